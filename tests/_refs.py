"""Independent reference computations used to pin the oracle.

None of these call the oracle's arithmetic; each is derived from the
mathematics the paper's method rests on, by a different route:

* ``beta_series``: the dispersion Taylor series beta(omega) itself, from
  which the phase mismatch is the four-wave-mixing difference
  beta(F_a) + beta(F_b) - beta(F_c) - beta(f) (App. A, Eq. phi).
* ``dispersion_of_betas``: D(lambda) = -(2 pi c / lambda^2) d^2beta/domega^2
  evaluated from a Taylor series in omega (the definition behind Sec. II,
  Eqs. d, d_slope, d_curve).
* ``zsum_closed_form``: the exact z-integral of a decaying exponential.
* ``one_d_sci``: a 1-D adaptive quadrature of the single-channel SCI
  integral in upsilon1 with the upsilon2-measure written in closed form.
* ``brute_sigma``: a Cartesian Gauss-Legendre quadrature in (f1, f2) with
  breakpoints at every discontinuity of the PSD product.
"""
from __future__ import annotations

import math

import numpy as np

C = 299792.458           # nm/ps


def beta_series(f, b2, b3, b4):
    """beta(f) - beta0 - beta1 w for w = 2 pi f (f in THz from the reference)."""
    w = 2.0 * np.pi * np.asarray(f, dtype=np.float64)
    return b2 / 2.0 * w ** 2 + b3 / 6.0 * w ** 3 + b4 / 24.0 * w ** 4


def phi_from_betas(f1, f2, fi, b2, b3, b4):
    """Four-wave-mixing phase mismatch per km: beta(Fa) + beta(Fb) - beta(Fc) - beta(f)."""
    fa, fb, fc = fi + f1, fi + f2, fi + f1 + f2
    return (beta_series(fa, b2, b3, b4) + beta_series(fb, b2, b3, b4)
            - beta_series(fc, b2, b3, b4) - beta_series(fi, b2, b3, b4))


def zsum_direct(z_edges, p_of_z, phi):
    """Discrete z-sum sum_m p(z_m) dz_m sinc(phi dz_m/2) e^{j phi z_m}, vectorised over phi."""
    ze = np.asarray(z_edges)
    zm = 0.5 * (ze[1:] + ze[:-1])
    dz = np.diff(ze)
    phi = np.asarray(phi, dtype=np.float64)[..., None]
    x = 0.5 * phi * dz
    sinc = np.where(np.abs(x) < 1e-8, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    return np.sum(p_of_z(zm) * dz * sinc * np.exp(1j * phi * zm), axis=-1)


def zsum_closed_form_abs2(a, phi, L):
    """|int_0^L e^{(-a + j phi) z} dz|^2."""
    return (1.0 - 2.0 * math.exp(-a * L) * math.cos(phi * L) + math.exp(-2.0 * a * L)) / (a * a + phi * phi)


# ---------------------------------------------------------------------------
# 1-D reference for one channel (SCI), C_r = 0, beta3 = beta4 = 0, uniform alpha
# ---------------------------------------------------------------------------
def one_d_sci(B, P, b2, z_edges, alpha, eps):
    """Sum over the four quadrants of int dv1 M(v1) (P/B)^3 |S(phi(v1))|^2.

    With only beta2, phi = -4 pi^2 beta2 s1 s2 v1 depends on v1 alone.  For a
    single channel of width B centred on the CUT, the v2-measure on which
    F_a, F_b and F_c all lie in the channel is
      same signs:     2 acosh(B / (4 sqrt v1))   for v1 < B^2/16  (|f1|+|f2| < B/2)
      opposite signs: 2 ln(B / (2 sqrt v1))      for v1 < B^2/4   (|f1|, |f2| < B/2)
    and the lower cut-off is v1 >= eps (B/2)^2 as in the 2-D grid.
    """
    from scipy.integrate import quad

    h = 0.5 * B
    v_lo, v_hi = eps * h * h, h * h
    psd3 = (P / B) ** 3

    def link(phi):
        return abs(zsum_direct(z_edges, lambda z: np.exp(-alpha * z), phi)) ** 2

    total = 0.0
    for s1s2 in (+1, -1):
        def integrand(s):
            v1 = math.exp(s)
            if s1s2 > 0:
                r = B / (4.0 * math.sqrt(v1))
                M = 2.0 * math.acosh(r) if r > 1.0 else 0.0
            else:
                r = B / (2.0 * math.sqrt(v1))
                M = 2.0 * math.log(r) if r > 1.0 else 0.0
            phi = -4.0 * math.pi ** 2 * b2 * s1s2 * v1
            return M * psd3 * float(link(phi)) * v1
        brk = [math.log(B * B / 16.0)] if s1s2 > 0 else []
        val, _ = quad(integrand, math.log(v_lo), math.log(v_hi), points=brk or None,
                      limit=2000, epsabs=0.0, epsrel=1e-11)
        total += 2.0 * val          # two quadrants of each sign pattern
    return total


# ---------------------------------------------------------------------------
# Cartesian brute force
# ---------------------------------------------------------------------------
def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def _panels(a, b, n_panels, x, w):
    """Composite Gauss-Legendre nodes/weights on [a, b]."""
    if not (b > a):
        return np.zeros(0), np.zeros(0)
    edges = np.linspace(a, b, n_panels + 1)
    h = np.diff(edges)[:, None]
    mid = 0.5 * (edges[1:] + edges[:-1])[:, None]
    return (mid + 0.5 * h * x[None, :]).ravel(), (0.5 * h * w[None, :]).ravel()


def lnrho_table(f, B, P, alpha, f_ref, Cr, alpha_R, zm):
    """Per channel c and step m: a[c, m] = ln rho(z_m, f_ref) contribution and kappa[m],
    so that ln rho(z_m, F in c) = -alpha_c z_m + lnPtot - lnN_m - kappa_m (F - f_ref).

    N(z) is the transmitted-PSD integral of e^{-kappa (nu - f_ref)}, evaluated here by
    Gauss-Legendre quadrature over each channel (no closed form used)."""
    Ptot = float(np.sum(P))
    leff = (1.0 - np.exp(-alpha_R * zm)) / alpha_R if alpha_R > 0 else zm
    kappa = Ptot * Cr * leff
    x, w = _gl(24)
    N = np.zeros_like(zm)
    for c in range(len(f)):
        nu = f[c] + 0.5 * B[c] * x
        N += (P[c] / B[c]) * 0.5 * B[c] * np.sum(w[None, :] * np.exp(-kappa[:, None] * (nu[None, :] - f_ref)), axis=1)
    return math.log(Ptot), np.log(N), kappa


def brute_sigma(f, B, P, alpha, fibre, z_edges, cut, cells="all", n_outer=64, n_inner=24, order=8):
    """Cartesian quadrature of the CUT's frequency integral.

    fibre = (L, f_ref, b2, b3, b4, Cr, alpha_R).  Integrates over each cell
    F_a in channel a, F_b in channel b with composite Gauss-Legendre; the inner
    f2 integral is broken at every channel edge crossed by F_c = f_i + f1 + f2
    so the integrand is smooth on each segment."""
    f, B, P, alpha = (np.asarray(v, dtype=np.float64) for v in (f, B, P, alpha))
    L, f_ref, b2, b3, b4, Cr, alpha_R = fibre
    ze = np.asarray(z_edges)
    zm = 0.5 * (ze[1:] + ze[:-1])
    dz = np.diff(ze)
    lnPtot, lnN, kappa = lnrho_table(f, B, P, alpha, f_ref, Cr, alpha_R, zm)
    fi = f[cut]
    x, w = _gl(order)
    lo_e, hi_e = f - 0.5 * B, f + 0.5 * B

    def chan(F):
        idx = np.searchsorted(lo_e, F, side="right") - 1
        ok = (idx >= 0) & (F < hi_e[np.clip(idx, 0, len(f) - 1)])
        return np.where(ok, idx, -1)

    def lnrho(c, F):
        return (-alpha[c][..., None] * zm + lnPtot - lnN - kappa * (F[..., None] - f_ref))

    total = 0.0
    n = len(f)
    for a in range(n):
        for b in range(n):
            if cells == "sci_xci" and a != cut and b != cut:
                continue
            A0, A1 = lo_e[a] - fi, hi_e[a] - fi
            C0, C1 = lo_e[b] - fi, hi_e[b] - fi
            brk1 = [A0, A1] + ([0.0] if A0 < 0.0 < A1 else [])
            brk1 = sorted(brk1)
            f1s, w1s = [], []
            for u0, u1 in zip(brk1[:-1], brk1[1:]):
                xx, ww = _panels(u0, u1, n_outer, x, w)
                f1s.append(xx); w1s.append(ww)
            f1s, w1s = np.concatenate(f1s), np.concatenate(w1s)
            for f1, w1 in zip(f1s, w1s):
                # breakpoints of F_c = fi + f1 + f2 at channel edges
                e = np.concatenate([lo_e, hi_e]) - fi - f1
                brk = sorted(set([C0, C1] + [v for v in e if C0 < v < C1]))
                f2s, w2s = [], []
                for v0, v1 in zip(brk[:-1], brk[1:]):
                    xx, ww = _panels(v0, v1, n_inner, x, w)
                    f2s.append(xx); w2s.append(ww)
                f2 = np.concatenate(f2s); w2 = np.concatenate(w2s)
                Fa = np.full_like(f2, fi + f1); Fb = fi + f2; Fc = fi + f1 + f2
                ca, cb, cc = chan(Fa), chan(Fb), chan(Fc)
                ok = (ca >= 0) & (cb >= 0) & (cc >= 0)
                if not np.any(ok):
                    continue
                f2, w2, Fa, Fb, Fc = f2[ok], w2[ok], Fa[ok], Fb[ok], Fc[ok]
                ca, cb, cc = ca[ok], cb[ok], cc[ok]
                W = (P[ca] / B[ca]) * (P[cb] / B[cb]) * (P[cc] / B[cc])
                lnp = 0.5 * (lnrho(ca, Fa) + lnrho(cb, Fb) + lnrho(cc, Fc)
                             - lnrho(np.full_like(ca, cut), np.full_like(Fa, fi)))
                ph = phi_from_betas(f1, f2, fi - f_ref, b2, b3, b4)[:, None]
                xarg = 0.5 * ph * dz
                sinc = np.where(np.abs(xarg) < 1e-8, 1.0, np.sin(xarg) / np.where(xarg == 0, 1.0, xarg))
                S = np.sum(np.exp(lnp) * dz * sinc * np.exp(1j * ph * zm), axis=1)
                total += w1 * float(np.sum(w2 * W * np.abs(S) ** 2))
    return total
