"""Conditioning of the coarse MCI sum near the zero-dispersion wavelength (a
reported check of the quadrature, independent of the CUDA path).

At the 589-ch CUT at 1260 nm with the Raman-ODE profile, the MCI cells carry
22 % of eta.  On an MCI grid of G_mci = 3 their sum is dominated by a few
points near phase-matched ridges, which are narrower in F_c than the FP32
spacing of a 59 THz offset.  This file evaluates that sum in numpy twice,
with FP64 z-sums both times:
  * with FP64 grid coordinates, reproducing the oracle's MCI part;
  * with the coordinates, the phase phi and the in-channel offsets formed
    in FP32, as the FP32 kernels form them.
Rounding the coordinates alone moves the 1260 nm CUT's MCI part by ~7e-4,
against ~5e-7 at the band centre.  That is the size of the FP32 path's
measured deviation there, which the GPU parity test therefore bounds
separately (reading R8: FP32 coordinates shift the sample point).
"""
import numpy as np

from paper_2401_18022_gb300 import workloads as W


def _mci_sum(orc, wl, i, fp32):
    """Sum over the MCI cells of CUT i on their own G_mci grid (folded
    mirror cells, rows uniform in ln upsilon1, columns in upsilon2), each
    point's z-sum of Eq. slow_vary in FP64 with ln p from the oracle's
    Raman-ODE tables (Eq. pk).  fp32: the point's coordinates formed in FP32."""
    G = wl.G_mci
    f, B = wl.f_THz, wl.B_THz
    n = len(f)
    fr = f - wl.f_ref_THz
    a_t, b_t, _ = orc.raman_profile(wl)
    ze = orc.zgrid(wl.L_km, wl.alpha_R_per_km, wl.n_edges)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    b2, b3, b4 = orc.beta_from_dispersion(299792.458 / wl.f_ref_THz, wl.D_ref, wl.S_ref, wl.Sdot_ref)
    pd = wl.P_W / B
    others = np.array([k for k in range(n) if k != i])
    ia, ib = np.triu_indices(len(others))
    ca, cb = others[ia], others[ib]
    mult = np.where(ca == cb, 1.0, 2.0)
    T = np.float32 if fp32 else np.float64
    rel, hb = (fr - fr[i]).astype(T), (0.5 * B).astype(T)
    ra, rb = rel[ca], rel[cb]
    s1, s2 = np.where(ra > 0, 1, -1).astype(T), np.where(rb > 0, 1, -1).astype(T)
    xlo, xhi = np.abs(ra) - hb[ca], np.abs(ra) + hb[ca]
    ylo, yhi = np.abs(rb) - hb[cb], np.abs(rb) + hb[cb]
    u1hi = xhi * yhi
    llo = np.log(np.maximum(xlo * ylo, T(wl.eps_v1) * u1hi))
    ds = (np.log(u1hi) - llo) / T(G)
    c3, c4, fi = T(np.pi * b3), T(2 * np.pi ** 2 / 3 * b4), T(fr[i])
    tot = 0.0
    for r in range(G):
        u1 = np.exp((T(r) + T(0.5)) * ds + llo)
        ymin, ymax = np.maximum(ylo, u1 / xhi), np.minimum(yhi, u1 / xlo)
        ok = ymax > ymin
        du2 = np.log1p((ymax - ymin) / np.where(ok, ymin, 1)) / T(G)
        yc = np.sqrt(ymin * ymax)
        xc = u1 / yc
        w = (u1 * ds * du2).astype(np.float64) * mult
        for j in range(G):
            e = np.exp((T(j) + T(0.5) - T(0.5) * T(G)) * du2)
            f1, f2 = s1 * (xc * e), s2 * (yc * (T(1) / e))
            u = f1 + f2
            c = np.clip(np.searchsorted(rel - hb, u, side="right") - 1, 0, n - 1)
            sel = np.nonzero(ok & (rel[c] - hb[c] <= u) & (u < rel[c] + hb[c]))[0]
            F1, F2, U, C, A, Bc = f1[sel], f2[sel], u[sel], c[sel], ca[sel], cb[sel]
            br = T(b2) + c3 * (U + T(2) * fi) + c4 * (F1 * F1 + T(1.5) * F1 * F2 + T(3) * fi * U + F2 * F2
                                                      + T(3) * fi * fi)
            phi = (T(-4 * np.pi ** 2) * F1 * F2 * br).astype(np.float64)[:, None]
            da = (F1 - rel[A]).astype(np.float64)[:, None]
            db = (F2 - rel[Bc]).astype(np.float64)[:, None]
            dc = (U - rel[C]).astype(np.float64)[:, None]
            lnp = 0.5 * (a_t[A] + b_t[A] * da + a_t[Bc] + b_t[Bc] * db + a_t[C] + b_t[C] * dc - a_t[i][None, :])
            x = 0.5 * phi * dz[None, :]
            sinc = np.where(np.abs(x) < 1e-8, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
            S = np.sum(np.exp(lnp) * dz[None, :] * sinc * np.exp(1j * phi * zm[None, :]), axis=1)
            tot += float(np.sum(w[sel] * pd[A] * pd[Bc] * pd[C] * np.abs(S) ** 2))
    return tot


def test_coordinate_rounding_moves_the_coarse_mci_sum_near_lambda0(orc):
    wl = W.raman(W.uwb(G=8, n_edges=33, cell_set=W.CELLS_ALL), ode_h_km=0.5).with_(G_mci=3)
    moved = {}
    for i in (294, 588):
        mci = orc.sigma(wl, cuts=[i])[0] - orc.sigma(wl.with_(cell_set=W.CELLS_SCI_XCI, G_mci=0), cuts=[i])[0]
        s64 = _mci_sum(orc, wl, i, False)
        assert abs(s64 / mci - 1) < 1e-10                  # the restatement is the oracle's MCI part
        moved[i] = abs(_mci_sum(orc, wl, i, True) / s64 - 1)
    assert moved[294] < 1e-5 and moved[588] > 2e-4, moved
