"""Pins of the FP64 oracle against mathematics that does not come from the oracle.

Each test fixes one function of ``oracle/`` to an independent fact: a
symbolic identity, a closed form, a conservation law, an ODE, a brute-force
quadrature of the same integral by another route, an invariant of the
integrand, or a value printed in the paper.  The mutation tests at the end
show that a plausible slip (a dropped dispersion term, a wrong sign, a
transposed argument) is caught by these pins.
"""
import math

import numpy as np
import pytest

import _refs
from paper_2401_18022_gb300 import workloads as W


# ---------------------------------------------------------------------------
# Sec. II, Eqs. d, d_slope, d_curve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lam,D,S,Sd", [(1550.116, 17.0, 0.057, 0.0),
                                        (1310.0, 0.0, 0.09, -2.061e-4),
                                        (1438.0, 17.74, 0.057, -5.975e-5)])
def test_beta_reproduces_dispersion_and_its_derivatives(orc, lam, D, S, Sd):
    """D(lambda) = -(2 pi c/lambda^2) beta2(omega) with beta2(omega) from the
    Taylor series; its value, slope and curvature at lambda_c must be D, S, Sdot."""
    import sympy as sp
    b2, b3, b4 = orc.beta_from_dispersion(lam, D, S, Sd)
    l = sp.symbols("l", positive=True)
    c = sp.Rational(299792458, 1000)
    dw = 2 * sp.pi * c * (1 / l - 1 / sp.Float(lam, 30))
    beta2_w = sp.Float(b2, 30) + sp.Float(b3, 30) * dw + sp.Float(b4, 30) / 2 * dw ** 2
    Dl = -(2 * sp.pi * c / l ** 2) * beta2_w
    vals = [float(sp.diff(Dl, l, k).subs(l, sp.Float(lam, 30)).evalf(30)) for k in range(3)]
    assert vals[0] == pytest.approx(D, abs=1e-12)
    assert vals[1] == pytest.approx(S, rel=1e-12, abs=1e-15)
    assert vals[2] == pytest.approx(Sd, rel=1e-10, abs=1e-15)


def test_gamma_textbook_values(orc):
    """Sec. II, Eq. gamma: SSMF at 1550 nm, n2 = 2.6e-20, Aeff = 80 um^2 gives
    the textbook ~1.3 /W/km; 1310 nm with 64.2 um^2 (the linear 60-95 um^2 Aeff model) gives ~1.94."""
    assert orc.gamma(1550.0, 2.6e-20, 80.0) == pytest.approx(1.3175, rel=2e-3)
    assert orc.gamma(1302.3, 2.6e-20, float(W.aeff_model_um2(1302.3))) == pytest.approx(2.0, rel=0.02)


# ---------------------------------------------------------------------------
# z-grid: equal power drop per step (Sec. III-A, App. A)
# ---------------------------------------------------------------------------
def test_zgrid_equal_power_drop(orc):
    L, a, n = 80.0, 0.0571, 113
    z = orc.zgrid(L, a, n)
    assert z[0] == 0.0 and z[-1] == L
    assert np.all(np.diff(z) > 0)
    drops = -np.diff(np.exp(-a * z))
    assert np.allclose(drops, (1 - math.exp(-a * L)) / (n - 1), rtol=1e-12)
    # density definition: (N_M - 1)/L = 1.4 steps/km at N_M = 113, L = 80 km
    assert W.n_edges_from_density(1.4, 80.0) == 113
    # no loss: uniform steps
    assert np.allclose(np.diff(orc.zgrid(10.0, 0.0, 11)), 1.0)


# ---------------------------------------------------------------------------
# App. A, Eq. phi
# ---------------------------------------------------------------------------
def test_phi_is_fwm_difference_of_taylor_betas_symbolically():
    """The printed polynomial equals beta(Fa)+beta(Fb)-beta(Fc)-beta(f) exactly."""
    import sympy as sp
    f1, f2, fi, b2, b3, b4 = sp.symbols("f1 f2 fi b2 b3 b4")
    pi = sp.pi

    def beta(f):
        w = 2 * pi * f
        return b2 / 2 * w ** 2 + b3 / 6 * w ** 3 + b4 / 24 * w ** 4
    fwm = beta(fi + f1) + beta(fi + f2) - beta(fi + f1 + f2) - beta(fi)
    printed = -4 * pi ** 2 * f1 * f2 * (b2 + pi * b3 * (f1 + f2 + 2 * fi) + 2 * pi ** 2 / 3 * b4 *
                                        (f1 ** 2 + sp.Rational(3, 2) * f1 * f2 + 3 * f1 * fi + f2 ** 2
                                         + 3 * f2 * fi + 3 * fi ** 2))
    assert sp.expand(fwm - printed) == 0


def test_phi_oracle_matches_beta_differences(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        f1, f2, fi = rng.uniform(-30, 30, 3)
        b = (rng.uniform(-25, 25), rng.uniform(-0.2, 0.2), rng.uniform(-1e-3, 1e-3))
        ref = _refs.phi_from_betas(f1, f2, fi, *b)
        got = orc.phi(f1, f2, fi, *b)
        scale = 4 * math.pi ** 2 * abs(f1 * f2) * (abs(b[0]) + math.pi * abs(b[1]) * 120
                                                   + 7 * math.pi ** 2 * abs(b[2]) * 3600)
        assert abs(got - ref) <= 1e-12 * scale


# ---------------------------------------------------------------------------
# ISRS power profile
# ---------------------------------------------------------------------------
def _plan3():
    f = np.array([193.0, 193.1, 193.25, 193.4, 193.6])
    B = np.array([0.05, 0.06, 0.096, 0.08, 0.1])
    P = np.array([2e-3, 1e-3, 5e-3, 3e-3, 4e-3])
    return f, B, P


def test_profile_without_raman_is_plain_attenuation(orc):
    f, B, P = _plan3()
    alpha = np.array([0.04, 0.045, 0.05, 0.055, 0.06])
    for z in (0.0, 3.0, 40.0, 80.0):
        for c in range(len(f)):
            lr = orc.lnrho(f, B, P, alpha, 193.3, 0.0, 0.046, z, f[c] + 0.01)
            assert lr == pytest.approx(-alpha[c] * z, abs=1e-13)


def test_profile_conserves_total_power(orc):
    """With uniform attenuation: int G_Tx(nu) rho(z, nu) dnu = P_tot e^{-alpha z}."""
    f, B, P = _plan3()
    a = 0.05
    alpha = np.full(len(f), a)
    x, w = np.polynomial.legendre.leggauss(12)
    for Cr in (0.028, 40.0):
        for z in (0.5, 10.0, 80.0):
            tot = 0.0
            for c in range(len(f)):
                nu = f[c] + 0.5 * B[c] * x
                vals = np.array([math.exp(orc.lnrho(f, B, P, alpha, 193.3, Cr, a, z, v)) for v in nu])
                tot += P[c] / B[c] * 0.5 * B[c] * np.sum(w * vals)
            assert tot == pytest.approx(P.sum() * math.exp(-a * z), rel=1e-12)


def test_profile_independent_of_reference_frequency(orc):
    f, B, P = _plan3()
    alpha = np.full(len(f), 0.05)
    for F in (193.02, 193.27, 193.61):
        a = orc.lnrho(f, B, P, alpha, 193.3, 30.0, 0.05, 20.0, F)
        b = orc.lnrho(f, B, P, alpha, 190.0, 30.0, 0.05, 20.0, F)
        assert a == pytest.approx(b, abs=1e-11)


def test_profile_solves_linear_slope_raman_ode(orc):
    """d/dz ln rho(z,f) = -alpha - C_r int (f - nu) G_Tx(nu) rho(z,nu) dnu, i.e. the
    Raman power-evolution ODE with a linear gain slope (triangular g_r, no cut-off)."""
    f, B, P = _plan3()
    a, Cr = 0.05, 25.0
    alpha = np.full(len(f), a)
    x, w = np.polynomial.legendre.leggauss(12)
    for z in (1.0, 15.0, 60.0):
        for F in (193.02, 193.42, 193.63):
            h = 1e-3
            d = (orc.lnrho(f, B, P, alpha, 193.3, Cr, a, z + h, F)
                 - orc.lnrho(f, B, P, alpha, 193.3, Cr, a, z - h, F)) / (2 * h)
            integ = 0.0
            for c in range(len(f)):
                nu = f[c] + 0.5 * B[c] * x
                rho = np.array([math.exp(orc.lnrho(f, B, P, alpha, 193.3, Cr, a, z, v)) for v in nu])
                integ += P[c] / B[c] * 0.5 * B[c] * np.sum(w * (F - nu) * rho)
            assert d == pytest.approx(-a - Cr * integ, rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------------------
# App. A, Eq. slow_vary (z-sum)
# ---------------------------------------------------------------------------
def test_zsum_telescopes_exactly_for_constant_power(orc):
    """With p = 1 the sum of dz sinc(phi dz/2) e^{j phi z_m} over any partition is
    (e^{j phi L} - 1)/(j phi)."""
    rng = np.random.default_rng(3)
    ze = np.concatenate([[0.0], np.sort(rng.uniform(0, 80, 40)), [80.0]])
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    for ph in (1e-6, 0.013, 0.7, 31.0, 1234.5):
        got = orc.zsum(zm, dz, np.ones_like(zm), ph)
        ref = (np.exp(1j * ph * 80.0) - 1) / (1j * ph)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)) + 1e-12 * 80


def test_zsum_converges_to_closed_form_link(orc):
    """p = e^{-a z}: |S|^2 -> (1 - 2e^{-aL}cos phi L + e^{-2aL})/(a^2 + phi^2).
    Second order in dz while phi dz << 1; for large phi the piecewise-constant
    power leaves an O(dz) oscillating error that still vanishes."""
    a, L = 0.046, 80.0

    def err(ph, n):
        ze = orc.zgrid(L, a, n)
        zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
        S = orc.zsum(zm, dz, np.exp(-a * zm), ph)
        return abs(abs(S) ** 2 / _refs.zsum_closed_form_abs2(a, ph, L) - 1)
    for ph in (0.0, 0.05):
        e = [err(ph, n) for n in (51, 101, 201)]
        assert e[2] < 1e-4
        assert 0.2 < e[1] / e[0] < 0.3 and 0.2 < e[2] / e[1] < 0.3
    for ph in (2.0, 50.0):
        e = [err(ph, n) for n in (401, 1601, 6401)]
        assert e[2] < (1e-5 if ph < 10 else 1e-2) and e[2] < e[0]


# ---------------------------------------------------------------------------
# Pieces and the hyperbolic grid (App. A, Eqs. q1a..q4d, q1..q4)
# ---------------------------------------------------------------------------
def test_pieces_tile_the_cells(orc):
    f, B, _ = _plan3()
    for cut in range(len(f)):
        for cs in (0, 1):
            pcs = orc.pieces(f, B, cut, cs)
            area = np.sum((pcs[:, 5] - pcs[:, 4]) * (pcs[:, 7] - pcs[:, 6]))
            if cs == 1:
                ref = B.sum() ** 2
            else:
                ref = 2 * B[cut] * B.sum() - B[cut] ** 2
            assert area == pytest.approx(ref, rel=1e-12)
        sci = [p for p in orc.pieces(f, B, cut, 0) if p[0] == cut and p[1] == cut]
        assert len(sci) == 4
        assert {(int(p[2]), int(p[3])) for p in sci} == {(1, 1), (1, -1), (-1, 1), (-1, -1)}
        for p in sci:
            assert (p[4], p[5], p[6], p[7]) == pytest.approx((0, B[cut] / 2, 0, B[cut] / 2))


def test_hyperbolic_grid_covers_piece_area(orc):
    """With the integrand set to 1 the Riemann sum converges to the cell area
    (minus the cut-off strip of relative size ~ eps ln(1/eps)), at second order."""
    f, B, P = _plan3()
    wl = W.tiny().with_(f_THz=f, B_THz=B, P_W=P, alpha_per_km=np.full(5, 0.05),
                        lambda_nm=W.nm_from_thz(f), aeff_um2=np.full(5, 80.0), nf_dB=np.full(5, 5.0),
                        cell_set=1, n_edges=3)
    ref = B.sum() ** 2
    errs = []
    for G in (16, 64, 256):
        s = orc.sigma(wl.with_(G=G), cuts=[2], unit_integrand=True)[0]
        errs.append(abs(s / ref - 1))
    # second order: each 4x refinement gains more than 10x
    assert errs[2] < 1e-3
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 10


def test_quadrature_matches_1d_semi_analytic_sci(orc):
    """Single channel, C_r = 0, beta3 = beta4 = 0, uniform alpha: phi depends on
    upsilon1 only, so the 2-D integral reduces to a 1-D one with a closed-form
    upsilon2-measure (see _refs.one_d_sci)."""
    Bw, P, a, L, b2 = 0.096, 1e-3, 0.046, 80.0, -21.7
    wl = W.tiny().with_(f_THz=np.array([193.4]), B_THz=np.array([Bw]), P_W=np.array([P]),
                        alpha_per_km=np.array([a]), lambda_nm=np.array([1550.0]),
                        aeff_um2=np.array([80.0]), nf_dB=np.array([5.0]), Cr=0.0,
                        alpha_R_per_km=a, cell_set=0, G=256)
    fib = np.array([L, 193.4, b2, 0.0, 0.0, 0.0, a])
    ze = orc.zgrid(L, a, 113)
    ref = _refs.one_d_sci(Bw, P, b2, ze, a, 1e-10)
    got = orc.sigma(wl, fibre=fib)[0]
    assert got == pytest.approx(ref, rel=3e-4)


def _brute_case():
    f = np.array([193.3, 193.4, 193.5])
    B = np.array([0.096, 0.080, 0.096])
    P = np.array([10e-3, 5e-3, 20e-3])
    alpha = np.array([0.05, 0.046, 0.06])
    fib = np.array([10.0, 193.9, -21.7, 1.5, -0.4, 3.0, 0.046])
    wl = W.tiny().with_(f_THz=f, B_THz=B, P_W=P, alpha_per_km=alpha, lambda_nm=W.nm_from_thz(f),
                        aeff_um2=np.full(3, 80.0), nf_dB=np.full(3, 5.0), Cr=3.0, alpha_R_per_km=0.046,
                        L_km=10.0, n_edges=17, cell_set=1, G=512)
    return f, B, P, alpha, fib, wl


@pytest.fixture(scope="module")
def brute_refs():
    import oracle
    f, B, P, alpha, fib, wl = _brute_case()
    ze = oracle.zgrid(fib[0], fib[6], wl.n_edges)
    return {cut: _refs.brute_sigma(f, B, P, alpha, fib, ze, cut, n_outer=40, n_inner=10)
            for cut in (0, 1)}


def test_quadrature_matches_cartesian_brute_force(orc, brute_refs):
    """3 uneven channels, all cells (SCI, XCI and MCI), strong beta3/beta4 and
    Raman tilt: the hyperbolic Riemann sum agrees with an independent Cartesian
    Gauss-Legendre quadrature that breaks at every PSD discontinuity."""
    f, B, P, alpha, fib, wl = _brute_case()
    got = orc.sigma(wl, fibre=fib, cuts=[0, 1])
    for k, cut in enumerate((0, 1)):
        assert got[k] == pytest.approx(brute_refs[cut], rel=6e-4)


@pytest.mark.parametrize("mutation", ["drop_beta3", "drop_beta4", "flip_tilt", "no_raman"])
def test_brute_force_pin_catches_mutations(orc, brute_refs, mutation):
    """Plant a plausible mistake in the oracle's inputs: the pin must fail by
    far more than its tolerance."""
    f, B, P, alpha, fib, wl = _brute_case()
    fib = fib.copy()
    if mutation == "drop_beta3":
        fib[3] = 0.0
    elif mutation == "drop_beta4":
        fib[4] = 0.0
    elif mutation == "flip_tilt":
        fib[5] = -fib[5]
    elif mutation == "no_raman":
        fib[5] = 0.0
    got = orc.sigma(wl.with_(G=128), fibre=fib, cuts=[0, 1])
    err = max(abs(got[0] / brute_refs[0] - 1), abs(got[1] / brute_refs[1] - 1))
    assert err > 5 * 6e-4


# ---------------------------------------------------------------------------
# Invariants of the integrand
# ---------------------------------------------------------------------------
def test_mirror_pieces_and_cells_are_equal(orc):
    """Psi(f1, f2) = Psi(f2, f1): quadrant pieces (+,-) and (-,+) of the SCI cell
    (Q4 = Q2) and cells (a,b), (b,a) have equal Riemann sums."""
    wl = W.tiny(G=32, cell_set=1)
    s, pcs_val = orc.sigma(wl, cuts=[1], return_pieces=True)
    pcs = orc.pieces(wl.f_THz, wl.B_THz, 1, 1)
    key = {(int(p[0]), int(p[1]), int(p[2]), int(p[3])): v for p, v in zip(pcs, pcs_val)}
    for (a, b, s1, s2), v in key.items():
        assert v == pytest.approx(key[(b, a, s2, s1)], rel=1e-11)


def test_eta_scales_with_gamma_squared_and_is_power_invariant_without_raman(orc):
    wl = W.tiny(G=24, n_edges=41).with_(Cr=0.0)
    s1 = orc.sigma(wl)
    e1, _ = orc.eta(wl, s1)
    e2, _ = orc.eta(wl.with_(gamma_fixed=2.6), s1)
    assert np.allclose(e2 / e1, 4.0, rtol=1e-14)
    s3 = orc.sigma(wl, P=wl.P_W * 3.7)
    e3, _ = orc.eta(wl, s3, P=wl.P_W * 3.7)
    assert np.allclose(e3, e1, rtol=1e-12)


def test_mirror_symmetric_plan(orc):
    """beta3 = beta4 = 0, uniform alpha, no Raman, symmetric plan: eta_i = eta_{N-1-i}."""
    wl = W.tiny(G=24, n_edges=41).with_(Cr=0.0, S_ref=0.0)
    fib = orc.fibre_params(wl)
    fib[3] = fib[4] = 0.0
    s = orc.sigma(wl, fibre=fib)
    assert np.allclose(s, s[::-1], rtol=1e-9)


def test_snr_ase_textbook(orc):
    """No NLI, no Raman: G = e^{alpha L} and P_ASE = NF h nu (G - 1) B."""
    wl = W.tiny(G=8, n_edges=5).with_(Cr=0.0)
    snr, pase, T = orc.snr_throughput(wl, np.zeros(5))
    a, L = wl.alpha_per_km[0], wl.L_km
    nf = 10 ** (wl.nf_dB / 10)
    ref = nf * 6.62607015e-34 * wl.f_THz * 1e12 * (math.exp(a * L) - 1) * wl.B_THz * 1e12
    assert np.allclose(pase, ref, rtol=1e-12)
    assert np.allclose(snr, wl.P_W / ref, rtol=1e-12)
    assert T == pytest.approx(float(np.sum(2 * wl.B_THz * np.log2(1 + wl.P_W / ref))), rel=1e-12)


def test_multispan_sum_is_phased_array_times_one_span(orc):
    """Identical spans: |sum_k S e^{j phi (k-1) L}|^2 = |S|^2 sin^2(n phi L/2)/sin^2(phi L/2)
    (the phased-array term the multi-span sum reduces to)."""
    L = 80.0
    ze = orc.zgrid(L, 0.05, 41)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    p = np.exp(-0.05 * zm)
    for n in (1, 2, 5, 13):
        for ph in (1e-4, 0.013, 0.9, 37.0):
            one = abs(orc.zsum(zm, dz, p, ph)) ** 2
            x = ph * L / 2
            af = (math.sin(n * x) / math.sin(x)) ** 2 if abs(math.sin(x)) > 1e-12 else n * n
            got = abs(orc.zsum_spans(zm, dz, p, ph, L, n)) ** 2
            assert got == pytest.approx(one * af, rel=1e-9, abs=1e-12 * one * n * n)


def test_multispan_quadrature_and_ase(orc):
    """n spans: Sigma grows between n and n^2 times (coherent array factor), the
    ASE adds over the n amplifiers."""
    wl = W.tiny(G=16, n_edges=17)
    s1 = orc.sigma(wl)
    for n in (2, 4):
        sn = orc.sigma(wl.with_(n_spans=n))
        assert np.all(sn > n * s1 * 0.999) and np.all(sn < n * n * s1)
        snr1, pase1, _ = orc.snr_throughput(wl, np.zeros(5))
        snrn, pasen, _ = orc.snr_throughput(wl.with_(n_spans=n), np.zeros(5))
        np.testing.assert_allclose(pasen, n * pase1, rtol=1e-14)


# ---------------------------------------------------------------------------
# App. A, Eq. gain_fin: the eta prefactor, end to end
# ---------------------------------------------------------------------------
def _one_channel_no_dispersion(G, cell_set=0):
    """One 96 GBaud channel, beta2 = beta3 = beta4 = 0, C_r = 0, uniform alpha."""
    Bw, P, a, L, g = 0.096, 2e-3, 0.046, 80.0, 1.3
    wl = W.tiny().with_(f_THz=np.array([193.4]), B_THz=np.array([Bw]), P_W=np.array([P]),
                        alpha_per_km=np.array([a]), lambda_nm=np.array([1550.0]),
                        aeff_um2=np.array([80.0]), nf_dB=np.array([5.0]), Cr=0.0, gamma_fixed=g,
                        alpha_R_per_km=a, cell_set=cell_set, G=G, n_edges=113)
    fib = np.array([L, 193.4, 0.0, 0.0, 0.0, 0.0, a])
    return wl, fib, (Bw, P, a, L, g)


def _eta_no_dispersion_exact(orc, a, L, g):
    """phi = 0 at every grid point, so every point's z-sum is the same real
    number S = sum_m e^{-alpha z_m} dz_m (Eq. slow_vary with sinc(0) = 1 and
    p_m = e^{-alpha z_m}: the three PSD frequencies and the CUT share alpha).
    F_a, F_b and F_c = F_a + F_b - f_i all lie in the channel on the hexagon
    |f1|, |f2|, |f1 + f2| <= B/2, whose area is B^2 - 2 (B/2)^2 / 2 = (3/4) B^2,
    and G_Tx = P/B there.  So the frequency integral is (P/B)^3 (3/4) B^2 S^2,
    and Eq. gain_fin with P_NLI = G(f_i) B gives
        eta = (16/27) gamma^2 B (P/B)^3 (3/4) B^2 S^2 / P^3 = (4/9) gamma^2 S^2,
    the zero-dispersion limit of the GN model ((4/9) gamma^2 L_eff^2 when the
    z-sum is replaced by its integral)."""
    ze = _refs_zgrid(L, a, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    S = float(np.sum(np.exp(-a * zm) * dz))
    return 4.0 / 9.0 * g * g * S * S, S


def _refs_zgrid(L, a, n):
    """Equal power drop per step, written out here (not the oracle's routine)."""
    t = np.arange(n) / (n - 1)
    z = -np.log1p(-t * (1.0 - math.exp(-a * L))) / a
    z[-1] = L
    return z


@pytest.mark.parametrize("cell_set", [0, 1])
def test_eta_prefactor_single_channel_zero_dispersion(orc, cell_set):
    """The whole chain Sigma -> eta (Eq. gain_fin, 16/27 gamma^2 B_i, P_NLI =
    G(f_i) B_i) against the closed form (4/9) gamma^2 S^2.  The hexagon's
    oblique edge |f1 + f2| = B/2 cuts grid cells, so the Riemann sum
    converges to it at first order with an oscillating sign: the error must
    shrink from G = 32 to G >= 128 and stay within 5e-4 there."""
    errs = {}
    for G in (32, 128, 256, 512):
        wl, fib, (Bw, P, a, L, g) = _one_channel_no_dispersion(G, cell_set)
        s = orc.sigma(wl, fibre=fib)
        e, pn = orc.eta(wl, s)
        ref, S = _eta_no_dispersion_exact(orc, a, L, g)
        errs[G] = abs(e[0] / ref - 1)
        assert pn[0] == pytest.approx(e[0] * P ** 3, rel=1e-14)
    assert errs[32] > 5 * max(errs[128], errs[256], errs[512])
    assert max(errs[128], errs[256], errs[512]) < 5e-4
    # the continuous z-integral: S -> L_eff = (1 - e^{-alpha L})/alpha
    assert S == pytest.approx((1 - math.exp(-a * L)) / a, rel=1e-3)


def test_eta_prefactor_full_square_pieces(orc):
    """The (+,-) and (-,+) quadrant pieces of the SCI cell are full squares
    [0, B/2] x [-B/2, 0] (|f1 + f2| <= B/2 holds everywhere), so each carries
    (P/B)^3 (B/2)^2 S^2 exactly.  The hyperbolic grid converges to it at second
    order in the row spacing of s = ln upsilon1, whose range is ln(1/eps) = 23
    (the eps cut-off strip itself is ~eps ln(1/eps) = 2e-9 of the area): the
    error must fall by ~4x per doubling of G."""
    errs = []
    for G in (128, 256, 512):
        wl, fib, (Bw, P, a, L, g) = _one_channel_no_dispersion(G, 0)
        _, S = _eta_no_dispersion_exact(orc, a, L, g)
        s, pv = orc.sigma(wl, fibre=fib, return_pieces=True)
        pcs = orc.pieces(wl.f_THz, wl.B_THz, 0, 0)
        mixed = [v for p, v in zip(pcs, pv) if p[2] != p[3]]
        assert len(mixed) == 2 and mixed[0] == pytest.approx(mixed[1], rel=1e-13)
        ref = (P / Bw) ** 3 * (Bw / 2) ** 2 * S * S
        errs.append(abs(mixed[0] / ref - 1))
    assert errs[2] < 2e-4
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("mutation", ["8/27", "drop_B", "B_squared", "gamma_not_squared"])
def test_eta_prefactor_pin_catches_mutations(orc, mutation):
    """Plant a slip in the oracle's eta (as a rescaling of its output): the
    closed-form pin above must fail by far more than its 5e-4 tolerance."""
    wl, fib, (Bw, P, a, L, g) = _one_channel_no_dispersion(256, 0)
    s = orc.sigma(wl, fibre=fib)
    e, _ = orc.eta(wl, s)
    mutated = {"8/27": e[0] / 2.0, "drop_B": e[0] / Bw, "B_squared": e[0] * Bw,
               "gamma_not_squared": e[0] / g}[mutation]
    ref, _ = _eta_no_dispersion_exact(orc, a, L, g)
    assert abs(mutated / ref - 1) > 100 * 5e-4


# ---------------------------------------------------------------------------
# Sec. IV, Eq. loss: SNR with NLI and transceiver noise
# ---------------------------------------------------------------------------
def test_snr_optimum_launch_power_textbook(orc):
    """With a power-independent ASE (C_r = 0) and a fixed eta, SNR(P) =
    P / (eta P^3 + P_ASE) peaks where the NLI power is half the ASE power,
    P_opt = (P_ASE / (2 eta))^(1/3), at SNR = P_opt / (1.5 P_ASE): the GN
    model's optimum launch power."""
    wl = W.tiny(G=8, n_edges=5).with_(Cr=0.0)
    eta = np.array([1.0e3, 2.5e3, 4.0e2, 7.0e2, 1.5e3])        # 1/W^2
    _, pase, _ = orc.snr_throughput(wl, eta, P=np.full(5, 1e-3))
    p_opt = (pase / (2 * eta)) ** (1.0 / 3.0)
    snr_opt, _, _ = orc.snr_throughput(wl, eta, P=p_opt)
    np.testing.assert_allclose(snr_opt, p_opt / (1.5 * pase), rtol=1e-12)
    for f in (0.97, 1.03):
        snr_f, _, _ = orc.snr_throughput(wl, eta, P=p_opt * f)
        assert np.all(snr_f < snr_opt)


def test_snr_transceiver_limited_and_guard(orc):
    """No NLI and a negligible ASE (NF -300 dB): 1/SNR = 1/SNR_ASE + 1/SNR_TRX
    leaves SNR = SNR_TRX, and T = 2 B log2(1 + SNR_TRX) over the channels that
    are neither guards nor empty."""
    wl = W.tiny(G=8, n_edges=5).with_(Cr=0.0, nf_dB=np.full(5, -300.0), snr_trx_dB=20.0,
                                      guard=np.array([0, 0, 1, 0, 0], dtype=np.uint8))
    snr, pase, T = orc.snr_throughput(wl, np.zeros(5))
    lit = np.array([True, True, False, True, True])
    np.testing.assert_allclose(snr[lit], 100.0, rtol=1e-12)
    assert snr[2] == 0.0
    assert T == pytest.approx(float(np.sum(2 * wl.B_THz[lit] * np.log2(101.0))), rel=1e-12)
