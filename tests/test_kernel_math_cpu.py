"""CPU checks of evaluation strategies the FP32 kernel relies on.

The kernel evaluates the z-sum of Eq. slow_vary in one of three exact-to-FP32
forms chosen per grid point; two of them rest on identities checked here
against the oracle's direct z-sum (independent code)."""
import numpy as np


def test_small_phi_second_order_expansion(orc):
    """For |phi| L <= 0.02: |S|^2 = M0^2 - phi^2 (M0 M2 - M1^2) with
    M_k = sum p dz z^k (M2 with z^2 + dz^2/12) to better than 1e-8."""
    L = 80.0
    ze = orc.zgrid(L, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(60):
        a, k = rng.uniform(0.02, 0.2), rng.uniform(-0.1, 0.1)
        p = np.exp(-a * zm + k * np.sin(zm / 7)) * rng.uniform(0.5, 2)
        w = p * dz
        M0, M1, M2 = w.sum(), (w * zm).sum(), (w * (zm ** 2 + dz ** 2 / 12)).sum()
        for x in rng.uniform(-0.02, 0.02, 10):
            ph = x / L
            exact = abs(orc.zsum(zm, dz, p, ph)) ** 2
            approx = M0 ** 2 - ph ** 2 * (M0 * M2 - M1 ** 2)
            worst = max(worst, abs(approx / exact - 1))
    assert worst < 1e-8


def test_telescoped_step_identity(orc):
    """dz sinc(phi dz/2) e^{j phi z_m} = (E_{m+1} - E_m)/(j phi), E = e^{j phi z}."""
    ze = orc.zgrid(80.0, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    rng = np.random.default_rng(2)
    p = np.exp(-0.05 * zm) * (1 + 0.1 * rng.standard_normal(len(zm)))
    for ph in (0.7, 13.0, 812.5):
        E = np.exp(1j * ph * ze)
        tele = np.sum(p * (E[1:] - E[:-1])) / (1j * ph)
        assert abs(tele - orc.zsum(zm, dz, p, ph)) < 1e-10 * np.sum(np.abs(p * dz))


def test_sinc_polynomial_on_direct_range():
    """Even Taylor polynomial of sinc to x^10 on |x| <= pi/2: error < 4e-8."""
    x = np.linspace(-np.pi / 2, np.pi / 2, 20001)
    c = [1.0, -1 / 6, 1 / 120, -1 / 5040, 1 / 362880, -1 / 39916800]
    poly = sum(ck * x ** (2 * k) for k, ck in enumerate(c))
    ref = np.sinc(x / np.pi)
    assert np.max(np.abs(poly - ref)) < 4e-8


def _bessel_i(n, a):
    """Modified Bessel I_n(a) by its power series (|a| small)."""
    from math import factorial
    return sum((a / 2) ** (2 * k + n) / (factorial(k) * factorial(k + n)) for k in range(8))


def test_chebyshev_contraction_of_small_phase_moments(orc):
    """For F_c = F0 + h x in one channel, the moments M_k = sum_m w_m(F_c) g_k(m)
    with w_m = 2^(A_m + K_m F_c) equal sum_n C_kn T_n(x), n <= 3, where
    C_kn = sum_m 2^(A_m + K_m F0) g_k(m) b_n(K_m h ln 2), b_0 = I_0, b_n = 2 I_n
    (the Chebyshev expansion of e^{a x}); truncation about (a/2)^4/12, below
    4e-8 for |a| <= 0.05 (the kernel's bound)."""
    import math
    ze = orc.zgrid(80.0, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    rng = np.random.default_rng(4)
    kappa = np.linspace(0.0, 0.36, len(zm))              # ISRS exponent per THz along z
    K = -kappa / math.log(2.0)                            # log2 slope per THz
    A = np.log2(dz) - 0.05 * zm / math.log(2.0)
    g = [np.ones_like(zm), zm, zm ** 2 + dz ** 2 / 12]
    for h in (0.048, 0.19):                               # a_max = 0.017 and 0.068
        F0 = rng.uniform(-30, 30)
        a = K * h * math.log(2.0)
        b = np.array([[_bessel_i(n, am) * (1 if n == 0 else 2) for n in range(4)] for am in a])
        base = 2.0 ** (A + K * F0)
        C = np.array([[np.sum(base * gk * b[:, n]) for n in range(4)] for gk in g])
        for x in np.linspace(-1, 1, 21):
            T = [1.0, x, 2 * x * x - 1, x * (4 * x * x - 3)]
            w = 2.0 ** (A + K * (F0 + h * x))
            for k in range(3):
                exact = np.sum(w * g[k])
                approx = sum(C[k, n] * T[n] for n in range(4))
                amax = float(np.max(np.abs(a)))
                assert abs(approx / exact - 1) < max(1e-12, (amax / 2) ** 4 / 6)


def test_small_phi_centred_moment_series(orc):
    """The contracted small-phase form: about the span centre z0 = L/2,
    S e^{-j phi z0} = sum_n (j phi)^n / n! nu_n with nu_n = sum_m p_m dz_m g_n(m)
    and g_n(m) the mean of (zeta - z0)^n over step m (the step's sinc times its
    phasor is the mean of e^{j phi zeta} over the step).  |S|^2 = A^2 + B^2
    matches the direct z-sum within the truncation bound 2 (phi L / 2)^{N+1} /
    (N+1)!: to 5e-8 for N = 10 and |phi| L <= 2 (the adjoint), to 2e-8 for
    N = 18 and |phi| L <= 6 (the forward kernels)."""
    import math
    L = 80.0
    ze = orc.zgrid(L, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    lo, hi = ze[:-1] - L / 2, ze[1:] - L / 2
    rng = np.random.default_rng(5)
    for N, T, tol in ((10, 2.0, 5e-8), (18, 6.0, 2e-8)):
        g = np.array([(hi ** (n + 1) - lo ** (n + 1)) / ((n + 1) * (hi - lo)) for n in range(N + 1)])
        f = np.array([(-1) ** (n // 2) / math.factorial(n) for n in range(N + 1)])
        worst, worst_bound = 0.0, -1.0
        for _ in range(40):
            a, k = rng.uniform(0.0, 0.2), rng.uniform(-0.1, 0.1)
            p = np.exp(-a * zm + k * np.sin(zm / 7)) * rng.uniform(0.5, 2)
            nu = f * (g @ (p * dz))
            for x in np.concatenate([rng.uniform(-T, T, 12), [T, -T, 1e-4]]):
                ph = x / L
                A = sum(nu[n] * ph ** n for n in range(0, N + 1, 2))
                B = sum(nu[n] * ph ** n for n in range(1, N + 1, 2))
                exact = abs(orc.zsum(zm, dz, p, ph)) ** 2
                err = abs((A * A + B * B) / exact - 1)
                worst = max(worst, err)
                # within the truncation bound, up to FP64 rounding of the sums
                worst_bound = max(worst_bound, err - 2 * (abs(x) / 2) ** (N + 1) / math.factorial(N + 1))
        assert worst < tol, (N, worst)
        assert worst_bound < 1e-12, (N, worst_bound)


def test_chebyshev_contraction_two_offsets(orc):
    """The tabulated (Raman-ODE) profile: log2 w_m = Ad_m + Sa_m da + Sb_m db
    with da = h_a x, db = h_b y the offsets of F_a, F_b inside their channels.
    Then w_m = base_m e^{alpha_m x} e^{beta_m y} (alpha = Sa h_a ln 2, beta =
    Sb h_b ln 2), and the moments nu_n = sum_m w_m g_n(m) equal
    sum_{k,l <= 3} C_nkl T_k(x) T_l(y) with C_nkl = sum_m base_m b_k(alpha_m)
    b_l(beta_m) g_n(m); the truncation is that of each 1-D expansion."""
    import math
    L = 80.0
    ze = orc.zgrid(L, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    lo, hi = ze[:-1] - L / 2, ze[1:] - L / 2
    g = np.array([(hi ** (n + 1) - lo ** (n + 1)) / ((n + 1) * (hi - lo)) for n in range(11)])
    rng = np.random.default_rng(6)
    Ad = np.log2(dz) - 0.05 * zm / math.log(2.0) + rng.normal(0, 0.1, len(zm))
    Sa = -np.linspace(0.0, 0.5, len(zm)) / math.log(2.0)
    Sb = -np.linspace(0.0, 0.4, len(zm)) / math.log(2.0) + 0.02
    for ha, hb in ((0.048, 0.048), (0.048, 0.19)):
        alpha, beta = Sa * ha * math.log(2.0), Sb * hb * math.log(2.0)
        bk = np.array([[_bessel_i(k, a) * (1 if k == 0 else 2) for k in range(4)] for a in alpha])
        bl = np.array([[_bessel_i(k, b) * (1 if k == 0 else 2) for k in range(4)] for b in beta])
        base = 2.0 ** Ad
        C = np.einsum("m,mk,ml,nm->nkl", base, bk, bl, g)
        amax = float(max(np.max(np.abs(alpha)), np.max(np.abs(beta))))
        tol = max(1e-12, 2 * (amax / 2) ** 4 / 6)
        for x, y in rng.uniform(-1, 1, (25, 2)):
            Tx = np.array([1.0, x, 2 * x * x - 1, x * (4 * x * x - 3)])
            Ty = np.array([1.0, y, 2 * y * y - 1, y * (4 * y * y - 3)])
            w = 2.0 ** (Ad + Sa * ha * x + Sb * hb * y)
            for n in (0, 1, 2, 5, 10):
                exact = np.sum(w * g[n])
                approx = Tx @ C[n] @ Ty
                scale = np.sum(np.abs(w * g[n]))
                assert abs(approx - exact) <= tol * scale, (n, abs(approx - exact) / scale, tol)


def test_segmented_moment_series(orc):
    """The segmented small-phase form: cut the span at step edges into J
    segments (centres c_s) and S = sum_s e^{j phi c_s} sum_n (j phi)^n / n!
    nu_n^s, nu_n^s = sum_{m in s} p_m dz_m g_n^s(m), g_n^s(m) the mean of
    (zeta - c_s)^n over step m, an exact rewriting of the z-sum; with 19
    moments and |phi| (longest segment) <= 6 each segment is truncated below
    2e-8 of its size.  |S|^2 matches the oracle's direct z-sum on the 80 km
    grid for J = 2, 4, 8 (boundaries at the edges nearest s L / J) up to the
    phase each J allows (|phi| L ~ 12, 22, 42), where segments cancel."""
    import math
    L, N = 80.0, 18
    ze = orc.zgrid(L, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    M = len(zm)
    f = np.array([(-1) ** (n // 2) / math.factorial(n) for n in range(N + 1)])
    rng = np.random.default_rng(9)
    for J in (2, 4, 8):
        b = [0]
        for s in range(1, J):
            e = int(np.argmin(np.abs(ze - s * L / J)))
            if b[-1] < e < M:
                b.append(e)
        b.append(M)
        lmax = max(ze[b[i + 1]] - ze[b[i]] for i in range(len(b) - 1))
        phmax = 6.0 / lmax
        for _ in range(20):
            a, k = rng.uniform(0.0, 0.2), rng.uniform(-0.1, 0.1)
            p = np.exp(-a * zm + k * np.sin(zm / 7)) * rng.uniform(0.5, 2)
            for ph in np.concatenate([rng.uniform(-phmax, phmax, 8), [phmax, -phmax]]):
                S = 0j
                for i in range(len(b) - 1):
                    m0, m1 = b[i], b[i + 1]
                    c = 0.5 * (ze[m0] + ze[m1])
                    lo, hi = ze[m0:m1] - c, ze[m0 + 1:m1 + 1] - c
                    g = np.array([(hi ** (n + 1) - lo ** (n + 1)) / ((n + 1) * (hi - lo)) for n in range(N + 1)])
                    nu = f * (g @ (p[m0:m1] * dz[m0:m1]))
                    A = sum(ph ** n * nu[n] for n in range(0, N + 1, 2))
                    B = sum(ph ** n * nu[n] for n in range(1, N + 1, 2))
                    S += np.exp(1j * ph * c) * (A + 1j * B)
                exact = orc.zsum(zm, dz, p, ph)
                # each segment within 2e-8 of its size; the parts cancel in S
                bound = 2e-8 * np.sum(p * dz) + 1e-13 * abs(exact)
                assert abs(S - exact) < bound, (J, ph * L, abs(S - exact), bound)
        assert phmax * L > {2: 11.0, 4: 21.0, 8: 40.0}[J]


def test_mci_cell_rows_with_tabulated_profile(orc):
    """k_quad_mci_f32_tab forms log2 p_m of an MCI point from its cell's row
    {A + log2 dz, S_a, S_b} (A = (a_a + a_b - a_i)/2 log2 e, S = b/2 log2 e)
    and the FP32 row {a_c, b_c}/2 log2 e of its F_c channel:
        log2 p_m dz_m = row.x + S_a da + S_b db + T_c.x + T_c.y dc,
    da, db, dc the point's offsets from the channel centres.  This equals
    log2 of p_m dz_m from the oracle's ln rho (Eq. pk with the Raman-ODE
    tables) to FP32 rounding (measured 8.7e-7 in log2 units on the 589-ch
    plan, a 6e-7 relative error of p; bound 4e-6)."""
    from paper_2401_18022_gb300 import workloads as W
    wl = W.raman(W.uwb(G=8, n_edges=57), ode_h_km=1.0)
    a, b, _ = orc.raman_profile(wl)
    f = wl.f_THz
    ze = orc.zgrid(wl.L_km, wl.alpha_R_per_km, wl.n_edges)
    dz = np.diff(ze)
    l2e = 1.0 / np.log(2.0)
    af = (0.5 * l2e * a).astype(np.float32)
    bf = (0.5 * l2e * b).astype(np.float32)
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(200):
        i, ca, cb = rng.integers(0, wl.n_ch, 3)
        Fa = f[ca] + rng.uniform(-0.048, 0.048)
        Fb = f[cb] + rng.uniform(-0.048, 0.048)
        Fc = Fa + Fb - f[i]
        cc = int(np.argmin(np.abs(f - Fc)))
        if abs(Fc - f[cc]) > 0.048:
            continue
        # the oracle's definition, FP64
        lnp = 0.5 * ((a[ca] + b[ca] * (Fa - f[ca])) + (a[cb] + b[cb] * (Fb - f[cb]))
                     + (a[cc] + b[cc] * (Fc - f[cc])) - a[i])
        ref = lnp * l2e + np.log2(dz)
        # the kernel's rows and FP32 arithmetic
        A = (af[ca] + af[cb]) - af[i]
        rowx = A + np.log2(dz).astype(np.float32)
        da, db, dc = np.float32(Fa - f[ca]), np.float32(Fb - f[cb]), np.float32(Fc - f[cc])
        got = rowx + bf[ca] * da + bf[cb] * db + bf[cc] * dc + af[cc]
        worst = max(worst, float(np.max(np.abs(got.astype(np.float64) - ref))))
    assert worst < 4e-6, worst
