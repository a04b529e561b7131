"""Pins of the oracle's Raman-ODE power profile (profile model R2: Sec. III
and App. A, the Raman power-evolution ODEs with Aeff-scaled gain).

Each pin is a fact that holds independently of the oracle's RK4 code:
  * with uniform attenuation, no cut-off, no photon ratio and equal scales
    the ODE has the closed-form linear-slope solution (the R1 profile with
    line channels), which the oracle's R1 function also gives;
  * two channels with a photon ratio and unequal Aeff scales obey a logistic
    law (a conserved weighted photon number);
  * without loss the photon number sum P_i / f_i is conserved, and without
    the photon ratio the power sum is;
  * channels farther apart than the cut-off only attenuate;
  * an empty slot is a zero-power probe: it changes nothing else;
  * RK4 converges at fourth order.
"""
import math

import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W


def _closed_form(f, P, alpha, Cr, f_ref, z):
    """ln rho_c(z) of line channels under a linear gain slope, uniform alpha."""
    Pt = P.sum()
    kap = Pt * Cr * (1 - math.exp(-alpha * z)) / alpha
    lnN = np.log(np.sum(P * np.exp(-kap * (f - f_ref))))
    return -alpha * z + math.log(Pt) - lnN - kap * (f - f_ref)


def _nodes(L, n_seg):
    z = np.linspace(0.0, L, n_seg + 1)
    return z


def test_linear_slope_limit_matches_closed_form(orc):
    rng = np.random.default_rng(3)
    n = 12
    f = 190.0 + np.sort(rng.uniform(0, 12, n))
    P = W.dbm_to_w(rng.uniform(-2, 6, n))
    alpha, Cr, f_ref = 0.05, 0.5, 195.0
    z = _nodes(80.0, 16)
    y = orc.raman_solve(f, P, np.full(n, alpha), Cr, 0.0, 0, z, np.full(16, 100))
    for s in (4, 9, 16):
        want = _closed_form(f, P, alpha, Cr, f_ref, z[s])
        np.testing.assert_allclose(y[s] - y[0], want, atol=1e-10)
        # the oracle's own closed-form profile with vanishing channel width
        tiny_B = np.full(n, 1e-9)
        r1 = [orc.lnrho(f, tiny_B, P, np.full(n, alpha), f_ref, Cr, alpha, z[s], fc) for fc in f]
        np.testing.assert_allclose(y[s] - y[0], r1, atol=1e-10)
    # the tilt is large enough to matter: several nepers across the plan
    assert np.ptp(y[-1] - y[0]) > 1.5


def test_rk4_fourth_order(orc):
    n = 6
    f = 191.0 + 2.0 * np.arange(n)
    P = W.dbm_to_w(np.array([3.0, 0.0, 5.0, 1.0, 4.0, 2.0]))
    alpha, Cr, f_ref = 0.05, 0.2, 196.0
    z = np.array([0.0, 80.0])
    exact = _closed_form(f, P, alpha, Cr, f_ref, 80.0)
    err = []
    for ns in (8, 16, 32):
        y = orc.raman_solve(f, P, np.full(n, alpha), Cr, 0.0, 0, z, [ns])
        err.append(np.max(np.abs(y[1] - y[0] - exact)))
    assert 12.0 < err[0] / err[1] < 20.0 and 12.0 < err[1] / err[2] < 20.0


def test_two_channel_logistic_with_photon_ratio_and_scales(orc):
    fs, fp = 190.0, 201.0
    f = np.array([fs, fp])
    P0 = np.array([2e-3, 30e-3])
    alpha, Cr = 0.045, 0.05
    sc = np.array([1.3, 0.8])                  # s_s, s_p
    z = _nodes(60.0, 6)
    y = orc.raman_solve(f, P0, np.full(2, alpha), Cr, 15.0, 1, z, np.full(6, 200), scale=sc)
    g, r = Cr * (fp - fs), fp / fs
    K = sc[1] * r * P0[0] + sc[0] * P0[1]      # s_p r Q_s + s_s Q_p is conserved
    for s in range(1, 7):
        zeta = (1 - math.exp(-alpha * z[s])) / alpha
        e = math.exp(g * K * zeta)
        Qs = P0[0] * e / (1 + sc[1] * r * P0[0] / K * (e - 1))
        Qp = (K - sc[1] * r * Qs) / sc[0]
        np.testing.assert_allclose(y[s], np.log([Qs, Qp]) - alpha * z[s], atol=1e-11)
    assert y[-1][0] - y[0][0] > -alpha * 60.0 + 0.1     # the signal gains


@pytest.mark.parametrize("photon", [0, 1])
def test_lossless_invariants(orc, photon):
    rng = np.random.default_rng(5)
    n = 30
    f = 185.0 + np.sort(rng.uniform(0, 40, n))
    P = W.dbm_to_w(rng.uniform(0, 10, n))
    z = _nodes(80.0, 8)
    y = orc.raman_solve(f, P, np.zeros(n), 0.05, 15.0, photon, z, np.full(8, 80))
    Pz = np.exp(y)
    if photon:
        photons = (Pz / f).sum(1)
        np.testing.assert_allclose(photons, photons[0], rtol=1e-10)
        assert Pz[-1].sum() < Pz[0].sum() * (1 - 1e-4)          # energy lost to the photon defect
    else:
        np.testing.assert_allclose(Pz.sum(1), Pz[0].sum(), rtol=1e-10)
    assert np.ptp(y[-1] - y[0]) > 0.5


def test_cutoff_leaves_distant_channels_alone(orc):
    f = np.array([185.0, 205.0])                # 20 THz apart, cut-off 15 THz
    P = np.array([0.05, 0.05])
    a = np.array([0.04, 0.06])
    z = _nodes(80.0, 4)
    y = orc.raman_solve(f, P, a, 0.05, 15.0, 1, z, np.full(4, 7))
    for s in range(5):
        np.testing.assert_allclose(y[s], np.log(P) - a * z[s], rtol=0, atol=1e-13)
    # without the cut-off they interact
    y2 = orc.raman_solve(f, P, a, 0.05, 0.0, 1, z, np.full(4, 7))
    assert y2[-1][0] - y[-1][0] > 0.1


def test_empty_slot_is_a_probe(orc):
    f = np.array([190.0, 193.0, 199.0])
    P = np.array([5e-3, 0.0, 40e-3])
    a = np.full(3, 0.046)
    z = _nodes(80.0, 5)
    y = orc.raman_solve(f, P, a, 0.05, 15.0, 1, z, np.full(5, 40))
    y2 = orc.raman_solve(f[[0, 2]], P[[0, 2]], a[[0, 2]], 0.05, 15.0, 1, z, np.full(5, 40))
    np.testing.assert_allclose(y[:, [0, 2]], y2, atol=1e-14)
    P3 = P.copy()
    P3[1] = 1e-30                               # a real channel of negligible power
    y3 = orc.raman_solve(f, P3, a, 0.05, 15.0, 1, z, np.full(5, 40))
    np.testing.assert_allclose(y[:, 1], y3[:, 1] - y3[0, 1], atol=1e-12)


def test_profile_tables_reduce_to_closed_form_inside_channels(orc):
    """Linear-slope limit with equal channel widths B: the closed form of a
    channel with a rectangular spectrum differs from the line-channel one by
    the normaliser factor sinhc(kappa B / 2), the same for every F, so
      a + b (F - f_c) = ln rho_R1(z_m, F) + ln sinhc(kappa_m B / 2)."""
    wl = W.tiny(G=8, n_edges=17).with_(Cr=0.3)
    wl2 = W.raman(wl, raman_max_THz=0.0, photon=0, ode_h_km=0.02, aeff_scaling=False)
    a, b, aL = orc.raman_profile(wl2)
    z = orc.zgrid(wl.L_km, wl.alpha_R_per_km, wl.n_edges)
    zm = 0.5 * (z[1:] + z[:-1])
    Pt = wl.P_W.sum()
    B = wl.B_THz[0]
    for m in (0, 7, 15):
        kap = Pt * wl.Cr * orc.leff(zm[m], wl.alpha_R_per_km)
        corr = math.log(math.sinh(0.5 * kap * B) / (0.5 * kap * B))
        for c in range(wl.n_ch):
            for F in (wl.f_THz[c] - 0.047, wl.f_THz[c], wl.f_THz[c] + 0.03):
                r1 = orc.lnrho(wl.f_THz, wl.B_THz, wl.P_W, wl.alpha_per_km, wl.f_ref_THz, wl.Cr,
                               wl.alpha_R_per_km, zm[m], F)
                got = a[c, m] + b[c, m] * (F - wl.f_THz[c])
                assert got == pytest.approx(r1 + corr, abs=1e-10)
    kapL = Pt * wl.Cr * orc.leff(wl.L_km, wl.alpha_R_per_km)
    corrL = math.log(math.sinh(0.5 * kapL * B) / (0.5 * kapL * B))
    for c in range(wl.n_ch):
        r1 = orc.lnrho(wl.f_THz, wl.B_THz, wl.P_W, wl.alpha_per_km, wl.f_ref_THz, wl.Cr,
                       wl.alpha_R_per_km, wl.L_km, wl.f_THz[c])
        assert aL[c] == pytest.approx(r1 + corrL, abs=1e-10)


def test_sigma_r2_without_raman_equals_r1(orc):
    """C_r = 0: both profiles are pure attenuation (RK4 is exact for a
    constant right-hand side)."""
    wl = W.tiny(G=16, n_edges=25).with_(Cr=0.0, alpha_per_km=np.linspace(0.04, 0.05, 5))
    s1 = orc.sigma(wl)
    s2 = orc.sigma(W.raman(wl))
    np.testing.assert_allclose(s2, s1, rtol=1e-12)
    e1, _ = orc.eta(wl, s1)
    r1 = orc.snr_throughput(wl, e1)
    r2 = orc.snr_throughput(W.raman(wl), e1)
    np.testing.assert_allclose(r2[1], r1[1], rtol=1e-12)


def test_sigma_r2_linear_limit_matches_r1_for_narrow_channels(orc):
    """Narrow channels (B = 1 GHz, kappa B / 2 < 2e-4): the R1 and R2 profiles
    agree to (kappa B)^2 / 24 inside every channel, so Sigma does too."""
    wl = W.tiny(G=12, n_edges=25).with_(Cr=0.1, B_THz=np.full(5, 0.001))
    s1 = orc.sigma(wl)
    s2 = orc.sigma(W.raman(wl, raman_max_THz=0.0, photon=0, ode_h_km=0.05, aeff_scaling=False))
    np.testing.assert_allclose(s2, s1, rtol=1e-7)


def test_uwb_cutoff_bounds_the_tilt(orc):
    """With the 15 THz cut-off the end-of-span tilt over 59 THz stays a few
    nepers, far below the linear-slope closed form's."""
    wl = W.uwb(G=8, n_edges=17)
    _, _, aL = orc.raman_profile(W.raman(wl, ode_h_km=0.5))
    r2 = aL + wl.alpha_per_km * wl.L_km
    Pt = wl.P_W.sum()
    kapL = Pt * wl.Cr * orc.leff(wl.L_km, wl.alpha_R_per_km)
    assert np.ptp(r2) < 0.25 * kapL * np.ptp(wl.f_THz)
    assert r2[0] > r2[-1]                       # low frequencies gain, high ones deplete
