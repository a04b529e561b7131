"""GPU checks of the hand-written adjoint (isrs_gn_grad) of the throughput.

The adjoint differentiates the FP32 quadrature analytically.  It is compared
with central finite differences, in dB of launch power with a 1e-4 dB step,
of (a) the plain FP64 GPU path and (b) the FP64 CPU oracle.  Finite
differences are never taken on the FP32 path: a 1e-4 dB step changes P by
2.3e-5 relative, close to the FP32 rounding of its tables.

Tolerance: 1e-3 relative per channel (floored at 1e-3 of the largest
component), the target stated for the method.
"""
import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_DB = 1e-4
RTOL = 1e-3


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    return api.Engine(0)


def _fd(T_of_P, P, chans):
    """dT/dP_j by central differences in dBm: dT/dP = (dT/dx) / (P ln10/10)."""
    g = np.zeros(len(chans))
    for k, j in enumerate(chans):
        Pp, Pm = P.copy(), P.copy()
        Pp[j] = P[j] * 10 ** (STEP_DB / 10)
        Pm[j] = P[j] * 10 ** (-STEP_DB / 10)
        dTdx = (T_of_P(Pp) - T_of_P(Pm)) / (2 * STEP_DB)
        g[k] = dTdx / (P[j] * np.log(10) / 10)
    return g


def _check(adj, fd):
    floor = RTOL * np.max(np.abs(fd))
    err = np.abs(adj - fd) / np.maximum(np.abs(fd), floor)
    assert err.max() < RTOL, (err.max(), adj, fd)


@pytest.mark.parametrize("trx", [0.0, 20.0])
@pytest.mark.parametrize("cells", [W.CELLS_SCI_XCI, W.CELLS_ALL])
def test_adjoint_vs_fd_of_fp64_path_tiny(eng, trx, cells):
    wl = W.tiny(G=48, n_edges=57, cell_set=cells).with_(snr_trx_dB=trx)
    P = wl.P_W * W.dbm_to_w(W.random_profile_dbm(5, seed=5)) / 1e-3
    r = eng.grad(wl, P=P)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], P, range(5))
    _check(r["dT_dP"], fd)
    # the forward outputs of the gradient call equal those of isrs_gn_snr
    s = eng.snr(wl, P=P, precision=0)
    np.testing.assert_allclose(r["snr"], s["snr"], rtol=1e-6)
    # the two kernels truncate the small-phase series at different orders
    # (19 and 11 moments), each within 5e-8 of the exact z-sum
    assert r["T"] == pytest.approx(s["T"], rel=1e-7)


def test_adjoint_vs_fd_of_oracle(eng, orc):
    wl = W.tiny(G=16, n_edges=17).with_(Cr=0.5)          # strong ISRS tilt
    P = W.dbm_to_w(W.random_profile_dbm(5, seed=7, lo=-1, hi=4))
    r = eng.grad(wl, P=P)
    fd = _fd(lambda Q: orc.evaluate(wl, P=Q)["T"], P, range(5))
    _check(r["dT_dP"], fd)


def test_adjoint_oband_zero_dispersion(eng):
    """41 channels at lambda0: beta2 = 0, MCI-heavy low dispersion, all cells."""
    wl = W.oband(G=12, n_edges=33)
    chans = [0, 9, 20, 31, 40]
    r = eng.grad(wl)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], wl.P_W, chans)
    _check(r["dT_dP"][chans], fd)


def test_adjoint_uwb_589_sampled_channels(eng):
    """The 589-channel system: FD on the 16 seeded channels (G = 8 to bound
    the cost of the 32 FP64 evaluations)."""
    wl = W.uwb(G=8)
    chans = W.gradient_fd_channels()
    r = eng.grad(wl)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], wl.P_W, chans)
    _check(r["dT_dP"][chans], fd)


def test_grad_rejects_bad_arguments(eng):
    from paper_2401_18022_gb300._capi import IsrsError
    wl = W.tiny(G=8)
    P = wl.P_W.copy()
    P[2] = 0.0
    with pytest.raises(IsrsError):
        eng.grad(wl, P=P)
    with pytest.raises(IsrsError):
        eng.grad(wl.with_(n_edges=200))


def test_adjoint_multispan(eng):
    wl = W.tiny(G=32, n_edges=41).with_(n_spans=4)
    r = eng.grad(wl)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], wl.P_W, range(5))
    _check(r["dT_dP"], fd)


def test_adjoint_strong_raman_tilt_per_step_small_phase(eng):
    """kappa(L) B/2 > 0.05: no contracted small-phase points; the adjoint's
    small-phase points are walked step by step on half-warps."""
    wl = W.tiny(G=32, n_edges=41).with_(Cr=8.0)
    P = np.full(wl.n_ch, W.dbm_to_w(4.0)) * W.dbm_to_w(W.random_profile_dbm(5, seed=9, lo=-1, hi=1)) / 1e-3
    r = eng.grad(wl, P=P)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], P, range(5))
    _check(r["dT_dP"], fd)


def test_adjoint_many_fc_candidates(eng):
    from _plans import wide_cut_plan
    wl = wide_cut_plan(G=32)
    r = eng.grad(wl)
    chans = [0, 4, 5, 6, 10]
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], wl.P_W, chans)
    _check(r["dT_dP"][chans], fd)
    # the gradient call's forward outputs equal the forward kernel's
    s = eng.snr(wl, precision=0)
    np.testing.assert_allclose(r["snr"], s["snr"], rtol=1e-6)


@pytest.mark.parametrize("G,n_edges", [(8, 2), (5, 3), (1, 18)])
def test_adjoint_degenerate_grids(eng, G, n_edges):
    """One z-step (15 of the 16 half-warp lanes hold padding steps), two
    steps, and a single grid point per piece."""
    wl = W.tiny(G=G, n_edges=n_edges, cell_set=W.CELLS_SCI_XCI)
    P = wl.P_W * W.dbm_to_w(W.random_profile_dbm(5, seed=11)) / 1e-3
    r = eng.grad(wl, P=P)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], P, range(5))
    _check(r["dT_dP"], fd)


@pytest.mark.parametrize("case", ["uwb", "wide", "raman", "mci"])
def test_gradient_is_bit_reproducible(eng, case):
    """Every reduction of the adjoints has a fixed order (each tile's buckets go
    to rows only that tile writes, summed per CUT or per channel in tile order),
    so two gradient calls return the same bits: the 589-ch plan, a plan with six
    F_c candidates per piece (past the four register buckets), the Raman-ODE
    profile and the MCI cells of a separate grid."""
    from _plans import wide_cut_plan
    wl = {"uwb": W.uwb(G=16, n_edges=33),
          "wide": wide_cut_plan(G=24).with_(n_edges=33),
          "raman": W.raman(W.uwb(G=8, n_edges=33), ode_h_km=0.5),
          "mci": W.tiny(G=16, n_edges=33).with_(G_mci=8)}[case]
    a = eng.grad(wl)
    b = eng.grad(wl)
    np.testing.assert_array_equal(a["dT_dP"], b["dT_dP"])
    np.testing.assert_array_equal(a["eta"], b["eta"])
    assert a["T"] == b["T"]


def test_adjoint_single_channel_zero_dispersion_closed_form(eng):
    """One channel, beta2 = beta3 = beta4 = 0, C_r = 0, uniform alpha: phi = 0
    and the profile does not depend on P, so eta is a constant and Sigma is
    P^3 times a constant (the adjoint's PSD bucket gives dSigma/dP = 3 Sigma/P,
    its profile buckets vanish).  With N = eta P^3 + P_ASE (P_ASE fixed,
    G = e^{alpha L}): dT/dP = 2B / (ln 2 (1 + SNR)) (N - 3 eta P^3) / N^2."""
    import math
    Bw, a, L = 0.096, 0.046, 80.0
    wl = W.tiny(G=64, n_edges=57).with_(
        f_THz=np.array([193.4]), B_THz=np.array([Bw]), P_W=np.array([2e-3]), alpha_per_km=np.array([a]),
        lambda_nm=np.array([1550.0]), aeff_um2=np.array([80.0]), nf_dB=np.array([5.0]), Cr=0.0,
        gamma_fixed=1.3, alpha_R_per_km=a, D_ref=0.0, S_ref=0.0, Sdot_ref=0.0, cell_set=W.CELLS_SCI_XCI)
    for P in (1e-3, 5e-3, 2e-2):
        g = eng.grad(wl, P=np.array([P]))
        eta = float(g["eta"][0])
        pase = 10 ** 0.5 * 6.62607015e-34 * 193.4e12 * (math.exp(a * L) - 1) * Bw * 1e12
        N = eta * P ** 3 + pase
        snr = P / N
        ref = 2 * Bw / (math.log(2) * (1 + snr)) * (N - 3 * eta * P ** 3) / N ** 2
        assert float(g["snr"][0]) == pytest.approx(snr, rel=1e-9)
        # the PSD bucket of F_c is an FP32 (uncompensated) lane sum: ~1e-6 relative
        assert float(g["dT_dP"][0]) == pytest.approx(ref, rel=1e-5)
