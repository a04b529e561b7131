"""GPU parity of the multi-channel-interference (MCI) cells on their own grid
(App. A: the integral of Eq. gain_fin over the whole band) against the FP64
oracle with the same grids, through the C ABI.

The SCI and XCI cells keep their G x G pieces; every cell (a, b) with
neither F_a nor F_b in the CUT's channel gets a G_mci x G_mci grid and is
enumerated on the device.  Tolerances are those of the single-grid path:
1e-9 (FP64), 2e-4 (FP32).
"""
import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL_F64 = 1e-9
RTOL_F32 = 2e-4


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    return api.Engine(0)


@pytest.mark.parametrize("prec,rtol", [(1, RTOL_F64), (0, RTOL_F32)])
def test_tiny_all_cuts(eng, orc, prec, rtol):
    wl = W.tiny(G=32, n_edges=41, cell_set=W.CELLS_ALL).with_(G_mci=8)
    np.testing.assert_allclose(eng.eta(wl, precision=prec)["sigma"], orc.sigma(wl), rtol=rtol)


@pytest.mark.parametrize("prec,rtol", [(1, RTOL_F64), (0, RTOL_F32)])
def test_oband_zero_dispersion(eng, orc, prec, rtol):
    """41 channels at lambda0: MCI is about half of eta at the centre."""
    wl = W.oband(G=16, n_edges=33, cell_set=W.CELLS_ALL).with_(G_mci=6)
    cuts = [0, 11, 20, 33, 40]
    ref = orc.sigma(wl, cuts=cuts)
    np.testing.assert_allclose(eng.eta(wl, cuts=cuts, precision=prec)["sigma"], ref, rtol=rtol)
    sx = orc.sigma(wl.with_(cell_set=W.CELLS_SCI_XCI, G_mci=0), cuts=cuts)
    assert 1 - sx[2] / ref[2] > 0.3


def test_same_grid_equals_single_grid(eng):
    wl = W.tiny(G=12, n_edges=25, cell_set=W.CELLS_ALL)
    a = eng.eta(wl, precision=1)["sigma"]
    b = eng.eta(wl.with_(G_mci=12), precision=1)["sigma"]
    np.testing.assert_allclose(b, a, rtol=1e-12)


def test_uwb_sampled_cuts(eng, orc):
    """589 channels: 173,166 MCI cells per CUT, phases up to ~1e7
    revolutions in the far cells (the wide FP32 phase reduction)."""
    wl = W.uwb(G=8, n_edges=33, cell_set=W.CELLS_ALL).with_(G_mci=3)
    cuts = [0, 294, 588]
    ref = orc.sigma(wl, cuts=cuts)
    np.testing.assert_allclose(eng.eta(wl, cuts=cuts, precision=0)["sigma"], ref, rtol=RTOL_F32)


def test_snr_and_batched(eng, orc):
    wl = W.oband(G=12, n_edges=25, cell_set=W.CELLS_ALL).with_(G_mci=4)
    r = orc.evaluate(wl)
    s = eng.snr(wl, precision=1)
    np.testing.assert_allclose(s["snr"], r["snr"], rtol=1e-9)
    bw = W.BatchedWorkload(plans=[wl, W.subset_plan(wl, np.arange(0, 41, 2), "odd").with_(G_mci=4)],
                           plan_of_profile=np.array([0, 1, 0]),
                           P_W=[wl.P_W, wl.P_W[::2].copy(), wl.P_W * 1.3])
    eta_b = eng.eta_batched(bw)
    off = 0
    for p in range(3):
        pl = bw.plans[bw.plan_of_profile[p]]
        np.testing.assert_array_equal(eta_b[off:off + pl.n_ch], eng.eta(pl, P=bw.P_W[p])["eta"])
        off += pl.n_ch


def test_rejections(eng):
    from paper_2401_18022_gb300._capi import IsrsError
    wl = W.tiny(G=8, n_edges=17)
    with pytest.raises(IsrsError):
        eng.eta(wl.with_(cell_set=W.CELLS_SCI_XCI, G_mci=4))
    with pytest.raises(IsrsError):
        eng.eta(wl.with_(cell_set=W.CELLS_ALL, G_mci=33))
    with pytest.raises(IsrsError):
        eng.grad(W.raman(wl.with_(cell_set=W.CELLS_ALL, G_mci=4)))


STEP_DB = 1e-4


def _fd(T_of_P, P, chans):
    """dT/dP_j by central differences in dBm (1e-4 dB) of the FP64 path."""
    g = np.zeros(len(chans))
    for k, j in enumerate(chans):
        Pp, Pm = P.copy(), P.copy()
        Pp[j] = P[j] * 10 ** (STEP_DB / 10)
        Pm[j] = P[j] * 10 ** (-STEP_DB / 10)
        g[k] = (T_of_P(Pp) - T_of_P(Pm)) / (2 * STEP_DB) / (P[j] * np.log(10) / 10)
    return g


@pytest.mark.parametrize("case", ["tiny", "oband"])
def test_adjoint_with_mci_grid_vs_fd(eng, case):
    """The gradient over SCI/XCI pieces plus the MCI cells of their own grid
    against central differences of the FP64 path (same cells, same grids),
    1e-3 relative per channel (floored at 1e-3 of the largest component)."""
    if case == "tiny":
        wl = W.tiny(G=32, n_edges=41, cell_set=W.CELLS_ALL).with_(G_mci=8)
        P = wl.P_W * W.dbm_to_w(W.random_profile_dbm(5, seed=12)) / 1e-3
        chans = list(range(5))
    else:
        wl = W.oband(G=12, n_edges=33, cell_set=W.CELLS_ALL).with_(G_mci=6)
        P = wl.P_W
        chans = [0, 9, 20, 31, 40]
    r = eng.grad(wl, P=P)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], P, chans)
    adj = np.asarray(r["dT_dP"].cpu() if hasattr(r["dT_dP"], "cpu") else r["dT_dP"])[chans]
    floor = 1e-3 * np.max(np.abs(fd))
    err = np.abs(adj - fd) / np.maximum(np.abs(fd), floor)
    assert err.max() < 1e-3, (err.max(), adj, fd)
    # the gradient call's forward outputs include the MCI cells
    s = eng.snr(wl, P=P, precision=0)
    snr_g = np.asarray(r["snr"].cpu() if hasattr(r["snr"], "cpu") else r["snr"])
    np.testing.assert_allclose(snr_g, np.asarray(s["snr"]), rtol=1e-6)


def test_adjoint_with_mci_grid_multispan(eng):
    """Three identical spans: the phased-array factor in the MCI cells too."""
    wl = W.tiny(G=24, n_edges=33, cell_set=W.CELLS_ALL).with_(G_mci=6, n_spans=3)
    r = eng.grad(wl)
    fd = _fd(lambda Q: eng.snr(wl, P=Q, precision=1)["T"], wl.P_W, range(5))
    adj = np.asarray(r["dT_dP"].cpu() if hasattr(r["dT_dP"], "cpu") else r["dT_dP"])
    floor = 1e-3 * np.max(np.abs(fd))
    err = np.abs(adj - fd) / np.maximum(np.abs(fd), floor)
    assert err.max() < 1e-3, (err.max(), adj, fd)
