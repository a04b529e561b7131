"""Host logic of the segment optimiser (Sec. IV): the guarded channel plan and
segment counts against the paper's tables, the interpolation map, the chain
rule of the loss gradient, and L-BFGS-B on a closed-form model whose optimum
is known.

The closed-form model replaces the NLI integral by SNR_i = P_i / (a_i +
P_i sum_j c_ij P_j^2): with c diagonal (c_ii = b_i) each channel's optimum is
P* = (a_i / 2 b_i)^(1/3), the textbook GN optimum launch power.
"""
import json
import math

import numpy as np
import pytest

from paper_2401_18022_gb300 import segments as S
from paper_2401_18022_gb300 import workloads as W


class ToyEngine:
    """grad/snr of T = 2 B sum log2(1 + P_i / (a_i + P_i sum_j c_ij P_j^2))."""

    def __init__(self, a, c):
        self.a, self.c = np.asarray(a, float), np.asarray(c, float)
        self.calls = 0

    def _parts(self, wl, P):
        P = np.asarray(P, float)
        N = self.a + P * (self.c @ (P * P))
        return P, N, P / N

    def snr(self, wl, P=None, precision=0):
        P, N, s = self._parts(wl, P)
        if wl.snr_trx_dB > 0:
            s = 1.0 / (1.0 / s + 10 ** (-wl.snr_trx_dB / 10))
        return {"snr": s, "T": float(2 * np.sum(wl.B_THz * np.log2(1 + s)))}

    def grad(self, wl, P=None):
        self.calls += 1
        P, N, s = self._parts(wl, P)
        q = self.c @ (P * P)
        # dN_i/dP_k = delta_ik q_i + 2 P_i c_ik P_k
        dN = np.diag(q) + 2.0 * P[:, None] * self.c * P[None, :]
        dS = np.diag(1.0 / N) - (P / N ** 2)[:, None] * dN
        w = 2 * wl.B_THz / (math.log(2.0) * (1 + s))
        return {"T": float(2 * np.sum(wl.B_THz * np.log2(1 + s))), "dT_dP": w @ dS, "snr": s}


def _toy_for(wl, p_opt_dbm, coupling=0.0, seed=0):
    """a_i, b_i placing each channel's uncoupled optimum at p_opt_dbm[i]."""
    rng = np.random.default_rng(seed)
    a = 1e-5 * 10 ** (rng.uniform(-0.5, 0.5, wl.n_ch) / 10)
    Pstar = W.dbm_to_w(p_opt_dbm)
    b = a / (2 * Pstar ** 3)
    c = np.diag(b)
    if coupling:
        d = np.abs(wl.f_THz[:, None] - wl.f_THz[None, :])
        c = c + coupling * np.sqrt(b[:, None] * b[None, :]) * np.exp(-d / 2.0) * (1 - np.eye(wl.n_ch))
    return ToyEngine(a, c)


def test_guard_plan_matches_paper_tables():
    loaded, band, guards = W.guard_plan()
    assert len(loaded) == 557 and len(guards) == 32          # N_ch - N_A and N_A
    for b, name in enumerate(W.BAND_NAMES):
        assert int((band == b).sum()) == {"O": 171, "E": 143, "S": 88, "C": 38, "L": 65, "U": 52}[name]
    assert sorted(np.concatenate([loaded, guards]).tolist()) == list(range(589))
    # gaps at U/L, L/C, C/S, S/E, E/O: whole 100 GHz slots within 5 nm
    gaps = [W.guard_gap_slots(e) for e in (1625.0, 1565.0, 1530.0, 1460.0, 1360.0)]
    assert gaps == [5, 6, 6, 7, 8]
    for e, g in zip((1625.0, 1565.0, 1530.0, 1460.0, 1360.0), gaps):
        df = 299792.458 * 5.0 / e ** 2
        assert g * 0.1 <= df < (g + 1) * 0.1
    # every loaded channel sits inside its band's wavelength range; every gap
    # straddles the nominal band edge
    wl = W.uwb_guarded(G=8)
    assert np.array_equal(S.band_of(wl), band)
    lam_g = W.nm_from_thz(W.uwb_slots()[guards])
    for e in (1625.0, 1565.0, 1530.0, 1460.0, 1360.0):
        near = lam_g[np.abs(lam_g - e) < 5.0]
        assert near.min() < e < near.max()


def test_guarded_plan_is_the_full_plan_without_guards():
    full, wl = W.uwb(G=8), W.uwb_guarded(G=8)
    loaded, _, _ = W.guard_plan()
    np.testing.assert_array_equal(wl.f_THz, full.f_THz[loaded])
    np.testing.assert_array_equal(wl.nf_dB, full.nf_dB[loaded])
    assert wl.f_ref_THz == full.f_ref_THz and wl.n_ch == 557


def test_segment_counts_match_paper_table():
    # Table "Per band characteristics": 23/10/6/3/4/3 segments
    want = {"O": 23, "E": 10, "S": 6, "C": 3, "L": 4, "U": 3}
    for name, n in W.TABLE_BAND_COUNTS.items():
        bp = 0.75 if name == "O" else 1.5
        assert S.n_segments(n, bp) == want[name]
    wl = W.uwb_guarded(G=8)
    par = S.segments(wl.f_THz, S.band_of(wl))
    assert par.n_var == sum(v + 1 for v in want.values())     # N_B + 1 edges per band
    assert S.n_segments(5, 1.5) == 0 and S.n_segments(8, 1.5) == 1


def test_interpolation_map_properties():
    wl = W.uwb_guarded(G=8)
    band = S.band_of(wl)
    par = S.segments(wl.f_THz, band)
    M = par.M
    assert np.all(M >= 0) and np.allclose(M.sum(1), 1.0, atol=1e-14)
    assert np.all((M > 0).sum(1) <= 2)
    for i in range(M.shape[0]):
        nz = np.flatnonzero(M[i])
        assert nz.size == 1 or nz[1] == nz[0] + 1            # two adjacent edges
    # a profile linear in frequency inside each band is reproduced exactly
    x = 0.3 + 0.05 * (par.edges_thz - 200.0)
    np.testing.assert_allclose(par.x_ch(x), 0.3 + 0.05 * (wl.f_THz - 200.0), atol=1e-12)
    # the first and last channel of each band take their edge's value
    for b in range(6):
        idx = np.flatnonzero(band == b)
        for i in (idx[0], idx[-1]):
            assert np.isclose(M[i].max(), 1.0)
    # edges equally spaced between the band's first and last channel
    off = 0
    for b in range(5, -1, -1):
        fb = wl.f_THz[band == b]
        n_e = S.n_segments(len(fb), 0.75 if b == 0 else 1.5) + 1
        e = par.edges_thz[off:off + n_e]
        np.testing.assert_allclose(e, np.linspace(fb[0], fb[-1], n_e), rtol=1e-15)
        off += n_e
    # one-channel band: a single edge
    one = S.segments(np.array([200.0, 200.1, 205.0]), np.array([1, 1, 0]))
    assert one.n_var == 3 and np.array_equal(one.M[2], [0.0, 0.0, 1.0])
    np.testing.assert_allclose(one.M[:2], [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


@pytest.mark.parametrize("kind", ["segments", "uniform", "per_channel"])
def test_loss_gradient_chain_rule(kind):
    wl = W.tiny(G=8).with_(B_THz=np.full(5, 0.096))
    band = np.array([5, 5, 4, 4, 4])
    eng = _toy_for(wl, np.linspace(-2, 3, 5), coupling=0.3)
    par = {"segments": S.segments(wl.f_THz, band, {"L": 0.1, "U": 0.1}),
           "uniform": S.uniform(5), "per_channel": S.per_channel(5)}[kind]
    obj = S.Objective(eng, wl, par)
    x = np.random.default_rng(1).uniform(-3, 3, par.n_var)
    L, g = obj(x)
    # L is minus the sum of log2(1 + SNR)
    r = eng.snr(wl, P=obj.powers(x))
    assert L == pytest.approx(-np.sum(np.log2(1 + r["snr"])), rel=1e-14)
    h = 1e-5
    fd = np.array([(obj(x + h * e)[0] - obj(x - h * e)[0]) / (2 * h) for e in np.eye(par.n_var)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())


def test_lbfgsb_reaches_closed_form_optimum():
    wl = W.tiny(G=8).with_(B_THz=np.full(5, 0.096))
    p_opt = np.array([-2.0, -0.5, 0.7, 1.9, 3.3])
    eng = _toy_for(wl, p_opt)
    obj = S.Objective(eng, wl, S.per_channel(5))
    res = S.optimise(obj, gtol=1e-9)
    np.testing.assert_allclose(res["x_dbm"], p_opt, atol=1e-4)
    # the paper's stop condition alone
    obj2 = S.Objective(eng, wl, S.per_channel(5))
    res2 = S.optimise(obj2)
    assert res2["pg_inf"] <= 0.01 and res2["converged"]
    assert res2["T"] > obj2.history[0]["T"]


def test_uniform_case_and_bounds():
    wl = W.tiny(G=8).with_(B_THz=np.full(5, 0.096))
    eng = _toy_for(wl, np.full(5, 1.87), seed=4)
    eng.a[:] = eng.a[0]
    eng.c = np.diag(np.full(5, eng.c[0, 0]))
    res = S.optimise(S.Objective(eng, wl, S.uniform(5)), gtol=1e-10)
    assert res["x_dbm"][0] == pytest.approx(1.87, abs=1e-4)
    # an optimum beyond +5 dBm stops on the bound with a vanishing projected gradient
    eng2 = _toy_for(wl, np.array([0.0, 1.0, 7.0, 9.0, 2.0]))
    res2 = S.optimise(S.Objective(eng2, wl, S.per_channel(5)), gtol=1e-8)
    assert res2["x_dbm"][2] == 5.0 and res2["x_dbm"][3] == 5.0
    assert res2["pg_inf"] <= 1e-6
    assert S.projected_grad_inf([5.0, 0.0], [-3.0, 0.0], -5, 5) == 0.0     # pushing out: inactive
    assert S.projected_grad_inf([5.0, 0.0], [3.0, 0.0], -5, 5) == 3.0


def test_checkpoint_resume(tmp_path):
    wl = W.tiny(G=8).with_(B_THz=np.full(5, 0.096))
    p_opt = np.array([-1.0, 0.5, 1.5, 2.5, -3.0])
    eng = _toy_for(wl, p_opt, coupling=0.2)
    ck = str(tmp_path / "seg.json")
    r1 = S.optimise(S.Objective(eng, wl, S.per_channel(5)), maxiter=2, ckpt=ck)
    x_mid = np.asarray(json.load(open(ck))["x_dbm"])
    np.testing.assert_allclose(x_mid, r1["x_dbm"])
    r2 = S.optimise(S.Objective(eng, wl, S.per_channel(5)), ckpt=ck, gtol=1e-9)
    r3 = S.optimise(S.Objective(eng, wl, S.per_channel(5)), gtol=1e-9)
    np.testing.assert_allclose(r2["x_dbm"], r3["x_dbm"], atol=1e-4)


def test_objective_rejects_mixed_bandwidths():
    wl = W.tiny(G=8).with_(B_THz=np.array([0.096, 0.096, 0.05, 0.096, 0.096]))
    with pytest.raises(ValueError):
        S.Objective(ToyEngine(np.ones(5), np.eye(5)), wl, S.per_channel(5))
    with pytest.raises(ValueError):
        S.Objective(ToyEngine(np.ones(5), np.eye(5)), W.tiny(G=8), S.per_channel(4))


def test_band_report_with_transceiver_noise():
    wl = W.tiny(G=8).with_(B_THz=np.full(5, 0.096))
    eng = _toy_for(wl, np.zeros(5))
    band = np.array([5, 5, 4, 4, 3])
    P = W.dbm_to_w(np.zeros(5))
    r0 = S.band_report(eng, wl, P, band)
    r20 = S.band_report(eng, wl, P, band, snr_trx_dB=20.0)
    assert r0["bands"]["U"]["pow_dBm"] == pytest.approx(10 * np.log10(2), abs=1e-12)
    assert sum(b["cap_Tbps"] for b in r0["bands"].values()) == pytest.approx(r0["T"], rel=1e-12)
    assert r20["T"] < r0["T"]


class _CellsEngine(ToyEngine):
    """ToyEngine that records the cells of every SNR call and adds 1 % more
    noise when the MCI cells are included (whole band)."""

    def __init__(self, a, c):
        super().__init__(a, c)
        self.seen = []

    def snr(self, wl, P=None, precision=0):
        self.seen.append((wl.cell_set, wl.G_mci))
        a0 = self.a
        if wl.cell_set == W.CELLS_ALL and wl.G_mci > 0:
            self.a = a0 * 1.01
        try:
            return super().snr(wl, P, precision)
        finally:
            self.a = a0


def test_run_stages_reports_the_optimum_over_the_whole_band():
    """run_stages optimises over the SCI/XCI cells and, with g_mci > 0,
    evaluates the optimum again with every MCI cell on its own grid."""
    wl = W.uwb_guarded(G=8)
    base = _toy_for(wl, np.full(wl.n_ch, 1.5), seed=5)
    eng = _CellsEngine(base.a, base.c)
    out = S.run_stages(eng, case=2, stages=(8,), g_mci=4)
    assert out["report_mci"]["G_mci"] == 4
    assert out["report_mci"]["T"] < out["report"]["T"]
    assert out["report_mci_trx20"]["T"] < out["report_mci"]["T"]
    assert (W.CELLS_ALL, 4) in eng.seen and (W.CELLS_SCI_XCI, 0) in eng.seen
    plain = S.run_stages(_CellsEngine(base.a, base.c), case=2, stages=(8,))
    assert "report_mci" not in plain
