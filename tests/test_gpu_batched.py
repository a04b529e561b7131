"""Batched persistent launch: CUDA-graph replay and the tile autotuner."""
import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    return api.Engine(0)


def test_graph_replay_reproduces_direct_run(eng):
    import torch
    bw = W.batched(n_prof=9, G=16, n_edges=33, sizes=(60, 31, 12))
    P = torch.tensor(np.concatenate(bw.P_W), dtype=torch.float64, device="cuda")
    first = eng.eta_batched(bw, P).clone()
    assert not eng.last_graph_replay()
    second = eng.eta_batched(bw, P).clone()
    assert eng.last_graph_replay()
    assert torch.equal(first, second)
    # new powers through the same graph
    P2 = P * 1.7
    third = eng.eta_batched(bw, P2)
    assert eng.last_graph_replay()
    direct = np.concatenate([eng.eta(bw.plans[bw.plan_of_profile[p]], P=bw.P_W[p] * 1.7)["eta"]
                             for p in range(9)])
    np.testing.assert_array_equal(third.cpu().numpy(), direct)
    # a single-profile call in between must not break the replay (workspace may move)
    eng.eta(W.uwb(G=8), P=W.uwb().P_W)
    fourth = eng.eta_batched(bw, P2)
    np.testing.assert_array_equal(fourth.cpu().numpy(), direct)


def test_autotuner_picks_a_candidate_and_keeps_results(eng, tmp_path, monkeypatch):
    from paper_2401_18022_gb300 import autotune
    monkeypatch.setenv("ISRS_TILE_CACHE", str(tmp_path / "tiles.json"))
    bw = W.batched(n_prof=6, G=16, n_edges=33, sizes=(60, 31, 12))
    cands = [(1 << 14, 128), (1 << 16, 256), (1 << 18, 256)]
    r = autotune.tune(eng, bw, candidates=cands)
    assert (r["points_per_item"], r["threads"]) in cands and not r["cached"]
    assert (tmp_path / "tiles.json").exists()
    r2 = autotune.tune(eng, bw, candidates=cands)
    assert r2["cached"] and r2["points_per_item"] == r["points_per_item"]
    eta = eng.eta_batched(bw)
    off = 0
    for p in range(6):
        wl = bw.plans[bw.plan_of_profile[p]]
        np.testing.assert_array_equal(eta[off:off + wl.n_ch], eng.eta(wl, P=bw.P_W[p])["eta"])
        off += wl.n_ch
    eng.set_tile(0, 0)
