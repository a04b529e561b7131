"""The multi-GPU strong-scaling split, run as sequential shards on one GPU.

Every CUT's eta is independent: the CUTs of a system are split into shards
balanced by their piece counts (dist.shard_cuts), each shard is evaluated by
its own call, and the per-CUT results are assembled.  A CUT's work tiles and
their summation order do not depend on which other CUTs a call evaluates, so
the assembled result equals one call over all CUTs bit for bit.
"""
import numpy as np
import pytest

from paper_2401_18022_gb300 import dist as D, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    return api.Engine(0)


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("prec", [0, 1])
def test_sequential_shards_equal_one_call(eng, orc, world, prec):
    wl = W.oband(G=12, n_edges=33)                 # all cells: uneven work per CUT
    weights = [len(orc.pieces(wl.f_THz - wl.f_ref_THz, wl.B_THz, c, wl.cell_set)) for c in range(wl.n_ch)]
    full = eng.eta(wl, precision=prec)
    out = np.full(wl.n_ch, np.nan)
    seen = []
    for r in range(world):
        cuts = D.shard_cuts(wl.n_ch, r, world, weights)
        seen += cuts
        got = eng.eta(wl, cuts=cuts, precision=prec)
        out[cuts] = np.asarray(got["eta"].cpu() if hasattr(got["eta"], "cpu") else got["eta"])[:len(cuts)]
    assert sorted(seen) == list(range(wl.n_ch))
    ref = np.asarray(full["eta"].cpu() if hasattr(full["eta"], "cpu") else full["eta"])
    np.testing.assert_array_equal(out, ref)


def _np(x):
    return np.asarray(x.cpu() if hasattr(x, "cpu") else x)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", ["tiny", "oband", "uwb", "raman_tiny", "raman_uwb"])
def test_split_gradient_shards_sum_to_one_gradient(eng, orc, world, case):
    """The gradient split by CUT shards (isrs_gn_grad_shard_fwd/_bwd), run as
    sequential ranks on one GPU with one handle each: eta gathered from the
    shards, each shard's part of dT/dP from the gathered eta, rank 0 adding
    the terms outside eta.  The parts sum to one isrs_gn_grad call; only the
    order of the FP64 sums over tiles differs.  With the Raman-ODE profile
    each shard runs the discrete adjoint of the RK4 steps on its own bucket
    terms (the adjoint is linear in them)."""
    from paper_2401_18022_gb300 import api
    wl = {"tiny": lambda: W.tiny(G=16, n_edges=33),
          "oband": lambda: W.oband(G=12, n_edges=33),
          "uwb": lambda: W.uwb(G=8, n_edges=33),
          "raman_tiny": lambda: W.raman(W.tiny(G=16, n_edges=33).with_(Cr=0.4), raman_max_THz=0.25),
          "raman_uwb": lambda: W.raman(W.uwb(G=8, n_edges=33), ode_h_km=0.5)}[case]()
    weights = [len(orc.pieces(wl.f_THz - wl.f_ref_THz, wl.B_THz, c, wl.cell_set)) for c in range(wl.n_ch)]
    full = eng.grad(wl)
    ranks = [api.Engine(0) for _ in range(world)]
    cuts = [D.shard_cuts(wl.n_ch, r, world, weights) for r in range(world)]
    eta_all = np.full(wl.n_ch, np.nan)
    for r in range(world):
        eta_all[cuts[r]] = _np(ranks[r].grad_shard_fwd(wl, cuts[r]))
    np.testing.assert_allclose(eta_all, _np(full["eta"]), rtol=1e-12)
    parts = [ranks[r].grad_shard_bwd(eta_all, with_direct=(r == 0)) for r in range(world)]
    g = np.sum([_np(p["dT_dP"]) for p in parts], axis=0)
    ref = _np(full["dT_dP"])
    np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))
    for p in parts:
        assert p["T"] == pytest.approx(full["T"], rel=1e-13)
        np.testing.assert_allclose(_np(p["snr"]), _np(full["snr"]), rtol=1e-12)


def test_split_gradient_one_rank_and_misuse(eng):
    """grad_split with one rank is one shard holding every CUT; the second
    phase without a first, or after another call on the handle, is refused."""
    from paper_2401_18022_gb300 import api
    from paper_2401_18022_gb300._capi import IsrsError
    wl = W.tiny(G=16, n_edges=33)
    full = eng.grad(wl)
    out = D.grad_split(eng, wl, wl.P_W, 0, 1)
    np.testing.assert_allclose(_np(out["dT_dP"]), _np(full["dT_dP"]), rtol=1e-12,
                               atol=1e-14 * np.max(np.abs(_np(full["dT_dP"]))))
    fresh = api.Engine(0)
    with pytest.raises(IsrsError) as ei:
        fresh.grad_shard_bwd(_np(full["eta"]), True)
    assert ei.value.status == 1
    fresh.grad_shard_fwd(wl, [0, 1])
    fresh.eta(wl)                                   # overwrites the shard's workspace
    with pytest.raises(IsrsError) as ei:
        fresh.grad_shard_bwd(_np(full["eta"]), True)
    assert ei.value.status == 1
