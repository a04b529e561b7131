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
