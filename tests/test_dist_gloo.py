"""Multi-process (gloo, world size 2, CPU) checks of the sharding host logic:
a system's CUTs split across ranks and gathered equal the single-process
result; per-rank weak-scaling profiles are independent; the timing reduction
takes the max over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_2401_18022_gb300 import dist as D, workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = W.tiny(G=12, n_edges=17)
    cuts = D.shard_cuts(wl.n_ch, rank, world)
    sig = oracle.sigma(wl, cuts=cuts, threads=1)
    full = D.gather_by_cut(sig, cuts, wl.n_ch)
    P = D.rank_powers(wl, rank)
    t = D.max_over_ranks(1.0 + rank)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([full, P, [t]]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_gather_and_reductions_world2(tmp_path, orc):
    import torch.multiprocessing as mp
    from paper_2401_18022_gb300 import workloads as W
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    wl = W.tiny(G=12, n_edges=17)
    ref = orc.sigma(wl, threads=1)
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    n = wl.n_ch
    np.testing.assert_array_equal(r0[:n], r1[:n])
    np.testing.assert_allclose(r0[:n], ref, rtol=1e-13)
    assert not np.allclose(r0[n:2 * n], r1[n:2 * n])          # independent profiles
    np.testing.assert_array_equal(r0[n:2 * n], wl.P_W)
    assert r0[-1] == r1[-1] == 2.0


def test_shard_cuts_partitions_and_balances():
    from paper_2401_18022_gb300 import dist as D
    for n, world in [(589, 8), (5, 2), (41, 3), (3, 4)]:
        parts = [D.shard_cuts(n, r, world) for r in range(world)]
        assert sorted(sum(parts, [])) == list(range(n))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    w = np.r_[np.full(10, 5.0), np.ones(40)]
    parts = [D.shard_cuts(50, r, 2, w) for r in range(2)]
    assert abs(sum(w[parts[0]]) - sum(w[parts[1]])) <= 5.0
    with pytest.raises(ValueError):
        D.shard_cuts(5, 2, 2)
