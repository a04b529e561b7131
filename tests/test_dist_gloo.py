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


class _OracleShards:
    """Stand-in for the engine's two split-gradient phases, computed by the FP64
    oracle with central differences in dB-power (CPU): phase 1 gives eta of the
    shard's CUTs; phase 2 gives sum over the shard's CUTs of dT/deta_i
    deta_i/dP_j, plus, with with_direct, dT/dP_j at fixed eta."""

    H_DB = 1e-3

    def __init__(self):
        import oracle
        self.orc = oracle

    def _eta(self, P):
        s = self.orc.sigma(self.wl, P=P, cuts=self.cuts, threads=1)
        return self.orc.eta(self.wl, s, cuts=self.cuts, P=P)[0]

    def _T(self, eta_all, P):
        return self.orc.snr_throughput(self.wl, eta_all, P=P)[2]

    def grad_shard_fwd(self, wl, cuts, P):
        self.wl, self.cuts, self.P = wl, list(cuts), np.asarray(P, dtype=np.float64)
        return self._eta(self.P)

    def grad_shard_bwd(self, eta_all, with_direct):
        eta_all, P = np.asarray(eta_all, dtype=np.float64), self.P
        n = len(P)
        ybar = np.zeros(n)
        for i in self.cuts:
            d = 1e-4 * eta_all[i]
            ep, em = eta_all.copy(), eta_all.copy()
            ep[i] += d
            em[i] -= d
            ybar[i] = (self._T(ep, P) - self._T(em, P)) / (2 * d)
        g = np.zeros(n)
        f = 10 ** (self.H_DB / 10)
        for j in range(n):
            Pp, Pm = P.copy(), P.copy()
            Pp[j] *= f
            Pm[j] /= f
            dP = Pp[j] - Pm[j]
            g[j] = ybar[self.cuts] @ ((self._eta(Pp) - self._eta(Pm)) / dP)
            if with_direct:
                g[j] += (self._T(eta_all, Pp) - self._T(eta_all, Pm)) / dP
        snr, _, T = self.orc.snr_throughput(self.wl, eta_all, P=P)
        return {"dT_dP": g, "snr": snr, "T": T}


def _split_wl(profile):
    from paper_2401_18022_gb300 import workloads as W
    wl = W.tiny(G=8, n_edges=9)
    if profile == "raman":
        # the Raman-ODE profile: the ASE gain of every channel depends on
        # every launch power through the ODE, one of the terms outside eta
        wl = W.raman(wl.with_(Cr=0.4), raman_max_THz=0.25, ode_h_km=2.0)
    return wl


def _split_worker(rank, world, port, out_dir, profile):
    import torch.distributed as dist
    from paper_2401_18022_gb300 import dist as D
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = _split_wl(profile)
    out = D.grad_split(_OracleShards(), wl, wl.P_W, rank, world)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), np.concatenate([out["dT_dP"], out["eta"], [out["T"]]]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("profile", ["closed", "raman"])
def test_split_gradient_world2_equals_full_gradient(tmp_path, orc, profile):
    """The split gradient's host logic (shards, eta gathered by an all-reduce,
    exactly one rank adding the terms outside eta, all-reduce of the parts),
    with the oracle standing in for each rank's GPU phases, equals the central
    difference of the single-process oracle throughput, for both profiles."""
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_split_worker, args=(2, port, str(tmp_path), profile), nprocs=2, start_method="spawn")
    wl = _split_wl(profile)
    n = wl.n_ch
    r0, r1 = np.load(tmp_path / "g0.npy"), np.load(tmp_path / "g1.npy")
    np.testing.assert_array_equal(r0, r1)                     # every rank holds the full result
    ref_eta = orc.evaluate(wl, threads=1)["eta"]
    np.testing.assert_allclose(r0[n:2 * n], ref_eta, rtol=1e-13)
    f = 10 ** (_OracleShards.H_DB / 10)
    ref = np.zeros(n)
    for j in range(n):
        Pp, Pm = wl.P_W.copy(), wl.P_W.copy()
        Pp[j] *= f
        Pm[j] /= f
        ref[j] = (orc.evaluate(wl, P=Pp, threads=1)["T"] - orc.evaluate(wl, P=Pm, threads=1)["T"]) / (Pp[j] - Pm[j])
    np.testing.assert_allclose(r0[:n], ref, rtol=1e-5)
    assert r0[-1] == pytest.approx(orc.evaluate(wl, threads=1)["T"], rel=1e-13)

