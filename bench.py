"""Benchmark of the ISRS GN hot path on the 589-channel O-to-U band system.

One step = one full pass of the hot path on the 589 x 96 GBaud, 1260-1675 nm,
80 km workload (G = 256 per piece, 113 z-edges, SCI + XCI cells): ISRS
profile tables, the hyperbolic Riemann sum for every CUT, eta, SNR and
throughput, and the gradient of the throughput with respect to all 589
launch powers (the hand-written adjoint).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "589-ch SNR eval time & grid-pts/s; SNR+gradient time vs plain FP64 at 0.01 dB"
UNIT = "grid-pts/s"
N_SMS = 152


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _workload(G: int, rank: int = 0):
    """The 589-ch system; under torchrun each rank evaluates its own
    independent launch-power profile (weak scaling)."""
    from paper_2401_18022_gb300 import dist as D, workloads as W
    wl = W.uwb(G=G)
    return wl.with_(P_W=D.rank_powers(wl, rank))


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str = None):
        self.device = device
        self.proc = None
        if path is None:
            fd, path = tempfile.mkstemp(prefix=f"isrs_clocks_rank{device}_", suffix=".csv")
            os.close(fd)
        self.path = path

    def start(self):
        try:
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(G: int, budget_core_s: float = 20.0):
    """Time the FP64 oracle as it stands on a bounded sample of the workload:
    every k-th piece of the centre CUT, k chosen for ~budget_core_s of CPU work."""
    import oracle
    wl = _workload(G)
    cut = wl.n_ch // 2
    oracle.build()
    threads = os.cpu_count() or 1
    probe = oracle.time_sample(wl, [cut], 64, threads=threads)
    per_pt_core = probe["seconds"] * threads / max(1, probe["points"])
    n_pieces = probe["pieces_total"]
    want_pts = budget_core_s / max(per_pt_core, 1e-12)
    stride = int(max(1, min(n_pieces, round(n_pieces * G * G / max(want_pts, 1.0)))))
    r = oracle.time_sample(wl, [cut], stride, threads=threads)
    return {"value": r["points"] / r["seconds"], "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 CPU oracle, CUT {cut} of the 589-ch plan, G={G}, every {stride}th of its "
                      f"{n_pieces} pieces ({r['pieces']} pieces, {r['points']} grid points, "
                      f"{r['point_steps']} point-steps) in {r['seconds']:.2f} s on {threads} threads",
            "seconds": r["seconds"], "points": r["points"]}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    wl = _workload(args.G)
    oracle.build()
    threads = os.cpu_count() or 1
    cut = wl.n_ch // 2
    n_pieces = len(oracle.pieces(wl.f_THz, wl.B_THz, cut, wl.cell_set))
    stride = max(1, n_pieces // 24)        # ~24 pieces (~1.6e6 points) per step
    for _ in range(args.warmup):
        oracle.time_sample(wl, [cut], stride * 4, threads=threads)
    secs, pts = 0.0, 0
    for _ in range(args.steps):
        r = oracle.time_sample(wl, [cut], stride, threads=threads)
        secs += r["seconds"]
        pts += r["points"]
    value = pts / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "uwb-589ch-80km-G256-N113-sci_xci (bounded sample per step)",
                       "n_ch": wl.n_ch, "G": wl.G, "n_edges": wl.n_edges, "cells": "sci_xci",
                       "l2": "CPU run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"every {stride}th of the {n_pieces} pieces of CUT {cut} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2401_18022_gb300 import api
    eng = api.Engine(local)
    split = args.split == "cuts" and world > 1
    if args.split == "cuts" and args.mode != "grad":
        raise SystemExit("--split cuts times the gradient (--mode grad)")
    # weak scaling: an independent profile per rank; strong: one system split by CUT shards
    wl = _workload(args.G, 0 if args.split == "cuts" else rank)
    dev = torch.device("cuda", local)
    P = torch.tensor(wl.P_W, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    use_grad = args.mode == "grad"
    from paper_2401_18022_gb300 import dist as D
    weights = None
    if split:
        weights = [4 + 4 * (wl.n_ch - 1)] * wl.n_ch      # SCI+XCI: equal pieces per CUT

    def step():
        if split:
            return D.grad_split(eng, wl, P, rank, world, weights=weights)
        if use_grad:
            return eng.grad(wl, P=P)
        return eng.snr(wl, P=P)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    info = eng.last_launch_info()
    launches_per_step = info["launches"]
    if split:
        # prep + fused forward/adjoint + finish, then SNR from eta + 6 chain kernels
        launches_per_step = 3 + 7
        eng.grad_shard_fwd(wl, D.shard_cuts(wl.n_ch, rank, world, weights), P)
        info = eng.last_launch_info()

    clk = Clocks(local, args.clocks_csv.format(rank=local) if args.clocks_csv else None)
    clk.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    quad_ms = []
    for k in range(args.steps):
        flush.zero_()                                  # L2 flushed between timed iterations
        starts[k].record(stream)
        out = step()
        ends[k].record(stream)
        quad_ms.append(eng.last_kernel_ms(1 if use_grad else 0))   # events around the dominant kernel
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_total = sum(step_ms) / 1e3
    if world > 1:
        from paper_2401_18022_gb300 import dist as D
        t_total = D.max_over_ranks(t_total)

    # grid points of the method's Riemann grid (every piece, as the oracle counts them)
    n_eval = info["points"]
    n_grid = _unfolded_points(wl)
    # weak: every rank evaluates a whole system; strong (split): the ranks share one
    value = (1 if split else world) * n_grid * args.steps / t_total

    quad_ms = float(np.mean(quad_ms))
    paths = eng.last_path_counts()          # z-sum forms of the last timed launch (both kernels count)
    roof = _roofline(eng, wl, paths, n_eval, quad_ms, use_grad, clocks)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "uwb-589ch-80km-G256-N113-sci_xci" + ("+grad" if use_grad else ""),
                       "parallelism": (f"cut shards x{world} (eta all-reduce gather, dT/dP all-reduce)" if split
                                       else f"independent profile per rank x{world}"),
                       "n_ch": wl.n_ch, "G": wl.G, "n_edges": wl.n_edges, "cells": "sci_xci",
                       "profile": "R1 closed-form ISRS, flat 1 dBm/ch",
                       "l2": "flushed (256 MB write) between timed iterations",
                       "grid_points_per_step": n_grid, "evaluated_points_per_step": n_eval,
                       "step": "isrs_gn_grad (SNR + dT/dP)" if use_grad else "isrs_gn_snr (eta, SNR, T)"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks, "roofline": roof, "wall_s": wall}
    if rank == 0 and use_grad:
        line["snr_eval"] = _snr_eval(eng, wl, P, dev, n_grid)
    if rank == 0 and args.extras:
        line["extras"] = _extras(eng, wl, P, dev)
    if rank == 0 and not args.quick:
        line["batched"] = _batched_record(eng, local)
        line["ascent"] = _ascent_record(eng, local)
        line["e2e"] = _e2e(eng, wl, args, world, n_grid)
        line["fp64_path"] = _fp64_path(eng, wl, P, args)
        line["cpu_baseline"] = cpu_baseline(args.G) if world == 1 else None
        line["T_Tbps"] = float(out["T"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _snr_eval(eng, wl, P, dev, n_grid, reps: int = 2):
    """The forward-only 589-ch SNR evaluation (isrs_gn_snr), timed with CUDA
    events on the launching stream."""
    import torch
    st = torch.cuda.current_stream(dev)
    eng.snr(wl, P=P)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        eng.snr(wl, P=P)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    t = float(np.median(ms))
    return {"ms": t, "grid_pts_per_s": n_grid / (t / 1e3), "kernel": "k_quad_f32",
            "kernel_ms": eng.last_kernel_ms(0)}


# Per-launch counters of the dominant kernels from the ncu captures kept in
# profiles/ (the 148-ch G = 256 profiling cases, --profile-case adjoint256 /
# quad256): DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum), executed
# warp instructions (smsp__inst_executed.sum) and FP32-pipe warp instructions
# (FFMA + FADD + FMUL of sass__inst_executed_per_opcode), with the grid points
# that launch evaluated.  The kernels' work per evaluated point is the same at
# full size (same G, same per-piece shape), so each count is scaled to a full
# launch by evaluated points.
ADJ_CAPTURE = {"profile": "k_quad_adj_uwb148_every4th_G256.md", "points": 2880700416,
               "dram_bytes": 4.861e6, "warp_inst": 1.587e11, "fp32_warp_inst": 8.530e10}
FWD_CAPTURE = {"profile": "k_quad_f32_uwb148_every4th_G256.md", "points": 2880700416,
               "dram_bytes": 4.126e6, "warp_inst": 7.114e10, "fp32_warp_inst": 4.469e10}
ISSUE_PER_CLK_PER_SM = 4         # one warp instruction per clock per SM sub-partition


def _roofline(eng, wl, paths, n_eval, kernel_ms, use_grad, clocks):
    """Roofline of the dominant kernel (k_quad_adj for the gradient step,
    k_quad_f32 for the SNR evaluation): plain ALU work, no tensor cores, not
    memory-bound.  Four fractions, each with its own peak:
      * sfu_algorithmic (the headline, `frac`): the work the method states per
        evaluated point-step, 3 SFU operations (sin, cos, exp), over every
        evaluated point and all N_M - 1 steps, against the SFU throughput
        measured by isrs_probe_alu_peaks in this run.  The contracted
        small-phase form (its z-sum from moments, exact to < 2e-8) needs none
        of them, so this fraction can exceed 1: it measures the method's
        rate, not pipe use;
      * sfu_executed: the SFU operations the kernel actually issues (3 per
        step of its direct and telescoped points, from its path counts);
      * issue: executed warp instructions (ncu capture, scaled by evaluated
        points) over 152 SMs x 4 per clock at the SM clock sampled during the
        timed region: the limiter of these kernels;
      * fp32_pipe: FP32 lane operations (FFMA, FADD, FMUL) over the measured
        FFMA throughput."""
    peaks = eng.probe_alu_peaks()
    n_steps = wl.n_edges - 1
    t = kernel_ms / 1e3
    sfu_alg = 3.0 * n_eval * n_steps
    sfu_exec = 3.0 * n_steps * (paths["direct"] + paths["telescoped"])
    cap = ADJ_CAPTURE if use_grad else FWD_CAPTURE
    scale = n_eval / cap["points"]
    warp_inst = cap["warp_inst"] * scale
    fp32_ops = cap["fp32_warp_inst"] * scale * 32
    mhz = clocks.get("sm_mhz") or float(_peaks().get("sm_max_mhz", 2070.0))
    issue_peak = N_SMS * ISSUE_PER_CLK_PER_SM * mhz * 1e6
    sfu_peak = peaks["sfu_ops_per_s"]
    fp32_peak = peaks["fp32_ops_per_s"]
    tot_pts = max(1, sum(paths.values()))
    return {"bound": "alu", "unit": "Tops/s (SFU ops of the method: 3 per evaluated point-step)",
            "achieved": sfu_alg / t / 1e12, "peak": sfu_peak / 1e12, "frac": sfu_alg / t / sfu_peak,
            "traffic": cap["dram_bytes"] * scale,
            "traffic_note": "DRAM bytes per launch from the ncu capture in profiles/%s, scaled by "
                            "evaluated points" % cap["profile"],
            "fractions": {"sfu_algorithmic": sfu_alg / t / sfu_peak, "sfu_executed": sfu_exec / t / sfu_peak,
                          "issue": warp_inst / t / issue_peak, "fp32_pipe": fp32_ops / t / fp32_peak},
            "peaks": {"sfu_ops_per_s": sfu_peak, "fp32_fma_per_s": fp32_peak, "issue_warp_inst_per_s": issue_peak,
                      "source": "SFU and FFMA: isrs_probe_alu_peaks in this run (measured); issue: 152 SMs x 4 "
                                "x %.0f MHz (SM clock sampled during the timed region)" % mhz,
                      "probe_ms": {"sfu": peaks["sfu_probe_ms"], "fp32": peaks["fp32_probe_ms"]}},
            "kernel": "k_quad_adj" if use_grad else "k_quad_f32", "kernel_ms": kernel_ms,
            "sfu_ops_per_launch": {"algorithmic": sfu_alg, "executed": sfu_exec},
            "warp_inst_per_launch": warp_inst,
            "path_fraction": {k: v / tot_pts for k, v in paths.items()}}


def _batched_record(eng, dev_index, reps: int = 1):
    """C4: 512 launch-power profiles over the 589/295/147-channel plans (G = 64)
    in one persistent launch with the autotuned tile, replayed from its
    captured CUDA graph; one direct (capturing) call, then `reps` timed
    replays with CUDA events on the launching stream."""
    import torch
    from paper_2401_18022_gb300 import api, autotune, workloads as W
    beng = api.Engine(dev_index)
    bw = W.batched(n_prof=512, G=64)
    tile = autotune.tune(beng, bw)
    dev = torch.device("cuda", dev_index)
    P = torch.tensor(np.concatenate(bw.P_W), dtype=torch.float64, device=dev)
    beng.eta_batched(bw, P)
    torch.cuda.synchronize(dev)
    st = torch.cuda.current_stream(dev)
    ms, replays = [], []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        beng.eta_batched(bw, P)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
        replays.append(beng.last_graph_replay())
    n_grid = sum(_unfolded_points(bw.plans[k]) for k in bw.plan_of_profile)
    t = float(np.median(ms))
    beng.close()
    return {"workload": "batched-512-profiles-589/295/147ch-G64-N113-sci_xci", "ms": t,
            "grid_pts_per_s": n_grid / (t / 1e3), "grid_points": n_grid, "graph_replayed": all(replays),
            "tile": {k: tile[k] for k in ("points_per_item", "threads")}, "tile_cached": tile.get("cached", False)}


def _ascent_record(eng, dev_index, iters: int = 50, G: int = 64):
    """C5: projected gradient ascent of the throughput over the 589 launch
    powers (dBm in [-5, 5], adjoint gradient every iteration, Armijo
    backtracking with forward calls) at G = 64; the result checked against the
    plain FP64 GPU path on 16 CUTs spread over the band."""
    import torch
    from paper_2401_18022_gb300 import optim, workloads as W
    wl = W.uwb(G=G)
    dev = torch.device("cuda", dev_index)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = optim.ascent(eng, wl, iters=iters)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    P = torch.tensor(res["P_W"], dtype=torch.float64, device=dev)
    r32 = eng.snr(wl, P=P)
    cuts = [int(c) for c in np.linspace(0, wl.n_ch - 1, 16)]
    e64 = eng.eta(wl, P=P, cuts=cuts, precision=1)["eta"].cpu().numpy()
    e32 = r32["eta"].cpu().numpy()[cuts]
    s32 = r32["snr"].cpu().numpy()[cuts]
    Pc = res["P_W"][cuts]
    pase = Pc / s32 - e32 * Pc ** 3
    s64 = Pc / (e64 * Pc ** 3 + pase)
    return {"iters": len(res["history"]), "G": G, "seconds": dt, "iters_per_s": len(res["history"]) / dt,
            "T_start_Tbps": res["history"][0].get("T_before", res["history"][0]["T"]), "T_final_Tbps": r32["T"],
            "x_dbm_minmax": [float(res["x_dbm"].min()), float(res["x_dbm"].max())],
            "fp64_check": {"cuts": cuts, "max_snr_err_dB": float(np.max(np.abs(10 * np.log10(s32 / s64)))),
                           "max_eta_err_dB": float(np.max(np.abs(10 * np.log10(e32 / e64))))}}


def _timed(fn, dev, reps: int = 2):
    """Median of `reps` calls timed with CUDA events on the current stream
    (after one untimed call)."""
    import torch
    st = torch.cuda.current_stream(dev)
    fn()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms))


def _extras(eng, wl, P, dev):
    """Side measurements of the widened rows on the same 589-ch workload:
    the Raman-ODE power profile (SNR and gradient), the MCI cells on their
    own grid (SNR, gradient, and the MCI share of eta per band), and both
    together (SNR and the MCI share with the Raman-ODE profile)."""
    from paper_2401_18022_gb300 import workloads as W
    out = {}
    wr = W.raman(wl)
    out["raman_snr_ms"] = _timed(lambda: eng.snr(wr, P=P), dev)
    out["raman_snr_quad_kernel_ms"] = eng.last_kernel_ms(0)
    out["raman_grad_ms"] = _timed(lambda: eng.grad(wr, P=P), dev)
    out["raman_grad_adjoint_kernel_ms"] = eng.last_kernel_ms(1)
    r2 = eng.snr(wr, P=P)
    out["raman_T_Tbps"] = r2["T"]
    g_mci = 8
    wm = wl.with_(cell_set=W.CELLS_ALL, G_mci=g_mci)
    out["mci_G"] = g_mci
    out["mci_snr_ms"] = _timed(lambda: eng.snr(wm, P=P), dev)
    out["mci_quad_kernels_ms"] = eng.last_kernel_ms(0)
    out["mci_grad_ms"] = _timed(lambda: eng.grad(wm, P=P), dev)
    out["mci_grad_adjoint_kernels_ms"] = eng.last_kernel_ms(1)
    e_all = eng.eta(wm, P=P)["eta"]
    e_sx = eng.eta(wl, P=P)["eta"]
    e_all = e_all.cpu().numpy() if hasattr(e_all, "cpu") else np.asarray(e_all)
    e_sx = e_sx.cpu().numpy() if hasattr(e_sx, "cpu") else np.asarray(e_sx)
    share = 1.0 - e_sx / e_all
    lam = W.nm_from_thz(wl.f_THz)
    band = np.clip(np.searchsorted(W.BAND_EDGES_NM, lam, side="right") - 1, 0, 5)
    out["mci_share_of_eta_by_band"] = {W.BAND_NAMES[b]: [float(share[band == b].min()), float(share[band == b].max())]
                                       for b in range(6)}
    n = wl.n_ch
    out["mci_cells_per_cut"] = (n - 1) * n // 2
    # the Raman-ODE profile with the MCI cells on their own grid (forward)
    wrm = W.raman(wm)
    out["raman_mci_snr_ms"] = _timed(lambda: eng.snr(wrm, P=P), dev)
    out["raman_mci_quad_kernels_ms"] = eng.last_kernel_ms(0)
    e_rm = eng.eta(wrm, P=P)["eta"]
    e_rs = eng.eta(wr, P=P)["eta"]
    e_rm = e_rm.cpu().numpy() if hasattr(e_rm, "cpu") else np.asarray(e_rm)
    e_rs = e_rs.cpu().numpy() if hasattr(e_rs, "cpu") else np.asarray(e_rs)
    share_r = 1.0 - e_rs / e_rm
    out["raman_mci_share_of_eta_by_band"] = {
        W.BAND_NAMES[b]: [float(share_r[band == b].min()), float(share_r[band == b].max())] for b in range(6)}
    out["raman_mci_T_Tbps"] = eng.snr(wrm, P=P)["T"]
    return out


def _unfolded_points(wl):
    """Grid points of the Riemann sum as defined (App. A, Eqs. q1..q4: every
    piece of every CUT, mirror pieces included, as the oracle evaluates them).
    With SCI + XCI cells and disjoint channels a CUT has 4 + 4 (N - 1) pieces:
    the SCI cell's four quadrants, and two pieces (split at f1 = 0 or f2 = 0,
    where the CUT's channel straddles the axis) for each of the cells (i, k)
    and (k, i).  The kernels evaluate the mirror-folded half."""
    n = wl.n_ch
    per_cut = 4 + 4 * (n - 1) if wl.cell_set == 0 else None
    if per_cut is None:
        raise ValueError("bench counts SCI+XCI grids only")
    return n * per_cut * wl.G * wl.G


def _e2e(eng, wl, args, world, n_grid):
    """Same metric through the C ABI with host buffers: H2D of the launch
    powers and D2H of SNR, eta and T inside the timed region."""
    import torch
    P_host = np.ascontiguousarray(wl.P_W)
    k = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        r = eng.grad(wl, P=P_host) if args.mode == "grad" else eng.snr(wl, P=P_host)
    dt = time.perf_counter() - t0
    n_out = 3 if args.mode == "grad" else 2
    return {"value": world * n_grid * k / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * wl.n_ch,
            "d2h_bytes_per_step": 8 * wl.n_ch * n_out + 8, "steps": k, "seconds": dt,
            "T_Tbps": float(r["T"])}


def _fp64_path(eng, wl, P, args):
    """The plain FP64 GPU path on a subset of CUTs (it is ~165x slower on
    GB300's FP64 units): time per CUT extrapolated to 589 CUTs, and the
    FP32-vs-FP64 eta/SNR error on those CUTs."""
    import torch
    cuts = [0, wl.n_ch // 2, wl.n_ch - 1]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r64 = eng.eta(wl, P=P, cuts=cuts, precision=1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    r32 = eng.eta(wl, P=P, cuts=cuts, precision=0)
    e64 = r64["eta"].cpu().numpy()
    e32 = r32["eta"].cpu().numpy()
    err_db = float(np.max(np.abs(10 * np.log10(e32 / e64))))
    per_cut = dt / len(cuts)
    return {"cuts": cuts, "seconds_for_cuts": dt, "extrapolated_589ch_s": per_cut * wl.n_ch,
            "max_eta_err_dB_fp32_vs_fp64": err_db, "note": "extrapolated linearly (equal work per CUT)"}


def run_batched(args) -> int:
    """512 launch-power profiles over the 589/295/147-channel plans (G = 64)
    in one persistent, graph-replayed launch with autotuned tiles."""
    import torch
    from paper_2401_18022_gb300 import api, autotune, workloads as W
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    eng = api.Engine(local)
    bw = W.batched(n_prof=512, G=64)
    tile = autotune.tune(eng, bw)
    dev = torch.device("cuda", local)
    P = torch.tensor(np.concatenate(bw.P_W), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        eng.eta_batched(bw, P)
    torch.cuda.synchronize(dev)
    ms, replays = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        eng.eta_batched(bw, P)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
        replays.append(eng.last_graph_replay())
    n_grid = sum(_unfolded_points(bw.plans[k]) for k in bw.plan_of_profile)
    t = sum(ms) / 1e3
    line = {"metric": METRIC, "value": n_grid * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched-512-profiles-589/295/147ch-G64-N113-sci_xci",
                       "grid_points_per_step": n_grid, "tile": {k: tile[k] for k in ("points_per_item", "threads")},
                       "graph_replayed_steps": int(sum(replays)), "l2": "flushed between timed iterations"},
            "gpu_launches": 3 * args.steps}
    print(json.dumps(line), flush=True)
    return 0


def run_accuracy(args) -> int:
    """The accuracy gate: every CUT of the 589-ch workload (G = 256 unless
    --G; --profile raman for the Raman-ODE profile, --G-mci for the MCI cells
    on their own grid), the FP32 path against the plain FP64 GPU path, as the
    per-CUT error in dB of eta and of SNR (the method's target: 0.01 dB of
    SNR per channel).  The FP64 path runs in chunks of CUTs (~1 min each);
    SNR_64 = P / (eta_64 P^3 + P_ASE) with the ASE of the same plan (no
    transceiver noise in this workload).  Prints one JSON line; with --out,
    writes the per-CUT errors there as JSON."""
    import torch
    from paper_2401_18022_gb300 import api, workloads as W
    torch.cuda.set_device(0)
    eng = api.Engine(0)
    wl = _workload(args.G)
    label = "uwb-589ch-80km-G%d-N113-sci_xci" % wl.G
    if args.G_mci > 0:
        wl = wl.with_(cell_set=W.CELLS_ALL, G_mci=args.G_mci)
        label = "uwb-589ch-80km-G%d-N113-all_cells-Gmci%d" % (wl.G, args.G_mci)
    if args.profile == "raman":
        wl = W.raman(wl)
        label += "-raman_ode"
    P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
    r32 = eng.snr(wl, P=P, precision=0)
    e32, s32 = r32["eta"].cpu().numpy(), r32["snr"].cpu().numpy()
    Ph = wl.P_W
    pase = Ph / s32 - e32 * Ph ** 3
    e64 = np.empty(wl.n_ch)
    t0 = time.perf_counter()
    for chunk in np.array_split(np.arange(wl.n_ch), args.chunks):
        e64[chunk] = eng.eta(wl, P=P, cuts=[int(c) for c in chunk], precision=1)["eta"].cpu().numpy()
    t64 = time.perf_counter() - t0
    s64 = Ph / (e64 * Ph ** 3 + pase)
    de = np.abs(10 * np.log10(e32 / e64))
    ds = np.abs(10 * np.log10(s32 / s64))
    lam = W.nm_from_thz(wl.f_THz)
    band = np.clip(np.searchsorted(W.BAND_EDGES_NM, lam, side="right") - 1, 0, 5)
    line = {"accuracy_gate": label + " FP32 vs plain FP64 GPU, all CUTs",
            "n_cuts": int(wl.n_ch), "fp64_seconds": t64,
            "eta_dB": {"max": float(de.max()), "mean": float(de.mean()), "argmax": int(de.argmax())},
            "snr_dB": {"max": float(ds.max()), "mean": float(ds.mean()), "argmax": int(ds.argmax())},
            "cuts_within_0.01dB_snr": int(np.sum(ds < 0.01)),
            "snr_dB_max_by_band": {W.BAND_NAMES[b]: float(ds[band == b].max()) for b in range(6)},
            "T_fp32_Tbps": float(r32["T"]),
            "T_fp64_Tbps": float(np.sum(2 * wl.B_THz * np.log2(1 + s64)))}
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"eta_dB": de.tolist(), "snr_dB": ds.tolist(), "eta32": e32.tolist(),
                       "eta64": e64.tolist()}, f)
    return 0


def profile_case(kind: str) -> int:
    """One launch for kernel captures: the 589-ch plan at the bench's G = 256
    for 16 CUTs spread over the band (1.2e9 points, ~1.2e3 work tiles, about
    0.1 s), so every SM is busy as in the full run."""
    import torch
    from paper_2401_18022_gb300 import api
    eng = api.Engine(0)
    wl = _workload(256)
    P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
    cuts = [int(c) for c in np.linspace(0, wl.n_ch - 1, 16)]
    if kind == "adjoint":
        eng.grad(wl.with_(G=64), P=P)          # all 589 CUTs at G = 64 (~0.6 s)
    elif kind == "raman256":
        # the same 148-ch subset with the Raman-ODE profile: the gradient (fused
        # tabulated forward + adjoint), then the tabulated forward alone (SNR)
        from paper_2401_18022_gb300 import workloads as W
        sub = W.raman(W.subset_plan(wl, np.arange(0, wl.n_ch, 4), "uwb-148ch-every4th"))
        Ps = torch.tensor(sub.P_W, dtype=torch.float64, device="cuda")
        eng.grad(sub, P=Ps)
        eng.snr(sub, P=Ps)
    elif kind == "mci256":
        # the 148-ch subset with every cell: SCI/XCI at G = 256, the MCI cells on an 8 x 8 grid
        from paper_2401_18022_gb300 import workloads as W
        sub = W.subset_plan(wl, np.arange(0, wl.n_ch, 4), "uwb-148ch-every4th").with_(cell_set=W.CELLS_ALL, G_mci=8)
        eng.grad(sub, P=torch.tensor(sub.P_W, dtype=torch.float64, device="cuda"))
    elif kind == "raman_mci":
        # the Raman-ODE profile with every cell (SCI/XCI at G = 256, MCI on an
        # 8 x 8 grid) on 48 CUTs of the 589-ch plan: 528 MCI work tiles, so the
        # MCI kernel fills every SM as in the full run
        from paper_2401_18022_gb300 import workloads as W
        wr = W.raman(wl.with_(cell_set=W.CELLS_ALL, G_mci=8))
        eng.eta(wr, P=P, cuts=[int(c) for c in np.linspace(0, wl.n_ch - 1, 48)])
    elif kind in ("adjoint256", "quad256"):
        # every 4th slot of the 589-ch grid (148 ch over the whole band) at the
        # bench's G = 256: the production per-piece shape, ~1.4e9 points
        from paper_2401_18022_gb300 import workloads as W
        sub = W.subset_plan(wl, np.arange(0, wl.n_ch, 4), "uwb-148ch-every4th")
        Ps = torch.tensor(sub.P_W, dtype=torch.float64, device="cuda")
        if kind == "adjoint256":
            eng.grad(sub, P=Ps)
        else:
            eng.eta(sub, P=Ps)
    elif kind == "probe":                  # the SFU and FFMA throughput probes alone
        print(json.dumps({"profile_case": kind, **eng.probe_alu_peaks()}))
        return 0
    elif kind == "quad64":                 # FP64 is ~200x slower: 4 CUTs at G = 64
        eng.eta(wl.with_(G=64), P=P, cuts=cuts[::4], precision=1)
    else:
        eng.eta(wl, P=P, cuts=cuts, precision=1 if kind == "quad64" else 0)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": kind, **eng.last_launch_info()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--G", type=int, default=256)
    ap.add_argument("--mode", default="grad", choices=["snr", "grad"],
                    help="grad: SNR + dT/dP (all hot-path steps); snr: forward only")
    ap.add_argument("--quick", action="store_true", help="skip e2e, FP64 and CPU legs")
    ap.add_argument("--clocks-csv", default=None,
                    help="where to keep the nvidia-smi clock samples ({rank} is replaced); default: a temp file")
    ap.add_argument("--extras", action="store_true",
                    help="also time the Raman-ODE profile and the MCI cells on the same workload")
    ap.add_argument("--split", default="profiles", choices=["profiles", "cuts"],
                    help="N > 1: profiles = weak scaling, an independent system per rank; cuts = one "
                         "system's gradient split by CUT shards (strong scaling)")
    ap.add_argument("--workload", default="uwb", choices=["uwb", "batched", "accuracy"],
                    help="uwb: the 589-ch system (default); batched: 512 profiles over 3 plans; "
                         "accuracy: all 589 CUTs FP32 vs the plain FP64 GPU path")
    ap.add_argument("--chunks", type=int, default=16, help="accuracy: FP64 launches over the CUTs")
    ap.add_argument("--out", default=None, help="accuracy: write per-CUT errors (JSON) here")
    ap.add_argument("--profile", default="closed", choices=["closed", "raman"],
                    help="accuracy: closed-form profile or the Raman ODEs")
    ap.add_argument("--G-mci", dest="G_mci", type=int, default=0,
                    help="accuracy: > 0 adds every MCI cell on its own G_mci grid")
    ap.add_argument("--profile-case", default=None,
                    choices=["quad", "quad64", "adjoint", "adjoint256", "quad256", "raman256", "mci256", "raman_mci",
                             "probe"],
                    help="run one small launch of a kernel (for ncu captures) and exit")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "accuracy":
        return run_accuracy(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
