"""The benchmark's output contract, on the CPU: `bench.py --impl reference`
(the FP64 oracle on a bounded sample of the 589-ch workload) prints one JSON
line with the keys and types the driver reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                     ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                     ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict),
                     ("impl", str)):
        assert isinstance(d[key], typ), (key, d.get(key))
    assert d["impl"] == "reference" and d["value"] > 0 and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("uwb-589ch")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_bench_grid_point_count_matches_the_oracles_pieces(orc):
    """The benchmark's grid-point count is the oracle's: G^2 times the pieces
    the oracle evaluates for every CUT (the 589-ch plan and the uneven
    295/147-ch plans of the batched workload)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2401_18022_gb300 import workloads as W
    plans = [W.uwb(G=4)] + list(W.batched(n_prof=3, G=4).plans)
    for wl in plans:
        f = wl.f_THz - wl.f_ref_THz
        n_pieces = sum(len(orc.pieces(f, wl.B_THz, i, wl.cell_set)) for i in range(wl.n_ch))
        assert bench._unfolded_points(wl) == n_pieces * wl.G * wl.G, wl.name


def test_roofline_record_with_a_stand_in_engine():
    """The GPU line's roofline object, built from a stand-in for the engine's
    measured peaks: keys, the four fractions and their defining formulas."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2401_18022_gb300 import workloads as W

    class FakeEng:
        def probe_alu_peaks(self):
            return {"sfu_ops_per_s": 1.0e13, "sfu_probe_ms": 8.0, "fp32_ops_per_s": 4.0e13, "fp32_probe_ms": 16.0}

    wl = W.uwb(G=4)
    paths = {"small": 600, "direct": 100, "telescoped": 300}
    r = bench._roofline(FakeEng(), wl, paths, 1000, 2.0, True, {"sm_mhz": 2000.0})
    f = r["fractions"]
    assert set(f) == {"sfu_algorithmic", "sfu_executed", "issue", "fp32_pipe"}
    steps = wl.n_edges - 1
    assert r["frac"] == f["sfu_algorithmic"] == 3 * 1000 * steps / 2e-3 / 1e13
    assert f["sfu_executed"] == 3 * steps * 400 / 2e-3 / 1e13
    cap = bench.ADJ_CAPTURE
    assert abs(f["issue"] / (cap["warp_inst"] * 1000 / cap["points"] / 2e-3 / (152 * 4 * 2e9)) - 1) < 1e-12
    assert r["bound"] == "alu" and r["peak"] == 10.0 and r["kernel"] == "k_quad_adj"
    json.dumps(r)
