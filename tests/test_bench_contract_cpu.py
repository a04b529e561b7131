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
