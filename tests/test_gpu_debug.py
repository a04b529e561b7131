"""The bounds-checked debug build (ISRS_DEBUG) on the GPU: every check passes
on the method's workloads, and its results equal the release build's.

The debug library is loaded in a child process (ISRS_GN_DEBUG=1), since one
process loads one build.  The child evaluates SNR and the gradient on the
tiny plan (all cells, MCI on its own grid), the Raman-ODE profile (also with
the MCI grid, SNR only, FP32 and FP64), and the 589-channel plan at G = 160;
a failed device check would surface as
ISRS_ERR_CHECK from the call.  The parent evaluates the same with the
release library and compares."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {root!r} + "/tests")
from paper_2401_18022_gb300 import api, workloads as W
from _debug_cases import cases
eng = api.Engine(0)
out = {{"debug_build": eng.debug_build}}
for name, wl, grad in cases(W):
    g = np.asarray(eng.grad(wl)["dT_dP"]).tolist() if grad else []
    s = eng.snr(wl)
    e32 = np.asarray(s["eta"]).tolist()
    e64 = np.asarray(eng.snr(wl, precision=1)["eta"]).tolist() if not grad else []
    out[name] = {{"dT_dP": g, "eta": e32, "eta64": e64, "T": s["T"]}}
json.dump(out, open(sys.argv[1], "w"))
"""


def test_debug_build_passes_every_check_and_matches_release(tmp_path):
    import torch
    from paper_2401_18022_gb300 import api, build as B, workloads as W
    from _debug_cases import cases

    assert torch.cuda.is_available()
    B.build(debug=True)
    script = tmp_path / "child.py"
    script.write_text(_CHILD.format(root=ROOT))
    res = tmp_path / "debug.json"
    env = dict(os.environ, ISRS_GN_DEBUG="1")
    p = subprocess.run([sys.executable, str(script), str(res)], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-3000:]
    dbg = json.load(open(res))
    assert dbg["debug_build"] is True

    eng = api.Engine(0)
    assert not eng.debug_build
    for name, wl, grad in cases(W):
        s = eng.snr(wl)
        e_rel, e_dbg = np.asarray(s["eta"]), np.array(dbg[name]["eta"])
        fin = np.isfinite(e_rel)
        assert np.array_equal(fin, np.isfinite(e_dbg)), name
        np.testing.assert_allclose(e_dbg[fin], e_rel[fin], rtol=1e-12, err_msg=name)
        assert abs(dbg[name]["T"] / s["T"] - 1) < 1e-13, name
        if grad:
            g_rel, g_dbg = np.asarray(eng.grad(wl)["dT_dP"]), np.array(dbg[name]["dT_dP"])
            np.testing.assert_allclose(g_dbg, g_rel, rtol=1e-10, atol=1e-12 * np.max(np.abs(g_rel)), err_msg=name)
        else:
            e64 = np.asarray(eng.snr(wl, precision=1)["eta"])
            np.testing.assert_allclose(np.array(dbg[name]["eta64"])[fin], e64[fin], rtol=1e-12, err_msg=name)
