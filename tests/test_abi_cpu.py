"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function declared in include/isrs_gn.h; host helpers agree
with the paper's Sec. II formulas through an independent route."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:isrs_status|double|int|const char \*)\s*\*?\s*(isrs_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_18022_gb300 import _capi
    return _capi.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for s in range(8):
        assert lib.isrs_status_string(s)
    assert lib.isrs_status_string(7) == b"debug bounds check failed"


def test_debug_build_is_separate_and_reports_itself(lib):
    """The bounds-checked variant (ISRS_DEBUG) builds from the same sources
    into its own library; each library reports which one it is."""
    from paper_2401_18022_gb300 import build as B
    assert lib.isrs_debug_build() == 0
    path = B.build(debug=True)
    assert path == B.LIB_DEBUG and path != B.LIB
    dbg = ctypes.CDLL(path)
    dbg.isrs_debug_build.restype = ctypes.c_int
    assert dbg.isrs_debug_build() == 1
    for n in _declared():
        assert hasattr(dbg, n), n


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    st = lib.isrs_create(ctypes.byref(h), 0)
    assert st in (1, 2) and not h.value


def test_host_beta_helper_matches_oracle(lib, orc):
    """Both implement Eqs. d..d_curve independently; they must agree."""
    from paper_2401_18022_gb300 import _capi
    for lam, D, S, Sd in [(1550.1, 17.0, 0.057, 0.0), (1310.0, 0.0, 0.09, -2.06e-4)]:
        out = np.zeros(3)
        assert lib.isrs_beta_from_dispersion(lam, D, S, Sd, out.ctypes.data_as(_capi.c_double_p)) == 0
        assert np.allclose(out, orc.beta_from_dispersion(lam, D, S, Sd), rtol=1e-14, atol=0)
    assert lib.isrs_beta_from_dispersion(-1.0, 1, 1, 1, out.ctypes.data_as(_capi.c_double_p)) == 1
    g = lib.isrs_gamma_from_aeff(1550.0, 2.6e-20, 80.0)
    assert g == pytest.approx(orc.gamma(1550.0, 2.6e-20, 80.0), rel=1e-14)
    assert np.isnan(lib.isrs_gamma_from_aeff(0.0, 2.6e-20, 80.0))


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of isrs_fibre / isrs_channels / isrs_quad have the
    C header's field offsets and sizes (compiled with the host C compiler)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2401_18022_gb300 import _capi
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    structs = {"isrs_fibre": _capi.Fibre, "isrs_channels": _capi.Channels, "isrs_quad": _capi.Quad}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "isrs_gn.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_pointer_classification_rejects_other_devices(tmp_path):
    """The rule the entry points apply to every caller pointer (csrc/ptr_class.h):
    device memory of the current device and managed memory are used in place,
    host memory is copied through, device memory of another GPU is rejected
    (a kernel on this device would otherwise write into that GPU's memory)."""
    import subprocess
    src = tmp_path / "t.cpp"
    src.write_text('#include "ptr_class.h"\n#include <cstdio>\nint main(){\n'
                   'for (int t = 0; t < 4; ++t) for (int d = 0; d < 3; ++d)\n'
                   '  std::printf("%d %d %d\\n", t, d, isrs::ptr_class(t, d, 1));\n}\n')
    exe = tmp_path / "t"
    subprocess.check_call(["g++", "-std=c++17", "-I", os.path.join(ROOT, "paper_2401_18022_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).split("\n"):
        if line:
            t, d, c = map(int, line.split())
            got[(t, d)] = c
    HOST, DEV, OTHER = 0, 1, 2
    for d in range(3):
        assert got[(0, d)] == HOST and got[(1, d)] == HOST      # unregistered / pinned host
        assert got[(3, d)] == DEV                               # managed
        assert got[(2, d)] == (DEV if d == 1 else OTHER)        # device memory: only the current GPU
