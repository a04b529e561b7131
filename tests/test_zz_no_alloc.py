"""The allocation-free entry point isrs_gn_eta_noalloc, through the C ABI.

It serves callers that cannot allocate device memory (a host framework that
owns the allocator, a memory-budgeted real-time loop); all its scratch sits in
a fixed 4 MiB device array inside the library.  This file is collected last
so that a run stopping at the first failure has run every other test first;
it passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL_F32 = 2e-4     # tolerance of the FP32 parity tests
RTOL_F64 = 1e-9


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import _capi, api
    eng = api.Engine(0)
    lib = _capi.load()
    lib.isrs_gn_eta_noalloc.argtypes = [ctypes.POINTER(_capi.Fibre), ctypes.POINTER(_capi.Channels),
                                        ctypes.c_void_p, ctypes.POINTER(_capi.Quad), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    lib.isrs_gn_eta_noalloc.restype = ctypes.c_int
    return eng, lib


def _noalloc(eng, lib, wl, P, precision):
    import torch
    fb, (ch, keep), q = eng.fibre(wl), eng.channels(wl), eng.quad(wl, precision)
    eta = torch.full((wl.n_ch,), float("nan"), dtype=torch.float64, device="cuda")
    pnli = torch.full((wl.n_ch,), float("nan"), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.isrs_gn_eta_noalloc(ctypes.byref(fb), ctypes.byref(ch), ctypes.c_void_p(P.data_ptr()),
                                 ctypes.byref(q), ctypes.c_void_p(eta.data_ptr()),
                                 ctypes.c_void_p(pnli.data_ptr()), st)
    torch.cuda.synchronize()
    return rc, eta.cpu().numpy(), pnli.cpu().numpy()


@pytest.mark.parametrize("precision,rtol", [(0, RTOL_F32), (1, RTOL_F64)])
def test_noalloc_matches_eta_on_two_calls_in_a_row(setup, precision, rtol):
    import torch
    eng, lib = setup
    cases = [W.tiny(G=40, n_edges=57),
             W.oband(G=10, n_edges=33, cell_set=W.CELLS_SCI_XCI)]
    for wl in cases:                               # two different calls back to back
        P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
        ref = eng.eta(wl, P=P, precision=precision)
        rc, eta, pnli = _noalloc(eng, lib, wl, P, precision)
        assert rc == 0
        np.testing.assert_allclose(eta, ref["eta"].cpu().numpy(), rtol=rtol)
        np.testing.assert_allclose(pnli, ref["pnli"].cpu().numpy(), rtol=rtol)


def test_noalloc_rejects_what_does_not_fit_or_host_pointers(setup):
    import torch
    eng, lib = setup
    big = W.uwb(G=16)                               # ~7e5 pieces: far beyond the scratch
    P = torch.tensor(big.P_W, dtype=torch.float64, device="cuda")
    rc, eta, _ = _noalloc(eng, lib, big, P, 0)
    assert rc == 6 and np.all(np.isnan(eta))
    wl = W.tiny(G=8)
    fb, (ch, keep), q = eng.fibre(wl), eng.channels(wl), eng.quad(wl, 0)
    Ph = np.ascontiguousarray(wl.P_W)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    rc = lib.isrs_gn_eta_noalloc(ctypes.byref(fb), ctypes.byref(ch), ctypes.c_void_p(Ph.ctypes.data),
                                 ctypes.byref(q), ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == 1


def test_noalloc_on_a_capturing_stream_returns_unsupported(setup):
    """The call reads the powers back and synchronises its stream, which a
    stream capture forbids: on a capturing stream it must return UNSUPPORTED
    before issuing any work, and the caller's capture must stay usable."""
    import torch
    eng, lib = setup
    wl = W.tiny(G=8, n_edges=17)
    P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
    fb, (ch, keep), q = eng.fibre(wl), eng.channels(wl), eng.quad(wl, 0)
    eta = torch.full((wl.n_ch,), float("nan"), dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        x.add_(1.0)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.isrs_gn_eta_noalloc(ctypes.byref(fb), ctypes.byref(ch), ctypes.c_void_p(P.data_ptr()),
                                     ctypes.byref(q), ctypes.c_void_p(eta.data_ptr()), None, st)
        x.add_(1.0)
    assert rc == 6
    graph.replay()
    torch.cuda.synchronize()
    assert torch.all(x == 2.0)
    assert torch.all(torch.isnan(eta))
    # the entry point still works afterwards
    rc2, e2, _ = _noalloc(eng, lib, wl, P, 0)
    assert rc2 == 0 and np.all(np.isfinite(e2))
