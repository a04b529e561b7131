"""Failure paths of the handle API, with the failure made on the host.

isrs_debug_inject_fault arms one simulated failure: a device allocation that
fails as if cudaMalloc had run out of memory, or a CUDA runtime call that
fails as if the runtime had returned an error.  Nothing faults on the GPU;
the simulated call is simply not executed.  Each test checks that the call
returns the documented status, writes nothing to its outputs, and that the
same handle then computes the same results as a clean one.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ALLOC, CUDA = 3, 2


@pytest.fixture(scope="module")
def ref():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    wl = W.tiny(G=12, n_edges=17)
    clean = api.Engine(0)
    return wl, clean.eta(wl)["eta"], clean.grad(wl)["dT_dP"]


def _eta_into(eng, wl, eta_out, pnli_out):
    """isrs_gn_eta through the C ABI into caller-owned device outputs."""
    import torch
    fb, (ch, keep), q = eng.fibre(wl), eng.channels(wl), eng.quad(wl, 0)
    P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = eng.lib.isrs_gn_eta(eng.h, ctypes.byref(fb), ctypes.byref(ch), ctypes.c_void_p(P.data_ptr()),
                             ctypes.byref(q), None, 0, ctypes.c_void_p(eta_out.data_ptr()),
                             ctypes.c_void_p(pnli_out.data_ptr()), None, st)
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("kind,after,status", [(1, 1, ALLOC), (1, 4, ALLOC), (1, 12, ALLOC),
                                               (2, 1, CUDA), (2, 3, CUDA), (2, 9, CUDA)])
def test_injected_failure_fresh_handle(ref, kind, after, status):
    """On a fresh handle (every workspace buffer and plan table still to be
    allocated): the call fails with the injected status, the outputs keep
    their NaN fill, and the next call on the same handle is correct."""
    import torch
    from paper_2401_18022_gb300 import api
    wl, eta_ref, _ = ref
    eng = api.Engine(0)
    eng.inject_fault(kind, after)
    eta = torch.full((wl.n_ch,), float("nan"), dtype=torch.float64, device="cuda")
    pnli = torch.full((wl.n_ch,), float("nan"), dtype=torch.float64, device="cuda")
    assert _eta_into(eng, wl, eta, pnli) == status
    assert eng.lib.isrs_last_error(eng.h)
    assert torch.all(torch.isnan(eta)) and torch.all(torch.isnan(pnli))
    eng.inject_fault(0)
    np.testing.assert_array_equal(eng.eta(wl)["eta"], eta_ref)


@pytest.mark.parametrize("after", [1, 2, 6])
def test_injected_cuda_failure_warm_handle_gradient(ref, after):
    """A handle whose tables are cached: a CUDA failure inside the gradient
    call returns ISRS_ERR_CUDA, leaves dT/dP unwritten, and the next gradient
    equals a clean handle's (to FP64 rounding: its PSD buckets are summed with
    atomics)."""
    import torch
    from paper_2401_18022_gb300 import api
    from paper_2401_18022_gb300._capi import IsrsError
    wl, _, g_ref = ref
    eng = api.Engine(0)
    eng.grad(wl)
    eng.inject_fault(2, after)
    P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
    g = torch.full((wl.n_ch,), float("nan"), dtype=torch.float64, device="cuda")
    fb, (ch, keep), q = eng.fibre(wl), eng.channels(wl), eng.quad(wl, 0)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = eng.lib.isrs_gn_grad(eng.h, ctypes.byref(fb), ctypes.byref(ch), ctypes.c_void_p(P.data_ptr()),
                              ctypes.byref(q), ctypes.c_void_p(g.data_ptr()), None, None, None, st)
    torch.cuda.synchronize()
    assert rc == CUDA
    assert torch.all(torch.isnan(g))
    eng.inject_fault(0)
    np.testing.assert_allclose(eng.grad(wl)["dT_dP"], g_ref, rtol=1e-12)
    with pytest.raises(IsrsError):
        eng.inject_fault(3, 1)
