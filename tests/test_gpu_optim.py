"""torch.autograd wrapper of the adjoint and the gradient-ascent optimiser on the GPU."""
import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    return api.Engine(0)


def test_autograd_function_returns_adjoint(eng):
    import torch
    from paper_2401_18022_gb300 import optim
    wl = W.tiny(G=32, n_edges=57)
    P = torch.tensor(wl.P_W * 1.3, dtype=torch.float64, device="cuda", requires_grad=True)
    T = optim.throughput(P, eng, wl)
    T.backward()
    ref = eng.grad(wl, P=P.detach())
    np.testing.assert_allclose(P.grad.cpu().numpy(), ref["dT_dP"].cpu().numpy(), rtol=0, atol=0)
    assert T.item() == pytest.approx(ref["T"], rel=1e-12)
    with torch.no_grad():
        T2 = optim.throughput(P.detach(), eng, wl)
    assert T2.item() == pytest.approx(ref["T"], rel=1e-7)     # forward vs adjoint small-phase orders


def test_gradient_ascent_on_uwb_raises_throughput(eng):
    from paper_2401_18022_gb300 import optim
    wl = W.uwb(G=8, n_edges=57)
    res = optim.ascent(eng, wl, iters=6)
    Ts = [h["T"] for h in res["history"]]
    assert Ts[-1] > res["history"][0]["T_before"]
    assert all(b >= a - 1e-9 for a, b in zip(Ts, Ts[1:]))
    T64 = eng.snr(wl, P=res["P_W"], precision=1)["T"]       # FP64 path beside it
    assert T64 == pytest.approx(Ts[-1], rel=1e-5)
