"""Parity at the full sizes the benchmark times, on sampled outputs.

* 589 channels, G = 256, 113 edges, SCI + XCI (the bench launch): all 589 CUTs
  in one FP32 launch; CUTs 0, 294 and 588 (both band edges and the centre)
  checked against the FP64 oracle, 8 CUTs against the plain FP64 GPU path;
  at G = 16 all 589 CUTs against the FP64 GPU path (per-CUT dB error of eta
  and SNR).
* The gradient call at that size returns the same SNR, eta and T as the
  forward call, and its directional derivatives along seeded directions
  agree with central differences of the FP32 forward throughput.
* Batched: 512 profiles over the 589/295/147-channel plans at G = 64 in one
  persistent launch; sampled profiles equal single-profile launches bit for
  bit and one (profile, CUT) pair matches the oracle.

Tolerances as in test_gpu_forward.py (FP32 2e-4 relative on eta).
"""
import os

import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL_F32 = 2e-4


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_18022_gb300 import api
    return api.Engine(0)


@pytest.fixture(scope="module")
def uwb_full(eng):
    import torch
    wl = W.uwb(G=256)
    P = torch.tensor(wl.P_W, dtype=torch.float64, device="cuda")
    r = eng.eta(wl, P=P)
    return wl, P, {k: v.cpu().numpy() for k, v in r.items()}


@pytest.mark.parametrize("cut", [0, 294, 588])
def test_uwb_full_cuts_vs_oracle(uwb_full, orc, cut):
    """Both band edges (CUT 0: strongest ISRS gain; CUT 588: strongest loss and
    the largest |beta| terms) and the centre, at the benchmark's G = 256,
    against the FP64 oracle (~20 s of host cores per CUT)."""
    wl, _, r = uwb_full
    ref = orc.sigma(wl, cuts=[cut], threads=os.cpu_count())
    np.testing.assert_allclose(r["sigma"][cut], ref[0], rtol=RTOL_F32)


def test_uwb_full_fp64_gpu_vs_oracle(eng, orc):
    """The plain FP64 GPU path against the FP64 oracle at the benchmark's
    G = 256, on the centre CUT of the 589-ch plan: same algorithm and
    precision, so they agree to summation order (1e-9)."""
    wl = W.uwb(G=256)
    got = eng.eta(wl, cuts=[294], precision=1)["sigma"]
    ref = orc.sigma(wl, cuts=[294], threads=os.cpu_count())
    np.testing.assert_allclose(got, ref, rtol=1e-9)


def test_uwb_full_vs_fp64_gpu_sampled(eng, uwb_full):
    wl, P, r = uwb_full
    cuts = [0, 1, 97, 200, 294, 401, 587, 588]
    r64 = eng.eta(wl, P=P, cuts=cuts, precision=1)
    e64 = r64["eta"].cpu().numpy()
    np.testing.assert_allclose(r["eta"][cuts], e64, rtol=RTOL_F32)
    assert np.max(np.abs(10 * np.log10(r["eta"][cuts] / e64))) < 1e-3


def test_uwb_full_grad_forward_consistent(eng, uwb_full):
    wl, P, r = uwb_full
    g = eng.grad(wl, P=P)
    s = eng.snr(wl, P=P)
    np.testing.assert_allclose(g["eta"].cpu().numpy(), r["eta"], rtol=1e-6)
    np.testing.assert_allclose(g["snr"].cpu().numpy(), s["snr"].cpu().numpy(), rtol=1e-6)
    # the forward kernel sums small phases with the 19-moment series up to
    # |phi| L = 6, the adjoint with 11 moments up to |phi| L = 2 and per step
    # beyond: each form is within 5e-8 of the exact z-sum, so T agrees to ~1e-8
    assert g["T"] == pytest.approx(s["T"], rel=1e-7)
    d = g["dT_dP"].cpu().numpy()
    assert np.all(np.isfinite(d))


def test_uwb_full_grad_directional_derivatives(eng, uwb_full):
    """The adjoint at the benchmark's configuration (589 ch, G = 256, Eq. loss):
    along three seeded directions delta (per-channel dB, N(0, 1)), g . dP/dt
    against the central difference of the FP32 forward T(P 10^{t delta/10}) at
    t = +-0.02 dB.  The FP32 forward is a smooth function of P here (the z-sum
    form of a point depends on phi only, and the contraction's eligibility
    kappa(L) B/2 <= 0.05 holds with margin), and its rounding (~1e-8 of T) is
    far below the ~1e-4 change of T, so the difference is accurate to its
    O(t^2) truncation (~4e-6).  Tolerance: 1e-3 relative, the method's target
    for the gradient."""
    wl, P, _ = uwb_full
    import torch
    g = eng.grad(wl, P=P)["dT_dP"].cpu().numpy()
    rng = np.random.default_rng(3)
    h = 0.02
    for _ in range(3):
        d = rng.standard_normal(wl.n_ch)
        Pp = torch.tensor(wl.P_W * 10 ** (h * d / 10), dtype=torch.float64, device="cuda")
        Pm = torch.tensor(wl.P_W * 10 ** (-h * d / 10), dtype=torch.float64, device="cuda")
        fd = (eng.snr(wl, P=Pp)["T"] - eng.snr(wl, P=Pm)["T"]) / (2 * h)
        ad = float(np.sum(g * wl.P_W * np.log(10) / 10 * d))
        assert ad == pytest.approx(fd, rel=1e-3), (ad, fd)


def test_batched_full_512_profiles(eng, orc):
    bw = W.batched(n_prof=512, G=64)
    eta = eng.eta_batched(bw)
    offs = np.concatenate([[0], np.cumsum([bw.plans[k].n_ch for k in bw.plan_of_profile])])
    for p in (0, 1, 2, 257, 511):
        wl = bw.plans[bw.plan_of_profile[p]]
        single = eng.eta(wl, P=bw.P_W[p])["eta"]
        np.testing.assert_array_equal(eta[offs[p]:offs[p + 1]], single)
    p, cut = 2, 73                                    # the 147-channel plan
    wl = bw.plans[bw.plan_of_profile[p]]
    ref, _ = orc.eta(wl, orc.sigma(wl, P=bw.P_W[p], cuts=[cut]), cuts=[cut], P=bw.P_W[p])
    np.testing.assert_allclose(eta[offs[p] + cut], ref[0], rtol=RTOL_F32)


def test_uwb_all_cuts_fp32_vs_fp64_gpu(eng):
    """Every one of the 589 CUTs, FP32 against the plain FP64 GPU path, at
    G = 16 (the FP64 path is ~600x slower): per-CUT error in dB of eta and
    of SNR, both well inside the method's 0.01 dB target."""
    wl = W.uwb(G=16)
    r32 = eng.snr(wl, precision=0)
    r64 = eng.snr(wl, precision=1)
    e32, e64 = np.asarray(r32["eta"]), np.asarray(r64["eta"])
    s32, s64 = np.asarray(r32["snr"]), np.asarray(r64["snr"])
    err_eta_db = np.abs(10 * np.log10(e32 / e64))
    err_snr_db = np.abs(10 * np.log10(s32 / s64))
    assert err_eta_db.shape == (589,)
    assert err_eta_db.max() < 1e-3, (err_eta_db.max(), int(err_eta_db.argmax()))
    assert err_snr_db.max() < 1e-3, (err_snr_db.max(), int(err_snr_db.argmax()))
