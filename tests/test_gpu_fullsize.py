"""Parity at the full sizes the benchmark times, on sampled outputs.

* 589 channels, G = 256, 113 edges, SCI + XCI (the bench launch): all 589 CUTs
  in one FP32 launch; CUT 0 (band edge, strongest ISRS gain) checked against
  the FP64 oracle, 8 CUTs against the plain FP64 GPU path; at G = 16 all
  589 CUTs against the FP64 GPU path (per-CUT dB error of eta and SNR).
* The gradient call at that size returns the same SNR, eta and T as the
  forward call.
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


def test_uwb_full_cut0_vs_oracle(uwb_full, orc):
    wl, _, r = uwb_full
    ref = orc.sigma(wl, cuts=[0], threads=os.cpu_count())
    np.testing.assert_allclose(r["sigma"][0], ref[0], rtol=RTOL_F32)


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
