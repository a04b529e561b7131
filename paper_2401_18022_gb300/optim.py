"""Differentiable throughput and launch-power optimisation (Sec. IV).

``throughput(P, engine, wl)`` is a ``torch.autograd.Function``: its forward
is ``isrs_gn_snr`` (or, when P requires grad, the fused ``isrs_gn_grad``
call) and its backward returns the adjoint dT/dP computed by the library.

``ascent`` maximises the Shannon throughput T over the per-channel launch
powers in dBm, within bounds [lo, hi] (the paper bounds its optimiser at
-5..5 dBm), by projected gradient ascent with Armijo backtracking.  The paper
uses L-BFGS-B with finite-difference gradients over power segments; here the
gradient of every channel comes from one adjoint pass.  The state can be
checkpointed to a JSON file every few iterations and resumed.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

import numpy as np

LN10_10 = math.log(10.0) / 10.0


def _torch():
    import torch
    return torch


class _Throughput:
    """Holder so that the Function class is only built when torch is imported."""
    fn = None


def _function():
    if _Throughput.fn is None:
        torch = _torch()

        class ThroughputFn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, P, engine, wl):
                Pd = P.detach().to(torch.float64).contiguous()
                if ctx.needs_input_grad[0]:
                    r = engine.grad(wl, P=Pd)
                    ctx.save_for_backward(r["dT_dP"].to(P.dtype))
                else:
                    r = engine.snr(wl, P=Pd)
                return torch.tensor(r["T"], dtype=P.dtype, device=P.device)

            @staticmethod
            def backward(ctx, gT):
                (g,) = ctx.saved_tensors
                return gT * g, None, None

        _Throughput.fn = ThroughputFn
    return _Throughput.fn


def throughput(P, engine, wl):
    """Throughput T [Tb/s] of launch powers P [W] (a torch tensor), differentiable in P."""
    return _function().apply(P, engine, wl)


def ascent(engine, wl, P0_W=None, iters: int = 50, lo_dbm: float = -5.0, hi_dbm: float = 5.0,
           step_db: float = 1.0, armijo: float = 1e-4, ckpt: Optional[str] = None, ckpt_every: int = 5,
           resume: bool = False, log=None) -> dict:
    """Projected gradient ascent of T in dBm with Armijo backtracking.

    Every iteration: one adjoint call (dT/dP), then forward-only calls
    until the Armijo condition T(x') >= T(x) + c g.(x' - x) holds.  Both
    sides of the condition are forward-call values: the adjoint call's own T
    can differ from the forward's in the last digits (its FP32 z-sum takes a
    different form for some points), which near the optimum would reject
    every trial step.  The first trial step moves the largest-gradient channel
    by `step_db` dB; the step grows by 2 after an accepted first trial and
    halves on each rejection.
    """
    torch = _torch()
    dev = getattr(engine, "torch_device", None) or torch.device("cuda", engine.device)
    x = 10.0 * np.log10(np.asarray(wl.P_W if P0_W is None else P0_W, dtype=np.float64) / 1e-3)
    x = np.clip(x, lo_dbm, hi_dbm)
    scale = step_db
    hist = []
    start = 0
    if resume and ckpt and os.path.exists(ckpt):
        st = json.load(open(ckpt))
        x, scale, hist, start = np.asarray(st["x_dbm"]), st["scale"], st["history"], st["iter"]

    def P_of(xd):
        return torch.tensor(1e-3 * 10.0 ** (xd / 10.0), dtype=torch.float64, device=dev)

    Tf = None      # forward T at x
    for it in range(start, iters):
        P = P_of(x)
        r = engine.grad(wl, P=P)
        T0 = r["T"]
        if Tf is None:
            Tf = engine.snr(wl, P=P)["T"]
        gx = r["dT_dP"].cpu().numpy() * (1e-3 * 10.0 ** (x / 10.0)) * LN10_10   # dT/dx [Tb/s per dB]
        # projected direction: drop components pushing against an active bound
        free = ~(((x <= lo_dbm) & (gx < 0)) | ((x >= hi_dbm) & (gx > 0)))
        d = np.where(free, gx, 0.0)
        gmax = float(np.max(np.abs(d))) if d.size else 0.0
        if gmax == 0.0:
            hist.append({"iter": it, "T": T0, "step": 0.0, "evals": 0})
            break
        alpha = scale / gmax
        evals = 0
        accepted = False
        while evals < 30:
            xn = np.clip(x + alpha * d, lo_dbm, hi_dbm)
            Tn = engine.snr(wl, P=P_of(xn))["T"]
            evals += 1
            if Tn >= Tf + armijo * float(np.dot(gx, xn - x)):
                accepted = True
                break
            alpha *= 0.5
        step = float(np.max(np.abs(xn - x))) if accepted else 0.0
        if accepted:
            x = xn
            Tf = Tn
            scale = min(4.0 * step_db, 2.0 * alpha * gmax) if evals == 1 else alpha * gmax
        else:
            scale *= 0.25
        hist.append({"iter": it, "T": float(Tn if accepted else T0), "T_before": T0, "step_db": step,
                     "evals": evals, "grad_inf_per_dB": gmax})
        if log:
            log(hist[-1])
        if ckpt and ((it + 1) % ckpt_every == 0 or it + 1 == iters):
            tmp = ckpt + ".tmp"
            json.dump({"x_dbm": x.tolist(), "scale": scale, "history": hist, "iter": it + 1}, open(tmp, "w"))
            os.replace(tmp, ckpt)
    return {"x_dbm": x, "P_W": 1e-3 * 10.0 ** (x / 10.0), "history": hist}


def main(argv=None):
    import argparse
    from . import api, workloads as W
    ap = argparse.ArgumentParser(description="gradient-ascent launch-power optimisation, 589-ch system")
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--G", type=int, default=64)
    ap.add_argument("--ckpt", default=None)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    eng = api.Engine(0)
    wl = W.uwb(G=a.G)
    res = ascent(eng, wl, iters=a.iters, ckpt=a.ckpt, resume=a.resume,
                 log=lambda h: print(json.dumps(h), flush=True))
    T32 = eng.snr(wl, P=res["P_W"])["T"]
    # the plain forward-only FP64 path beside the FP32 result
    T64 = eng.snr(wl, P=res["P_W"], precision=1)["T"]
    out = {"T_start": res["history"][0]["T_before"], "T_final_fp32": T32, "T_final_fp64": T64,
           "iters": len(res["history"]), "G": a.G, "x_dbm_minmax": [float(res["x_dbm"].min()),
                                                                   float(res["x_dbm"].max())]}
    print(json.dumps(out), flush=True)
    if a.out:
        json.dump({**out, "history": res["history"], "x_dbm": res["x_dbm"].tolist()}, open(a.out, "w"))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
