"""Launch-power optimisation over power segments (Sec. IV, Eq. loss).

The optimisation variables are launch powers in dBm at segment edges.  Each
band b is split into N_B = round(B_band / B_p) equal segments (B_band: the
band's loaded bandwidth, n_b slots x 100 GHz; B_p = 750 GHz in the O band,
1.5 THz elsewhere) with at least two edges per band, and every channel's dBm
value is the linear interpolation, in frequency, of its two neighbouring
edges.  All of this is a fixed linear map x_ch = M x from the variables to
the per-channel dBm values (``PowerParam``); the spectrally uniform case
(Case 2) is the one-column map and the per-channel case the identity.

The cost is the paper's loss

    L(x) = -sum_{i not in A} log2(1 + SNR_i(P)),   P_i = 1 mW * 10^(x_ch,i / 10),

with the guard set A left out of the plan (its slots carry no power).  With a
common channel bandwidth B the throughput is T = -2 B L, so L and its
gradient follow from one ``isrs_gn_grad`` call:

    dL/dx = M^T ( -(1 / 2B) dT/dP  *  P ln10 / 10 ).

The gradient is the library's adjoint instead of the paper's finite
differences.  ``optimise`` runs SciPy's L-BFGS-B within [-5, 5] dBm from a
uniform 0 dBm start and stops when the largest projected gradient component
is at most 0.01 (the paper's stop condition); ``run_stages`` repeats it on a
finer quadrature from the coarse result, as the paper does.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import workloads as W

LN10_10 = math.log(10.0) / 10.0
B_P_THZ = {"O": 0.75}               # segment bandwidth B_p per band; others use the default
B_P_DEFAULT_THZ = 1.5


def n_segments(n_channels: int, b_p_thz: float, slot_thz: float = W.SLOT_THZ) -> int:
    """N_B = round(B_band / B_p), with B_band = n_channels * slot (halves round up)."""
    return int(math.floor(n_channels * slot_thz / b_p_thz + 0.5))


@dataclass
class PowerParam:
    """Linear map from optimisation variables (dBm) to per-channel dBm values."""
    M: np.ndarray                           # [n_ch, n_var]
    labels: List[str] = field(default_factory=list)
    edges_thz: Optional[np.ndarray] = None  # frequency of each variable (segment edges)

    @property
    def n_var(self) -> int:
        return self.M.shape[1]

    def x_ch(self, x) -> np.ndarray:
        return self.M @ np.asarray(x, dtype=np.float64)


def per_channel(n_ch: int) -> PowerParam:
    return PowerParam(np.eye(n_ch), [f"ch{i}" for i in range(n_ch)])


def uniform(n_ch: int) -> PowerParam:
    """Case 2: one launch power for every loaded channel."""
    return PowerParam(np.ones((n_ch, 1)), ["all"])


def segments(f_thz: np.ndarray, band: np.ndarray, b_p_thz: Optional[Dict[str, float]] = None,
             slot_thz: float = W.SLOT_THZ) -> PowerParam:
    """Segment-edge parameterisation of channels at `f_thz` grouped by `band`
    (indices into W.BAND_NAMES).  Edges are equally spaced from the band's
    first to its last channel centre; a band of one channel has one edge."""
    f = np.asarray(f_thz, dtype=np.float64)
    band = np.asarray(band)
    b_p = dict(B_P_THZ if b_p_thz is None else b_p_thz)
    cols, labels, edges_all = [], [], []
    M_blocks = []
    for b in sorted(set(band.tolist()), key=lambda k: -k):     # increasing frequency
        idx = np.flatnonzero(band == b)
        fb = f[idx]
        name = W.BAND_NAMES[b]
        nb = n_segments(len(idx), b_p.get(name, B_P_DEFAULT_THZ), slot_thz)
        if len(idx) == 1:
            e = fb[:1].copy()
        else:
            e = np.linspace(fb.min(), fb.max(), max(nb, 1) + 1)
        Mb = np.zeros((len(f), len(e)))
        if len(e) == 1:
            Mb[idx, 0] = 1.0
        else:
            k = np.clip(np.searchsorted(e, fb, side="right") - 1, 0, len(e) - 2)
            t = np.clip((fb - e[k]) / (e[k + 1] - e[k]), 0.0, 1.0)
            Mb[idx, k] = 1.0 - t
            Mb[idx, k + 1] = t
        M_blocks.append(Mb)
        labels += [f"{name}{j}" for j in range(len(e))]
        edges_all.append(e)
    return PowerParam(np.concatenate(M_blocks, axis=1), labels, np.concatenate(edges_all))


def band_of(wl) -> np.ndarray:
    """Band index (0 = O ... 5 = U) of each channel from its wavelength."""
    return np.clip(np.searchsorted(W.BAND_EDGES_NM, wl.lambda_nm, side="right") - 1, 0, 5)


class Objective:
    """L(x) and dL/dx through one gradient call of `engine` per evaluation.

    `engine` is anything with ``grad(wl, P=...) -> {"T", "dT_dP", "snr"}``
    (T in Tb/s with bandwidths in THz); the library's Engine is the product
    one.  Every evaluation is appended to ``history``.
    """

    def __init__(self, engine, wl, param: PowerParam):
        B = np.asarray(wl.B_THz, dtype=np.float64)
        if B.size == 0 or np.ptp(B) > 1e-12 * B.max():
            raise ValueError("the loss of Eq. loss needs one common channel bandwidth")
        if param.M.shape[0] != wl.n_ch:
            raise ValueError("parameterisation does not match the channel plan")
        self.engine, self.wl, self.param = engine, wl, param
        self.two_b = 2.0 * float(B[0])
        self.history: List[dict] = []
        self.seconds = 0.0

    def powers(self, x) -> np.ndarray:
        return 1e-3 * np.power(10.0, self.param.x_ch(x) / 10.0)

    def __call__(self, x):
        t0 = time.perf_counter()
        P = self.powers(x)
        r = self.engine.grad(self.wl, P=P)
        dTdP = np.asarray(r["dT_dP"], dtype=np.float64)
        L = -float(r["T"]) / self.two_b
        g_ch = -(dTdP / self.two_b) * P * LN10_10
        g = self.param.M.T @ g_ch
        self.seconds += time.perf_counter() - t0
        self.history.append({"eval": len(self.history), "T": float(r["T"]), "L": L,
                             "grad_inf": float(np.max(np.abs(g)))})
        return L, g


def projected_grad_inf(x, g, lo: float, hi: float) -> float:
    """max_i |proj g_i| of a minimisation within [lo, hi] (L-BFGS-B's measure)."""
    x, g = np.asarray(x), np.asarray(g)
    pg = np.where(g > 0, np.minimum(g, x - lo), np.maximum(g, x - hi))
    return float(np.max(np.abs(pg))) if pg.size else 0.0


def optimise(obj: Objective, x0=None, lo: float = -5.0, hi: float = 5.0, gtol: float = 0.01,
             maxiter: int = 500, ckpt: Optional[str] = None, log: Optional[Callable] = None) -> dict:
    """L-BFGS-B on `obj` within [lo, hi] dBm, stopping at max |proj grad| <= gtol.

    With `ckpt`, the current iterate is written to that JSON file after every
    iteration; a later call with the same file starts from it (L-BFGS-B's
    curvature memory is rebuilt from there).
    """
    from scipy.optimize import minimize
    n = obj.param.n_var
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    if ckpt and os.path.exists(ckpt):
        x = np.asarray(json.load(open(ckpt))["x_dbm"], dtype=np.float64)
    x = np.clip(x, lo, hi)
    iters = []

    def cb(xk):
        h = obj.history[-1] if obj.history else {}
        iters.append({"iter": len(iters), "L": h.get("L"), "T": h.get("T"), "evals": len(obj.history)})
        if log:
            log(iters[-1])
        if ckpt:
            tmp = ckpt + ".tmp"
            json.dump({"x_dbm": np.asarray(xk).tolist(), "iter": len(iters)}, open(tmp, "w"))
            os.replace(tmp, ckpt)

    res = minimize(obj, x, jac=True, method="L-BFGS-B", bounds=[(lo, hi)] * n, callback=cb,
                   options={"gtol": gtol, "ftol": 1e-13, "maxiter": maxiter, "maxcor": 10})
    L, g = float(res.fun), np.asarray(res.jac, dtype=np.float64)
    return {"x_dbm": np.asarray(res.x), "L": L, "T": -obj.two_b * L,
            "pg_inf": projected_grad_inf(res.x, g, lo, hi), "converged": bool(res.success),
            "message": str(res.message), "nit": int(res.nit), "nfev": int(res.nfev),
            "seconds": obj.seconds, "iters": iters}


def band_report(engine, wl, P, band: np.ndarray, snr_trx_dB: float = 0.0, precision: int = 0) -> dict:
    """Total launch power (dBm) and Shannon capacity (Tb/s) per band."""
    r = engine.snr(wl.with_(snr_trx_dB=snr_trx_dB), P=np.asarray(P), precision=precision)
    snr = np.asarray(r["snr"], dtype=np.float64)
    cap = 2.0 * np.asarray(wl.B_THz) * np.log2(1.0 + snr)
    out = {}
    for b in range(6):
        m = band == b
        if m.any():
            out[W.BAND_NAMES[b]] = {"pow_dBm": float(10 * np.log10(np.sum(P[m]) / 1e-3)),
                                    "cap_Tbps": float(cap[m].sum()),
                                    "snr_dB_min_max": [float(10 * np.log10(snr[m].min())),
                                                       float(10 * np.log10(snr[m].max()))]}
    return {"T": float(r["T"]), "total_dBm": float(10 * np.log10(np.sum(P) / 1e-3)), "bands": out}


def run_stages(engine, case: int = 1, stages: Sequence[int] = (32, 64), n_edges: int = 113,
               gtol: float = 0.01, maxiter: int = 500, log: Optional[Callable] = None,
               profile: str = "closed", g_mci: int = 0) -> dict:
    """Case 1 (segments) or Case 2 (uniform) on the guarded 557-channel plan:
    one L-BFGS-B run per quadrature size G in `stages`, each started from the
    previous result (the first from 0 dBm).  profile "raman" uses the
    Raman-ODE power profile (15 THz gain cut-off, photon ratio, Aeff
    scaling), "closed" the linear-slope closed form.  The optimisation sums
    the SCI and XCI cells; with g_mci > 0 the optimum is also evaluated over
    the whole band (every other cell on its own g_mci grid, App. A's integral
    over all frequencies), reported as report_mci."""
    x = None
    out = {"case": case, "profile": profile, "stages": []}
    for G in stages:
        wl = W.uwb_guarded(G=G, n_edges=n_edges)
        if profile == "raman":
            wl = W.raman(wl)
        band = band_of(wl)
        param = segments(wl.f_THz, band) if case == 1 else uniform(wl.n_ch)
        obj = Objective(engine, wl, param)
        res = optimise(obj, x0=x, gtol=gtol, maxiter=maxiter, log=log)
        x = res["x_dbm"]
        res.pop("iters")
        out["stages"].append({"G": G, "n_var": param.n_var, **{k: (v.tolist() if isinstance(v, np.ndarray)
                                                                  else v) for k, v in res.items()}})
    P = obj.powers(x)
    out["report"] = band_report(engine, wl, P, band)
    out["report_trx20"] = band_report(engine, wl, P, band, snr_trx_dB=20.0)
    if g_mci > 0:
        wm = wl.with_(cell_set=W.CELLS_ALL, G_mci=int(g_mci))
        out["report_mci"] = {"G_mci": int(g_mci), **band_report(engine, wm, P, band)}
        out["report_mci_trx20"] = band_report(engine, wm, P, band, snr_trx_dB=20.0)
    out["x_ch_dBm_min_max"] = [float(param.x_ch(x).min()), float(param.x_ch(x).max())]
    return out


def main(argv=None):
    import argparse
    from . import api
    ap = argparse.ArgumentParser(description="segment (Case 1) or uniform (Case 2) launch-power "
                                             "optimisation of the guarded 557-channel system")
    ap.add_argument("--case", type=int, default=1, choices=(1, 2))
    ap.add_argument("--stages", default="32,64", help="quadrature sizes G, comma separated")
    ap.add_argument("--gtol", type=float, default=0.01)
    ap.add_argument("--maxiter", type=int, default=500)
    ap.add_argument("--profile", default="raman", choices=("raman", "closed"))
    ap.add_argument("--mci", type=int, default=0,
                    help="> 0: also evaluate the optimum with every MCI cell on its own grid of this size")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    eng = api.Engine(0)
    stages = [int(s) for s in a.stages.split(",")]
    res = run_stages(eng, a.case, stages, gtol=a.gtol, maxiter=a.maxiter,
                     log=lambda h: print(json.dumps(h), flush=True), profile=a.profile, g_mci=a.mci)
    print(json.dumps({k: v for k, v in res.items()}), flush=True)
    if a.out:
        json.dump(res, open(a.out, "w"), indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
