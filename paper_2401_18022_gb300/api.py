"""Python binding of the ISRS GN C ABI (argument marshalling only).

Every step of the computation runs in the CUDA library; this module turns a
:class:`~paper_2401_18022_gb300.workloads.Workload` and launch powers (numpy
arrays on the host, or torch tensors on the host or the GPU) into the ABI's
structs and pointers.  Outputs live where the powers live: numpy in, numpy
out; a CUDA tensor in, CUDA tensors out (asynchronous on torch's current
stream).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _capi
from ._capi import CELLS_ALL, CELLS_SCI_XCI, PREC_FP32, PREC_FP64, check  # noqa: F401


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _as_f64(x):
    if _is_torch(x):
        import torch
        return x.to(torch.float64).contiguous()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(x) -> int:
    if _is_torch(x):
        return x.data_ptr()
    return x.ctypes.data


def _empty_like(x, n: int):
    if _is_torch(x):
        import torch
        return torch.empty(n, dtype=torch.float64, device=x.device)
    return np.empty(n, dtype=np.float64)


def _stream_of(x):
    if _is_torch(x) and x.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


class Engine:
    """A handle on one CUDA device owning workspace and cached plan tables."""

    def __init__(self, device: int = 0):
        self.lib = _capi.load()
        self.h = ctypes.c_void_p()
        check(self.lib.isrs_create(ctypes.byref(self.h), int(device)))
        self.device = device

    @property
    def debug_build(self) -> bool:
        """Whether the loaded library is the bounds-checked debug build."""
        return bool(self.lib.isrs_debug_build())

    def close(self):
        if self.h:
            self.lib.isrs_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- structs ---------------------------------------------------------
    def beta(self, wl) -> np.ndarray:
        out = np.zeros(3)
        check(self.lib.isrs_beta_from_dispersion(wl.lambda_ref_nm, wl.D_ref, wl.S_ref, wl.Sdot_ref,
                                                 out.ctypes.data_as(_capi.c_double_p)))
        return out

    def gammas(self, wl) -> np.ndarray:
        if wl.gamma_fixed is not None:
            return np.full(wl.n_ch, float(wl.gamma_fixed))
        return np.array([self.lib.isrs_gamma_from_aeff(l, wl.n2_m2_per_W, a)
                         for l, a in zip(wl.lambda_nm, wl.aeff_um2)])

    def fibre(self, wl) -> _capi.Fibre:
        b = self.beta(wl)
        return _capi.Fibre(wl.L_km, wl.f_ref_THz, b[0], b[1], b[2], wl.Cr, wl.alpha_R_per_km,
                           int(getattr(wl, "n_spans", 1)), int(getattr(wl, "profile", 0)),
                           float(getattr(wl, "raman_max_THz", 15.0)), int(getattr(wl, "raman_photon", 1)))

    def channels(self, wl):
        keep = {k: np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for k, v in
                (("f", wl.f_THz), ("B", wl.B_THz), ("a", wl.alpha_per_km), ("g", self.gammas(wl)),
                 ("nf", wl.nf_dB))}
        dp = lambda a: a.ctypes.data_as(_capi.c_double_p)  # noqa: E731
        guard = None
        if getattr(wl, "guard", None) is not None:
            keep["guard"] = np.ascontiguousarray(np.asarray(wl.guard, dtype=np.uint8))
            guard = keep["guard"].ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        scale = None
        if getattr(wl, "raman_scale", None) is not None:
            keep["scale"] = np.ascontiguousarray(np.asarray(wl.raman_scale, dtype=np.float64))
            scale = dp(keep["scale"])
        ch = _capi.Channels(wl.n_ch, dp(keep["f"]), dp(keep["B"]), dp(keep["a"]), dp(keep["g"]),
                            dp(keep["nf"]), guard, scale)
        return ch, keep

    @staticmethod
    def quad(wl, precision: int = PREC_FP32) -> _capi.Quad:
        return _capi.Quad(int(wl.G), int(wl.n_edges), float(wl.eps_v1), int(wl.cell_set), int(precision),
                          float(wl.snr_trx_dB), float(getattr(wl, "ode_h_km", 0.25)),
                          int(getattr(wl, "G_mci", 0)))

    def inject_fault(self, kind: int, after: int = 1):
        """Arm one simulated failure (1: the after-th device allocation, 2: the
        after-th checked CUDA call of this handle); 0 disarms."""
        check(self.lib.isrs_debug_inject_fault(self.h, int(kind), int(after)), self.h)

    def set_tile(self, points_per_item: int = 0, threads_per_block: int = 0):
        check(self.lib.isrs_set_tile(self.h, points_per_item, threads_per_block), self.h)

    def last_launch_info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        check(self.lib.isrs_last_launch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"points": a.value, "point_steps": b.value, "launches": c.value}

    def last_kernel_ms(self, which: int = 0) -> float:
        """Duration of the last quadrature (0) or adjoint (1) kernel, from
        CUDA events recorded on its launch stream."""
        ms = ctypes.c_float()
        check(self.lib.isrs_last_kernel_ms(self.h, int(which), ctypes.byref(ms)), self.h)
        return ms.value

    def probe_alu_peaks(self):
        """Measured SFU (MUFU ex2) and FP32 FMA throughput of this device [ops/s]."""
        out = {}
        for which, name in ((0, "sfu"), (1, "fp32")):
            v, ms = ctypes.c_double(), ctypes.c_float()
            check(self.lib.isrs_probe_alu_peaks(int(self.device), which, ctypes.byref(v), ctypes.byref(ms)))
            out[f"{name}_ops_per_s"] = v.value
            out[f"{name}_probe_ms"] = ms.value
        return out

    def last_graph_replay(self) -> bool:
        """Whether the last batched call replayed its captured CUDA graph."""
        v = ctypes.c_int()
        check(self.lib.isrs_last_graph_replay(self.h, ctypes.byref(v)), self.h)
        return bool(v.value)

    def last_path_counts(self):
        """Grid points of the last FP32 launch per z-sum form."""
        c = (ctypes.c_int64 * 3)()
        check(self.lib.isrs_last_path_counts(self.h, c), self.h)
        return {"small": c[0], "direct": c[1], "telescoped": c[2]}

    # ---- calls -----------------------------------------------------------
    def eta(self, wl, P=None, cuts: Optional[Sequence[int]] = None, precision: int = PREC_FP32,
            want_sigma: bool = True):
        """isrs_gn_eta: eta, P_NLI and Sigma for the listed CUTs (all if None)."""
        P = _as_f64(wl.P_W if P is None else P)
        fb, (ch, keep), q = self.fibre(wl), self.channels(wl), self.quad(wl, precision)
        n = wl.n_ch if cuts is None else len(cuts)
        cuts_arr = None
        cp = None
        if cuts is not None:
            cuts_arr = np.ascontiguousarray(np.asarray(cuts, dtype=np.int32))
            cp = cuts_arr.ctypes.data_as(_capi.c_int_p)
        eta, pnli = _empty_like(P, n), _empty_like(P, n)
        sig = _empty_like(P, n) if want_sigma else None
        check(self.lib.isrs_gn_eta(self.h, ctypes.byref(fb), ctypes.byref(ch), _ptr(P), ctypes.byref(q), cp,
                                   n, _ptr(eta), _ptr(pnli), _ptr(sig) if sig is not None else None,
                                   _stream_of(P)), self.h)
        return {"eta": eta, "pnli": pnli, "sigma": sig}

    def snr(self, wl, P=None, precision: int = PREC_FP32):
        """isrs_gn_snr: per-channel SNR, eta and the throughput T [Tb/s]."""
        P = _as_f64(wl.P_W if P is None else P)
        fb, (ch, keep), q = self.fibre(wl), self.channels(wl), self.quad(wl, precision)
        snr, eta = _empty_like(P, wl.n_ch), _empty_like(P, wl.n_ch)
        T = ctypes.c_double()
        check(self.lib.isrs_gn_snr(self.h, ctypes.byref(fb), ctypes.byref(ch), _ptr(P), ctypes.byref(q),
                                   _ptr(snr), _ptr(eta), ctypes.byref(T), _stream_of(P)), self.h)
        return {"snr": snr, "eta": eta, "T": T.value}

    def grad(self, wl, P=None):
        """isrs_gn_grad: dT/dP_j, SNR, eta and T of the FP32 path."""
        P = _as_f64(wl.P_W if P is None else P)
        fb, (ch, keep), q = self.fibre(wl), self.channels(wl), self.quad(wl, PREC_FP32)
        g, snr, eta = _empty_like(P, wl.n_ch), _empty_like(P, wl.n_ch), _empty_like(P, wl.n_ch)
        T = ctypes.c_double()
        check(self.lib.isrs_gn_grad(self.h, ctypes.byref(fb), ctypes.byref(ch), _ptr(P), ctypes.byref(q),
                                    _ptr(g), _ptr(snr), _ptr(eta), ctypes.byref(T), _stream_of(P)), self.h)
        return {"dT_dP": g, "snr": snr, "eta": eta, "T": T.value}

    def grad_shard_fwd(self, wl, cuts: Sequence[int], P=None):
        """isrs_gn_grad_shard_fwd: fused forward + adjoint over the CUTs of one
        shard; returns eta of those CUTs (the buckets stay in the handle)."""
        P = _as_f64(wl.P_W if P is None else P)
        fb, (ch, keep), q = self.fibre(wl), self.channels(wl), self.quad(wl, PREC_FP32)
        cuts_arr = np.ascontiguousarray(np.asarray(cuts, dtype=np.int32))
        eta = _empty_like(P, len(cuts_arr))
        check(self.lib.isrs_gn_grad_shard_fwd(self.h, ctypes.byref(fb), ctypes.byref(ch), _ptr(P), ctypes.byref(q),
                                              cuts_arr.ctypes.data_as(_capi.c_int_p), len(cuts_arr), _ptr(eta),
                                              _stream_of(P)), self.h)
        return eta

    def grad_shard_bwd(self, eta_all, with_direct: bool):
        """isrs_gn_grad_shard_bwd: this shard's part of dT/dP from the gathered
        eta of every channel, with the SNR of every channel and T."""
        eta_all = _as_f64(eta_all)
        n = int(eta_all.shape[0])
        g, snr = _empty_like(eta_all, n), _empty_like(eta_all, n)
        T = ctypes.c_double()
        check(self.lib.isrs_gn_grad_shard_bwd(self.h, _ptr(eta_all), 1 if with_direct else 0, _ptr(g), _ptr(snr),
                                              ctypes.byref(T), _stream_of(eta_all)), self.h)
        return {"dT_dP": g, "snr": snr, "T": T.value}

    def eta_batched(self, bw, P_cat=None, precision: int = PREC_FP32):
        """isrs_gn_eta_batched over a BatchedWorkload; P_cat concatenates the profiles."""
        if P_cat is None:
            P_cat = np.concatenate(bw.P_W)
        P_cat = _as_f64(P_cat)
        wl0 = bw.plans[0]
        fb, q = self.fibre(wl0), self.quad(wl0, precision)
        chs, keeps = zip(*(self.channels(p) for p in bw.plans))
        arr = (_capi.Channels * len(chs))(*chs)
        pop = np.ascontiguousarray(np.asarray(bw.plan_of_profile, dtype=np.int32))
        n_tot = int(sum(bw.plans[k].n_ch for k in pop))
        eta = _empty_like(P_cat, n_tot)
        check(self.lib.isrs_gn_eta_batched(self.h, ctypes.byref(fb), len(chs), arr, len(pop),
                                           pop.ctypes.data_as(_capi.c_int_p), _ptr(P_cat), ctypes.byref(q),
                                           _ptr(eta), _stream_of(P_cat)), self.h)
        return eta


_default = {}


def engine(device: int = 0) -> Engine:
    if device not in _default:
        _default[device] = Engine(device)
    return _default[device]
