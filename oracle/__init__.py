"""FP64 CPU oracle of the ISRS GN integral model (arXiv 2401.18022).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library and never imports it; it takes plain
arrays (or any object carrying the workload attributes) and returns numpy
arrays.

The arithmetic lives in ``isrs_oracle.c`` (plain C, double precision, built
with gcc by :func:`build`).  Pins for every function are in
``tests/test_oracle_*.py``.  Parity unpinned: nothing — each exported
function has at least one independent pin.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isrs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, f"liborc_{platform.machine()}.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_beta_from_dispersion.argtypes = [ctypes.c_double] * 4 + [_D]
        lib.orc_gamma.argtypes = [ctypes.c_double] * 3
        lib.orc_gamma.restype = ctypes.c_double
        lib.orc_zgrid.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]
        lib.orc_phi.argtypes = [ctypes.c_double] * 6
        lib.orc_phi.restype = ctypes.c_double
        lib.orc_leff.argtypes = [ctypes.c_double] * 2
        lib.orc_leff.restype = ctypes.c_double
        lib.orc_lnrho.argtypes = [ctypes.c_int, _D, _D, _D, _D] + [ctypes.c_double] * 5
        lib.orc_lnrho.restype = ctypes.c_double
        lib.orc_zsum.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, _D]
        lib.orc_zsum_spans.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _D]
        lib.orc_pieces_flat.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, ctypes.c_int, _D]
        lib.orc_pieces_flat.restype = ctypes.c_int
        lib.orc_sigma.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, _I, ctypes.c_double, _I,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_sigma.restype = ctypes.c_int
        lib.orc_sigma_sampled.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, _I, ctypes.c_double,
                                          _I, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _D, _D]
        lib.orc_sigma_sampled.restype = ctypes.c_int
        lib.orc_eta_from_sigma.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D]
        lib.orc_snr_throughput.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, ctypes.c_int, _D, _D,
                                           ctypes.c_double, ctypes.POINTER(ctypes.c_ubyte), _D, _D]
        lib.orc_snr_throughput.restype = ctypes.c_double
        lib.orc_raman_solve.argtypes = [ctypes.c_int, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, _D, _I, _D]
        lib.orc_raman_solve.restype = ctypes.c_int
        lib.orc_raman_profile.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, ctypes.c_int, _D, _D, _D]
        lib.orc_raman_profile.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# Elementary functions (each a direct statement of one equation)
# --------------------------------------------------------------------------
def beta_from_dispersion(lambda_nm: float, D: float, S: float, Sdot: float) -> np.ndarray:
    """Sec. II, Eqs. d, d_slope, d_curve -> [beta2, beta3, beta4] (ps^k/km)."""
    out = np.zeros(3)
    _load().orc_beta_from_dispersion(lambda_nm, D, S, Sdot, _dp(out))
    return out


def gamma(lambda_nm: float, n2: float, aeff_um2: float) -> float:
    """Sec. II, Eq. gamma [1/(W km)]."""
    return float(_load().orc_gamma(lambda_nm, n2, aeff_um2))


def zgrid(L: float, alpha: float, n_edges: int) -> np.ndarray:
    """Equal-power-drop z edges (Sec. III-A, App. A)."""
    z = np.zeros(n_edges)
    if _load().orc_zgrid(L, alpha, n_edges, _dp(z)) != 0:
        raise ValueError("bad z-grid arguments")
    return z


def phi(f1: float, f2: float, fi: float, b2: float, b3: float, b4: float) -> float:
    """App. A, Eq. phi [rad/km]."""
    return float(_load().orc_phi(f1, f2, fi, b2, b3, b4))


def leff(z: float, alpha_R: float) -> float:
    return float(_load().orc_leff(z, alpha_R))


def lnrho(f, B, P, alpha, f_ref, Cr, alpha_R, z, F) -> float:
    """ln of the ISRS power profile rho(z, F) (linear Raman slope closed form)."""
    f, B, P, alpha = _f64(f), _f64(B), _f64(P), _f64(alpha)
    return float(_load().orc_lnrho(len(f), _dp(f), _dp(B), _dp(P), _dp(alpha),
                                   f_ref, Cr, alpha_R, z, F))


def zsum(z_mid, dz, p, phi_: float) -> complex:
    """App. A, Eq. slow_vary for given per-step powers p_m."""
    z_mid, dz, p = _f64(z_mid), _f64(dz), _f64(p)
    out = np.zeros(2)
    _load().orc_zsum(len(z_mid), _dp(z_mid), _dp(dz), _dp(p), phi_, _dp(out))
    return complex(out[0], out[1])


def zsum_spans(z_mid, dz, p, phi_: float, L: float, n_spans: int) -> complex:
    """Eq. new_gn_model: the z-sum over n identical spans with offsets (k-1) L."""
    z_mid, dz, p = _f64(z_mid), _f64(dz), _f64(p)
    out = np.zeros(2)
    _load().orc_zsum_spans(len(z_mid), _dp(z_mid), _dp(dz), _dp(p), phi_, L, int(n_spans), _dp(out))
    return complex(out[0], out[1])


def pieces(f, B, cut: int, cell_set: int) -> np.ndarray:
    """Pieces of one CUT: rows (a, b, s1, s2, xlo, xhi, ylo, yhi)."""
    f, B = _f64(f), _f64(B)
    n = _load().orc_pieces_flat(len(f), _dp(f), _dp(B), cut, cell_set,
                                None)
    out = np.zeros((n, 8))
    _load().orc_pieces_flat(len(f), _dp(f), _dp(B), cut, cell_set, _dp(out))
    return out


# --------------------------------------------------------------------------
# Workload-level evaluation
# --------------------------------------------------------------------------
def _raman_tail(wl) -> list:
    return [float(getattr(wl, "profile", 0)), float(getattr(wl, "raman_max_THz", 15.0)),
            float(getattr(wl, "raman_photon", 1)), float(getattr(wl, "ode_h_km", 0.25))]


def fibre_params(wl) -> np.ndarray:
    """[L, f_ref, beta2, beta3, beta4, Cr, alpha_R, n_spans, profile, df_max, photon, h_max]
    of a workload-like object."""
    b = beta_from_dispersion(C_NM_PER_PS / wl.f_ref_THz, wl.D_ref, wl.S_ref, wl.Sdot_ref)
    return np.array([wl.L_km, wl.f_ref_THz, b[0], b[1], b[2], wl.Cr, wl.alpha_R_per_km,
                     float(getattr(wl, "n_spans", 1))] + _raman_tail(wl))


def _fib12(fib, wl) -> np.ndarray:
    """Accepts the 7- or 8-entry forms (single span, closed-form profile) and
    completes them from the workload."""
    fib = _f64(fib)
    if fib.shape[0] == 7:
        fib = np.concatenate([fib, [float(getattr(wl, "n_spans", 1))]])
    if fib.shape[0] == 8:
        fib = np.concatenate([fib, _raman_tail(wl)])
    return np.ascontiguousarray(fib)


def _scale(wl):
    sc = getattr(wl, "raman_scale", None)
    return None if sc is None else _f64(sc)


def raman_solve(f, P, alpha, Cr, df_max, photon, z_nodes, n_sub, scale=None) -> np.ndarray:
    """RK4 solution of the Raman ODE (profile model R2) at the given nodes:
    rows = nodes, columns = channels, values y = ln P (0 at z = 0 for empty slots)."""
    f, P, alpha, z = _f64(f), _f64(P), _f64(alpha), _f64(z_nodes)
    ns = np.ascontiguousarray(np.asarray(n_sub, dtype=np.int32))
    sc = None if scale is None else _f64(scale)
    out = np.zeros((len(z), len(f)))
    rc = _load().orc_raman_solve(len(f), _dp(f), _dp(P), _dp(alpha), None if sc is None else _dp(sc),
                                 float(Cr), float(df_max), int(photon), len(z) - 1, _dp(z),
                                 ns.ctypes.data_as(_I), _dp(out))
    if rc != 0:
        raise ValueError("bad Raman ODE arguments")
    return out


def raman_profile(wl, P=None):
    """Profile model R2 on the workload's z-grid: (a [n, M], b [n, M], a_L [n])
    with ln rho(z_m, F) = a[c, m] + b[c, m] (F - f_c) inside channel c."""
    f, alpha = _f64(wl.f_THz), _f64(wl.alpha_per_km)
    P = _f64(wl.P_W if P is None else P)
    fib = fibre_params(wl)
    fib[8] = 1.0
    n, M = len(f), wl.n_edges - 1
    a, b, aL = np.zeros((n, M)), np.zeros((n, M)), np.zeros(n)
    sc = _scale(wl)
    rc = _load().orc_raman_profile(n, _dp(f), _dp(P), _dp(alpha), None if sc is None else _dp(sc),
                                   _dp(fib), int(wl.n_edges), _dp(a), _dp(b), _dp(aL))
    if rc != 0:
        raise ValueError("bad Raman profile arguments")
    return a, b, aL


C_NM_PER_PS = 299792.458


def gammas(wl) -> np.ndarray:
    if getattr(wl, "gamma_fixed", None) is not None:
        return np.full(len(wl.f_THz), float(wl.gamma_fixed))
    return np.array([gamma(l, wl.n2_m2_per_W, a) for l, a in zip(wl.lambda_nm, wl.aeff_um2)])


def sigma(wl, P=None, cuts: Optional[Sequence[int]] = None, threads: Optional[int] = None,
          unit_integrand: bool = False, fibre: Optional[np.ndarray] = None,
          return_pieces: bool = False):
    """Sigma_i: the frequency integral at f_i (Eq. gain_fin without 16/27 gamma^2)."""
    f, B = _f64(wl.f_THz), _f64(wl.B_THz)
    P = _f64(wl.P_W if P is None else P)
    alpha = _f64(wl.alpha_per_km)
    fib = _fib12(fibre_params(wl) if fibre is None else fibre, wl)
    quad = np.array([wl.G, wl.n_edges, wl.cell_set, int(getattr(wl, "G_mci", 0))], dtype=np.int32)
    cuts = np.arange(len(f), dtype=np.int32) if cuts is None else np.asarray(cuts, dtype=np.int32)
    cuts = np.ascontiguousarray(cuts)
    threads = threads or os.cpu_count() or 1
    out = np.zeros(len(cuts))
    n_pieces = sum(_load().orc_pieces_flat(len(f), _dp(f), _dp(B), int(c), int(wl.cell_set),
                                           None) for c in cuts)
    pout = np.zeros(max(n_pieces, 1))
    sc = _scale(wl)
    rc = _load().orc_sigma(len(f), _dp(f), _dp(B), _dp(P), _dp(alpha), None if sc is None else _dp(sc),
                           _dp(fib),
                           quad.ctypes.data_as(_I), float(wl.eps_v1),
                           cuts.ctypes.data_as(_I), len(cuts), int(threads),
                           1 if unit_integrand else 0, _dp(out), _dp(pout))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    if return_pieces:
        return out, pout[:n_pieces]
    return out


def time_sample(wl, cuts, stride: int, threads: Optional[int] = None) -> dict:
    """Time the oracle on every stride-th piece of the given CUTs (a bounded
    sample of a workload).  Returns the wall time and the grid points and
    point-steps the sample evaluated."""
    import time
    f, B = _f64(wl.f_THz), _f64(wl.B_THz)
    P, alpha = _f64(wl.P_W), _f64(wl.alpha_per_km)
    fib = _fib12(fibre_params(wl), wl)
    quad = np.array([wl.G, wl.n_edges, wl.cell_set, int(getattr(wl, "G_mci", 0))], dtype=np.int32)
    cuts = np.ascontiguousarray(np.asarray(cuts, dtype=np.int32))
    threads = threads or os.cpu_count() or 1
    n_pieces = sum(_load().orc_pieces_flat(len(f), _dp(f), _dp(B), int(c), int(wl.cell_set), None)
                   for c in cuts)
    pout = np.zeros(max(n_pieces, 1))
    out = np.zeros(len(cuts))
    t0 = time.perf_counter()
    sc = _scale(wl)
    rc = _load().orc_sigma_sampled(len(f), _dp(f), _dp(B), _dp(P), _dp(alpha),
                                   None if sc is None else _dp(sc), _dp(fib),
                                   quad.ctypes.data_as(_I), float(wl.eps_v1), cuts.ctypes.data_as(_I),
                                   len(cuts), int(threads), 0, int(stride), _dp(out), _dp(pout))
    dt = time.perf_counter() - t0
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    n_eval = len(range(0, n_pieces, max(1, int(stride))))
    pts = n_eval * wl.G * wl.G
    return {"seconds": dt, "points": pts, "point_steps": pts * (wl.n_edges - 1), "threads": threads,
            "pieces": n_eval, "pieces_total": n_pieces}


def eta(wl, sigma_: np.ndarray, cuts=None, P=None):
    """eta_i = 16/27 gamma_i^2 B_i Sigma_i / P_i^3 and P_NLI,i."""
    P = _f64(wl.P_W if P is None else P)
    cuts = np.arange(len(P)) if cuts is None else np.asarray(cuts)
    g = _f64(gammas(wl)[cuts])
    Bc, Pc, s = _f64(np.asarray(wl.B_THz)[cuts]), _f64(P[cuts]), _f64(sigma_)
    e, pn = np.zeros(len(cuts)), np.zeros(len(cuts))
    _load().orc_eta_from_sigma(len(cuts), _dp(s), _dp(g), _dp(Bc), _dp(Pc), _dp(e), _dp(pn))
    return e, pn


def snr_throughput(wl, eta_all: np.ndarray, P=None, fibre=None):
    """Per-channel SNR (Sec. IV, Eq. loss), ASE power, and throughput T [Tb/s]."""
    f, B, alpha = _f64(wl.f_THz), _f64(wl.B_THz), _f64(wl.alpha_per_km)
    P = _f64(wl.P_W if P is None else P)
    fib = _fib12(fibre_params(wl) if fibre is None else fibre, wl)
    nf = _f64(wl.nf_dB)
    e = _f64(eta_all)
    g = getattr(wl, "guard", None)
    gp = None
    if g is not None:
        g = np.ascontiguousarray(np.asarray(g, dtype=np.uint8))
        gp = g.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    snr, pase = np.zeros(len(f)), np.zeros(len(f))
    sc = _scale(wl)
    T = _load().orc_snr_throughput(len(f), _dp(f), _dp(B), _dp(P), _dp(alpha),
                                   None if sc is None else _dp(sc), _dp(fib), int(wl.n_edges), _dp(e),
                                   _dp(nf), float(wl.snr_trx_dB), gp, _dp(snr), _dp(pase))
    return snr, pase, float(T)


def evaluate(wl, P=None, threads=None):
    """Full oracle pass: Sigma, eta, P_NLI, SNR, ASE and throughput for all CUTs."""
    s = sigma(wl, P=P, threads=threads)
    e, pn = eta(wl, s, P=P)
    snr, pase, T = snr_throughput(wl, e, P=P)
    return {"sigma": s, "eta": e, "pnli": pn, "snr": snr, "pase": pase, "T": T}
