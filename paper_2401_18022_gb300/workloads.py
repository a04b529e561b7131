"""Seeded synthetic workloads: channel plans, fibre models and launch powers.

This module is shared by the CUDA path, the tests, the benchmark and the
oracle's callers.  It holds none of the ISRS GN method's arithmetic: it only
lays out channel grids, evaluates the *configuration* models of the fibre
(attenuation, effective area and the dispersion model with its analytic
wavelength derivatives), converts units and draws seeded random powers.
The method's own steps (beta from D, gamma from n2/Aeff, the power profile,
the quadrature) live in the CUDA library and, independently, in the oracle.

Units everywhere: frequency THz, time ps, length km, power W,
dispersion ps/(nm km), slope ps/(nm^2 km), curvature ps/(nm^3 km).

The fibre data of the paper (mode solver, measured Raman gain, Sec. II) is
not available, so analytic stand-ins are used:
  * attenuation  alpha_dB(lambda) = 0.962 / lambda_um^4 + 0.0233  dB/km
    (Rayleigh term plus a constant floor; 0.35 dB/km at 1310 nm);
  * effective area linear from 60 um^2 at 1260 nm to 95 um^2 at 1675 nm;
  * dispersion D(lambda) = S0/4 (lambda - lambda0^4 / lambda^3),
    lambda0 = 1310 nm, S0 = 0.09 ps/(nm^2 km);
  * n2 = 2.6e-20 m^2/W, Raman slope C_r = 0.028 1/(W km THz).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

C_NM_PER_PS = 299792.458          # speed of light [nm/ps]: f[THz] = C / lambda[nm]
DB_PER_NEPER_POWER = 10.0 / np.log(10.0)   # 4.3429 dB per neper of power

# Amplifier noise figure per band (Table "Per band characteristics"), band
# edges in nm: O 1260-1360, E 1360-1460, S 1460-1530, C 1530-1565,
# L 1565-1625, U 1625-1675.
BAND_EDGES_NM = [1260.0, 1360.0, 1460.0, 1530.0, 1565.0, 1625.0, 1675.0]
BAND_NAMES = ["O", "E", "S", "C", "L", "U"]
BAND_NF_DB = [7.0, 7.0, 7.0, 5.0, 6.0, 8.0]

CELLS_SCI_XCI = 0
CELLS_ALL = 1


def thz_from_nm(lam_nm):
    return C_NM_PER_PS / np.asarray(lam_nm, dtype=np.float64)


def nm_from_thz(f_thz):
    return C_NM_PER_PS / np.asarray(f_thz, dtype=np.float64)


def dbm_to_w(p_dbm):
    return 1e-3 * np.power(10.0, np.asarray(p_dbm, dtype=np.float64) / 10.0)


def w_to_dbm(p_w):
    return 10.0 * np.log10(np.asarray(p_w, dtype=np.float64) / 1e-3)


def db_per_km_to_per_km(a_db):
    return np.asarray(a_db, dtype=np.float64) / DB_PER_NEPER_POWER


def alpha_model_db(lam_nm):
    """Attenuation stand-in (Rayleigh + floor) [dB/km]."""
    lam_um = np.asarray(lam_nm, dtype=np.float64) * 1e-3
    return 0.962 / lam_um ** 4 + 0.0233


def aeff_model_um2(lam_nm):
    """Effective area stand-in, linear 60 -> 95 um^2 over 1260 -> 1675 nm."""
    lam = np.asarray(lam_nm, dtype=np.float64)
    return 60.0 + 35.0 * (lam - 1260.0) / (1675.0 - 1260.0)


def dispersion_model(lam_nm, lam0_nm=1310.0, s0=0.09):
    """D, dD/dlambda and d2D/dlambda2 of D = S0/4 (l - l0^4/l^3).

    Returns (D [ps/nm/km], S [ps/nm^2/km], Sdot [ps/nm^3/km]).
    """
    lam = float(lam_nm)
    d = s0 / 4.0 * (lam - lam0_nm ** 4 / lam ** 3)
    s = s0 / 4.0 * (1.0 + 3.0 * lam0_nm ** 4 / lam ** 4)
    sdot = -3.0 * s0 * lam0_nm ** 4 / lam ** 5
    return d, s, sdot


def band_nf_db(lam_nm):
    lam = np.asarray(lam_nm, dtype=np.float64)
    idx = np.clip(np.searchsorted(BAND_EDGES_NM, lam, side="right") - 1, 0, 5)
    return np.asarray(BAND_NF_DB)[idx]


@dataclass
class Workload:
    """One transmission scenario: a channel plan, a fibre and a quadrature."""
    name: str
    f_THz: np.ndarray               # channel centre frequencies, sorted
    B_THz: np.ndarray               # channel bandwidths (symbol rate)
    P_W: np.ndarray                 # launch power per channel
    alpha_per_km: np.ndarray        # power attenuation per channel [1/km]
    lambda_nm: np.ndarray           # channel wavelengths
    aeff_um2: np.ndarray            # effective area per channel
    nf_dB: np.ndarray               # amplifier noise figure per channel
    n2_m2_per_W: float
    gamma_fixed: Optional[float]    # if set, gamma is this constant [1/W/km]
    L_km: float
    f_ref_THz: float                # reference frequency of the beta Taylor series
    D_ref: float                    # D, S, Sdot at the reference wavelength
    S_ref: float
    Sdot_ref: float
    Cr: float                       # Raman gain slope [1/(W km THz)]
    alpha_R_per_km: float           # attenuation used for L_eff and the z-grid
    G: int = 64                     # grid points per dimension per piece
    n_edges: int = 113              # z-grid edges (n_edges - 1 steps)
    eps_v1: float = 1e-10           # lower cut-off of upsilon1 (relative)
    cell_set: int = CELLS_SCI_XCI
    G_mci: int = 0                  # with CELLS_ALL: grid of the MCI cells (a, b != CUT); 0 = G
    snr_trx_dB: float = 0.0         # <= 0: no transceiver noise
    guard: Optional[np.ndarray] = None
    n_spans: int = 1                # identical spans, launch profile restored per span
    profile: int = 0                # power profile: 0 closed form (linear slope), 1 Raman ODE
    raman_max_THz: float = 15.0     # Raman ODE: triangular gain cut-off
    raman_photon: int = 1           # Raman ODE: photon-number ratio in the pump depletion
    ode_h_km: float = 0.25          # Raman ODE: largest RK4 step
    raman_scale: Optional[np.ndarray] = None   # Raman ODE: Aeff(f_ref) / Aeff(f_i); None -> 1

    @property
    def n_ch(self) -> int:
        return int(self.f_THz.shape[0])

    @property
    def lambda_ref_nm(self) -> float:
        return float(C_NM_PER_PS / self.f_ref_THz)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def n_edges_from_density(nbar_per_km: float, L_km: float) -> int:
    """N_M edges from the mean number of steps per km, (N_M - 1) = Nbar L."""
    return int(round(nbar_per_km * L_km)) + 1


def _plan(name, f, B, P, alpha, lam, aeff, nf, **kw) -> Workload:
    return Workload(name=name, f_THz=np.asarray(f, np.float64), B_THz=np.asarray(B, np.float64),
                    P_W=np.asarray(P, np.float64), alpha_per_km=np.asarray(alpha, np.float64),
                    lambda_nm=np.asarray(lam, np.float64), aeff_um2=np.asarray(aeff, np.float64),
                    nf_dB=np.asarray(nf, np.float64), **kw)


def tiny(G: int = 64, n_edges: int = 113, cell_set: int = CELLS_ALL) -> Workload:
    """5 x 96 GBaud at 100 GHz around 193.4 THz, 80 km, flat 0.2 dB/km,
    D = 17, S = 0.057 at the centre, gamma = 1.3, C_r = 0.028, 0 dBm/ch."""
    n = 5
    f = 193.4 + 0.1 * (np.arange(n) - 2)
    lam = nm_from_thz(f)
    a = np.full(n, db_per_km_to_per_km(0.2))
    return _plan("tiny-5ch", f, np.full(n, 0.096), dbm_to_w(np.zeros(n)), a, lam,
                 aeff_model_um2(lam), band_nf_db(lam), n2_m2_per_W=2.6e-20,
                 gamma_fixed=1.3, L_km=80.0, f_ref_THz=193.4, D_ref=17.0, S_ref=0.057,
                 Sdot_ref=0.0, Cr=0.028, alpha_R_per_km=float(a[0]), G=G,
                 n_edges=n_edges, cell_set=cell_set)


def _wdm_models(name, f, P, L_km, f_ref, Cr, G, n_edges, cell_set, **kw) -> Workload:
    lam = nm_from_thz(f)
    alpha = db_per_km_to_per_km(alpha_model_db(lam))
    d, s, sd = dispersion_model(C_NM_PER_PS / f_ref)
    alpha_r = float(db_per_km_to_per_km(alpha_model_db(C_NM_PER_PS / f_ref)))
    return _plan(name, f, np.full(f.shape, 0.096), P, alpha, lam, aeff_model_um2(lam),
                 band_nf_db(lam), n2_m2_per_W=2.6e-20, gamma_fixed=None, L_km=L_km,
                 f_ref_THz=f_ref, D_ref=d, S_ref=s, Sdot_ref=sd, Cr=Cr,
                 alpha_R_per_km=alpha_r, G=G, n_edges=n_edges, cell_set=cell_set, **kw)


def oband(G: int = 64, n_edges: int = 113, seed: int = 0, cell_set: int = CELLS_ALL) -> Workload:
    """41 x 96 GBaud at 100 GHz around 1310 nm, powers U[-2, 2] dBm (seed)."""
    n = 41
    fc = float(thz_from_nm(1310.0))
    f = fc + 0.1 * (np.arange(n) - 20)
    rng = np.random.default_rng(seed)
    P = dbm_to_w(rng.uniform(-2.0, 2.0, size=n))
    return _wdm_models("oband-41ch", f, P, 80.0, fc, 0.028, G, n_edges, cell_set)


UWB_F_LO = float(thz_from_nm(1675.0))    # 178.98 THz


def uwb_slots(n: int = 589) -> np.ndarray:
    """The 589 slot centres of the fully loaded 1260-1675 nm grid."""
    return UWB_F_LO + 0.05 + 0.1 * np.arange(n)


def uwb(G: int = 256, n_edges: int = 113, p_dbm: float = 1.0,
        cell_set: int = CELLS_SCI_XCI, n: int = 589) -> Workload:
    """589 x 96 GBaud over 1260-1675 nm, 80 km, flat p_dbm per channel."""
    f = uwb_slots(n)
    f_ref = 0.5 * (f[0] + f[-1])
    P = dbm_to_w(np.full(n, p_dbm))
    return _wdm_models("uwb-589ch", f, P, 80.0, f_ref, 0.028, G, n_edges, cell_set)


# Loaded channels per band (Table "Per band characteristics"), the guard-band
# gap between adjacent bands (Table "Simulation parameters") and the slot
# pitch of the 589-slot grid.
TABLE_BAND_COUNTS = {"O": 171, "E": 143, "S": 88, "C": 38, "L": 65, "U": 52}
GUARD_GAP_NM = 5.0
SLOT_THZ = 0.1


def guard_gap_slots(edge_nm: float, gap_nm: float = GUARD_GAP_NM, slot_thz: float = SLOT_THZ) -> int:
    """Whole slots inside a gap of `gap_nm` at wavelength `edge_nm`:
    floor(c * gap / lambda^2 / slot)."""
    return int(np.floor(C_NM_PER_PS * gap_nm / edge_nm ** 2 / slot_thz + 1e-9))


def guard_plan(n_slots: int = 589, counts=None, gap_nm: float = GUARD_GAP_NM):
    """Loaded slots, their band, and the guard set A of the 589-slot grid.

    Walking the grid from its low-frequency end (U band), each band takes the
    table's number of consecutive slots and every boundary between two bands
    leaves guard_gap_slots(boundary) slots empty.  Returns
    (loaded slot indices, band index per loaded slot (0 = O ... 5 = U),
    guard slot indices).
    """
    counts = TABLE_BAND_COUNTS if counts is None else counts
    loaded, band, guards = [], [], []
    pos = 0
    for b in range(5, -1, -1):                       # U, L, C, S, E, O: increasing frequency
        n = int(counts[BAND_NAMES[b]])
        loaded.extend(range(pos, pos + n))
        band.extend([b] * n)
        pos += n
        if b > 0:
            g = guard_gap_slots(BAND_EDGES_NM[b], gap_nm)
            guards.extend(range(pos, pos + g))
            pos += g
    if pos != n_slots:
        raise ValueError(f"band counts and guard gaps cover {pos} slots, not {n_slots}")
    return np.asarray(loaded), np.asarray(band), np.asarray(guards)


def uwb_guarded(G: int = 64, n_edges: int = 113, p_dbm: float = 0.0,
                cell_set: int = CELLS_SCI_XCI) -> Workload:
    """The 589-slot grid with the guard set A left empty: 557 loaded channels.
    An empty slot carries no power, so it adds nothing to the Raman
    normaliser, the integrand or the throughput: the plan simply omits it."""
    base = uwb(G=G, n_edges=n_edges, p_dbm=p_dbm, cell_set=cell_set)
    loaded, _, _ = guard_plan(base.n_ch)
    return subset_plan(base, loaded, "uwb-557ch-guarded")


def subset_plan(base: Workload, idx: np.ndarray, name: str) -> Workload:
    idx = np.sort(np.asarray(idx))
    sc = None if base.raman_scale is None else np.asarray(base.raman_scale)[idx]
    return base.with_(name=name, f_THz=base.f_THz[idx], B_THz=base.B_THz[idx],
                      P_W=base.P_W[idx], alpha_per_km=base.alpha_per_km[idx],
                      lambda_nm=base.lambda_nm[idx], aeff_um2=base.aeff_um2[idx],
                      nf_dB=base.nf_dB[idx], raman_scale=sc)


def raman(wl: Workload, raman_max_THz: float = 15.0, photon: int = 1, ode_h_km: float = 0.25,
          aeff_scaling: bool = True) -> Workload:
    """The same scenario with the Raman-ODE power profile: triangular gain
    C_r |df| up to raman_max_THz, scaled per channel by Aeff(f_ref)/Aeff(f_i)
    (Aeff at f_ref interpolated linearly in frequency over the plan)."""
    sc = None
    if aeff_scaling:
        a_ref = float(np.interp(wl.f_ref_THz, wl.f_THz, wl.aeff_um2))
        sc = a_ref / np.asarray(wl.aeff_um2, dtype=np.float64)
    return wl.with_(profile=1, raman_max_THz=float(raman_max_THz), raman_photon=int(photon),
                    ode_h_km=float(ode_h_km), raman_scale=sc)


@dataclass
class BatchedWorkload:
    plans: List[Workload]
    plan_of_profile: np.ndarray            # [n_prof] int
    P_W: List[np.ndarray] = field(default_factory=list)   # per profile


def batched(n_prof: int = 512, G: int = 64, n_edges: int = 113, seed_plans: int = 1,
            seed_powers: int = 2, sizes=(589, 295, 147)) -> BatchedWorkload:
    """Random launch-power profiles (dBm ~ N(1, 1.5^2) clipped to [-4, 5])
    over three channel plans: the 589-slot grid and two sorted random
    subsets of its slots.  Profile p uses plan p mod 3."""
    full = uwb(G=G, n_edges=n_edges)
    rng = np.random.default_rng(seed_plans)
    plans = []
    for s in sizes:
        if s == full.n_ch:
            plans.append(full.with_(name=f"uwb-{s}ch"))
        else:
            idx = rng.choice(full.n_ch, size=s, replace=False)
            plans.append(subset_plan(full, idx, f"uwb-subset-{s}ch"))
    rng_p = np.random.default_rng(seed_powers)
    plan_of = np.arange(n_prof) % len(plans)
    P = []
    for p in range(n_prof):
        n = plans[plan_of[p]].n_ch
        dbm = np.clip(rng_p.normal(1.0, 1.5, size=n), -4.0, 5.0)
        P.append(dbm_to_w(dbm))
    return BatchedWorkload(plans=plans, plan_of_profile=plan_of, P_W=P)


def gradient_fd_channels(n_ch: int = 589, k: int = 16, seed: int = 3) -> np.ndarray:
    """The channels on which the gradient is checked by finite differences."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_ch, size=k, replace=False))


def random_profile_dbm(n: int, seed: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=n)
