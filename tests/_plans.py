"""Channel plans shared by GPU tests (synthetic, seeded where random)."""
import numpy as np

from paper_2401_18022_gb300 import workloads as W


def wide_cut_plan(G):
    """A 300 GHz channel between five narrow 25 GBaud channels at 30 GHz
    spacing on each side: the wide channel's SCI pieces have six F_c
    candidates, and in the lower quadrant its own channel (where the
    small-phase points fall) is the sixth, beyond the adjoint's contracted
    candidates, so those points take the per-step forms."""
    base = W.tiny(G=G, n_edges=41)
    f = np.concatenate([193.115 + 0.03 * np.arange(5), [193.40], 193.565 + 0.03 * np.arange(5)])
    B = np.array([0.025] * 5 + [0.30] + [0.025] * 5)
    n = len(f)
    lam = W.nm_from_thz(f)
    return base.with_(f_THz=f, B_THz=B, P_W=W.dbm_to_w(np.where(B > 0.1, 5.0, -2.0)),
                      alpha_per_km=np.full(n, base.alpha_per_km[0]), lambda_nm=lam,
                      aeff_um2=np.full(n, base.aeff_um2[0]), nf_dB=np.full(n, base.nf_dB[0]),
                      cell_set=W.CELLS_SCI_XCI)
