"""Pins of the oracle's separate grid for multi-channel-interference cells
(cells (a, b) of the CUT's plane with neither F_a nor F_b in the CUT's
channel; App. A's integral over the whole band includes them).

  * G_mci = G reproduces the single-grid result exactly;
  * the MCI part (ALL minus SCI+XCI) converges as G_mci grows, towards the
    value of a fine grid, at the midpoint rule's rate;
  * at zero dispersion (O band at lambda0) MCI is a large part of eta, far
    from it a small one (the paper's reason for including it).
"""
import numpy as np

from paper_2401_18022_gb300 import workloads as W


def test_gmci_equal_to_g_is_the_single_grid(orc):
    wl = W.tiny(G=12, n_edges=25, cell_set=W.CELLS_ALL)
    np.testing.assert_array_equal(orc.sigma(wl.with_(G_mci=12)), orc.sigma(wl))


def test_mci_part_converges_with_its_grid(orc):
    wl = W.oband(G=16, n_edges=25, cell_set=W.CELLS_ALL)
    wl = wl.with_(f_THz=wl.f_THz[14:27], B_THz=wl.B_THz[14:27], P_W=wl.P_W[14:27],
                  alpha_per_km=wl.alpha_per_km[14:27], lambda_nm=wl.lambda_nm[14:27],
                  aeff_um2=wl.aeff_um2[14:27], nf_dB=wl.nf_dB[14:27])
    cuts = [0, 6, 12]
    sx = orc.sigma(wl.with_(cell_set=W.CELLS_SCI_XCI), cuts=cuts)
    ref = orc.sigma(wl.with_(G_mci=48), cuts=cuts) - sx
    errs = []
    for g in (4, 8, 16):
        mci = orc.sigma(wl.with_(G_mci=g), cuts=cuts) - sx
        errs.append(np.max(np.abs(mci / ref - 1)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3
    assert np.all(ref > 0)


def test_mci_share_large_at_zero_dispersion(orc):
    """41-ch O band centred on lambda0: MCI adds a large share of eta; the
    same plan moved to 1550 nm (D ~ 17 ps/nm/km) gets a small share."""
    wl = W.oband(G=12, n_edges=25, cell_set=W.CELLS_ALL).with_(G_mci=6)
    cuts = [20]
    allc = orc.sigma(wl, cuts=cuts)
    sx = orc.sigma(wl.with_(cell_set=W.CELLS_SCI_XCI), cuts=cuts)
    share0 = 1 - sx / allc
    far = W.subset_plan(W.uwb(G=12, n_edges=25), np.arange(41) + 180, "c-41").with_(cell_set=W.CELLS_ALL,
                                                                                    G_mci=6)
    allf = orc.sigma(far, cuts=cuts)
    sxf = orc.sigma(far.with_(cell_set=W.CELLS_SCI_XCI), cuts=cuts)
    share1 = 1 - sxf / allf
    assert share0[0] > 0.3 and share1[0] < 0.1 and share0[0] > 4 * share1[0]



def test_gmci_with_raman_ode_profile(orc):
    """With the Raman-ODE profile (R2) the separate grid follows the same grid
    rule: G_mci = G reproduces the single grid exactly, and on the O-band
    subset at lambda0 (MCI 30-66 % of eta) the MCI part converges at the
    midpoint rule's rate as G_mci grows."""
    tiny = W.raman(W.tiny(G=12, n_edges=25, cell_set=W.CELLS_ALL).with_(Cr=0.4), raman_max_THz=0.25)
    np.testing.assert_array_equal(orc.sigma(tiny.with_(G_mci=12)), orc.sigma(tiny))
    wl = W.oband(G=16, n_edges=25, cell_set=W.CELLS_ALL)
    wl = wl.with_(f_THz=wl.f_THz[14:27], B_THz=wl.B_THz[14:27], P_W=wl.P_W[14:27],
                  alpha_per_km=wl.alpha_per_km[14:27], lambda_nm=wl.lambda_nm[14:27],
                  aeff_um2=wl.aeff_um2[14:27], nf_dB=wl.nf_dB[14:27])
    wl = W.raman(wl.with_(Cr=0.4), raman_max_THz=0.5)
    cuts = [0, 6, 12]
    sx = orc.sigma(wl.with_(cell_set=W.CELLS_SCI_XCI), cuts=cuts)
    ref = orc.sigma(wl.with_(G_mci=48), cuts=cuts) - sx
    errs = [np.max(np.abs((orc.sigma(wl.with_(G_mci=g), cuts=cuts) - sx) / ref - 1)) for g in (4, 8, 16)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2] and errs[2] < 5e-3
    assert np.all(ref > 0.25 * (ref + sx))
