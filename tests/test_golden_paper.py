"""Pins against values printed in the paper (tests/golden/paper_values.json)."""
import json
import os

import numpy as np
import pytest

from paper_2401_18022_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_gamma_at_zero_dispersion_wavelength(orc):
    g = GOLD["gamma_at_lambda_zd"]
    lam = g["lambda_nm"]
    assert orc.gamma(lam, 2.6e-20, float(W.aeff_model_um2(lam))) == pytest.approx(g["value"], rel=g["rel_tol"])


def test_step_density_definition():
    g = GOLD["steps_per_km_definition"]
    assert W.n_edges_from_density(g["nbar_per_km"], g["L_km"]) == g["n_edges"]


def test_band_noise_figures():
    g = GOLD["band_noise_figures_dB"]
    centres = {"O": 1310, "E": 1410, "S": 1495, "C": 1547, "L": 1595, "U": 1650}
    for band, lam in centres.items():
        assert W.band_nf_db(lam) == g[band]


def test_uwb_plan_matches_paper():
    g = GOLD["uwb_plan"]
    wl = W.uwb(G=8)
    assert wl.n_ch == g["n_ch"]
    assert np.allclose(np.diff(wl.f_THz), g["spacing_GHz"] / 1000.0)
    assert np.allclose(wl.B_THz, g["symbol_rate_GBd"] / 1000.0)
    lo, hi = W.nm_from_thz(wl.f_THz[-1] + 0.05), W.nm_from_thz(wl.f_THz[0] - 0.05)
    assert lo >= g["band_nm"][0] - 0.5 and hi <= g["band_nm"][1] + 0.5


def test_oracle_reproduces_its_stored_record(orc):
    """Regression record written by tests/golden/make_golden.py (oracle only)."""
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny.json")))
    for name, cells in (("all_cells", W.CELLS_ALL), ("sci_xci", W.CELLS_SCI_XCI)):
        wl = W.tiny(G=32, n_edges=57, cell_set=cells).with_(snr_trx_dB=20.0)
        r = orc.evaluate(wl, threads=1)
        np.testing.assert_allclose(r["sigma"], rec[name]["sigma"], rtol=1e-12)
        np.testing.assert_allclose(r["snr"], rec[name]["snr"], rtol=1e-12)
        assert r["T"] == pytest.approx(rec[name]["T_Tbps"], rel=1e-12)
