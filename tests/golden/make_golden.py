"""Writes tests/golden/oracle_tiny.json from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The stored values are a regression record of the oracle (not of the CUDA
path): tests/test_golden_paper.py checks that the oracle still reproduces
them, so a change to the oracle's arithmetic shows up as a diff of this file.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2401_18022_gb300 import workloads as W  # noqa: E402


def main():
    out = {"_source": "FP64 oracle, tiny 5-ch workload; written by tests/golden/make_golden.py"}
    for name, cells in (("all_cells", W.CELLS_ALL), ("sci_xci", W.CELLS_SCI_XCI)):
        wl = W.tiny(G=32, n_edges=57, cell_set=cells).with_(snr_trx_dB=20.0)
        r = oracle.evaluate(wl, threads=1)
        out[name] = {"G": 32, "n_edges": 57, "snr_trx_dB": 20.0,
                     "sigma": r["sigma"].tolist(), "eta": r["eta"].tolist(),
                     "snr": r["snr"].tolist(), "T_Tbps": r["T"]}
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
