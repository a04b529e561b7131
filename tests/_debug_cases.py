"""Workloads of the debug-build GPU test: every quadrature kernel and its
adjoint (closed form with the MCI grid, Raman-ODE profile, and the 589-channel
plan at a G large enough for the segmented series)."""


def cases(W):
    tiny = W.tiny(G=32, n_edges=41, cell_set=W.CELLS_ALL).with_(G_mci=8)
    return [("tiny_mci", tiny),
            ("raman", W.raman(W.tiny(G=24, n_edges=41, cell_set=W.CELLS_SCI_XCI))),
            ("uwb_G160", W.uwb(G=160))]
