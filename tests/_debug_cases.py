"""Workloads of the debug-build GPU test: every quadrature kernel and its
adjoint (closed form with the MCI grid, Raman-ODE profile, and the 589-channel
plan at a G large enough for the segmented series), and the forward of the
Raman-ODE profile with the MCI grid (no gradient there).  Each case is
(name, workload, with_gradient)."""


def cases(W):
    tiny = W.tiny(G=32, n_edges=41, cell_set=W.CELLS_ALL).with_(G_mci=8)
    return [("tiny_mci", tiny, True),
            ("raman", W.raman(W.tiny(G=24, n_edges=41, cell_set=W.CELLS_SCI_XCI)), True),
            ("raman_mci", W.raman(tiny, raman_max_THz=0.25), False),
            ("uwb_G160", W.uwb(G=160), True)]
