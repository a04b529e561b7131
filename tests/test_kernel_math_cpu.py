"""CPU checks of evaluation strategies the FP32 kernel relies on.

The kernel evaluates the z-sum of Eq. slow_vary in one of three exact-to-FP32
forms chosen per grid point; two of them rest on identities checked here
against the oracle's direct z-sum (independent code)."""
import numpy as np


def test_small_phi_second_order_expansion(orc):
    """For |phi| L <= 0.02: |S|^2 = M0^2 - phi^2 (M0 M2 - M1^2) with
    M_k = sum p dz z^k (M2 with z^2 + dz^2/12) to better than 1e-8."""
    L = 80.0
    ze = orc.zgrid(L, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(60):
        a, k = rng.uniform(0.02, 0.2), rng.uniform(-0.1, 0.1)
        p = np.exp(-a * zm + k * np.sin(zm / 7)) * rng.uniform(0.5, 2)
        w = p * dz
        M0, M1, M2 = w.sum(), (w * zm).sum(), (w * (zm ** 2 + dz ** 2 / 12)).sum()
        for x in rng.uniform(-0.02, 0.02, 10):
            ph = x / L
            exact = abs(orc.zsum(zm, dz, p, ph)) ** 2
            approx = M0 ** 2 - ph ** 2 * (M0 * M2 - M1 ** 2)
            worst = max(worst, abs(approx / exact - 1))
    assert worst < 1e-8


def test_telescoped_step_identity(orc):
    """dz sinc(phi dz/2) e^{j phi z_m} = (E_{m+1} - E_m)/(j phi), E = e^{j phi z}."""
    ze = orc.zgrid(80.0, 0.0571, 113)
    zm, dz = 0.5 * (ze[1:] + ze[:-1]), np.diff(ze)
    rng = np.random.default_rng(2)
    p = np.exp(-0.05 * zm) * (1 + 0.1 * rng.standard_normal(len(zm)))
    for ph in (0.7, 13.0, 812.5):
        E = np.exp(1j * ph * ze)
        tele = np.sum(p * (E[1:] - E[:-1])) / (1j * ph)
        assert abs(tele - orc.zsum(zm, dz, p, ph)) < 1e-10 * np.sum(np.abs(p * dz))


def test_sinc_polynomial_on_direct_range():
    """Even Taylor polynomial of sinc to x^10 on |x| <= pi/2: error < 4e-8."""
    x = np.linspace(-np.pi / 2, np.pi / 2, 20001)
    c = [1.0, -1 / 6, 1 / 120, -1 / 5040, 1 / 362880, -1 / 39916800]
    poly = sum(ck * x ** (2 * k) for k, ck in enumerate(c))
    ref = np.sinc(x / np.pi)
    assert np.max(np.abs(poly - ref)) < 4e-8
