"""Pins of the oracle's full anisotropic edge correction (N = zeta R solved on
the real, l1 + l2 even coefficients) against things other than its own
coupling code: products of functions evaluated pointwise on a quadrature grid
(scipy Y), the isotropic limit (bin-wise division by RRR_00^0), the identity
N = R, and the Gaunt coefficients against exact sympy values.  CPU only."""
import math

import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from tests import bruteforce as bf


def _grid(n_mu, n_phi):
    x, w = np.polynomial.legendre.leggauss(n_mu)
    th = np.arccos(x)
    ph = 2 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    W = np.outer(w, np.full(n_phi, 2 * math.pi / n_phi))
    return T.ravel(), P.ravel(), W.ravel()


def _basis(l1, l2, m, T, P):
    """B^m_{l1 l2}(r1, r2) = Y_l1^m(r1) Y_l2^m*(r2) on the product grid [n1, n2]."""
    return np.outer(bf.sph_y(l1, m, T, P), np.conj(bf.sph_y(l2, m, T, P)))


def _function(coef, modes, T, P):
    """sum over modes of c (B^m + B^-m) (once for m = 0): a real-coefficient,
    +-m symmetric function of the two directions."""
    F = 0
    for c, (l1, l2, m) in zip(coef, modes):
        F = F + c * _basis(l1, l2, m, T, P)
        if m > 0:
            F = F + c * _basis(l1, l2, -m, T, P)
    return F


@pytest.mark.parametrize("L,seed", [(2, 1), (3, 2)])
def test_solution_recovers_zeta_from_pointwise_products(ora, L, seed):
    """zeta and R given by coefficients; N = zeta R formed pointwise on a grid that
    integrates the products exactly; projecting N and solving returns zeta_hat."""
    rng = np.random.default_rng(seed)
    modes = ora.edge_modes(L)
    zhat = rng.normal(size=len(modes))
    rc = 0.15 * rng.normal(size=len(modes))
    rc[modes.index((0, 0, 0))] = 3.0
    T, P, W = _grid(2 * L + 2, 4 * L + 4)
    N = _function(4 * math.pi * zhat, modes, T, P) * _function(rc, modes, T, P)
    WW = np.outer(W, W)
    proj = np.array([np.sum(WW * N * np.conj(_basis(l1, l2, m, T, P))) for (l1, l2, m) in modes])
    assert np.abs(proj.imag).max() < 1e-10 * np.abs(proj).max()
    rr = np.zeros((2 * L + 1, L + 1, L + 1))
    for c, (l1, l2, m) in zip(rc, modes):
        rr[m + L, l1, l2] = rr[-m + L, l1, l2] = c
    _, M = ora.edge_matrix(rr, L)
    np.testing.assert_allclose(np.linalg.solve(M, proj.real), zhat, rtol=1e-9, atol=1e-9)


def test_isotropic_randoms_reduce_to_binwise_division(ora):
    L, nb = 3, 2
    rng = np.random.default_rng(4)
    nnn = rng.normal(size=(2 * L + 1, L + 1, L + 1, nb, nb)) + 0j
    rrr = np.zeros_like(nnn)
    rrr[L, 0, 0] = rng.uniform(1, 2, size=(nb, nb))
    z = ora.edge_correct(nnn, rrr, L)
    for (l1, l2, m) in ora.edge_modes(L):
        np.testing.assert_allclose(z[m + L, l1, l2].real, nnn[m + L, l1, l2].real / rrr[L, 0, 0].real, rtol=1e-12)


def test_n_equal_r_gives_unit_zeta(ora):
    """zeta = 1 for every direction pair: zeta_hat^0_00 = 1, all other modes 0."""
    L, nb = 4, 2
    rng = np.random.default_rng(6)
    rrr = np.zeros((2 * L + 1, L + 1, L + 1, nb, nb), dtype=complex)
    for (l1, l2, m) in ora.edge_modes(L):
        v = rng.normal(size=(nb, nb)) * (0.05 if (l1, l2, m) != (0, 0, 0) else 0.0) + (2.0 if (l1, l2, m) == (0, 0, 0) else 0.0)
        rrr[m + L, l1, l2] = rrr[-m + L, l1, l2] = v
    z = ora.edge_correct(rrr, rrr, L)
    for (l1, l2, m) in ora.edge_modes(L):
        np.testing.assert_allclose(z[m + L, l1, l2].real, 1.0 if (l1, l2, m) == (0, 0, 0) else 0.0, atol=1e-12)


def test_gaunt_vs_exact_sympy(ora):
    from sympy.physics.wigner import gaunt as sg
    rng = np.random.default_rng(7)
    for _ in range(40):
        l1, l2, l3 = rng.integers(0, 5, size=3)
        m1 = int(rng.integers(-l1, l1 + 1))
        m2 = int(rng.integers(-l2, l2 + 1))
        m3 = m1 + m2
        # sympy's gaunt is int Y Y Y; Y_l3^(m3)* = (-1)^m3 Y_l3^-m3
        ref = float(sg(int(l1), int(l2), int(l3), m1, m2, -m3)) * (-1) ** m3 if abs(m3) <= l3 else 0.0
        assert abs(ora.gaunt(int(l1), m1, int(l2), m2, int(l3)) - ref) < 1e-13


def test_full_estimate_matches_binwise_for_nearly_isotropic_randoms(ora):
    """Randoms filling a periodic box (no edges): RRR is isotropic up to shot
    noise, so the full correction moves the multipoles only by that noise."""
    cfg = ora.Config(10.0, 40.0, 3, 2, (0, 2), True, 150.0)
    d, dw = synth.lognormal(1500, 150.0, 3, mesh=32)
    r, rw = synth.randoms(6000, 4)
    full = ora.estimate(cfg, d, dw, r, rw, edge="full", nthreads=4)
    binw = ora.estimate(cfg, d, dw, r, rw, nthreads=4)
    rf = full.extra["rrr_full"]
    aniso = max(np.abs(rf[m + 2, l1, l2]).max() for (l1, l2, m) in ora.edge_modes(2) if (l1, l2, m) != (0, 0, 0))
    assert aniso < 0.05 * np.abs(rf[2, 0, 0]).max()
    assert np.abs(full.zeta[0] - binw.zeta[0]).max() <= 0.1 * np.abs(binw.zeta[0]).max()
