"""Pins of the plain tree-level model (the emulator's reference) and of the FP64
network reference, against closed forms, exact symmetries and finite
differences.  CPU only."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import spherical_jn

from oracle import mlp_oracle as MO
from oracle import treelevel as T


@pytest.fixture(scope="module")
def small():
    """A coarse but complete setup (fast on a CPU)."""
    return T.ModelSetup(n_bins=6, r_min=20.0, r_max=110.0, k_max=0.6, n_log=20, dk=0.025,
                        grid=T.AngularGrid(24, 6, 6))


def per_mult(z, ref):
    return max(np.abs(z[q] - ref[q]).max() / max(np.abs(ref[q]).max(), 1e-300) for q in range(ref.shape[0]))


def test_s_basis_projection_is_identity():
    """Projecting S_{l1 l2 L} itself gives coefficient 1 on itself and 0 elsewhere
    (orthogonality normalisation of Eq. TSHbasis)."""
    g = T.AngularGrid(48, 8, 8).build(T.MULTIPOLES)
    ct, cb = g.k2hat[:, 2], g.n[:, 2]
    ph = np.arctan2(g.n[:, 1], g.n[:, 0])
    M = np.array([g.proj @ T.s_basis(l1, l2, L, 0 * ct, 0 * ct, np.arccos(ct), 0 * ct, np.arccos(cb), ph)
                  for (l1, l2, L) in T.MULTIPOLES])
    assert np.abs(M - np.eye(len(T.MULTIPOLES))).max() < 1e-12


def test_s_ll0_is_legendre_of_the_opening_angle():
    """S_{l l 0}(k1, k2, n) = P_l(k1 . k2) for any n (addition theorem)."""
    rng = np.random.default_rng(1)
    th1, ph1, th2, ph2, thn, phn = rng.uniform(0, math.pi, 6)
    from scipy.special import eval_legendre
    c12 = math.cos(th1) * math.cos(th2) + math.sin(th1) * math.sin(th2) * math.cos(ph1 - ph2)
    for l in range(5):
        s = T.s_basis(l, l, 0, th1, ph1, th2, ph2, thn, phn)
        assert abs(s - eval_legendre(l, c12)) < 1e-12


def test_monomial_split_matches_direct_kernels():
    """The 11 monomial coefficient arrays reproduce Z1 Z1 Z2 evaluated directly."""
    rng = np.random.default_rng(2)
    n = 50
    ka, kb = rng.uniform(0.01, 0.5, n), rng.uniform(0.01, 0.5, n)
    cab = rng.uniform(-1, 1, n)
    ma, mb = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    kab = np.sqrt(ka ** 2 + kb ** 2 + 2 * ka * kb * cab)
    mab = (ka * ma + kb * mb) / kab
    parts = T._kernel_parts(ka, kb, cab, ma, mb, mab, kab)
    b1, b2, f = 1.7, -0.4, 0.73
    got = sum(c * p for c, p in zip(T.monomial_coeffs(b1, b2, f), parts))
    F2 = 5 / 7 + 0.5 * cab * (ka / kb + kb / ka) + 2 / 7 * cab ** 2
    G2 = 3 / 7 + 0.5 * cab * (ka / kb + kb / ka) + 4 / 7 * cab ** 2
    Z1a, Z1b = b1 + f * ma ** 2, b1 + f * mb ** 2
    Z2 = (b1 * F2 + f * mab ** 2 * G2 + 0.5 * f * mab * kab * (ma / ka * Z1b + mb / kb * Z1a) + 0.5 * b2)
    np.testing.assert_allclose(got, Z1a * Z1b * Z2, rtol=1e-13)


def test_separable_legendre_bispectrum_gives_products_of_1d_hankel(small):
    """B = P(k1) P(k2) P_l(k1 . k2) has the single coefficient B_{l l 0} = P1 P2, so
    zeta_{l l 0}(r1, r2) = (-1)^l xi_l(r1) xi_l(r2) with the bin-averaged 1D
    transforms xi_l(r) = int dk k^2 P j_l(k r) / (2 pi^2) (Eq. TriRelBtoZ)."""
    from scipy.special import eval_legendre
    pk = small.pk

    def bispec(k1v, k2v, n):
        k1, k2 = np.linalg.norm(k1v, axis=-1), np.linalg.norm(k2v, axis=-1)
        c = np.sum(k1v * k2v, axis=-1) / (k1 * k2)
        return np.stack([pk(k1) * pk(k2) * eval_legendre(l, c) for l in range(3)])

    B = T.triposh_monomials(small.k, small.grid, pk, bispec=bispec)
    z = T.hankel_2d(B, small.k, small.edges, T.MULTIPOLES)
    e = small.edges
    for l in range(3):
        xi = []
        for b in range(len(e) - 1):
            # bin average of the 1D transform, by adaptive quadrature in r and k
            def integrand(r):
                return quad(lambda k: k * k * pk(k) * spherical_jn(l, k * r) / (2 * math.pi ** 2),
                            1e-4, 0.6, limit=400)[0] * r * r
            xi.append(quad(integrand, e[b], e[b + 1], limit=50)[0] * 3 / (e[b + 1] ** 3 - e[b] ** 3))
        xi = np.array(xi)
        q = T.MULTIPOLES.index((l, l, 0))
        ref = (-1) ** l * np.outer(xi, xi)
        assert np.abs(z[l, q] - ref).max() / np.abs(ref).max() < 2e-3, l
        for q2, m in enumerate(T.MULTIPOLES):
            if m != (l, l, 0):
                assert np.abs(z[l, q2]).max() < 1e-8 * np.abs(ref).max()


def test_real_space_has_no_anisotropic_multipoles(small):
    """f = 0, alpha = 1, eps = 0: the bispectrum does not depend on n, so every
    L > 0 multipole vanishes."""
    z = T.model_direct(small, (0.0, 2.0, 0.5, 0.8, 1.0, 0.0))
    iso = max(np.abs(z[q]).max() for q, m in enumerate(T.MULTIPOLES) if m[2] == 0)
    for q, m in enumerate(T.MULTIPOLES):
        if m[2] > 0:
            assert np.abs(z[q]).max() < 1e-10 * iso, m


def test_exchange_symmetry(small):
    """zeta_{l1 l2 L}(r1, r2) = zeta_{l2 l1 L}(r2, r1)."""
    z = T.model_direct(small, (0.8, 2.2, 0.3, 0.8, 1.02, 0.02))
    scale = np.abs(z).max()
    for q, (l1, l2, L) in enumerate(T.MULTIPOLES):
        q2 = T.MULTIPOLES.index((l2, l1, L))
        assert np.abs(z[q] - z[q2].T).max() < 1e-10 * scale


def test_ap_map_matches_eqs_k_prime_mu_prime():
    """The vector map reproduces the printed k' and mu' (Eqs. k_prime, mu_prime)."""
    rng = np.random.default_rng(5)
    kv = rng.normal(size=(20, 3))
    n = rng.normal(size=(20, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    for alpha, eps in [(1.03, 0.02), (0.96, -0.04)]:
        kp = T.ap_map(kv, n, alpha, eps)
        k = np.linalg.norm(kv, axis=-1)
        mu = np.sum(kv * n, axis=-1) / k
        fac = np.sqrt(1 + mu ** 2 * ((1 + eps) ** -6 - 1))
        np.testing.assert_allclose(np.linalg.norm(kp, axis=-1), (1 + eps) / alpha * k * fac, rtol=1e-13)
        np.testing.assert_allclose(np.sum(kp * n, axis=-1) / np.linalg.norm(kp, axis=-1),
                                   mu * (1 + eps) ** -3 / fac, rtol=1e-12, atol=1e-14)


def test_isotropic_dilation_rescales_wavenumbers():
    """With eps = 0, B_obs(k; alpha) = alpha^-6 B(k / alpha): the TripoSH
    coefficients at alpha equal those at alpha = 1 on the scaled wavenumbers."""
    pk = T.PowerNW()
    g = T.AngularGrid(24, 6, 6).build(T.MULTIPOLES)
    k = np.array([0.02, 0.05, 0.11, 0.3])
    a = 1.04
    B = T.triposh_monomials(k, g, pk, a, 0.0)
    ref = T.triposh_monomials(k / a, g, pk, 1.0, 0.0) / a ** 6
    assert np.abs(B - ref).max() <= 1e-12 * np.abs(ref).max()


def test_template_decomposition_is_exact(small):
    """The model is sigma8^4 times a polynomial in (b1, b2, f): the template sum at
    one (alpha, eps) reproduces direct evaluations at other bias values."""
    Tm = T.templates(small, 0.98, -0.01)
    for th in [(0.6, 1.2, -0.5, 0.7), (0.95, 2.8, 1.5, 0.95)]:
        f, b1, b2, s8 = th
        direct = T.model_direct(small, th + (0.98, -0.01))
        via = s8 ** 4 * np.tensordot(T.monomial_coeffs(b1, b2, f), Tm, axes=(0, 0))
        assert np.abs(direct - via).max() <= 1e-12 * np.abs(direct).max()


def test_bicubic_template_interpolation(small):
    """Catmull-Rom interpolation on the (alpha, eps) grid against direct evaluation
    off the nodes."""
    al = np.linspace(0.94, 1.06, 7)
    ep = np.linspace(-0.06, 0.06, 7)
    tm = T.TemplateModel.build(small, al, ep)
    th = np.array([0.8, 2.0, 0.4, 0.85, 1.013, 0.017])
    got = tm(th)[0]
    ref = T.flatten_upper(T.model_direct(small, th))
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-3


def test_mlp_reference_gradient_by_finite_differences():
    rng = np.random.default_rng(4)
    widths = [6, 9, 7, 5]
    n_p = sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(3))
    p = rng.normal(0, 0.5, n_p)
    x = rng.uniform(-2, 3, (13, 6))
    y = rng.normal(0, 1, (13, 5))
    lo, hi = np.full(6, -2.0), np.full(6, 3.0)
    mu, sd = rng.normal(0, 0.1, 5), rng.uniform(0.5, 2, 5)
    _, g = MO.loss_and_grad(p, widths, x, y, lo, hi, mu, sd, rounding=False)
    h = 1e-6
    for i in rng.choice(n_p, 25, replace=False):
        e = np.zeros(n_p)
        e[i] = h
        fp = MO.loss_and_grad(p + e, widths, x, y, lo, hi, mu, sd, rounding=False)[0]
        fm = MO.loss_and_grad(p - e, widths, x, y, lo, hi, mu, sd, rounding=False)[0]
        assert abs((fp - fm) / (2 * h) - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_bf16_rounding_ties_to_even():
    vals = np.array([1.0, 1.00390625, 1.01171875, 1.0 + 2 ** -9, -3.5, 65504.0], dtype=np.float32)
    got = MO.bf16_round(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1.0) wins
    assert got[0] == 1.0 and got[1] == 1.0
    assert got[2] == 1.015625      # 1 + 3 * 2^-8 ties to 1 + 2^-6 (even)
    assert got[3] == 1.0
    assert got[4] == -3.5 and got[5] == 65536.0
