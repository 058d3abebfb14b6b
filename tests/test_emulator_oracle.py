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


# ------------------------------------------------------------------------------
# Pins of the perturbation-theory kernels, the P(k) normalisation and the real-
# space 3PCF against results published independently of the model's own
# formulas (Bernardeau et al. 2002 for F2 / G2; Kaiser 1987 for Z1; the
# configuration-space tree-level 3PCF built from 1D Hankel transforms).

def _kernels(ka, kb, cab, ma, mb, mab, kab, b1, b2, f):
    """Z1(k_a) Z1(k_b) Z2(k_a, k_b) from the model's monomial split."""
    parts = T._kernel_parts(ka, kb, cab, ma, mb, mab, kab)
    return sum(c * p for c, p in zip(T.monomial_coeffs(b1, b2, f), parts))


def _f2_g2(ka, kb, c):
    """F2 and G2 isolated from the monomial parts: the b1^3 coefficient is
    Z1 Z1 (b1 part) x F2 = F2; with both LOS cosines 0 and a unit LOS cosine of
    k_a + k_b the b1^2 f coefficient is G2 alone."""
    z = np.zeros_like(np.asarray(c, dtype=float))
    kab = np.sqrt(ka ** 2 + kb ** 2 + 2 * ka * kb * c)
    parts = T._kernel_parts(ka, kb, c, z, z, z + 1.0, kab)
    return parts[T.MONOMIALS.index((3, 0, 0))], parts[T.MONOMIALS.index((2, 0, 1))]


def test_f2_g2_special_values():
    """F2(k, -k) = G2(k, -k) = 0 (momentum conservation) and F2 = G2 = 2 for two
    equal parallel wavevectors."""
    for k in (0.01, 0.1, 0.37):
        F, G = _f2_g2(np.array([k, k]), np.array([k, k]), np.array([-1.0, 1.0]))
        assert abs(F[0]) < 1e-14 and abs(G[0]) < 1e-14
        assert abs(F[1] - 2.0) < 1e-14 and abs(G[1] - 2.0) < 1e-14


def test_f2_g2_legendre_multipoles():
    """In the cosine mu of the angle between k1 and k2:
    F2 = 17/21 + (k1/k2 + k2/k1)/2 P1(mu) + 4/21 P2(mu),
    G2 = 13/21 + (k1/k2 + k2/k1)/2 P1(mu) + 8/21 P2(mu)."""
    from scipy.special import eval_legendre, roots_legendre
    x, wx = roots_legendre(16)
    for ka, kb in [(0.05, 0.05), (0.02, 0.11), (0.3, 0.07)]:
        F, G = _f2_g2(np.full(16, ka), np.full(16, kb), x)
        r = 0.5 * (ka / kb + kb / ka)
        for l, (cf, cg) in enumerate([(17 / 21, 13 / 21), (r, r), (4 / 21, 8 / 21)]):
            pf = (2 * l + 1) / 2 * np.sum(wx * F * eval_legendre(l, x))
            pg = (2 * l + 1) / 2 * np.sum(wx * G * eval_legendre(l, x))
            assert abs(pf - cf) < 1e-13 and abs(pg - cg) < 1e-13, (l, pf, pg)
        for l in range(3, 8):
            assert abs(np.sum(wx * F * eval_legendre(l, x))) < 1e-13


def test_kaiser_factor_of_z1():
    """Z1 = b1 + f mu^2: averaged over the LOS angle, Z1(mu)^2 gives the Kaiser
    factor b1^2 + 2 b1 f / 3 + f^2 / 5.  Z1(k_a) Z1(k_b) is twice the b2
    derivative of Z1 Z1 Z2 (Z2 carries b2 / 2)."""
    from scipy.special import roots_legendre
    x, wx = roots_legendre(12)
    k = np.full(12, 0.1)
    b1, f = 1.6, 0.7
    z1z1 = 2.0 * (_kernels(k, k, np.ones(12), x, x, x, 2 * k, b1, 1.0, f)
                  - _kernels(k, k, np.ones(12), x, x, x, 2 * k, b1, 0.0, f))
    assert abs(0.5 * np.sum(wx * z1z1) - (b1 ** 2 + 2 * b1 * f / 3 + f ** 2 / 5)) < 1e-13


def test_z2_squeezed_limit_is_the_redshift_space_shift():
    """As k2 -> 0 the long mode only displaces the short one; in redshift space
    the displacement has the extra f (Psi . n) n part, so
    Z2(k1, k2) -> (k1 / 2 k2) (k1_hat . k2_hat + f mu1 mu2) Z1(k1)
    (leading order in k2 / k1)."""
    rng = np.random.default_rng(11)
    b1, f = 1.9, 0.8
    for _ in range(10):
        v1, v2, n = rng.normal(size=(3, 3))
        n /= np.linalg.norm(n)
        k1 = 0.2 * v1 / np.linalg.norm(v1)
        k2 = 0.2e-6 * v2 / np.linalg.norm(v2)
        ka, kb = np.linalg.norm(k1), np.linalg.norm(k2)
        kab = np.linalg.norm(k1 + k2)
        c = k1 @ k2 / (ka * kb)
        m1, m2, m12 = k1 @ n / ka, k2 @ n / kb, (k1 + k2) @ n / kab
        a = [np.array([v]) for v in (ka, kb, c, m1, m2, m12, kab)]
        tot0 = _kernels(*a, b1, 0.0, f)[0]
        z1z1 = 2.0 * (_kernels(*a, b1, 1.0, f)[0] - tot0)
        z2 = tot0 / z1z1
        z1 = b1 + f * m1 ** 2
        lim = ka / (2 * kb) * (c + f * m1 * m2) * z1
        assert abs(z2 - lim) <= 1e-5 * abs(ka / (2 * kb) * z1), (z2, lim)


def test_power_spectrum_sigma8_is_one():
    """PowerNW is normalised to sigma(R = 8 Mpc/h) = 1 with the top-hat window:
    adaptive quadrature in linear k (the model itself uses a trapezoid in ln k)."""
    pk = T.PowerNW()
    R = 8.0

    def integrand(k):
        x = k * R
        wth = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3
        return k * k * float(pk(k)) * wth * wth / (2.0 * math.pi ** 2)

    edges = [1e-6, 1e-3, 0.01, 0.1, 0.5, 1.0, 2.0, 5.0, 20.0, 100.0, 1000.0]
    s2 = sum(quad(integrand, a, b, limit=500, epsrel=1e-11)[0] for a, b in zip(edges[:-1], edges[1:]))
    assert abs(math.sqrt(s2) - 1.0) < 1e-4


def _xi_tables(pk, r, k_hi=1.6, nk=16001):
    """xi_l^[n](r) = int dk k^(2+n) P(k) j_l(k r) / (2 pi^2) for (l, n) = (0, 0),
    (1, 1), (1, -1), (2, 0), on a fine k grid (P is Gaussian-damped)."""
    k = np.linspace(1e-6, k_hi, nk)
    P = pk(k)
    out = {}
    for (l, n) in ((0, 0), (1, 1), (1, -1), (2, 0)):
        f = (k ** (2 + n) * P)[None, :] * spherical_jn(l, np.outer(r, k)) / (2 * math.pi ** 2)
        out[(l, n)] = np.trapezoid(f, k, axis=1)
    return out


def test_real_space_isotropic_multipoles_against_configuration_space():
    """f = 0, alpha = 1, eps = 0: the model's zeta_{l l 0} (l = 0, 1, 2) against the
    tree-level 3PCF computed in configuration space.  Each vertex with legs a, b
    and opening cosine g contributes
        2 b1^3 [17/21 xi0(a) xi0(b) - 1/2 (xi1+(a) xi1-(b) + xi1-(a) xi1+(b)) g
                + 4/21 xi2(a) xi2(b) P2(g)] + b1^2 b2 xi0(a) xi0(b)
    (the Legendre form of F2 transformed leg by leg), summed over the three
    vertices of the triangle (r1, r2, r3 = |r2 - r1|), projected on P_l(mu) and
    bin-averaged with r^2 weights.  The model instead integrates the bispectrum
    multipoles of Eq. bisp with the 2D transform of Eq. TriRelBtoZ.  P is damped
    by exp(-(k / 0.25)^2) on both sides so that the model's k cut does not enter."""
    from scipy.interpolate import CubicSpline
    from scipy.special import eval_legendre, roots_legendre
    base = T.PowerNW()

    def pk(k):
        k = np.asarray(k, dtype=np.float64)
        return base(k) * np.exp(-(k / 0.25) ** 2)

    setup = T.ModelSetup(n_bins=6, r_min=20.0, r_max=110.0, k_max=0.6, n_log=40, dk=0.0125,
                         grid=T.AngularGrid(48, 4, 4))
    setup.pk = pk
    b1, b2 = 1.7, 0.6
    z = T.model_direct(setup, (0.0, b1, b2, 1.0, 1.0, 0.0))
    rg = np.linspace(0.0, 240.0, 961)
    X = {key: CubicSpline(rg, v) for key, v in _xi_tables(pk, rg).items()}

    def vertex(a, b, g):
        t = 2 * b1 ** 3 * (17 / 21 * X[0, 0](a) * X[0, 0](b)
                           - 0.5 * (X[1, 1](a) * X[1, -1](b) + X[1, -1](a) * X[1, 1](b)) * g
                           + 4 / 21 * X[2, 0](a) * X[2, 0](b) * eval_legendre(2, g))
        return t + b1 ** 2 * b2 * X[0, 0](a) * X[0, 0](b)

    xr, wr = roots_legendre(16)
    xm, wm = roots_legendre(64)
    e = setup.edges
    nb = len(e) - 1
    ref = np.zeros((3, nb, nb))
    for i in range(nb):
        r1 = 0.5 * (e[i + 1] - e[i]) * xr + 0.5 * (e[i + 1] + e[i])
        w1 = wr * r1 ** 2
        for j in range(nb):
            r2 = 0.5 * (e[j + 1] - e[j]) * xr + 0.5 * (e[j + 1] + e[j])
            w2 = wr * r2 ** 2
            R1, R2, MU = np.meshgrid(r1, r2, xm, indexing="ij")
            R3 = np.sqrt(np.maximum(R1 ** 2 + R2 ** 2 - 2 * R1 * R2 * MU, 1e-12))
            zz = vertex(R1, R2, MU) + vertex(R1, R3, (R1 - R2 * MU) / R3) + vertex(R2, R3, (R2 - R1 * MU) / R3)
            for l in range(3):
                c = (2 * l + 1) / 2 * np.einsum("abm,m->ab", zz, wm * eval_legendre(l, xm))
                ref[l, i, j] = np.einsum("ab,a,b->", c, w1, w2) / (w1.sum() * w2.sum())
    for l, tol in ((0, 2e-3), (1, 6e-3), (2, 2e-3)):
        q = T.MULTIPOLES.index((l, l, 0))
        err = np.abs(z[q] - ref[l]).max() / np.abs(ref[l]).max()
        assert err < tol, (l, err)
