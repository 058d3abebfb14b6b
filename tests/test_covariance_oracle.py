"""Pins of the covariance oracle (Eqs. covariance, Hartlap, Perc1, Perc) against
exact rational arithmetic, a library routine, Wishart and inverse-Wishart
expectations and closed-form counts.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import covariance as CV


def test_sample_covariance_exact_rationals_and_numpy():
    rng = np.random.default_rng(1)
    d = rng.integers(-9, 10, size=(7, 4)).astype(np.float64)
    mean, C = CV.sample_covariance(d)
    n = d.shape[0]
    for i in range(4):
        mi = sum(Fraction(int(v)) for v in d[:, i]) / n
        assert mean[i] == float(mi)
        for j in range(4):
            mj = sum(Fraction(int(v)) for v in d[:, j]) / n
            cij = sum((Fraction(int(d[k, i])) - mi) * (Fraction(int(d[k, j])) - mj) for k in range(n)) / (n - 1)
            assert abs(C[i, j] - float(cij)) <= 1e-14 * max(1.0, abs(float(cij)))
    x = rng.normal(size=(50, 9))
    np.testing.assert_allclose(CV.sample_covariance(x)[1], np.cov(x, rowvar=False, ddof=1), rtol=1e-13, atol=1e-15)


def _true_cov(nd, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(nd, nd))
    return a @ a.T / nd + np.eye(nd)


def test_sample_covariance_is_unbiased_wishart_mean():
    """E[C_hat] = C for Gaussian mocks (the 1/(N_m - 1) normalisation)."""
    nd, nm, draws = 5, 8, 20000
    C = _true_cov(nd, 2)
    L = np.linalg.cholesky(C)
    rng = np.random.default_rng(3)
    acc = np.zeros((nd, nd))
    for _ in range(draws):
        acc += CV.sample_covariance(rng.normal(size=(nm, nd)) @ L.T)[1]
    est = acc / draws
    # a 1/N_m normalisation would be low by 1/8; the scatter of the mean is ~1 %
    assert np.abs(est - C).max() <= 0.03 * np.abs(C).max()


def test_hartlap_debiases_the_inverse_covariance():
    """Inverse-Wishart mean: E[C_hat^-1] = (N_m - 1)/(N_m - N_d - 2) C^-1, so the
    Hartlap factor times the mean inverse recovers C^-1."""
    nd, nm, draws = 6, 20, 20000
    C = _true_cov(nd, 4)
    L = np.linalg.cholesky(C)
    Ci = np.linalg.inv(C)
    rng = np.random.default_rng(5)
    acc = np.zeros((nd, nd))
    for _ in range(draws):
        acc += np.linalg.inv(CV.sample_covariance(rng.normal(size=(nm, nd)) @ L.T)[1])
    est = CV.hartlap(nm, nd) * acc / draws
    # the alternatives (N_m - N_d - 1) or (N_m - N_d) in the numerator move it by 8 % / 17 %
    assert np.abs(np.diag(est) / np.diag(Ci) - 1).max() < 0.02
    assert np.abs(est - Ci).max() <= 0.03 * np.abs(Ci).max()


@pytest.mark.parametrize("nd,npar", [(336, 6), (48, 4), (288, 7)])
def test_percival_m1_limits(nd, npar):
    """m1 -> 1 as N_m grows, with N_m (m1 - 1) -> N_d - 2 N_p - 1 (B ~ 1/N_m,
    A ~ 2/N_m^2)."""
    for nm in (10**7, 10**8):
        m1 = CV.percival_m1(nm, nd, npar)
        assert abs(nm * (m1 - 1.0) - (nd - 2 * npar - 1)) < 1e-3 * nd
    assert CV.percival_m1(3000, nd, npar) > 1.0


def test_data_vector_index_counts_and_order():
    mults = [(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2)]
    # 12 bins, eta = 3: (12 - 3)(12 - 3 + 1)/2 = 45 triangles per multipole
    idx = CV.data_vector_index(12, mults, [(0, 0, 0), (2, 0, 2)], 3)
    assert idx.size == 90
    b1, b2 = (idx % 144) // 12, idx % 12
    assert (b2 - b1 >= 3).all()
    assert set(idx[:45] // 144) == {0} and set(idx[45:] // 144) == {3}
    assert (np.diff(idx) > 0).all()
    assert CV.data_vector_index(5, mults, [(1, 1, 0)], 0).size == 15
