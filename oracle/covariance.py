"""Plain FP64 oracle of the covariance step (Sec. 4.3 of arXiv:2408.03036).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU leg are the only
callers.  Nothing here is shared with, imported by, or imports the CUDA path.

  * Eq. covariance: C_ij = sum_k (d_i^k - dbar_i)(d_j^k - dbar_j) / (N_m - 1),
    dbar the mean over the N_m mocks;
  * Eq. Hartlap: the inverse covariance is debiased by (N_m - N_d - 2)/(N_m - 1);
  * Eqs. Perc1, Perc: the factor m1 on the parameters' variance, with
    A = 2 / ((N_m - N_d - 1)(N_m - N_d - 4)) and
    B = (N_m - N_d - 2) / ((N_m - N_d - 1)(N_m - N_d - 4));
  * the data vector takes, per selected multipole, the triangles r1 <= r2
    whose bins differ by at least eta (|r1 - r2| >= eta * dr, Sec. 4.3), in the
    order multipole, b1, b2.
"""
from __future__ import annotations

import numpy as np


def sample_covariance(d):
    """(mean [N_d], C [N_d][N_d]) of d [N_m][N_d] by Eq. covariance."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    mean = d.sum(axis=0) / n
    x = d - mean
    return mean, (x.T @ x) / (n - 1)


def hartlap(n_mocks: int, n_dv: int) -> float:
    """Eq. Hartlap's factor on the inverse of the sample covariance."""
    return (n_mocks - n_dv - 2) / (n_mocks - 1)


def percival_m1(n_mocks: int, n_dv: int, n_params: int) -> float:
    """Eq. Perc1 with A and B of Eq. Perc."""
    q = (n_mocks - n_dv - 1) * (n_mocks - n_dv - 4)
    A = 2.0 / q
    B = (n_mocks - n_dv - 2) / q
    return (1.0 + B * (n_dv - n_params)) / (1.0 + A + B * (n_params + 1))


def data_vector_index(n_bins: int, mults: list, selected: list, eta: int):
    """Flat indices into a [n_mult][n_bins][n_bins] zeta array: for every
    selected (l1, l2, L) in order, every b1 <= b2 with b2 - b1 >= eta."""
    out = []
    for sel in selected:
        k = mults.index(tuple(sel))
        for b1 in range(n_bins):
            for b2 in range(b1, n_bins):
                if b2 - b1 >= eta:
                    out.append((k * n_bins + b1) * n_bins + b2)
    return np.array(out, dtype=np.int64)
