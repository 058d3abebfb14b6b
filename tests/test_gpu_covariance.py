"""Covariance from mocks (Eq. covariance) through the C ABI against the FP64
oracle: plain matrices with ragged sizes, selections by index, the batch's
zeta array used in place, and the index check."""
import numpy as np
import pytest

from oracle import covariance as CV
from paper_2408_03036_gb300 import synth
from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu

# FP64 throughout; the two sides sum in different orders
TOL = 1e-12


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    return torch


def check(mean, cov, ref_mean, ref_cov):
    m, c = mean.cpu().numpy(), cov.cpu().numpy()
    assert np.abs(m - ref_mean).max() <= TOL * max(np.abs(ref_mean).max(), 1.0)
    assert np.abs(c - ref_cov).max() <= TOL * np.abs(ref_cov).max()
    assert np.array_equal(c, c.T)


@pytest.mark.parametrize("nm,nd", [(2, 1), (37, 333), (300, 64), (1000, 130), (16, 1)])
def test_plain_matrix(gpu, nm, nd):
    """Ragged sizes: mocks not a multiple of the 16-mock chunk, entries not a
    multiple of the 64-wide tile; correlated columns with a large common offset."""
    torch = gpu
    rng = np.random.default_rng(nm * 1000 + nd)
    a = rng.normal(size=(nd, nd)) / np.sqrt(nd)
    d = 1e3 + rng.normal(size=(nm, nd)) @ a.T
    mean, cov = tpcf.covariance(torch.from_numpy(d).cuda())
    tpcf.stream_status()
    check(mean, cov, *CV.sample_covariance(d))


def test_selection_by_index(gpu):
    torch = gpu
    rng = np.random.default_rng(3)
    d = rng.normal(size=(50, 24, 9, 9))
    idx = rng.choice(24 * 81, size=200, replace=False)
    mean, cov = tpcf.covariance(torch.from_numpy(d).cuda(), idx=idx)
    tpcf.stream_status()
    check(mean, cov, *CV.sample_covariance(d.reshape(50, -1)[:, idx]))


def test_batch_zeta_in_place(gpu, ora):
    """The batch's zeta array [n_mocks][n_mult][nb][nb] with the eta-selected
    data vector of six multipoles, against the oracle on the same numbers."""
    torch = gpu
    cfg = tpcf.Config(r_min=10.0, r_max=60.0, n_bins=8, l_max=3, Ls=(0, 2), periodic=True, box=250.0)
    sizes = [2000 + 37 * k for k in range(24)]
    xyz = np.concatenate([synth.poisson(n, 500 + k)[0] for k, n in enumerate(sizes)])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    z, _ = tpcf.estimate_3pcf_batched(cfg, xyz, None, off, want_counts=False)
    sel = [(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2), (3, 1, 2)]
    idx = tpcf.data_vector_index(cfg, sel, 2)
    assert idx.size == 6 * 21
    mean, cov = tpcf.covariance(z.contiguous(), idx=idx)
    tpcf.stream_status()
    zc = z.cpu().numpy().reshape(len(sizes), -1)[:, idx]
    check(mean, cov, *CV.sample_covariance(zc))


def test_index_outside_the_row_is_reported(gpu):
    """An out-of-range index is caught by the kernels' own bounds check (no load)
    and reported by the stream status; the row becomes NaN."""
    torch = gpu
    d = torch.ones((5, 10), dtype=torch.float64, device="cuda")
    idx = np.array([0, 3, 10], dtype=np.int64)
    mean, cov = tpcf.covariance(d, idx=idx)
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.stream_status()
    assert ei.value.code == -6
    assert torch.isnan(mean[2]).item() and not torch.isnan(mean[:2]).any().item()
    tpcf.stream_status()
