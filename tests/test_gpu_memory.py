"""Device scratch kept in the library's own memory pool between calls, and
tpcf_trim_memory handing it back to the driver.

The per-primary harmonic sums a_l^m[b] of one estimate are the largest scratch
buffer (n_prim x n_bins x (l_max + 1)^2 floats).  With the pool they stay cached
after the call, so the next call reuses them without mapping new device memory;
after tpcf_trim_memory the device's free memory rises by at least their size.
The second estimate, served from the cached blocks, matches the first (counts
exactly, multipoles at the FP32 bar: the pair stage's FP32 sums may add in a
different order).
"""
import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    return torch


def test_scratch_cached_between_calls_and_trimmed(gpu):
    torch = gpu
    n = 400_000
    cfg = tpcf.Config(r_min=10.0, r_max=60.0, n_bins=20, l_max=4, Ls=(0, 2, 4), periodic=True, box=1000.0)
    xyz, w = synth.poisson(n, 31)
    alm_bytes = n * cfg.n_bins * (cfg.l_max + 1) ** 2 * 4
    d_x = torch.from_numpy(xyz.view(np.int32)).cuda()
    d_w = torch.as_tensor(w).cuda()
    torch.cuda.synchronize()
    tpcf.trim_memory()
    free0 = torch.cuda.mem_get_info()[0]
    r1 = tpcf.estimate_3pcf(cfg, d_x, d_w)
    tpcf.stream_status()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # the a_l^m block (and the grid's) stay in the pool after the call
    assert free0 - free1 >= 0.9 * alm_bytes, (free0, free1, alm_bytes)
    r2 = tpcf.estimate_3pcf(cfg, d_x, d_w)
    tpcf.stream_status()
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    # served from the cached blocks: no further growth beyond a few MB
    assert free1 - free2 <= 64 << 20, (free1, free2)
    tpcf.trim_memory()
    free3 = torch.cuda.mem_get_info()[0]
    assert free3 - free2 >= 0.9 * alm_bytes, (free2, free3, alm_bytes)
    assert np.array_equal(r1.pair_counts.cpu().numpy(), r2.pair_counts.cpu().numpy())
    assert np.array_equal(r1.triplet_counts.cpu().numpy(), r2.triplet_counts.cpu().numpy())
    z1, z2 = r1.zeta.cpu().numpy(), r2.zeta.cpu().numpy()
    for k in range(z1.shape[0]):
        den = np.abs(z1[k]).max()
        assert np.abs(z2[k] - z1[k]).max() <= TOL_FP32 * den
    # a third call after the trim maps fresh memory and still agrees
    r3 = tpcf.estimate_3pcf(cfg, d_x, d_w)
    tpcf.stream_status()
    assert np.array_equal(r1.pair_counts.cpu().numpy(), r3.pair_counts.cpu().numpy())
