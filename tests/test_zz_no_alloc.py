"""The coupling entry point that allocates nothing (tpcf_couple_multipoles_static).

It serves callers that may not allocate GPU memory while they run; it uses a
fixed scratch block inside the library instead.  Checked here through the C ABI
against tpcf_couple_multipoles on the same inputs, on two calls in a row (the
second call finds the block holding the first call's contents and must clear
what has to start at zero).  This file sorts last so a run that stops at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32 path's parity tolerance (per block, normalised by the block's max)


def _block_err(a, b, lmax):
    worst = 0.0
    for m in range(lmax + 1):
        for l1 in range(m, lmax + 1):
            for l2 in range(m, lmax + 1):
                den = np.abs(b[m, l1, l2]).max()
                if den > 0:
                    worst = max(worst, np.abs(a[m, l1, l2] - b[m, l1, l2]).max() / den)
    return worst


def test_static_scratch_coupling_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    cases = [
        (tpcf.Config(r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0), 8000, 1),
        (tpcf.Config(r_min=10.0, r_max=70.0, n_bins=12, l_max=2, Ls=(0, 2), box=300.0), 5000, 2),
    ]
    for cfg, n, seed in cases:
        xyz, w = synth.poisson(n, seed)
        grid = tpcf.Grid(cfg, xyz, w)
        alm, counts, diag, wsp, _ = tpcf.accumulate_alm(grid, cfg, monopole_weight=float(n))
        _, pw, _ = grid.points()
        ref_nnn, ref_tc = tpcf.couple_multipoles(cfg, alm, pw, counts, diag, wsp)
        for _ in range(2):   # two calls in a row on the shared block
            nnn, tc = tpcf.couple_multipoles_static(cfg, alm, pw, counts, diag, wsp)
            tpcf.stream_status()
            assert np.array_equal(tc.cpu().numpy(), ref_tc.cpu().numpy())
            assert _block_err(nnn.cpu().numpy(), ref_nnn.cpu().numpy(), cfg.l_max) <= TOL
        grid.close()


def test_static_scratch_rejects_oversize_requests():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = tpcf.Config(r_min=5.0, r_max=155.0, n_bins=30, l_max=6, Ls=(0, 2), box=500.0)
    dev = torch.device("cuda")
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    alm = torch.zeros((4, nb, L1 * L1), dtype=torch.float32, device=dev)
    diag = torch.zeros((L1 * (L1 + 1) // 2, nb), dtype=torch.float64, device=dev)
    wsp = torch.zeros((L1, nb), dtype=torch.float64, device=dev)
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.couple_multipoles_static(cfg, alm, None, None, diag, wsp)
    assert ei.value.code == -1 and "static scratch" in str(ei.value)


def test_static_scratch_coupling_matches_the_oracle(ora):
    """NNN^m and the triplet counts of the static-scratch coupling against the FP64
    oracle's (periodic, analytic randoms): FP32 bar per (m, l1, l2) block, counts
    exact."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    cfg = tpcf.Config(r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    o = ora.Config(20.0, 120.0, 10, 4, (0, 2, 4), True, 500.0)
    xyz, w = synth.poisson(6000, 21)
    grid = tpcf.Grid(cfg, xyz, w)
    alm, counts, diag, wsp, _ = tpcf.accumulate_alm(grid, cfg, monopole_weight=float(w.astype(np.float64).sum()))
    _, pw, _ = grid.points()
    nnn, tc = tpcf.couple_multipoles_static(cfg, alm, pw, counts, diag, wsp)
    tpcf.stream_status()
    grid.close()
    est = ora.estimate(o, xyz, w)
    assert np.array_equal(tc.cpu().numpy(), est.trip_counts)
    ng, L = nnn.cpu().numpy(), cfg.l_max
    worst = 0.0
    for m in range(L + 1):
        for l1 in range(m, L + 1):
            for l2 in range(m, L + 1):
                if (l1 + l2) % 2:
                    continue
                ref = est.nnn[m + L, l1, l2].real
                den = np.abs(ref).max()
                if den > 0:
                    worst = max(worst, np.abs(ng[m, l1, l2] - ref).max() / den)
    assert worst <= TOL, worst
