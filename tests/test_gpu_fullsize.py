"""Parity at the full size of the clustered-halo workload that the benchmark
times: a lognormal catalogue of 400,000 points (512^3 mesh) and 1,200,000
uniform randoms in an open cube of side 1000 Mpc/h, 20 bins 10-150 Mpc/h,
l_max = 4.  At this density every primary has about 2.3e4 neighbours, the
pair stage's queues overflow and drain several times per primary, and the
cell size is chosen automatically, none of which the small parity cases
reach.  The oracle cannot run every primary in seconds, so seeded samples of
primaries are compared one by one: their harmonic sums a_l^m[b] (Eq. alm) of
the D - R field against all 1.6 M secondaries, and the integer pair counts of
the random-only pass against all 1.2 M randoms.
"""
import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu

ND, NR, BOX, MESH = 400_000, 1_200_000, 1000.0, 512
TOL = 1e-5   # FP32 bar: per (l, m) block, max error / max |a| over sampled primaries and bins


@pytest.fixture(scope="module")
def field():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    d, dw = synth.lognormal(ND, BOX, 2, mesh=MESH)
    r, rw = synth.randoms(NR, 3)
    alpha = float(dw.astype(np.float64).sum() / rw.astype(np.float64).sum())
    x = np.concatenate([d, r])
    w = np.concatenate([dw, (-alpha * rw.astype(np.float64)).astype(np.float32)])
    return x, w, r


def test_harmonic_sums_of_sampled_primaries(field, ora):
    x, w, _ = field
    cfg = tpcf.Config(r_min=10.0, r_max=150.0, n_bins=20, l_max=4, Ls=(0, 2, 4), periodic=False, box=BOX)
    o = ora.Config(10.0, 150.0, 20, 4, (0, 2, 4), False, BOX)
    sel = np.sort(np.random.default_rng(101).choice(x.shape[0], size=2000, replace=False))
    grid = tpcf.Grid(cfg, x, w)
    alm, counts, _, _, _ = tpcf.accumulate_alm(grid, cfg, x[sel], w[sel], monopole_weight=-1.0)
    tpcf.stream_status()
    ro = ora.run(o, x, w.astype(np.float64), prim=sel, want_alm=True)
    got_c = counts.cpu().numpy()
    assert np.array_equal(got_c, ro.cnt)
    assert got_c.sum(1).mean() > 1.5e4          # the dense regime this test is for
    a = alm.cpu().numpy().astype(np.float64)
    for l in range(5):
        for m in range(l + 1):
            ref = ro.alm[:, :, l * l + l + m]
            parts = [(a[:, :, l * l], ref.real)] if m == 0 else \
                [(a[:, :, l * l + 2 * m - 1], ref.real), (a[:, :, l * l + 2 * m], ref.imag)]
            for got, want in parts:
                err = np.abs(got - want).max() / np.abs(want).max()
                assert err <= TOL, (l, m, err)
    grid.close()


def test_random_pair_counts_of_sampled_primaries(field, ora):
    _, _, r = field
    cfg = tpcf.Config(r_min=10.0, r_max=150.0, n_bins=20, l_max=4, Ls=(0, 2, 4), periodic=False, box=BOX)
    o = ora.Config(10.0, 150.0, 20, 0, (0,), False, BOX)
    sel = np.sort(np.random.default_rng(102).choice(r.shape[0], size=3000, replace=False))
    grid = tpcf.Grid(cfg, r)
    counts, pc = tpcf.pair_counts(grid, cfg, r[sel])
    tpcf.stream_status()
    ro = ora.run(o, r, np.ones(r.shape[0]), prim=sel, want_alm=True, l_max=0)
    got = counts.cpu().numpy()
    assert np.array_equal(got, ro.cnt)
    assert np.array_equal(pc.cpu().numpy(), got.sum(0).astype(np.int64))
    grid.close()
