"""The slab-sharded form on the GPU: every rank's partials (tpcf_estimate_3pcf_partial)
computed one after the other on the one device, summed as the reduction would,
and finished (tpcf_estimate_3pcf_finish), against the unsplit estimate on the
GPU and against the FP64 oracle.  (Ranks that wait on one another are never
run on one GPU; these partial computations are independent.)"""
import numpy as np
import pytest

from paper_2408_03036_gb300 import shard, synth, tpcf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    return torch


def sharded(cfg, d, dw, r, rw, world, want_xi=True):
    """What estimate_3pcf_sharded computes over `world` ranks, the reduction done here."""
    dw = np.ones(d.shape[0], np.float32) if dw is None else dw
    w_d = float(dw.astype(np.float64).sum())
    w_r, weighted = 0.0, False
    if r is not None:
        w_r = float(rw.astype(np.float64).sum())
        weighted = bool(np.any(rw != 1.0))
    pf = pi = None
    for rank in range(world):
        pd, sd = shard.partition(cfg, d, rank, world)
        kw = dict(d_xyz=d[sd], d_w=dw[sd], dp_xyz=d[pd], dp_w=dw[pd], r_xyz=None, r_w=None, rp_xyz=None, rp_w=None)
        if r is not None:
            pr, sr = shard.partition(cfg, r, rank, world)
            kw.update(r_xyz=r[sr], r_w=rw[sr], rp_xyz=r[pr], rp_w=rw[pr])
        f, i = tpcf.estimate_3pcf_partial(cfg, w_d_total=w_d, w_r_total=w_r, weighted_randoms=weighted, **kw)
        pf = f if pf is None else pf + f
        pi = i if pi is None else pi + i
    return tpcf.estimate_3pcf_finish(cfg, pf, pi, w_d, w_r, r is not None, weighted, want_xi=want_xi)


def check(ora, res, cfg, d, dw, r, rw):
    full = tpcf.estimate_3pcf(cfg, d, dw, r, rw, want_xi=True)
    tpcf.stream_status()
    assert np.array_equal(res.pair_counts.cpu().numpy(), full.pair_counts.cpu().numpy())
    assert np.array_equal(res.triplet_counts.cpu().numpy(), full.triplet_counts.cpu().numpy())
    zs, zf = res.zeta.cpu().numpy(), full.zeta.cpu().numpy()
    # FP32 sums grouped differently (each shard's own cell grid and primaries): the FP32 bar
    for k in range(zf.shape[0]):
        assert np.abs(zs[k] - zf[k]).max() <= 1e-5 * np.abs(zf[k]).max(), k
    o = ora.Config(cfg.r_min, cfg.r_max, cfg.n_bins, cfg.l_max, cfg.Ls, cfg.periodic, cfg.box, los=cfg.los,
                   observer=cfg.observer)
    est = ora.estimate(o, d, dw, r, rw, want_xi=True)
    assert np.array_equal(res.triplet_counts.cpu().numpy(), est.trip_counts)
    for k in range(est.zeta.shape[0]):
        assert np.abs(zs[k] - est.zeta[k]).max() <= 1e-5 * np.abs(est.zeta[k]).max(), k
    xs, xo = res.xi.cpu().numpy(), est.extra["xi"]
    for e in range(xo.shape[0]):
        assert np.abs(xs[e] - xo[e]).max() <= 1e-5 * np.abs(xo[e]).max(), e


@pytest.mark.parametrize("world", [2, 3])
def test_periodic_analytic(gpu, ora, world):
    cfg = tpcf.Config(r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    d, dw = synth.poisson(20000, 1)
    check(ora, sharded(cfg, d, dw, None, None, world), cfg, d, dw, None, None)


@pytest.mark.parametrize("world", [2, 4])
def test_open_volume_unit_randoms(gpu, ora, world):
    cfg = tpcf.Config(r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False)
    d, dw = synth.lognormal(8000, 600.0, 3, mesh=64)
    r, rw = synth.randoms(24000, 4)
    check(ora, sharded(cfg, d, dw, r, rw, world), cfg, d, dw, r, rw)


def test_open_volume_weighted_randoms_varying_los(gpu, ora):
    cfg = tpcf.Config(r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False,
                      los="observer", observer=(-300.0, -180.0, -480.0))
    d, _ = synth.lognormal(8000, 600.0, 13, mesh=64)
    r, _ = synth.randoms(24000, 14)
    rng = np.random.default_rng(15)
    dw = rng.uniform(0.5, 1.5, d.shape[0]).astype(np.float32)
    rw = rng.uniform(0.2, 1.8, r.shape[0]).astype(np.float32)
    check(ora, sharded(cfg, d, dw, r, rw, 3), cfg, d, dw, r, rw)


def test_single_rank_wrapper_matches(gpu, ora):
    """estimate_3pcf_sharded with no process group (one rank) is the plain estimate."""
    cfg = tpcf.Config(r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False)
    d, dw = synth.lognormal(8000, 600.0, 3, mesh=64)
    r, rw = synth.randoms(24000, 4)
    res = shard.estimate_3pcf_sharded(cfg, d, dw, r, rw, want_xi=True)
    check(ora, res, cfg, d, dw, r, rw)
