"""Batches of periodic catalogues of uneven sizes (covariance mocks) and the
autotuner, through the C ABI, against one-catalogue estimates and the oracle.

A batch must give, for every mock, what the one-catalogue entry point gives for
that mock alone: counts bit-exact, multipoles within the FP32 bar (the two
paths sum each primary's pairs in different orders, so they agree to rounding,
not to the bit).
"""
import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    return torch


def per_mult_err(zg, zo):
    out = []
    for k in range(zo.shape[0]):
        den = np.abs(zo[k]).max()
        out.append(np.abs(zg[k] - zo[k]).max() / den if den > 0 else np.abs(zg[k] - zo[k]).max())
    return np.array(out)


def make_mocks(sizes, seed, box=500.0, clustered=()):
    """Concatenated mocks: Poisson, or lognormal for the indices in `clustered`."""
    xs, ws = [], []
    for k, n in enumerate(sizes):
        if n and k in clustered:
            x, w = synth.lognormal(int(n), box, seed + k, mesh=64)
        else:
            x, w = synth.poisson(int(n), seed + k)
        xs.append(x)
        ws.append(w)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(xs).reshape(-1, 3), np.concatenate(ws), off


def base_cfg(**kw):
    d = dict(r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), periodic=True, box=500.0)
    d.update(kw)
    return d


def check_against_single(gpu, cfg, xyz, w, off, zb, tb, tol):
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        if b - a < 2:
            assert not tb[k].any()
            continue
        res = tpcf.estimate_3pcf(cfg, xyz[a:b], w[a:b])
        tpcf.stream_status()
        assert np.array_equal(tb[k], res.triplet_counts.cpu().numpy()), k
        err = per_mult_err(zb[k], res.zeta.cpu().numpy())
        assert err.max() <= tol, (k, err)


def test_batch_matches_single_and_oracle(gpu, ora):
    sizes = [2500, 1200, 0, 3100, 1, 1800, 2200]
    xyz, w, off = make_mocks(sizes, seed=100, clustered=(3, 6))
    cfg = tpcf.Config(**base_cfg())
    zb, tb = tpcf.estimate_3pcf_batched(cfg, xyz, w, off)
    tpcf.stream_status()
    zb, tb = zb.cpu().numpy(), tb.cpu().numpy()
    check_against_single(gpu, cfg, xyz, w, off, zb, tb, TOL_FP32)
    ocfg = ora.Config(20.0, 120.0, 10, 4, (0, 2, 4), True, 500.0, True, "S_COEFF")
    for k in (0, 3):
        a, b = off[k], off[k + 1]
        est = ora.estimate(ocfg, xyz[a:b], w[a:b])
        assert np.array_equal(tb[k], est.trip_counts)
        err = per_mult_err(zb[k], est.zeta)
        assert err.max() <= TOL_FP32, (k, dict(zip(map(str, est.mults), err)))


def test_batch_tile_sizes_agree(gpu):
    """Tiles of 1, 3 and the automatic number of primaries (8 here), each within
    one mock, over mocks of uneven sizes (empty and one-point mocks included) and
    two groups: triplet counts identical, multipoles at the FP32 bar."""
    sizes = [1700, 0, 2300, 1, 900, 2600, 5]
    xyz, w, off = make_mocks(sizes, seed=300, clustered=(2,))
    ref = None
    for tp in (1, 3, 0):
        cfg = tpcf.Config(**base_cfg(tile_primaries=tp))
        b = tpcf.Batch(cfg, off, group_points=5000)
        z = b.zeta_buffer()
        t = gpu.zeros((len(sizes), cfg.n_bins, cfg.n_bins), dtype=gpu.int64, device="cuda")
        b.run(gpu.from_numpy(synth.as_int32_bits(xyz)).cuda(), gpu.from_numpy(w).cuda(), z, t)
        tpcf.stream_status()
        b.close()
        z, t = z.cpu().numpy(), t.cpu().numpy()
        if ref is None:
            ref = (z, t)
            continue
        assert np.array_equal(t, ref[1]), tp
        for k in range(len(sizes)):
            if sizes[k] >= 2:
                assert per_mult_err(z[k], ref[0][k]).max() <= TOL_FP32, (tp, k)


def test_batch_weighted_and_grouped(gpu):
    """Positive weights, and the batch split into several groups (persistent launches)."""
    sizes = [1500, 2600, 900, 2000, 1700]
    xyz, _, off = make_mocks(sizes, seed=300, clustered=(1,))
    w = np.random.default_rng(7).uniform(0.5, 2.0, size=xyz.shape[0]).astype(np.float32)
    cfg = tpcf.Config(**base_cfg(n_bins=8, r_min=15.0, r_max=95.0))
    torch = gpu
    dx = torch.from_numpy(synth.as_int32_bits(xyz)).cuda()
    dw = torch.from_numpy(w).cuda()
    b = tpcf.Batch(cfg, off, group_points=4000)
    n_groups, _ = b.info()
    assert n_groups >= 3
    z = b.zeta_buffer()
    t = torch.empty((len(sizes), cfg.n_bins, cfg.n_bins), dtype=torch.int64, device="cuda")
    b.run(dx, dw, z, t)
    tpcf.stream_status()
    zb, tb = z.cpu().numpy(), t.cpu().numpy()
    b.close()
    # one group holding everything gives the same numbers
    z1, t1 = tpcf.estimate_3pcf_batched(cfg, xyz, w, off)
    assert np.array_equal(t1.cpu().numpy(), tb)
    z1 = z1.cpu().numpy()
    for k in range(len(sizes)):
        assert per_mult_err(zb[k], z1[k]).max() <= TOL_FP32, k
    check_against_single(gpu, cfg, xyz, w, off, zb, tb, TOL_FP32)


def test_batch_graph_replay_reads_new_inputs(gpu):
    """A captured batch replays on whatever the same buffers hold at launch."""
    torch = gpu
    sizes = [1800, 2400, 1300]
    cfg = tpcf.Config(**base_cfg())
    xyz1, w1, off = make_mocks(sizes, seed=500)
    xyz2, w2, _ = make_mocks(sizes, seed=600, clustered=(0, 2))
    dx = torch.from_numpy(synth.as_int32_bits(xyz1)).cuda()
    dw = torch.from_numpy(w1).cuda()
    b = tpcf.Batch(cfg, off)
    z = b.zeta_buffer()
    t = torch.empty((len(sizes), cfg.n_bins, cfg.n_bins), dtype=torch.int64, device="cuda")
    b.run_graph(dx, dw, z, t)          # eager run + capture
    tpcf.stream_status()
    first = z.clone()
    dx.copy_(torch.from_numpy(synth.as_int32_bits(xyz2)))
    dw.copy_(torch.from_numpy(w2))
    b.run_graph(dx, dw, z, t)          # graph launch on the new contents
    tpcf.stream_status()
    ref, tref = tpcf.estimate_3pcf_batched(cfg, xyz2, w2, off)
    assert np.array_equal(t.cpu().numpy(), tref.cpu().numpy())
    # per-primary FP32 sums and FP64 atomics may add in another order: rounding-level agreement
    zg, zr = z.cpu().numpy(), ref.cpu().numpy()
    for k in range(len(sizes)):
        assert per_mult_err(zg[k], zr[k]).max() <= TOL_FP32, k
    dx_other = torch.from_numpy(synth.as_int32_bits(xyz1)).cuda()
    dw_other = torch.from_numpy(w1).cuda()
    b.run_graph(dx_other, dw_other, z, t)   # new pointers: eager run and a new capture
    tpcf.stream_status()
    zg, zf = z.cpu().numpy(), first.cpu().numpy()
    for k in range(len(sizes)):
        assert per_mult_err(zg[k], zf[k]).max() <= TOL_FP32, k
    b.close()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_batch_tensor_core_vs_oracle(gpu, ora, prec):
    sizes = [2600, 1900, 3000]
    xyz, w, off = make_mocks(sizes, seed=700, clustered=(1,))
    cfg = tpcf.Config(**base_cfg(precision=prec))
    zb, tb = tpcf.estimate_3pcf_batched(cfg, xyz, w, off)
    tpcf.stream_status()
    zb = zb.cpu().numpy()
    ocfg = ora.Config(20.0, 120.0, 10, 4, (0, 2, 4), True, 500.0, True, "S_COEFF")
    for k in range(len(sizes)):
        a, b = off[k], off[k + 1]
        est = ora.estimate(ocfg, xyz[a:b], w[a:b])
        assert np.array_equal(tb[k].cpu().numpy(), est.trip_counts)
        err = per_mult_err(zb[k], est.zeta)
        assert err.max() <= TOL_MIXED, (k, err)


def test_batch_rejects_bad_requests(gpu):
    cfg = tpcf.Config(**base_cfg())
    with pytest.raises(tpcf.TpcfError):
        tpcf.Batch(cfg, [0, 10, 5])                       # decreasing offsets
    with pytest.raises(tpcf.TpcfError):
        tpcf.Batch(tpcf.Config(**base_cfg(periodic=False)), [0, 10])
    with pytest.raises(tpcf.TpcfError):
        tpcf.Batch(cfg, [0, 100, 300], group_points=150)  # one mock above the group cap


def test_autotune_returns_a_valid_faster_choice(gpu, ora):
    xyz, w = synth.lognormal(20000, 500.0, 11, mesh=64)
    cfg = tpcf.Config(**base_cfg())
    tuned = tpcf.autotune(cfg, xyz, w)
    assert tuned.cell_div in (2, 3, 4, 5, 6)
    assert tuned.tile_primaries in (1, 2, 4)
    assert tuned.chunk in (12288, 15360, 24576)
    res = tpcf.estimate_3pcf(tuned, xyz[:4000], w[:4000])
    tpcf.stream_status()
    ocfg = ora.Config(20.0, 120.0, 10, 4, (0, 2, 4), True, 500.0, True, "S_COEFF")
    est = ora.estimate(ocfg, xyz[:4000], w[:4000])
    assert np.array_equal(res.triplet_counts.cpu().numpy(), est.trip_counts)
    assert per_mult_err(res.zeta.cpu().numpy(), est.zeta).max() <= TOL_FP32


def test_per_mock_status_isolates_a_bad_mock(gpu):
    """A non-finite weight in one mock and a one-point mock: the call succeeds, the
    per-mock status names exactly those two mocks (TPCF_ERR_DATA, TPCF_ERR_ARG),
    and every other mock's multipoles equal their one-catalogue estimates."""
    cfg = tpcf.Config(**base_cfg())
    sizes = [2000, 1500, 1, 2500, 1800]
    xyz, w, off = make_mocks(sizes, seed=300)
    w = w.copy()
    w[off[3] + 17] = np.nan
    zb, tb, st = tpcf.estimate_3pcf_batched(cfg, xyz, w, off, want_status=True)
    tpcf.stream_status()   # no device-wide error was latched
    assert list(st) == [0, 0, -1, -6, 0], st
    zb, tb = zb.cpu().numpy(), tb.cpu().numpy()
    assert not np.isfinite(zb[3]).all()
    good = [0, 1, 4]
    for k in good:
        a, b = off[k], off[k + 1]
        res = tpcf.estimate_3pcf(cfg, xyz[a:b], w[a:b])
        tpcf.stream_status()
        assert np.array_equal(tb[k], res.triplet_counts.cpu().numpy()), k
        assert per_mult_err(zb[k], res.zeta.cpu().numpy()).max() <= TOL_FP32, k
    # the batch object reports the same after a graph run
    import torch
    bt = tpcf.Batch(cfg, off)
    dx = torch.from_numpy(synth.as_int32_bits(xyz)).cuda()
    dw = torch.from_numpy(w).cuda()
    z = bt.zeta_buffer()
    bt.run_graph(dx, dw, z)
    bt.run_graph(dx, dw, z)
    assert list(bt.status()) == [0, 0, -1, -6, 0]
    tpcf.stream_status()
    bt.close()
