"""CUDA path vs the FP64 oracle, element by element, on the same seeded inputs.

Bar (the benchmark spec's tolerance): per multipole,
    max_{b1,b2} |zeta_gpu - zeta_oracle| / max_{b1,b2} |zeta_oracle| <= 1e-5
for the FP32 path, and pair / triplet counts bit-exact.
"""
import math

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


def cfg_pair(ora, **kw):
    """The same configuration for the CUDA path and the oracle."""
    g = tpcf.Config(**kw)
    o = ora.Config(kw["r_min"], kw["r_max"], kw["n_bins"], kw["l_max"], kw.get("Ls", (0, 2, 4)),
                   kw.get("periodic", True), kw.get("box", 500.0), kw.get("remove_self", True),
                   kw.get("convention", "S_COEFF"), kw.get("los", "z"), kw.get("observer", (0.0, 0.0, 0.0)))
    return g, o


def per_mult_err(zg, zo):
    out = []
    for k in range(zo.shape[0]):
        den = np.abs(zo[k]).max()
        num = np.abs(zg[k] - zo[k]).max()
        out.append(num / den if den > 0 else num)
    return np.array(out)


def nnn_err(ng, no, lmax):
    """Worst normalised error over the (m, l1, l2) blocks with l1 + l2 even."""
    worst = 0.0
    for m in range(lmax + 1):
        for l1 in range(m, lmax + 1):
            for l2 in range(m, lmax + 1):
                if (l1 + l2) % 2:
                    continue
                ref = no[m + lmax, l1, l2].real
                den = np.abs(ref).max()
                if den == 0:
                    continue
                worst = max(worst, np.abs(ng[m, l1, l2] - ref).max() / den)
    return worst


def compare(gpu, gcfg, ocfg, ora, d_xyz, d_w, r_xyz=None, r_w=None, tol=TOL_FP32, xi=False, rrr_exact=True):
    """zeta, NNN, the counts and RRR against the oracle; with xi also the even 2PCF
    multipoles (per multipole, max error over bins / max |xi| over bins <= tol).
    RRR is bit-for-bit up to FP64 rounding for analytic and unit-weight randoms
    (integer triplet counts); for weighted randoms it comes from FP32 harmonic
    sums and is held to tol."""
    res = tpcf.estimate_3pcf(gcfg, d_xyz, d_w, r_xyz, r_w, want_xi=xi)
    tpcf.stream_status()
    est = ora.estimate(ocfg, d_xyz, d_w, r_xyz, r_w, want_xi=xi)
    assert res.mults == est.mults
    zg = res.zeta.cpu().numpy()
    err = per_mult_err(zg, est.zeta)
    assert np.array_equal(res.pair_counts.cpu().numpy(), est.pair_counts)
    assert np.array_equal(res.triplet_counts.cpu().numpy(), est.trip_counts)
    rg = res.rrr.cpu().numpy()
    if rrr_exact:
        assert np.allclose(rg, est.rrr, rtol=1e-12, atol=0)
    else:
        assert np.abs(rg - est.rrr).max() <= tol * np.abs(est.rrr).max()
    assert err.max() <= tol, dict(zip(map(str, est.mults), err))
    assert nnn_err(res.nnn.cpu().numpy(), est.nnn, gcfg.l_max) <= tol
    if xi:
        xg, xo = res.xi.cpu().numpy(), est.extra["xi"]
        assert xg.shape == xo.shape
        for e in range(xo.shape[0]):
            assert np.abs(xg[e] - xo[e]).max() <= tol * np.abs(xo[e]).max(), (2 * e, xg[e], xo[e])
    return err


def test_small_periodic(gpu, ora):
    g, o = cfg_pair(ora, r_min=10.0, r_max=60.0, n_bins=5, l_max=2, Ls=(0, 2), box=250.0)
    xyz, w = synth.poisson(3000, 5)
    compare(gpu, g, o, ora, xyz, w, xi=True)


def test_config1_poisson_periodic(gpu, ora):
    """Plain estimator workload: N = 20,000 uniform points, periodic L = 500,
    10 bins 20-120, l <= 4, L in {0, 2, 4}, analytic randoms."""
    g, o = cfg_pair(ora, r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    xyz, w = synth.poisson(20000, 1)
    compare(gpu, g, o, ora, xyz, w, xi=True)


def test_paper_eq_convention(gpu, ora):
    g, o = cfg_pair(ora, r_min=20.0, r_max=120.0, n_bins=6, l_max=3, Ls=(0, 2), box=500.0,
                    convention="PAPER_EQ")
    xyz, w = synth.poisson(8000, 2)
    compare(gpu, g, o, ora, xyz, w)


def test_open_volume_data_minus_randoms(gpu, ora):
    """Clustered lognormal data with 3x uniform randoms in an open (non-periodic) cube."""
    g, o = cfg_pair(ora, r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False)
    d, dw = synth.lognormal(8000, 600.0, 3, mesh=64)
    r, rw = synth.randoms(24000, 4)
    compare(gpu, g, o, ora, d, dw, r, rw, xi=True)


def test_open_volume_weighted_randoms(gpu, ora):
    """Randoms with non-unit weights: RRR_00^0 and the 2PCF normaliser come from the
    weighted l = 0 sums of a random-only harmonic pass, not from integer counts."""
    g, o = cfg_pair(ora, r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False)
    d, _ = synth.lognormal(8000, 600.0, 13, mesh=64)
    r, _ = synth.randoms(24000, 14)
    rng = np.random.default_rng(15)
    dw = rng.uniform(0.5, 1.5, d.shape[0]).astype(np.float32)
    rw = rng.uniform(0.2, 1.8, r.shape[0]).astype(np.float32)
    compare(gpu, g, o, ora, d, dw, r, rw, xi=True, rrr_exact=False)


def test_xi_lmax6_open(gpu, ora):
    """Four even 2PCF multipoles (l_max = 6) with unit-weight randoms given as an
    array of ones (the integer-count normaliser)."""
    g, o = cfg_pair(ora, r_min=5.0, r_max=80.0, n_bins=15, l_max=6, Ls=(0, 2), box=500.0, periodic=False)
    d, dw = synth.lognormal(5000, 500.0, 23, mesh=64)
    r, rw = synth.randoms(10000, 24)
    compare(gpu, g, o, ora, d, dw, r, rw, xi=True)


@pytest.mark.parametrize("tile,chunk,div", [(1, 512, 1), (3, 768, 2), (8, 2048, 3), (2, 4096, 4)])
def test_schedules_agree(gpu, ora, tile, chunk, div):
    """Every tiling / staging / cell-size choice gives the same answer."""
    g, o = cfg_pair(ora, r_min=15.0, r_max=90.0, n_bins=8, l_max=4, Ls=(0, 2, 4), box=400.0,
                    tile_primaries=tile, chunk=chunk, cell_div=div)
    xyz, w = synth.poisson(9001, 6)   # ragged: not a multiple of any tile
    compare(gpu, g, o, ora, xyz, w)


@pytest.mark.parametrize("tile,chunk,div", [(1, 512, 2), (3, 768, 3), (6, 2048, 4)])
def test_open_volume_random_counts_with_the_harmonic_pass(gpu, ora, tile, chunk, div):
    """Unit randoms in an open volume: their pair counts per random primary (for
    RRR_00^0 and the 2PCF normaliser) are taken by the D - R harmonic pass from the
    records of negative weight, under every tile / queue / cell schedule; RRR must
    equal the oracle's integer-triplet value."""
    g, o = cfg_pair(ora, r_min=12.0, r_max=90.0, n_bins=7, l_max=2, Ls=(0, 2), box=420.0, periodic=False,
                    tile_primaries=tile, chunk=chunk, cell_div=div)
    d, dw = synth.lognormal(5001, 420.0, 41, mesh=64)   # ragged sizes
    r, rw = synth.randoms(12007, 42)
    dw = np.random.default_rng(43).uniform(0.0, 2.0, d.shape[0]).astype(np.float32)
    dw[::7] = 0.0                                       # zero weights are data too
    compare(gpu, g, o, ora, d, dw, r, rw, xi=True)


def test_open_volume_signed_data_weights_unit_randoms(gpu, ora):
    """Data weights of both signs with unit randoms: the randoms are then not the only
    records of negative weight, and their counts come from the separate count pass."""
    g, o = cfg_pair(ora, r_min=12.0, r_max=90.0, n_bins=7, l_max=2, Ls=(0, 2), box=500.0, periodic=False)
    d, _ = synth.lognormal(5000, 500.0, 44, mesh=64)
    r, rw = synth.randoms(12000, 45)
    dw = np.random.default_rng(46).uniform(0.5, 2.0, d.shape[0]).astype(np.float32)
    dw[::5] *= -1
    compare(gpu, g, o, ora, d, dw, r, rw, xi=True)


def test_signed_weights_and_clustering(gpu, ora):
    """Non-unit signed weights and strong clustering (many points per cell)."""
    g, o = cfg_pair(ora, r_min=5.0, r_max=60.0, n_bins=11, l_max=3, Ls=(0, 2), box=300.0)
    d, _ = synth.lognormal(6000, 300.0, 8, mesh=64, sigma_g=1.6)
    rng = np.random.default_rng(9)
    w = rng.uniform(0.5, 2.0, size=d.shape[0]).astype(np.float32)
    w[::4] *= -1
    compare(gpu, g, o, ora, d, w)


def test_lmax6_thirty_bins(gpu, ora):
    """l <= 6, 30 bins 5-155 on a Poisson catalogue in a periodic L = 500 box
    (the precision workload's shape at 6000 points)."""
    g, o = cfg_pair(ora, r_min=5.0, r_max=155.0, n_bins=30, l_max=6, Ls=(0, 2, 4, 6), box=500.0)
    xyz, w = synth.poisson(6000, 1)
    compare(gpu, g, o, ora, xyz, w)


@pytest.mark.parametrize("prec,tol", [("fp32", TOL_FP32), ("bf16x3", 1e-4), ("tf32x3", 1e-4)])
def test_precision_workload_full(gpu, ora, prec, tol):
    """The precision workload at full size: Poisson N = 20,000 in a periodic
    L = 500 box, 30 bins 5-155 Mpc/h, l <= 6, L in {0, 2, 4, 6} (58 multipoles).
    Every multipole within 1e-5 of the FP64 oracle on the FP32 path (1e-4 with
    the split-precision tensor-core coupling); pair and triplet counts exact.
    The innermost bins hold about 0.6 pairs per primary, so their diagonal
    b1 = b2 entries are almost all j = k term: this is where the removal of
    degenerate triangles must cancel to the last bits."""
    g, o = cfg_pair(ora, r_min=5.0, r_max=155.0, n_bins=30, l_max=6, Ls=(0, 2, 4, 6), box=500.0)
    g.precision = prec
    xyz, w = synth.poisson(20000, 1)
    err = compare(gpu, g, o, ora, xyz, w, tol=tol)
    print(prec, "max per-multipole error %.2e, median %.2e" % (err.max(), np.median(err)))


def test_single_point_and_tiny(gpu, ora):
    g, o = cfg_pair(ora, r_min=10.0, r_max=60.0, n_bins=5, l_max=2, Ls=(0, 2), box=250.0)
    for n in (1, 2, 7):
        xyz, w = synth.poisson(n, 40 + n)
        res = tpcf.estimate_3pcf(g, xyz, w)
        tpcf.stream_status()
        est = ora.estimate(o, xyz, w)
        assert np.array_equal(res.pair_counts.cpu().numpy(), est.pair_counts)
        assert np.array_equal(res.triplet_counts.cpu().numpy(), est.trip_counts)
        zg = res.zeta.cpu().numpy()
        if n == 1:   # no pairs and W - 1 = 0: 0/0 on both sides
            assert np.isnan(zg).all() and np.isnan(est.zeta).all()
        else:
            # a handful of points: several multipoles are exact cancellations (zero in
            # FP64), so the error is measured against the largest multipole value
            assert np.abs(zg - est.zeta).max() <= TOL_FP32 * np.abs(est.zeta).max()


def test_per_primary_alm_explicit_primaries(gpu, ora):
    """tpcf_accumulate_alm with explicit primaries reproduces the oracle's a_l^m
    per primary (real and imaginary parts, m >= 0)."""
    import torch
    g, o = cfg_pair(ora, r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    xyz, w = synth.poisson(20000, 1)
    prim = np.arange(0, 20000, 97)
    grid = tpcf.Grid(g, xyz, w)
    alm, counts, diag, wsp, pc = tpcf.accumulate_alm(grid, g, xyz[prim], w[prim], monopole_weight=-1.0)
    tpcf.stream_status()
    ro = ora.run(o, xyz, w, prim=prim, want_alm=True)
    assert np.array_equal(counts.cpu().numpy(), ro.cnt)
    a = alm.cpu().numpy().astype(np.float64)
    L = 4
    for l in range(L + 1):
        for m in range(l + 1):
            ref = ro.alm[:, :, l * l + l + m]
            if m == 0:
                got = a[:, :, l * l]
                assert np.abs(got - ref.real).max() <= 2e-6 * max(1.0, np.abs(ref).max())
            else:
                gre, gim = a[:, :, l * l + 2 * m - 1], a[:, :, l * l + 2 * m]
                assert np.abs(gre - ref.real).max() <= 2e-6 * max(1.0, np.abs(ref).max())
                assert np.abs(gim - ref.imag).max() <= 2e-6 * max(1.0, np.abs(ref).max())
    grid.close()
    del torch


def test_host_entry_point_matches_device(gpu, ora):
    g, o = cfg_pair(ora, r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    xyz, w = synth.poisson(20000, 1)
    a = tpcf.estimate_3pcf(g, xyz, w)
    b = tpcf.estimate_3pcf_host(g, xyz, w)
    assert np.array_equal(a.triplet_counts.cpu().numpy(), b.triplet_counts)
    # same inputs, same kernels; only the order of floating-point atomics differs
    assert per_mult_err(b.zeta, a.zeta.cpu().numpy()).max() <= 1e-6


def test_bad_weights_are_reported(gpu):
    g = tpcf.Config(r_min=10.0, r_max=60.0, n_bins=5, l_max=2, Ls=(0, 2), box=250.0)
    xyz, w = synth.poisson(500, 3)
    w = w.copy()
    w[7] = np.nan
    tpcf.estimate_3pcf(g, xyz, w)
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.stream_status()
    assert ei.value.code == -6
    tpcf.stream_status()   # latch cleared


TOL_MIXED = 1e-4   # split-precision tensor-core coupling (bf16x3 / tf32x3) vs the FP64 oracle


@pytest.mark.parametrize("prec,tol", [("bf16x3", TOL_MIXED), ("tf32x3", TOL_MIXED)])
def test_tensor_core_coupling_config1(gpu, ora, prec, tol):
    """tcgen05 Gram (split precision, FP32 accumulate in tensor memory, FP64 flush)
    on the plain-estimator workload."""
    g, o = cfg_pair(ora, r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    g.precision = prec
    xyz, w = synth.poisson(20000, 1)
    compare(gpu, g, o, ora, xyz, w, tol=tol)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tensor_core_coupling_open_volume_and_two_row_tiles(gpu, ora, prec):
    """Signed D - R primary weights, and an m = 0 block of 30 x 7 = 210 rows
    (two 128-row tiles) at l_max = 6."""
    g, o = cfg_pair(ora, r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False)
    g.precision = prec
    d, dw = synth.lognormal(8000, 600.0, 3, mesh=64)
    r, rw = synth.randoms(24000, 4)
    compare(gpu, g, o, ora, d, dw, r, rw, tol=TOL_MIXED)
    g, o = cfg_pair(ora, r_min=5.0, r_max=155.0, n_bins=30, l_max=6, Ls=(0, 2, 4, 6), box=500.0)
    g.precision = prec
    xyz, w = synth.poisson(6000, 1)
    compare(gpu, g, o, ora, xyz, w, tol=TOL_MIXED)


@pytest.mark.parametrize("nb,lmax", [(32, 4), (25, 4), (7, 6), (1, 0), (3, 2), (32, 6), (13, 5)])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tensor_core_tile_plans_match_fp32_gram(gpu, prec, nb, lmax):
    """Every packing of the m blocks into tensor-core tiles and CTA groups (blocks
    above 128 rows, shared tiles, several groups) against the FP32 Gram on the
    same per-primary sums, block by block."""
    import dataclasses
    import torch
    cfg = tpcf.Config(r_min=10.0, r_max=90.0, n_bins=nb, l_max=lmax, Ls=(0,), box=400.0)
    xyz, w = synth.lognormal(5000, 400.0, 21, mesh=64)
    wt = np.random.default_rng(3).uniform(-1.0, 2.0, size=w.shape[0]).astype(np.float32)
    grid = tpcf.Grid(cfg, xyz, wt)
    alm, counts, diag, wsp, _ = tpcf.accumulate_alm(grid, cfg, prim_xyz=xyz, prim_w=wt)
    pw = torch.from_numpy(wt).cuda()
    ref, tref = tpcf.couple_multipoles(cfg, alm, pw, counts, diag, wsp)
    got, tgot = tpcf.couple_multipoles(dataclasses.replace(cfg, precision=prec), alm, pw, counts, diag, wsp)
    tpcf.stream_status()
    assert torch.equal(tref, tgot)
    ref, got = ref.cpu().numpy(), got.cpu().numpy()
    worst = 0.0
    for m in range(lmax + 1):
        for l1 in range(m, lmax + 1):
            for l2 in range(m, lmax + 1):
                den = np.abs(ref[m, l1, l2]).max()
                if den > 0:
                    worst = max(worst, np.abs(got[m, l1, l2] - ref[m, l1, l2]).max() / den)
    assert worst <= 1e-4, worst
    grid.close()


# ------------------------------------------------------- full edge correction
def compare_full_edge(gpu, gcfg, ocfg, ora, d, dw, r, rw, tol=TOL_FP32):
    """zeta, RRR^m_{l1 l2}, NNN and xi of the full anisotropic edge correction
    against the oracle.  RRR is held to tol of its largest (l = 0) block."""
    res = tpcf.estimate_3pcf_full_edge(gcfg, d, dw, r, rw, want_xi=True)
    tpcf.stream_status()
    est = ora.estimate(ocfg, d, dw, r, rw, want_xi=True, edge="full")
    L = gcfg.l_max
    err = per_mult_err(res.zeta.cpu().numpy(), est.zeta)
    assert err.max() <= tol, dict(zip(map(str, est.mults), err))
    rg, ro = res.rrr.cpu().numpy(), est.extra["rrr_full"]
    scale = np.abs(ro[L, 0, 0].real).max()
    for (l1, l2, m) in ora.edge_modes(L):
        assert np.abs(rg[m, l1, l2] - ro[m + L, l1, l2].real).max() <= tol * scale, (l1, l2, m)
    assert nnn_err(res.nnn.cpu().numpy(), est.nnn, L) <= tol
    xg, xo = res.xi.cpu().numpy(), est.extra["xi"]
    for e in range(xo.shape[0]):
        assert np.abs(xg[e] - xo[e]).max() <= tol * np.abs(xo[e]).max(), e
    return res, est


def test_full_edge_open_volume(gpu, ora):
    g, o = cfg_pair(ora, r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False)
    d, dw = synth.lognormal(8000, 600.0, 3, mesh=64)
    r, rw = synth.randoms(24000, 4)
    compare_full_edge(gpu, g, o, ora, d, dw, r, rw)


def test_full_edge_weighted_randoms(gpu, ora):
    g, o = cfg_pair(ora, r_min=10.0, r_max=80.0, n_bins=7, l_max=2, Ls=(0, 2), box=500.0, periodic=False)
    d, _ = synth.lognormal(6000, 500.0, 31, mesh=64)
    r, _ = synth.randoms(18000, 32)
    rng = np.random.default_rng(33)
    dw = rng.uniform(0.5, 1.5, d.shape[0]).astype(np.float32)
    rw = rng.uniform(0.2, 1.8, r.shape[0]).astype(np.float32)
    compare_full_edge(gpu, g, o, ora, d, dw, r, rw)


def test_full_edge_thin_slab(gpu, ora):
    """Data and randoms confined to a slab a third of the box thick in z: RRR is
    strongly anisotropic, and the full correction moves the multipoles well
    away from the bin-wise division (which it must, to undo the window)."""
    g, o = cfg_pair(ora, r_min=10.0, r_max=70.0, n_bins=6, l_max=4, Ls=(0, 2), box=500.0, periodic=False)
    d, dw = synth.lognormal(20000, 500.0, 41, mesh=64)
    r, rw = synth.randoms(40000, 42)
    cut = 2 ** 32 // 3
    d, dw = d[d[:, 2] < cut], dw[d[:, 2] < cut]
    r, rw = r[r[:, 2] < cut], rw[r[:, 2] < cut]
    res, est = compare_full_edge(gpu, g, o, ora, d, dw, r, rw)
    rf = est.extra["rrr_full"]
    L = 4
    assert np.abs(rf[L, 2, 0].real).max() > 0.05 * np.abs(rf[L, 0, 0].real).max()
    binwise = ora.project(o, est.nnn, est.rrr, est.mults)[0]
    k = est.mults.index((0, 0, 0))
    assert np.abs(binwise[k] - est.zeta[k]).max() > 0.01 * np.abs(est.zeta[k]).max()


# ------------------------------------------------------ varying line of sight
def test_varying_los_open_volume(gpu, ora):
    """Line of sight from an observer outside the cube to each primary (survey
    geometry): harmonics in each primary's frame; zeta, NNN and xi vs the oracle."""
    g, o = cfg_pair(ora, r_min=10.0, r_max=100.0, n_bins=9, l_max=4, Ls=(0, 2, 4), box=600.0, periodic=False,
                    los="observer", observer=(-300.0, -180.0, -480.0))
    d, dw = synth.lognormal(8000, 600.0, 51, mesh=64)
    r, rw = synth.randoms(24000, 52)
    compare(gpu, g, o, ora, d, dw, r, rw, xi=True)


@pytest.mark.parametrize("lmax,tile", [(2, 4), (6, 0)])
def test_varying_los_observer_inside_periodic(gpu, ora, lmax, tile):
    """Observer at the box centre (lines of sight in every direction), analytic
    randoms, several primaries per tile (each slot with its own frame)."""
    g, o = cfg_pair(ora, r_min=10.0, r_max=60.0, n_bins=5, l_max=lmax, Ls=(0, 2), box=250.0,
                    los="observer", observer=(125.0, 125.0, 125.0), tile_primaries=tile)
    xyz, w = synth.lognormal(6000, 250.0, 53, mesh=32)
    compare(gpu, g, o, ora, xyz, w, xi=True)


def test_varying_los_full_edge(gpu, ora):
    g, o = cfg_pair(ora, r_min=10.0, r_max=80.0, n_bins=6, l_max=2, Ls=(0, 2), box=500.0, periodic=False,
                    los="observer", observer=(250.0, 250.0, -900.0))
    d, dw = synth.lognormal(6000, 500.0, 55, mesh=64)
    r, rw = synth.randoms(18000, 56)
    compare_full_edge(gpu, g, o, ora, d, dw, r, rw)


def test_pair_stage_rsqrt_against_correctly_rounded(gpu):
    """The pair stage's reciprocal square root (estimate + one Newton step) stays
    within one unit in the last place of __frsqrt_rn on 2^24 log-uniform inputs,
    and |n|^2 - 1 carries no bias beyond that of the correctly rounded result
    (a biased |n|^2 would break the j = k cancellation on diagonal bins)."""
    s = tpcf.check_rsqrt(1 << 24, seed=7)
    print(s)
    assert s["max_ulp"] <= 1
    assert abs(s["mean_rel_diff"]) < 5e-9
    assert abs(s["mean_norm_err"] - s["mean_norm_err_rn"]) < 5e-9
