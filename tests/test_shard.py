"""Slab sharding of the estimator over ranks (host logic, CPU only).

The partition pins: primaries fall in exactly one slab, and every neighbour
within r_max of a slab's primary is among that slab's secondaries (brute force,
periodic and open).  The multi-rank path: world-size-2 process groups on the
gloo backend, each rank computing its slab's additive partials with the FP64
oracle, one sum all-reduce, and the result against the unsplit oracle
(NNN^m, RRR, zeta to 1e-12, counts exact).  A rank that never reports ends the
other's reduction with an error within the group's timeout.
"""
import datetime
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest

from paper_2408_03036_gb300 import shard, synth, tpcf


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("world", [2, 3, 5])
def test_partition_covers_every_neighbour(periodic, world):
    cfg = tpcf.Config(r_min=5.0, r_max=70.0, n_bins=4, l_max=2, Ls=(0,), box=300.0, periodic=periodic)
    xyz, _ = synth.poisson(1500, 7)
    masks = [shard.partition(cfg, xyz, r, world) for r in range(world)]
    prim_count = sum(m[0].astype(int) for m in masks)
    assert np.array_equal(prim_count, np.ones(xyz.shape[0], dtype=int))   # a partition
    u = 2.0 ** 32 / cfg.box
    d = xyz[None, :, :].astype(np.int64) - xyz[:, None, :].astype(np.int64)
    if periodic:
        d = (d + 2 ** 31) % 2 ** 32 - 2 ** 31
    r = np.sqrt((d.astype(np.float64) ** 2).sum(-1)) / u
    near = r < cfg.r_max
    for prim, sec in masks:
        assert prim[sec].sum() == prim.sum()               # primaries are secondaries
        need = near[prim].any(axis=0)                        # every neighbour of a primary
        assert not np.any(need & ~sec)


def _rank_partials(ora, cfg, o, d, dw, r, rw, rank, world):
    """One rank's additive partials with the oracle: (nnn, rrr, pair counts, triplet counts)."""
    wd = float(dw.astype(np.float64).sum())
    pd, sd = shard.partition(cfg, d, rank, world)
    if r is None:
        idx = np.flatnonzero(pd[sd])
        out = ora.run(o, d[sd], dw[sd].astype(np.float64), offset_weight=wd, prim=idx)
        return out.nnn, None, out.pair_counts, out.trip_counts
    alpha = wd / float(rw.astype(np.float64).sum())
    pr, sr = shard.partition(cfg, r, rank, world)
    xyz = np.concatenate([d[sd], r[sr]])
    w = np.concatenate([dw[sd].astype(np.float64), -alpha * rw[sr].astype(np.float64)])
    idx = np.concatenate([np.flatnonzero(pd[sd]), sd.sum() + np.flatnonzero(pr[sr])])
    out = ora.run(o, xyz, w, prim=idx)
    rr = ora.run(o, r[sr], alpha * rw[sr].astype(np.float64), l_max=0, prim=np.flatnonzero(pr[sr]))
    return out.nnn, rr.nnn[0, 0, 0].real, out.pair_counts, out.trip_counts


def _cases():
    d, dw = synth.lognormal(2500, 300.0, 31, mesh=32)
    r, rw = synth.randoms(5000, 32)
    rw2 = np.random.default_rng(33).uniform(0.5, 1.5, r.shape[0]).astype(np.float32)
    pc = dict(r_min=10.0, r_max=60.0, n_bins=5, l_max=3, Ls=(0, 2), box=300.0)
    return {
        "periodic": (dict(pc, periodic=True), d, dw, None, None),
        "open": (dict(pc, periodic=False), d, dw, r, rw),
        "open_weighted": (dict(pc, periodic=False), d, dw, r, rw2),
    }


def _worker(rank, world, port, case, q):
    import torch.distributed as dist
    from oracle import oracle as ora
    os.environ["GLOO_SOCKET_IFNAME"] = os.environ.get("GLOO_SOCKET_IFNAME", "lo")
    try:
        dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=20))
        import torch
        kw, d, dw, r, rw = _cases()[case]
        cfg = tpcf.Config(**kw)
        o = ora.Config(kw["r_min"], kw["r_max"], kw["n_bins"], kw["l_max"], kw["Ls"], kw["periodic"], kw["box"])
        nnn, rrr, pc, tc = _rank_partials(ora, cfg, o, d, dw, r, rw, rank, world)
        t = [torch.from_numpy(np.ascontiguousarray(nnn.real)), torch.from_numpy(np.ascontiguousarray(nnn.imag)),
             torch.from_numpy(pc.astype(np.int64)), torch.from_numpy(tc.astype(np.int64))]
        if rrr is not None:
            t.append(torch.from_numpy(np.ascontiguousarray(rrr)))
        for x in t:
            shard.all_reduce_sum(x)
        q.put((rank, [x.numpy() for x in t]))
        dist.destroy_process_group()
    except Exception as e:   # reported to the parent
        q.put((rank, "error: %r" % (e,)))


def _run_ranks(target, world, *args, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=target, args=(r, world, port) + args + (q,)) for r in range(world)]
    for p in ps:
        p.start()
    out = {}
    t0 = time.time()
    while len(out) < world and time.time() - t0 < timeout:
        try:
            rank, v = q.get(timeout=1.0)
            out[rank] = v
        except Exception:
            pass
    for p in ps:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return out, time.time() - t0


@pytest.mark.parametrize("case", ["periodic", "open", "open_weighted"])
def test_two_ranks_reproduce_the_unsplit_estimate(ora, case):
    kw, d, dw, r, rw = _cases()[case]
    o = ora.Config(kw["r_min"], kw["r_max"], kw["n_bins"], kw["l_max"], kw["Ls"], kw["periodic"], kw["box"])
    out, _ = _run_ranks(_worker, 2, case)
    assert set(out) == {0, 1}, out
    for rank in (0, 1):
        assert not isinstance(out[rank], str), out[rank]
    a, b = out[0], out[1]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)                          # every rank holds the same sums
    est = ora.estimate(o, d, dw, r, rw)
    nnn = a[0] + 1j * a[1]
    assert np.abs(nnn - est.nnn).max() <= 1e-12 * np.abs(est.nnn).max()
    assert np.array_equal(a[2], est.pair_counts)
    assert np.array_equal(a[3], est.trip_counts)
    rrr = est.rrr if r is None else a[4]
    assert np.abs(rrr - est.rrr).max() <= 1e-12 * np.abs(est.rrr).max()
    z, _ = ora.project(o, nnn, rrr, est.mults)
    assert np.abs(z - est.zeta).max() <= 1e-12 * np.abs(est.zeta).max()


def _silent_worker(rank, world, port, q):
    """Rank 1 leaves before the reduction; rank 0 must get an error, not wait forever."""
    import torch
    import torch.distributed as dist
    try:
        dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=5))
        if rank == 1:
            q.put((rank, "left"))
            return          # never reduces (the process ends)
        t0 = time.time()
        try:
            shard.all_reduce_sum(torch.ones(4, dtype=torch.float64))
            q.put((rank, "reduced"))
        except Exception as e:
            q.put((rank, ("error", time.time() - t0, type(e).__name__)))
    except Exception as e:
        q.put((rank, ("setup-error", repr(e))))


def test_a_rank_that_never_reports_ends_in_an_error():
    out, elapsed = _run_ranks(_silent_worker, 2, timeout=90)
    assert out.get(1) == "left"
    r0 = out.get(0)
    assert isinstance(r0, tuple) and r0[0] == "error", r0
    assert r0[1] < 60.0
