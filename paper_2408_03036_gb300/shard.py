"""Slab-sharded estimator: several ranks (one GPU each) share one catalogue.

The estimator is a sum over primaries (Sec. 4.2: NNN^m is the average over
positions x of the local products of Eq. measured_mult), so it shards by
primaries.  Rank k of R takes the primaries whose z lies in the k-th slab
[k 2^32 / R, (k + 1) 2^32 / R) of the fixed-point box, and as secondaries every
point within r_max of that slab along z (wrapping around in periodic boxes):
that is every neighbour any of its primaries can have.  Each rank computes its
additive partials through tpcf_estimate_3pcf_partial (FP64 NNN^m, the 2PCF
sums, the randoms' triplet counts or l = 0 coupling, integer pair and triplet
counts) with the weight totals of the whole catalogue; one sum reduction over
the process group adds them, and tpcf_estimate_3pcf_finish normalises and
projects.  Only the reduction crosses ranks; its process group's timeout bounds
the wait for a rank that never reports.

This module routes points and moves partial results; every step of the
estimator itself runs in the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

TWO32 = 1 << 32


def slab(rank: int, world: int):
    """[lo, hi) of rank's slab in fixed-point z units."""
    if not (0 <= rank < world):
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return (rank * TWO32) // world, ((rank + 1) * TWO32) // world


def margin_units(cfg) -> int:
    """r_max in fixed-point units, rounded up, plus two units of slack."""
    return int(math.ceil(cfg.r_max / cfg.box * TWO32)) + 2


def partition(cfg, xyz, rank: int, world: int):
    """(primary mask, secondary mask) of rank's slab for uint32 coordinates xyz [n, 3]:
    primaries with z in the slab, secondaries with z within r_max of it (the
    primaries included)."""
    z = np.asarray(xyz)[:, 2].astype(np.int64)
    if world == 1:
        ones = np.ones(z.shape[0], dtype=bool)
        return ones, ones
    lo, hi = slab(rank, world)
    prim = (z >= lo) & (z < hi)
    m = margin_units(cfg)
    if cfg.periodic:
        below = (lo - z) % TWO32          # distance from z up to the slab's start
        above = (z - (hi - 1)) % TWO32    # distance from the slab's last unit up to z
        sec = prim | (below <= m) | (above <= m)
    else:
        sec = (z >= lo - m) & (z < hi + m)
    return prim, sec


def _dist():
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist
    except ImportError:
        pass
    return None


def all_reduce_sum(t, group=None):
    """Sum of a tensor over the process group (in place).  NCCL reduces device
    tensors directly; gloo goes through host memory."""
    dist = _dist()
    if dist is None or dist.get_world_size(group) == 1:
        return t
    if t.is_cuda and dist.get_backend(group) != "nccl":
        h = t.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


class ShardInputs:
    """One rank's share of a catalogue on its device: the secondaries within r_max of
    its slab, the slab's primaries, and the catalogue-wide weight totals."""

    def __init__(self, cfg, d_xyz, d_w=None, r_xyz=None, r_w=None, rank=0, world=1, device="cuda"):
        from paper_2408_03036_gb300 import tpcf
        d_xyz = np.ascontiguousarray(d_xyz, dtype=np.uint32)
        d_w = np.ones(d_xyz.shape[0], np.float32) if d_w is None else np.ascontiguousarray(d_w, dtype=np.float32)
        self.w_d = float(d_w.astype(np.float64).sum())
        self.explicit = r_xyz is not None
        self.w_r, self.weighted = 0.0, False
        pd, sd = partition(cfg, d_xyz, rank, world)
        dev = lambda a, f: None if a is None else f(a, device)
        self.kw = dict(d_xyz=dev(d_xyz[sd], tpcf._as_dev_xyz), d_w=dev(d_w[sd], tpcf._as_dev_w),
                       dp_xyz=dev(d_xyz[pd], tpcf._as_dev_xyz), dp_w=dev(d_w[pd], tpcf._as_dev_w),
                       r_xyz=None, r_w=None, rp_xyz=None, rp_w=None)
        self.n_primaries = int(pd.sum())
        if self.explicit:
            r_xyz = np.ascontiguousarray(r_xyz, dtype=np.uint32)
            r_w = np.ones(r_xyz.shape[0], np.float32) if r_w is None else np.ascontiguousarray(r_w, dtype=np.float32)
            self.w_r = float(r_w.astype(np.float64).sum())
            self.weighted = bool(np.any(r_w != 1.0))
            pr, sr = partition(cfg, r_xyz, rank, world)
            self.kw.update(r_xyz=dev(r_xyz[sr], tpcf._as_dev_xyz), r_w=dev(r_w[sr], tpcf._as_dev_w),
                           rp_xyz=dev(r_xyz[pr], tpcf._as_dev_xyz), rp_w=dev(r_w[pr], tpcf._as_dev_w))
            self.n_primaries += int(pr.sum())
        self.device, self.world = device, world


def estimate_prepared(cfg, inp: ShardInputs, group=None, want_xi=False, stream=None):
    """The whole catalogue's estimate from this rank's prepared share (the partials of
    its slab, summed over the process group, then finished)."""
    from paper_2408_03036_gb300 import tpcf
    pf, pi = tpcf.estimate_3pcf_partial(cfg, w_d_total=inp.w_d, w_r_total=inp.w_r, weighted_randoms=inp.weighted,
                                        stream=stream, device=inp.device, **inp.kw)
    if inp.world > 1:
        all_reduce_sum(pf, group)
        all_reduce_sum(pi, group)
    return tpcf.estimate_3pcf_finish(cfg, pf, pi, inp.w_d, inp.w_r, inp.explicit, inp.weighted, want_xi=want_xi,
                                     stream=stream)


def estimate_3pcf_sharded(cfg, d_xyz, d_w=None, r_xyz=None, r_w=None, rank=None, world=None, group=None,
                          device="cuda", want_xi=False, stream=None):
    """The estimate of the whole catalogue (the same Result as tpcf.estimate_3pcf),
    this rank computing the partials of its slab.  rank / world default to the
    initialised torch.distributed process group (else a single rank)."""
    dist = _dist()
    if world is None:
        world = dist.get_world_size(group) if dist else 1
    if rank is None:
        rank = dist.get_rank(group) if dist else 0
    inp = ShardInputs(cfg, d_xyz, d_w, r_xyz, r_w, rank, world, device)
    return estimate_prepared(cfg, inp, group, want_xi, stream)
