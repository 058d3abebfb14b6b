"""Checkpoint / resume of per-mock results for long covariance batches.

A results directory holds `header.json` (a hash of the estimator configuration,
the seed the mocks were drawn with, the number of mocks and the multipole list)
and one `mock_<id>.npz` per finished mock (zeta [n_mult][n_b][n_b] FP64, the
triplet counts and the mock's status word), each written to a temporary file
and renamed into place, so an interrupted run leaves only whole results.  A
rerun with the same configuration and seed skips the mocks already stored; a
different configuration or seed is refused rather than mixed in.

The estimates themselves run in the CUDA library (tpcf_estimate_3pcf_batched on
the mocks still to do, in groups); this module only moves results to and from
files.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os

import numpy as np


def config_hash(cfg) -> str:
    """SHA-256 of the configuration's fields (dataclass), in a fixed order."""
    d = dataclasses.asdict(cfg)
    text = json.dumps(d, sort_keys=True, default=str)
    return hashlib.sha256(text.encode()).hexdigest()


class MockResults:
    """The results directory of one batch of `n_mocks` mocks."""

    def __init__(self, path, cfg, seed: int, n_mocks: int, multipoles=None):
        self.path = str(path)
        os.makedirs(self.path, exist_ok=True)
        head = {"config_hash": config_hash(cfg), "seed": int(seed), "n_mocks": int(n_mocks),
                "multipoles": [list(map(int, m)) for m in (multipoles or [])]}
        hp = os.path.join(self.path, "header.json")
        if os.path.exists(hp):
            with open(hp) as f:
                old = json.load(f)
            for k in ("config_hash", "seed", "n_mocks"):
                if old.get(k) != head[k]:
                    raise ValueError("results in %s were made with a different %s" % (self.path, k))
            self.header = old
        else:
            tmp = hp + ".tmp"
            with open(tmp, "w") as f:
                json.dump(head, f)
            os.replace(tmp, hp)
            self.header = head
        self.n_mocks = int(n_mocks)

    def _file(self, k: int) -> str:
        return os.path.join(self.path, "mock_%06d.npz" % k)

    def done(self) -> set:
        """Ids of the mocks whose results are stored."""
        return {k for k in range(self.n_mocks) if os.path.exists(self._file(k))}

    def save(self, k: int, zeta, triplet_counts=None, status: int = 0):
        if not (0 <= k < self.n_mocks):
            raise ValueError("mock id %d outside 0..%d" % (k, self.n_mocks - 1))
        tmp = self._file(k) + ".tmp.npz"
        tc = np.zeros(0, dtype=np.int64) if triplet_counts is None else np.asarray(triplet_counts)
        np.savez(tmp, zeta=np.asarray(zeta, dtype=np.float64), triplet_counts=tc, status=np.int32(status))
        os.replace(tmp, self._file(k))

    def load(self, k: int):
        """(zeta, triplet counts, status) of mock k."""
        with np.load(self._file(k)) as f:
            return f["zeta"], f["triplet_counts"], int(f["status"])

    def load_all(self):
        """zeta of every mock [n_mocks][...] (all must be stored) and the status words."""
        missing = sorted(set(range(self.n_mocks)) - self.done())
        if missing:
            raise ValueError("%d mocks have no results yet (first %d)" % (len(missing), missing[0]))
        zs, st = [], []
        for k in range(self.n_mocks):
            z, _, s = self.load(k)
            zs.append(z)
            st.append(s)
        return np.stack(zs), np.asarray(st, dtype=np.int32)


def estimate_mocks_resumable(cfg, xyz, w, offsets, path, seed: int, group: int = 32, stream=None,
                             device="cuda", on_group=None):
    """The batched estimate of every mock (xyz, w and offsets as for
    tpcf.estimate_3pcf_batched: mock k is rows offsets[k]..offsets[k+1]-1) with its
    results kept in `path`: mocks already stored are skipped, the others run in
    groups of `group` mocks (one batched call each) and are stored as each group
    finishes.  on_group(ids), if given, is called after a group is stored (a test
    hook; raising from it interrupts the run like a crash would).  Returns
    (zeta [n_mocks][n_mult][n_b][n_b], status words)."""
    import torch

    from . import tpcf
    off = np.asarray(offsets, dtype=np.int64)
    n = len(off) - 1
    res = MockResults(path, cfg, seed, n, tpcf.multipole_index(cfg))
    todo = [k for k in range(n) if k not in res.done()]
    xyz = np.asarray(xyz) if not isinstance(xyz, torch.Tensor) else xyz
    for g0 in range(0, len(todo), group):
        ids = todo[g0:g0 + group]
        # the group's mocks as one catalogue of consecutive row blocks
        rows = [np.arange(off[k], off[k + 1]) for k in ids]
        sel = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
        sub_off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
        if isinstance(xyz, torch.Tensor):
            gx = xyz[torch.from_numpy(sel).to(xyz.device)]
        else:
            gx = xyz[sel]
        gw = None
        if w is not None:
            gw = w[torch.from_numpy(sel).to(w.device)] if isinstance(w, torch.Tensor) else np.asarray(w)[sel]
        z, tc, st = tpcf.estimate_3pcf_batched(cfg, gx, gw, sub_off, stream=stream, device=device, want_status=True)
        z = z.cpu().numpy()
        tcn = tc.cpu().numpy() if tc is not None else None
        for j, k in enumerate(ids):
            res.save(k, z[j], None if tcn is None else tcn[j], int(st[j]))
        if on_group is not None:
            on_group(ids)
    return res.load_all()
