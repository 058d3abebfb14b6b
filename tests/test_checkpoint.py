"""Checkpoint / resume of per-mock results on the host: the header guards against
mixing configurations or seeds, stored mocks are reported as done, writes are
whole files, and a batch is only complete when every mock is stored."""
import dataclasses
import os

import numpy as np
import pytest

from paper_2408_03036_gb300 import checkpoint as ck


@dataclasses.dataclass
class FakeConfig:
    r_min: float = 20.0
    r_max: float = 120.0
    n_bins: int = 4
    l_max: int = 2


def test_config_hash_tracks_every_field():
    a = ck.config_hash(FakeConfig())
    assert a == ck.config_hash(FakeConfig())
    assert a != ck.config_hash(FakeConfig(n_bins=5))
    assert a != ck.config_hash(FakeConfig(r_max=121.0))


def test_results_round_trip_and_resume(tmp_path):
    cfg = FakeConfig()
    res = ck.MockResults(tmp_path, cfg, seed=7, n_mocks=5, multipoles=[(0, 0, 0), (1, 1, 0)])
    assert res.done() == set()
    rng = np.random.default_rng(1)
    z = {k: rng.normal(size=(2, 4, 4)) for k in (0, 3)}
    for k, zk in z.items():
        res.save(k, zk, np.arange(16).reshape(4, 4) + k, status=k)
    # nothing but whole files and the header
    assert sorted(os.listdir(tmp_path)) == ["header.json", "mock_000000.npz", "mock_000003.npz"]
    again = ck.MockResults(tmp_path, cfg, seed=7, n_mocks=5)
    assert again.done() == {0, 3}
    zz, tc, st = again.load(3)
    assert np.array_equal(zz, z[3]) and np.array_equal(tc, np.arange(16).reshape(4, 4) + 3) and st == 3
    with pytest.raises(ValueError):
        again.load_all()                                   # mocks 1, 2, 4 missing
    for k in (1, 2, 4):
        again.save(k, np.zeros((2, 4, 4)))
    allz, stat = again.load_all()
    assert allz.shape == (5, 2, 4, 4) and np.array_equal(allz[0], z[0]) and list(stat) == [0, 0, 0, 3, 0]


@pytest.mark.parametrize("change", [dict(seed=8), dict(n_mocks=6), dict(cfg=FakeConfig(l_max=4))])
def test_a_different_run_is_refused(tmp_path, change):
    ck.MockResults(tmp_path, FakeConfig(), seed=7, n_mocks=5)
    kw = dict(cfg=FakeConfig(), seed=7, n_mocks=5)
    kw.update(change)
    with pytest.raises(ValueError):
        ck.MockResults(tmp_path, kw["cfg"], kw["seed"], kw["n_mocks"])


def test_mock_ids_are_checked(tmp_path):
    res = ck.MockResults(tmp_path, FakeConfig(), seed=1, n_mocks=2)
    with pytest.raises(ValueError):
        res.save(2, np.zeros(1))
