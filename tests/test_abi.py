"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/tpcf.h declares; host-only entry points agree with the oracle.
No GPU is needed: nothing here launches a kernel."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_2408_03036_gb300 import build as B
from paper_2408_03036_gb300 import tpcf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return tpcf.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tpcf_\w+)\s*\(", txt))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) <= set(tpcf.EXPORTS) | set(decl)
    for name in tpcf.EXPORTS:
        assert name in decl, name


def test_version_and_error_string(lib):
    assert lib.tpcf_version() >= 100
    cfg = tpcf.Config(20.0, 10.0, 10, 4)
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.multipole_index(cfg)
    assert ei.value.code == -1 and "r_max" in str(ei.value)


@pytest.mark.parametrize("lmax,Ls", [(4, (0, 2, 4)), (6, (0, 2, 4, 6)), (4, (0, 2)), (2, (0,))])
def test_multipole_list_matches_oracle(lib, ora, lmax, Ls):
    cfg = tpcf.Config(20.0, 120.0, 10, lmax, Ls)
    assert tpcf.multipole_index(cfg) == ora.multipoles(lmax, Ls)


def test_counts_of_multipoles(lib):
    assert len(tpcf.multipole_index(tpcf.Config(20.0, 120.0, 10, 4, (0, 2, 4)))) == 24
    assert len(tpcf.multipole_index(tpcf.Config(5.0, 155.0, 30, 6, (0, 2, 4, 6)))) == 58
    assert len(tpcf.multipole_index(tpcf.Config(10.0, 150.0, 20, 4, (0, 2)))) == 15


@pytest.mark.parametrize("rmin,rmax,nb,box", [(20.0, 120.0, 10, 500.0), (10.0, 150.0, 20, 1000.0),
                                              (5.0, 155.0, 30, 500.0), (0.3, 7.7, 7, 33.3)])
def test_bin_edges_match_oracle(lib, ora, rmin, rmax, nb, box):
    cfg = tpcf.Config(rmin, rmax, nb, 2, (0,), box=box)
    ocfg = ora.Config(rmin, rmax, nb, 2, (0,), box=box)
    E, _ = ora.edges(ocfg)
    assert tpcf.bin_edges(cfg) == [int(e) for e in E]


@pytest.mark.parametrize("bad", [dict(n_bins=0), dict(n_bins=33), dict(l_max=7), dict(r_min=0.0),
                                 dict(r_max=300.0), dict(Ls=(1,)), dict(Ls=(10,)), dict(precision="fp16"),
                                 dict(chunk=100), dict(chunk=256), dict(tile_primaries=9)])
def test_config_validation(lib, bad):
    kw = dict(r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), box=500.0)
    if bad.get("precision") == "fp16":
        cfg = tpcf.Config(**kw)
        c = cfg.c()
        c.precision = 9
        n = ctypes.c_int32(0)
        assert lib.tpcf_multipole_count(ctypes.byref(c), ctypes.addressof(n)) == -1
        return
    kw.update(bad)
    with pytest.raises(tpcf.TpcfError):
        tpcf.multipole_index(tpcf.Config(**kw))


@pytest.mark.parametrize("nb,eta,sel", [(12, 3, [(0, 0, 0), (2, 0, 2)]), (20, 0, [(1, 1, 0)]),
                                        (20, 2, [(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2), (3, 1, 2)])])
def test_data_vector_index_matches_oracle(lib, ora, nb, eta, sel):
    from oracle import covariance as CV
    cfg = tpcf.Config(10.0, 130.0, nb, 4, (0, 2, 4))
    got = tpcf.data_vector_index(cfg, sel, eta)
    ref = CV.data_vector_index(nb, ora.multipoles(4, (0, 2, 4)), sel, eta)
    assert np.array_equal(got, ref)
    with pytest.raises(tpcf.TpcfError):
        tpcf.data_vector_index(tpcf.Config(10.0, 130.0, nb, 4, (0, 2)), [(1, 3, 4)], eta)


@pytest.mark.parametrize("nm,nd,npar", [(3000, 336, 6), (3000, 288, 7), (40, 20, 3)])
def test_covariance_factors_match_oracle(lib, nm, nd, npar):
    from oracle import covariance as CV
    h, m1 = tpcf.covariance_factors(nm, nd, npar)
    assert abs(h - CV.hartlap(nm, nd)) < 1e-15
    assert abs(m1 - CV.percival_m1(nm, nd, npar)) < 1e-14
    with pytest.raises(tpcf.TpcfError):
        tpcf.covariance_factors(nd + 4, nd, npar)


def test_entry_points_reject_bad_arguments_before_device_work(lib):
    """Argument errors are reported by the host checks, with a message, before
    any CUDA call (so they run here without a GPU)."""
    cfg = tpcf.Config(10.0, 60.0, 5, 2, (0, 2), box=250.0)
    c = cfg.c()
    z = ctypes.c_void_p(1)   # never dereferenced: the checks fail first
    # no data points
    rc = lib.tpcf_estimate_3pcf_xi(ctypes.byref(c), None, None, 0, None, None, 0, z, None, None, None, None, None,
                                   None)
    assert rc == -1 and b"data point" in lib.tpcf_last_error()
    # analytic randoms in an open volume
    oc = tpcf.Config(10.0, 60.0, 5, 2, (0, 2), periodic=False, box=250.0).c()
    rc = lib.tpcf_estimate_3pcf(ctypes.byref(oc), z, None, 10, None, None, 0, z, None, None, None, None, None)
    assert rc == -1 and b"periodic" in lib.tpcf_last_error()
    # the full edge correction needs explicit randoms
    rc = lib.tpcf_estimate_3pcf_full_edge(ctypes.byref(c), z, None, 10, None, None, 0, z, None, None, None, None)
    assert rc == -1 and b"randoms" in lib.tpcf_last_error()
    # a covariance needs two mocks and a consistent selection
    rc = lib.tpcf_covariance(z, 1, 10, None, 5, z, z, None)
    assert rc == -1 and b"two mocks" in lib.tpcf_last_error()
    rc = lib.tpcf_covariance(z, 5, 10, None, 11, z, z, None)
    assert rc == -1 and b"stride" in lib.tpcf_last_error()
    # the rsqrt check needs inputs and an output
    assert lib.tpcf_check_rsqrt(0, 1, None, None) == -1
    # the count pass needs a grid
    rc = lib.tpcf_pair_counts(None, None, 10, ctypes.byref(c), None, None, None)
    assert rc == -1 and b"grid" in lib.tpcf_last_error()
    # a varying line of sight needs a finite observer
    vc = tpcf.Config(10.0, 60.0, 5, 2, (0, 2), box=250.0, los="observer", observer=(float("nan"), 0.0, 0.0))
    with pytest.raises(tpcf.TpcfError):
        tpcf.multipole_index(vc)


def test_quantize_host_matches_the_fixed_point_rule(lib):
    """tpcf_quantize_host against the generators' rule (floor(x / box * 2^32) in
    FP64) bit for bit, the box edges, and out-of-range or non-finite positions."""
    from paper_2408_03036_gb300 import synth
    rng = np.random.default_rng(11)
    box = 1000.0
    x = rng.uniform(0.0, box, size=(5000, 3)).astype(np.float32)
    x[0] = [0.0, np.nextafter(np.float32(box), np.float32(0)), 500.0]
    u = tpcf.quantize_host(x, box)
    assert u.shape == x.shape and u.dtype == np.uint32
    assert np.array_equal(u, synth.quantize(x, box))
    assert u[0, 0] == 0 and u[0, 2] == 2 ** 31
    for bad in (-1e-3, box, np.inf, np.nan):
        y = x.copy()
        y[7, 1] = bad
        with pytest.raises(tpcf.TpcfError) as ei:
            tpcf.quantize_host(y, box)
        assert ei.value.code == -6
    with pytest.raises(tpcf.TpcfError):
        tpcf.quantize_host(x, 0.0)
