"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's code: closed forms, a library routine, an
exact-rational computation, brute-force triplet sums, exact invariances, the
exact expectation of the estimator on Poisson points, and a quadrature
identity of the TripoSH basis.
"""
import math

import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from tests import bruteforce as bf

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ------------------------------------------------------------------ edges

def test_edges_are_exact_ceil_of_square(ora):
    for (rmin, rmax, nb, box) in [(20.0, 120.0, 10, 500.0), (10.0, 150.0, 20, 1000.0),
                                  (5.0, 155.0, 30, 500.0), (0.3, 7.7, 7, 33.3)]:
        cfg = ora.Config(rmin, rmax, nb, 2, box=box)
        E, r = ora.edges(cfg)
        ref = bf.exact_edges(rmin, rmax, nb, box)
        assert [int(e) for e in E] == ref
        assert r[0] == rmin and abs(r[-1] - rmax) < 1e-12


# -------------------------------------------------------- spherical harmonics

def _unit_vectors(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


def test_ylm_closed_forms(ora):
    pi = math.pi
    for x, y, z in _unit_vectors(20, 3):
        Y = ora.ylm((x, y, z), 3)
        xy = x + 1j * y
        ref = {
            (0, 0): 0.5 / math.sqrt(pi),
            (1, 0): math.sqrt(3 / (4 * pi)) * z,
            (1, 1): -math.sqrt(3 / (8 * pi)) * xy,
            (1, -1): math.sqrt(3 / (8 * pi)) * np.conj(xy),
            (2, 0): math.sqrt(5 / (16 * pi)) * (3 * z * z - 1),
            (2, 1): -math.sqrt(15 / (8 * pi)) * z * xy,
            (2, 2): math.sqrt(15 / (32 * pi)) * xy * xy,
            (3, 0): math.sqrt(7 / (16 * pi)) * (5 * z ** 3 - 3 * z),
            (3, 3): -math.sqrt(35 / (64 * pi)) * xy ** 3,
        }
        for (l, m), v in ref.items():
            assert abs(Y[l * l + l + m] - v) < 1e-13


def test_ylm_matches_scipy_and_unsold(ora):
    for v in _unit_vectors(30, 4):
        Y = ora.ylm(v, 8)
        th = math.acos(np.clip(v[2], -1, 1))
        ph = math.atan2(v[1], v[0])
        for l in range(9):
            s = 0.0
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - bf.sph_y(l, m, th, ph)) < 1e-12
                s += abs(Y[l * l + l + m]) ** 2
            assert abs(s - (2 * l + 1) / (4 * math.pi)) < 1e-12   # Unsold's theorem


def test_ylm_orthonormal_by_quadrature(ora):
    L = 6
    xg, wg = np.polynomial.legendre.leggauss(L + 2)
    nphi = 2 * L + 3
    G = np.zeros(((L + 1) ** 2, (L + 1) ** 2), dtype=np.complex128)
    for ct, wt in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = ora.ylm((st * math.cos(ph), st * math.sin(ph), ct), L)
            G += wt * (2 * math.pi / nphi) * np.outer(Y, np.conj(Y))
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-12


# ------------------------------------------------------------------- 3j

def test_wigner3j_special_values(ora):
    for l in range(9):
        for m in range(-l, l + 1):
            assert abs(ora.wigner3j(l, l, 0, m, -m, 0) - (-1) ** (l - m) / math.sqrt(2 * l + 1)) < 1e-14
    assert abs(ora.wigner3j(1, 1, 2, 0, 0, 0) - math.sqrt(2 / 15)) < 1e-15
    assert ora.wigner3j(1, 1, 1, 0, 0, 0) == 0.0          # odd l1 + l2 + L with m = 0
    assert ora.wigner3j(2, 2, 5, 0, 0, 0) == 0.0          # triangle rule


def test_wigner3j_vs_exact_sympy(ora):
    for j1 in range(5):
        for j2 in range(5):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for m1 in range(-j1, j1 + 1):
                    for m2 in range(-j2, j2 + 1):
                        m3 = -m1 - m2
                        if abs(m3) > j3:
                            continue
                        assert abs(ora.wigner3j(j1, j2, j3, m1, m2, m3)
                                   - bf.w3j_exact(j1, j2, j3, m1, m2, m3)) < 1e-14


def test_wigner3j_orthogonality(ora):
    for j1, j2 in [(3, 4), (6, 6), (2, 5)]:
        for j3 in range(abs(j1 - j2), j1 + j2 + 1):
            for j3p in range(abs(j1 - j2), j1 + j2 + 1):
                s = sum(ora.wigner3j(j1, j2, j3, m1, m2, -m1 - m2) * ora.wigner3j(j1, j2, j3p, m1, m2, -m1 - m2)
                        for m1 in range(-j1, j1 + 1) for m2 in range(-j2, j2 + 1)
                        if abs(m1 + m2) <= min(j3, j3p))
                # summed over M as well: delta_{j3 j3'} (2 j3 + 1) / (2 j3 + 1)
                assert abs(s - (1.0 if j3 == j3p else 0.0)) < 1e-13


# --------------------------------------------------------- counts / brute force

def _dense_tiny(seed, n=160, box=150.0):
    xyz, w = synth.poisson(n, seed)
    return xyz, w


@pytest.mark.parametrize("periodic", [True, False])
def test_pair_and_triplet_counts_vs_brute_force(ora, periodic):
    xyz, w = _dense_tiny(11, n=300)
    cfg = ora.Config(8.0, 40.0, 6, 0, (0,), periodic, 150.0)
    E, _ = ora.edges(cfg)
    o = ora.run(cfg, xyz, w, l_max=0, nthreads=2)
    nbl = bf.neighbours(xyz, periodic, E)
    pc = np.zeros(cfg.n_bins, dtype=np.int64)
    tc = np.zeros((cfg.n_bins, cfg.n_bins), dtype=np.int64)
    for ok, bins, _ in nbl:
        n_b = np.bincount(bins, minlength=cfg.n_bins).astype(np.int64)
        pc += n_b
        tc += np.outer(n_b, n_b) - np.diag(n_b)
    assert np.array_equal(o.pair_counts, pc)
    assert np.array_equal(o.trip_counts, tc)


@pytest.mark.parametrize("periodic,signed", [(True, False), (False, True)])
def test_nnn_vs_brute_force_triplets(ora, periodic, signed):
    """NNN^m from the factorised a_l^m equals the explicit j != k triplet sum."""
    xyz, w = _dense_tiny(12, n=150)
    w = w.astype(np.float64)
    if signed:  # a data-minus-random style signed field
        w[::3] = -0.4
    cfg = ora.Config(10.0, 45.0, 4, 3, (0, 2), periodic, 150.0)
    E, _ = ora.edges(cfg)
    o = ora.run(cfg, xyz, w, nthreads=2)
    nnn, leg, trip = bf.triplets(xyz, w, periodic, E, cfg.n_bins, cfg.l_max)
    scale = np.abs(nnn).max()
    assert np.abs(o.nnn - nnn).max() <= 1e-12 * scale
    assert np.array_equal(o.trip_counts, trip)
    # addition theorem: sum_m Y_l^m(a) Y_l^m*(b) = (2l+1)/(4 pi) P_l(a.b), no Y used on this side
    for l in range(cfg.l_max + 1):
        s = sum(o.nnn[m + cfg.l_max, l, l] for m in range(-l, l + 1))
        ref = (2 * l + 1) / (4 * math.pi) * leg[l]
        assert np.abs(s.imag).max() < 1e-12 * scale
        assert np.abs(s.real - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_projection_vs_tripolar_basis(ora):
    """Eq. slep2sugy on the oracle's NNN equals the triplet sum of S_{l1 l2 L}(r1, r2, z)
    built from its definition (Eq. TSHbasis) with Schmidt y, times
    (2L+1) H^2 sqrt((2 l1+1)(2 l2+1)) / (4 pi)."""
    xyz, w = _dense_tiny(13, n=140)
    cfg = ora.Config(10.0, 45.0, 3, 3, (0, 2, 4), True, 150.0, convention="PAPER_EQ")
    E, _ = ora.edges(cfg)
    o = ora.run(cfg, xyz, w, nthreads=2)
    mults = [(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (3, 1, 2), (2, 2, 4), (1, 3, 4), (3, 3, 2)]
    zr, zi = ora.project(cfg, o.nnn, np.ones((cfg.n_bins, cfg.n_bins)), mults)
    for k, (l1, l2, LL) in enumerate(mults):
        H = bf.w3j_exact(l1, l2, LL, 0, 0, 0)
        ref = (2 * LL + 1) * H * H * math.sqrt((2 * l1 + 1) * (2 * l2 + 1)) / (4 * math.pi) \
            * bf.tsh_sum(xyz, w, True, E, cfg.n_bins, l1, l2, LL)
        assert np.abs(zr[k] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (l1, l2, LL)
        assert np.abs(zi[k]).max() <= 1e-11 * max(1.0, np.abs(ref).max())


def test_quadrature_identity_fixes_convention(ora):
    """Feeding NNN^m of a pure basis function S_{abc} (angular quadrature over both
    triangle sides, uniform measure) through the S_COEFF projection returns the unit
    coefficient on (a, b, c) and zero elsewhere; PAPER_EQ returns 1/sqrt((2a+1)(2b+1))."""
    L = 4
    xg, wg = np.polynomial.legendre.leggauss(6)
    nphi = 11
    th, ph, wq = [], [], []
    for ct, wt in zip(xg, wg):
        for k in range(nphi):
            th.append(math.acos(ct)); ph.append(2 * math.pi * k / nphi); wq.append(wt / (2 * nphi))
    th, ph, wq = map(np.array, (th, ph, wq))
    Y = {(l, m): bf.sph_y(l, m, th, ph) for l in range(L + 1) for m in range(-l, l + 1)}

    def S(a, b, c):
        H = bf.w3j_exact(a, b, c, 0, 0, 0)
        out = np.zeros((th.size, th.size), dtype=np.complex128)
        for m in range(-min(a, b), min(a, b) + 1):
            y1 = math.sqrt(4 * math.pi / (2 * a + 1)) * Y[(a, m)]
            y2 = math.sqrt(4 * math.pi / (2 * b + 1)) * Y[(b, -m)]
            out += bf.w3j_exact(a, b, c, m, -m, 0) * np.outer(y1, y2)
        return out / H   # y_c^0(z) = 1

    W = np.outer(wq, wq)
    cfg = ora.Config(1.0, 2.0, 1, L, (0, 2, 4), True, 10.0)
    mults = ora.multipoles(L, cfg.Ls)
    for (a, b, c) in [(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (3, 1, 2), (2, 2, 4), (4, 2, 2)]:
        f = S(a, b, c)
        assert np.abs(f.imag).max() < 1e-12
        nnn = np.zeros((2 * L + 1, L + 1, L + 1, 1, 1), dtype=np.complex128)
        for m in range(-L, L + 1):
            for l1 in range(abs(m), L + 1):
                for l2 in range(abs(m), L + 1):
                    nnn[m + L, l1, l2, 0, 0] = np.sum(W * f * np.outer(Y[(l1, m)], np.conj(Y[(l2, m)])))
        rrr = np.full((1, 1), np.sum(W) / (4 * math.pi))   # uniform triplets, Y_0^0 Y_0^0
        for conv in ("S_COEFF", "PAPER_EQ"):
            cfg.convention = conv
            zr, zi = ora.project(cfg, nnn, rrr, mults)
            for k, m3 in enumerate(mults):
                want = 0.0
                if m3 == (a, b, c):
                    want = 1.0 if conv == "S_COEFF" else 1.0 / math.sqrt((2 * a + 1) * (2 * b + 1))
                assert abs(zr[k, 0, 0] - want) < 1e-10, (conv, (a, b, c), m3)
                assert abs(zi[k, 0, 0]) < 1e-10


# ------------------------------------------------------------- invariances

def _zeta(ora, cfg, xyz, w):
    return ora.estimate(cfg, xyz, w, nthreads=4).zeta


def test_exact_invariances(ora):
    xyz, w = synth.poisson(1500, 21)
    cfg = ora.Config(20.0, 120.0, 5, 4, (0, 2, 4), True, 500.0)
    base = ora.estimate(cfg, xyz, w, nthreads=4)
    z0 = base.zeta
    tol = 1e-10 * np.abs(z0).max()
    # r1 <-> r2 with l1 <-> l2
    idx = {m: k for k, m in enumerate(base.mults)}
    for k, (l1, l2, L) in enumerate(base.mults):
        assert np.abs(z0[k] - z0[idx[(l2, l1, L)]].T).max() <= tol
    # reflection z -> -z (exact in fixed point: u -> -u mod 2^32)
    r = xyz.copy(); r[:, 2] = (np.uint64(2**32) - r[:, 2].astype(np.uint64)).astype(np.uint32)
    assert np.abs(_zeta(ora, cfg, r, w) - z0).max() <= tol
    # 90 degree rotation about the line of sight: (x, y) -> (-y, x)
    r = xyz.copy(); r[:, 0] = (np.uint64(2**32) - xyz[:, 1].astype(np.uint64)).astype(np.uint32); r[:, 1] = xyz[:, 0]
    assert np.abs(_zeta(ora, cfg, r, w) - z0).max() <= tol
    # periodic integer translation
    r = (xyz.astype(np.uint64) + np.array([123456789, 2**31 + 7, 3999999999], dtype=np.uint64)) % np.uint64(2**32)
    assert np.abs(_zeta(ora, cfg, r.astype(np.uint32), w) - z0).max() <= tol
    # counts are invariant exactly
    assert np.array_equal(ora.estimate(cfg, r.astype(np.uint32), w, nthreads=4).trip_counts, base.trip_counts)


# ----------------------------------------------------- expectation on Poisson

def test_poisson_null_expectation(ora):
    """On N uniform points in a periodic box (a multinomial draw of the other N-1),
    the analytic-random estimator has E[zeta_000] = -1/(N-1) exactly (integral
    constraint of a fixed-N catalogue; PAPER_EQ convention), and every other
    multipole has zero expectation.  Checked against the spread over seeds."""
    N, seeds = 3000, 24
    cfg = ora.Config(10.0, 50.0, 4, 2, (0, 2), True, 200.0, convention="PAPER_EQ")
    ests = [ora.estimate(cfg, *synth.poisson(N, 1000 + s), nthreads=4) for s in range(seeds)]
    zs = np.array([e.zeta for e in ests])
    mults = ora.multipoles(cfg.l_max, cfg.Ls)
    mean = zs.mean(0)
    sem = zs.std(0, ddof=1) / math.sqrt(seeds)
    for k, m in enumerate(mults):
        want = -1.0 / (N - 1) if m == (0, 0, 0) else 0.0
        dev = np.abs(mean[k] - want) / sem[k]
        assert dev.max() < 5.0, (m, dev.max())
    # zeta_000 over all bins at once (sum of NNN over sum of RRR) resolves the
    # -1/(N-1) term: an offset using N instead of N-1 in c_b would move it by
    # about 2/N, several standard errors away
    tot = np.array([e.nnn[cfg.l_max, 0, 0].real.sum() / e.rrr.sum() for e in ests])
    sem_tot = tot.std(ddof=1) / math.sqrt(seeds)
    assert abs(tot.mean() + 1.0 / (N - 1)) < 4.0 * sem_tot
    assert (2.0 / N) / sem_tot > 3.0


def test_nonperiodic_rrr_is_integer_triplet_count(ora):
    """RRR_00^0 from the random-only pass equals alpha^3 T_RR / (4 pi) exactly."""
    rxyz, rw = synth.randoms(900, 31)
    cfg = ora.Config(10.0, 60.0, 4, 0, (0,), False, 300.0)
    alpha = 0.25
    o = ora.run(cfg, rxyz, alpha * rw.astype(np.float64), l_max=0, nthreads=2)
    ref = alpha ** 3 * o.trip_counts / (4 * math.pi)
    assert np.abs(o.nnn[0, 0, 0].real - ref).max() <= 1e-12 * np.abs(ref).max()


# ------------------------------------------------------------ 2PCF multipoles
@pytest.mark.parametrize("periodic", [True, False])
def test_xi_numerator_vs_brute_force_pairs(ora, periodic):
    """sum_i w_i a_l^0[b] equals the brute-force pair sum sum w_i w_j Y_l^0(r_ij)
    (with the analytic-random offset c_b W on l = 0 for the periodic form)."""
    from scipy.special import eval_legendre
    box = 150.0
    xyz, _ = synth.poisson(400, 77)
    w = np.random.default_rng(3).uniform(0.5, 1.5, 400)
    cfg = ora.Config(5.0, 40.0, 5, 4, (0,), periodic, box)
    E = bf.exact_edges(5.0, 40.0, 5, box)
    off = float(w.sum()) if periodic else -1.0
    o = ora.run(cfg, xyz, w, offset_weight=off, want_alm=True)
    S = ora.m0_sums(o.alm, w, 4)
    ref = np.zeros((3, 5))
    for i, (js, bins, d) in enumerate(bf.neighbours(xyz, periodic, E)):
        mu = d[:, 2] / np.sqrt((d * d).sum(1))
        for e, l in enumerate((0, 2, 4)):
            np.add.at(ref[e], bins, w[i] * w[js] * math.sqrt((2 * l + 1) / (4 * math.pi)) * eval_legendre(l, mu))
    if periodic:
        ref[0] -= float(w.sum()) * ora.shell_offsets(cfg, float(w.sum()))
    np.testing.assert_allclose(S, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_xi_poisson_null(ora):
    """Uniform points in a periodic box: every 2PCF multipole of the analytic-random
    form has zero expectation (E[DD_b] = N (N - 1) V_b / L^3 and the separation
    directions are isotropic), checked against the spread over seeds."""
    N, seeds = 3000, 24
    cfg = ora.Config(10.0, 50.0, 4, 2, (0,), True, 200.0)
    xs = np.array([ora.estimate(cfg, *synth.poisson(N, 2000 + s), nthreads=4, want_xi=True).extra["xi"]
                   for s in range(seeds)])
    dev = np.abs(xs.mean(0)) / (xs.std(0, ddof=1) / math.sqrt(seeds))
    assert dev.max() < 5.0, dev.max()


def test_xi_normaliser_is_the_random_pair_sum(ora):
    """RR_b is alpha^2 times the ordered random pair count for unit random weights,
    and alpha^2 sum_{i != j} w_i w_j over the random pairs of bin b (brute force)
    for weighted randoms."""
    box = 150.0
    d, dw = synth.poisson(600, 5)
    r, rw = synth.randoms(1800, 6)
    cfg = ora.Config(5.0, 40.0, 5, 2, (0,), False, box)
    est = ora.estimate(cfg, d, dw, r, rw, want_xi=True)
    alpha = dw.astype(np.float64).sum() / rw.astype(np.float64).sum()
    pc = ora.run(cfg, r, rw, l_max=0).pair_counts
    np.testing.assert_allclose(est.extra["rr"], alpha ** 2 * pc, rtol=1e-12)
    rw2 = np.random.default_rng(7).uniform(0.2, 1.8, r.shape[0])
    est2 = ora.estimate(cfg, d, dw, r, rw2, want_xi=True)
    alpha2 = dw.astype(np.float64).sum() / rw2.sum()
    ref = np.zeros(5)
    for i, (js, bins, _) in enumerate(bf.neighbours(r, False, bf.exact_edges(5.0, 40.0, 5, box))):
        np.add.at(ref, bins, alpha2 ** 2 * rw2[i] * rw2[js])
    np.testing.assert_allclose(est2.extra["rr"], ref, rtol=1e-12)


# ------------------------------------------------------ varying line of sight
def test_varying_los_vs_brute_force_with_scipy_frames(ora):
    """NNN^m with the line of sight from an observer to each primary equals the
    brute-force triplet sum in frames from scipy's Rotation.align_vectors (a
    different azimuth about the line of sight, to which NNN^m is blind)."""
    from scipy.spatial.transform import Rotation
    box = 150.0
    xyz, w = _dense_tiny(21, n=150)
    w = w.astype(np.float64)
    w[::4] = -0.5
    obs = (-0.7 * box, 0.3 * box, 1.6 * box)
    cfg = ora.Config(10.0, 45.0, 4, 3, (0, 2), False, box, los="observer", observer=obs)
    E, _ = ora.edges(cfg)
    o = ora.run(cfg, xyz, w, nthreads=2)
    ou = np.array(obs) / box * 2.0 ** 32

    def frame(i):
        n = xyz[i].astype(np.float64) - ou
        return Rotation.align_vectors([[0.0, 0.0, 1.0]], [n / np.linalg.norm(n)])[0].as_matrix()

    nnn, _, _ = bf.triplets(xyz, w, False, E, cfg.n_bins, cfg.l_max, frame=frame)
    assert np.abs(o.nnn - nnn).max() <= 1e-11 * np.abs(nnn).max()
    fixed = ora.run(ora.Config(10.0, 45.0, 4, 3, (0, 2), False, box), xyz, w, nthreads=2)
    assert np.abs(o.nnn - fixed.nnn).max() > 1e-3 * np.abs(nnn).max()   # the frames matter


def test_distant_observer_on_the_z_axis_is_the_fixed_los(ora):
    box = 150.0
    xyz, w = _dense_tiny(22, n=150)
    base = dict(r_min=10.0, r_max=45.0, n_bins=4, l_max=3, Ls=(0, 2), periodic=False, box=box)
    far = ora.run(ora.Config(**base, los="observer", observer=(0.5 * box, 0.5 * box, -1e7 * box)), xyz, w)
    fixed = ora.run(ora.Config(**base), xyz, w)
    assert np.abs(far.nnn - fixed.nnn).max() <= 1e-6 * np.abs(fixed.nnn).max()


def test_varying_los_is_rotation_invariant(ora):
    """Cycling the axes of the catalogue and of the observer (exact in fixed point)
    leaves the varying-LOS multipoles unchanged; the fixed-z ones change."""
    box = 150.0
    d, _ = synth.lognormal(1200, box, 23, mesh=32)
    w = np.ones(d.shape[0])
    obs = (0.2 * box, -1.1 * box, 0.4 * box)
    cyc = np.ascontiguousarray(d[:, [2, 0, 1]])        # (x, y, z) -> (z, x, y)
    obs_c = (obs[2], obs[0], obs[1])
    base = dict(r_min=10.0, r_max=40.0, n_bins=3, l_max=2, Ls=(0, 2), periodic=False, box=box)
    a = ora.run(ora.Config(**base, los="observer", observer=obs), d, w, nthreads=4).nnn
    b = ora.run(ora.Config(**base, los="observer", observer=obs_c), cyc, w, nthreads=4).nnn
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    fa = ora.run(ora.Config(**base), d, w, nthreads=4).nnn
    fb = ora.run(ora.Config(**base), cyc, w, nthreads=4).nnn
    assert np.abs(fa - fb).max() > 1e-3 * np.abs(fa).max()
