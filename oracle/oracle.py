"""Plain FP64 CPU oracle of the anisotropic 3PCF estimator (Python side).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke() and the benchmark's
CPU-baseline / reference leg are the only callers.  Nothing here is shared
with, imported by, or imports the CUDA path.

The heavy loop (neighbour search, a_l^m, the local products) lives in
``tpcf_oracle.c``; this module builds and loads it, assembles the
data-minus-random field, forms the normaliser and applies the TripoSH
projection of Eq. slep2sugy:

    zeta_{l1 l2 L}(r1, r2) = (2L+1) H_{l1 l2 L}
        sum_m (l1 l2 L; m -m 0) (-1)^m zeta^m_{l1 l2}(r1, r2),

with H_{l1 l2 L} = (l1 l2 L; 0 0 0) (Sec. 2.2, TripoSH basis) and
zeta^m = NNN^m / RRR_{00}^0 (Eq. ssest: (D-R)^3 / R^3, bin-wise by the l = 0
random triplet count).

Readings of the paper recorded here:
  * the second a_l^m of Eq. measured_mult is conjugated (Eq. zeta_meas puts
    Y* on r_hat_2);
  * degenerate j = k triangles are removed (remove_self = 1);
  * periodic boxes use analytic randoms: a_0^0[b] is offset by
    c_b = (W - 1)/L^3 V_b Y_0^0 and RRR_00^0[b1][b2] = W c_b1 c_b2;
  * non-periodic volumes use explicit randoms with weights -W_D/W_R, and
    RRR_00^0 from the randoms alone with weights +W_D/W_R;
  * the 2PCF multipoles (Eq. xi_meas_leg) take P_l(mu) of every pair exactly
    (the limit of vanishing mu bins), share the 3PCF's radial bins, and use
    the natural estimator (Eq. xi_natest) on the same D - R field, i.e.
    (DD - 2DR + RR) / RR with explicit randoms;
  * the full edge correction (``edge="full"``, for explicit randoms) solves
    N = zeta R for zeta on the real, l1 + l2 even coefficients (the ones the
    L-even multipoles use), dropping the imaginary and odd-parity parts of
    RRR, which vanish for a random catalogue symmetric under the reflections
    z -> -z and y -> -y and are shot noise otherwise;
  * ``los="observer"`` replaces the fixed z line of sight (Sec. 4.1) by the
    direction from an observer to each primary: every separation is turned
    by R_y(-theta_i) R_z(-phi_i), which takes that direction to z, before
    its harmonics are taken (the coupling and projection are unchanged);
  * ``convention="PAPER_EQ"`` is Eq. slep2sugy as printed with orthonormal
    Y; ``"S_COEFF"`` (default) multiplies it by sqrt((2 l1 + 1)(2 l2 + 1)), the
    coefficient of the Schmidt-normalised basis function S_{l1 l2 L} of
    Eq. TSHbasis.
"""
from __future__ import annotations

import ctypes
import functools
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpcf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("r_min", ctypes.c_double), ("r_max", ctypes.c_double),
                ("n_bins", ctypes.c_int32), ("l_max", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("remove_self", ctypes.c_int32),
                ("box", ctypes.c_double), ("offset_weight", ctypes.c_double),
                ("los_mode", ctypes.c_int32), ("observer", ctypes.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.ora_run.argtypes = [ctypes.POINTER(_Cfg), P, P, ctypes.c_int64, P, ctypes.c_int64,
                              P, P, P, P, P, P, P, ctypes.c_int]
        L.ora_run.restype = ctypes.c_int
        L.ora_edges.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, P, P]
        L.ora_edges.restype = None
        L.ora_wigner3j.argtypes = [ctypes.c_int] * 6
        L.ora_wigner3j.restype = ctypes.c_double
        L.ora_ylm.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int, P]
        L.ora_ylm.restype = None
        L.ora_max_threads.argtypes = []
        L.ora_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


@dataclass
class Config:
    r_min: float
    r_max: float
    n_bins: int
    l_max: int
    Ls: tuple = (0, 2, 4)
    periodic: bool = True
    box: float = 500.0
    remove_self: bool = True
    convention: str = "S_COEFF"
    los: str = "z"               # "z": fixed line of sight; "observer": from observer to primary
    observer: tuple = (0.0, 0.0, 0.0)   # observer position (length units, box coordinates)


def edges(cfg: Config):
    """(E uint64 [nb+1], r float64 [nb+1]): exact integer edges^2 and physical edges."""
    E = np.zeros(cfg.n_bins + 1, dtype=np.uint64)
    r = np.zeros(cfg.n_bins + 1, dtype=np.float64)
    lib().ora_edges(cfg.r_min, cfg.r_max, cfg.n_bins, cfg.box, _p(E), _p(r))
    return E, r


def wigner3j(j1, j2, j3, m1, m2, m3) -> float:
    return lib().ora_wigner3j(j1, j2, j3, m1, m2, m3)


def ylm(vec, lmax):
    """Orthonormal complex Y_l^m at a unit vector, index l*l + l + m."""
    out = np.zeros((lmax + 1) ** 2, dtype=np.complex128)
    lib().ora_ylm(float(vec[0]), float(vec[1]), float(vec[2]), lmax, _p(out))
    return out


def multipoles(l_max: int, Ls) -> list:
    """(l1, l2, L) kept by the TripoSH projection: triangle rule and even l1+l2+L."""
    out = []
    for L in Ls:
        for l1 in range(l_max + 1):
            for l2 in range(l_max + 1):
                if abs(l1 - l2) <= L <= l1 + l2 and (l1 + l2 + L) % 2 == 0:
                    out.append((l1, l2, L))
    return out


def shell_offsets(cfg: Config, weight_sum: float):
    """c_b = (W - 1)/L^3 * V_b * Y_0^0 with V_b the volume of radial shell b."""
    _, r = edges(cfg)
    nbar = (weight_sum - 1.0) / cfg.box ** 3
    vb = 4.0 * math.pi / 3.0 * (r[1:] ** 3 - r[:-1] ** 3)
    return nbar * vb / math.sqrt(4.0 * math.pi)


@dataclass
class RunOut:
    nnn: np.ndarray            # complex [2L+1][L+1][L+1][nb][nb], m index m + L
    pair_counts: np.ndarray    # int64 [nb]
    trip_counts: np.ndarray    # int64 [nb][nb]
    alm: np.ndarray | None = None   # complex [n_prim][nb][(L+1)^2]
    cnt: np.ndarray | None = None   # int32 [n_prim][nb]


def run(cfg: Config, xyz, w, offset_weight=-1.0, prim=None, want_alm=False, nthreads=0,
        l_max=None) -> RunOut:
    """One pass of the estimator loop over a single signed-weight field."""
    L = cfg.l_max if l_max is None else l_max
    xyz = np.ascontiguousarray(xyz, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = xyz.shape[0]
    nb = cfg.n_bins
    if cfg.los not in ("z", "observer"):
        raise ValueError(cfg.los)
    obs = (ctypes.c_double * 3)(*[float(v) / cfg.box * 4294967296.0 for v in cfg.observer])
    c = _Cfg(cfg.r_min, cfg.r_max, nb, L, int(cfg.periodic), int(cfg.remove_self), cfg.box,
             float(offset_weight), 1 if cfg.los == "observer" else 0, obs)
    nm = 2 * L + 1
    re = np.zeros((nm, L + 1, L + 1, nb, nb))
    im = np.zeros_like(re)
    pc = np.zeros(nb, dtype=np.int64)
    tc = np.zeros((nb, nb), dtype=np.int64)
    pr = None
    npr = 0
    if prim is not None:
        pr = np.ascontiguousarray(prim, dtype=np.int64)
        npr = pr.shape[0]
    nlm = (L + 1) ** 2
    ar = ai = cn = None
    if want_alm:
        k = npr if prim is not None else n
        ar = np.zeros((k, nb, nlm))
        ai = np.zeros((k, nb, nlm))
        cn = np.zeros((k, nb), dtype=np.int32)
    rc = lib().ora_run(ctypes.byref(c), _p(xyz), _p(w), n, _p(pr), npr,
                       _p(re), _p(im), _p(pc), _p(tc), _p(ar), _p(ai), _p(cn), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    out = RunOut(re + 1j * im, pc, tc)
    if want_alm:
        out.alm = ar + 1j * ai
        out.cnt = cn
    return out


def project(cfg: Config, nnn: np.ndarray, rrr: np.ndarray, mults=None, l_max=None):
    """Eq. slep2sugy applied bin by bin, divided by RRR_00^0; returns (real, imag)."""
    L = cfg.l_max if l_max is None else l_max
    mults = multipoles(L, cfg.Ls) if mults is None else mults
    nb = cfg.n_bins
    z = np.zeros((len(mults), nb, nb), dtype=np.complex128)
    for k, (l1, l2, LL) in enumerate(mults):
        H = wigner3j(l1, l2, LL, 0, 0, 0)
        s = np.zeros((nb, nb), dtype=np.complex128)
        for m in range(-min(l1, l2), min(l1, l2) + 1):
            s += wigner3j(l1, l2, LL, m, -m, 0) * (-1.0) ** m * nnn[m + L, l1, l2]
        v = (2 * LL + 1) * H * s / rrr
        if cfg.convention == "S_COEFF":
            v = v * math.sqrt((2 * l1 + 1) * (2 * l2 + 1))
        elif cfg.convention != "PAPER_EQ":
            raise ValueError(cfg.convention)
        z[k] = v
    return z.real, z.imag


@dataclass
class Estimate:
    zeta: np.ndarray
    zeta_imag: np.ndarray
    mults: list
    nnn: np.ndarray
    rrr: np.ndarray
    pair_counts: np.ndarray
    trip_counts: np.ndarray
    extra: dict = field(default_factory=dict)


def m0_sums(alm, w, L, step=2):
    """S_l[b] = sum_i w_i Re a_l^0[b](x_i) for l = 0, step, ..., L: the weighted
    pair sums sum_{i != j in b} w_i w_j Y_l^0(r_hat_ij) behind the Legendre
    multipoles of Eq. xi_meas_leg (Y_l^0 = sqrt((2l+1)/4pi) P_l(mu), mu the
    cosine to the z line of sight)."""
    w = np.asarray(w, dtype=np.float64)
    return np.array([w @ alm[:, :, l * l + l].real for l in range(0, L + 1, step)])


def xi_multipoles(S, rr, step=2):
    """Eq. xi_meas_leg in the limit of vanishing mu bins, with the natural
    estimator of Eq. xi_natest generalised to the D - R field:
    xi_l[b] = (2l+1) sum_pairs w w P_l(mu) / RR_b = sqrt(4pi (2l+1)) S_l[b] / RR_b,
    with RR_b the (isotropic) weighted random pair count of bin b."""
    out = np.zeros_like(S)
    for e in range(S.shape[0]):
        l = step * e
        out[e] = math.sqrt(4.0 * math.pi * (2 * l + 1)) * S[e] / rr
    return out


def estimate(cfg: Config, d_xyz, d_w, r_xyz=None, r_w=None, nthreads=0, want_xi=False,
             edge="binwise") -> Estimate:
    """Full estimator: (D - R)^3 / R^3 multipoles (Eq. ssest with Eq. slep2sugy).

    Without randoms (periodic only) the analytic-random form is used.  With
    want_xi the even 2PCF multipoles xi_l, l = 0, 2, ..., l_max, of the same
    field and radial bins go to extra["xi"] (their normaliser RR_b to
    extra["rr"])."""
    d_w = np.asarray(d_w, dtype=np.float64)
    WD = float(d_w.sum())
    if r_xyz is None:
        if not cfg.periodic:
            raise ValueError("analytic randoms need a periodic box")
        w = d_w
        o = run(cfg, d_xyz, d_w, offset_weight=WD, nthreads=nthreads, want_alm=want_xi)
        cb = shell_offsets(cfg, WD)
        rrr = WD * np.outer(cb, cb)
        # analytic RR_b = W (W - 1) V_b / L^3
        rr = WD * math.sqrt(4.0 * math.pi) * cb
    else:
        r_w = np.asarray(r_w, dtype=np.float64)
        alpha = WD / float(r_w.sum())
        xyz = np.concatenate([np.asarray(d_xyz, np.uint32), np.asarray(r_xyz, np.uint32)])
        w = np.concatenate([d_w, -alpha * r_w])
        o = run(cfg, xyz, w, nthreads=nthreads, want_alm=want_xi)
        orr = run(cfg, r_xyz, alpha * r_w, nthreads=nthreads, l_max=0, want_alm=want_xi)
        rrr = orr.nnn[0, 0, 0].real
        if want_xi:
            # sum over ordered random pairs of alpha^2 w_i w_j, from the l = 0 sums
            rr = math.sqrt(4.0 * math.pi) * m0_sums(orr.alm, alpha * r_w, 0)[0]
    mults = multipoles(cfg.l_max, cfg.Ls)
    if edge == "full":
        # the full anisotropic edge correction: RRR^m_{l1 l2} of the randoms at l_max
        if r_xyz is None:
            raise ValueError("the full edge correction needs explicit randoms")
        rfull = run(cfg, r_xyz, alpha * r_w, nthreads=nthreads).nnn
        zhat = edge_correct(o.nnn, rfull, cfg.l_max)
        zr, zi = project(cfg, zhat, np.ones_like(rrr), mults)
        est = Estimate(zr, zi, mults, o.nnn, rrr, o.pair_counts, o.trip_counts)
        est.extra["rrr_full"] = rfull
        est.extra["zeta_hat"] = zhat
    elif edge == "binwise":
        zr, zi = project(cfg, o.nnn, rrr, mults)
        est = Estimate(zr, zi, mults, o.nnn, rrr, o.pair_counts, o.trip_counts)
    else:
        raise ValueError(edge)
    if want_xi:
        est.extra["xi"] = xi_multipoles(m0_sums(o.alm, w, cfg.l_max), rr)
        est.extra["rr"] = rr
    return est


def gaunt(l1: int, m1: int, l2: int, m2: int, l3: int) -> float:
    """int Y_l1^m1 Y_l2^m2 (Y_l3^(m1+m2))* dOmega, the coefficient of Y_l3^(m1+m2)
    in the product Y_l1^m1 Y_l2^m2 (real for orthonormal Y)."""
    m3 = m1 + m2
    if abs(m1) > l1 or abs(m2) > l2 or abs(m3) > l3:
        return 0.0
    pre = math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4.0 * math.pi))
    return pre * wigner3j(l1, l2, l3, 0, 0, 0) * wigner3j(l1, l2, l3, m1, m2, -m3) * (-1.0) ** m3


def edge_modes(L: int) -> list:
    """(l1, l2, m), m >= 0, l1, l2 in [m, L], l1 + l2 even: the real coefficients the
    edge-correction system is solved for (its unknowns and its equations)."""
    return [(l1, l2, m) for m in range(L + 1) for l1 in range(m, L + 1) for l2 in range(m, L + 1)
            if (l1 + l2) % 2 == 0]


@functools.lru_cache(maxsize=None)
def _edge_terms(L: int):
    """The nonzero Gaunt products of the coupling matrix (they do not depend on
    the bins): (row, column, m'', l1'', l2'', gaunt * gaunt)."""
    modes = edge_modes(L)
    terms = []
    for r, (l1, l2, m) in enumerate(modes):
        for c, (p1, p2, mp) in enumerate(modes):
            for mq in ((mp, -mp) if mp > 0 else (0,)):
                mr = m - mq
                if abs(mr) > L:
                    continue
                for q1 in range(abs(mr), L + 1):
                    for q2 in range(abs(mr), L + 1):
                        if (q1 + q2) % 2:
                            continue
                        g = gaunt(p1, mq, q1, mr, l1) * gaunt(p2, mq, q2, mr, l2)
                        if g != 0.0:
                            terms.append((r, c, mr, q1, q2, g))
    return modes, terms


def edge_matrix(rrr_real, L: int):
    """The coupling matrix of N = zeta R in the basis Y_l1^m(r1) Y_l2^m*(r2).

    Functions of (r_hat_1, r_hat_2) about the fixed line of sight expand as
    F = sum_{l1 l2 m} F^m_{l1 l2} Y_l1^m(r_hat_1) Y_l2^m*(r_hat_2); a product
    couples them through one Gaunt coefficient per angle:
      (F G)^m_{l1 l2} = sum F^m'_{l1' l2'} G^(m-m')_{l1'' l2''}
                        gaunt(l1', m', l1'', m-m', l1) gaunt(l2', m', l2'', m-m', l2).
    The unknowns are real with zeta^-m = zeta^m, so the columns of +m' and -m'
    are added.  rrr_real[m][l1][l2][...] (m = -L..L at index m + L; any trailing
    bin axes) holds Re RRR^m.  The factor 4 pi makes the solution the
    bin-wise-normalised zeta_hat^m = zeta^m / 4 pi, which equals
    NNN^m / RRR_00^0 for isotropic R.  Returns (modes, M[row][col][...])."""
    modes, terms = _edge_terms(L)
    M = np.zeros((len(modes), len(modes)) + rrr_real.shape[3:])
    for r, c, mr, q1, q2, g in terms:
        M[r, c] += g * rrr_real[mr + L, q1, q2]
    return modes, 4.0 * math.pi * M


def edge_correct(nnn, rrr, L: int):
    """Solves Re NNN^m_{l1 l2} = sum M (zeta_hat) bin pair by bin pair (N = zeta R
    with the full anisotropic RRR^m_{l1 l2} of the randoms, truncated at l_max)
    on the real, l1 + l2 even coefficients; returns zeta_hat in the layout of
    nnn (complex [2L+1][L+1][L+1][nb][nb], zeta_hat^-m = zeta_hat^m, zero
    outside the solved modes)."""
    nb = nnn.shape[-1]
    out = np.zeros(nnn.shape, dtype=np.complex128)
    modes, M = edge_matrix(rrr.real, L)
    for b1 in range(nb):
        for b2 in range(nb):
            rhs = np.array([nnn[m + L, l1, l2, b1, b2].real for (l1, l2, m) in modes])
            z = np.linalg.solve(M[:, :, b1, b2], rhs)
            for (l1, l2, m), v in zip(modes, z):
                out[m + L, l1, l2, b1, b2] = v
                out[-m + L, l1, l2, b1, b2] = v
    return out


def max_threads() -> int:
    return lib().ora_max_threads()
