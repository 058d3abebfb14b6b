"""Brute-force triplet sums on tiny catalogues, used only to pin the oracle.

Independent of the oracle's own arithmetic: neighbours come from an O(N^2)
exact-integer distance matrix, spherical harmonics from scipy, 3j symbols from
sympy (exact), Legendre polynomials from scipy, and every j != k pair of
secondaries is enumerated explicitly (the diagonal of the pair matrix is
removed), as the definition of a triplet count states.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sps

if hasattr(sps, "sph_harm_y"):  # scipy >= 1.15: (l, m, polar, azimuth)
    def sph_y(l, m, theta, phi):
        return sps.sph_harm_y(l, m, theta, phi)
else:  # pragma: no cover - older scipy: (m, l, azimuth, polar)
    def sph_y(l, m, theta, phi):
        return sps.sph_harm(m, l, phi, theta)


def w3j_exact(j1, j2, j3, m1, m2, m3) -> float:
    from sympy.physics.wigner import wigner_3j
    return float(wigner_3j(j1, j2, j3, m1, m2, m3))


def exact_edges(r_min, r_max, n_bins, box):
    """ceil(s_b^2) with exact rational arithmetic on the same FP64 s_b."""
    from fractions import Fraction
    out = []
    for b in range(n_bins + 1):
        r = r_min + ((r_max - r_min) * b) / n_bins
        s = (r * 4294967296.0) / box
        out.append(math.ceil(Fraction(s) ** 2))
    return out


def neighbours(xyz, periodic, E):
    """All (i, j, bin, dvec) with E_0 <= r^2 < E_nb, by brute force."""
    u = np.asarray(xyz, dtype=np.uint32)
    n = u.shape[0]
    out = []
    Eu = np.array([int(e) for e in E], dtype=np.uint64)
    for i in range(n):
        if periodic:
            d = (u - u[i]).view(np.int32).astype(np.int64)
        else:
            d = u.astype(np.int64) - u[i].astype(np.int64)
        near = (np.abs(d) < 2**31).all(axis=1)      # farther pairs are beyond r_max < L/2
        d = np.where(near[:, None], d, 0)
        r2 = (d[:, 0] * d[:, 0]).astype(np.uint64) + (d[:, 1] * d[:, 1]).astype(np.uint64) \
            + (d[:, 2] * d[:, 2]).astype(np.uint64)
        ok = np.nonzero(near & (r2 >= Eu[0]) & (r2 < Eu[-1]))[0]
        ok = ok[ok != i]
        bins = np.searchsorted(Eu, r2[ok], side="right").astype(np.int64) - 1
        out.append((ok, bins, d[ok].astype(np.float64)))
    return out


def dirs(d):
    r = np.sqrt((d * d).sum(axis=1))
    v = d / r[:, None]
    theta = np.arccos(np.clip(v[:, 2], -1, 1))
    phi = np.arctan2(v[:, 1], v[:, 0])
    return v, theta, phi


def triplets(xyz, w, periodic, E, n_bins, lmax, prim=None, frame=None):
    """Brute-force NNN^m_{l1 l2}[b1][b2] = sum_i w_i sum_{j != k} w_j w_k Y Y*,
    the addition-theorem sums A_l = sum_i w_i sum_{j != k} w_j w_k P_l(r_j . r_k),
    and the integer triplet counts.  frame(i), if given, is a 3 x 3 matrix that
    turns primary i's separations into the frame their harmonics are taken in."""
    w = np.asarray(w, dtype=np.float64)
    nb = n_bins
    L = lmax
    nnn = np.zeros((2 * L + 1, L + 1, L + 1, nb, nb), dtype=np.complex128)
    leg = np.zeros((L + 1, nb, nb))
    trip = np.zeros((nb, nb), dtype=np.int64)
    nbl = neighbours(xyz, periodic, E)
    prims = range(len(nbl)) if prim is None else prim
    for i in prims:
        ok, bins, d = nbl[i]
        if ok.size == 0:
            continue
        if frame is not None:
            d = d @ np.asarray(frame(i)).T
        v, th, ph = dirs(d)
        wj = w[ok]
        B = np.zeros((ok.size, nb))
        B[np.arange(ok.size), bins] = 1.0
        offd = 1.0 - np.eye(ok.size)
        trip += np.rint(B.T @ offd @ B).astype(np.int64)
        cosg = np.clip(v @ v.T, -1.0, 1.0)
        for l in range(L + 1):
            F = np.outer(wj, wj) * sps.eval_legendre(l, cosg) * offd
            leg[l] += w[i] * (B.T @ F @ B)
        Y = {}
        for l in range(L + 1):
            for m in range(-l, l + 1):
                Y[(l, m)] = sph_y(l, m, th, ph)
        for m in range(-L, L + 1):
            for l1 in range(abs(m), L + 1):
                for l2 in range(abs(m), L + 1):
                    F = np.outer(wj * Y[(l1, m)], np.conj(wj * Y[(l2, m)])) * offd
                    nnn[m + L, l1, l2] += w[i] * (B.T @ F @ B)
    return nnn, leg, trip


def tsh_sum(xyz, w, periodic, E, n_bins, l1, l2, LL):
    """sum_i w_i sum_{j != k} w_j w_k S_{l1 l2 L}(r_j, r_k, z) from the TripoSH
    definition with Schmidt semi-normalised y_l^m = sqrt(4 pi/(2l+1)) Y_l^m."""
    w = np.asarray(w, dtype=np.float64)
    nb = n_bins
    out = np.zeros((nb, nb))
    H = w3j_exact(l1, l2, LL, 0, 0, 0)
    nbl = neighbours(xyz, periodic, E)
    c1 = math.sqrt(4 * math.pi / (2 * l1 + 1))
    c2 = math.sqrt(4 * math.pi / (2 * l2 + 1))
    cL = math.sqrt(4 * math.pi / (2 * LL + 1))
    yL_z = {M: cL * sph_y(LL, M, 0.0, 0.0) for M in range(-LL, LL + 1)}
    for i, (ok, bins, d) in enumerate(nbl):
        if ok.size == 0:
            continue
        _, th, ph = dirs(d)
        wj = w[ok]
        B = np.zeros((ok.size, nb))
        B[np.arange(ok.size), bins] = 1.0
        S = np.zeros((ok.size, ok.size), dtype=np.complex128)
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                M = -m1 - m2
                if abs(M) > LL:
                    continue
                c = w3j_exact(l1, l2, LL, m1, m2, M)
                if c == 0.0:
                    continue
                S += c * np.outer(c1 * sph_y(l1, m1, th, ph), c2 * sph_y(l2, m2, th, ph)) * yL_z[M]
        S = S / H
        F = np.outer(wj, wj) * S.real * (1.0 - np.eye(ok.size))
        out += w[i] * (B.T @ F @ B)
    return out
