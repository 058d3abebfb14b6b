"""Plain FP64 tree-level model of the anisotropic halo 3PCF multipoles (Sec. 2.3-2.5
of arXiv:2408.03036): the reference that the MLP emulator is trained on and judged
against.

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke() and the benchmark's
CPU-baseline leg are the only callers; nothing in the CUDA library imports it.

Steps, in the paper's order:
  1. linear power spectrum without wiggles, P_w = 0 (Eq. Pk_IR with no BAO part):
     BBKS transfer function with the Sugiyama shape parameter, n_s tilt,
     normalised to sigma_8 = 1 in spheres of 8 Mpc/h (sigma_8 scales P by sigma_8^2);
  2. redshift-space kernels Z_1 = b_1 + f mu^2 and the second-order Z_2 with the
     density and velocity kernels F_2, G_2 and local bias b_2 (b_G2 = 0);
  3. the tree-level bispectrum of Eq. bisp, three cyclic terms;
  4. Alcock-Paczynski and isotropic dilation (Eqs. k_prime, mu_prime): every
     wavevector is mapped by k_par' = k_par / (alpha (1+eps)^2),
     k_perp' = k_perp (1+eps) / alpha, and B_obs = B(k') / alpha^6;
  5. TripoSH coefficients B_{l1 l2 L}(k1, k2) of Eq. TripoSH, by projecting on
     S_{l1 l2 L} (Eq. TSHbasis) with the orthogonality of the S basis,
     <S S'> = delta / (H^2 (2 l1 + 1)(2 l2 + 1)(2 L + 1)), evaluated by quadrature
     in the frame of Eq. Scoord1 (k1 along z, k2 in the x-z plane, n over the
     sphere);
  6. the 2D Hankel transform of Eq. TriRelBtoZ, bin-averaged over radial bins
     with r^2 weights, as a separable quadrature: B_{l1 l2 L} on nodes in k
     (logarithmic, then linear) is interpolated by cubic splines in ln k and the
     oscillating bin-averaged Bessel factors are integrated against those spline
     basis functions (Gauss-Legendre inside every interval).
The model is a polynomial in (b1, b2, f) times sigma_8^4 for fixed (alpha, eps):
zeta = sigma_8^4 sum_t c_t(b1, b2, f) T_t(alpha, eps), with the 11 monomials c_t
listed in MONOMIALS; TemplateModel tabulates T_t on an (alpha, eps) grid and
interpolates bicubically (the template approach of Sec. 2.5).

Readings (the paper names the Minerva cosmology and an analytic no-wiggle P(k)
without listing numbers): Omega_m = 0.285, Omega_b h^2 = 0.02247, h = 0.695,
n_s = 0.9632; b_G2 = 0; eps is the AP warp with 1 + eps in [0.95, 1.05].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import roots_legendre, spherical_jn, sph_harm_y

from oracle.oracle import wigner3j

OMEGA_M, OMEGA_B_H2, H0, N_S = 0.285, 0.02247, 0.695, 0.9632

# multipoles of the emulator output: l1, l2 <= 4, L in {0, 2}, both (l1, l2) orders
MULTIPOLES = [(l1, l2, L) for L in (0, 2) for l1 in range(5) for l2 in range(5)
              if (l1 + l2 + L) % 2 == 0 and abs(l1 - l2) <= L <= l1 + l2]

# monomials in (b1, b2, f) of the tree-level bispectrum (exponents of b1, b2, f)
MONOMIALS = [(3, 0, 0), (2, 0, 1), (3, 0, 1), (2, 0, 2), (2, 1, 0), (1, 0, 2), (1, 0, 3), (1, 1, 1),
             (0, 0, 3), (0, 0, 4), (0, 1, 2)]


# ---------------------------------------------------------------- 1. power spectrum

def bbks_transfer(k):
    """BBKS transfer function (Bardeen et al. 1986) with the Sugiyama (1995) shape
    Gamma = Omega_m h exp(-Omega_b (1 + sqrt(2 h) / Omega_m)); k in h/Mpc."""
    ob = OMEGA_B_H2 / H0 ** 2
    gamma = OMEGA_M * H0 * math.exp(-ob * (1.0 + math.sqrt(2.0 * H0) / OMEGA_M))
    q = np.asarray(k, dtype=np.float64) / gamma
    return (np.log1p(2.34 * q) / (2.34 * q)
            * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)


def _sigma_r(pk, R=8.0):
    k = np.logspace(-5, 3, 20001)
    x = k * R
    wth = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    f = k ** 3 * pk(k) * wth ** 2 / (2.0 * math.pi ** 2)
    return math.sqrt(np.trapezoid(f, np.log(k)))


class PowerNW:
    """P_nw(k) = A k^n_s T(k)^2 with sigma_8 = 1."""

    def __init__(self):
        self.A = 1.0
        self.A = 1.0 / _sigma_r(self) ** 2

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        return self.A * k ** N_S * bbks_transfer(k) ** 2


# ---------------------------------------------------------------- 2-4. bispectrum

def _kernel_parts(ka, kb, c_ab, ma, mb, mab, kab):
    """Z_1 Z_1 Z_2 of one cyclic term split by monomial (Eq. bisp): returns the
    coefficient arrays of the 11 MONOMIALS (without the factor 2 P_a P_b).
    ka, kb: magnitudes; c_ab: cosine between them; ma, mb: LOS cosines;
    mab, kab: LOS cosine and magnitude of k_a + k_b."""
    r = ka / kb + kb / ka
    F2 = 5.0 / 7.0 + 0.5 * c_ab * r + 2.0 / 7.0 * c_ab ** 2
    G2 = 3.0 / 7.0 + 0.5 * c_ab * r + 4.0 / 7.0 * c_ab ** 2
    mk = mab * kab                     # (k_a + k_b) . n
    # Z2 = b1 F2 + f mu^2 G2 + f b1 (mk/2)(ma/ka + mb/kb) + f^2 (mk/2)(ma mb^2/ka + mb ma^2/kb) + b2/2
    z2_b1, z2_f, z2_fb1 = F2, mab ** 2 * G2, 0.5 * mk * (ma / ka + mb / kb)
    z2_f2, z2_b2 = 0.5 * mk * (ma * mb ** 2 / ka + mb * ma ** 2 / kb), 0.5
    # Z1 Z1 = b1^2 + b1 f (ma^2 + mb^2) + f^2 ma^2 mb^2
    y_b1b1, y_b1f, y_ff = 1.0, ma ** 2 + mb ** 2, ma ** 2 * mb ** 2
    one = np.ones_like(F2)
    out = {}

    def add(key, v):
        out[key] = out.get(key, 0.0) + v

    for (yk, yv) in (((2, 0, 0), y_b1b1 * one), ((1, 0, 1), y_b1f), ((0, 0, 2), y_ff)):
        for (zk, zv) in (((1, 0, 0), z2_b1), ((0, 0, 1), z2_f), ((1, 0, 1), z2_fb1), ((0, 0, 2), z2_f2),
                         ((0, 1, 0), z2_b2 * one)):
            add((yk[0] + zk[0], yk[1] + zk[1], yk[2] + zk[2]), yv * zv)
    return [out.get(m, 0.0 * one) for m in MONOMIALS]


def ap_map(kv, n, alpha, eps):
    """Wavevector seen through the AP distortion: the component along n divided by
    alpha (1 + eps)^2, the perpendicular part by alpha / (1 + eps); its length and
    LOS cosine are those of Eqs. k_prime and mu_prime."""
    apar, aperp = alpha * (1.0 + eps) ** 2, alpha / (1.0 + eps)
    kp = np.sum(kv * n, axis=-1, keepdims=True)
    return (kv - kp * n) / aperp + (kp / apar) * n


def bispectrum_monomials(k1v, k2v, n, pk, alpha=1.0, eps=0.0):
    """Tree-level redshift-space bispectrum with AP, per monomial (sigma_8 = 1):
    array [11, ...].  k1v, k2v: [..., 3] wavevectors; n: [..., 3] unit LOS."""
    vs = [ap_map(k1v, n, alpha, eps), ap_map(k2v, n, alpha, eps)]
    vs.append(-vs[0] - vs[1])
    mags = [np.linalg.norm(v, axis=-1) for v in vs]
    mus = [np.sum(v * n, axis=-1) / m for v, m in zip(vs, mags)]
    P = [pk(m) for m in mags]
    tot = None
    for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        cab = np.sum(vs[a] * vs[b], axis=-1) / (mags[a] * mags[b])
        # k_a + k_b = -k_c: its LOS cosine is -mu_c, its magnitude |k_c|
        parts = _kernel_parts(mags[a], mags[b], cab, mus[a], mus[b], -mus[c], mags[c])
        term = np.stack([2.0 * p * P[a] * P[b] for p in parts])
        tot = term if tot is None else tot + term
    return tot / alpha ** 6


# ---------------------------------------------------------------- 5. TripoSH projection

def schmidt_y(l, m, theta, phi):
    """Schmidt semi-normalised y_l^m = sqrt(4 pi / (2l + 1)) Y_l^m (complex)."""
    return math.sqrt(4.0 * math.pi / (2 * l + 1)) * sph_harm_y(l, m, theta, phi)


def s_basis(l1, l2, L, th1, ph1, th2, ph2, thn, phn):
    """S_{l1 l2 L}(k1, k2, n) of Eq. TSHbasis (real for l1 + l2 + L even)."""
    H = wigner3j(l1, l2, L, 0, 0, 0)
    s = 0.0
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            M = -m1 - m2
            if abs(M) > L:
                continue
            c = wigner3j(l1, l2, L, m1, m2, M)
            if c == 0.0:
                continue
            s = s + c * schmidt_y(l1, m1, th1, ph1) * schmidt_y(l2, m2, th2, ph2) * schmidt_y(L, M, thn, phn)
    return np.real(s) / H


@dataclass
class AngularGrid:
    """Frame of Eq. Scoord1: k1 = z, k2 = (sin t, 0, cos t), n over the sphere;
    composite Gauss-Legendre in cos t (n_t nodes over the panels T_PANELS),
    Gauss-Legendre in cos(beta), uniform in phi.  weights sum to 1."""
    n_t: int = 32
    n_b: int = 12
    n_p: int = 12

    # panels in cos t, crowded towards -1 where k3 = |k1 + k2| -> 0 for k1 = k2
    T_PANELS = (-1.0, -0.999, -0.99, -0.9, -0.5, 0.2, 1.0)

    def build(self, mults):
        per = max(2, self.n_t // (len(self.T_PANELS) - 1))
        x0, w0 = roots_legendre(per)
        xt, wt = [], []
        for a, b in zip(self.T_PANELS[:-1], self.T_PANELS[1:]):
            xt.append(0.5 * (b - a) * x0 + 0.5 * (a + b))
            wt.append(0.5 * (b - a) * w0)
        xt, wt = np.concatenate(xt), np.concatenate(wt)
        xb, wb = roots_legendre(self.n_b)
        ph = (np.arange(self.n_p) + 0.5) * 2.0 * math.pi / self.n_p
        T, B, Pn = np.meshgrid(xt, xb, ph, indexing="ij")
        W = (np.meshgrid(wt, wb, np.full(self.n_p, 1.0 / self.n_p), indexing="ij"))
        self.w = (W[0] * W[1] * W[2] / 4.0).ravel()            # (1/2)(1/2) GL normalisation
        ct, cb, ph = T.ravel(), B.ravel(), Pn.ravel()
        st, sb = np.sqrt(1 - ct ** 2), np.sqrt(1 - cb ** 2)
        self.k2hat = np.stack([st, 0 * st, ct], axis=-1)
        self.n = np.stack([sb * np.cos(ph), sb * np.sin(ph), cb], axis=-1)
        th2, thn = np.arccos(ct), np.arccos(cb)
        # projection weights: (2l1+1)(2l2+1)(2L+1) H^2 S w  (coefficient of S, Eq. TripoSH)
        self.proj = []
        for (l1, l2, L) in mults:
            H = wigner3j(l1, l2, L, 0, 0, 0)
            S = s_basis(l1, l2, L, 0.0 * ct, 0.0 * ct, th2, 0.0 * ct, thn, ph)
            self.proj.append((2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1) * H ** 2 * S * self.w)
        self.proj = np.array(self.proj)   # [n_mult, n_ang]
        return self


def triposh_monomials(k, grid, pk, alpha=1.0, eps=0.0, mults=None, bispec=None):
    """B^t_{l1 l2 L}(k_i, k_j) for every monomial t: array [11, n_mult, Nk, Nk].
    Only k_j >= k_i is integrated; the rest follows from the exchange symmetry
    B_{l1 l2 L}(k1, k2) = B_{l2 l1 L}(k2, k1) of the cyclic bispectrum."""
    mults = MULTIPOLES if mults is None else mults
    swap = [mults.index((l2, l1, L)) for (l1, l2, L) in mults]
    Nk = len(k)
    out = None
    zhat = np.array([0.0, 0.0, 1.0])
    for i in range(Nk):
        k2v = k[i:, None, None] * grid.k2hat[None, :, :]             # [Nk - i, n_ang, 3]
        k1v = np.broadcast_to((k[i] * zhat)[None, None, :], k2v.shape)
        n = np.broadcast_to(grid.n[None, :, :], k2v.shape)
        if bispec is None:
            Bm = bispectrum_monomials(k1v, k2v, n, pk, alpha, eps)   # [11, Nk - i, n_ang]
        else:
            Bm = bispec(k1v, k2v, n)                                 # [T, Nk - i, n_ang]
        proj = np.einsum("tja,ma->tmj", Bm, grid.proj)
        if out is None:
            out = np.zeros((Bm.shape[0], grid.proj.shape[0], Nk, Nk))
        out[:, :, i, i:] = proj
        out[:, :, i:, i] = proj[:, swap, :]
        # k_i = k_j: both orders are the same integral; keep their mean
        out[:, :, i, i] = 0.5 * (proj[:, :, 0] + proj[:, swap, 0])
    return out


# ---------------------------------------------------------------- 6. Hankel transform

def bin_bessel(l, k, edges, n_gl=64):
    """r^2-weighted bin averages of j_l(k r): array [n_bins, Nk]."""
    x, w = roots_legendre(n_gl)
    out = np.zeros((len(edges) - 1, len(k)))
    for b in range(len(edges) - 1):
        a, c = edges[b], edges[b + 1]
        r = 0.5 * (c - a) * x + 0.5 * (c + a)
        wr = 0.5 * (c - a) * w * r ** 2
        out[b] = (wr[:, None] * spherical_jn(l, np.outer(r, k))).sum(0) / wr.sum()
    return out


def hankel_weights(l, k, edges, n_sub=16):
    """J[bin][i] = int dk k^2 / (2 pi^2) jbar_l(k; bin) s_i(k), with s_i the
    cardinal cubic splines in ln k on the nodes k (natural ends): B_{l1 l2 L} is
    interpolated by a cubic spline in ln k between nodes while the oscillating
    bin-averaged Bessel factor is integrated on n_sub Gauss-Legendre points per
    interval."""
    from scipy.interpolate import CubicSpline
    x, wx = roots_legendre(n_sub)
    a, b = k[:-1], k[1:]
    kk = 0.5 * (b - a)[:, None] * x[None, :] + 0.5 * (a + b)[:, None]       # [intervals, n_sub]
    ww = 0.5 * (b - a)[:, None] * wx[None, :]
    jb = bin_bessel(l, kk.ravel(), edges)                                    # [bins, points]
    f = jb * (ww * kk ** 2 / (2.0 * math.pi ** 2)).ravel()[None, :]
    card = CubicSpline(np.log(k), np.eye(len(k)), bc_type="natural")(np.log(kk.ravel()))   # [points, nodes]
    return f @ card


def hankel_2d(Bm, k, edges, mults):
    """Eq. TriRelBtoZ, bin-averaged: zeta[t, mult, b1, b2] from B[t, mult, k1, k2]
    on the nodes k (linear interpolation between them)."""
    J = {l: hankel_weights(l, k, edges) for l in range(5)}
    out = np.zeros(Bm.shape[:2] + (len(edges) - 1, len(edges) - 1))
    for q, (l1, l2, L) in enumerate(mults):
        phase = (-1) ** ((l1 + l2) // 2)                 # i^(l1 + l2), l1 + l2 even
        out[:, q] = phase * np.einsum("ai,tij,bj->tab", J[l1], Bm[:, q], J[l2])
    return out


def k_nodes(k_min, k_split, k_max, n_log, dk):
    """Nodes: logarithmic below k_split, linear (step dk) up to k_max."""
    kl = np.logspace(math.log10(k_min), math.log10(k_split), n_log)
    kh = np.arange(k_split, k_max + 0.5 * dk, dk)
    return np.concatenate([kl, kh[1:]])


# ---------------------------------------------------------------- the model

@dataclass
class ModelSetup:
    r_min: float = 10.0
    r_max: float = 150.0
    n_bins: int = 20
    k_min: float = 1e-4            # nodes of B in k: log below k_split, linear above
    k_split: float = 0.05
    k_max: float = 1.0
    n_log: int = 16
    dk: float = 0.025
    grid: AngularGrid = None

    def __post_init__(self):
        if self.grid is None:
            self.grid = AngularGrid(48, 8, 8)
        self.edges = np.linspace(self.r_min, self.r_max, self.n_bins + 1)
        self.k = k_nodes(self.k_min, self.k_split, self.k_max, self.n_log, self.dk)
        self.pk = PowerNW()
        self.grid.build(MULTIPOLES)


def templates(setup: ModelSetup, alpha=1.0, eps=0.0):
    """T_t(alpha, eps): zeta per monomial, array [11, n_mult, n_bins, n_bins]."""
    Bm = triposh_monomials(setup.k, setup.grid, setup.pk, alpha, eps)
    return hankel_2d(Bm, setup.k, setup.edges, MULTIPOLES)


def monomial_coeffs(b1, b2, f):
    b1, b2, f = (np.asarray(x, dtype=np.float64) for x in (b1, b2, f))
    return np.stack([b1 ** e1 * b2 ** e2 * f ** e3 for (e1, e2, e3) in MONOMIALS], axis=-1)


def model_direct(setup: ModelSetup, theta):
    """The full model at theta = (f, b1, b2, sigma8, alpha, eps): [n_mult, n_bins, n_bins]."""
    f, b1, b2, s8, alpha, eps = theta
    T = templates(setup, alpha, eps)
    return s8 ** 4 * np.tensordot(monomial_coeffs(b1, b2, f), T, axes=(0, 0))


def upper_pairs(n_bins):
    """Index pairs (i, j), i <= j, in row-major order: the r1 <= r2 triangles."""
    return [(i, j) for i in range(n_bins) for j in range(i, n_bins)]


def flatten_upper(z):
    """[..., n_mult, n_bins, n_bins] -> [..., n_mult * n_pairs] over r1 <= r2."""
    nb = z.shape[-1]
    iu = np.triu_indices(nb)
    return z[..., iu[0], iu[1]].reshape(z.shape[:-3] + (-1,))


class TemplateModel:
    """Templates on an (alpha, eps) grid with bicubic interpolation (Sec. 2.5)."""

    def __init__(self, setup: ModelSetup, alphas, epss, tables):
        self.setup, self.alphas, self.epss = setup, np.asarray(alphas), np.asarray(epss)
        self.tables = tables      # [n_a, n_e, 11, n_out] (upper-triangle flattened)

    @staticmethod
    def build(setup: ModelSetup, alphas, epss, pool=None):
        nodes = [(a, e) for a in alphas for e in epss]
        if pool is None:
            res = [flatten_upper(templates(setup, a, e)) for (a, e) in nodes]
        else:
            res = pool.starmap(_template_node, [(setup, a, e) for (a, e) in nodes])
        tab = np.array(res).reshape(len(alphas), len(epss), len(MONOMIALS), -1)
        return TemplateModel(setup, alphas, epss, tab)

    def _cubic_weights(self, grid, x):
        """Catmull-Rom weights on a uniform grid: (index of the 4-point stencil start, weights)."""
        h = grid[1] - grid[0]
        u = (x - grid[0]) / h
        i = np.clip(np.floor(u).astype(int), 1, len(grid) - 3)
        t = u - i
        w = np.stack([(-t ** 3 + 2 * t ** 2 - t) / 2, (3 * t ** 3 - 5 * t ** 2 + 2) / 2,
                      (-3 * t ** 3 + 4 * t ** 2 + t) / 2, (t ** 3 - t ** 2) / 2], axis=-1)
        return i - 1, w

    def __call__(self, theta, chunk=512):
        """theta [..., 6] = (f, b1, b2, sigma8, alpha, eps) -> flattened zeta [..., n_out]."""
        theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
        out = np.empty((theta.shape[0], self.tables.shape[-1]))
        for c0 in range(0, theta.shape[0], chunk):
            th = theta[c0:c0 + chunk]
            f, b1, b2, s8, a, e = th.T
            ia, wa = self._cubic_weights(self.alphas, a)
            ie, we = self._cubic_weights(self.epss, e)
            c = monomial_coeffs(b1, b2, f) * (s8 ** 4)[:, None]
            acc = np.zeros((th.shape[0], self.tables.shape[-1]))
            for p in range(4):
                for q in range(4):
                    wpq = (wa[:, p] * we[:, q])[:, None] * c                       # [n, 11]
                    acc += np.einsum("nt,nto->no", wpq, self.tables[ia + p, ie + q])
            out[c0:c0 + chunk] = acc
        return out


def _template_node(setup, a, e):
    return flatten_upper(templates(setup, a, e))


def latin_hypercube(n, seed, box=((0.5, 1.0), (1.0, 3.0), (-1.0, 2.0), (0.6, 1.0), (0.95, 1.05), (-0.05, 0.05))):
    """Seeded Latin-hypercube samples of (f, b1, b2, sigma8, alpha, eps)."""
    rng = np.random.default_rng(seed)
    d = len(box)
    u = (rng.permuted(np.tile(np.arange(n), (d, 1)), axis=1).T + rng.random((n, d))) / n
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    return lo + u * (hi - lo)
