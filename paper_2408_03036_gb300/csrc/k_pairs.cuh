// Pair stage of the anisotropic 3PCF estimator (Eq. alm of arXiv:2408.03036,
// Sec. 4.2): for every primary, neighbour search to r_max over a cell list,
// exact integer radial binning, and per-bin sums of w_j Y_l^m(r_hat_ij) with
// the line of sight along z (or, in the VLOS variant, from an observer to the
// primary).  Also the per-bin sums of w_j^2 f_j(mu) that give
// the degenerate j = k triangle term, and integer pair counts.
//
// Both kernels are persistent: a CTA takes tiles of P primaries from an atomic
// counter.  For a tile, the cell rows within reach of each primary become
// contiguous record ranges (cells are stored x-fastest, so a run of cells along
// x is one range), trimmed to the sphere of radius r_max; warps take ranges in
// a strided order (which mixes radii) and sweep them 32 candidates per step,
// binning each candidate exactly (cand_bin2, two per lane).  k_counts adds
// integer counts; k_pairs_q (below) accumulates the harmonic sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

// Constant tables, passed by value (kernel parameter space is a constant bank,
// fine for warp-uniform reads) and as a device copy (PairParams::harm) for the
// tile epilogue, whose lanes read different entries.
//
// Harmonics are accumulated unnormalised: for a unit vector (x, y, z),
//     Y_l^m = K_lm V_l^m(z) (x + i y)^m,
// where V_m^m = 1, V_{m+1}^m = (2m + 1) z and
//     V_l^m = (2l - 1) z V_{l-1}^m - (l + m - 1)(l - m - 1) V_{l-2}^m,
// (the associated-Legendre recurrence divided through by (l - m)! / (2m - 1)!!),
// and K_lm = (-1)^m N_lm (2m - 1)!! / (l - m)!.  Every recurrence coefficient is
// a small integer, exact in single precision, so the float evaluation carries
// only rounding error; the normalisation enters once, as K_lm at write-out.
// (Rounded polynomial coefficients would instead give Y_l^m a small non-zero
// mean over the sphere, a coherent bias that grows with the pair count.)
struct HarmTables {
    double K[TPCF_MAX_LMAX + 1][TPCF_MAX_LMAX + 1];
    // The self accumulator j sums w^2 f_j(z) with f_0 = 1 and f_j = V_{2j}^0 = (2j)! P_{2j}.
    // gd_hi + gd_lo [jd][j]: V_l^m(z)^2 (1 - z^2)^m = sum_j gd[jd][j] f_j(z) exactly,
    // jd = (l, m >= 0); the j = k term of the diagonal is K_lm^2 sum_j gd[jd][j] * acc_j.
    float gd_hi[(TPCF_MAX_LMAX + 1) * (TPCF_MAX_LMAX + 2) / 2][TPCF_MAX_LMAX + 1];
    float gd_lo[(TPCF_MAX_LMAX + 1) * (TPCF_MAX_LMAX + 2) / 2][TPCF_MAX_LMAX + 1];
    // K_lm as an unevaluated float pair (hi, lo) per real index k (l^2 for m = 0,
    // l^2 + 2m - 1 and l^2 + 2m for m >= 1), and K_lm^2 rounded to float per
    // jd = (l, m >= 0): the tile epilogue scales in FP32 (FP64 arithmetic runs at a
    // small fraction of the FP32 rate on this part)
    float kout[(TPCF_MAX_LMAX + 1) * (TPCF_MAX_LMAX + 1)][2];
    float k2[(TPCF_MAX_LMAX + 1) * (TPCF_MAX_LMAX + 2) / 2];
};

// Direct j = k sums for l_max >= 5: sum_j w_j^2 |V_l^m(z_j) (x_j + i y_j)^m|^2 per
// (l, m >= 0), accumulated from the same rounded values as the harmonic sums.
// The polynomial identity behind the shared self sums (below) assumes |n| = 1;
// FP32 unit vectors miss it by about an ulp, and for m >= 1 the miss
// (|x + iy|^2 versus 1 - z^2) is amplified near the poles, which at l = 5, 6
// leaves about 1e-6 of |Y|^2 per pair in |a|^2 - self.  Bins with one or two
// pairs per primary, where |a|^2 - self is almost all j = k term, then carry
// that into the diagonal.  Pairs of consecutive l at one m share a float2.
template <int LMAX>
struct Direct {
    static constexpr bool ON = LMAX >= 5;
    static constexpr int np(int m) { return (LMAX - m + 2) / 2; }
    static constexpr int off(int m)
    {
        int o = 0;
        for (int k = 0; k < m; ++k) o += np(k);
        return o;
    }
    static constexpr int N2 = ON ? off(LMAX + 1) : 1;
};

template <int LMAX>
struct Layout {
    static constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    static constexpr int NSP = LMAX + 1;
    static constexpr int NDIAG = (LMAX + 1) * (LMAX + 2) / 2;
    static constexpr int NDS = Direct<LMAX>::ON ? NDIAG : 0;   // direct j = k sums, index l(l+1)/2 + m
    static constexpr int NACC = NLM + NSP + NDS;
    // odd row stride (distinct banks for distinct keys) with one spare column: the
    // key's count of secondaries of negative weight, as an integer
    static constexpr int NACCP = (NACC + 1) | 1;
};

__device__ __forceinline__ void latch_error(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// 1/sqrt(x) for finite x >= 1: the hardware estimate y0 = rsqrtf(x) refined by
// one Newton-Raphson step for f(y) = y^-2 - x, y1 = y0 + y0 (1 - x y0^2) / 2.
// The step leaves a truncation error of -(3/2) e0^2 for a relative estimate
// error e0 (below 1e-13), so what remains is the rounding of its last
// operations, with no coherent bias in x y1^2 - 1 over many pairs; the j = k
// cancellation on diagonal bins needs that (the raw estimate alone is biased).
// tpcf_check_rsqrt compares it with the correctly rounded __frsqrt_rn.
__device__ __forceinline__ float rsqrt_newton(float x)
{
    const float y0 = rsqrtf(x);
    const float r = fmaf(-x * y0, y0, 1.0f);
    return fmaf(0.5f * y0, r, y0);
}

// Packed accumulators of one lane (float2, so that every update is one paired
// FP32 instruction with the rounding of the two scalar ones):
//   A[l]          = (sum w V_l^0,  sum w^2 f_l)            l = 0..LMAX
//   A[q(l, m)]    = (Re, Im of sum w V_l^m (x + i y)^m)    m = 1..LMAX, l = m..LMAX
// f_0 = 1 and f_l = V_{2l}^0 (the self-sum polynomials).  unpack() maps them to
// the tile layout: index l^2 (m = 0), l^2 + 2m - 1 / l^2 + 2m (Re / Im), NLM + l.
template <int LMAX>
struct Packed {
    static constexpr int N0 = LMAX + 1;
    static constexpr int N2 = N0 + LMAX * (LMAX + 1) / 2;
    static __host__ __device__ constexpr int q(int l, int m)
    {
        int o = N0;
        for (int k = 1; k < m; ++k) o += LMAX - k + 1;
        return o + (l - m);
    }
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Accumulates one pair (unit vector x, y, z and weight w) into the packed sums.
// Every chain is streamed (each value used as soon as it is formed, two values
// of a recurrence kept), which keeps the live registers to the accumulators and
// a handful of temporaries.
template <int LMAX>
__device__ __forceinline__ void accum_pair(float x, float y, float z, float w, float2 (&A)[Packed<LMAX>::N2],
                                           float2 (&S)[Direct<LMAX>::N2])
{
    constexpr int LZ = (2 * LMAX > 1) ? 2 * LMAX : 1;
    const float w2 = w * w;
    // m = 0: V_l^0 for l <= 2 LMAX; a_l^0 (l <= LMAX) and the self sums w^2 f_j, f_j = V_2j^0
    A[0] = __fadd2_rn(A[0], f2(w, w2));
    {
        float vm2 = 1.f, vm1 = z;   // V_0^0, V_1^0
        if (LMAX >= 1) A[1].x = fmaf(vm1, w, A[1].x);
        if constexpr (Direct<LMAX>::ON) S[0] = __fadd2_rn(S[0], f2(w2, w2 * z * z));
#pragma unroll
        for (int l = 2; l <= LZ; ++l) {
            const float v = fmaf((float)(2 * l - 1) * z, vm1, -(float)((l - 1) * (l - 1)) * vm2);
            if (l <= LMAX) A[l].x = fmaf(v, w, A[l].x);
            if ((l & 1) == 0) A[l / 2].y = fmaf(v, w2, A[l / 2].y);
            if constexpr (Direct<LMAX>::ON) {
                if (l <= LMAX) {   // w^2 V_l^0^2 into slot (l, 0)
                    const float t = v * v * w2;
                    if (l & 1) S[l / 2].y += t;
                    else S[l / 2].x += t;
                }
            }
            vm2 = vm1;
            vm1 = v;
        }
    }
    // m >= 1: cs = w (x + i y)^m advanced by one complex product per m
    float cr = w, ci = 0.f;
#pragma unroll
    for (int m = 1; m <= LMAX; ++m) {
        const float nr = fmaf(cr, x, -ci * y), ni = fmaf(cr, y, ci * x);
        cr = nr;
        ci = ni;
        float qm = 0.f;
        if constexpr (Direct<LMAX>::ON) qm = fmaf(cr, cr, ci * ci);
        float vm2 = 0.f, vm1 = 0.f;
#pragma unroll
        for (int l = m; l <= LMAX; ++l) {
            float v;
            if (l == m) v = 1.f;
            else if (l == m + 1) v = (float)(2 * m + 1) * z;
            else v = fmaf((float)(2 * l - 1) * z, vm1, -(float)((l + m - 1) * (l - m - 1)) * vm2);
            vm2 = vm1;
            vm1 = v;
            const int qi = Packed<LMAX>::q(l, m);
            if (l == m) A[qi] = __fadd2_rn(A[qi], f2(cr, ci));
            else A[qi] = __ffma2_rn(f2(v, v), f2(cr, ci), A[qi]);
            if constexpr (Direct<LMAX>::ON) {
                const int si = Direct<LMAX>::off(m) + (l - m) / 2;
                const float t = v * v * qm;
                if ((l - m) & 1) S[si].y += t;
                else S[si].x += t;
            }
        }
    }
}

// Writes the packed sums of one lane to a row of the tile layout.
template <int LMAX>
__device__ __forceinline__ void unpack(const float2 (&A)[Packed<LMAX>::N2], const float2 (&S)[Direct<LMAX>::N2],
                                       float *row)
{
    constexpr int NLM = Layout<LMAX>::NLM;
    constexpr int NSP = Layout<LMAX>::NSP;
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
        row[l * l] = A[l].x;
        row[NLM + l] = A[l].y;
    }
#pragma unroll
    for (int m = 1; m <= LMAX; ++m)
#pragma unroll
        for (int l = m; l <= LMAX; ++l) {
            row[l * l + 2 * m - 1] = A[Packed<LMAX>::q(l, m)].x;
            row[l * l + 2 * m] = A[Packed<LMAX>::q(l, m)].y;
        }
    if constexpr (Direct<LMAX>::ON) {
#pragma unroll
        for (int m = 0; m <= LMAX; ++m)
#pragma unroll
            for (int p = 0; p < Direct<LMAX>::np(m); ++p) {
                const int l = m + 2 * p;
                const float2 v = S[Direct<LMAX>::off(m) + p];
                row[NLM + NSP + l * (l + 1) / 2 + m] = v.x;
                if (l + 1 <= LMAX) row[NLM + NSP + (l + 1) * (l + 2) / 2 + m] = v.y;
            }
    }
}

// Compensated evaluation of a^2 + b^2 - c: the squares are split exactly
// (TwoProduct with an FMA) and the sums carried as unevaluated pairs (Knuth's
// TwoSum), so the one rounding is of the result, however much a^2 + b^2 and c
// cancel.  The round-to-nearest intrinsics keep the compiler from fusing the
// steps.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return s;
}

__device__ __forceinline__ float sq2_minus(float a, float b, float ch, float cl)
{
    const float p = __fmul_rn(a, a), ep = fmaf(a, a, -p);
    const float q = __fmul_rn(b, b), eq = fmaf(b, b, -q);
    float e1, e2;
    const float s = two_sum(p, q, e1);
    const float t = two_sum(s, -ch, e2);
    return __fadd_rn(t, __fadd_rn(__fadd_rn(ep, eq), __fadd_rn(__fadd_rn(e1, e2), -cl)));
}

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__device__ __forceinline__ int gcd_int(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Two independent bisections in lockstep on the x words of the records (the
// records of a cell are sorted by x): on return a is the first index in [a, b)
// whose record has x >= ta, and c the first in [c, d) with x >= tc.  The two
// loads of a round are in flight together, so a row's two chord ends cost one
// chain of L2 round trips, not two.
__device__ __forceinline__ void lower_x2(const int4 *rec, int &a, int b, long long ta, int &c, int d, long long tc)
{
    const int *xw = reinterpret_cast<const int *>(rec);
    while (a < b || c < d) {
        const int ma = (a + b) >> 1, mc = (c + d) >> 1;
        const long long va = a < b ? (long long)(uint32_t)__ldg(xw + 4 * (size_t)ma) : 0;
        const long long vc = c < d ? (long long)(uint32_t)__ldg(xw + 4 * (size_t)mc) : 0;
        if (a < b) {
            if (va < ta) a = ma + 1;
            else b = ma;
        }
        if (c < d) {
            if (vc < tc) c = mc + 1;
            else d = mc;
        }
    }
}

// Candidate record ranges of a tile (all threads): for every (slot, row of cells
// within reach) up to two contiguous runs of cells along x (two where a periodic
// row wraps), trimmed to the sphere of radius r_max around the primary: to whole
// cells, then, since every cell's records are sorted by x, to the records of the
// two end cells that lie inside the row's chord; only non-empty runs are listed,
// in any order, with the count in *s_nr.
__device__ inline void tile_ranges(const PairParams &p, int np, long long mock_cells, const int4 *sPc,
                                   const float4 *sPf, int *rstart, int *rlen, int *rslot, int *s_nr)
{
    const int s = p.s, nc = p.nc, side = 2 * s + 1, rows = side * side;
    for (int r = threadIdx.x; r < np * rows; r += blockDim.x) {
        const int slot = r / rows, row = r % rows;
        const int dz = row / side - s, dy = row % side - s;
        const int4 pc = sPc[slot];
        const float4 pf = sPf[slot];
        const int cy = pc.y + dy, cz = pc.z + dz;
        int a0 = 0, l0 = 0, a1 = 0, l1 = 0;
        const float ylo = (float)cy * p.h_u, zlo = (float)cz * p.h_u;
        const float dyv = fmaxf(0.f, fmaxf(ylo - pf.y, pf.y - (ylo + p.h_u)));
        const float dzv = fmaxf(0.f, fmaxf(zlo - pf.z, pf.z - (zlo + p.h_u)));
        const float rr = p.rmax_trim;
        const float d2 = dyv * dyv + dzv * dzv;
        bool row_ok = d2 <= rr * rr;
        int wy = cy, wz = cz;
        if (p.periodic) {
            wy = (cy % nc + nc) % nc;
            wz = (cz % nc + nc) % nc;
        } else if (cy < 0 || cz < 0 || cy >= nc || cz >= nc) {
            row_ok = false;
        }
        if (row_ok) {
            const float wx = sqrtf(fmaxf(rr * rr - d2, 0.f)) * 1.0001f + 4096.f;
            int x0 = (int)floorf((pf.x - wx) / p.h_u);
            int x1 = (int)floorf((pf.x + wx) / p.h_u);
            x0 = max(x0, pc.x - s);
            x1 = min(x1, pc.x + s);
            if (!p.periodic) {
                x0 = max(x0, 0);
                x1 = min(x1, nc - 1);
            }
            if (x1 >= x0) {
                const long long base = mock_cells + ((long long)wz * nc + wy) * nc;
                // the chord [pf.x - wx, pf.x + wx] in whole units (wx carries margins
                // far above the float roundings of pf.x and of these bounds); a
                // wrapped run's records sit 2^32 units from their unwrapped place
                const long long clo = (long long)floorf(pf.x - wx), chi = (long long)ceilf(pf.x + wx);
                long long lo0 = clo, hi1 = chi;
                int sa = x0, sb = x1, ta = 1, tb = 0;   // second run empty
                if (p.periodic) {
                    if (x0 < 0) { sa = x0 + nc; sb = nc - 1; ta = 0; tb = x1; lo0 += 4294967296ll; }
                    else if (x1 >= nc) { sa = x0; sb = nc - 1; ta = 0; tb = x1 - nc; hi1 -= 4294967296ll; }
                }
                const bool two = tb >= ta;
                // the low end of the chord lies in cell sa, the high end in the last
                // cell of the run that ends the row (tb when the row wraps, else sb);
                // the two searches are independent (same sorted cell when sa = sb,
                // later cells otherwise)
                const int hc = two ? tb : sb;
                int lo_a = p.cell_start[base + sa];
                const int lo_b = p.cell_start[base + sa + 1];
                int hi_a = p.cell_start[base + hc];
                const int hi_b = p.cell_start[base + hc + 1];
                const int end0 = two ? p.cell_start[base + sb + 1] : 0;
                const int start1 = two ? p.cell_start[base + ta] : 0;
                lower_x2(p.rec, lo_a, lo_b, lo0, hi_a, hi_b, hi1 + 1);
                a0 = lo_a;
                if (two) {
                    a1 = start1;
                    l1 = hi_a - a1;
                    l0 = end0 - a0;
                } else {
                    l0 = hi_a - a0;
                }
            }
        }
        if (l0 > 0) {
            const int at = atomicAdd(s_nr, 1);
            rstart[at] = a0; rlen[at] = l0; rslot[at] = slot;
        }
        if (l1 > 0) {
            const int at = atomicAdd(s_nr, 1);
            rstart[at] = a1; rlen[at] = l1; rslot[at] = slot;
        }
    }
}

// Exact radial bin of one candidate (all lanes of the warp call it together).
// The float bin coordinate t = (r - r_min) / dr from the float r^2 decides unless
// it lies within p.tdelta of an integer (a proven bound on its rounding error),
// where the exact 64-bit integer r^2 is compared with the integer edges E.
// Returns the bin, or -1 outside [r_min, r_max) or for an invalid lane.
__device__ __forceinline__ int cand_bin(const PairParams &p, const unsigned long long *sE, int nb, bool valid,
                                        int dx, int dy, int dz, float fx, float fy, float fz)
{
    const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
    const float rg = fmaxf(r2f, 1.f);
    const float t = fmaf(rg * rsqrtf(rg), p.inv_dr_u, p.t_off);
    const float tf = floorf(t);
    int b = (int)tf;
    const float fr = t - tf;
    const bool sure = fr > p.tdelta && fr < 1.f - p.tdelta;
    bool ok = valid && sure && b >= 0 && b < nb;
    const bool unsure = valid && !sure && t > -1.f && t < (float)(nb + 1);
    if (__any_sync(0xffffffffu, unsure)) {
        if (unsure) {
            const long long lx = dx, ly = dy, lz = dz;
            const unsigned long long r2 = (unsigned long long)(lx * lx) + (unsigned long long)(ly * ly)
                                        + (unsigned long long)(lz * lz);
            ok = r2 >= sE[0] && r2 < sE[nb];
            b = min(max(b, 0), nb - 1);
            while (b > 0 && r2 < sE[b]) --b;
            while (b < nb - 1 && r2 >= sE[b + 1]) ++b;
        }
    }
    return ok ? b : -1;
}

// cand_bin for a lane's two candidates at once: the float steps as paired FP32
// instructions (the scalar steps' roundings, so the same bins) and one warp vote
// for the exact fallback.
__device__ __forceinline__ int2 cand_bin2(const PairParams &p, const unsigned long long *sE, int nb, bool valid0,
                                          bool valid1, int dx0, int dy0, int dz0, int dx1, int dy1, int dz1,
                                          float fx0, float fy0, float fz0, float fx1, float fy1, float fz1)
{
    const float2 r2 = __ffma2_rn(make_float2(fx0, fx1), make_float2(fx0, fx1),
                                 __ffma2_rn(make_float2(fy0, fy1), make_float2(fy0, fy1),
                                            __fmul2_rn(make_float2(fz0, fz1), make_float2(fz0, fz1))));
    const float rg0 = fmaxf(r2.x, 1.f), rg1 = fmaxf(r2.y, 1.f);
    const float2 r = __fmul2_rn(make_float2(rg0, rg1), make_float2(rsqrtf(rg0), rsqrtf(rg1)));
    const float2 t = __ffma2_rn(r, make_float2(p.inv_dr_u, p.inv_dr_u), make_float2(p.t_off, p.t_off));
    const float tf0 = floorf(t.x), tf1 = floorf(t.y);
    const float2 fr = __fadd2_rn(t, make_float2(-tf0, -tf1));
    int b0 = (int)tf0, b1 = (int)tf1;
    const bool sure0 = fr.x > p.tdelta && fr.x < 1.f - p.tdelta, sure1 = fr.y > p.tdelta && fr.y < 1.f - p.tdelta;
    bool ok0 = valid0 && sure0 && b0 >= 0 && b0 < nb;
    bool ok1 = valid1 && sure1 && b1 >= 0 && b1 < nb;
    const bool unsure0 = valid0 && !sure0 && t.x > -1.f && t.x < (float)(nb + 1);
    const bool unsure1 = valid1 && !sure1 && t.y > -1.f && t.y < (float)(nb + 1);
    if (__any_sync(0xffffffffu, unsure0 || unsure1)) {
        if (unsure0) {
            const long long lx = dx0, ly = dy0, lz = dz0;
            const unsigned long long q = (unsigned long long)(lx * lx) + (unsigned long long)(ly * ly)
                                       + (unsigned long long)(lz * lz);
            ok0 = q >= sE[0] && q < sE[nb];
            b0 = min(max(b0, 0), nb - 1);
            while (b0 > 0 && q < sE[b0]) --b0;
            while (b0 < nb - 1 && q >= sE[b0 + 1]) ++b0;
        }
        if (unsure1) {
            const long long lx = dx1, ly = dy1, lz = dz1;
            const unsigned long long q = (unsigned long long)(lx * lx) + (unsigned long long)(ly * ly)
                                       + (unsigned long long)(lz * lz);
            ok1 = q >= sE[0] && q < sE[nb];
            b1 = min(max(b1, 0), nb - 1);
            while (b1 > 0 && q < sE[b1]) --b1;
            while (b1 < nb - 1 && q >= sE[b1 + 1]) ++b1;
        }
    }
    return make_int2(ok0 ? b0 : -1, ok1 ? b1 : -1);
}

// ---------------------------------------------------------------------------
// Integer pair counts only (the random-only RRR pass): the same tiles, ranges
// and exact binning.  With one primary per tile every thread counts into its own
// column of a [bin][thread] array (no atomics, no bank conflicts), added up per
// tile; with several, one shared atomic per pair on the (slot, bin) counts.
constexpr int kCountThreads = 256;

struct CMap {
    int off_E, off_prim, off_pf, off_pc, off_rstart, off_rlen, off_rslot, off_cnt, off_red, off_pairs, off_misc;
    int total;
};

__host__ __device__ inline CMap make_cmap(int P, int nb, int s)
{
    CMap m;
    const int maxr = 2 * P * (2 * s + 1) * (2 * s + 1);
    int o = 0;
    m.off_E = o;      o = align_up(o + 8 * (TPCF_MAX_BINS + 1), 16);
    m.off_prim = o;   o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pf = o;     o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pc = o;     o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_rstart = o; o = align_up(o + 4 * maxr, 16);
    m.off_rlen = o;   o = align_up(o + 4 * maxr, 16);
    m.off_rslot = o;  o = align_up(o + 4 * maxr, 16);
    m.off_cnt = o;    o = align_up(o + 4 * (P == 1 ? nb * kCountThreads : P * nb), 16);
    m.off_red = o;    o = align_up(o + 4 * TPCF_MAX_BINS, 16);
    m.off_pairs = o;  o = align_up(o + 8 * nb, 16);
    m.off_misc = o;   o = align_up(o + 16, 16);
    m.total = o;
    return m;
}

template <int UNUSED = 0>   // a template so that every translation unit may include it
__global__ void __launch_bounds__(256, 2) k_counts(const PairParams p)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int nb = p.nb, P = p.P, nc = p.nc;
    const CMap M = make_cmap(P, nb, p.s);
    unsigned long long *sE = reinterpret_cast<unsigned long long *>(smem + M.off_E);
    int4 *sPrim = reinterpret_cast<int4 *>(smem + M.off_prim);
    float4 *sPf = reinterpret_cast<float4 *>(smem + M.off_pf);
    int4 *sPc = reinterpret_cast<int4 *>(smem + M.off_pc);
    int *rstart = reinterpret_cast<int *>(smem + M.off_rstart);
    int *rlen = reinterpret_cast<int *>(smem + M.off_rlen);
    int *rslot = reinterpret_cast<int *>(smem + M.off_rslot);
    int *cnt = reinterpret_cast<int *>(smem + M.off_cnt);
    int *red = reinterpret_cast<int *>(smem + M.off_red);
    unsigned long long *spairs = reinterpret_cast<unsigned long long *>(smem + M.off_pairs);
    int *misc = reinterpret_cast<int *>(smem + M.off_misc);
    const bool own = P == 1;   // per-thread counters [bin][thread]
    int &s_tile = misc[0];
    int &s_next = misc[1];
    int &s_nr = misc[2];

    for (int i = tid; i <= nb; i += blockDim.x) sE[i] = p.E[i];
    for (int i = tid; i < nb; i += blockDim.x) spairs[i] = 0ull;
    int cta_mock = -1;
    __syncthreads();
    auto flush = [&](int mk) {
        __syncthreads();
        for (int b = tid; b < nb; b += blockDim.x) {
            if (p.pair_counts && spairs[b]) atomicAdd(p.pair_counts + (size_t)mk * nb + b, spairs[b]);
            spairs[b] = 0ull;
        }
        __syncthreads();
    };
    for (;;) {
        if (tid == 0) {
            s_tile = atomicAdd(p.work, 1);
            s_next = 0;
            s_nr = 0;
        }
        __syncthreads();
        const long long t0 = (long long)s_tile * P;
        if (t0 >= p.n_prim) break;
        const int np = (int)min((long long)P, p.n_prim - t0);
        const int mock = p.prim_mock ? p.prim_mock[t0] : 0;
        if (mock != cta_mock) {
            if (cta_mock >= 0) flush(cta_mock);
            cta_mock = mock;
        }
        if (tid < np) {
            const int4 q = p.prim[t0 + tid];
            sPrim[tid] = q;
            const uint32_t ux = (uint32_t)q.x, uy = (uint32_t)q.y, uz = (uint32_t)q.z;
            sPf[tid] = make_float4((float)ux, (float)uy, (float)uz, __int_as_float(q.w));
            sPc[tid] = make_int4((int)(((unsigned long long)ux * nc) >> 32), (int)(((unsigned long long)uy * nc) >> 32),
                                 (int)(((unsigned long long)uz * nc) >> 32), 0);
        }
        for (int i = tid; i < (own ? nb * kCountThreads : np * nb); i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        tile_ranges(p, np, (long long)mock * p.ncell_mock, sPc, sPf, rstart, rlen, rslot, &s_nr);
        __syncthreads();
        const int nr = s_nr;
        int stride = (nr * 5) / 8 + 1;
        while (nr > 1 && gcd_int(stride, nr) != 1) ++stride;
        for (;;) {
            int r = 0;
            if (lane == 0) r = atomicAdd(&s_next, 1);
            r = __shfl_sync(FULL, r, 0);
            if (r >= nr) break;
            const int rr = (int)(((unsigned)r * (unsigned)stride) % (unsigned)nr);
            const int start = rstart[rr], len = rlen[rr], sl = rslot[rr];
            const int4 pr = sPrim[sl];
            for (int pos = 0; pos < len; pos += 64) {
                const int i0 = pos + lane, i1 = i0 + 32;
                const int4 q0 = p.rec[start + min(i0, len - 1)];
                const int4 q1 = p.rec[start + min(i1, len - 1)];
                const int dx0 = (int)((uint32_t)q0.x - (uint32_t)pr.x), dx1 = (int)((uint32_t)q1.x - (uint32_t)pr.x);
                const int dy0 = (int)((uint32_t)q0.y - (uint32_t)pr.y), dy1 = (int)((uint32_t)q1.y - (uint32_t)pr.y);
                const int dz0 = (int)((uint32_t)q0.z - (uint32_t)pr.z), dz1 = (int)((uint32_t)q1.z - (uint32_t)pr.z);
                const int2 bb = cand_bin2(p, sE, nb, i0 < len, i1 < len, dx0, dy0, dz0, dx1, dy1, dz1, (float)dx0,
                                          (float)dy0, (float)dz0, (float)dx1, (float)dy1, (float)dz1);
                const int b0 = bb.x, b1 = bb.y;
                if (own) {
                    if (b0 >= 0) cnt[b0 * kCountThreads + tid] += 1;
                    if (b1 >= 0) cnt[b1 * kCountThreads + tid] += 1;
                } else {
                    if (b0 >= 0) atomicAdd(&cnt[sl * nb + b0], 1);
                    if (b1 >= 0) atomicAdd(&cnt[sl * nb + b1], 1);
                }
            }
        }
        __syncthreads();
        const int *tc = cnt;   // the tile's (slot, bin) counts
        if (own) {
            // one warp per bin adds the threads' columns
            const int warp = tid >> 5, nw = blockDim.x >> 5;
            for (int b = warp; b < nb; b += nw) {
                int v = 0;
                for (int t = lane; t < kCountThreads; t += 32) v += cnt[b * kCountThreads + t];
                v = __reduce_add_sync(FULL, v);
                if (lane == 0) red[b] = v;
            }
            __syncthreads();
            tc = red;
        }
        if (p.counts)
            for (int i = tid; i < np * nb; i += blockDim.x) p.counts[t0 * nb + i] = tc[i];
        for (int b = tid; b < nb; b += blockDim.x) {
            unsigned long long t = 0;
            for (int q = 0; q < np; ++q) t += (unsigned long long)tc[q * nb + b];
            spairs[b] += t;
        }
        __syncthreads();
    }
    if (cta_mock >= 0) flush(cta_mock);
}

// ---------------------------------------------------------------------------
// Queued pair stage (harmonic sums).  Same tile / range / window scheme as
// k_pairs, but the CTA keeps one lane assignment for the whole tile:
//   * every key (slot, bin) of the tile owns g_k lanes and a queue of cap_k
//     entries in shared memory, both in proportion to the key's expected share
//     of the pairs (a per-CTA running histogram over bins, seeded with the
//     shell volumes);
//   * gathering warps compute the exact bin of every candidate that passes the
//     window test and append it to its key's queue (one shared atomic per
//     entry); an entry that finds its queue full stays in the lane and raises
//     the flag;
//   * when the flag is up (or every warp is out of ranges) the CTA drains the
//     queues: each lane sums its key's entries, strided by g_k, into registers
//     that it keeps for the whole tile; queue counters are double-buffered, so
//     a drain costs two barriers;
//   * at the end of the tile the g_k lanes of every key are added through one
//     shared-memory transpose.
// Compared with k_pairs there is no per-chunk sort, key histogram or per-chunk
// reduction, and staged pairs are written and read once.
struct QMap {
    int off_E, off_prim, off_pf, off_pc;
    int off_rstart, off_rlen, off_rslot;
    int off_qinfo, off_qcnt, off_cnt, off_gfirst, off_gsize, off_lanekey, off_hist;
    int off_sacc, off_queue;
    int off_d64, off_w64, off_pairs, off_misc;
    int total;
    int maxr;
};

template <int LMAX>
__host__ __device__ inline QMap make_qmap(int P, int nb, int s, int chunk, int block)
{
    QMap m;
    const int rows = (2 * s + 1) * (2 * s + 1);
    const int W = block / 32;
    m.maxr = 2 * P * rows;
    const int nk = P * nb;
    constexpr int naccp = Layout<LMAX>::NACCP;
    int o = 0;
    m.off_E = o;       o = align_up(o + 8 * (TPCF_MAX_BINS + 1), 16);
    m.off_prim = o;    o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pf = o;      o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pc = o;      o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_rstart = o;  o = align_up(o + 4 * m.maxr, 16);
    m.off_rlen = o;    o = align_up(o + 4 * m.maxr, 16);
    m.off_rslot = o;   o = align_up(o + 4 * m.maxr, 16);
    m.off_qinfo = o;   o = align_up(o + 8 * nk, 16);
    m.off_qcnt = o;    o = align_up(o + 4 * 2 * nk, 16);
    m.off_cnt = o;     o = align_up(o + 4 * nk, 16);
    m.off_gfirst = o;  o = align_up(o + 4 * nk, 16);
    m.off_gsize = o;   o = align_up(o + 4 * nk, 16);
    m.off_lanekey = o; o = align_up(o + 4 * block, 16);
    m.off_hist = o;    o = align_up(o + 4 * TPCF_MAX_BINS, 16);
    m.off_sacc = o;    o = align_up(o + 4 * nk * naccp, 16);
    // the queues (one record index per entry); reused as the [block][NACCP]
    // transpose area at the end of a tile
    const int qbytes = 4 * chunk, stage = 4 * block * naccp;
    m.off_queue = o;   o = align_up(o + (qbytes > stage ? qbytes : stage), 16);
    m.off_d64 = o;     o = align_up(o + 8 * nb * Layout<LMAX>::NDIAG, 16);
    m.off_w64 = o;     o = align_up(o + 8 * nb * Layout<LMAX>::NSP, 16);
    m.off_pairs = o;   o = align_up(o + 2 * 8 * nb, 16);   // all pairs, then random-random pairs
    m.off_misc = o;    o = align_up(o + 4 * (16 + W), 16);
    m.total = o;
    return m;
}

// static shared memory of the harmonic kernel (one double), and the extra of the
// varying-line-of-sight variant (the frames of a tile)
constexpr int kPairsStaticSmem = 16;
constexpr int kVlosStaticSmem = 3 * TPCF_MAX_TILE * 16;

template <int LMAX, bool VLOS = false>
__global__ void __launch_bounds__(256, (LMAX <= 4 ? 3 : 1)) k_pairs_q(const PairParams p, const HarmTables H)
{
    constexpr int NLM = Layout<LMAX>::NLM;
    constexpr int NACC = Layout<LMAX>::NACC;
    constexpr int NACCP = Layout<LMAX>::NACCP;
    constexpr int NDIAG = Layout<LMAX>::NDIAG;
    constexpr int NSP = Layout<LMAX>::NSP;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = T >> 5;
    const int nb = p.nb, P = p.P, s = p.s, nc = p.nc, C = p.chunk;
    const QMap M = make_qmap<LMAX>(P, nb, s, C, T);
    const int nkmax = P * nb;

    unsigned long long *sE = reinterpret_cast<unsigned long long *>(smem + M.off_E);
    int4 *sPrim = reinterpret_cast<int4 *>(smem + M.off_prim);
    float4 *sPf = reinterpret_cast<float4 *>(smem + M.off_pf);
    int4 *sPc = reinterpret_cast<int4 *>(smem + M.off_pc);
    int *rstart = reinterpret_cast<int *>(smem + M.off_rstart);
    int *rlen = reinterpret_cast<int *>(smem + M.off_rlen);
    int *rslot = reinterpret_cast<int *>(smem + M.off_rslot);
    int2 *qinfo = reinterpret_cast<int2 *>(smem + M.off_qinfo);   // (first entry, capacity) per key
    int *qcnt = reinterpret_cast<int *>(smem + M.off_qcnt);      // [2][nkmax]
    int *cnt = reinterpret_cast<int *>(smem + M.off_cnt);
    int *gfirst = reinterpret_cast<int *>(smem + M.off_gfirst);
    int *gsize = reinterpret_cast<int *>(smem + M.off_gsize);
    int *lanekey = reinterpret_cast<int *>(smem + M.off_lanekey);
    float *hist = reinterpret_cast<float *>(smem + M.off_hist);  // expected share of every bin
    float *sacc = reinterpret_cast<float *>(smem + M.off_sacc);  // [nk][NACCP] tile sums
    int *queue = reinterpret_cast<int *>(smem + M.off_queue);          // record index per entry
    float *stage = reinterpret_cast<float *>(smem + M.off_queue);
    double *d64 = reinterpret_cast<double *>(smem + M.off_d64);
    double *w64 = reinterpret_cast<double *>(smem + M.off_w64);
    unsigned long long *spairs = reinterpret_cast<unsigned long long *>(smem + M.off_pairs);
    unsigned long long *spairs_r = spairs + nb;
    int *misc = reinterpret_cast<int *>(smem + M.off_misc);
    int &s_tile = misc[0];
    int &s_next = misc[1];
    volatile int &s_flag = misc[2];   // a queue is full
    int &s_nr = misc[3];              // non-empty candidate ranges of the tile
    int *wdone = misc + 16;           // [W] warp has no more ranges and nothing pending
    // VLOS: rows e1, e2, e3 of each slot's rotation (e3 = line of sight), as float4
    __shared__ float4 sRot[VLOS ? 3 * TPCF_MAX_TILE : 1];   // kVlosStaticSmem bytes

    for (int i = tid; i <= nb; i += T) {
        sE[i] = p.E[i];
    }
    for (int i = tid; i < nb * NDIAG; i += T) d64[i] = 0.0;
    for (int i = tid; i < nb * NSP; i += T) w64[i] = 0.0;
    for (int i = tid; i < 2 * nb; i += T) spairs[i] = 0ull;
    for (int i = tid; i < 2 * nkmax; i += T) qcnt[i] = 0;
    if (tid < nb) {
        // seed: the shell volumes, r^3 in units of the bin edges' squares
        const float a = sqrtf(p.Ef[tid]), b = sqrtf(p.Ef[tid + 1]);
        hist[tid] = b * b * b - a * a * a;
    }
    if (tid == 0) s_flag = 0;
    // the periodic offset's total weight, in shared memory (read only at the tile ends)
    __shared__ double s_mono_w;
    if (tid == 0) s_mono_w = p.use_mono ? (p.mono_w_dev ? *p.mono_w_dev : p.mono_w) : 0.0;
    int cta_mock = -1;
    int par = 0;                      // live half of the double-buffered queue counters
    __syncthreads();

    auto a00 = [&](float wsum, int b) -> float {
        double v = (double)wsum * H.K[0][0];
        if (p.use_mono) v -= (s_mono_w - 1.0) * p.mono_coef[b];
        return (float)v;
    };

    auto flush_cta = [&](int mk) {
        __syncthreads();
        for (int i = tid; i < nb * NDIAG; i += T) {
            const double v = d64[i];
            const int b = i / NDIAG, jd = i % NDIAG;
            if (p.diag && v != 0.0) atomicAdd(p.diag + ((size_t)mk * NDIAG + jd) * nb + b, v);
            d64[i] = 0.0;
        }
        for (int i = tid; i < nb * NSP; i += T) {
            const double v = w64[i];
            const int b = i / NSP, j = i % NSP;
            if (p.wsp && v != 0.0) atomicAdd(p.wsp + ((size_t)mk * NSP + j) * nb + b, v);
            w64[i] = 0.0;
        }
        for (int b = tid; b < nb; b += T) {
            if (p.pair_counts && spairs[b]) atomicAdd(p.pair_counts + (size_t)mk * nb + b, spairs[b]);
            if (p.pair_counts_r && spairs_r[b]) atomicAdd(p.pair_counts_r + (size_t)mk * nb + b, spairs_r[b]);
            spairs[b] = 0ull;
            spairs_r[b] = 0ull;
        }
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) {
            s_tile = atomicAdd(p.work, 1);
            s_next = 0;
            s_nr = 0;
        }
        __syncthreads();
        long long t0;
        int np;
        if (p.tile_start) {
            if (s_tile >= p.n_tiles) break;
            t0 = p.tile_start[s_tile];
            np = (int)(p.tile_start[s_tile + 1] - t0);
        } else {
            t0 = (long long)s_tile * P;
            if (t0 >= p.n_prim) break;
            np = (int)min((long long)P, p.n_prim - t0);
        }
        const int nk = np * nb;
        const int mock = p.prim_mock ? p.prim_mock[t0] : 0;
        if (mock != cta_mock) {
            if (cta_mock >= 0) flush_cta(cta_mock);
            cta_mock = mock;
            if (p.prim_mock && p.use_mono && tid == 0) s_mono_w = p.mono_w_mock[mock];
        }
        const long long mock_cells = (long long)mock * p.ncell_mock;

        if (tid < np) {
            const int4 q = p.prim[t0 + tid];
            sPrim[tid] = q;
            const uint32_t ux = (uint32_t)q.x, uy = (uint32_t)q.y, uz = (uint32_t)q.z;
            sPf[tid] = make_float4((float)ux, (float)uy, (float)uz, __int_as_float(q.w));
            sPc[tid] = make_int4((int)(((unsigned long long)ux * nc) >> 32),
                                 (int)(((unsigned long long)uy * nc) >> 32),
                                 (int)(((unsigned long long)uz * nc) >> 32), 0);
            const float wq = __int_as_float(q.w);
            if (!(wq == wq) || isinf(wq)) latch_error(p.mock_status ? p.mock_status + mock : p.err, DEV_ERR_DATA);
            if constexpr (VLOS) {
                // line of sight n = (x_i - obs) / |x_i - obs| and an orthonormal frame
                // (e1, e2, n); the harmonics of the m = m' coupling do not depend on
                // the azimuth of e1 about n
                double n0 = (double)ux - p.obs[0], n1 = (double)uy - p.obs[1], n2 = (double)uz - p.obs[2];
                const double nr = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
                if (nr > 0.0) {
                    n0 /= nr;
                    n1 /= nr;
                    n2 /= nr;
                } else {   // a primary at the observer keeps z
                    n0 = 0.0;
                    n1 = 0.0;
                    n2 = 1.0;
                }
                // e1 = normalise(a x n) with a the coordinate axis least aligned with n
                double a0 = 0.0, a1 = 0.0, a2 = 0.0;
                if (fabs(n0) <= fabs(n1) && fabs(n0) <= fabs(n2)) a0 = 1.0;
                else if (fabs(n1) <= fabs(n2)) a1 = 1.0;
                else a2 = 1.0;
                double e0 = a1 * n2 - a2 * n1, e1 = a2 * n0 - a0 * n2, e2 = a0 * n1 - a1 * n0;
                const double er = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
                e0 /= er;
                e1 /= er;
                e2 /= er;
                const double f0 = n1 * e2 - n2 * e1, f1 = n2 * e0 - n0 * e2, f2 = n0 * e1 - n1 * e0;
                sRot[3 * tid + 0] = make_float4((float)e0, (float)e1, (float)e2, 0.f);
                sRot[3 * tid + 1] = make_float4((float)f0, (float)f1, (float)f2, 0.f);
                sRot[3 * tid + 2] = make_float4((float)n0, (float)n1, (float)n2, 0.f);
            }
        }
        // tile plan (warp 0): queue capacities and lane groups in proportion to the
        // expected share e_b / np of every key; at least 32 entries and one lane each
        if (warp == 0) {
            float e = lane < nb ? hist[lane] : 0.f;
            float tot = e;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
            e = lane < nb ? 0.999f * e / (tot * (float)np) : 0.f;   // sum over keys < 1
            const int capb = lane < nb ? 32 + (int)((float)(C - 32 * nk) * e) : 0;
            const int gb = lane < nb ? 1 + (int)((float)(T - nk) * e) : 0;
            int cs = capb, gs = gb;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t1 = __shfl_up_sync(FULL, cs, o);
                const int t2 = __shfl_up_sync(FULL, gs, o);
                if (lane >= o) { cs += t1; gs += t2; }
            }
            const int ctot = __shfl_sync(FULL, cs, 31), gtot = __shfl_sync(FULL, gs, 31);
            for (int i = lane; i < T; i += 32) lanekey[i] = -1;
            __syncwarp();
            if (lane < nb) {
                for (int sl = 0; sl < np; ++sl) {
                    const int k = sl * nb + lane;
                    qinfo[k] = make_int2(sl * ctot + cs - capb, capb);
                    const int g0 = sl * gtot + gs - gb;
                    gfirst[k] = g0;
                    gsize[k] = gb;
                    cnt[k] = 0;
                    for (int q = 0; q < gb; ++q) lanekey[g0 + q] = k;
                }
            }
        }
        __syncthreads();

        tile_ranges(p, np, mock_cells, sPc, sPf, rstart, rlen, rslot, &s_nr);
        __syncthreads();
        const int nr = s_nr;

        const int myk = lanekey[tid];
        const int myg = myk >= 0 ? gsize[myk] : 1;
        const int myr = myk >= 0 ? tid - gfirst[myk] : 0;
        const int myq = myk >= 0 ? qinfo[myk].x : 0;
        const int mycap = myk >= 0 ? qinfo[myk].y : 0;
        float2 acc[Packed<LMAX>::N2];
        float2 dacc[Direct<LMAX>::N2];
        // secondaries of negative weight (the randoms of a D - R field) in this lane's share
        int rcnt = 0;
#pragma unroll
        for (int j = 0; j < Packed<LMAX>::N2; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < Direct<LMAX>::N2; ++j) dacc[j] = make_float2(0.f, 0.f);

        // drains the queues (all threads); returns whether every warp has finished
        auto drain = [&]() -> bool {
            __syncthreads();                                   // (A) appends are visible
            int alldone = 1;
            for (int w = 0; w < W; ++w) alldone &= wdone[w];
            const int *live = qcnt + par * nkmax;
            if (tid < nk) cnt[tid] += min(live[tid], qinfo[tid].y);
            if (tid < nkmax) qcnt[(par ^ 1) * nkmax + tid] = 0;   // the other half: free since the last drain
            if (tid == 0) s_flag = 0;
            if (myk >= 0) {
                const int n = min(live[myk], mycap);
                const int *qq = queue + myq;
                // entries are record indices: the record is re-read (from L2) one
                // entry ahead of its use and its separation from the primary formed
                // again, exactly as in the sweep
                int4 nxt = make_int4(0, 0, 0, 0);
                if (myr < n) nxt = p.rec[qq[myr]];
                for (int e = myr; e < n; e += myg) {
                    const int4 q = nxt;
                    if (e + myg < n) nxt = p.rec[qq[e + myg]];
                    const int4 pr = sPrim[myk / nb];
                    float4 v = make_float4((float)(int)((uint32_t)q.x - (uint32_t)pr.x),
                                           (float)(int)((uint32_t)q.y - (uint32_t)pr.y),
                                           (float)(int)((uint32_t)q.z - (uint32_t)pr.z), __int_as_float(q.w));
                    rcnt += (int)(__float_as_uint(v.w) >> 31);
                    if constexpr (VLOS) {
                        // the separation in the primary's frame (e1, e2, line of sight)
                        const float4 *R = sRot + 3 * (myk / nb);
                        const float4 r0 = R[0], r1 = R[1], r2 = R[2];
                        const float x = fmaf(r0.x, v.x, fmaf(r0.y, v.y, r0.z * v.z));
                        const float y = fmaf(r1.x, v.x, fmaf(r1.y, v.y, r1.z * v.z));
                        const float z = fmaf(r2.x, v.x, fmaf(r2.y, v.y, r2.z * v.z));
                        v.x = x;
                        v.y = y;
                        v.z = z;
                    }
                    const float r2f = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
                    // |n|^2 = 1 up to unbiased rounding (see rsqrt_newton)
                    const float inv = rsqrt_newton(r2f);
                    accum_pair<LMAX>(v.x * inv, v.y * inv, v.z * inv, v.w, acc, dacc);
                }
            }
            __syncthreads();                                   // (B) queues consumed
            par ^= 1;
            return alldone != 0;
        };

        // ----- gather: warps take ranges (in a strided order that mixes radii, so the
        // queues fill evenly) and sweep them 32 candidates per step
        int stride = (nr * 5) / 8 + 1;
        while (nr > 1 && gcd_int(stride, nr) != 1) ++stride;
        int my_start = 0, my_len = 0, my_pos = 0, my_sl = 0;
        // two candidates per lane and step (i and i + 32): independent loads and bins
        bool done = false, have0 = false, have1 = false;
        int ent0 = 0, ent1 = 0;   // record indices
        int ek0 = 0, ek1 = 0;
        // appends a pending entry (one shared atomic); an entry that finds its queue
        // full stays pending and raises the flag.  (Aggregating equal keys across the
        // warp with a match instruction measured slower.)
        auto append = [&](bool &have, int ent, int ek) {
            if (!have) return;
            const int pos = atomicAdd(&qcnt[par * nkmax + ek], 1);
            const int2 qi = qinfo[ek];
            if (pos < qi.y) {
                queue[qi.x + pos] = ent;
                have = false;
            } else {
                s_flag = 1;   // stays pending until the queues are drained
            }
        };
        for (;;) {
            // bit 0: an entry of the warp waits for room; bit 1: a queue is full
            const unsigned st = __reduce_or_sync(FULL, (have0 || have1 ? 1u : 0u) | (s_flag ? 2u : 0u));
            const bool fin = done && !(st & 1u);
            if ((st & 2u) || fin) {
                if (lane == 0) wdone[warp] = fin ? 1 : 0;
                if (drain()) break;
                continue;
            }
            if (!(st & 1u)) {
                if (my_pos >= my_len) {   // ranges are never empty
                    int r = 0;
                    if (lane == 0) r = atomicAdd(&s_next, 1);
                    r = __shfl_sync(FULL, r, 0);
                    if (r >= nr) {
                        done = true;
                        continue;
                    }
                    const int rr = (int)(((unsigned)r * (unsigned)stride) % (unsigned)nr);
                    my_start = rstart[rr];
                    my_len = rlen[rr];
                    my_sl = rslot[rr];
                    my_pos = 0;
                }
                const int i0 = my_pos + lane, i1 = i0 + 32;
                const bool v0 = i0 < my_len, v1 = i1 < my_len;
                const int j0 = my_start + min(i0, my_len - 1), j1 = my_start + min(i1, my_len - 1);
                const int4 q0 = p.rec[j0];
                const int4 q1 = p.rec[j1];
                my_pos += 64;
                // the range's primary, re-read every step (fewer registers live across the
                // drains; a register prefetch of the next step measured 2 % at two CTAs per
                // SM but costs the third)
                const int4 pr = sPrim[my_sl];
                const uint32_t px = (uint32_t)pr.x, py = (uint32_t)pr.y, pz = (uint32_t)pr.z;
                const int kb = my_sl * nb;
                const int dx0 = (int)((uint32_t)q0.x - px), dx1 = (int)((uint32_t)q1.x - px);
                const int dy0 = (int)((uint32_t)q0.y - py), dy1 = (int)((uint32_t)q1.y - py);
                const int dz0 = (int)((uint32_t)q0.z - pz), dz1 = (int)((uint32_t)q1.z - pz);
                const float fx0 = (float)dx0, fy0 = (float)dy0, fz0 = (float)dz0;
                const float fx1 = (float)dx1, fy1 = (float)dy1, fz1 = (float)dz1;
                const int2 bb = cand_bin2(p, sE, nb, v0, v1, dx0, dy0, dz0, dx1, dy1, dz1, fx0, fy0, fz0, fx1, fy1,
                                          fz1);
                const int b0 = bb.x, b1 = bb.y;
                have0 = b0 >= 0;
                have1 = b1 >= 0;
                ent0 = j0;
                ent1 = j1;
                ek0 = kb + b0;
                ek1 = kb + b1;
            }
            append(have0, ent0, ek0);
            append(have1, ent1, ek1);
        }

        // ----- tile sums: every key's lanes added through one transpose
        {
            float *st = stage + (size_t)tid * NACCP;
            unpack<LMAX>(acc, dacc, st);
            st[NACC] = __int_as_float(rcnt);
        }
        __syncthreads();
        for (int i = tid; i < nk * (NACC + 1); i += T) {
            const int k = i / (NACC + 1), j = i % (NACC + 1);
            const int g0 = gfirst[k], g = gsize[k];
            if (j < NACC) {
                float t = 0.f;
                for (int q = 0; q < g; ++q) t += stage[(g0 + q) * NACCP + j];
                sacc[k * NACCP + j] = t;
            } else {
                int t = 0;
                for (int q = 0; q < g; ++q) t += __float_as_int(stage[(g0 + q) * NACCP + j]);
                sacc[k * NACCP + j] = __int_as_float(t);
            }
        }
        __syncthreads();

        // ----- tile outputs (as in k_pairs)
        // the tile's first primary (re-read: t0 is not kept)
        const long long g0 = p.tile_start ? p.tile_start[s_tile] : (long long)s_tile * P;
        if (p.alm) {
            for (int i = tid; i < np * nb * NLM; i += T) {
                const int slot = i / (nb * NLM), rem = i % (nb * NLM);
                const int b = rem / NLM, k = rem % NLM;
                const float raw = sacc[(slot * nb + b) * NACCP + k];
                float v;
                if (k == 0) {
                    v = a00(raw, b);
                } else {   // raw K_lm, rounded once up to the rounding of raw K_lo
                    const float kh = __ldg(&p.harm->kout[k][0]), kl = __ldg(&p.harm->kout[k][1]);
                    v = fmaf(raw, kh, __fmul_rn(raw, kl));
                }
                p.alm[(g0 + slot) * nb * NLM + rem] = v;
            }
        }
        if (p.counts)
            for (int i = tid; i < np * nb; i += T) p.counts[g0 * nb + i] = cnt[i];
        // random-random counts: a primary of negative weight with its secondaries of
        // negative weight (zero rows for the other primaries)
        if (p.counts_r)
            for (int i = tid; i < np * nb; i += T)
                p.counts_r[g0 * nb + i] =
                    (sPrim[i / nb].w < 0) ? __float_as_int(sacc[i * NACCP + NACC]) : 0;
        for (int b = tid; b < nb; b += T) {
            unsigned long long t = 0, tr = 0;
            for (int sl = 0; sl < np; ++sl) {
                t += (unsigned long long)cnt[sl * nb + b];
                if (sPrim[sl].w < 0) tr += (unsigned long long)__float_as_int(sacc[(sl * nb + b) * NACCP + NACC]);
            }
            spairs[b] += t;
            spairs_r[b] += tr;
        }
        // diagonal residuals w_i (|a_l^m[b]|^2 - s_ll^m[b]), the j = k term s removed: for
        // l >= 1 compensated (sq2_minus) on the unnormalised sums, then scaled by K_lm^2;
        // for l = 0 (where the periodic offset enters) in FP64; exactly zero for keys
        // with at most one pair (no j != k term) unless the offset makes a_0^0 differ
        // from the single pair's own term.  For l >= 1 the products with K_lm^2 and
        // w_i are FP32 (their roundings vary with the sums, so they carry no common
        // bias) and only the sum is FP64.  Summed into FP64 every tile.
        for (int i = tid; i < nb * NDIAG; i += T) {
            const int b = i / NDIAG, jd = i % NDIAG;
            int l = 0;
            while ((l + 1) * (l + 2) / 2 <= jd) ++l;
            const int m = jd - l * (l + 1) / 2;
            const float k2 = __ldg(&p.harm->k2[jd]);
            double acc2 = 0.0;
            for (int sl = 0; sl < np; ++sl) {
                const float *a = sacc + (sl * nb + b) * NACCP;
                const bool single = cnt[sl * nb + b] <= 1;
                const float wq = __int_as_float(sPrim[sl].w);
                if (l == 0) {
                    const double kd = __ldg(&p.harm->K[0][0]);
                    double d;
                    const double raw = (double)a[0];
                    double dd = raw * raw - (p.remove_self ? (double)a[NLM] : 0.0);
                    if (p.remove_self && single) dd = 0.0;   // raw^2 = w^2 up to the rounding of the self sum
                    d = kd * kd * dd;
                    if (p.use_mono) {
                        const double c = (s_mono_w - 1.0) * p.mono_coef[b];
                        d += c * (c - 2.0 * kd * raw);
                    }
                    acc2 = fma((double)wq, d, acc2);
                } else {
                    const float re = a[l * l + (m ? 2 * m - 1 : 0)];
                    const float im = m ? a[l * l + 2 * m] : 0.f;
                    float dq;
                    if (!p.remove_self) {
                        dq = fmaf(re, re, im * im);
                    } else if (single) {
                        dq = 0.f;
                    } else {
                        float ch = 0.f, cl = 0.f;
                        if constexpr (Direct<LMAX>::ON) {
                            ch = a[NLM + NSP + jd];
                        } else {
                            // s = sum_j (gd_hi + gd_lo)[j] acc_j as an unevaluated pair
#pragma unroll
                            for (int j = 0; j <= LMAX; ++j) {
                                const float h = __ldg(&p.harm->gd_hi[jd][j]), lo = __ldg(&p.harm->gd_lo[jd][j]);
                                const float x = a[NLM + j];
                                const float ph = __fmul_rn(h, x);
                                float pe = fmaf(h, x, -ph);
                                pe = fmaf(lo, x, pe);
                                float e;
                                ch = two_sum(ch, ph, e);
                                cl = __fadd_rn(cl, __fadd_rn(e, pe));
                            }
                        }
                        dq = sq2_minus(re, im, ch, cl);
                    }
                    acc2 += (double)__fmul_rn(__fmul_rn(k2, dq), wq);
                }
            }
            d64[i] += acc2;
        }
        for (int i = tid; i < nb * NSP; i += T) {
            const int b = i / NSP, j = i % NSP;
            double acc2 = 0.0;
            for (int sl = 0; sl < np; ++sl)
                acc2 += (double)__fmul_rn(__int_as_float(sPrim[sl].w), sacc[(sl * nb + b) * NACCP + NLM + j]);
            w64[i] += acc2;
        }
        // the bin shares for the next tile: half the old estimate, half this tile's counts
        if (warp == 0) {
            int c = 0;
            if (lane < nb)
                for (int sl = 0; sl < np; ++sl) c += cnt[sl * nb + lane];
            const float h = lane < nb ? hist[lane] : 0.f;
            int ct = c;
            float ht = h;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ct += __shfl_xor_sync(FULL, ct, o);
                ht += __shfl_xor_sync(FULL, ht, o);
            }
            if (lane < nb && ct > 0) hist[lane] = 0.5f * h / ht + 0.5f * (float)c / (float)ct + 1e-4f;
        }
        __syncthreads();
    }

    if (cta_mock >= 0) flush_cta(cta_mock);
}

}  // namespace tpcf
