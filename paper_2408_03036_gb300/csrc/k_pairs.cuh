// Pair stage of the anisotropic 3PCF estimator (Eq. alm of arXiv:2408.03036,
// Sec. 4.2): for every primary, neighbour search to r_max over a cell list,
// exact integer radial binning, and per-bin sums of w_j Y_l^m(r_hat_ij) with
// the line of sight along z.  Also the per-bin sums of w_j^2 f_j(mu) that give
// the degenerate j = k triangle term, and integer pair counts.
//
// One CTA works on a tile of P primaries at a time (persistent grid, tiles taken
// from an atomic counter).  For a tile:
//   1. the cell rows within reach of each primary are listed as contiguous
//      point ranges (cells are stored x-fastest, so a run of cells along x is
//      one range), trimmed per primary to the sphere of radius r_max;
//   2. warps take ranges one at a time (in a strided order that mixes radii)
//      and sweep them 32 candidates per step (coalesced 16-byte records); a
//      float window test on r^2 keeps the candidates that may lie in
//      [r_min, r_max), appended to the shared chunk with one reservation per
//      warp step;
//   3. when the chunk fills, every warp stops and the CTA processes it:
//      exact bin and unit vector per staged pair (float decision with a proven
//      margin, 64-bit integer comparison near an edge), per-warp key
//      histograms, a counting sort by key = slot * n_bins + bin, lanes grouped
//      per key in proportion to the key's run, the harmonic sums in registers,
//      and a per-warp transpose that adds each key's lanes into the warp's own
//      accumulator copy (no atomics);
//   4. the tile's sums are written out, and the diagonal-bin residuals
//      w_i (|a_l^m[b]|^2 - s^m_ll[b]) are summed per CTA, flushed to FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

// Constant tables passed by value (kernel parameter space is a constant bank).
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
};

template <int LMAX>
struct Layout {
    static constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    static constexpr int NSP = LMAX + 1;
    static constexpr int NACC = NLM + NSP;
    static constexpr int NACCP = NACC | 1;  // odd row stride: distinct banks for distinct keys
    static constexpr int NDIAG = (LMAX + 1) * (LMAX + 2) / 2;
};

__device__ __forceinline__ void latch_error(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// Accumulates one pair (unit vector x, y, z and weight w) into acc:
// acc[l^2 + ...] += w V_l^m(z) (x + i y)^m (real / imaginary parts), and the
// self sums acc[NLM + j] += w^2 f_j(z).
template <int LMAX>
__device__ __forceinline__ void accum_pair(float x, float y, float z, float w, float (&acc)[Layout<LMAX>::NACC])
{
    constexpr int NLM = Layout<LMAX>::NLM;
    constexpr int LZ = (2 * LMAX > 1) ? 2 * LMAX : 1;
    float wc[LMAX + 1], ws[LMAX + 1];
    wc[0] = w;
    ws[0] = 0.f;
    if (LMAX >= 1) {
        wc[1] = w * x;
        ws[1] = w * y;
    }
#pragma unroll
    for (int m = 2; m <= LMAX; ++m) {
        wc[m] = fmaf(wc[m - 1], x, -ws[m - 1] * y);
        ws[m] = fmaf(wc[m - 1], y, ws[m - 1] * x);
    }
    float zl[LZ + 1];                 // zl[l] = (2l - 1) z
    zl[0] = 0.f;
#pragma unroll
    for (int l = 1; l <= LZ; ++l) zl[l] = (float)(2 * l - 1) * z;
    float v0[LZ + 1];                 // V_l^0, kept for the self sums
#pragma unroll
    for (int m = 0; m <= LMAX; ++m) {
        float vm2 = 0.f, vm1 = 0.f;
#pragma unroll
        for (int l = m; l <= LMAX; ++l) {
            float v;
            if (l == m) v = 1.f;
            else if (l == m + 1) v = zl[m + 1];
            else v = fmaf(zl[l], vm1, -(float)((l + m - 1) * (l - m - 1)) * vm2);
            vm2 = vm1;
            vm1 = v;
            if (m == 0) {
                v0[l] = v;
                if (l == 0) acc[0] += w;
                else acc[l * l] = fmaf(v, wc[0], acc[l * l]);
            } else {
                if (l == m) {
                    acc[l * l + 2 * m - 1] += wc[m];
                    acc[l * l + 2 * m] += ws[m];
                } else {
                    acc[l * l + 2 * m - 1] = fmaf(v, wc[m], acc[l * l + 2 * m - 1]);
                    acc[l * l + 2 * m] = fmaf(v, ws[m], acc[l * l + 2 * m]);
                }
            }
        }
    }
    // continue V_l^0 up to l = 2 LMAX for the self sums
#pragma unroll
    for (int l = LMAX + 1; l <= 2 * LMAX; ++l) {
        if (l == 1) v0[1] = zl[1];
        else v0[l] = fmaf(zl[l], v0[l - 1], -(float)((l - 1) * (l - 1)) * v0[l - 2]);
    }
    const float w2 = w * w;
    acc[NLM] += w2;
#pragma unroll
    for (int j = 1; j <= LMAX; ++j) acc[NLM + j] = fmaf(w2, v0[2 * j], acc[NLM + j]);
}

// Shared-memory carve-up of the pair kernel (byte offsets).
struct SmemMap {
    int off_E, off_Ef, off_Elo, off_Ehi, off_prim, off_pf, off_pc;
    int off_rstart, off_rlen, off_rslot;
    int off_whist, off_wcur, off_cnt, off_cstart, off_clen, off_gfirst, off_gsize, off_lanekey;
    int off_acc, off_ent, off_key, off_sent;
    int off_d32, off_w32, off_d64, off_w64, off_pairs, off_misc;
    int total;
    int maxr;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

template <int LMAX, bool COUNTS>
__host__ __device__ inline SmemMap make_smem_map(int P, int nb, int s, int chunk, int block)
{
    SmemMap m;
    const int rows = (2 * s + 1) * (2 * s + 1);
    const int W = block / 32;
    m.maxr = 2 * P * rows;
    const int nk = P * nb;
    int o = 0;
    m.off_E = o;       o = align_up(o + 8 * (TPCF_MAX_BINS + 1), 16);
    m.off_Ef = o;      o = align_up(o + 4 * (TPCF_MAX_BINS + 1), 16);
    m.off_Elo = o;     o = align_up(o + 4 * (TPCF_MAX_BINS + 1), 16);
    m.off_Ehi = o;     o = align_up(o + 4 * (TPCF_MAX_BINS + 1), 16);
    m.off_prim = o;    o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pf = o;      o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pc = o;      o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_rstart = o;  o = align_up(o + 4 * m.maxr, 16);
    m.off_rlen = o;    o = align_up(o + 4 * m.maxr, 16);
    m.off_rslot = o;   o = align_up(o + 4 * m.maxr, 16);
    m.off_whist = o;   o = align_up(o + 4 * W * nk, 16);
    m.off_wcur = o;    o = align_up(o + 4 * W * nk, 16);
    m.off_cnt = o;     o = align_up(o + 4 * nk, 16);
    m.off_cstart = o;  o = align_up(o + 4 * nk, 16);
    m.off_clen = o;    o = align_up(o + 4 * nk, 16);
    m.off_gfirst = o;  o = align_up(o + 4 * nk, 16);
    m.off_gsize = o;   o = align_up(o + 4 * nk, 16);
    m.off_lanekey = o; o = align_up(o + 4 * block, 16);
    const int naccp = COUNTS ? 0 : Layout<LMAX>::NACCP;
    const int ndiag = COUNTS ? 0 : Layout<LMAX>::NDIAG;
    const int nsp = COUNTS ? 0 : Layout<LMAX>::NSP;
    const int cap = COUNTS ? 0 : chunk;
    // one accumulator copy per warp (warp-private: plain adds, no atomics)
    m.off_acc = o;     o = align_up(o + 4 * W * nk * naccp, 16);
    // staging segments (one per warp); reused as the per-warp transpose area once sorted
    const int ent_bytes = 16 * cap;
    const int stage_bytes = COUNTS ? 0 : 4 * block * naccp;
    m.off_ent = o;     o = align_up(o + (ent_bytes > stage_bytes ? ent_bytes : stage_bytes), 16);
    m.off_key = o;     o = align_up(o + 4 * cap, 16);
    m.off_sent = o;    o = align_up(o + 16 * cap, 16);
    m.off_d32 = o;     o = align_up(o + 4 * nb * ndiag, 16);
    m.off_w32 = o;     o = align_up(o + 4 * nb * nsp, 16);
    m.off_d64 = o;     o = align_up(o + 8 * nb * ndiag, 16);
    m.off_w64 = o;     o = align_up(o + 8 * nb * nsp, 16);
    m.off_pairs = o;   o = align_up(o + 8 * nb, 16);
    m.off_misc = o;    o = align_up(o + 4 * (16 + W), 16);
    m.total = o;
    return m;
}

__device__ __forceinline__ int gcd_int(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Block-wide exclusive scan of n ints in place at a (any n); returns the total.
__device__ inline int block_exclusive_scan(int *a, int n, int *scratch32)
{
    const int tid = threadIdx.x, T = blockDim.x;
    const int per = (n + T - 1) / T;
    const int b0 = tid * per;
    int local = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < n) local += a[b0 + i];
    const int lane = tid & 31, warp = tid >> 5;
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) scratch32[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = T >> 5;
        int x = lane < nw ? scratch32[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane < nw) scratch32[lane] = x;
    }
    __syncthreads();
    int run = v - local + (warp > 0 ? scratch32[warp - 1] : 0);
    const int total = scratch32[(T >> 5) - 1];
    for (int i = 0; i < per; ++i) {
        if (b0 + i < n) {
            int x = a[b0 + i];
            a[b0 + i] = run;
            run += x;
        }
    }
    __syncthreads();
    return total;
}

template <int LMAX, bool COUNTS>
__global__ void __launch_bounds__(256, (LMAX <= 4 ? 2 : 1)) k_pairs(const PairParams p, const HarmTables H)
{
    constexpr int NLM = Layout<LMAX>::NLM;
    constexpr int NACC = Layout<LMAX>::NACC;
    constexpr int NACCP = Layout<LMAX>::NACCP;
    constexpr int NDIAG = Layout<LMAX>::NDIAG;
    constexpr int NSP = Layout<LMAX>::NSP;
    constexpr float TOL = 1.0e-6f;        // > 5 * 2^-24 relative error of the float r^2

    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = T >> 5;
    const int nb = p.nb, P = p.P, s = p.s, nc = p.nc;
    const int side = 2 * s + 1, rows = side * side;
    const SmemMap M = make_smem_map<LMAX, COUNTS>(P, nb, s, p.chunk, T);
    const int nk = P * nb;
    const int room = COUNTS ? 0 : p.chunk - 32 * W;   // fill at which the chunk must be processed
    const unsigned lt_mask = (1u << lane) - 1u;

    unsigned long long *sE = reinterpret_cast<unsigned long long *>(smem + M.off_E);
    float *sEf = reinterpret_cast<float *>(smem + M.off_Ef);
    float *sElo = reinterpret_cast<float *>(smem + M.off_Elo);
    float *sEhi = reinterpret_cast<float *>(smem + M.off_Ehi);
    int4 *sPrim = reinterpret_cast<int4 *>(smem + M.off_prim);
    float4 *sPf = reinterpret_cast<float4 *>(smem + M.off_pf);
    int4 *sPc = reinterpret_cast<int4 *>(smem + M.off_pc);
    int *rstart = reinterpret_cast<int *>(smem + M.off_rstart);
    int *rlen = reinterpret_cast<int *>(smem + M.off_rlen);
    int *rslot = reinterpret_cast<int *>(smem + M.off_rslot);
    int *whist = reinterpret_cast<int *>(smem + M.off_whist);    // [W][nk]
    int *wcur = reinterpret_cast<int *>(smem + M.off_wcur);      // [W][nk]
    int *cnt = reinterpret_cast<int *>(smem + M.off_cnt);
    int *cstart = reinterpret_cast<int *>(smem + M.off_cstart);
    int *clen = reinterpret_cast<int *>(smem + M.off_clen);
    int *gfirst = reinterpret_cast<int *>(smem + M.off_gfirst);
    int *gsize = reinterpret_cast<int *>(smem + M.off_gsize);
    int *lanekey = reinterpret_cast<int *>(smem + M.off_lanekey);
    float *saccw = reinterpret_cast<float *>(smem + M.off_acc);   // [W][nk][NACCP]
    float *sacc = saccw;                                         // copy 0 holds the tile total
    float4 *ent = reinterpret_cast<float4 *>(smem + M.off_ent);  // [chunk] staged pairs
    float *stage = reinterpret_cast<float *>(smem + M.off_ent);  // [T][NACCP] after the scatter
    int *key = reinterpret_cast<int *>(smem + M.off_key);        // [chunk]: slot | candidate << 3
    float4 *sent = reinterpret_cast<float4 *>(smem + M.off_sent);
    float *d32 = reinterpret_cast<float *>(smem + M.off_d32);
    float *w32 = reinterpret_cast<float *>(smem + M.off_w32);
    double *d64 = reinterpret_cast<double *>(smem + M.off_d64);
    double *w64 = reinterpret_cast<double *>(smem + M.off_w64);
    unsigned long long *spairs = reinterpret_cast<unsigned long long *>(smem + M.off_pairs);
    int *misc = reinterpret_cast<int *>(smem + M.off_misc);
    int &s_tile = misc[0];
    int &s_next = misc[1];        // next range to hand out
    int &s_count = misc[3];       // staged pairs in the chunk
    volatile int &s_flag = misc[2];   // a staging segment is full
    int *scratch32 = misc + 8;    // 8 ints: per-warp totals for the scans (W <= 8)
    int *wdone = misc + 16;       // [W] warp has no more ranges

    for (int i = tid; i <= nb; i += T) {
        sE[i] = p.E[i];
        sEf[i] = p.Ef[i];
        sElo[i] = p.Ef[i] * (1.f + TOL);   // a float r^2 at or above this is surely >= E_i
        sEhi[i] = p.Ef[i] * (1.f - TOL);   // a float r^2 below this is surely < E_i
    }
    if (!COUNTS) {
        for (int i = tid; i < nb * NDIAG; i += T) { d32[i] = 0.f; d64[i] = 0.0; }
        for (int i = tid; i < nb * NSP; i += T) { w32[i] = 0.f; w64[i] = 0.0; }
    }
    for (int i = tid; i < nb; i += T) spairs[i] = 0ull;
    for (int i = tid; i < W * nk; i += T) whist[i] = 0;
    if (tid == 0) {
        s_flag = 0;
        s_count = 0;
    }
    double mono_w = p.use_mono ? (p.mono_w_dev ? *p.mono_w_dev : p.mono_w) : 0.0;
    int tiles_since_flush = 0;
    int cta_mock = -1;            // catalogue whose sums the CTA is accumulating
    __syncthreads();
    const int accw = nk * NACCP;   // floats per warp copy

    // a_0^0[b] from the raw weight sum, in double: Y_0^0 sum w - c_b
    auto a00 = [&](float wsum, int b) -> float {
        double v = (double)wsum * H.K[0][0];
        if (p.use_mono) v -= (mono_w - 1.0) * p.mono_coef[b];
        return (float)v;
    };

    // Exact radial bin from a float r^2 (computed as fma(x,x,fma(y,y,z*z)) from the
    // float separations); the float decision stands unless r^2 is within a relative
    // TOL of an edge, where the exact 64-bit integer separation decides.
    auto bin_of = [&](float r2f, int dx, int dy, int dz, bool have_int) -> int {
        if (!(r2f >= p.r2_lo && r2f < p.r2_hi)) return -1;
        int b = (int)((r2f * rsqrtf(r2f) - p.rmin_u) * p.inv_dr_u);
        b = min(max(b, 0), nb - 1);
        if (r2f >= sElo[b] && r2f < sEhi[b + 1]) return b;
        (void)have_int;
        const long long lx = dx, ly = dy, lz = dz;
        const unsigned long long r2 = (unsigned long long)(lx * lx) + (unsigned long long)(ly * ly)
                                    + (unsigned long long)(lz * lz);
        if (r2 < sE[0] || r2 >= sE[nb]) return -1;
        while (b > 0 && r2 < sE[b]) --b;
        while (b < nb - 1 && r2 >= sE[b + 1]) ++b;
        return b;
    };

    // ----- chunk processing (all threads; the chunk holds s_count staged pairs)
    auto process_chunk = [&]() {
        const int n_all = s_count;
        const int wb = (int)(((long long)n_all * warp) / W);
        const int n_w = (int)(((long long)n_all * (warp + 1)) / W) - wb;   // this warp's part
        // 0. per warp, over its part of the chunk: exact bin and unit vector; key histogram
        {
            float4 *went = ent + wb;
            int *wkeyv = key + wb;
            int *hist = whist + warp * nk;
            for (int base = 0; base < n_w; base += 32) {
                const int i = base + lane;
                int k = -1 - lane;   // unique per lane: never matches a real key
                if (i < n_w) {
                    const float4 v = went[i];
                    const int kv = wkeyv[i];
                    const int slot = kv & 7;
                    const float r2f = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
                    int b;
                    if (r2f >= p.r2_lo && r2f < p.r2_hi) {
                        int bb = (int)((r2f * rsqrtf(r2f) - p.rmin_u) * p.inv_dr_u);
                        bb = min(max(bb, 0), nb - 1);
                        if (r2f >= sElo[bb] && r2f < sEhi[bb + 1]) {
                            b = bb;
                        } else {
                            // near an edge: recover the exact integer separation
                            const int4 q = p.rec[(unsigned)kv >> 3];
                            const int4 pr = sPrim[slot];
                            b = bin_of(r2f, (int)((uint32_t)q.x - (uint32_t)pr.x),
                                       (int)((uint32_t)q.y - (uint32_t)pr.y),
                                       (int)((uint32_t)q.z - (uint32_t)pr.z), true);
                        }
                    } else {
                        b = -1;
                    }
                    if (b >= 0) {
                        // correctly rounded 1/sqrt: |n|^2 = 1 up to unbiased rounding,
                        // which the j = k cancellation on diagonal bins needs
                        const float inv = __frsqrt_rn(r2f);
                        went[i] = make_float4(v.x * inv, v.y * inv, v.z * inv, v.w);
                        k = slot * nb + b;
                    }
                    wkeyv[i] = k < 0 ? -1 : k;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, k);
                if (k >= 0 && lane == __ffs(peers) - 1) hist[k] += __popc(peers);
            }
        }
        __syncthreads();
        // 1. key totals and per-warp offsets; warp 0 scans the totals and assigns lanes
        for (int k = tid; k < nk; k += T) {
            int run = 0;
            for (int w = 0; w < W; ++w) {
                wcur[w * nk + k] = run;
                run += whist[w * nk + k];
                whist[w * nk + k] = 0;
            }
            clen[k] = run;
        }
        __syncthreads();
        int n_tot = 0;
        if (warp == 0) {
            const int per = (nk + 31) >> 5;     // <= 4 keys per lane (nk <= 128)
            const int k0 = lane * per;
            int len[4], loc = 0, act = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                len[i] = (i < per && k0 + i < nk) ? clen[k0 + i] : 0;
                loc += len[i];
                act += len[i] > 0;
            }
            int v = loc, a = act;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t1 = __shfl_up_sync(0xffffffffu, v, o);
                const int t2 = __shfl_up_sync(0xffffffffu, a, o);
                if (lane >= o) { v += t1; a += t2; }
            }
            n_tot = __shfl_sync(0xffffffffu, v, 31);
            const int K = __shfl_sync(0xffffffffu, a, 31);
            const int lam = n_tot > 0 ? (n_tot + (T - K) - 1) / (T - K) : 1;
            int gl[4], gsum = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                gl[i] = (len[i] + lam - 1) / lam;
                gsum += gl[i];
            }
            int gv = gsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t1 = __shfl_up_sync(0xffffffffu, gv, o);
                if (lane >= o) gv += t1;
            }
            for (int i = lane; i < T; i += 32) lanekey[i] = -1;
            __syncwarp();
            int run = v - loc, g0 = gv - gsum;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i < per && k0 + i < nk) {
                    const int k = k0 + i;
                    cstart[k] = run;
                    gfirst[k] = g0;
                    gsize[k] = gl[i];
                    cnt[k] += len[i];
                    for (int q = 0; q < gl[i]; ++q) lanekey[g0 + q] = k;
                    run += len[i];
                    g0 += gl[i];
                }
            }
        }
        __syncthreads();
        // 2. counting-sort scatter of every warp's part (warp-private cursors)
        {
            const float4 *went = ent + wb;
            const int *wkeyv = key + wb;
            int *cur = wcur + warp * nk;
            for (int base = 0; base < n_w; base += 32) {
                const int i = base + lane;
                const int k0 = i < n_w ? wkeyv[i] : -1;
                const bool valid = k0 >= 0;
                const int k = valid ? k0 : -1 - lane;
                const unsigned peers = __match_any_sync(0xffffffffu, k);
                const int leader = __ffs(peers) - 1;
                int b0 = 0;
                if (valid && lane == leader) {
                    b0 = cstart[k] + cur[k];
                    cur[k] += __popc(peers);
                }
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                if (valid) sent[b0 + __popc(peers & lt_mask)] = went[i];
            }
        }
        __syncthreads();
        // 3. every lane accumulates its key's run (stride g_k) in registers
        float acc[NACC];
#pragma unroll
        for (int j = 0; j < NACC; ++j) acc[j] = 0.f;
        const int myk = lanekey[tid];
        if (myk >= 0) {
            const int g = gsize[myk];
            const int end = cstart[myk] + clen[myk];
            for (int e = cstart[myk] + (tid - gfirst[myk]); e < end; e += g) {
                const float4 v = sent[e];
                accum_pair<LMAX>(v.x, v.y, v.z, v.w, acc);
            }
        }
        // 4. per warp: sum each key's lanes (a contiguous lane range) column by column
        float *st = stage + (size_t)tid * NACCP;
#pragma unroll
        for (int j = 0; j < NACC; ++j) st[j] = acc[j];
        __syncwarp();
        {
            float *mine = saccw + (size_t)warp * accw;
            const float *wst = stage + (size_t)warp * 32 * NACCP;
            const int *wkey = lanekey + warp * 32;
            int l = 0;
            while (l < 32) {
                const int k = wkey[l];
                if (k < 0) break;
                const int e = min(32, gfirst[k] + gsize[k] - warp * 32);
                for (int j = lane; j < NACC; j += 32) {
                    float s0 = 0.f, s1 = 0.f;
                    int q = l;
                    for (; q + 1 < e; q += 2) {
                        s0 += wst[q * NACCP + j];
                        s1 += wst[(q + 1) * NACCP + j];
                    }
                    if (q < e) s0 += wst[q * NACCP + j];
                    mine[k * NACCP + j] += s0 + s1;
                }
                l = e;
            }
        }
        __syncthreads();
        if (tid == 0) {
            s_flag = 0;
            s_count = 0;
        }
        __syncthreads();
    };

    // adds the CTA's FP64 diagonal / self / pair-count sums to catalogue `mk`'s
    // slice of the outputs and clears them (all threads)
    auto flush_cta = [&](int mk) {
        __syncthreads();
        if (!COUNTS) {
            for (int i = tid; i < nb * NDIAG; i += T) {
                const double v = d64[i] + (double)d32[i];
                const int b = i / NDIAG, jd = i % NDIAG;
                if (p.diag && v != 0.0) atomicAdd(p.diag + ((size_t)mk * NDIAG + jd) * nb + b, v);
                d64[i] = 0.0;
                d32[i] = 0.f;
            }
            for (int i = tid; i < nb * NSP; i += T) {
                const double v = w64[i] + (double)w32[i];
                const int b = i / NSP, j = i % NSP;
                if (p.wsp && v != 0.0) atomicAdd(p.wsp + ((size_t)mk * NSP + j) * nb + b, v);
                w64[i] = 0.0;
                w32[i] = 0.f;
            }
        }
        for (int b = tid; b < nb; b += T) {
            if (p.pair_counts && spairs[b]) atomicAdd(p.pair_counts + (size_t)mk * nb + b, spairs[b]);
            spairs[b] = 0ull;
        }
        tiles_since_flush = 0;
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) {
            s_tile = atomicAdd(p.work, 1);
            s_next = 0;
        }
        __syncthreads();
        const long long t0 = (long long)s_tile * P;
        if (t0 >= p.n_prim) break;
        const int np = (int)min((long long)P, p.n_prim - t0);
        const int mock = p.prim_mock ? p.prim_mock[t0] : 0;
        if (mock != cta_mock) {
            if (cta_mock >= 0) flush_cta(cta_mock);
            cta_mock = mock;
            if (p.prim_mock && p.use_mono) mono_w = p.mono_w_mock[mock];
        }
        const long long mock_cells = (long long)mock * p.ncell_mock;

        // primaries of the tile
        if (tid < np) {
            const int4 q = p.prim[t0 + tid];
            sPrim[tid] = q;
            const uint32_t ux = (uint32_t)q.x, uy = (uint32_t)q.y, uz = (uint32_t)q.z;
            sPf[tid] = make_float4((float)ux, (float)uy, (float)uz, __int_as_float(q.w));
            sPc[tid] = make_int4((int)(((unsigned long long)ux * nc) >> 32),
                                 (int)(((unsigned long long)uy * nc) >> 32),
                                 (int)(((unsigned long long)uz * nc) >> 32), 0);
            const float wq = __int_as_float(q.w);
            if (!(wq == wq) || isinf(wq)) latch_error(p.err, DEV_ERR_DATA);
        }
        for (int i = tid; i < np * nb; i += T) cnt[i] = 0;
        if (!COUNTS)
            for (int i = tid; i < W * accw; i += T) saccw[i] = 0.f;
        __syncthreads();

        // candidate ranges: per (slot, row) up to two contiguous runs of cells
        const int nr = 2 * np * rows;
        for (int r = tid; r < np * rows; r += T) {
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
                    int sa = x0, sb = x1, ta = 1, tb = 0;   // second run empty
                    if (p.periodic) {
                        if (x0 < 0) { sa = x0 + nc; sb = nc - 1; ta = 0; tb = x1; }
                        else if (x1 >= nc) { sa = x0; sb = nc - 1; ta = 0; tb = x1 - nc; }
                    }
                    a0 = p.cell_start[base + sa];
                    l0 = p.cell_start[base + sb + 1] - a0;
                    if (tb >= ta) {
                        a1 = p.cell_start[base + ta];
                        l1 = p.cell_start[base + tb + 1] - a1;
                    }
                }
            }
            rstart[2 * r] = a0; rlen[2 * r] = l0; rslot[2 * r] = slot;
            rstart[2 * r + 1] = a1; rlen[2 * r + 1] = l1; rslot[2 * r + 1] = slot;
        }
        __syncthreads();

        // ----- gather: warps take ranges and sweep them 32 candidates per step
        // ranges are handed out in a strided order so that every chunk mixes rows
        // from across the sphere (all radii), which keeps the key groups balanced
        int stride = (nr * 5) / 8 + 1;
        while (nr > 1 && gcd_int(stride, nr) != 1) ++stride;
        int my_start = 0, my_len = 0, my_pos = 0, my_slot = 0;
        bool done = false;
        for (;;) {
            while (!done && my_pos >= my_len) {
                int r = 0;
                if (lane == 0) r = atomicAdd(&s_next, 1);
                r = __shfl_sync(0xffffffffu, r, 0);
                if (r >= nr) {
                    done = true;
                } else {
                    const int rr = (int)(((long long)r * stride) % nr);
                    my_start = rstart[rr];
                    my_len = rlen[rr];
                    my_slot = rslot[rr];
                    my_pos = 0;
                }
            }
            if (COUNTS) {
                if (done) break;
                const int i = my_pos + lane;
                if (i < my_len) {
                    const int4 q = p.rec[my_start + i];
                    const int4 pr = sPrim[my_slot];
                    const int dx = (int)((uint32_t)q.x - (uint32_t)pr.x);
                    const int dy = (int)((uint32_t)q.y - (uint32_t)pr.y);
                    const int dz = (int)((uint32_t)q.z - (uint32_t)pr.z);
                    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
                    const int b = bin_of(fmaf(fx, fx, fmaf(fy, fy, fz * fz)), dx, dy, dz, true);
                    if (b >= 0) atomicAdd(&cnt[my_slot * nb + b], 1);
                }
                my_pos += 32;
                continue;
            }
            if (done || s_flag) {
                if (lane == 0) wdone[warp] = done ? 1 : 0;
                __syncthreads();
                int alldone = 1;
                for (int w = 0; w < W; ++w) alldone &= wdone[w];
                process_chunk();   // every warp here is done or the chunk is full
                if (alldone) break;
                continue;
            }
            const int i = my_pos + lane;
            bool ok = false;
            float4 e;
            int kv = 0;
            if (i < my_len) {
                const int idx = my_start + i;
                const int4 q = p.rec[idx];
                const int4 pr = sPrim[my_slot];
                const float fx = (float)(int)((uint32_t)q.x - (uint32_t)pr.x);
                const float fy = (float)(int)((uint32_t)q.y - (uint32_t)pr.y);
                const float fz = (float)(int)((uint32_t)q.z - (uint32_t)pr.z);
                const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                ok = (r2f >= p.r2_lo && r2f < p.r2_hi);
                e = make_float4(fx, fy, fz, __int_as_float(q.w));
                kv = my_slot | (idx << 3);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (bal) {
                // one reservation per warp step; a warp that takes the fill past
                // `room` raises the flag, and every warp stops after at most one
                // more step, so the chunk never overflows
                int b0 = 0;
                if (lane == 0) {
                    b0 = atomicAdd(&s_count, __popc(bal));
                    if (b0 + __popc(bal) > room) s_flag = 1;
                }
                b0 = __shfl_sync(0xffffffffu, b0, 0);
                if (ok) {
                    const int at = b0 + __popc(bal & lt_mask);
                    ent[at] = e;
                    key[at] = kv;
                }
            }
            my_pos += 32;
        }
        if (!COUNTS) {
            for (int i = tid; i < np * nb * NACCP; i += T) {
                float t = 0.f;
                for (int w = 0; w < W; ++w) t += saccw[(size_t)w * accw + i];
                sacc[i] = t;
            }
        }
        __syncthreads();

        // ----- tile outputs
        const long long g0 = t0;
        if (!COUNTS && p.alm) {
            for (int i = tid; i < np * nb * NLM; i += T) {
                const int slot = i / (nb * NLM), rem = i % (nb * NLM);
                const int b = rem / NLM, k = rem % NLM;
                const float raw = sacc[(slot * nb + b) * NACCP + k];
                float v;
                if (k == 0) {
                    v = a00(raw, b);
                } else {
                    int l = 1;
                    while ((l + 1) * (l + 1) <= k) ++l;
                    const int m = (k - l * l + 1) >> 1;
                    v = (float)((double)raw * H.K[l][m]);
                }
                p.alm[(g0 + slot) * nb * NLM + rem] = v;
            }
        }
        if (p.counts)
            for (int i = tid; i < np * nb; i += T) p.counts[g0 * nb + i] = cnt[i];
        for (int b = tid; b < nb; b += T) {
            unsigned long long t = 0;
            for (int sl = 0; sl < np; ++sl) t += (unsigned long long)cnt[sl * nb + b];
            spairs[b] += t;
        }
        if (!COUNTS) {
            // diagonal-bin residuals and self sums, FP32 per tile
            for (int i = tid; i < nb * NDIAG; i += T) {
                const int b = i / NDIAG, jd = i % NDIAG;
                int l = 0;
                while ((l + 1) * (l + 2) / 2 <= jd) ++l;
                const int m = jd - l * (l + 1) / 2;
                // residual in unnormalised units, then one common scale K_lm^2, so the
                // cancellation between |a|^2 and the j = k term is exact in exact arithmetic
                float acc = 0.f;
                const float k2 = (float)(H.K[l][m] * H.K[l][m]);
                for (int sl = 0; sl < np; ++sl) {
                    const float *a = sacc + (sl * nb + b) * NACCP;
                    float self = 0.f;
                    if (p.remove_self)
                        for (int j = 0; j <= LMAX; ++j) {
                            self = fmaf(H.gd_hi[jd][j], a[NLM + j], self);
                            self = fmaf(H.gd_lo[jd][j], a[NLM + j], self);
                        }
                    float d;
                    if (l == 0) {
                        const float re = a00(a[0], b);   // includes the analytic-random offset
                        d = fmaf(re, re, -k2 * self);
                    } else {
                        const float re = a[l * l + (m ? 2 * m - 1 : 0)];
                        const float im = m ? a[l * l + 2 * m] : 0.f;
                        d = k2 * (fmaf(re, re, im * im) - self);
                    }
                    acc += __int_as_float(sPrim[sl].w) * d;
                }
                d32[i] += acc;
            }
            for (int i = tid; i < nb * NSP; i += T) {
                const int b = i / NSP, j = i % NSP;
                float acc = 0.f;
                for (int sl = 0; sl < np; ++sl)
                    acc += __int_as_float(sPrim[sl].w) * sacc[(sl * nb + b) * NACCP + NLM + j];
                w32[i] += acc;
            }
            if (++tiles_since_flush >= 16) {
                tiles_since_flush = 0;
                for (int i = tid; i < nb * NDIAG; i += T) { d64[i] += (double)d32[i]; d32[i] = 0.f; }
                for (int i = tid; i < nb * NSP; i += T) { w64[i] += (double)w32[i]; w32[i] = 0.f; }
            }
        }
        __syncthreads();
    }

    // ----- CTA totals to global
    if (cta_mock >= 0) flush_cta(cta_mock);
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
    int off_E, off_Ef, off_Elo, off_Ehi, off_prim, off_pf, off_pc;
    int off_rstart, off_rlen, off_rslot;
    int off_qbase, off_qcap, off_qcnt, off_cnt, off_gfirst, off_gsize, off_lanekey, off_hist;
    int off_sacc, off_queue;
    int off_d32, off_w32, off_d64, off_w64, off_pairs, off_misc;
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
    m.off_Ef = o;      o = align_up(o + 4 * (TPCF_MAX_BINS + 1), 16);
    m.off_Elo = o;     o = align_up(o + 4 * (TPCF_MAX_BINS + 1), 16);
    m.off_Ehi = o;     o = align_up(o + 4 * (TPCF_MAX_BINS + 1), 16);
    m.off_prim = o;    o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pf = o;      o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_pc = o;      o = align_up(o + 16 * TPCF_MAX_TILE, 16);
    m.off_rstart = o;  o = align_up(o + 4 * m.maxr, 16);
    m.off_rlen = o;    o = align_up(o + 4 * m.maxr, 16);
    m.off_rslot = o;   o = align_up(o + 4 * m.maxr, 16);
    m.off_qbase = o;   o = align_up(o + 4 * nk, 16);
    m.off_qcap = o;    o = align_up(o + 4 * nk, 16);
    m.off_qcnt = o;    o = align_up(o + 4 * 2 * nk, 16);
    m.off_cnt = o;     o = align_up(o + 4 * nk, 16);
    m.off_gfirst = o;  o = align_up(o + 4 * nk, 16);
    m.off_gsize = o;   o = align_up(o + 4 * nk, 16);
    m.off_lanekey = o; o = align_up(o + 4 * block, 16);
    m.off_hist = o;    o = align_up(o + 4 * TPCF_MAX_BINS, 16);
    m.off_sacc = o;    o = align_up(o + 4 * nk * naccp, 16);
    // the queues; reused as the [block][NACCP] transpose area at the end of a tile
    const int qbytes = 16 * chunk, stage = 4 * block * naccp;
    m.off_queue = o;   o = align_up(o + (qbytes > stage ? qbytes : stage), 16);
    m.off_d32 = o;     o = align_up(o + 4 * nb * Layout<LMAX>::NDIAG, 16);
    m.off_w32 = o;     o = align_up(o + 4 * nb * Layout<LMAX>::NSP, 16);
    m.off_d64 = o;     o = align_up(o + 8 * nb * Layout<LMAX>::NDIAG, 16);
    m.off_w64 = o;     o = align_up(o + 8 * nb * Layout<LMAX>::NSP, 16);
    m.off_pairs = o;   o = align_up(o + 8 * nb, 16);
    m.off_misc = o;    o = align_up(o + 4 * (16 + W), 16);
    m.total = o;
    return m;
}

template <int LMAX>
__global__ void __launch_bounds__(256, (LMAX <= 4 ? 2 : 1)) k_pairs_q(const PairParams p, const HarmTables H)
{
    constexpr int NLM = Layout<LMAX>::NLM;
    constexpr int NACC = Layout<LMAX>::NACC;
    constexpr int NACCP = Layout<LMAX>::NACCP;
    constexpr int NDIAG = Layout<LMAX>::NDIAG;
    constexpr int NSP = Layout<LMAX>::NSP;
    constexpr float TOL = 1.0e-6f;        // > 5 * 2^-24 relative error of the float r^2
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = T >> 5;
    const int nb = p.nb, P = p.P, s = p.s, nc = p.nc, C = p.chunk;
    const int side = 2 * s + 1, rows = side * side;
    const QMap M = make_qmap<LMAX>(P, nb, s, C, T);
    const int nkmax = P * nb;

    unsigned long long *sE = reinterpret_cast<unsigned long long *>(smem + M.off_E);
    float *sEf = reinterpret_cast<float *>(smem + M.off_Ef);
    float *sElo = reinterpret_cast<float *>(smem + M.off_Elo);
    float *sEhi = reinterpret_cast<float *>(smem + M.off_Ehi);
    int4 *sPrim = reinterpret_cast<int4 *>(smem + M.off_prim);
    float4 *sPf = reinterpret_cast<float4 *>(smem + M.off_pf);
    int4 *sPc = reinterpret_cast<int4 *>(smem + M.off_pc);
    int *rstart = reinterpret_cast<int *>(smem + M.off_rstart);
    int *rlen = reinterpret_cast<int *>(smem + M.off_rlen);
    int *rslot = reinterpret_cast<int *>(smem + M.off_rslot);
    int *qbase = reinterpret_cast<int *>(smem + M.off_qbase);
    int *qcap = reinterpret_cast<int *>(smem + M.off_qcap);
    int *qcnt = reinterpret_cast<int *>(smem + M.off_qcnt);      // [2][nkmax]
    int *cnt = reinterpret_cast<int *>(smem + M.off_cnt);
    int *gfirst = reinterpret_cast<int *>(smem + M.off_gfirst);
    int *gsize = reinterpret_cast<int *>(smem + M.off_gsize);
    int *lanekey = reinterpret_cast<int *>(smem + M.off_lanekey);
    float *hist = reinterpret_cast<float *>(smem + M.off_hist);  // expected share of every bin
    float *sacc = reinterpret_cast<float *>(smem + M.off_sacc);  // [nk][NACCP] tile sums
    float4 *queue = reinterpret_cast<float4 *>(smem + M.off_queue);
    float *stage = reinterpret_cast<float *>(smem + M.off_queue);
    float *d32 = reinterpret_cast<float *>(smem + M.off_d32);
    float *w32 = reinterpret_cast<float *>(smem + M.off_w32);
    double *d64 = reinterpret_cast<double *>(smem + M.off_d64);
    double *w64 = reinterpret_cast<double *>(smem + M.off_w64);
    unsigned long long *spairs = reinterpret_cast<unsigned long long *>(smem + M.off_pairs);
    int *misc = reinterpret_cast<int *>(smem + M.off_misc);
    int &s_tile = misc[0];
    int &s_next = misc[1];
    volatile int &s_flag = misc[2];   // a queue is full
    int &s_nr = misc[3];              // non-empty candidate ranges of the tile
    int *wdone = misc + 16;           // [W] warp has no more ranges and nothing pending

    for (int i = tid; i <= nb; i += T) {
        sE[i] = p.E[i];
        sEf[i] = p.Ef[i];
        sElo[i] = p.Ef[i] * (1.f + TOL);
        sEhi[i] = p.Ef[i] * (1.f - TOL);
    }
    for (int i = tid; i < nb * NDIAG; i += T) { d32[i] = 0.f; d64[i] = 0.0; }
    for (int i = tid; i < nb * NSP; i += T) { w32[i] = 0.f; w64[i] = 0.0; }
    for (int i = tid; i < nb; i += T) spairs[i] = 0ull;
    for (int i = tid; i < 2 * nkmax; i += T) qcnt[i] = 0;
    if (tid < nb) {
        // seed: the shell volumes, r^3 in units of the bin edges' squares
        const float a = sqrtf(p.Ef[tid]), b = sqrtf(p.Ef[tid + 1]);
        hist[tid] = b * b * b - a * a * a;
    }
    if (tid == 0) s_flag = 0;
    double mono_w = p.use_mono ? (p.mono_w_dev ? *p.mono_w_dev : p.mono_w) : 0.0;
    int tiles_since_flush = 0;
    int cta_mock = -1;
    int par = 0;                      // live half of the double-buffered queue counters
    __syncthreads();

    auto a00 = [&](float wsum, int b) -> float {
        double v = (double)wsum * H.K[0][0];
        if (p.use_mono) v -= (mono_w - 1.0) * p.mono_coef[b];
        return (float)v;
    };

    auto flush_cta = [&](int mk) {
        __syncthreads();
        for (int i = tid; i < nb * NDIAG; i += T) {
            const double v = d64[i] + (double)d32[i];
            const int b = i / NDIAG, jd = i % NDIAG;
            if (p.diag && v != 0.0) atomicAdd(p.diag + ((size_t)mk * NDIAG + jd) * nb + b, v);
            d64[i] = 0.0;
            d32[i] = 0.f;
        }
        for (int i = tid; i < nb * NSP; i += T) {
            const double v = w64[i] + (double)w32[i];
            const int b = i / NSP, j = i % NSP;
            if (p.wsp && v != 0.0) atomicAdd(p.wsp + ((size_t)mk * NSP + j) * nb + b, v);
            w64[i] = 0.0;
            w32[i] = 0.f;
        }
        for (int b = tid; b < nb; b += T) {
            if (p.pair_counts && spairs[b]) atomicAdd(p.pair_counts + (size_t)mk * nb + b, spairs[b]);
            spairs[b] = 0ull;
        }
        tiles_since_flush = 0;
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
        const int nk = np * nb;
        const int mock = p.prim_mock ? p.prim_mock[t0] : 0;
        if (mock != cta_mock) {
            if (cta_mock >= 0) flush_cta(cta_mock);
            cta_mock = mock;
            if (p.prim_mock && p.use_mono) mono_w = p.mono_w_mock[mock];
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
            if (!(wq == wq) || isinf(wq)) latch_error(p.err, DEV_ERR_DATA);
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
                    qbase[k] = sl * ctot + cs - capb;
                    qcap[k] = capb;
                    const int g0 = sl * gtot + gs - gb;
                    gfirst[k] = g0;
                    gsize[k] = gb;
                    cnt[k] = 0;
                    for (int q = 0; q < gb; ++q) lanekey[g0 + q] = k;
                }
            }
        }
        __syncthreads();

        // candidate ranges (as in k_pairs), non-empty ones listed in any order
        for (int r = tid; r < np * rows; r += T) {
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
                    int sa = x0, sb = x1, ta = 1, tb = 0;
                    if (p.periodic) {
                        if (x0 < 0) { sa = x0 + nc; sb = nc - 1; ta = 0; tb = x1; }
                        else if (x1 >= nc) { sa = x0; sb = nc - 1; ta = 0; tb = x1 - nc; }
                    }
                    a0 = p.cell_start[base + sa];
                    l0 = p.cell_start[base + sb + 1] - a0;
                    if (tb >= ta) {
                        a1 = p.cell_start[base + ta];
                        l1 = p.cell_start[base + tb + 1] - a1;
                    }
                }
            }
            if (l0 > 0) {
                const int at = atomicAdd(&s_nr, 1);
                rstart[at] = a0; rlen[at] = l0; rslot[at] = slot;
            }
            if (l1 > 0) {
                const int at = atomicAdd(&s_nr, 1);
                rstart[at] = a1; rlen[at] = l1; rslot[at] = slot;
            }
        }
        __syncthreads();
        const int nr = s_nr;

        const int myk = lanekey[tid];
        const int myg = myk >= 0 ? gsize[myk] : 1;
        const int myr = myk >= 0 ? tid - gfirst[myk] : 0;
        const int myq = myk >= 0 ? qbase[myk] : 0;
        const int mycap = myk >= 0 ? qcap[myk] : 0;
        float acc[NACC];
#pragma unroll
        for (int j = 0; j < NACC; ++j) acc[j] = 0.f;

        // drains the queues (all threads); returns whether every warp has finished
        auto drain = [&]() -> bool {
            __syncthreads();                                   // (A) appends are visible
            int alldone = 1;
            for (int w = 0; w < W; ++w) alldone &= wdone[w];
            const int *live = qcnt + par * nkmax;
            if (tid < nk) cnt[tid] += min(live[tid], qcap[tid]);
            if (tid < nkmax) qcnt[(par ^ 1) * nkmax + tid] = 0;   // the other half: free since the last drain
            if (tid == 0) s_flag = 0;
            if (myk >= 0) {
                const int n = min(live[myk], mycap);
                const float4 *qq = queue + myq;
                for (int e = myr; e < n; e += myg) {
                    const float4 v = qq[e];
                    const float r2f = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
                    // correctly rounded 1/sqrt: |n|^2 = 1 up to unbiased rounding,
                    // which the j = k cancellation on diagonal bins needs
                    const float inv = __frsqrt_rn(r2f);
                    accum_pair<LMAX>(v.x * inv, v.y * inv, v.z * inv, v.w, acc);
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
        int my_start = 0, my_len = 0, my_pos = 0, kb = 0;
        uint32_t px = 0, py = 0, pz = 0;
        bool done = false, have = false;
        float4 ent = make_float4(0.f, 0.f, 0.f, 0.f);
        int ek = 0;
        for (;;) {
            // bit 0: an entry of the warp waits for room; bit 1: a queue is full
            const unsigned st = __reduce_or_sync(FULL, (have ? 1u : 0u) | (s_flag ? 2u : 0u));
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
                    const int sl = rslot[rr];
                    const int4 pr = sPrim[sl];
                    px = (uint32_t)pr.x;
                    py = (uint32_t)pr.y;
                    pz = (uint32_t)pr.z;
                    kb = sl * nb;
                    my_pos = 0;
                }
                const int i = my_pos + lane;
                my_pos += 32;
                const bool valid = i < my_len;
                const int4 q = p.rec[my_start + min(i, my_len - 1)];
                const int dx = (int)((uint32_t)q.x - px);
                const int dy = (int)((uint32_t)q.y - py);
                const int dz = (int)((uint32_t)q.z - pz);
                const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
                const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                // bin coordinate t = (r - r_min) / dr; its integer part is the bin unless
                // t is within tdelta of an integer, where the 64-bit separation decides
                const float rg = fmaxf(r2f, 1.f);
                const float t = fmaf(rg * rsqrtf(rg), p.inv_dr_u, p.t_off);
                const float tf = floorf(t);
                int b = (int)tf;
                const float fr = t - tf;
                const bool sure = fr > p.tdelta && fr < 1.f - p.tdelta;
                bool ok = valid && sure && b >= 0 && b < nb;
                const bool unsure = valid && !sure && t > -1.f && t < (float)(nb + 1);
                if (__any_sync(FULL, unsure)) {
                    if (unsure) {
                        const long long lx = dx, ly = dy, lz = dz;
                        const unsigned long long r2 = (unsigned long long)(lx * lx)
                                                    + (unsigned long long)(ly * ly)
                                                    + (unsigned long long)(lz * lz);
                        ok = r2 >= sE[0] && r2 < sE[nb];
                        b = min(max(b, 0), nb - 1);
                        while (b > 0 && r2 < sE[b]) --b;
                        while (b < nb - 1 && r2 >= sE[b + 1]) ++b;
                    }
                }
                have = ok;
                ent = make_float4(fx, fy, fz, __int_as_float(q.w));
                ek = kb + b;
            }
            if (have) {
                const int pos = atomicAdd(&qcnt[par * nkmax + ek], 1);
                if (pos < qcap[ek]) {
                    queue[qbase[ek] + pos] = ent;
                    have = false;
                } else {
                    s_flag = 1;   // stays pending until the queues are drained
                }
            }
        }

        // ----- tile sums: every key's lanes added through one transpose
        {
            float *st = stage + (size_t)tid * NACCP;
#pragma unroll
            for (int j = 0; j < NACC; ++j) st[j] = acc[j];
        }
        __syncthreads();
        for (int i = tid; i < nk * NACC; i += T) {
            const int k = i / NACC, j = i % NACC;
            const int g0 = gfirst[k], g = gsize[k];
            float t = 0.f;
            for (int q = 0; q < g; ++q) t += stage[(g0 + q) * NACCP + j];
            sacc[k * NACCP + j] = t;
        }
        __syncthreads();

        // ----- tile outputs (as in k_pairs)
        const long long g0 = t0;
        if (p.alm) {
            for (int i = tid; i < np * nb * NLM; i += T) {
                const int slot = i / (nb * NLM), rem = i % (nb * NLM);
                const int b = rem / NLM, k = rem % NLM;
                const float raw = sacc[(slot * nb + b) * NACCP + k];
                float v;
                if (k == 0) {
                    v = a00(raw, b);
                } else {
                    int l = 1;
                    while ((l + 1) * (l + 1) <= k) ++l;
                    const int m = (k - l * l + 1) >> 1;
                    v = (float)((double)raw * H.K[l][m]);
                }
                p.alm[(g0 + slot) * nb * NLM + rem] = v;
            }
        }
        if (p.counts)
            for (int i = tid; i < np * nb; i += T) p.counts[g0 * nb + i] = cnt[i];
        for (int b = tid; b < nb; b += T) {
            unsigned long long t = 0;
            for (int sl = 0; sl < np; ++sl) t += (unsigned long long)cnt[sl * nb + b];
            spairs[b] += t;
        }
        for (int i = tid; i < nb * NDIAG; i += T) {
            const int b = i / NDIAG, jd = i % NDIAG;
            int l = 0;
            while ((l + 1) * (l + 2) / 2 <= jd) ++l;
            const int m = jd - l * (l + 1) / 2;
            float acc2 = 0.f;
            const float k2 = (float)(H.K[l][m] * H.K[l][m]);
            for (int sl = 0; sl < np; ++sl) {
                const float *a = sacc + (sl * nb + b) * NACCP;
                float self = 0.f;
                if (p.remove_self)
                    for (int j = 0; j <= LMAX; ++j) {
                        self = fmaf(H.gd_hi[jd][j], a[NLM + j], self);
                        self = fmaf(H.gd_lo[jd][j], a[NLM + j], self);
                    }
                float d;
                if (l == 0) {
                    const float re = a00(a[0], b);
                    d = fmaf(re, re, -k2 * self);
                } else {
                    const float re = a[l * l + (m ? 2 * m - 1 : 0)];
                    const float im = m ? a[l * l + 2 * m] : 0.f;
                    d = k2 * (fmaf(re, re, im * im) - self);
                }
                acc2 += __int_as_float(sPrim[sl].w) * d;
            }
            d32[i] += acc2;
        }
        for (int i = tid; i < nb * NSP; i += T) {
            const int b = i / NSP, j = i % NSP;
            float acc2 = 0.f;
            for (int sl = 0; sl < np; ++sl)
                acc2 += __int_as_float(sPrim[sl].w) * sacc[(sl * nb + b) * NACCP + NLM + j];
            w32[i] += acc2;
        }
        if (++tiles_since_flush >= 16) {
            tiles_since_flush = 0;
            for (int i = tid; i < nb * NDIAG; i += T) { d64[i] += (double)d32[i]; d32[i] = 0.f; }
            for (int i = tid; i < nb * NSP; i += T) { w64[i] += (double)w32[i]; w32[i] = 0.f; }
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
