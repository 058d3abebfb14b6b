// Coupling over primaries on the 5th-generation tensor cores (tcgen05, TMEM).
//
// G_m = sum_i w_i (Re v_i Re v_i^T + Im v_i Im v_i^T) for every azimuthal m
// (Eq. measured_mult summed over primaries, Sec. 4.2 of arXiv:2408.03036), with
// v_i the per-primary harmonic sums a_l^m[b], l = m..l_max, b = 0..n_b-1.  As a
// matrix product D = A B^T with K running over (primary, real/imaginary part):
// A = (w v)^T rows, B = v^T rows, both K-major.
//
// Split precision: every operand value x is written as hi + lo in the MMA type
// (bf16 or tf32) and D accumulates hi_A hi_B + hi_A lo_B + lo_A hi_B in FP32 in
// tensor memory; the dropped lo_A lo_B term is below 2^-16 (bf16) or 2^-22 (tf32)
// of each product.  Partial sums are moved to FP64 every kFlushK K-rows.
//
// The m blocks are packed into 128-row tiles (blocks above 128 rows take two
// units of 128 rows against all their rows) and the tiles into CTA groups of at
// most 512 TMEM columns; one CTA covers its group for one slice of primaries, so
// a primary's row of a_l^m is read once per group.  A stage holds 16 primaries
// (8 for tf32) x (real, imaginary part) of every staged row, written as 16-byte
// core-matrix rows of the canonical no-swizzle K-major layout (core matrices
// adjacent in K 128 bytes apart, 8-row groups KS/8 x 128 bytes apart), and is
// double-buffered: threads stage one buffer while the tensor cores read the
// other.  One elected thread issues the MMAs and commits them to an mbarrier
// per buffer.  Every wait is bounded; a timeout latches an error flag, waits for
// the MMAs in flight, releases tensor memory and returns.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace tpcf {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kRowTile = 128;                 // M of every MMA (TMEM lanes)

// Two values at once: hi = bf16x2(a, b) rounded to nearest, lo = bf16x2 of the
// exact FP32 remainders; element a in the low half (lower K index).
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

constexpr int kMaxM = TPCF_MAX_LMAX + 1;
constexpr int kMaxUnits = 2 * kMaxM;
constexpr int kMaxRows = 384;                 // staged operand rows per CTA (two stages fit)

// One MMA target: D[128 x n] at TMEM column tmem_col = A rows a_row.. (128) times
// B rows b_row.. (n), both in the CTA's staged rows; part_off locates the unit's
// [128][n] FP64 block in every slice's partial sums.
struct TcUnit {
    int a_row, b_row, n, tmem_col;
    long long part_off;
};
// Staged rows row .. row + rows - 1 hold the m block (rows = n_b (l_max - m + 1)).
struct TcSeg {
    int row, m, rows;
};
struct TcGroup {
    int unit0, n_units, seg0, n_segs, rows_alloc, tmem_alloc;
};
// G_m[i][j] = D_{unit_lo}[off + i][off + j] (one tile) or, for blocks above 128
// rows, D_{unit_lo}[i][j] for i < 128 and D_{unit_hi}[i - 128][j].
struct TcMap {
    int unit_lo, unit_hi, off;
};
struct TcPlan {
    int n_groups, n_units, n_segs;
    TcGroup g[kMaxM];
    TcUnit u[kMaxUnits];
    TcSeg s[kMaxM];
    TcMap map[kMaxM];
    long long slice_size;   // doubles of partial sums per slice
};

struct TcParams {
    const float *alm;
    const float *w;
    int64_t K;            // primaries
    int nb, lmax;
    int64_t per_slice;    // primaries per slice
    int n_slices;
    // slice boundaries [n_slices + 1] in device memory (a batch: slices never
    // straddle two catalogues); null: slice s is [s per_slice, (s + 1) per_slice) of K
    const int64_t *slice_k;
    double *partial;      // [n_slices][slice_size], zeroed before the launch
    int *err;
    long long wait_limit; // polls of a per-stage mbarrier wait before giving up
    int wait_unmet;       // test mode: one more wait on a phase that nothing completes
    TcPlan plan;
};

__host__ __device__ inline int pad16(int n) { return (n + 15) / 16 * 16; }

// Packs the m blocks into CTA groups.  Blocks above 128 rows take two 128-row
// units against all their rows; smaller blocks share 128-row tiles (first fit,
// largest first), whose unit computes the tile's full square (cross-block entries
// are not used).  A group holds at most 512 TMEM columns and kMaxRows staged rows.
bool make_tc_plan(int nb, int lmax, TcPlan &P)
{
    std::memset(&P, 0, sizeof(P));
    struct Item { int rows, cols; bool big; int ms[kMaxM], mo[kMaxM], nm; };
    Item items[kMaxM];
    int ni = 0;
    int order[kMaxM];
    for (int m = 0; m <= lmax; ++m) order[m] = m;   // n_m decreases with m
    for (int k = 0; k <= lmax; ++k) {
        const int m = order[k];
        const int n = nb * (lmax - m + 1);
        if (n > 256) return false;
        if (n > 128) {
            Item &it = items[ni++];
            it.rows = n; it.cols = 2 * pad16(n); it.big = true; it.nm = 1; it.ms[0] = m; it.mo[0] = 0;
            continue;
        }
        int t = -1;
        for (int q = 0; q < ni; ++q)
            if (!items[q].big && items[q].rows + n <= 128) { t = q; break; }
        if (t < 0) {
            t = ni++;
            items[t].rows = 0; items[t].big = false; items[t].nm = 0;
        }
        Item &it = items[t];
        it.ms[it.nm] = m; it.mo[it.nm] = it.rows; ++it.nm;
        it.rows += n;
        it.cols = pad16(it.rows);
    }
    // groups: first fit in item order (largest first)
    int grp_of[kMaxM], g_cols[kMaxM], g_rows[kMaxM], g_alloc[kMaxM];
    int ng = 0;
    for (int q = 0; q < ni; ++q) {
        const Item &it = items[q];
        const int r8 = (it.rows + 7) / 8 * 8;
        int g = -1;
        for (int h = 0; h < ng; ++h) {
            const int start = g_rows[h];
            const int need = std::max(g_alloc[h], std::max(start + r8, start + (it.big ? 256 : 128)));
            if (g_cols[h] + it.cols <= 512 && need <= kMaxRows) { g = h; break; }
        }
        if (g < 0) {
            g = ng++;
            g_cols[g] = 0; g_rows[g] = 0; g_alloc[g] = 0;
        }
        const int start = g_rows[g];
        g_alloc[g] = std::max(g_alloc[g], std::max(start + r8, start + (it.big ? 256 : 128)));
        if (g_alloc[g] > kMaxRows) return false;
        g_rows[g] = start + r8;
        g_cols[g] += it.cols;
        grp_of[q] = g;
    }
    // units and segments, group by group
    long long part = 0;
    for (int g = 0; g < ng; ++g) {
        TcGroup &G = P.g[g];
        G.unit0 = P.n_units; G.seg0 = P.n_segs;
        int row = 0, col = 0;
        for (int q = 0; q < ni; ++q) {
            if (grp_of[q] != g) continue;
            const Item &it = items[q];
            const int n = pad16(it.rows);
            if (it.big) {
                const int m = it.ms[0];
                P.map[m] = {P.n_units, P.n_units + 1, 0};
                P.u[P.n_units++] = {row, row, n, col, part};
                part += 128LL * n;
                P.u[P.n_units++] = {row + 128, row, n, col + n, part};
                part += 128LL * n;
                col += 2 * n;
                P.s[P.n_segs++] = {row, m, it.rows};
            } else {
                for (int j = 0; j < it.nm; ++j) {
                    P.map[it.ms[j]] = {P.n_units, -1, it.mo[j]};
                    P.s[P.n_segs++] = {row + it.mo[j], it.ms[j], nb * (lmax - it.ms[j] + 1)};
                }
                P.u[P.n_units++] = {row, row, n, col, part};
                part += 128LL * n;
                col += n;
            }
            row += (it.rows + 7) / 8 * 8;
        }
        G.n_units = P.n_units - G.unit0;
        G.n_segs = P.n_segs - G.seg0;
        G.rows_alloc = g_alloc[g];
        int alloc = 32;
        while (alloc < col) alloc <<= 1;
        G.tmem_alloc = alloc;
    }
    P.n_groups = ng;
    P.slice_size = part;
    return true;
}

template <bool TF32>
__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(const TcParams p)
{
    constexpr int KP = TF32 ? 8 : 16;          // primaries per stage
    constexpr int KS = 2 * KP;                 // K entries per stage (real and imaginary part)
    constexpr int ESZ = TF32 ? 4 : 2;
    constexpr int KSTEP = TF32 ? 8 : 16;       // K per MMA
    constexpr int NKS = KS / KSTEP;
    constexpr int PER_CM = 16 / ESZ;           // elements per 16-byte core-matrix row
    constexpr uint32_t SBO = (KS / PER_CM) * 128;   // bytes between 8-row groups
    constexpr int FLUSH_P = 512;               // primaries (1024 K rows) per FP32 accumulation run

    extern __shared__ __align__(128) unsigned char smem[];
    const TcGroup G = p.plan.g[blockIdx.x];
    const int slice = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = p.nb, nlm = (p.lmax + 1) * (p.lmax + 1);
    const int R = G.rows_alloc;
    const uint32_t op_bytes = (uint32_t)R * KS * ESZ;
    const uint32_t stage_bytes = 4 * op_bytes;        // A_hi, A_lo, B_hi, B_lo
    int4 *rowinfo = reinterpret_cast<int4 *>(smem + 2 * stage_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes + 16 * R);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 2 * stage_bytes + 16 * R + 16);
    volatile int *s_abort = reinterpret_cast<int *>(smem + 2 * stage_bytes + 16 * R + 20);

    const int64_t i_beg = p.slice_k ? p.slice_k[slice] : (int64_t)slice * p.per_slice;
    const int64_t i_end = p.slice_k ? p.slice_k[slice + 1] : min(p.K, i_beg + p.per_slice);
    const int64_t nst = i_end > i_beg ? (i_end - i_beg + KP - 1) / KP : 0;

    // row table; unused rows stay zero in both stages for the whole launch
    for (int r = tid; r < R; r += kThreads) {
        int4 ri = make_int4(0, -1, 0, 0);
        for (int q = 0; q < G.n_segs; ++q) {
            const TcSeg sg = p.plan.s[G.seg0 + q];
            if (r >= sg.row && r < sg.row + sg.rows) {
                const int within = r - sg.row, l = sg.m + within / nb;
                ri = make_int4(l * l + (sg.m ? 2 * sg.m - 1 : 0), sg.m ? l * l + 2 * sg.m : -1, within % nb, 1);
            }
        }
        rowinfo[r] = ri;
    }
    for (uint32_t q = tid; q < 2 * stage_bytes / 16; q += kThreads)
        reinterpret_cast<uint4 *>(smem)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(G.tmem_alloc));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    double *part = p.partial + (int64_t)slice * p.plan.slice_size;

    uint32_t phase[2] = {0u, 0u};
    bool used[2] = {false, false};
    bool acc_on = false, ok = true;
    int since = 0;

    // TMEM (FP32) -> this slice's FP64 partial sums (all threads)
    auto flush = [&]() {
        if (tid == 0)
            for (int s = 0; s < 2; ++s)
                if (used[s] && !mbar_wait(&bars[s], phase[s] ^ 1u, p.wait_limit)) *s_abort = 1;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        used[0] = used[1] = false;
        if (*s_abort) return;
        // warp w reads TMEM lanes 32 (w % 4) ..; the warps sharing a lane quarter split the columns
        constexpr int NSETS = kThreads / 128;
        const int quarter = warp & 3, set = warp >> 2;
        const int row = 32 * quarter + lane;
        for (int q = 0; q < G.n_units; ++q) {
            const TcUnit u = p.plan.u[G.unit0 + q];
            double *dst = part + u.part_off + (int64_t)row * u.n;
            for (int c0 = 16 * set; c0 < u.n; c0 += 16 * NSETS) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(u.tmem_col + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) dst[c0 + j] += (double)v[j];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        acc_on = false;
    };

    // software pipeline: the values of stage st + 1 are loaded into registers while
    // stage st is written to shared memory and its MMAs are issued.  A thread's
    // items (octet o of row r) are the same in every stage: their source columns
    // and destination offsets are computed once.
    constexpr int OCT = KP / 4;                                  // octets per row and stage
    constexpr int MAXI = (kMaxRows * OCT + kThreads - 1) / kThreads;
    const int n_items = R * OCT;
    const int64_t RL = (int64_t)nb * nlm;                        // floats per primary
    int it_col[MAXI], it_dsin[MAXI], it_o[MAXI];
    uint32_t it_off[MAXI];
    bool it_on[MAXI];
#pragma unroll
    for (int it = 0; it < MAXI; ++it) {
        const int item = tid + it * kThreads;
        const int r = item % R, o = item / R;
        const int4 ri = item < n_items ? rowinfo[r] : make_int4(0, -1, 0, 0);
        it_on[it] = item < n_items && ri.w;
        it_col[it] = ri.z * nlm + ri.x;
        it_dsin[it] = ri.y >= 0 ? ri.y - ri.x : -1;
        it_o[it] = o;
        it_off[it] = TF32 ? (uint32_t)(((r >> 3) * (KS / 4) + (8 * o) / 4) * 128 + (r & 7) * 16)
                          : (uint32_t)(((r >> 3) * (KS / 8) + o) * 128 + (r & 7) * 16);
    }
    float xv[MAXI][8], wq[MAXI][4];
    auto load_stage = [&](int64_t st) {
        const int64_t i0 = i_beg + st * KP;
#pragma unroll
        for (int it = 0; it < MAXI; ++it) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t i = i0 + 4 * it_o[it] + q;
                float xc = 0.f, xs = 0.f, wi = 0.f;
                if (it_on[it] && i < i_end) {
                    const float *src = p.alm + i * RL + it_col[it];
                    xc = __ldg(src);
                    xs = it_dsin[it] >= 0 ? __ldg(src + it_dsin[it]) : 0.f;
                    wi = p.w ? __ldg(p.w + i) : 1.f;
                }
                xv[it][2 * q] = xc;
                xv[it][2 * q + 1] = xs;
                wq[it][q] = wi;
            }
        }
    };
    if (nst > 0) load_stage(0);

    for (int64_t st = 0; st < nst; ++st) {
        const int s = (int)(st & 1);
        unsigned char *stg = smem + s * stage_bytes;
        // the MMAs that last read this stage must have completed
        if (tid == 0 && used[s] && !mbar_wait(&bars[s], phase[s] ^ 1u, p.wait_limit)) *s_abort = 1;
        __syncthreads();
        if (*s_abort) { ok = false; break; }
        // stage: item (octet o, row r) = 8 K entries (4 primaries x real/imaginary) of row r
#pragma unroll
        for (int it = 0; it < MAXI; ++it) {
            if (!it_on[it]) continue;
            float wv[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                wv[2 * q] = wq[it][q] * xv[it][2 * q];
                wv[2 * q + 1] = wq[it][q] * xv[it][2 * q + 1];
            }
            const uint32_t off = it_off[it];
            if (TF32) {
                uint32_t bh[8], bl[8], ah[8], al[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    split_tf32(xv[it][j], bh[j], bl[j]);
                    split_tf32(wv[j], ah[j], al[j]);
                }
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const uint32_t o2 = off + 128u * half;   // the next core matrix along K
                    const int j0 = 4 * half;
                    *reinterpret_cast<uint4 *>(stg + o2) = make_uint4(ah[j0], ah[j0 + 1], ah[j0 + 2], ah[j0 + 3]);
                    *reinterpret_cast<uint4 *>(stg + op_bytes + o2) = make_uint4(al[j0], al[j0 + 1], al[j0 + 2], al[j0 + 3]);
                    *reinterpret_cast<uint4 *>(stg + 2 * op_bytes + o2) = make_uint4(bh[j0], bh[j0 + 1], bh[j0 + 2], bh[j0 + 3]);
                    *reinterpret_cast<uint4 *>(stg + 3 * op_bytes + o2) = make_uint4(bl[j0], bl[j0 + 1], bl[j0 + 2], bl[j0 + 3]);
                }
            } else {
                uint32_t bh[4], bl[4], ah[4], al[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    split_bf16x2(xv[it][2 * j], xv[it][2 * j + 1], bh[j], bl[j]);
                    split_bf16x2(wv[2 * j], wv[2 * j + 1], ah[j], al[j]);
                }
                *reinterpret_cast<uint4 *>(stg + off) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
                *reinterpret_cast<uint4 *>(stg + op_bytes + off) = make_uint4(al[0], al[1], al[2], al[3]);
                *reinterpret_cast<uint4 *>(stg + 2 * op_bytes + off) = make_uint4(bh[0], bh[1], bh[2], bh[3]);
                *reinterpret_cast<uint4 *>(stg + 3 * op_bytes + off) = make_uint4(bl[0], bl[1], bl[2], bl[3]);
            }
        }
        if (st + 1 < nst) load_stage(st + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(stg);
            for (int q = 0; q < G.n_units; ++q) {
                const TcUnit u = p.plan.u[G.unit0 + q];
                const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, kRowTile, u.n);
                const uint32_t d = tmem + (uint32_t)u.tmem_col;
                const uint32_t aoff = (uint32_t)(u.a_row >> 3) * SBO, boff = (uint32_t)(u.b_row >> 3) * SBO;
#pragma unroll
                for (int ks = 0; ks < NKS; ++ks) {
                    const uint32_t kb = 256u * ks;
                    const uint64_t ahi = make_desc(base + aoff + kb, 128, SBO);
                    const uint64_t alo = make_desc(base + op_bytes + aoff + kb, 128, SBO);
                    const uint64_t bhi = make_desc(base + 2 * op_bytes + boff + kb, 128, SBO);
                    const uint64_t blo = make_desc(base + 3 * op_bytes + boff + kb, 128, SBO);
                    mma_issue<TF32>(d, ahi, bhi, idesc, (acc_on || ks > 0) ? 1u : 0u);
                    mma_issue<TF32>(d, ahi, blo, idesc, 1u);
                    mma_issue<TF32>(d, alo, bhi, idesc, 1u);
                }
            }
            mma_commit(&bars[s]);
        }
        used[s] = true;
        phase[s] ^= 1u;
        acc_on = true;
        since += KP;
        if (since >= FLUSH_P) {
            flush();
            since = 0;
            if (*s_abort) { ok = false; break; }
        }
    }
    if (ok && acc_on) flush();
    // test mode: after the last flush (both buffers' commits complete), buffer 0's
    // next phase, which no commit completes
    if (p.wait_unmet && tid == 0 && !*s_abort && !mbar_wait(&bars[0], phase[0], p.wait_limit)) *s_abort = 1;
    __syncthreads();
    if (*s_abort || !ok) {
        if (tid == 0) {
            atomicCAS(p.err, 0, DEV_ERR_TIMEOUT);
            // wait (bounded) for anything still in flight before releasing TMEM
            for (int s = 0; s < 2; ++s)
                if (used[s]) mbar_wait(&bars[s], phase[s] ^ 1u);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.tmem_alloc));
}

// G_m[i][j] = sum over slices of the unit entries that hold it.  With a slice
// range per catalogue (mslice [n_cat + 1], grid y = catalogue), catalogue c sums
// its own slices into G + c * gram_offset(nb, lmax, lmax + 1).
__global__ void k_gram_tc_reduce(const double *partial, int n_slices, long long slice_size, int nb, int lmax,
                                 TcPlan plan, double *G, const int *mslice = nullptr)
{
    const int64_t total = gram_offset(nb, lmax, lmax + 1);
    int s0 = 0, s1 = n_slices;
    if (mslice) {
        s0 = mslice[blockIdx.y];
        s1 = mslice[blockIdx.y + 1];
        G += (int64_t)blockIdx.y * total;
    }
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int m = 0;
        while (m < lmax && idx >= gram_offset(nb, lmax, m + 1)) ++m;
        const int n_m = nb * (lmax - m + 1);
        const int64_t r = idx - gram_offset(nb, lmax, m);
        const int i = (int)(r / n_m), j = (int)(r % n_m);
        const TcMap mp = plan.map[m];
        int unit = mp.unit_lo, ri = mp.off + i;
        const int cj = mp.off + j;
        if (mp.unit_hi >= 0 && i >= 128) {
            unit = mp.unit_hi;
            ri = i - 128;
        }
        const TcUnit u = plan.u[unit];
        const int64_t src = u.part_off + (int64_t)ri * u.n + cj;
        double s = 0.0;
        for (int sl = s0; sl < s1; ++sl) s += partial[sl * slice_size + src];
        G[idx] = s;
    }
}

// ---------------------------------------------------------------------------
// The plain FP32 Gram on the same tile plan: one CTA per (unit, column half,
// slice of primaries) computes its 128 x (up to 128) block of D with FP32 FMAs,
// 8 x 8 outputs per thread; the staged operands are FP32 (A = w x, B = x),
// [K entry][row]; FP32 runs of 256 primaries are added to FP64 partial sums.
constexpr int kSimtKP = 16;          // primaries per stage (32 K entries)
constexpr int kSimtFlush = 256;      // primaries per FP32 accumulation run

__global__ void __launch_bounds__(256, 2) k_gram_simt(const TcParams p)
{
    __shared__ __align__(16) float sA[2 * kSimtKP][128];
    __shared__ __align__(16) float sB[2 * kSimtKP][128];
    __shared__ int4 rowinfoA[128], rowinfoB[128];
    // work item -> (unit, column half)
    int item = blockIdx.x, unit = 0, half = 0;
    for (unit = 0; unit < p.plan.n_units; ++unit) {
        const int halves = (p.plan.u[unit].n + 127) / 128;
        if (item < halves) { half = item; break; }
        item -= halves;
    }
    if (unit >= p.plan.n_units) return;
    const TcUnit U = p.plan.u[unit];
    int grp = 0;
    while (grp + 1 < p.plan.n_groups && p.plan.g[grp + 1].unit0 <= unit) ++grp;
    const TcGroup G = p.plan.g[grp];
    const int ncols = min(128, U.n - 128 * half);
    const int brow0 = U.b_row + 128 * half;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int nb = p.nb, nlm = (p.lmax + 1) * (p.lmax + 1);
    const int64_t RL = (int64_t)nb * nlm;
    // row tables of the 128 A rows and the ncols B rows (staged-row numbering of the group)
    for (int r = tid; r < 256; r += blockDim.x) {
        const int row = r < 128 ? U.a_row + r : brow0 + (r - 128);
        int4 ri = make_int4(0, -1, 0, 0);
        if (r < 128 || r - 128 < ncols)
            for (int q = 0; q < G.n_segs; ++q) {
                const TcSeg sg = p.plan.s[G.seg0 + q];
                if (row >= sg.row && row < sg.row + sg.rows) {
                    const int within = row - sg.row, l = sg.m + within / nb;
                    ri = make_int4(l * l + (sg.m ? 2 * sg.m - 1 : 0), sg.m ? l * l + 2 * sg.m : -1, within % nb, 1);
                }
            }
        if (r < 128) rowinfoA[r] = ri;
        else rowinfoB[r - 128] = ri;
    }
    const int64_t i_beg = p.slice_k ? p.slice_k[blockIdx.y] : (int64_t)blockIdx.y * p.per_slice;
    const int64_t i_end = p.slice_k ? p.slice_k[blockIdx.y + 1] : min(p.K, i_beg + p.per_slice);
    double *part = p.partial + (int64_t)blockIdx.y * p.plan.slice_size + U.part_off;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    auto flush = [&]() {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int r = ty * 8 + a;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int c = tx * 8 + b;
                if (c < ncols) part[(int64_t)r * U.n + 128 * half + c] += (double)acc[a][b];
                acc[a][b] = 0.f;
            }
        }
    };
    int since = 0;
    __syncthreads();
    for (int64_t i0 = i_beg; i0 < i_end; i0 += kSimtKP) {
        __syncthreads();
        // stage: entry k = 2 p + part of primary i0 + p, rows of A (w-scaled) and B
        for (int e = tid; e < 2 * 128 * kSimtKP; e += blockDim.x) {
            const int which = e / (128 * kSimtKP);            // 0: A rows, 1: B rows
            const int rem = e % (128 * kSimtKP);
            const int pp = rem / 128, r = rem % 128;
            const int64_t i = i0 + pp;
            const int4 ri = which ? rowinfoB[r] : rowinfoA[r];
            float xc = 0.f, xs = 0.f;
            if (ri.w && i < i_end) {
                const float *src = p.alm + i * RL + ri.z * nlm;
                xc = __ldg(src + ri.x);
                xs = ri.y >= 0 ? __ldg(src + ri.y) : 0.f;
                if (!which && p.w) {
                    const float wi = __ldg(p.w + i);
                    xc *= wi;
                    xs *= wi;
                }
            }
            float (*dst)[128] = which ? sB : sA;
            dst[2 * pp][r] = xc;
            dst[2 * pp + 1][r] = xs;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < 2 * kSimtKP; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&sA[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sA[k][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&sB[k][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&sB[k][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        since += kSimtKP;
        if (since >= kSimtFlush) {
            flush();
            since = 0;
        }
    }
    if (since > 0) flush();
}

// The tensor-core Gram's shared-memory limit, set once per device (before any
// stream capture: the first call runs eagerly).
cudaError_t tc_smem_attr(bool tf32)
{
    static std::atomic<unsigned long long> attr_done[2];   // devices whose attribute is set
    const unsigned long long bit = device_bit();
    if (!(attr_done[tf32].load(std::memory_order_acquire) & bit)) {
        const cudaError_t e = cudaFuncSetAttribute(tf32 ? k_gram_tc<true> : k_gram_tc<false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr_done[tf32].fetch_or(bit, std::memory_order_acq_rel);
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t couple_gram_tc(const float *alm, const float *w, int64_t K, int nb, int lmax, bool tf32, double *G,
                           int *err, int sms, cudaStream_t st)
{
    TcParams p;
    if (!make_tc_plan(nb, lmax, p.plan)) return cudaErrorInvalidValue;
    if (K <= 0) return cudaMemsetAsync(G, 0, gram_offset(nb, lmax, lmax + 1) * sizeof(double), st);
    const int ng = p.plan.n_groups;
    int slices = sms / ng;
    if (slices < 1) slices = 1;
    const int64_t min_per = 1024;
    if ((K + slices - 1) / slices < min_per) slices = (int)((K + min_per - 1) / min_per);
    if (slices < 1) slices = 1;
    p.alm = alm;
    p.w = w;
    p.K = K;
    p.nb = nb;
    p.lmax = lmax;
    p.per_slice = (K + slices - 1) / slices;
    p.n_slices = slices;
    p.slice_k = nullptr;
    p.err = err;
    p.wait_limit = device_wait_limit();
    p.wait_unmet = device_wait_unmet();
    int rmax = 0;
    for (int g = 0; g < ng; ++g) rmax = std::max(rmax, p.plan.g[g].rows_alloc);
    const int ks = tf32 ? 16 : 32, esz = tf32 ? 4 : 2;
    // two stages of four operands, the row table, barriers; at least 116 KB so that
    // one CTA owns an SM and tensor-memory allocations never wait
    size_t smem = 2 * 4 * (size_t)rmax * ks * esz + 16 * (size_t)rmax + 64;
    if (smem < 116 * 1024) smem = 116 * 1024;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = tc_smem_attr(tf32);
    if (e != cudaSuccess) return e;
    const size_t pbytes = (size_t)slices * p.plan.slice_size * sizeof(double);
    e = scratch_malloc((void **)&p.partial, pbytes, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.partial, 0, pbytes, st);
    if (e == cudaSuccess) {
        const dim3 grid(ng, slices);
        if (tf32) k_gram_tc<true><<<grid, kThreads, smem, st>>>(p);
        else k_gram_tc<false><<<grid, kThreads, smem, st>>>(p);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t tot = gram_offset(nb, lmax, lmax + 1);
        int g = (int)((tot + 255) / 256);
        if (g > 4096) g = 4096;
        k_gram_tc_reduce<<<g, 256, 0, st>>>(p.partial, slices, p.plan.slice_size, nb, lmax, p.plan, G);
        note_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(p.partial, st);
    return e;
}

cudaError_t couple_gram_simt(const float *alm, const float *w, int64_t K, int nb, int lmax, double *G, int sms,
                             cudaStream_t st)
{
    TcParams p;
    if (!make_tc_plan(nb, lmax, p.plan)) return cudaErrorInvalidValue;
    if (K <= 0) return cudaMemsetAsync(G, 0, gram_offset(nb, lmax, lmax + 1) * sizeof(double), st);
    int items = 0;
    for (int u = 0; u < p.plan.n_units; ++u) items += (p.plan.u[u].n + 127) / 128;
    int slices = (2 * sms + items - 1) / items;
    const int64_t min_per = 2048;
    if ((K + slices - 1) / slices < min_per) slices = (int)((K + min_per - 1) / min_per);
    if (slices < 1) slices = 1;
    p.alm = alm;
    p.w = w;
    p.K = K;
    p.nb = nb;
    p.lmax = lmax;
    p.per_slice = (K + slices - 1) / slices;
    p.n_slices = slices;
    p.slice_k = nullptr;
    p.err = nullptr;
    p.wait_limit = device_wait_limit();
    p.wait_unmet = 0;
    const size_t pbytes = (size_t)slices * p.plan.slice_size * sizeof(double);
    cudaError_t e = scratch_malloc((void **)&p.partial, pbytes, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.partial, 0, pbytes, st);
    if (e == cudaSuccess) {
        k_gram_simt<<<dim3(items, slices), 256, 0, st>>>(p);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t tot = gram_offset(nb, lmax, lmax + 1);
        int g = (int)((tot + 255) / 256);
        if (g > 4096) g = 4096;
        k_gram_tc_reduce<<<g, 256, 0, st>>>(p.partial, slices, p.plan.slice_size, nb, lmax, p.plan, G);
        note_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(p.partial, st);
    return e;
}

namespace {

// Work items of the FP32 Gram: 128-row tiles of every unit.
int simt_items(const TcPlan &plan)
{
    int items = 0;
    for (int u = 0; u < plan.n_units; ++u) items += (plan.u[u].n + 127) / 128;
    return items;
}

}  // namespace

void gram_batch_slices(const int64_t *off, int n_cat, int nb, int lmax, bool simt, int sms,
                       std::vector<int64_t> &slice_k, std::vector<int> &mslice)
{
    slice_k.clear();
    mslice.clear();
    TcPlan plan;
    if (!make_tc_plan(nb, lmax, plan)) return;
    // about one launch wave over the whole group (two FP32 CTAs per SM, one
    // tensor-core CTA), slices of 1024 (tensor) / 2048 (FP32) to 65536 primaries
    const int per_wave = simt ? std::max(1, 2 * sms / std::max(1, simt_items(plan)))
                              : std::max(1, sms / std::max(1, plan.n_groups));
    const int64_t K = off[n_cat] - off[0];
    int64_t per = (K + per_wave - 1) / per_wave;
    per = std::max<int64_t>(per, simt ? 2048 : 1024);
    per = std::min<int64_t>(per, 65536);
    slice_k.push_back(0);
    for (int c = 0; c < n_cat; ++c) {
        mslice.push_back((int)slice_k.size() - 1);
        const int64_t a = off[c] - off[0], b = off[c + 1] - off[0];
        const int64_t ns = (b - a + per - 1) / per;
        for (int64_t q = 1; q <= ns; ++q) slice_k.push_back(a + ((b - a) * q) / ns);
    }
    mslice.push_back((int)slice_k.size() - 1);
}

cudaError_t couple_gram_batched(const float *alm, const float *w, int n_cat, const int64_t *d_slice_k,
                                int n_slices, const int *d_mslice, int nb, int lmax, int precision, double *G,
                                int *err, int sms, cudaStream_t st)
{
    TcParams p;
    if (!make_tc_plan(nb, lmax, p.plan)) return cudaErrorInvalidValue;
    const int64_t gsz = gram_offset(nb, lmax, lmax + 1);
    if (n_slices < 1) return cudaMemsetAsync(G, 0, (size_t)n_cat * gsz * sizeof(double), st);
    const bool simt = precision == TPCF_PREC_FP32, tf32 = precision == TPCF_PREC_TF32X3;
    p.alm = alm;
    p.w = w;
    p.K = 0;
    p.nb = nb;
    p.lmax = lmax;
    p.per_slice = 0;
    p.n_slices = n_slices;
    p.slice_k = d_slice_k;
    p.err = simt ? nullptr : err;
    p.wait_limit = device_wait_limit();
    p.wait_unmet = simt ? 0 : device_wait_unmet();
    size_t smem = 0;
    cudaError_t e = cudaSuccess;
    if (!simt) {
        int rmax = 0;
        for (int g = 0; g < p.plan.n_groups; ++g) rmax = std::max(rmax, p.plan.g[g].rows_alloc);
        const int ks = tf32 ? 16 : 32, esz = tf32 ? 4 : 2;
        smem = 2 * 4 * (size_t)rmax * ks * esz + 16 * (size_t)rmax + 64;
        if (smem < 116 * 1024) smem = 116 * 1024;
        if (smem > 227 * 1024) return cudaErrorInvalidValue;
        e = tc_smem_attr(tf32);
        if (e != cudaSuccess) return e;
    }
    const size_t pbytes = (size_t)n_slices * p.plan.slice_size * sizeof(double);
    e = scratch_malloc((void **)&p.partial, pbytes, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.partial, 0, pbytes, st);
    if (e == cudaSuccess) {
        if (simt) {
            k_gram_simt<<<dim3(simt_items(p.plan), n_slices), 256, 0, st>>>(p);
        } else {
            const dim3 grid(p.plan.n_groups, n_slices);
            if (tf32) k_gram_tc<true><<<grid, kThreads, smem, st>>>(p);
            else k_gram_tc<false><<<grid, kThreads, smem, st>>>(p);
        }
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        int g = (int)((gsz + 255) / 256);
        if (g > 4096) g = 4096;
        k_gram_tc_reduce<<<dim3(g, n_cat), 256, 0, st>>>(p.partial, n_slices, p.plan.slice_size, nb, lmax, p.plan, G,
                                                         d_mslice);
        note_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(p.partial, st);
    return e;
}

}  // namespace tpcf
