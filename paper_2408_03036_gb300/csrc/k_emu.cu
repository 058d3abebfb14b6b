// MLP emulator of the tree-level 3PCF multipoles: forward, backward and Adam
// kernels behind the tpcf_emu_* C ABI (include/tpcf_emu.h).
//
// Every product of the network runs on the 5th-generation tensor cores through
// one persistent, warp-specialised GEMM kernel (k_gemm): bf16 operands brought
// in by TMA (128-byte swizzle, K-major or MN-major), FP32 accumulation in tensor
// memory, and an epilogue per use that reads the accumulator back and fuses the
// elementwise work: bias and SiLU in the forward pass, the output scaling in
// inference, the loss, its gradient and the output bias gradient in training,
// SiLU'(z) and the bias gradient of every hidden layer in the backward product
// dA_prev = dZ W, and split-K partials for the weight gradients dW = A_prev^T dZ.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <atomic>

#include <cuda.h>   // CUtensorMap and the tensor-map encoder's types (the encoder is resolved at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_common.cuh"
#include "../../include/tpcf_emu.h"

namespace {

constexpr int kMaxLayers = 8;
constexpr int kMaxWidth = 4096;
constexpr int64_t kMaxChunk = 32768;  // most rows per internal pass (per-chunk buffer capacity)

struct Layer {
    int in, out;
    int ldi, ldo;                     // in and out rounded up to 8 (16-byte bf16 rows)
    int64_t w_off, b_off;             // offsets in the parameter vector
};

inline int round8(int n) { return (n + 7) / 8 * 8; }

// SiLU with an IEEE division (its result is rounded to bf16: a less accurate value
// flips that rounding more often); its derivative with the fast division (it scales
// a bf16-rounded gradient); z -> -inf gives 0 for both
__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = __fdividef(1.f, 1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Epilogues of the GEMM kernel (C = A B^T over one 128 x NT tile, FP32 in tensor memory):
//   EPI_HID   forward hidden layer: z = c + bias; pre-activation z (FP32, training
//             only) and the activation SiLU(z) (bf16, the next product's operand)
//   EPI_PRED  forward output layer, inference: y = (c + bias) sd + mean (FP32)
//   EPI_LOSS  forward output layer, training: d = c + bias - (y - mean) / sd against
//             the targets y; the gradient g = gscale d (bf16), its column sums into
//             the bias gradient, and sum d^2 / count into the loss
//   EPI_BWD   backward product dA_prev = dZ W: g = c SiLU'(z) with the previous
//             layer's pre-activation z (bf16), its column sums into that layer's
//             bias gradient
//   EPI_PART  weight gradient, split over K: the split's FP32 partial tile
enum { EPI_HID = 0, EPI_PRED = 1, EPI_LOSS = 2, EPI_BWD = 3, EPI_PART = 4 };

struct GemmArgs {
    int M, N, K;
    int a_mn, b_mn;          // 1: operand stored MN-major (contiguous along M or N)
    int NT;                  // tile columns: 64, 128 or 256
    int n_mt, n_nt, nkb;     // tiles along M and N, 64-wide K blocks
    int kper;                // K blocks per split
    int units;               // splits x n_mt x n_nt work units
    int stages;              // stages of the load ring (at most kMaxStages)
    int ncol;                // floats of each per-column parameter array in shared memory (0: none)
    const float *bias;       // [N]
    __nv_bfloat16 *out_b;    // bf16 rows, pitch ld_b (HID activation; LOSS, BWD gradient)
    int64_t ld_b;
    float *out_f;            // FP32 rows, pitch ld_f (HID pre-activation or null; PRED y; PART workspace)
    int64_t ld_f;
    int pair_f;              // out_f rows take 8-byte pair stores (even ld_f, 8-byte aligned)
    const float *in_f;       // FP32 rows read by the epilogue, pitch ld_in (LOSS targets; BWD pre-activation)
    int64_t ld_in;
    int pair_in;             // in_f rows take 8-byte pair loads
    const float *mean, *sd;  // output scaling [N]
    float gscale;            // LOSS: 2 / (rows x outputs of the whole batch)
    float inv_count;         // LOSS: 1 / (rows x outputs of the whole batch)
    double *loss;            // LOSS: += sum d^2 inv_count
    float *colsum;           // LOSS, BWD: += column sums of the gradient
    int64_t part_stride;     // PART: floats between the splits' partial outputs
    int *err;
    long long wait_limit;    // bound of a wait: wait_limit / 16 suspending polls (at least one)
    int wait_unmet;          // test mode: one more wait on a phase that nothing completes
};

constexpr int kGemmThreads = 320;       // warp 0 loads (TMA), warp 1 issues MMAs, warps 2-9 epilogue
constexpr int kEpiWarps = 8;
constexpr int kBM = 128;                // tile rows (tensor-memory lanes, the MMA's M)
constexpr int kBK = 64;                 // K per stage: one 128-byte swizzle row of bf16
constexpr int kMaxStages = 4;
constexpr uint32_t kATile = kBM * kBK * 2;
constexpr uint32_t kMNBox = 64 * kBK * 2;   // one 64 (MN) x 64 (K) box of an MN-major operand

// The epilogue works on 16-column chunks of the warp's 32 rows in a column-pair
// layout: the accumulator (one row per lane, as tensor memory hands it out) goes
// through a per-warp [32][kStg] staging area in shared memory, after which lane l
// holds columns 2 (l % 8) and 2 (l % 8) + 1 of rows 4 it + l / 8 (it = 0..7), as
// t[2 it] and t[2 it + 1].  Per-column values (bias, output scaling) are then two
// registers per lane, column sums are sums over `it` plus two shuffles, and global
// loads and stores are pairs running along rows: each instruction covers 16
// consecutive columns of four rows.
constexpr int kStg = 20;                                   // row pitch (floats): 16-byte rows
constexpr uint32_t kStgBytes = kEpiWarps * 32 * kStg * 4;

// the accumulator row r (this lane's, 16 raw 32-bit values) to the pair layout t
__device__ __forceinline__ void to_pairs(float *stg, const uint32_t (&r)[16], float (&t)[16], int lane)
{
    float4 *row = reinterpret_cast<float4 *>(stg + lane * kStg);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        row[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                             __uint_as_float(r[4 * q + 3]));
    __syncwarp();
    const int p = lane & 7, g4 = lane >> 3;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const float2 v = *reinterpret_cast<const float2 *>(stg + (4 * it + g4) * kStg + 2 * p);
        t[2 * it] = v.x;
        t[2 * it + 1] = v.y;
    }
    __syncwarp();
}

// Per-column parameters, two arrays in shared memory filled once per CTA (colA, colB):
//   HID   z = c + colB                       (colB = bias)
//   PRED  y = c colA + colB                  (colA = sd, colB = bias sd + mean)
//   LOSS  d = c + colB - y colA              (colA = 1 / sd, colB = bias + mean / sd)
template <int EPI>
__device__ __forceinline__ void col_params(const GemmArgs &g, int n, float &a, float &b)
{
    const float bias = g.bias ? g.bias[n] : 0.f;
    a = 1.f;
    b = bias;
    if (EPI == EPI_PRED) {
        a = g.sd[n];
        b = fmaf(bias, a, g.mean[n]);
    } else if (EPI == EPI_LOSS) {
        a = 1.f / g.sd[n];
        b = fmaf(g.mean[n], a, bias);
    }
}

// Per-chunk row inputs (LOSS targets, BWD pre-activations) in the pair layout, loaded
// one chunk ahead.
struct ChunkIn {
    float x[16];
};

template <int EPI>
__device__ __forceinline__ void chunk_load(const GemmArgs &g, int row_base, int n0, int lane, ChunkIn &in)
{
    if (EPI != EPI_LOSS && EPI != EPI_BWD) return;
    const int nval = min(16, g.N - n0);
    const int p = lane & 7, g4 = lane >> 3;
    const int c = 2 * p;
    const bool c0v = c < nval, c1v = c + 1 < nval;
    const float *base = g.in_f + (int64_t)(row_base + g4) * g.ld_in + n0 + c;
    const bool full = nval == 16 && row_base + 32 <= g.M && g.pair_in;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const float *a = base + (int64_t)(4 * it) * g.ld_in;
        const bool rv = row_base + 4 * it + g4 < g.M;
        if (full || (rv && c1v && g.pair_in)) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(a));
            in.x[2 * it] = v.x;
            in.x[2 * it + 1] = v.y;
        } else {
            in.x[2 * it] = (rv && c0v) ? __ldg(a) : 0.f;
            in.x[2 * it + 1] = (rv && c1v) ? __ldg(a + 1) : 0.f;
        }
    }
}

// stores of one row pair (FP32 or bf16), paired when both columns are valid and aligned
__device__ __forceinline__ void st_pair(float *a, float v0, float v1, bool c0v, bool c1v, bool pair)
{
    if (c1v && pair) {
        *reinterpret_cast<float2 *>(a) = make_float2(v0, v1);
    } else {
        if (c0v) a[0] = v0;
        if (c1v) a[1] = v1;
    }
}

__device__ __forceinline__ void st_pair(__nv_bfloat16 *a, float v0, float v1, bool c0v, bool c1v)
{
    if (c1v) {
        *reinterpret_cast<__nv_bfloat162 *>(a) = __floats2bfloat162_rn(v0, v1);
    } else if (c0v) {
        a[0] = __float2bfloat16_rn(v0);
    }
}

// One 16-column chunk of the epilogue; r holds this lane's accumulator row (row_base + lane).
// FULL: all 32 rows and 16 columns lie inside the output and FP32 rows take pair
// stores, so the chunk runs without predicates.
template <int EPI, bool FULL>
__device__ __forceinline__ void epi_chunk(const GemmArgs &g, int row_base, int n0, int split, const uint32_t (&r)[16],
                                          const ChunkIn &in, const float *colA, const float *colB, float *stg,
                                          float &lsum, int lane)
{
    const int nval = min(16, g.N - n0);
    const int p = lane & 7, g4 = lane >> 3;
    const int c = 2 * p;
    float2 pa = make_float2(1.f, 1.f), pb = make_float2(0.f, 0.f);
    if (EPI == EPI_HID || EPI == EPI_PRED || EPI == EPI_LOSS) {
        pa = *reinterpret_cast<const float2 *>(colA + n0 + c);
        pb = *reinterpret_cast<const float2 *>(colB + n0 + c);
    }
    const bool c0v = FULL || c < nval, c1v = FULL || c + 1 < nval;
    auto rowv = [&](int it) { return FULL || row_base + 4 * it + g4 < g.M; };
    float t[16];
    to_pairs(stg, r, t, lane);
    if (EPI == EPI_PART) {
        float *a = g.out_f + split * g.part_stride + (int64_t)(row_base + g4) * g.ld_f + n0 + c;
#pragma unroll
        for (int it = 0; it < 8; ++it)
            if (rowv(it)) st_pair(a + (int64_t)(4 * it) * g.ld_f, t[2 * it], t[2 * it + 1], c0v, c1v, true);
        return;
    }
    if (EPI == EPI_HID) {
        float *az = g.out_f ? g.out_f + (int64_t)(row_base + g4) * g.ld_f + n0 + c : nullptr;
        __nv_bfloat16 *aa = g.out_b + (int64_t)(row_base + g4) * g.ld_b + n0 + c;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            if (rowv(it)) {
                const float z0 = t[2 * it] + pb.x, z1 = t[2 * it + 1] + pb.y;
                if (az) st_pair(az + (int64_t)(4 * it) * g.ld_f, z0, z1, c0v, c1v, true);
                st_pair(aa + (int64_t)(4 * it) * g.ld_b, silu(z0), silu(z1), c0v, c1v);
            }
        }
        return;
    }
    if (EPI == EPI_PRED) {
        float *a = g.out_f + (int64_t)(row_base + g4) * g.ld_f + n0 + c;
#pragma unroll
        for (int it = 0; it < 8; ++it)
            if (rowv(it))
                st_pair(a + (int64_t)(4 * it) * g.ld_f, fmaf(t[2 * it], pa.x, pb.x), fmaf(t[2 * it + 1], pa.y, pb.y),
                        c0v, c1v, FULL || g.pair_f);
        return;
    }
    // LOSS, BWD: the gradient (zero outside the M x N output), stored as bf16, and its
    // column sums into the bias gradient
    __nv_bfloat16 *ag = g.out_b + (int64_t)(row_base + g4) * g.ld_b + n0 + c;
    float cs0 = 0.f, cs1 = 0.f;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const bool rv = rowv(it);
        float g0, g1;
        if (EPI == EPI_LOSS) {
            const float d0 = (rv && c0v) ? fmaf(-in.x[2 * it], pa.x, t[2 * it] + pb.x) : 0.f;
            const float d1 = (rv && c1v) ? fmaf(-in.x[2 * it + 1], pa.y, t[2 * it + 1] + pb.y) : 0.f;
            lsum = fmaf(d0, d0, fmaf(d1, d1, lsum));
            g0 = g.gscale * d0;
            g1 = g.gscale * d1;
        } else {
            g0 = (rv && c0v) ? t[2 * it] * silu_grad(in.x[2 * it]) : 0.f;
            g1 = (rv && c1v) ? t[2 * it + 1] * silu_grad(in.x[2 * it + 1]) : 0.f;
        }
        if (rv) st_pair(ag + (int64_t)(4 * it) * g.ld_b, g0, g1, c0v, c1v);
        cs0 += g0;
        cs1 += g1;
    }
    cs0 += __shfl_xor_sync(0xffffffffu, cs0, 8);
    cs1 += __shfl_xor_sync(0xffffffffu, cs1, 8);
    cs0 += __shfl_xor_sync(0xffffffffu, cs0, 16);
    cs1 += __shfl_xor_sync(0xffffffffu, cs1, 16);
    if (g4 == 0) {
        if (c0v) atomicAdd(g.colsum + n0 + c, cs0);
        if (c1v) atomicAdd(g.colsum + n0 + c + 1, cs1);
    }
}

// Persistent, warp-specialised tcgen05 GEMM: C[m][n] = sum_k A(m, k) B(n, k) in
// 128 x NT tiles (work units: K splits x row tiles x column tiles, taken by the
// CTAs in turn).  Warp 0 (one thread) loads 64-wide K blocks of A and B with TMA
// into a ring of g.stages 128-byte-swizzled stages (K-major operands: one box of
// 64 K x rows; MN-major operands: boxes of 64 MN x 64 K), completing each
// stage's `full` barrier; warp 1 (one thread) issues four K = 16 MMAs per stage
// into one of two tensor-memory accumulators and commits them to the stage's
// `empty` barrier and, after a unit's last stage, to the accumulator's `tfull`
// barrier; warps 2-5 read the accumulator (one 32-lane quarter each), run the
// epilogue and release it through `tempty`, so the epilogue of one unit overlaps
// the products of the next.  The waiting threads suspend in mbarrier.try_wait
// rather than spin, so they take no issue slots from the epilogue warps.  Every
// wait is bounded (wait_limit / 16 polls of up to a microsecond): a role that gives up raises
// the CTA's abort flag, the others stop, the loads and products in flight are
// waited for (long bound) before the tensor memory is released, and the kernel
// latches DEV_ERR_TIMEOUT.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b, const GemmArgs g)
{
    using namespace tpcf::tc;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);   // swizzled tiles: 1024-byte aligned
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NT = g.NT;
    const uint32_t stage_bytes = kATile + (uint32_t)NT * kBK * 2;
    const int S = g.stages;
    float *colA = reinterpret_cast<float *>(smem + S * stage_bytes + kStgBytes);   // per-column parameters
    float *colB = colA + g.ncol;
    uint64_t *full = reinterpret_cast<uint64_t *>(colB + g.ncol);
    uint64_t *empty = full + kMaxStages;
    uint64_t *tfull = empty + kMaxStages;
    uint64_t *tempty = tfull + 2;
    uint64_t *done = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *s_abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t tmem_cols = 2u * (uint32_t)NT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kEpiWarps);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int per_split = g.n_mt * g.n_nt;
    // polls of a suspending wait (up to a microsecond each)
    const long long polls = g.wait_limit > 16 ? g.wait_limit >> 4 : 1;

    if (warp == 0 && lane == 0) {
        // ---- loads
        uint32_t it = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
            const int sp = u / per_split, r = u % per_split, mt = r / g.n_nt, nt = r % g.n_nt;
            const int kb0 = sp * g.kper, kb1 = min(g.nkb, kb0 + g.kper);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = (int)(it % (uint32_t)S);
                const uint32_t ph = (it / (uint32_t)S) & 1u;
                if (!mbar_sleep_wait_or_abort(&empty[s], ph ^ 1u, polls, s_abort)) {
                    *s_abort = 1;
                    ok = false;
                    break;
                }
                unsigned char *sa = smem + s * stage_bytes, *sb = sa + kATile;
                mbar_expect_tx(&full[s], stage_bytes);
                const int k0 = kb * kBK;
                if (!g.a_mn) {
                    tma_load_2d(sa, &tma_a, k0, mt * kBM, &full[s]);
                } else {
                    tma_load_2d(sa, &tma_a, mt * kBM, k0, &full[s]);
                    tma_load_2d(sa + kMNBox, &tma_a, mt * kBM + 64, k0, &full[s]);
                }
                if (!g.b_mn) {
                    tma_load_2d(sb, &tma_b, k0, nt * NT, &full[s]);
                } else {
                    for (int h = 0; h < NT / 64; ++h) tma_load_2d(sb + h * kMNBox, &tma_b, nt * NT + 64 * h, k0, &full[s]);
                }
            }
        }
        if (!ok) {
            // the loads issued must land before the CTA's shared memory goes away
            for (int s = 0; s < S; ++s)
                if (it > (uint32_t)s) {
                    const uint32_t j = ((it - 1u - (uint32_t)s) / (uint32_t)S) * (uint32_t)S + (uint32_t)s;
                    mbar_wait(&full[s], (j / (uint32_t)S) & 1u);
                }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- products
        uint32_t it = 0, tc = 0;
        bool ok = true, any = false;
        const uint32_t idesc = make_idesc_major(1u, kBM, NT, g.a_mn, g.b_mn);
        for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
            const int sp = u / per_split;
            const int kb0 = sp * g.kper, kb1 = min(g.nkb, kb0 + g.kper);
            const uint32_t acc = tc & 1u, aph = (tc >> 1) & 1u;
            if (!mbar_sleep_wait_or_abort(&tempty[acc], aph ^ 1u, polls, s_abort)) {
                *s_abort = 1;
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d_tmem = tmem + acc * (uint32_t)NT;
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = (int)(it % (uint32_t)S);
                const uint32_t ph = (it / (uint32_t)S) & 1u;
                if (!mbar_sleep_wait_or_abort(&full[s], ph, polls, s_abort)) {
                    *s_abort = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_u32(smem + s * stage_bytes), sb = sa + kATile;
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k) {
                    const uint64_t da = g.a_mn ? make_desc_sw128(sa + 2048u * k, kMNBox, 1024)
                                               : make_desc_sw128(sa + 32u * k, 16, 1024);
                    const uint64_t db = g.b_mn ? make_desc_sw128(sb + 2048u * k, kMNBox, 1024)
                                               : make_desc_sw128(sb + 32u * k, 16, 1024);
                    mma_issue<false>(d_tmem, da, db, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
                any = true;
            }
            if (!ok) break;
            mma_commit(&tfull[acc]);
            ++tc;
        }
        // every product issued completes before the accumulators are released
        if (any) {
            mma_commit(done);
            mbar_wait(done, 0u);
        }
        // test mode: a phase of `done` that no commit completes
        if (g.wait_unmet && ok && !mbar_wait(done, any ? 1u : 0u, g.wait_limit)) *s_abort = 1;
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31; the two
        // warps of a lane quarter take alternate 16-column chunks, each loading the
        // next chunk's inputs before it works on the current one
        const int q = warp & 3;
        const int c_first = 16 * ((warp - 2) >> 2);
        float *stg = reinterpret_cast<float *>(smem + S * stage_bytes) + (warp - 2) * 32 * kStg;
        // the per-column parameters of all N columns, once; every epilogue thread
        // reaches this barrier (named barrier 1, the 256 epilogue threads) exactly once
        if (g.ncol > 0) {
            for (int n = threadIdx.x - 64; n < g.ncol; n += 32 * kEpiWarps) {
                float a = 1.f, b = 0.f;
                if (n < g.N) col_params<EPI>(g, n, a, b);
                colA[n] = a;
                colB[n] = b;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
        }
        uint32_t tc = 0;
        float lsum = 0.f;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x) {
            const int sp = u / per_split, r = u % per_split, mt = r / g.n_nt, nt = r % g.n_nt;
            const uint32_t acc = tc & 1u, aph = (tc >> 1) & 1u;
            const int row_base = mt * kBM + 32 * q;
            ChunkIn cur, nxt;
            if (c_first < NT && nt * NT + c_first < g.N) chunk_load<EPI>(g, row_base, nt * NT + c_first, lane, cur);
            // one poller per warp: the warp's tensor-memory loads below are collective
            int okw = 1;
            if (lane == 0) okw = mbar_sleep_wait_or_abort(&tfull[acc], aph, polls, s_abort) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) {
                if (lane == 0) *s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // the next chunk's tensor-memory load is in flight while this one is worked on
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + acc * (uint32_t)NT;
            uint32_t ra[16], rb[16];
            if (c_first < NT && nt * NT + c_first < g.N) {
                tmem_ld16_issue(tbase + (uint32_t)c_first, ra);
                tmem_ld_wait();
                reg_fence16(ra);
            }
            // one chunk: the next chunk's inputs and tensor-memory load go out first; the
            // two register sets swap roles from one chunk to the next
            const bool pair_ok = EPI == EPI_PRED ? g.pair_f != 0 : true;
            auto step = [&](uint32_t(&rc)[16], uint32_t(&rn)[16], const ChunkIn &ic, ChunkIn &inx, int c0) -> bool {
                const int n0 = nt * NT + c0;
                const bool more = c0 + 32 < NT && n0 + 32 < g.N;
                if (more) {
                    chunk_load<EPI>(g, row_base, n0 + 32, lane, inx);
                    tmem_ld16_issue(tbase + (uint32_t)(c0 + 32), rn);
                }
                if (n0 + 16 <= g.N && row_base + 32 <= g.M && pair_ok)
                    epi_chunk<EPI, true>(g, row_base, n0, sp, rc, ic, colA, colB, stg, lsum, lane);
                else
                    epi_chunk<EPI, false>(g, row_base, n0, sp, rc, ic, colA, colB, stg, lsum, lane);
                if (more) {
                    tmem_ld_wait();
                    reg_fence16(rn);
                }
                return more;
            };
            if (c_first < NT && nt * NT + c_first < g.N) {
                for (int c0 = c_first;; c0 += 64) {
                    if (!step(ra, rb, cur, nxt, c0)) break;
                    if (!step(rb, ra, nxt, cur, c0 + 32)) break;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            ++tc;
        }
        if (EPI == EPI_LOSS) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if (lane == 0 && g.loss && lsum != 0.f) atomicAdd(g.loss, (double)lsum * (double)g.inv_count);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0 && *s_abort && g.err) atomicCAS(g.err, 0, tpcf::DEV_ERR_TIMEOUT);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// grads[i][o] += sum over splits of the partial weight gradients ws[split][i][ldw]
__global__ void k_reduce_parts(const float *__restrict__ ws, int splits, int64_t stride, int in, int out, int ldw,
                               float *__restrict__ grads)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)in * out;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / out), o = (int)(idx % out);
        float s = 0.f;
        for (int sp = 0; sp < splits; ++sp) s += ws[sp * stride + (int64_t)i * ldw + o];
        grads[idx] += s;
    }
}

// scaled inputs 2 (x - lo) / (hi - lo) - 1 as bf16 rows of stride ld (padding stays zero)
__global__ void k_scale_in(const float *__restrict__ x, int64_t n, int w, const float *__restrict__ lo,
                           const float *__restrict__ hi, __nv_bfloat16 *__restrict__ xs, int ld)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * w; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % w);
        const int64_t r = i / w;
        xs[r * ld + c] = __float2bfloat16_rn(2.f * (x[i] - lo[c]) / (hi[c] - lo[c]) - 1.f);
    }
}

// Per-column FP64 sums of y and y^2 over a block of rows: block (cx, ry) takes 32
// columns (one per lane, coalesced rows) and rows ry, ry + R, ..., spread over its
// eight warps and added in a fixed order (deterministic).
__global__ void k_col_partial(const float *__restrict__ y, int64_t n, int w, double2 *__restrict__ part)
{
    __shared__ double2 red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const int64_t R = gridDim.y;
    double s = 0.0, s2 = 0.0;
    if (c < w)
        for (int64_t r = blockIdx.y + R * warp; r < n; r += 8 * R) {
            const double v = y[r * w + c];
            s += v;
            s2 += v * v;
        }
    red[warp][lane] = make_double2(s, s2);
    __syncthreads();
    if (warp == 0 && c < w) {
        double2 t = red[0][lane];
        for (int q = 1; q < 8; ++q) {
            t.x += red[q][lane].x;
            t.y += red[q][lane].y;
        }
        part[(int64_t)blockIdx.y * w + c] = t;
    }
}

// per-column mean and standard deviation from the R row-block partial sums
__global__ void k_col_stats(const double2 *__restrict__ part, int R, int64_t n, int w, float *__restrict__ mean,
                            float *__restrict__ sd)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    double s = 0.0, s2 = 0.0;
    for (int r = 0; r < R; ++r) {
        const double2 t = part[(int64_t)r * w + c];
        s += t.x;
        s2 += t.y;
    }
    const double mu = n > 0 ? s / n : 0.0;
    const double var = n > 1 ? fmax(s2 / n - mu * mu, 0.0) : 0.0;
    mean[c] = (float)mu;
    sd[c] = (float)(var > 0.0 ? sqrt(var) : 1.0);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr_t, float b1, float b2, float eps_t)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] = p[i] - lr_t * mi / (sqrtf(vi) + eps_t);
    }
}

// bf16 copies of one layer's weights W[in][out] (FP32 master): wT[o][ldi] = W[i][o]
// (the forward product's operand, contiguous in i) and wP[i][ldo] = W[i][o] (the
// backward product's, contiguous in o); the padding columns stay zero
__global__ void k_wcopy(const float *__restrict__ W, int in, int out, __nv_bfloat16 *__restrict__ wT, int ldi,
                        __nv_bfloat16 *__restrict__ wP, int ldo)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)in * out;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / out), o = (int)(idx % out);
        const __nv_bfloat16 b = __float2bfloat16_rn(W[idx]);
        wT[(int64_t)o * ldi + i] = b;
        wP[(int64_t)i * ldo + o] = b;
    }
}

// Glorot-uniform weights from splitmix64(seed ^ index) (a counter-based hash), zero biases
__global__ void k_init(float *__restrict__ p, int64_t w_off, int64_t w_count, float a, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < w_count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(w_off + i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
        p[w_off + i] = (float)((2.0 * u - 1.0) * a);
    }
}

int grid1(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), (int64_t)tpcf::sm_count() * 8); }

}  // namespace

struct tpcf_emu_s {
    int nl = 0;
    int widths[kMaxLayers + 1] = {0};
    Layer layers[kMaxLayers];
    int64_t n_params = 0;
    int maxw8 = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *in_lo = nullptr, *in_hi = nullptr, *out_mean = nullptr, *out_sd = nullptr;
    // bf16 weight copies (rows padded to multiples of 8): the products' B operands
    __nv_bfloat16 *wT[kMaxLayers] = {nullptr};   // [out][ldi]: forward, contiguous in the input index
    __nv_bfloat16 *wP[kMaxLayers] = {nullptr};   // [in][ldo]: backward, contiguous in the output index
    float *ws = nullptr;                         // split-K partial weight gradients
    int64_t ws_floats = 0;
    // per-chunk buffers for `cap` rows (grown on demand up to kMaxChunk)
    int64_t cap = 0;
    __nv_bfloat16 *xs = nullptr;                 // scaled inputs [cap][ldi of layer 0]
    __nv_bfloat16 *act[kMaxLayers] = {nullptr};  // hidden activations [cap][ldo]
    float *Z[kMaxLayers] = {nullptr};            // hidden pre-activations [cap][ldo] (FP32)
    __nv_bfloat16 *gA = nullptr, *gB = nullptr;  // output-gradient ping-pong [cap][maxw8]
    int64_t step = 0;
};

namespace {

int emu_fail(int code, const char *msg) { return tpcf::set_error(code, msg); }
int emu_cuda(cudaError_t e)
{
    return tpcf::set_error(e == cudaErrorMemoryAllocation ? TPCF_ERR_OOM : TPCF_ERR_CUDA, cudaGetErrorString(e));
}
#define ECK(call)                                        \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return emu_cuda(e_);      \
    } while (0)

// cuTensorMapEncodeTiled, reached through the runtime's driver entry-point query
// (the library does not link the driver library itself)
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static std::once_flag once;
    static EncodeTiled f = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f = reinterpret_cast<EncodeTiled>(p);
    });
    return f;
}

// 2D bf16 tensor map: `inner` contiguous elements, `outer` rows `ld` elements apart
// (a multiple of 8), boxes of 64 x box_outer with the 128-byte swizzle; reads
// outside the extents return zeros
cudaError_t make_tmap(CUtensorMap *m, const void *base, int64_t inner, int64_t outer, int64_t ld, int box_outer)
{
    const EncodeTiled f = encoder();
    if (!f) return cudaErrorNotSupported;
    if (((uintptr_t)base & 15u) || (ld * 2) % 16 || inner < 1 || outer < 1) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_outer};
    const cuuint32_t es[2] = {1u, 1u};
    const CUresult r = f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// whether rows of ld floats starting at p take 8-byte pair accesses
int pairable(const void *p, int64_t ld) { return ((uintptr_t)p % 8 == 0 && ld % 2 == 0) ? 1 : 0; }

// A bf16 operand: element (mn, k) at p[mn + k ld] when MN-major, p[k + mn ld] when K-major
struct Operand {
    const __nv_bfloat16 *p;
    int64_t ld;
    int mn;
};

// C = A B^T through k_gemm<EPI>; g carries M, N, K and the epilogue's fields.  For
// EPI_PART the K range is split over up to max_splits partial outputs (g.out_f, rows
// g.ld_f apart, M rows per split) and the number of splits is returned in *splits.
template <int EPI>
cudaError_t gemm(GemmArgs g, Operand A, Operand B, cudaStream_t st, int max_splits = 1, int *splits = nullptr)
{
    if (splits) *splits = 0;
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    const int sms = tpcf::sm_count();
    auto tiles = [&](int nt) { return ((g.M + kBM - 1) / kBM) * ((g.N + nt - 1) / nt); };
    // tile width: 256 unless narrower tiles are needed to spread the units over the SMs
    int NT = 256;
    while (NT > 64 && (NT / 2 >= g.N || tiles(NT) < 2 * sms)) NT >>= 1;
    g.NT = NT;
    g.n_mt = (g.M + kBM - 1) / kBM;
    g.n_nt = (g.N + NT - 1) / NT;
    g.nkb = (g.K + kBK - 1) / kBK;
    int sp = 1;
    if (EPI == EPI_PART) {
        const int t = g.n_mt * g.n_nt;
        sp = std::max(1, std::min({(2 * sms + t - 1) / t, g.nkb / 4, max_splits}));
    }
    g.kper = (g.nkb + sp - 1) / sp;
    sp = (g.nkb + g.kper - 1) / g.kper;
    g.units = sp * g.n_mt * g.n_nt;
    if (EPI == EPI_PART) g.part_stride = (int64_t)g.M * g.ld_f;
    if (splits) *splits = sp;
    g.a_mn = A.mn;
    g.b_mn = B.mn;
    g.err = tpcf::device_error_flag();
    g.wait_limit = tpcf::device_wait_limit();
    g.wait_unmet = tpcf::device_wait_unmet();
    CUtensorMap ta, tb;
    cudaError_t e = A.mn ? make_tmap(&ta, A.p, g.M, g.K, A.ld, 64) : make_tmap(&ta, A.p, g.K, g.M, A.ld, kBM);
    if (e != cudaSuccess) return e;
    e = B.mn ? make_tmap(&tb, B.p, g.N, g.K, B.ld, 64) : make_tmap(&tb, B.p, g.K, g.N, B.ld, NT);
    if (e != cudaSuccess) return e;
    // per-column parameter arrays, then as many load stages as fit beside them
    g.ncol = (EPI == EPI_HID || EPI == EPI_PRED || EPI == EPI_LOSS) ? (g.N + 15) / 16 * 16 : 0;
    const size_t fixed = kStgBytes + 2 * (size_t)g.ncol * sizeof(float) + 256 + 1024;
    const size_t stage_bytes = kATile + (size_t)NT * kBK * 2;
    g.stages = kMaxStages;
    while (g.stages > 2 && fixed + g.stages * stage_bytes > 227 * 1024) --g.stages;
    const size_t smem = fixed + g.stages * stage_bytes;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const unsigned long long bit = tpcf::device_bit();
    if (!(attr_done.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr_done.fetch_or(bit, std::memory_order_acq_rel);
    }
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm<EPI>, kGemmThreads, smem);
    if (e != cudaSuccess) return e;
    // co-resident CTAs never ask for more than the SM's 512 tensor-memory columns
    per_sm = std::max(1, std::min(per_sm, 512 / (2 * NT)));
    const int grid = std::min(g.units, sms * per_sm);
    k_gemm<EPI><<<grid, kGemmThreads, smem, st>>>(ta, tb, g);
    tpcf::note_launch();
    return cudaGetLastError();
}

// bf16 weight copies of every layer from the FP32 master parameters
cudaError_t weight_copies(tpcf_emu e, cudaStream_t st)
{
    for (int l = 0; l < e->nl; ++l) {
        const Layer &L = e->layers[l];
        k_wcopy<<<grid1((int64_t)L.in * L.out), 256, 0, st>>>(e->params + L.w_off, L.in, L.out, e->wT[l], L.ldi,
                                                               e->wP[l], L.ldo);
        tpcf::note_launch();
    }
    return cudaGetLastError();
}

void free_chunk_buffers(tpcf_emu e)
{
    for (void *p : {(void *)e->xs, (void *)e->gA, (void *)e->gB})
        if (p) cudaFree(p);
    e->xs = nullptr;
    e->gA = e->gB = nullptr;
    for (int l = 0; l < kMaxLayers; ++l) {
        if (e->act[l]) cudaFree(e->act[l]);
        if (e->Z[l]) cudaFree(e->Z[l]);
        e->act[l] = nullptr;
        e->Z[l] = nullptr;
    }
    e->cap = 0;
}

// per-chunk buffers for at least `rows` rows (at most kMaxChunk); synchronises the
// stream when they grow
int ensure_cap(tpcf_emu e, int64_t rows, cudaStream_t st)
{
    rows = std::min<int64_t>(std::max<int64_t>(rows, 1), kMaxChunk);
    if (e->cap >= rows) return TPCF_OK;
    const int64_t cap = std::min<int64_t>(kMaxChunk, std::max<int64_t>((rows + 127) / 128 * 128, 2 * e->cap));
    ECK(cudaStreamSynchronize(st));
    free_chunk_buffers(e);
    const size_t bf = sizeof(__nv_bfloat16);
    cudaError_t err = cudaMalloc((void **)&e->xs, (size_t)cap * e->layers[0].ldi * bf);
    for (int l = 0; l + 1 < e->nl && err == cudaSuccess; ++l) {
        const Layer &L = e->layers[l];
        err = cudaMalloc((void **)&e->act[l], (size_t)cap * L.ldo * bf);
        if (err == cudaSuccess) err = cudaMalloc((void **)&e->Z[l], (size_t)cap * L.ldo * sizeof(float));
    }
    if (err == cudaSuccess) err = cudaMalloc((void **)&e->gA, (size_t)cap * e->maxw8 * bf);
    if (err == cudaSuccess) err = cudaMalloc((void **)&e->gB, (size_t)cap * e->maxw8 * bf);
    if (err != cudaSuccess) {
        free_chunk_buffers(e);
        return emu_cuda(err);
    }
    e->cap = cap;
    return TPCF_OK;
}

// forward pass of `rows` rows of the scaled inputs in e->xs.  Inference writes the
// unscaled outputs to y_out (rows w_out apart); training keeps the hidden
// pre-activations and turns the output layer into the loss gradient (e->gA) against
// the targets yt, adding the output bias gradient and the loss.
cudaError_t forward(tpcf_emu e, int64_t rows, bool training, const float *yt, float *y_out, double *loss,
                    double inv_count, cudaStream_t st)
{
    Operand in = {e->xs, e->layers[0].ldi, 0};
    for (int l = 0; l < e->nl; ++l) {
        const Layer &L = e->layers[l];
        GemmArgs g;
        std::memset(&g, 0, sizeof(g));
        g.M = (int)rows;
        g.N = L.out;
        g.K = L.in;
        g.bias = e->params + L.b_off;
        const Operand W = {e->wT[l], L.ldi, 0};   // B(o, i) = W[i][o], contiguous in i
        cudaError_t err;
        if (l + 1 < e->nl) {
            g.out_b = e->act[l];
            g.ld_b = L.ldo;
            g.out_f = training ? e->Z[l] : nullptr;
            g.ld_f = L.ldo;
            err = gemm<EPI_HID>(g, in, W, st);
            in = {e->act[l], L.ldo, 0};
        } else {
            g.mean = e->out_mean;
            g.sd = e->out_sd;
            if (training) {
                g.in_f = yt;
                g.pair_in = pairable(yt, L.out);
                g.ld_in = L.out;
                g.gscale = (float)(2.0 * inv_count);
                g.inv_count = (float)inv_count;
                g.loss = loss;
                g.colsum = e->grads + L.b_off;
                g.out_b = e->gA;
                g.ld_b = L.ldo;
                err = gemm<EPI_LOSS>(g, in, W, st);
            } else {
                g.out_f = y_out;
                g.pair_f = pairable(y_out, L.out);
                g.ld_f = L.out;
                err = gemm<EPI_PRED>(g, in, W, st);
            }
        }
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// backward pass of one chunk from the output-layer gradient in e->gA: weight
// gradients (split-K partials reduced into e->grads) and, layer by layer, the
// gradient of the previous layer's pre-activation with its bias gradient
cudaError_t backward(tpcf_emu e, int64_t rows, cudaStream_t st)
{
    __nv_bfloat16 *gcur = e->gA, *gnext = e->gB;
    for (int l = e->nl - 1; l >= 0; --l) {
        const Layer &L = e->layers[l];
        const __nv_bfloat16 *aprev = l > 0 ? e->act[l - 1] : e->xs;
        // dW[i][o] = sum_r aprev[r][i] g[r][o]: A(i, r) and B(o, r) both MN-major
        GemmArgs g;
        std::memset(&g, 0, sizeof(g));
        g.M = L.in;
        g.N = L.out;
        g.K = (int)rows;
        g.out_f = e->ws;
        g.ld_f = L.ldo;
        int splits = 0;
        const int max_splits = (int)std::max<int64_t>(1, e->ws_floats / ((int64_t)L.in * L.ldo));
        cudaError_t err = gemm<EPI_PART>(g, {aprev, L.ldi, 1}, {gcur, L.ldo, 1}, st, max_splits, &splits);
        if (err != cudaSuccess) return err;
        k_reduce_parts<<<grid1((int64_t)L.in * L.out), 256, 0, st>>>(e->ws, splits, (int64_t)L.in * L.ldo, L.in,
                                                                     L.out, L.ldo, e->grads + L.w_off);
        tpcf::note_launch();
        if (l > 0) {
            // dA_prev[r][i] = sum_o g[r][o] W[i][o], times SiLU'(z_prev): A = g, B(i, o) = wP[i][o]
            const Layer &Lp = e->layers[l - 1];
            GemmArgs h;
            std::memset(&h, 0, sizeof(h));
            h.M = (int)rows;
            h.N = L.in;
            h.K = L.out;
            h.in_f = e->Z[l - 1];
            h.pair_in = 1;   // rows of ldo floats (a multiple of 8)
            h.ld_in = Lp.ldo;
            h.out_b = gnext;
            h.ld_b = Lp.ldo;
            h.colsum = e->grads + Lp.b_off;
            err = gemm<EPI_BWD>(h, {gcur, L.ldo, 0}, {e->wP[l], L.ldo, 0}, st);
            if (err != cudaSuccess) return err;
            std::swap(gcur, gnext);
        }
    }
    return cudaGetLastError();
}

// full-batch gradient (in chunks of up to kMaxChunk rows) into e->grads
int batch_gradient(tpcf_emu e, const float *x, const float *y, int64_t batch, double *loss, cudaStream_t st)
{
    const int w_in = e->widths[0], w_out = e->widths[e->nl];
    int rc = ensure_cap(e, batch, st);
    if (rc) return rc;
    const double inv = 1.0 / ((double)batch * w_out);
    ECK(cudaMemsetAsync(e->grads, 0, e->n_params * sizeof(float), st));
    if (loss) ECK(cudaMemsetAsync(loss, 0, sizeof(double), st));
    for (int64_t r0 = 0; r0 < batch; r0 += e->cap) {
        const int64_t rows = std::min<int64_t>(e->cap, batch - r0);
        k_scale_in<<<grid1(rows * w_in), 256, 0, st>>>(x + r0 * w_in, rows, w_in, e->in_lo, e->in_hi, e->xs,
                                                        e->layers[0].ldi);
        tpcf::note_launch();
        ECK(forward(e, rows, true, y + r0 * w_out, nullptr, loss, inv, st));
        ECK(backward(e, rows, st));
    }
    return TPCF_OK;
}

}  // namespace

extern "C" {

int tpcf_emu_create(const int32_t *widths, int32_t n_layers, uint64_t seed, tpcf_emu *out)
{
    if (!widths || !out) return emu_fail(TPCF_ERR_ARG, "widths and out are required");
    if (n_layers < 1 || n_layers > kMaxLayers) return emu_fail(TPCF_ERR_ARG, "n_layers must be 1..8");
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] < 1 || widths[l] > kMaxWidth) return emu_fail(TPCF_ERR_ARG, "widths must be 1..4096");
    if (!encoder()) return emu_fail(TPCF_ERR_UNSUPPORTED, "the driver has no tensor-map encoder");
    tpcf_emu e = new tpcf_emu_s();
    e->nl = n_layers;
    int64_t off = 0;
    for (int l = 0; l <= n_layers; ++l) e->widths[l] = widths[l];
    int64_t ws_need = 0;
    for (int l = 0; l < n_layers; ++l) {
        Layer &L = e->layers[l];
        L.in = widths[l];
        L.out = widths[l + 1];
        L.ldi = round8(L.in);
        L.ldo = round8(L.out);
        e->maxw8 = std::max({e->maxw8, L.ldo, L.ldi});
        ws_need = std::max<int64_t>(ws_need, (int64_t)L.in * L.ldo);
        L.w_off = off;
        off += (int64_t)L.in * L.out;
        L.b_off = off;
        off += L.out;
    }
    e->n_params = off;
    // room for at least 8 split-K partials of the largest weight gradient, 8 M floats at least
    e->ws_floats = std::max<int64_t>(8 * ws_need, (int64_t)8 << 20);
    cudaError_t err = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (err == cudaSuccess) err = cudaMalloc(p, bytes);
    };
    A((void **)&e->params, off * sizeof(float));
    A((void **)&e->grads, off * sizeof(float));
    A((void **)&e->m, off * sizeof(float));
    A((void **)&e->v, off * sizeof(float));
    A((void **)&e->in_lo, widths[0] * sizeof(float));
    A((void **)&e->in_hi, widths[0] * sizeof(float));
    A((void **)&e->out_mean, widths[n_layers] * sizeof(float));
    A((void **)&e->out_sd, widths[n_layers] * sizeof(float));
    A((void **)&e->ws, (size_t)e->ws_floats * sizeof(float));
    const size_t bf = sizeof(__nv_bfloat16);
    for (int l = 0; l < n_layers; ++l) {
        const Layer &L = e->layers[l];
        A((void **)&e->wT[l], (size_t)L.out * L.ldi * bf);
        A((void **)&e->wP[l], (size_t)L.in * L.ldo * bf);
    }
    // the padding of the weight copies is never written: zero it once
    for (int l = 0; l < n_layers && err == cudaSuccess; ++l) {
        const Layer &L = e->layers[l];
        err = cudaMemset(e->wT[l], 0, (size_t)L.out * L.ldi * bf);
        if (err == cudaSuccess) err = cudaMemset(e->wP[l], 0, (size_t)L.in * L.ldo * bf);
    }
    if (err == cudaSuccess) err = cudaMemset(e->params, 0, off * sizeof(float));
    if (err == cudaSuccess) err = cudaMemset(e->m, 0, off * sizeof(float));
    if (err == cudaSuccess) err = cudaMemset(e->v, 0, off * sizeof(float));
    if (err != cudaSuccess) {
        tpcf_emu_destroy(e);
        return emu_cuda(err);
    }
    for (int l = 0; l < n_layers; ++l) {
        const Layer &L = e->layers[l];
        const float a = (float)std::sqrt(6.0 / (L.in + L.out));
        k_init<<<grid1((int64_t)L.in * L.out), 256>>>(e->params, L.w_off, (int64_t)L.in * L.out, a, seed);
        tpcf::note_launch();
    }
    if (err == cudaSuccess) err = weight_copies(e, 0);
    std::vector<float> lo(widths[0], -1.f), hi(widths[0], 1.f), mu(widths[n_layers], 0.f), sd(widths[n_layers], 1.f);
    if (err == cudaSuccess) err = cudaMemcpy(e->in_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(e->in_hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(e->out_mean, mu.data(), mu.size() * 4, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(e->out_sd, sd.data(), sd.size() * 4, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        tpcf_emu_destroy(e);
        return emu_cuda(err);
    }
    *out = e;
    return TPCF_OK;
}

int tpcf_emu_destroy(tpcf_emu e)
{
    if (!e) return TPCF_OK;
    cudaDeviceSynchronize();
    free_chunk_buffers(e);
    for (void *p : {(void *)e->params, (void *)e->grads, (void *)e->m, (void *)e->v, (void *)e->in_lo,
                    (void *)e->in_hi, (void *)e->out_mean, (void *)e->out_sd, (void *)e->ws})
        if (p) cudaFree(p);
    for (int l = 0; l < kMaxLayers; ++l)
        for (void *p : {(void *)e->wT[l], (void *)e->wP[l]})
            if (p) cudaFree(p);
    delete e;
    return TPCF_OK;
}

int tpcf_emu_param_count(tpcf_emu e, int64_t *n)
{
    if (!e || !n) return emu_fail(TPCF_ERR_ARG, "handle and output are required");
    *n = e->n_params;
    return TPCF_OK;
}

int tpcf_emu_set_input_box(tpcf_emu e, const float *lo, const float *hi)
{
    if (!e || !lo || !hi) return emu_fail(TPCF_ERR_ARG, "handle, lo and hi are required");
    for (int i = 0; i < e->widths[0]; ++i)
        if (!(hi[i] > lo[i])) return emu_fail(TPCF_ERR_ARG, "every input needs hi > lo");
    ECK(cudaMemcpy(e->in_lo, lo, e->widths[0] * sizeof(float), cudaMemcpyHostToDevice));
    ECK(cudaMemcpy(e->in_hi, hi, e->widths[0] * sizeof(float), cudaMemcpyHostToDevice));
    return TPCF_OK;
}

int tpcf_emu_fit_output_scaling(tpcf_emu e, const float *y, int64_t n, void *stream)
{
    if (!e || !y || n < 1) return emu_fail(TPCF_ERR_ARG, "handle and at least one target row are required");
    const int w = e->widths[e->nl];
    // row blocks: enough CTAs to fill the GPU, partials in the split-K workspace
    int R = (int)std::min<int64_t>(256, (n + 1023) / 1024);
    R = std::max(1, std::min<int>(R, (int)(e->ws_floats * sizeof(float) / (sizeof(double2) * (size_t)w))));
    double2 *part = reinterpret_cast<double2 *>(e->ws);
    cudaStream_t st = (cudaStream_t)stream;
    k_col_partial<<<dim3((w + 31) / 32, R), 256, 0, st>>>(y, n, w, part);
    k_col_stats<<<(w + 127) / 128, 128, 0, st>>>(part, R, n, w, e->out_mean, e->out_sd);
    tpcf::note_launch(2);
    ECK(cudaGetLastError());
    return TPCF_OK;
}

int tpcf_emu_gradients(tpcf_emu e, const float *x, const float *y, int64_t batch, float *grad, double *loss,
                       void *stream)
{
    if (!e || !x || !y || !grad || batch < 1) return emu_fail(TPCF_ERR_ARG, "handle, x, y, grad and batch >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = batch_gradient(e, x, y, batch, loss, st);
    if (rc) return rc;
    ECK(cudaMemcpyAsync(grad, e->grads, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return TPCF_OK;
}

int tpcf_emu_train_step(tpcf_emu e, const float *x, const float *y, int64_t batch, float lr, double *loss,
                        void *stream)
{
    if (!e || !x || !y || batch < 1) return emu_fail(TPCF_ERR_ARG, "handle, x, y and batch >= 1 are required");
    if (!(lr > 0.f)) return emu_fail(TPCF_ERR_ARG, "lr must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = batch_gradient(e, x, y, batch, loss, st);
    if (rc) return rc;
    ++e->step;
    const double b1 = 0.9, b2 = 0.999;
    const double c1 = 1.0 - std::pow(b1, (double)e->step), c2 = 1.0 - std::pow(b2, (double)e->step);
    // bias-corrected step folded into the learning rate and epsilon
    const float lr_t = (float)(lr * std::sqrt(c2) / c1);
    const float eps_t = (float)(1e-8 * std::sqrt(c2));
    k_adam<<<grid1(e->n_params), 256, 0, st>>>(e->params, e->grads, e->m, e->v, e->n_params, lr_t, (float)b1,
                                               (float)b2, eps_t);
    tpcf::note_launch();
    ECK(weight_copies(e, st));
    ECK(cudaGetLastError());
    return TPCF_OK;
}

int tpcf_emu_predict(tpcf_emu e, const float *x, int64_t n, float *y, void *stream)
{
    if (!e || n < 0 || (n > 0 && (!x || !y))) return emu_fail(TPCF_ERR_ARG, "handle, x and y are required");
    if (n == 0) return TPCF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int w_in = e->widths[0], w_out = e->widths[e->nl];
    int rc = ensure_cap(e, n, st);
    if (rc) return rc;
    for (int64_t r0 = 0; r0 < n; r0 += e->cap) {
        const int64_t rows = std::min<int64_t>(e->cap, n - r0);
        k_scale_in<<<grid1(rows * w_in), 256, 0, st>>>(x + r0 * w_in, rows, w_in, e->in_lo, e->in_hi, e->xs,
                                                        e->layers[0].ldi);
        tpcf::note_launch();
        ECK(forward(e, rows, false, nullptr, y + r0 * w_out, nullptr, 0.0, st));
    }
    ECK(cudaGetLastError());
    return TPCF_OK;
}

int tpcf_emu_get_params(tpcf_emu e, float *params, void *stream)
{
    if (!e || !params) return emu_fail(TPCF_ERR_ARG, "handle and params are required");
    ECK(cudaMemcpyAsync(params, e->params, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_emu_set_params(tpcf_emu e, const float *params, void *stream)
{
    if (!e || !params) return emu_fail(TPCF_ERR_ARG, "handle and params are required");
    cudaStream_t st = (cudaStream_t)stream;
    ECK(cudaMemcpyAsync(e->params, params, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ECK(cudaMemsetAsync(e->m, 0, e->n_params * sizeof(float), st));
    ECK(cudaMemsetAsync(e->v, 0, e->n_params * sizeof(float), st));
    ECK(weight_copies(e, st));
    e->step = 0;
    ECK(cudaGetLastError());
    return TPCF_OK;
}

int tpcf_emu_set_output_scaling(tpcf_emu e, const float *mean, const float *std_dev)
{
    if (!e || !mean || !std_dev) return emu_fail(TPCF_ERR_ARG, "handle, mean and std_dev are required");
    const int w = e->widths[e->nl];
    for (int i = 0; i < w; ++i)
        if (!(std_dev[i] > 0.f) || !(mean[i] == mean[i])) return emu_fail(TPCF_ERR_ARG, "every std must be > 0");
    ECK(cudaDeviceSynchronize());
    ECK(cudaMemcpy(e->out_mean, mean, w * sizeof(float), cudaMemcpyHostToDevice));
    ECK(cudaMemcpy(e->out_sd, std_dev, w * sizeof(float), cudaMemcpyHostToDevice));
    return TPCF_OK;
}

int tpcf_emu_get_input_box(tpcf_emu e, float *lo, float *hi)
{
    if (!e || !lo || !hi) return emu_fail(TPCF_ERR_ARG, "handle, lo and hi are required");
    ECK(cudaMemcpy(lo, e->in_lo, e->widths[0] * sizeof(float), cudaMemcpyDeviceToHost));
    ECK(cudaMemcpy(hi, e->in_hi, e->widths[0] * sizeof(float), cudaMemcpyDeviceToHost));
    return TPCF_OK;
}

int tpcf_emu_get_optimizer(tpcf_emu e, float *m, float *v, int64_t *step, void *stream)
{
    if (!e || !m || !v || !step) return emu_fail(TPCF_ERR_ARG, "handle, m, v and step are required");
    cudaStream_t st = (cudaStream_t)stream;
    ECK(cudaMemcpyAsync(m, e->m, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ECK(cudaMemcpyAsync(v, e->v, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    *step = e->step;
    return TPCF_OK;
}

int tpcf_emu_set_optimizer(tpcf_emu e, const float *m, const float *v, int64_t step, void *stream)
{
    if (!e || !m || !v || step < 0) return emu_fail(TPCF_ERR_ARG, "handle, m, v and step >= 0 are required");
    cudaStream_t st = (cudaStream_t)stream;
    ECK(cudaMemcpyAsync(e->m, m, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ECK(cudaMemcpyAsync(e->v, v, e->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    e->step = step;
    return TPCF_OK;
}

int tpcf_emu_get_output_scaling(tpcf_emu e, float *mean, float *std_dev)
{
    if (!e || !mean || !std_dev) return emu_fail(TPCF_ERR_ARG, "handle, mean and std_dev are required");
    const int w = e->widths[e->nl];
    ECK(cudaDeviceSynchronize());
    ECK(cudaMemcpy(mean, e->out_mean, w * sizeof(float), cudaMemcpyDeviceToHost));
    ECK(cudaMemcpy(std_dev, e->out_sd, w * sizeof(float), cudaMemcpyDeviceToHost));
    return TPCF_OK;
}

}  // extern "C"
