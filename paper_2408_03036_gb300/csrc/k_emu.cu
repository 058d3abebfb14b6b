// MLP emulator of the tree-level 3PCF multipoles: forward, backward and Adam
// kernels behind the tpcf_emu_* C ABI (include/tpcf_emu.h).
//
// Every product of the network runs on the 5th-generation tensor cores: one GEMM
// kernel (k_gemm_tc) computes a 128-row x NT-column tile of C = A B with bf16
// operands (FP32 activations and gradients rounded to bf16 as they are staged,
// bf16 weights as stored) and FP32 accumulation in tensor memory; the epilogue
// reads the tile back from tensor memory and adds the bias and applies SiLU in
// the forward pass.  Backward: dZ = dA * SiLU'(Z), dW = A_prev^T dZ, db = column
// sums of dZ, dA_prev = dZ W^T, all three products on the same kernel.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_common.cuh"
#include "../../include/tpcf_emu.h"

namespace {

constexpr int kMaxLayers = 8;
constexpr int kMaxWidth = 4096;
constexpr int kChunk = 4096;          // rows per internal pass (scratch capacity)

struct Layer {
    int in, out;
    int ldi, ldo;                     // in and out rounded up to 8 (16-byte bf16 rows)
    int64_t w_off, b_off;             // offsets in the parameter vector
};

inline int round8(int n) { return (n + 7) / 8 * 8; }

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_SILU = 2 };

// C[m][n] = sum_k A(m, k) B(k, n) with A(m, k) = A[m sam + k sak] and
// B(k, n) = B[k sbk + n sbn], both bf16.
struct GemmArgs {
    const __nv_bfloat16 *A;
    int64_t sam, sak;
    const __nv_bfloat16 *B;
    int64_t sbk, sbn;
    int M, N, K;
    float *C;               // FP32 output, row stride ldc
    int64_t ldc;
    const float *bias;
    __nv_bfloat16 *act;     // bf16 SiLU(C), row stride ld_act (EPI_BIAS_SILU)
    int64_t ld_act;
    int a_vec, b_vec;       // operand contiguous in K with 16-byte aligned rows: 16-byte staging
    int NT;                 // tile columns: a power of two from 16 to 256
    int k_per;              // K values per split (a multiple of kKS); blockIdx.z takes split z
    int split;              // more than one split: the tiles are added into C (zeroed first)
    int tmem_cols;          // tensor-memory columns allocated: a power of two >= max(32, NT)
    int *err;
    long long wait_limit;   // polls of a per-stage mbarrier wait
    int wait_unmet;         // test mode: one more wait on a phase that nothing completes
};

constexpr int kGemmThreads = 256;
constexpr int kTM = 128;                 // tile rows (tensor-memory lanes, the MMA's M)
constexpr int kKS = 32;                  // K per stage: two MMAs of K = 16
constexpr uint32_t kRowBytes = kKS * 2;  // bytes of one operand row in a stage (bf16)
constexpr uint32_t kSBO = 4 * 128;       // bytes between 8-row core-matrix groups

// One CTA per (NT-column, 128-row) tile of C.  A stage holds the tile's 128 A rows
// and NT B columns for kKS values of K as bf16 in the canonical no-swizzle
// K-major layout (16-byte core-matrix rows, core matrices 128 bytes apart along K
// and kSBO apart across 8-row groups); stages are double-buffered (the next one
// is loaded into registers while the tensor cores read the current one), one
// thread issues the MMAs and commits them to the stage's mbarrier, and every
// wait is bounded: a timeout latches DEV_ERR_TIMEOUT, waits for the MMAs in
// flight, releases the tensor memory and returns.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 2) k_gemm_tc(const GemmArgs g)
{
    using namespace tpcf::tc;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * g.NT;
    const int NT = g.NT;
    const uint32_t a_bytes = kTM * kRowBytes, stage_bytes = a_bytes + (uint32_t)NT * kRowBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 2 * stage_bytes + 16);
    volatile int *s_abort = reinterpret_cast<int *>(smem + 2 * stage_bytes + 20);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // staging, per operand: 16-byte loads of 8 consecutive K values straight into a
    // core-matrix row when the operand is contiguous in K with aligned rows
    // (consecutive threads take consecutive octets of a row), otherwise one bf16
    // at a time with the lanes along whichever index is contiguous in memory
    // (every warp load one coalesced run)
    const bool a_kc = g.sak == 1, b_kc = g.sbk == 1;
    const int k_beg = blockIdx.z * g.k_per, k_end = min(g.K, k_beg + g.k_per);
    const int nbe = NT / 8;                      // scalar B elements per thread (NT x kKS / 256)
    const int nbu = NT * 4;                      // 16-byte B units (NT rows x 4 octets)
    uint4 va[2], vb[4];
    __nv_bfloat16 sa[16], sb[32];
    auto cm_off = [](int r, int k) -> uint32_t {   // byte offset of element (r, k) in an operand tile
        return (uint32_t)(((r >> 3) * 4 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
    };
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    auto load = [&](int st) {
        const int k0 = k_beg + st * kKS;
        if (g.a_vec) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int u = tid + kGemmThreads * q, r = u >> 2, k = k0 + 8 * (u & 3), m = m0 + r;
                va[q] = (m < g.M && k < k_end) ? __ldg(reinterpret_cast<const uint4 *>(g.A + m * g.sam + k))
                                                : make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                int r, k;
                if (a_kc) { r = (tid >> 5) + 8 * e; k = lane; }
                else { r = tid & (kTM - 1); k = (tid >> 7) + 2 * e; }
                const int m = m0 + r;
                k += k0;
                sa[e] = (m < g.M && k < k_end) ? g.A[m * g.sam + k * g.sak] : zero;
            }
        }
        if (g.b_vec) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = tid + kGemmThreads * q, nn = u >> 2, k = k0 + 8 * (u & 3), n = n0 + nn;
                vb[q] = (u < nbu && n < g.N && k < k_end)
                            ? __ldg(reinterpret_cast<const uint4 *>(g.B + n * g.sbn + k))
                            : make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (e >= nbe) break;
                int nn, k;
                if (b_kc) { nn = (tid >> 5) + 8 * e; k = lane; }
                else { nn = tid % NT; k = tid / NT + (kGemmThreads / NT) * e; }
                const int n = n0 + nn;
                k += k0;
                sb[e] = (n < g.N && k < k_end) ? g.B[k * g.sbk + n * g.sbn] : zero;
            }
        }
    };
    auto store = [&](int buf) {
        unsigned char *stg = smem + buf * stage_bytes;
        if (g.a_vec) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int u = tid + kGemmThreads * q;
                *reinterpret_cast<uint4 *>(stg + cm_off(u >> 2, 8 * (u & 3))) = va[q];
            }
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                int r, k;
                if (a_kc) { r = (tid >> 5) + 8 * e; k = lane; }
                else { r = tid & (kTM - 1); k = (tid >> 7) + 2 * e; }
                *reinterpret_cast<__nv_bfloat16 *>(stg + cm_off(r, k)) = sa[e];
            }
        }
        if (g.b_vec) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = tid + kGemmThreads * q;
                if (u < nbu) *reinterpret_cast<uint4 *>(stg + a_bytes + cm_off(u >> 2, 8 * (u & 3))) = vb[q];
            }
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (e >= nbe) break;
                int nn, k;
                if (b_kc) { nn = (tid >> 5) + 8 * e; k = lane; }
                else { nn = tid % NT; k = tid / NT + (kGemmThreads / NT) * e; }
                *reinterpret_cast<__nv_bfloat16 *>(stg + a_bytes + cm_off(nn, k)) = sb[e];
            }
        }
    };

    const int nst = k_end > k_beg ? (k_end - k_beg + kKS - 1) / kKS : 0;
    uint32_t phase[2] = {0u, 0u};
    bool used[2] = {false, false};
    bool ok = true;
    const uint32_t idesc = make_idesc(1u, kTM, NT);
    if (nst > 0) load(0);
    for (int st = 0; st < nst; ++st) {
        const int b = st & 1;
        // the MMAs that last read this buffer must have completed
        if (tid == 0 && used[b] && !mbar_wait(&bars[b], phase[b] ^ 1u, g.wait_limit)) *s_abort = 1;
        __syncthreads();
        if (*s_abort) { ok = false; break; }
        store(b);
        if (st + 1 < nst) load(st + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + b * stage_bytes);
#pragma unroll
            for (int ks = 0; ks < kKS / 16; ++ks) {
                const uint64_t da = make_desc(base + 256u * ks, 128, kSBO);
                const uint64_t db = make_desc(base + a_bytes + 256u * ks, 128, kSBO);
                mma_issue<false>(tmem, da, db, idesc, (st > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&bars[b]);
        }
        used[b] = true;
        phase[b] ^= 1u;
    }
    // the last MMAs: every buffer's latest commit
    if (ok && tid == 0) {
        for (int b = 0; b < 2; ++b)
            if (used[b] && !mbar_wait(&bars[b], phase[b] ^ 1u, g.wait_limit)) *s_abort = 1;
        // test mode: buffer 0's next phase, which no commit completes
        if (g.wait_unmet && !*s_abort && !mbar_wait(&bars[0], phase[0], g.wait_limit)) *s_abort = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*s_abort) ok = false;
    if (ok && nst > 0) {
        // warp w reads tensor-memory lanes 32 (w % 4) ..; the two warps of a lane
        // quarter take alternate 16-column chunks
        const int quarter = warp & 3, set = warp >> 2;
        const int row = m0 + 32 * quarter + lane;
        for (int c0 = 16 * set; c0 < NT; c0 += 32) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0, v);
            if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n >= g.N) break;
                    float z = v[j];
                    if (EPI != EPI_STORE) z += __ldg(g.bias + n);
                    if (EPI == EPI_STORE && g.split) atomicAdd(g.C + row * g.ldc + n, z);
                    else g.C[row * g.ldc + n] = z;
                    if (EPI == EPI_BIAS_SILU) g.act[row * g.ld_act + n] = __float2bfloat16_rn(silu(z));
                }
            }
        }
    } else if (!ok && tid == 0) {
        if (g.err) atomicCAS(g.err, 0, tpcf::DEV_ERR_TIMEOUT);
        // wait (on the long bound) for anything still in flight before releasing TMEM
        for (int b = 0; b < 2; ++b)
            if (used[b]) mbar_wait(&bars[b], phase[b] ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
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

// per-column mean and standard deviation (FP64 sums); one thread per column
__global__ void k_col_stats(const float *__restrict__ y, int64_t n, int w, float *__restrict__ mean,
                            float *__restrict__ sd)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        const double v = y[r * w + c];
        s += v;
        s2 += v * v;
    }
    const double mu = n > 0 ? s / n : 0.0;
    const double var = n > 1 ? fmax(s2 / n - mu * mu, 0.0) : 0.0;
    mean[c] = (float)mu;
    sd[c] = (float)(var > 0.0 ? sqrt(var) : 1.0);
}

// dY = 2 (yhat - (y - mean) / sd) / (rows * w); loss += mean squared error; dY also
// as bf16 rows of stride ld (the products' operand)
__global__ void k_loss_grad(const float *__restrict__ yhat, const float *__restrict__ y, int64_t rows, int w,
                            const float *__restrict__ mean, const float *__restrict__ sd, double inv_count,
                            float *__restrict__ dy, __nv_bfloat16 *__restrict__ dyb, int ld, double *__restrict__ loss)
{
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * w;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % w);
        const float d = yhat[i] - (y[i] - mean[c]) / sd[c];
        const float g = (float)(2.0 * inv_count) * d;
        dy[i] = g;
        dyb[(i / w) * ld + c] = __float2bfloat16_rn(g);
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(loss, t * inv_count);
    }
}

// d *= SiLU'(z) over rows x w, and the result as bf16 rows of stride ld
__global__ void k_silu_back(const float *__restrict__ z, float *__restrict__ d, int64_t rows, int w,
                            __nv_bfloat16 *__restrict__ db, int ld)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * w;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = d[i] * silu_grad(z[i]);
        d[i] = v;
        db[(i / w) * ld + (int)(i % w)] = __float2bfloat16_rn(v);
    }
}

// db[c] (+)= sum over rows of d[r][c]; one thread per column
__global__ void k_col_sum(const float *__restrict__ d, int64_t rows, int w, float *__restrict__ db, int accumulate)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    float s = 0.f;
    for (int64_t r = 0; r < rows; ++r) s += d[r * w + c];
    db[c] = accumulate ? db[c] + s : s;
}

__global__ void k_add(float *__restrict__ a, const float *__restrict__ b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

__global__ void k_unscale_out(const float *__restrict__ yhat, int64_t rows, int w, const float *__restrict__ mean,
                              const float *__restrict__ sd, float *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * w;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % w);
        y[i] = yhat[i] * sd[c] + mean[c];
    }
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
    int maxw = 0, maxw8 = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *in_lo = nullptr, *in_hi = nullptr, *out_mean = nullptr, *out_sd = nullptr;
    // bf16 operands of the products, rows padded to multiples of 8 (padding zero)
    __nv_bfloat16 *wT[kMaxLayers] = {nullptr};   // [out][ldi] transposed weights
    __nv_bfloat16 *wP[kMaxLayers] = {nullptr};   // [in][ldo] weights
    __nv_bfloat16 *xs = nullptr;                 // scaled inputs [kChunk][ldi of layer 0]
    __nv_bfloat16 *act[kMaxLayers] = {nullptr};  // hidden activations [kChunk][ldo]
    __nv_bfloat16 *db = nullptr;                 // output gradient of the current layer [kChunk][maxw8]
    float *Z[kMaxLayers] = {nullptr};            // pre-activations [kChunk][out] (FP32)
    float *d0 = nullptr, *d1 = nullptr;          // gradient ping-pong [kChunk][maxw] (FP32)
    float *gtmp = nullptr;                       // per-chunk gradient [n_params]
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

template <int EPI>
cudaError_t gemm(const __nv_bfloat16 *A, int64_t sam, int64_t sak, const __nv_bfloat16 *B, int64_t sbk, int64_t sbn,
                 int M, int N, int K, float *C, int64_t ldc, const float *bias, __nv_bfloat16 *act, int64_t ld_act,
                 cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    GemmArgs g;
    g.A = A;
    g.sam = sam;
    g.sak = sak;
    g.B = B;
    g.sbk = sbk;
    g.sbn = sbn;
    g.M = M;
    g.N = N;
    g.K = K;
    g.C = C;
    g.ldc = ldc;
    g.bias = bias;
    g.act = act;
    g.ld_act = ld_act;
    auto aligned16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    g.a_vec = sak == 1 && sam % 8 == 0 && aligned16(A);
    g.b_vec = sbk == 1 && sbn % 8 == 0 && aligned16(B);
    // tile width: 256 columns for wide outputs; narrow ones (hidden layers) in tiles
    // of at most 64 so that their few row tiles still spread over the SMs (a power
    // of two from 16 to 256: the staging map needs NT to divide 256)
    g.NT = 256;
    if (N <= 256) {
        g.NT = 16;
        while (g.NT < 64 && g.NT < N) g.NT <<= 1;
    }
    g.tmem_cols = 32;
    while (g.tmem_cols < g.NT) g.tmem_cols <<= 1;
    g.err = tpcf::device_error_flag();
    g.wait_limit = tpcf::device_wait_limit();
    g.wait_unmet = tpcf::device_wait_unmet();
    // split K when the output has too few tiles to fill the SMs (the weight
    // gradients: 256 x 256 outputs over thousands of rows); the splits' tiles
    // are added into the zeroed output with FP32 atomics
    const int tiles = ((N + g.NT - 1) / g.NT) * ((M + kTM - 1) / kTM);
    const int nst = (K + kKS - 1) / kKS;
    int splits = 1;
    if (EPI == EPI_STORE && tiles < 2 * tpcf::sm_count()) {
        splits = (2 * tpcf::sm_count() + tiles - 1) / tiles;
        splits = std::max(1, std::min(splits, nst / 4));
    }
    g.k_per = ((nst + splits - 1) / splits) * kKS;
    splits = (K + g.k_per - 1) / g.k_per;
    g.split = splits > 1 ? 1 : 0;
    if (g.split) {
        cudaError_t e = cudaMemsetAsync(C, 0, (size_t)M * ldc * sizeof(float), st);
        if (e != cudaSuccess) return e;
    }
    // two stages and the barriers; enough that the CTAs sharing an SM never ask for
    // more than its 512 tensor-memory columns (allocations never wait)
    size_t smem = 2 * ((size_t)kTM + g.NT) * kRowBytes + 64;
    const size_t floor_bytes = (size_t)(228 * 1024) / (512 / g.tmem_cols + 1) + 1024;
    if (smem < floor_bytes) smem = floor_bytes;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const unsigned long long bit = tpcf::device_bit();
    if (!(attr_done.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        if (e != cudaSuccess) return e;
        attr_done.fetch_or(bit, std::memory_order_acq_rel);
    }
    const dim3 grid((N + g.NT - 1) / g.NT, (M + kTM - 1) / kTM, splits);
    k_gemm_tc<EPI><<<grid, kGemmThreads, smem, st>>>(g);
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

// forward pass of rows [0, rows) of the scaled inputs already in e->xs
cudaError_t forward(tpcf_emu e, int64_t rows, cudaStream_t st)
{
    const __nv_bfloat16 *in = e->xs;
    int ld_in = e->layers[0].ldi;
    for (int l = 0; l < e->nl; ++l) {
        const Layer &L = e->layers[l];
        const float *b = e->params + L.b_off;
        // Z[r][o] = sum_i in[r][i] W[i][o] + b[o]: A = in (contiguous in i), B(i, o) = wT[o][i]
        cudaError_t err;
        if (l + 1 < e->nl)
            err = gemm<EPI_BIAS_SILU>(in, ld_in, 1, e->wT[l], 1, L.ldi, (int)rows, L.out, L.in, e->Z[l], L.out, b,
                                      e->act[l], L.ldo, st);
        else
            err = gemm<EPI_BIAS>(in, ld_in, 1, e->wT[l], 1, L.ldi, (int)rows, L.out, L.in, e->Z[l], L.out, b,
                                 nullptr, 0, st);
        if (err != cudaSuccess) return err;
        in = e->act[l];
        ld_in = L.ldo;
    }
    return cudaSuccess;
}

// loss gradient of one chunk into g (overwrites), loss added to *loss
cudaError_t backward_chunk(tpcf_emu e, const float *y, int64_t rows, double inv_count, float *g, double *loss,
                           cudaStream_t st)
{
    const int nl = e->nl, w_out = e->widths[nl];
    k_loss_grad<<<grid1(rows * w_out), 256, 0, st>>>(e->Z[nl - 1], y, rows, w_out, e->out_mean, e->out_sd,
                                                      inv_count, e->d0, e->db, e->layers[nl - 1].ldo, loss);
    tpcf::note_launch();
    float *dcur = e->d0, *dnext = e->d1;
    for (int l = nl - 1; l >= 0; --l) {
        const Layer &L = e->layers[l];
        if (l + 1 < nl) {
            k_silu_back<<<grid1(rows * L.out), 256, 0, st>>>(e->Z[l], dcur, rows, L.out, e->db, L.ldo);
            tpcf::note_launch();
        }
        const __nv_bfloat16 *aprev = l > 0 ? e->act[l - 1] : e->xs;
        const int ld_prev = L.ldi;
        // dW[i][o] = sum_r aprev[r][i] dZ[r][o]: A(i, r) = aprev[r][i], B(r, o) = db[r][o]
        cudaError_t err = gemm<EPI_STORE>(aprev, 1, ld_prev, e->db, L.ldo, 1, L.in, L.out, (int)rows,
                                          g + L.w_off, L.out, nullptr, nullptr, 0, st);
        if (err != cudaSuccess) return err;
        k_col_sum<<<(L.out + 127) / 128, 128, 0, st>>>(dcur, rows, L.out, g + L.b_off, 0);
        tpcf::note_launch();
        if (l > 0) {
            // dA_prev[r][i] = sum_o dZ[r][o] W[i][o]: A = db (contiguous in o), B(o, i) = wP[i][o]
            err = gemm<EPI_STORE>(e->db, L.ldo, 1, e->wP[l], 1, L.ldo, (int)rows, L.in, L.out, dnext, L.in, nullptr,
                                  nullptr, 0, st);
            if (err != cudaSuccess) return err;
            std::swap(dcur, dnext);
        }
    }
    return cudaGetLastError();
}

// full-batch gradient (in chunks of kChunk rows) into e->grads
int batch_gradient(tpcf_emu e, const float *x, const float *y, int64_t batch, double *loss, cudaStream_t st)
{
    const int w_in = e->widths[0], w_out = e->widths[e->nl];
    const double inv = 1.0 / ((double)batch * w_out);
    if (loss) ECK(cudaMemsetAsync(loss, 0, sizeof(double), st));
    for (int64_t r0 = 0; r0 < batch; r0 += kChunk) {
        const int64_t rows = std::min<int64_t>(kChunk, batch - r0);
        k_scale_in<<<grid1(rows * w_in), 256, 0, st>>>(x + r0 * w_in, rows, w_in, e->in_lo, e->in_hi, e->xs,
                                                        e->layers[0].ldi);
        tpcf::note_launch();
        ECK(forward(e, rows, st));
        float *g = r0 == 0 ? e->grads : e->gtmp;
        ECK(backward_chunk(e, y + r0 * w_out, rows, inv, g, loss, st));
        if (r0 > 0) {
            k_add<<<grid1(e->n_params), 256, 0, st>>>(e->grads, e->gtmp, e->n_params);
            tpcf::note_launch();
        }
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
    tpcf_emu e = new tpcf_emu_s();
    e->nl = n_layers;
    int64_t off = 0;
    for (int l = 0; l <= n_layers; ++l) {
        e->widths[l] = widths[l];
        e->maxw = std::max(e->maxw, (int)widths[l]);
    }
    for (int l = 0; l < n_layers; ++l) {
        Layer &L = e->layers[l];
        L.in = widths[l];
        L.out = widths[l + 1];
        L.ldi = round8(L.in);
        L.ldo = round8(L.out);
        e->maxw8 = std::max(e->maxw8, L.ldo);
        L.w_off = off;
        off += (int64_t)L.in * L.out;
        L.b_off = off;
        off += L.out;
    }
    e->n_params = off;
    cudaError_t err = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (err == cudaSuccess) err = cudaMalloc(p, bytes);
    };
    A((void **)&e->params, off * sizeof(float));
    A((void **)&e->grads, off * sizeof(float));
    A((void **)&e->gtmp, off * sizeof(float));
    A((void **)&e->m, off * sizeof(float));
    A((void **)&e->v, off * sizeof(float));
    A((void **)&e->in_lo, widths[0] * sizeof(float));
    A((void **)&e->in_hi, widths[0] * sizeof(float));
    A((void **)&e->out_mean, widths[n_layers] * sizeof(float));
    A((void **)&e->out_sd, widths[n_layers] * sizeof(float));
    const size_t bf = sizeof(__nv_bfloat16);
    A((void **)&e->xs, (size_t)kChunk * e->layers[0].ldi * bf);
    for (int l = 0; l < n_layers; ++l) {
        const Layer &L = e->layers[l];
        A((void **)&e->wT[l], (size_t)L.out * L.ldi * bf);
        A((void **)&e->wP[l], (size_t)L.in * L.ldo * bf);
        A((void **)&e->Z[l], (size_t)kChunk * L.out * sizeof(float));
        if (l + 1 < n_layers) A((void **)&e->act[l], (size_t)kChunk * L.ldo * bf);
    }
    A((void **)&e->db, (size_t)kChunk * e->maxw8 * bf);
    A((void **)&e->d0, (size_t)kChunk * e->maxw * sizeof(float));
    A((void **)&e->d1, (size_t)kChunk * e->maxw * sizeof(float));
    // zero the padded bf16 buffers once: their padding is never written
    if (err == cudaSuccess) err = cudaMemset(e->xs, 0, (size_t)kChunk * e->layers[0].ldi * bf);
    for (int l = 0; l < n_layers && err == cudaSuccess; ++l) {
        const Layer &L = e->layers[l];
        err = cudaMemset(e->wT[l], 0, (size_t)L.out * L.ldi * bf);
        if (err == cudaSuccess) err = cudaMemset(e->wP[l], 0, (size_t)L.in * L.ldo * bf);
        if (err == cudaSuccess && e->act[l]) err = cudaMemset(e->act[l], 0, (size_t)kChunk * L.ldo * bf);
    }
    if (err == cudaSuccess) err = cudaMemset(e->db, 0, (size_t)kChunk * e->maxw8 * bf);
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
    for (void *p : {(void *)e->params, (void *)e->grads, (void *)e->gtmp, (void *)e->m, (void *)e->v,
                    (void *)e->in_lo, (void *)e->in_hi, (void *)e->out_mean, (void *)e->out_sd, (void *)e->xs,
                    (void *)e->db, (void *)e->d0, (void *)e->d1})
        if (p) cudaFree(p);
    for (int l = 0; l < kMaxLayers; ++l)
        for (void *p : {(void *)e->Z[l], (void *)e->act[l], (void *)e->wT[l], (void *)e->wP[l]})
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
    k_col_stats<<<(w + 127) / 128, 128, 0, (cudaStream_t)stream>>>(y, n, w, e->out_mean, e->out_sd);
    tpcf::note_launch();
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
    cudaStream_t st = (cudaStream_t)stream;
    const int w_in = e->widths[0], w_out = e->widths[e->nl];
    for (int64_t r0 = 0; r0 < n; r0 += kChunk) {
        const int64_t rows = std::min<int64_t>(kChunk, n - r0);
        k_scale_in<<<grid1(rows * w_in), 256, 0, st>>>(x + r0 * w_in, rows, w_in, e->in_lo, e->in_hi, e->xs,
                                                        e->layers[0].ldi);
        tpcf::note_launch();
        ECK(forward(e, rows, st));
        k_unscale_out<<<grid1(rows * w_out), 256, 0, st>>>(e->Z[e->nl - 1], rows, w_out, e->out_mean, e->out_sd,
                                                           y + r0 * w_out);
        tpcf::note_launch();
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
