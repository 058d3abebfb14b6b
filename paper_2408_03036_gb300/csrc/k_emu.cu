// MLP emulator of the tree-level 3PCF multipoles: forward, backward and Adam
// kernels behind the tpcf_emu_* C ABI (include/tpcf_emu.h).
//
// Every product of the network is one tiled GEMM kernel (64 x 64 output tiles,
// 16-deep K slices in shared memory, 4 x 4 outputs per thread, FP32
// accumulation) with BF16 weights read through the same tile loader; the
// epilogue adds the bias and applies SiLU in the forward pass.  Backward:
// dZ = dA * SiLU'(Z), dW = A_prev^T dZ, db = column sums of dZ, dA_prev = dZ W^T.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "../../include/tpcf_emu.h"

namespace {

constexpr int kMaxLayers = 8;
constexpr int kMaxWidth = 4096;
constexpr int kChunk = 4096;          // rows per internal pass (scratch capacity)

struct Layer {
    int in, out;
    int64_t w_off, b_off;             // offsets in the parameter vector
};

__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_SILU = 2 };

// C[m][n] = sum_k A(m, k) B(k, n) with A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn].
template <class TA, class TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(const TA *__restrict__ A, int64_t sam, int64_t sak,
                                              const TB *__restrict__ B, int64_t sbk, int64_t sbn, int M, int N,
                                              int K, float *__restrict__ C, int64_t ldc,
                                              const float *__restrict__ bias, float *__restrict__ act)
{
    __shared__ __align__(16) float As[16][68];   // [k][m]
    __shared__ __align__(16) float Bs[16][68];   // [k][n]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            int mm, kk;
            if (sak == 1) { kk = e & 15; mm = e >> 4; } else { mm = e & 63; kk = e >> 6; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? ld(A + m * sam + k * sak) : 0.f;
            int nn;
            if (sbn == 1) { nn = e & 63; kk = e >> 6; } else { kk = e & 15; nn = e >> 4; }
            const int n = n0 + nn, k2 = k0 + kk;
            Bs[kk][nn] = (n < N && k2 < K) ? ld(B + k2 * sbk + n * sbn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float z = acc[i][j];
            if (EPI != EPI_STORE) z += bias[n];
            C[m * ldc + n] = z;
            if (EPI == EPI_BIAS_SILU) act[m * ldc + n] = silu(z);
        }
    }
}

__global__ void k_scale_in(const float *__restrict__ x, int64_t n, int w, const float *__restrict__ lo,
                           const float *__restrict__ hi, float *__restrict__ xs)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * w; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % w);
        xs[i] = 2.f * (x[i] - lo[c]) / (hi[c] - lo[c]) - 1.f;
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

// dY = 2 (yhat - (y - mean) / sd) / (rows * w); loss += mean squared error
__global__ void k_loss_grad(const float *__restrict__ yhat, const float *__restrict__ y, int64_t rows, int w,
                            const float *__restrict__ mean, const float *__restrict__ sd, double inv_count,
                            float *__restrict__ dy, double *__restrict__ loss)
{
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * w;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % w);
        const float d = yhat[i] - (y[i] - mean[c]) / sd[c];
        dy[i] = (float)(2.0 * inv_count) * d;
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

__global__ void k_silu_back(const float *__restrict__ z, float *__restrict__ d, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] *= silu_grad(z[i]);
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
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, int64_t n, float lr_t, float b1,
                       float b2, float eps_t)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr_t * mi / (sqrtf(vi) + eps_t);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
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
    int maxw = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pbf = nullptr;
    float *in_lo = nullptr, *in_hi = nullptr, *out_mean = nullptr, *out_sd = nullptr;
    float *xs = nullptr;                      // scaled inputs [kChunk][in]
    float *Z[kMaxLayers] = {nullptr}, *A[kMaxLayers] = {nullptr};   // [kChunk][out_l]
    float *d0 = nullptr, *d1 = nullptr;       // gradient ping-pong [kChunk][maxw]
    float *gtmp = nullptr;                    // per-chunk gradient [n_params]
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

template <class TA, class TB, int EPI>
cudaError_t gemm(const TA *A, int64_t sam, int64_t sak, const TB *B, int64_t sbk, int64_t sbn, int M, int N, int K,
                 float *C, int64_t ldc, const float *bias, float *act, cudaStream_t st)
{
    const dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<TA, TB, EPI><<<grid, 256, 0, st>>>(A, sam, sak, B, sbk, sbn, M, N, K, C, ldc, bias, act);
    tpcf::note_launch();
    return cudaGetLastError();
}

// forward pass of rows [0, rows) of the scaled inputs already in e->xs
cudaError_t forward(tpcf_emu e, int64_t rows, cudaStream_t st)
{
    const float *in = e->xs;
    for (int l = 0; l < e->nl; ++l) {
        const Layer &L = e->layers[l];
        const __nv_bfloat16 *W = e->pbf + L.w_off;
        const float *b = e->params + L.b_off;
        cudaError_t err;
        if (l + 1 < e->nl)
            err = gemm<float, __nv_bfloat16, EPI_BIAS_SILU>(in, L.in, 1, W, L.out, 1, (int)rows, L.out, L.in, e->Z[l],
                                                            L.out, b, e->A[l], st);
        else
            err = gemm<float, __nv_bfloat16, EPI_BIAS>(in, L.in, 1, W, L.out, 1, (int)rows, L.out, L.in, e->Z[l], L.out,
                                                       b, nullptr, st);
        if (err != cudaSuccess) return err;
        in = e->A[l];
    }
    return cudaSuccess;
}

// loss gradient of one chunk into g (overwrites), loss added to *loss
cudaError_t backward_chunk(tpcf_emu e, const float *y, int64_t rows, double inv_count, float *g, double *loss,
                           cudaStream_t st)
{
    const int nl = e->nl, w_out = e->widths[nl];
    k_loss_grad<<<grid1(rows * w_out), 256, 0, st>>>(e->Z[nl - 1], y, rows, w_out, e->out_mean, e->out_sd,
                                                      inv_count, e->d0, loss);
    tpcf::note_launch();
    float *dcur = e->d0, *dnext = e->d1;
    for (int l = nl - 1; l >= 0; --l) {
        const Layer &L = e->layers[l];
        if (l + 1 < nl) {
            k_silu_back<<<grid1(rows * L.out), 256, 0, st>>>(e->Z[l], dcur, rows * L.out);
            tpcf::note_launch();
        }
        const float *aprev = l > 0 ? e->A[l - 1] : e->xs;
        // dW[i][o] = sum_r aprev[r][i] dZ[r][o]
        cudaError_t err = gemm<float, float, EPI_STORE>(aprev, 1, L.in, dcur, L.out, 1, L.in, L.out, (int)rows,
                                                        g + L.w_off, L.out, nullptr, nullptr, st);
        if (err != cudaSuccess) return err;
        k_col_sum<<<(L.out + 127) / 128, 128, 0, st>>>(dcur, rows, L.out, g + L.b_off, 0);
        tpcf::note_launch();
        if (l > 0) {
            // dA_prev[r][i] = sum_o dZ[r][o] W[i][o]
            err = gemm<float, __nv_bfloat16, EPI_STORE>(dcur, L.out, 1, e->pbf + L.w_off, 1, L.out, (int)rows, L.in,
                                                        L.out, dnext, L.in, nullptr, nullptr, st);
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
        k_scale_in<<<grid1(rows * w_in), 256, 0, st>>>(x + r0 * w_in, rows, w_in, e->in_lo, e->in_hi, e->xs);
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
    A((void **)&e->pbf, off * sizeof(__nv_bfloat16));
    A((void **)&e->in_lo, widths[0] * sizeof(float));
    A((void **)&e->in_hi, widths[0] * sizeof(float));
    A((void **)&e->out_mean, widths[n_layers] * sizeof(float));
    A((void **)&e->out_sd, widths[n_layers] * sizeof(float));
    A((void **)&e->xs, (size_t)kChunk * widths[0] * sizeof(float));
    for (int l = 0; l < n_layers; ++l) {
        A((void **)&e->Z[l], (size_t)kChunk * widths[l + 1] * sizeof(float));
        A((void **)&e->A[l], (size_t)kChunk * widths[l + 1] * sizeof(float));
    }
    A((void **)&e->d0, (size_t)kChunk * e->maxw * sizeof(float));
    A((void **)&e->d1, (size_t)kChunk * e->maxw * sizeof(float));
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
    k_to_bf16<<<grid1(off), 256>>>(e->params, e->pbf, off);
    tpcf::note_launch();
    std::vector<float> lo(widths[0], -1.f), hi(widths[0], 1.f), mu(widths[n_layers], 0.f), sd(widths[n_layers], 1.f);
    err = cudaMemcpy(e->in_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice);
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
    for (void *p : {(void *)e->params, (void *)e->grads, (void *)e->gtmp, (void *)e->m, (void *)e->v, (void *)e->pbf,
                    (void *)e->in_lo, (void *)e->in_hi, (void *)e->out_mean, (void *)e->out_sd, (void *)e->xs,
                    (void *)e->d0, (void *)e->d1})
        if (p) cudaFree(p);
    for (int l = 0; l < kMaxLayers; ++l) {
        if (e->Z[l]) cudaFree(e->Z[l]);
        if (e->A[l]) cudaFree(e->A[l]);
    }
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
    k_adam<<<grid1(e->n_params), 256, 0, st>>>(e->params, e->grads, e->m, e->v, e->pbf, e->n_params, lr_t, (float)b1,
                                               (float)b2, eps_t);
    tpcf::note_launch();
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
        k_scale_in<<<grid1(rows * w_in), 256, 0, st>>>(x + r0 * w_in, rows, w_in, e->in_lo, e->in_hi, e->xs);
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
    k_to_bf16<<<grid1(e->n_params), 256, 0, st>>>(e->params, e->pbf, e->n_params);
    tpcf::note_launch();
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
