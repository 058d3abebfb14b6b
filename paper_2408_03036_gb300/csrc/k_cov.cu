// Sample covariance of data vectors over mocks (Eq. covariance of
// arXiv:2408.03036, Sec. 4.3): the mean over mocks, then a Gram over mocks of
// the centred data vectors, in FP64.  Data vector i of mock k is
// src[k * stride + idx[i]] (idx NULL: i), so the batch's zeta array is used in
// place with a selection of multipoles and triangles.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

namespace {

constexpr int CT = 64;   // covariance tile edge
constexpr int CK = 16;   // mocks per staged chunk

__device__ __forceinline__ int64_t dv_col(const int64_t *idx, int64_t i) { return idx ? idx[i] : i; }

// mean[i] = sum_k d_i^k / n; one thread per data-vector entry (coalesced over i
// for a contiguous selection).
// An index outside [0, stride) latches DEV_ERR_INDEX and yields NaN (no load).
__global__ void k_cov_mean(const double *__restrict__ src, int64_t n, int64_t stride,
                           const int64_t *__restrict__ idx, int64_t nd, double *__restrict__ mean, int *err)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nd) return;
    const int64_t c = dv_col(idx, i);
    if (c < 0 || c >= stride) {
        atomicCAS(err, 0, DEV_ERR_INDEX);
        mean[i] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += src[k * stride + c];
    mean[i] = s / (double)n;
}

// One CTA per upper-triangle 64 x 64 tile (ti <= tj) of C.  256 threads, each
// with a 4 x 4 block of outputs at rows ty + 16 a and columns tx + 16 b (so
// the shared-memory reads are conflict-free); CK mocks of centred values are
// staged at a time.  Off-diagonal tiles are written twice (C is symmetric).
__global__ void __launch_bounds__(256) k_cov_gram(const double *__restrict__ src, int64_t n, int64_t stride,
                                                  const int64_t *__restrict__ idx, int64_t nd,
                                                  const double *__restrict__ mean, int ntile,
                                                  double *__restrict__ cov)
{
    __shared__ double sA[CK][CT];
    __shared__ double sB[CK][CT];
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t k0 = 0; k0 < n; k0 += CK) {
        __syncthreads();
        for (int e = tid; e < 2 * CK * CT; e += 256) {
            const int which = e / (CK * CT), r = e % (CK * CT), kk = r / CT, c = r % CT;
            const int64_t i = (int64_t)(which ? tj : ti) * CT + c, k = k0 + kk;
            double v = 0.0;
            if (i < nd && k < n) {
                const int64_t col = dv_col(idx, i);
                v = (col >= 0 && col < stride) ? src[k * stride + col] - mean[i]
                                                : __longlong_as_double(0x7ff8000000000000ll);
            }
            if (which) sB[kk][c] = v;
            else sA[kk][c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < CK; ++kk) {
            double x[4], y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                x[a] = sA[kk][ty + 16 * a];
                y[a] = sB[kk][tx + 16 * a];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
        }
    }
    const double inv = 1.0 / (double)(n - 1);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t i = (int64_t)ti * CT + ty + 16 * a, j = (int64_t)tj * CT + tx + 16 * b;
            if (i < nd && j < nd) {
                const double v = acc[a][b] * inv;
                cov[i * nd + j] = v;
                if (ti != tj) cov[j * nd + i] = v;
            }
        }
}

}  // namespace

cudaError_t covariance(const double *src, int64_t n, int64_t stride, const int64_t *idx, int64_t nd, double *mean,
                       double *cov, int *err, cudaStream_t st)
{
    k_cov_mean<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(src, n, stride, idx, nd, mean, err);
    note_launch();
    const int64_t ntile = (nd + CT - 1) / CT;
    const int64_t nblk = ntile * (ntile + 1) / 2;
    if (nblk > 0x7fffffff) return cudaErrorInvalidValue;
    k_cov_gram<<<(unsigned)nblk, 256, 0, st>>>(src, n, stride, idx, nd, mean, (int)ntile, cov);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpcf
