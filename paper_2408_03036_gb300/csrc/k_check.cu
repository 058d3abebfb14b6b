// Self-check of the pair stage's reciprocal square root (rsqrt_newton) against
// CUDA's correctly rounded __frsqrt_rn on pseudo-random inputs.
#include <cstdint>
#include <cuda_runtime.h>

#include "k_pairs.cuh"

namespace tpcf {

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    // splitmix64 finaliser (Steele, Lea and Flood, 2014)
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// stats: [0] max |ulp difference| (atomicMax on an integer), [1] sum of relative
// differences, [2] sum of x y^2 - 1 for rsqrt_newton, [3] the same for __frsqrt_rn,
// [4] count of differing results.  Inputs are log-uniform on [1, 2^62).
__global__ void k_check_rsqrt(int64_t n, unsigned long long seed, double *stats, unsigned long long *maxulp)
{
    double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
    unsigned long long mu = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long h = mix64(seed ^ mix64((unsigned long long)i));
        const unsigned e = 127u + (unsigned)(h % 62ull);
        const unsigned mant = (unsigned)(h >> 40) & 0x7fffffu;
        const float x = __uint_as_float((e << 23) | mant);
        const float a = rsqrt_newton(x), b = __frsqrt_rn(x);
        const long long d = (long long)__float_as_uint(a) - (long long)__float_as_uint(b);
        const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
        mu = ad > mu ? ad : mu;
        s1 += ((double)a - (double)b) / (double)b;
        s2 += (double)x * (double)a * (double)a - 1.0;
        s3 += (double)x * (double)b * (double)b - 1.0;
        s4 += d != 0 ? 1.0 : 0.0;
    }
    atomicAdd(stats + 1, s1);
    atomicAdd(stats + 2, s2);
    atomicAdd(stats + 3, s3);
    atomicAdd(stats + 4, s4);
    atomicMax(maxulp, mu);
}

// FP32 FMA throughput: every thread runs 8 independent chains of `iters` fused
// multiply-adds (scalar fma.rn.f32 in inline PTX, or the paired FFMA2 form when
// PAIRED), enough independent work per scheduler to cover the pipe latency.  The
// chains' sum is written only if it equals an impossible value, so the work stays.
template <bool PAIRED>
__global__ void __launch_bounds__(256) k_ffma_peak(int iters, float *sink)
{
    const float s = 1.0f + 1e-7f * (float)(threadIdx.x & 7);
    if (PAIRED) {
        float2 a[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = make_float2(0.5f + 0.01f * j, 0.25f + 0.01f * j);
        const float2 m = make_float2(s, s), c = make_float2(1e-6f, -1e-6f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = __ffma2_rn(a[j], m, c);
        }
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) t += a[j].x + a[j].y;
        if (t == -12345.f) sink[threadIdx.x] = t;
    } else {
        float a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = 0.5f + 0.01f * j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[j]) : "f"(s), "f"(1e-6f));
        }
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) t += a[j];
        if (t == -12345.f) sink[threadIdx.x] = t;
    }
}

}  // namespace

// Launches the FMA microbenchmark on `blocks` CTAs of 256 threads; 16 FLOP per
// thread and iteration.
cudaError_t ffma_peak(bool paired, int blocks, int iters, float *sink, cudaStream_t st)
{
    if (paired) k_ffma_peak<true><<<blocks, 256, 0, st>>>(iters, sink);
    else k_ffma_peak<false><<<blocks, 256, 0, st>>>(iters, sink);
    note_launch();
    return cudaGetLastError();
}

cudaError_t check_rsqrt(int64_t n, unsigned long long seed, double *stats, unsigned long long *maxulp,
                        cudaStream_t st)
{
    k_check_rsqrt<<<sm_count() * 4, 256, 0, st>>>(n, seed, stats, maxulp);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpcf
