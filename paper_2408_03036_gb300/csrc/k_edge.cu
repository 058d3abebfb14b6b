// Full anisotropic edge correction: for every bin pair (r1, r2) solve
//   Re NNN^m_{l1 l2} = sum_{modes'} Mt[(l1 l2 m), (l1' l2' m')] zeta_hat^m'_{l1' l2'}
// where N = zeta R is the product of functions of (r_hat_1, r_hat_2) expanded
// in Y_l1^m(r_hat_1) Y_l2^m*(r_hat_2) (Eq. zeta_meas with the measured
// multipoles of Eq. measured_mult), so the matrix couples the randoms'
// RRR^m''_{l1'' l2''} through one Gaunt coefficient per direction:
//   Mt = 4 pi sum_{+-m'} sum_{l1'' l2''} RRR^{|m - m'|}_{l1'' l2''}
//        gaunt(l1', m', l1'', m - m', l1) gaunt(l2', m', l2'', m - m', l2).
// The host builds the sparse term list of Mt (coefficients and RRR block
// indices); the kernel evaluates it per bin pair and eliminates in FP64.
// Unknowns and equations are the real, l1 + l2 even coefficients with m >= 0
// (zeta_hat^-m = zeta_hat^m); for isotropic randoms the solution is
// NNN^m / RRR_00^0, the bin-wise estimate.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

namespace {

// One CTA per bin pair bb = b1 * nb + b2.  Shared memory: the augmented
// nu x (nu + 1) system, nu pivot factors, the pivot row index.
__global__ void __launch_bounds__(128) k_edge_solve(const double *__restrict__ nnn, const double *__restrict__ rfull,
                                                    int nb, int L1, int nu, const int *__restrict__ modes,
                                                    const int *__restrict__ tstart, const int *__restrict__ tridx,
                                                    const double *__restrict__ tcoef, double *__restrict__ zhat,
                                                    int *err)
{
    extern __shared__ double sm[];
    const int W = nu + 1;
    double *A = sm;                 // [nu][W]
    double *f = sm + (size_t)nu * W; // [nu]
    __shared__ int s_piv;
    const int bb = blockIdx.x, tid = threadIdx.x;
    const int64_t nbb = (int64_t)nb * nb;
    for (int e = tid; e < nu * nu; e += blockDim.x) {
        const int r = e / nu, c = e % nu;
        double v = 0.0;
        for (int t = tstart[e]; t < tstart[e + 1]; ++t) v += tcoef[t] * rfull[(int64_t)tridx[t] * nbb + bb];
        A[r * W + c] = v;
    }
    for (int r = tid; r < nu; r += blockDim.x) {
        const int l1 = modes[3 * r], l2 = modes[3 * r + 1], m = modes[3 * r + 2];
        A[r * W + nu] = nnn[(int64_t)((m * L1 + l1) * L1 + l2) * nbb + bb];
    }
    __syncthreads();
    bool singular = false;
    for (int k = 0; k < nu; ++k) {
        if (tid < 32) {
            // partial pivoting: the largest |A[i][k]|, i >= k
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < nu; i += 32) {
                const double a = fabs(A[i * W + k]);
                if (a > best) {
                    best = a;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) s_piv = bi;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k)
            for (int j = k + tid; j < W; j += blockDim.x) {
                const double t = A[k * W + j];
                A[k * W + j] = A[p * W + j];
                A[p * W + j] = t;
            }
        __syncthreads();
        const double piv = A[k * W + k];
        if (!(fabs(piv) > 0.0)) {
            singular = true;
            break;
        }
        for (int i = k + 1 + tid; i < nu; i += blockDim.x) f[i] = A[i * W + k] / piv;
        __syncthreads();
        const int ncol = W - k - 1;
        for (int e = tid; e < (nu - k - 1) * ncol; e += blockDim.x) {
            const int i = k + 1 + e / ncol, j = k + 1 + e % ncol;
            A[i * W + j] -= f[i] * A[k * W + j];
        }
        __syncthreads();
    }
    if (singular) {
        if (tid == 0) atomicCAS(err, 0, DEV_ERR_DATA);
        for (int r = tid; r < nu; r += blockDim.x) {
            const int l1 = modes[3 * r], l2 = modes[3 * r + 1], m = modes[3 * r + 2];
            zhat[(int64_t)((m * L1 + l1) * L1 + l2) * nbb + bb] = __longlong_as_double(0x7ff8000000000000ll);
        }
        return;
    }
    // back substitution (one thread; nu <= 72)
    if (tid == 0)
        for (int r = nu - 1; r >= 0; --r) {
            double s = A[r * W + nu];
            for (int c = r + 1; c < nu; ++c) s -= A[r * W + c] * A[c * W + nu];
            A[r * W + nu] = s / A[r * W + r];
        }
    __syncthreads();
    for (int r = tid; r < nu; r += blockDim.x) {
        const int l1 = modes[3 * r], l2 = modes[3 * r + 1], m = modes[3 * r + 2];
        zhat[(int64_t)((m * L1 + l1) * L1 + l2) * nbb + bb] = A[r * W + nu];
    }
}

__global__ void k_scale_alpha3(double *x, int64_t n, const double *__restrict__ wsums)
{
    const double a = wsums[0] / wsums[1];
    const double a3 = a * a * a;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= a3;
}

}  // namespace

size_t edge_solve_smem(int nu) { return ((size_t)nu * (nu + 1) + nu) * sizeof(double); }

cudaError_t edge_solve(const double *nnn, const double *rfull, int nb, int lmax, int nu, const int *modes,
                       const int *tstart, const int *tridx, const double *tcoef, double *zhat, int *err,
                       cudaStream_t st)
{
    static unsigned long long done = 0;
    const size_t smem = edge_solve_smem(nu);
    if (smem > 48 * 1024 && !(done & device_bit())) {
        cudaError_t e = cudaFuncSetAttribute(k_edge_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        done |= device_bit();
    }
    const size_t blk = (size_t)(lmax + 1) * (lmax + 1) * (lmax + 1) * nb * nb;
    cudaError_t e = cudaMemsetAsync(zhat, 0, blk * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_edge_solve<<<nb * nb, 128, smem, st>>>(nnn, rfull, nb, lmax + 1, nu, modes, tstart, tridx, tcoef, zhat, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scale_alpha3(double *x, int64_t n, const double *wsums, cudaStream_t st)
{
    int g = (int)((n + 255) / 256);
    if (g > 1024) g = 1024;
    if (n > 0) {
        k_scale_alpha3<<<g, 256, 0, st>>>(x, n, wsums);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace tpcf
