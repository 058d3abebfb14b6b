// Coupling of the per-primary harmonic sums (Eq. measured_mult of
// arXiv:2408.03036, summed over primaries as in Sec. 4.2), the integer triplet
// counts, the assembly of NNN^m, the TripoSH projection (Eq. slep2sugy), the
// random normalisers and the 2PCF multipoles of Eq. xi_meas_leg.
//
// Gram layout: for every m, the vector v_i of primary i collects
// a_l^m[b] for l = m..l_max, b = 0..n_b-1 (row (l - m) * n_b + b), real and
// imaginary parts separately; G_m = sum_i w_i (Re v_i Re v_i^T + Im v_i Im v_i^T)
// = sum_i w_i Re(v_i v_i^H).  Blocks are packed one after another (see
// gram_offset in internal.h).
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

namespace {

constexpr int GT = 32;        // Gram tile edge
constexpr int GK = 32;        // primaries per staged chunk
constexpr int GFLUSH = 8;     // chunks accumulated in FP32 before the FP64 flush

__device__ __forceinline__ int harm_index(int l, int m, int part)
{
    return l * l + (m == 0 ? 0 : 2 * m - 1 + part);
}

// One CTA: one 32x32 tile of one G_m block over a slice of primaries.
// 256 threads, 2x2 outputs each; FP32 partial sums over GFLUSH*GK primaries,
// then FP64 accumulation; FP64 atomics into G at the end.
__global__ void __launch_bounds__(256) k_gram_fp32(const float *__restrict__ alm, const float *__restrict__ w,
                                                   int64_t K, int nb, int lmax, const int *__restrict__ tiles,
                                                   int ntiles, double *__restrict__ G)
{
    __shared__ float sA[2][GK][GT + 1];
    __shared__ float sB[2][GK][GT + 1];
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const int m = tiles[3 * t], tr = tiles[3 * t + 1], tc = tiles[3 * t + 2];
    const int nlm = (lmax + 1) * (lmax + 1);
    const int n_m = nb * (lmax - m + 1);
    const int nparts = m == 0 ? 1 : 2;
    const int64_t per = (K + gridDim.y - 1) / gridDim.y;
    const int64_t k0 = blockIdx.y * per;
    const int64_t k1 = min(K, k0 + per);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc64[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    int nch = 0;
    for (int64_t kb = k0; kb < k1; kb += GK) {
        __syncthreads();
        // stage GK primaries x 32 rows (and cols) x parts
        for (int e = tid; e < 2 * nparts * GK * GT; e += 256) {
            const int which = e / (nparts * GK * GT);          // 0: rows (A), 1: cols (B)
            const int rem = e % (nparts * GK * GT);
            const int part = rem / (GK * GT);
            const int rem2 = rem % (GK * GT);
            const int kk = rem2 / GT, rr = rem2 % GT;
            const int64_t i = kb + kk;
            const int gidx = (which ? tc : tr) * GT + rr;
            float v = 0.f;
            if (i < k1 && gidx < n_m) {
                const int l = m + gidx / nb, b = gidx % nb;
                v = alm[(i * nb + b) * nlm + harm_index(l, m, part)];
                if (which == 0 && w) v *= w[i];
            }
            if (which == 0) sA[part][kk][rr] = v;
            else sB[part][kk][rr] = v;
        }
        __syncthreads();
        for (int part = 0; part < nparts; ++part) {
#pragma unroll 8
            for (int kk = 0; kk < GK; ++kk) {
                const float a0 = sA[part][kk][2 * ty], a1 = sA[part][kk][2 * ty + 1];
                const float b0 = sB[part][kk][2 * tx], b1 = sB[part][kk][2 * tx + 1];
                acc[0][0] = fmaf(a0, b0, acc[0][0]);
                acc[0][1] = fmaf(a0, b1, acc[0][1]);
                acc[1][0] = fmaf(a1, b0, acc[1][0]);
                acc[1][1] = fmaf(a1, b1, acc[1][1]);
            }
        }
        if (++nch == GFLUSH) {
            nch = 0;
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    acc64[a][b] += (double)acc[a][b];
                    acc[a][b] = 0.f;
                }
        }
    }
    const int64_t off = gram_offset(nb, lmax, m);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int r = tr * GT + 2 * ty + a, c = tc * GT + 2 * tx + b;
            const double v = acc64[a][b] + (double)acc[a][b];
            if (r < n_m && c < n_m && v != 0.0) atomicAdd(G + off + (int64_t)r * n_m + c, v);
        }
}

// T[b1][b2] += sum_i n_b1(i) (n_b2(i) - delta), exact in 64-bit integers.
// T[b1][b2] += sum_i c_i[b1] (c_i[b2] - [b1 == b2]) over the block's rows: tiles
// of kTripRows rows staged in shared memory with coalesced loads, one thread per
// (b1, b2) pair summing from there (integer sums: exact in any order).
constexpr int kTripRows = 128;
__global__ void k_triplets(const int32_t *__restrict__ counts, int64_t K, int nb, unsigned long long *T)
{
    __shared__ int32_t tile[kTripRows * TPCF_MAX_BINS];
    const int b1 = threadIdx.x / nb, b2 = threadIdx.x % nb;
    const bool mine = threadIdx.x < nb * nb;
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = blockIdx.x * per, k1 = min(K, k0 + per);
    unsigned long long s = 0;
    for (int64_t r0 = k0; r0 < k1; r0 += kTripRows) {
        const int rows = (int)min((int64_t)kTripRows, k1 - r0);
        __syncthreads();
        for (int q = threadIdx.x; q < rows * nb; q += blockDim.x) tile[q] = counts[r0 * nb + q];
        __syncthreads();
        if (mine) {
            const int d = b1 == b2 ? 1 : 0;
            for (int r = 0; r < rows; ++r) {
                const long long c1 = tile[r * nb + b1];
                const long long c2 = tile[r * nb + b2] - d;
                s += (unsigned long long)(c1 * c2);
            }
        }
    }
    if (mine && s) atomicAdd(T + threadIdx.x, s);
}

// nnn[m][l1][l2][b1][b2] from the Gram blocks, the diagonal residuals and the
// self sums.  gaunt[((m * (L+1) + l1) * (L+1) + l2) * (L+1) + j] multiplies
// wsp[j][b]: sum_i w_i sum_j w_j^2 Y_l1^m Y_l2^m* = sum_j gaunt * wsp_j.
__global__ void k_assemble(const double *__restrict__ G, const double *__restrict__ diag,
                           const double *__restrict__ wsp, int nb, int lmax, int remove_self,
                           const double *__restrict__ gaunt, double *__restrict__ nnn)
{
    const int L1 = lmax + 1;
    const int64_t tot = (int64_t)L1 * L1 * L1 * nb * nb;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx;
        const int b2 = r % nb; r /= nb;
        const int b1 = r % nb; r /= nb;
        const int l2 = r % L1; r /= L1;
        const int l1 = r % L1; r /= L1;
        const int m = (int)r;
        double v = 0.0;
        if (l1 >= m && l2 >= m && ((l1 + l2) & 1) == 0) {
            if (b1 == b2 && l1 == l2) {
                const int jd = l1 * (l1 + 1) / 2 + m;
                v = diag[(int64_t)jd * nb + b1];
            } else {
                const int n_m = nb * (lmax - m + 1);
                const int row = (l1 - m) * nb + b1, col = (l2 - m) * nb + b2;
                v = G[gram_offset(nb, lmax, m) + (int64_t)row * n_m + col];
                if (b1 == b2 && remove_self) {
                    const double *g = gaunt + ((int64_t)(m * L1 + l1) * L1 + l2) * L1;
                    double s = 0.0;
                    for (int j = 0; j <= lmax; ++j) s += g[j] * wsp[(int64_t)j * nb + b1];
                    v -= s;
                }
            }
        }
        nnn[idx] = v;
    }
}

// zeta[k][b1][b2] = sum_m coef[k][m] nnn[m][l1][l2][b1][b2] / rrr[b1][b2] (rrr NULL: no division)
__global__ void k_project(const double *__restrict__ nnn, const double *__restrict__ rrr, int nb, int lmax,
                          int n_mult, const double *__restrict__ coef, const int *__restrict__ mults,
                          double *__restrict__ zeta)
{
    const int L1 = lmax + 1;
    const int64_t tot = (int64_t)n_mult * nb * nb;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx / (nb * nb));
        const int bb = (int)(idx % (nb * nb));
        const int l1 = mults[3 * k], l2 = mults[3 * k + 1];
        double s = 0.0;
        for (int m = 0; m <= min(l1, l2); ++m)
            s += coef[k * L1 + m] * nnn[((int64_t)(m * L1 + l1) * L1 + l2) * nb * nb + bb];
        zeta[idx] = rrr ? s / rrr[bb] : s;
    }
}

__global__ void k_rrr_analytic(const double *__restrict__ wsum, const double *__restrict__ coef, int nb,
                               double *__restrict__ rrr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nb) return;
    const double W = wsum[0];
    const double c1 = (W - 1.0) * coef[i / nb], c2 = (W - 1.0) * coef[i % nb];
    rrr[i] = W * c1 * c2;
}

__global__ void k_rrr_counts(const unsigned long long *__restrict__ T, const double *__restrict__ wsums, int nb,
                             double *__restrict__ rrr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nb) return;
    const double a = wsums[0] / wsums[1];
    rrr[i] = a * a * a * (double)T[i] / (4.0 * 3.14159265358979323846);
}

// out[e][b] += sum_i w_i a_{lstep e}^0[b](i).  Each warp takes primaries in turn,
// its lanes the (e, b) outputs (at most 128, four per lane); FP64 sums, reduced
// in shared memory, then one FP64 atomic per output and CTA.
__global__ void __launch_bounds__(256) k_m0_sums(const float *__restrict__ alm, const float *__restrict__ w,
                                                 int64_t K, int nb, int lmax, int n_ell, int lstep,
                                                 double *__restrict__ out)
{
    __shared__ double s[128];
    const int n_out = n_ell * nb;
    for (int t = threadIdx.x; t < n_out; t += blockDim.x) s[t] = 0.0;
    __syncthreads();
    const int nlm = (lmax + 1) * (lmax + 1);
    const int lane = threadIdx.x & 31;
    int off[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int o = lane + 32 * q;
        const int l = lstep * (o / nb);
        off[q] = o < n_out ? (o % nb) * nlm + l * l : -1;
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < K; i += nwarp) {
        const double wi = w ? (double)w[i] : 1.0;
        const float *a = alm + i * nb * nlm;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (off[q] >= 0) acc[q] += wi * (double)a[off[q]];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (off[q] >= 0 && acc[q] != 0.0) atomicAdd(&s[lane + 32 * q], acc[q]);
    __syncthreads();
    for (int t = threadIdx.x; t < n_out; t += blockDim.x)
        if (s[t] != 0.0) atomicAdd(out + t, s[t]);
}

// 2PCF multipoles xi_l[b] = sqrt(4 pi (2l + 1)) S_l[b] / RR_b (Eq. xi_meas_leg with
// exact per-pair Legendre polynomials), l = lstep e.  RR_b by rr_mode:
//   0: analytic, W (W - 1) V_b / L^3 = W (W - 1) sqrt(4 pi) coef[b];
//   1: alpha^2 times the ordered random pair count pc[b] (unit random weights);
//   2: alpha^2 sqrt(4 pi) s0[b], s0 = sum_i w_i a_0^0[b] of the randoms.
__global__ void k_xi(int rr_mode, const double *__restrict__ wsums, const double *__restrict__ coef,
                     const unsigned long long *__restrict__ pc, const double *__restrict__ s0,
                     const double *__restrict__ S, int n_ell, int lstep, int nb, double *__restrict__ rr,
                     double *__restrict__ xi)
{
    const int b = threadIdx.x;
    if (b >= nb) return;
    const double sq4pi = 3.5449077018110320546;   // sqrt(4 pi)
    double r;
    if (rr_mode == 0) {
        const double W = wsums[0];
        r = W * (W - 1.0) * coef[b] * sq4pi;
    } else {
        const double a = wsums[0] / wsums[1];
        r = rr_mode == 1 ? a * a * (double)pc[b] : a * a * sq4pi * s0[b];
    }
    rr[b] = r;
    for (int e = 0; e < n_ell; ++e) {
        const int l = lstep * e;
        xi[e * nb + b] = sq4pi * sqrt(2.0 * l + 1.0) * S[e * nb + b] / r;
    }
}

// Fills the (m, tr, tc) tile table of the Gram blocks on the device.
__global__ void k_gram_tiles(int nb, int lmax, int *tiles, int ntiles)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int rem = t;
    for (int m = 0; m <= lmax; ++m) {
        const int n_m = nb * (lmax - m + 1);
        const int tm = (n_m + GT - 1) / GT;
        if (rem < tm * tm) {
            tiles[3 * t] = m;
            tiles[3 * t + 1] = rem / tm;
            tiles[3 * t + 2] = rem % tm;
            return;
        }
        rem -= tm * tm;
    }
}

__global__ void k_u64_to_i64(const unsigned long long *src, int64_t *dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (int64_t)src[i];
}

}  // namespace

int gram_tile_count(int nb, int lmax)
{
    int nt = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int t = (nb * (lmax - m + 1) + GT - 1) / GT;
        nt += t * t;
    }
    return nt;
}

// The FP32 Gram with a caller-provided device tile table (filled here) and no
// allocation of its own.
cudaError_t couple_gram_fp32_tiles(const float *alm, const float *w, int64_t K, int nb, int lmax, int *d_tiles,
                                   double *G, cudaStream_t st)
{
    const int nt = gram_tile_count(nb, lmax);
    k_gram_tiles<<<(nt + 127) / 128, 128, 0, st>>>(nb, lmax, d_tiles, nt);
    note_launch();
    int64_t ks = (sm_count() * 8 + nt - 1) / nt;
    const int64_t maxks = (K + 1023) / 1024;
    if (ks > maxks) ks = maxks;
    if (ks < 1) ks = 1;
    if (K > 0) {
        k_gram_fp32<<<dim3(nt, (unsigned)ks), 256, 0, st>>>(alm, w, K, nb, lmax, d_tiles, nt, G);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t triplet_counts(const int32_t *counts, int64_t K, int nb, unsigned long long *T, cudaStream_t st)
{
    int64_t g = (K + 1023) / 1024;
    if (g < 1) g = 1;
    if (g > sm_count() * 8) g = sm_count() * 8;
    if (K > 0) {
        k_triplets<<<(unsigned)g, ((nb * nb + 31) / 32) * 32, 0, st>>>(counts, K, nb, T);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t assemble_nnn(const double *G, const double *diag, const double *wsp, int nb, int lmax,
                         int remove_self, const double *gaunt, double *nnn, cudaStream_t st)
{
    const int64_t tot = (int64_t)(lmax + 1) * (lmax + 1) * (lmax + 1) * nb * nb;
    int g = (int)((tot + 255) / 256);
    if (g > 4096) g = 4096;
    k_assemble<<<g, 256, 0, st>>>(G, diag, wsp, nb, lmax, remove_self, gaunt, nnn);
    note_launch();
    return cudaGetLastError();
}

cudaError_t project_zeta(const double *nnn, const double *rrr, int nb, int lmax, int n_mult, const double *coef,
                         const int *mults, double *zeta, cudaStream_t st)
{
    const int64_t tot = (int64_t)n_mult * nb * nb;
    int g = (int)((tot + 255) / 256);
    if (g > 4096) g = 4096;
    if (tot > 0) {
        k_project<<<g, 256, 0, st>>>(nnn, rrr, nb, lmax, n_mult, coef, mults, zeta);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t rrr_analytic(const double *wsum, const double *coef, int nb, double *rrr, cudaStream_t st)
{
    k_rrr_analytic<<<(nb * nb + 255) / 256, 256, 0, st>>>(wsum, coef, nb, rrr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t rrr_from_counts(const unsigned long long *T, const double *wsums, int nb, double *rrr, cudaStream_t st)
{
    k_rrr_counts<<<(nb * nb + 255) / 256, 256, 0, st>>>(T, wsums, nb, rrr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t m0_sums(const float *alm, const float *w, int64_t K, int nb, int lmax, int n_ell, int lstep, double *out,
                    cudaStream_t st)
{
    if (n_ell * nb > 128 || lstep * (n_ell - 1) > lmax) return cudaErrorInvalidValue;
    if (K <= 0) return cudaSuccess;
    int64_t g = (K + 7) / 8;
    if (g > sm_count() * 4) g = sm_count() * 4;
    k_m0_sums<<<(unsigned)g, 256, 0, st>>>(alm, w, K, nb, lmax, n_ell, lstep, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t xi_from_sums(int rr_mode, const double *wsums, const double *coef, const unsigned long long *pc,
                         const double *s0, const double *S, int n_ell, int lstep, int nb, double *rr, double *xi,
                         cudaStream_t st)
{
    k_xi<<<1, 32, 0, st>>>(rr_mode, wsums, coef, pc, s0, S, n_ell, lstep, nb, rr, xi);
    note_launch();
    return cudaGetLastError();
}

cudaError_t i64_from_u64(const unsigned long long *src, int64_t *dst, int n, cudaStream_t st)
{
    if (n > 0) {
        k_u64_to_i64<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace tpcf
