// Internal declarations shared by the CUDA translation units of libtpcf.
// Not part of the public ABI (include/tpcf.h is).
#pragma once

#include <atomic>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/tpcf.h"

#define TPCF_MAX_BINS 32
#define TPCF_MAX_LMAX 6
#define TPCF_MAX_TILE 8

namespace tpcf {

struct HarmTables;   // harmonic normalisation and self-sum tables (k_pairs.cuh)

// Device-side error latch values (first error wins).
enum : int { DEV_OK = 0, DEV_ERR_DATA = 1, DEV_ERR_TIMEOUT = 2, DEV_ERR_CAPACITY = 3, DEV_ERR_INDEX = 4 };

// Cell list in device memory.  Records are int4 {x, y, z, float_as_int(w)} with
// x, y, z uint32 fixed-point bit patterns, sorted by cell index
// ((cz * nc + cy) * nc + cx), cell = floor(u * nc / 2^32).
struct GridDev {
    int4 *rec = nullptr;
    int64_t *order = nullptr;      // input index of each record
    int32_t *cell_start = nullptr; // [ncell + 1]
    int64_t n = 0;
    int nc = 0;
    int64_t ncell = 0;
};

// Parameters of the pair-stage kernel (one struct, passed by value).
struct PairParams {
    const int4 *rec;
    const int32_t *cell_start;
    int nc;
    int s;              // cells scanned on each side of the primary's cell
    int periodic;
    const int4 *prim;   // primaries as records
    int64_t n_prim;
    int nb;
    int P;              // primaries per tile
    int chunk;          // staged pairs per chunk
    unsigned long long E[TPCF_MAX_BINS + 1];
    float Ef[TPCF_MAX_BINS + 1];  // edges as floats (seed of the bin-share estimate)
    float rmin_u, inv_dr_u;   // float bin estimate b = (sqrt(r2) - rmin_u) * inv_dr_u
    float t_off, tdelta;      // t = sqrt(r2) * inv_dr_u + t_off is the bin coordinate; a float t
                              // within tdelta of an integer is decided in exact arithmetic
    float rmax_trim;          // conservative r_max (units) for row trimming
    float h_u;                // cell side in units (2^32 / nc)
    double mono_coef[TPCF_MAX_BINS];  // c_b = (W - 1) * mono_coef[b]
    double mono_w;            // W used when mono_w_dev is null
    const double *mono_w_dev; // device W (overrides mono_w)
    int use_mono;
    const HarmTables *harm;   // device copy of the harmonic tables
    int vlos;                 // 1: line of sight from obs to each primary (else z)
    double obs[3];            // observer in fixed-point units (may lie outside the box)
    int remove_self;
    float *alm;
    int32_t *counts;
    double *diag;
    double *wsp;
    unsigned long long *pair_counts;
    // D - R fields whose randoms are the only records of negative weight (sign bit
    // set): per primary and bin, the count of such secondaries for primaries of
    // negative weight (zero rows for the others), and its sum over those primaries
    // per bin; null when not wanted.  Harmonic kernel only.
    int32_t *counts_r;
    unsigned long long *pair_counts_r;
    int *work;                // tile counter (zeroed before launch)
    int *err;                 // device error latch
    // Batches of catalogues (null prim_mock: one catalogue).  Primary i belongs to
    // mock prim_mock[i]; its cells start at mock * ncell_mock in cell_start, its
    // W is mono_w_mock[mock], and its diag / wsp / pair_counts go to that mock's
    // slice of the outputs.  Requires tiles within one mock: P = 1, or tile_start.
    const int *prim_mock;
    int64_t ncell_mock;
    const double *mono_w_mock;
    // batches: bad input latches the mock's own status (DEV_ERR_*) instead of err
    int *mock_status;
    // batches with several primaries per tile: tile t is primaries
    // [tile_start[t], tile_start[t + 1]) (at most P, all of one catalogue);
    // null: tile t is [t P, min((t + 1) P, n_prim))
    const int64_t *tile_start;
    int64_t n_tiles;
};

// Bit of the current device in a per-device "done" mask (one-time attribute set-up).
inline unsigned long long device_bit()
{
    int d = 0;
    cudaGetDevice(&d);
    return 1ull << (d & 63);
}

// Streaming multiprocessors of the current device (queried once per device and
// cached), for grid sizing in multiples of the SM count.
inline int sm_count()
{
    static int cache[64] = {0};
    int d = 0;
    cudaGetDevice(&d);
    int &c = cache[d & 63];
    if (c <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) v = 1;
        c = v;
    }
    return c;
}

// Polls of a per-stage mbarrier wait in the tensor-core kernels before they give
// up and latch DEV_ERR_TIMEOUT (tpcf_set_wait_limit; default 2^26), and the
// current device's error latch (read and cleared by tpcf_stream_status).
long long device_wait_limit();
int device_wait_unmet();   // test mode: one extra wait on an mbarrier phase that nothing completes
int *device_error_flag();

// Counts kernel launches made by the library (reported by tpcf_kernel_launches).
void note_launch(int n = 1);

// Host-side launchers (defined in the .cu files).
cudaError_t build_grid_dev(const uint32_t *xyz, const float *w, int64_t n,
                           const uint32_t *xyz2, const float *w2, int64_t n2, const double *wsums,
                           int nc, GridDev &g, int *err, cudaStream_t st);
void free_grid_dev(GridDev &g, cudaStream_t st);
// One grid over many catalogues: points [offsets[k], offsets[k+1]) form mock k,
// whose cells are k * nc^3 ... (k+1) * nc^3 - 1; rec_mock[i] = mock of record i.
cudaError_t build_grid_batched_dev(const uint32_t *xyz, const float *w, int64_t n, const int64_t *d_offsets,
                                   int n_mocks, int nc, GridDev &g, int32_t *rec_mock, int *err, cudaStream_t st,
                                   int *mock_status = nullptr);
// *out (zeroed by the caller) += number of w[i] != 1.
cudaError_t count_not_one(const float *w, int64_t n, int *out, cudaStream_t st);
// out[0] += weights whose sign bit is set, out[1] += weights > 0 (out zeroed by the caller)
cudaError_t weight_signs(const float *w, int64_t n, int *out, cudaStream_t st);
cudaError_t weight_sums_mocks(const float *w, const int64_t *d_offsets, int n_mocks, double *out, cudaStream_t st);

// records of n points; wsums = {W_D, W_R} (device) turns the weights into -(W_D / W_R) w
cudaError_t pack_records(const uint32_t *xyz, const float *w, int64_t n, int4 *out, int *err,
                         cudaStream_t st, const double *wsums = nullptr);
cudaError_t weight_sums(const float *w1, int64_t n1, const float *w2, int64_t n2, double *out2,
                        cudaStream_t st);

// Coupling (Gram over primaries) and assembly.
cudaError_t triplet_counts(const int32_t *counts, int64_t K, int nb, unsigned long long *T,
                           cudaStream_t st);
int gram_tile_count(int nb, int lmax);
// The plain FP32 Gram on the tensor-core tile plan (SIMT FMAs, FP64 partial sums); fills all of G.
cudaError_t couple_gram_simt(const float *alm, const float *w, int64_t K, int nb, int lmax, double *G, int sms,
                             cudaStream_t st);
// Tensor-core (tcgen05) Gram with bf16 or tf32 hi/lo splits; fills all of G.
cudaError_t couple_gram_tc(const float *alm, const float *w, int64_t K, int nb, int lmax, bool tf32, double *G,
                           int *err, int sms, cudaStream_t st);
// The Gram of every catalogue of a batch group in one launch (precision: a
// TPCF_PREC_* value): catalogue c owns the slices [mslice[c], mslice[c + 1]) of
// the slice boundaries slice_k (primaries relative to alm / w, in device memory,
// made by gram_batch_slices: no slice straddles two catalogues) and its G goes to
// G + c * gram_offset(nb, lmax, lmax + 1).
cudaError_t couple_gram_batched(const float *alm, const float *w, int n_cat, const int64_t *d_slice_k,
                                int n_slices, const int *d_mslice, int nb, int lmax, int precision, double *G,
                                int *err, int sms, cudaStream_t st);
// Host slice table of a batch group with catalogue offsets off[0..n_cat] (off[0]
// need not be 0); empty when no tile plan exists for (nb, lmax).
void gram_batch_slices(const int64_t *off, int n_cat, int nb, int lmax, bool simt, int sms,
                       std::vector<int64_t> &slice_k, std::vector<int> &mslice);
// The FP32 Gram with a caller-provided tile table and no allocation (accumulates into G).
cudaError_t couple_gram_fp32_tiles(const float *alm, const float *w, int64_t K, int nb, int lmax, int *d_tiles,
                                   double *G, cudaStream_t st);
// j = k coefficients of the off-diagonal (l1 != l2) entries, [m][l1][l2][j] for one l_max
// (the same table tpcf_couple_multipoles uploads), written to host memory.
void self_term_table(int lmax, double *out);
// Host-side argument and configuration checks shared by the entry points.
int check_config_public(const tpcf_config *c);
int set_error(int code, const char *msg);
cudaError_t assemble_nnn(const double *G, const double *diag, const double *wsp, int nb, int lmax,
                         int remove_self, const double *gaunt, double *nnn, cudaStream_t st);
cudaError_t project_zeta(const double *nnn, const double *rrr, int nb, int lmax, int n_mult,
                         const double *coef, const int *mults, double *zeta, cudaStream_t st);
cudaError_t rrr_analytic(const double *wsum, const double *coef, int nb, double *rrr, cudaStream_t st);
// out[e][b] += sum_i w_i a_{lstep e}^0[b](i) (out zeroed by the caller; n_ell * nb <= 128).
cudaError_t m0_sums(const float *alm, const float *w, int64_t K, int nb, int lmax, int n_ell, int lstep, double *out,
                    cudaStream_t st);
// 2PCF multipoles from the m = 0 sums S and the pair normaliser (rr_mode 0 analytic,
// 1 random pair counts pc, 2 weighted random sums s0); rr [nb] is scratch.
cudaError_t xi_from_sums(int rr_mode, const double *wsums, const double *coef, const unsigned long long *pc,
                         const double *s0, const double *S, int n_ell, int lstep, int nb, double *rr, double *xi,
                         cudaStream_t st);
cudaError_t rrr_from_counts(const unsigned long long *T, const double *wsums, int nb, double *rrr,
                            cudaStream_t st);
// Sample covariance over n mocks of the data vectors d_i^k = src[k * stride + idx[i]]
// (idx NULL: i): mean [nd], cov [nd][nd] (Eq. covariance); bad indices latch DEV_ERR_INDEX.
cudaError_t covariance(const double *src, int64_t n, int64_t stride, const int64_t *idx, int64_t nd, double *mean,
                       double *cov, int *err, cudaStream_t st);
// Full edge correction: per bin pair, solve the Gaunt-coupled system of nu real
// unknowns (term list built on the host) for zeta_hat [L1][L1][L1][nb][nb].
cudaError_t edge_solve(const double *nnn, const double *rfull, int nb, int lmax, int nu, const int *modes,
                       const int *tstart, const int *tridx, const double *tcoef, double *zhat, int *err,
                       cudaStream_t st);
cudaError_t scale_alpha3(double *x, int64_t n, const double *wsums, cudaStream_t st);
// Self-check of the pair stage's reciprocal square root (see tpcf_check_rsqrt).
// FP32 FMA throughput microbenchmark (k_check.cu): blocks x 256 threads, 16 FLOP per
// thread and iteration; sink is never written in practice.
cudaError_t ffma_peak(bool paired, int blocks, int iters, float *sink, cudaStream_t st);
cudaError_t check_rsqrt(int64_t n, unsigned long long seed, double *stats, unsigned long long *maxulp,
                        cudaStream_t st);
cudaError_t i64_from_u64(const unsigned long long *src, int64_t *dst, int n, cudaStream_t st);

// Stream-ordered allocation of the library's device scratch and grids (released
// with cudaFreeAsync).  Outside a stream capture the memory comes from a pool of
// the library's own on the current device, which keeps freed blocks for later
// calls instead of handing them back to the driver at every synchronisation
// (tpcf_trim_memory hands them back); inside a capture from the device's default
// pool, as the graph's own allocations.
cudaError_t scratch_malloc(void **p, size_t bytes, cudaStream_t st);
// Unique id of the current CUDA context (0 if the driver does not report one).
unsigned long long context_id();

// Offsets of the per-m Gram blocks in the packed G array: block m is
// n_m x n_m doubles with n_m = nb * (lmax - m + 1); row index (l - m) * nb + b.
__host__ __device__ inline int64_t gram_offset(int nb, int lmax, int m)
{
    int64_t off = 0;
    for (int k = 0; k < m; ++k) {
        int64_t n = (int64_t)nb * (lmax - k + 1);
        off += n * n;
    }
    return off;
}

}  // namespace tpcf
