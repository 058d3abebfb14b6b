/*
 * tpcf.h - C ABI of the GB300 (sm_103a) anisotropic three-point correlation
 * function estimator (Slepian-Eisenstein pair-count estimator with TripoSH
 * multipoles about a fixed line of sight along z).
 *
 * Method (arXiv:2408.03036, Sec. 4.2 "3PCF estimator" and Sec. 4, Eq. ssest):
 *   for every primary x_i and radial bin b (step function phi of Eq. alm)
 *       a_l^m[b](x_i) = sum_{j in b} w_j Y_l^m(r_hat_ij)            (Eq. alm)
 *   the local products of Eq. measured_mult, kept for m = m' with the second
 *   factor conjugated, summed over primaries with the primary's weight
 *       NNN^m_{l1 l2}[b1][b2] = sum_i w_i ( a_{l1}^m[b1] a_{l2}^m[b2]*
 *                                - delta_{b1 b2} sum_j w_j^2 Y_{l1}^m Y_{l2}^m* )
 *   (the subtracted term removes degenerate j = k triangles), and the
 *   TripoSH projection of Eq. slep2sugy, divided by the random triplet
 *   normaliser RRR_00^0 (Eq. ssest, (D-R)^3 / R^3):
 *       zeta_{l1 l2 L} = (2L+1) H_{l1 l2 L} sum_m (l1 l2 L; m -m 0) (-1)^m
 *                        Re NNN^m_{l1 l2} / RRR_00^0.
 *
 * Coordinates are uint32 fixed point: u = floor(x / L * 2^32).  Separations are
 * exact integer differences (modulo 2^32 in periodic boxes), r^2 is an exact
 * 64-bit integer, and a pair is in bin b iff E_b <= r^2 < E_{b+1} with
 * E_b = ceil(s_b^2), s_b = (r_b * 2^32) / L, r_b = r_min + ((r_max - r_min) * b) / n_bins
 * (all in IEEE double).  Pair and triplet counts are therefore exact integers.
 *
 * General rules for every entry point:
 *   - returns TPCF_OK (0) or a negative tpcf_status; a message for the last
 *     error of the calling thread is available from tpcf_last_error();
 *   - never aborts or traps; arguments are validated on the host;
 *   - pointers marked "dev" are device pointers owned by the caller; "host"
 *     pointers are host memory owned by the caller;
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); work is enqueued asynchronously on it unless stated otherwise;
 *     data errors found on the device (coordinates outside [0, 2^32), NaN
 *     weights) are latched in a device flag and reported by
 *     tpcf_stream_status();
 *   - scratch memory is taken with stream-ordered allocation on the given
 *     stream and returned before the call's work completes.
 */
#ifndef TPCF_H
#define TPCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TPCF_OK = 0,
    TPCF_ERR_ARG = -1,          /* invalid argument or configuration */
    TPCF_ERR_OOM = -2,          /* device allocation failed */
    TPCF_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    TPCF_ERR_TIMEOUT = -4,      /* a bounded device-side wait ran out */
    TPCF_ERR_UNSUPPORTED = -5,  /* valid request the library does not implement */
    TPCF_ERR_DATA = -6          /* bad input data detected on the device */
} tpcf_status;

/* Precision of the coupling sum over primaries (the pair stage is always FP32,
 * final sums FP64). */
enum {
    TPCF_PREC_FP32 = 0,     /* plain FP32 SIMT Gram, FP64 flush */
    TPCF_PREC_BF16X3 = 1,   /* tcgen05 tensor cores, bf16 hi/lo split, 3 products, FP32 accumulate */
    TPCF_PREC_TF32X3 = 2    /* tcgen05 tensor cores, tf32 hi/lo split, 3 products, FP32 accumulate */
};

/* Normalisation of the reported multipoles. */
enum {
    TPCF_CONV_S_COEFF = 0,  /* coefficient of the Schmidt basis S_{l1 l2 L} (Eq. TSHbasis):
                               sqrt((2 l1 + 1)(2 l2 + 1)) times Eq. slep2sugy */
    TPCF_CONV_PAPER_EQ = 1  /* Eq. slep2sugy as printed with orthonormal Y */
};

typedef struct {
    double r_min;           /* inner edge of the first radial bin, > 0 */
    double r_max;           /* outer edge of the last radial bin, < box / 2 */
    int32_t n_bins;         /* number of linear radial bins, 1..32 */
    int32_t l_max;          /* harmonics l1, l2 <= l_max, 0..6 */
    int32_t n_L;            /* number of TripoSH L values in L[], 1..8 */
    int32_t L[8];           /* the L values (even, 0..2 l_max) */
    int32_t periodic;       /* 1: periodic cube (minimum image), 0: open volume */
    double box;             /* cube side L in the same length unit as r */
    int32_t precision;      /* TPCF_PREC_* */
    int32_t remove_self;    /* 1: drop degenerate j = k triangles (default) */
    int32_t convention;     /* TPCF_CONV_* */
    int32_t cell_div;       /* cells per r_max along an axis, 1..6; 0 = automatic */
    int32_t tile_primaries; /* primaries processed together by one CTA, 1..8 (capped so that
                               tile_primaries * n_bins <= 128); 0 = automatic */
    int32_t chunk;          /* staged pairs per CTA, 4 bytes each (multiple of 256, 512..49152,
                               above 32 per bin); 0 = automatic (15360 up to l_max 4, else 49152) */
    int32_t los;            /* line of sight: 0 = z for every primary (Sec. 4.1, default);
                               1 = from `observer` to each primary (survey geometry): every
                               separation's harmonics are taken in a frame whose polar axis is
                               the primary's line of sight */
    double observer[3];     /* observer position for los = 1 (box coordinates, same length unit;
                               it may lie outside the box; |x| <= 1e6 box) */
} tpcf_config;

typedef struct tpcf_grid_s *tpcf_grid;   /* library-owned cell list (opaque) */

/* Message describing the calling thread's most recent error ("" if none). */
const char *tpcf_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int tpcf_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (a diagnostic: the difference around a call is that call's launch count). */
int64_t tpcf_kernel_launches(void);

/* Host positions to the library's fixed-point coordinates: u = floor(x / box *
 * 2^32), the product taken in FP64 (Sec. 4.1's cube of side L = box), for n
 * values (host x[n], host u[n]; three per point for xyz).  Every x must lie in
 * [0, box); TPCF_ERR_DATA (nothing written past the first bad value) for one
 * outside or not finite, TPCF_ERR_ARG for box <= 0 or missing arrays.  Wrapping
 * periodic positions into the box is the caller's step.  No device work. */
int tpcf_quantize_host(const float *x, int64_t n, double box, uint32_t *u);

/* Number of (l1, l2, L) multipoles the configuration produces.  These are all
 * triples with l1, l2 <= l_max, L in cfg->L, |l1 - l2| <= L <= l1 + l2 and
 * l1 + l2 + L even (Eq. slep2sugy with H_{l1 l2 L} != 0), ordered by the
 * position of L in cfg->L, then l1, then l2. */
int tpcf_multipole_count(const tpcf_config *cfg, int32_t *n_mult);

/* Writes the multipole triples, host l1l2L[n_mult][3] (capacity cap triples). */
int tpcf_multipole_index(const tpcf_config *cfg, int32_t *l1l2L, int32_t cap);

/* The exact integer bin edges E_b (b = 0..n_bins), host E[n_bins + 1]. */
int tpcf_bin_edges(const tpcf_config *cfg, uint64_t *E);

/* Cell list of a catalogue (the linked-list partition of Sec. 4.1, built as a
 * counting sort by cell).  dev xyz[n][3] uint32 fixed point, dev w[n] float
 * weights (NULL: unit weights), n < 2^28.  The grid copies what it needs; the inputs may
 * be freed once the stream has passed this call.  *out receives a handle that
 * must be released with tpcf_grid_destroy. */
int tpcf_build_grid(const uint32_t *xyz, const float *w, int64_t n, const tpcf_config *cfg,
                    tpcf_grid *out, void *stream);

/* Releases a grid (synchronises its stream first). NULL is accepted. */
int tpcf_grid_destroy(tpcf_grid grid);

/* Number of points and cells per axis of a grid. */
int tpcf_grid_info(tpcf_grid grid, int64_t *n_points, int32_t *cells_per_axis);

/* Copies the grid's points in grid (cell) order: dev xyz[n][3], dev w[n], and
 * dev order[n] = input index of each point.  Any output may be NULL. */
int tpcf_grid_points(tpcf_grid grid, uint32_t *xyz, float *w, int64_t *order, void *stream);

/* Testing aid for the device-side failure path (the paper has no counterpart).
 *   polls: the bound of every mbarrier wait of a tensor-core kernel before it
 *     gives up: the split-precision coupling makes `polls` non-blocking polls,
 *     the emulator's products polls / 16 suspending polls of at most a
 *     microsecond each; 0 restores the default (2^26, far longer than any stage).
 *   unmet_wait: nonzero makes every such kernel, once its own tensor-core work
 *     has completed, wait once more on an mbarrier phase that nothing completes
 *     (a flag that nothing sets), with that limit.
 * A wait that gives up sets the device error latch (TPCF_ERR_TIMEOUT at the next
 * tpcf_stream_status), waits on the long bound for the kernel's own tensor-core
 * work in flight, releases its tensor memory and returns: no fault, and the
 * context stays usable.  Process-wide; TPCF_ERR_ARG for a negative count. */
int tpcf_set_wait_limit(int64_t polls, int32_t unmet_wait);

/* Pair stage (Eq. alm): for every primary, the neighbour search to r_max over
 * the secondaries in `grid`, exact radial binning and the FP32 harmonic sums.
 *   prim_xyz/prim_w: dev primaries [n_prim][3] / [n_prim] (NULL: unit weights).
 *     If prim_xyz is NULL the primaries are the grid's own points in grid order
 *     (n_prim must then equal the grid's point count).
 *   monopole_weight: >= 0 enables the periodic analytic-random offset
 *     a_0^0[b] -= (monopole_weight - 1) / L^3 * V_b * Y_0^0; < 0 disables it.
 *   Outputs (dev, any may be NULL):
 *     alm[n_prim][n_bins][(l_max+1)^2]  real harmonic sums, per (l, m >= 0) the
 *        real part at index l^2 + max(2m - 1, 0) and, for m > 0, the imaginary
 *        part at l^2 + 2m (orthonormal Y with the Condon-Shortley phase);
 *     counts[n_prim][n_bins] int32 pair counts per primary;
 *     diag[(l_max+1)(l_max+2)/2][n_bins]  += sum_i w_i (|a_l^m[b]|^2 - s_{ll}^m[b]),
 *        (l, m) in the order l = 0..l_max, m = 0..l, where s is the j = k term
 *        (omitted when cfg->remove_self is 0);
 *     wsp[l_max+1][n_bins]  += sum_i w_i sum_j w_j^2 f_k(mu_ij), k = 0..l_max, with f_0 = 1
 *        and f_k = (2k)! P_{2k} (an intermediate consumed by tpcf_couple_multipoles
 *        for the j = k term of the l1 != l2 entries);
 *     pair_counts[n_bins]  int64, += total pairs per bin. */
int tpcf_accumulate_alm(tpcf_grid grid, const uint32_t *prim_xyz, const float *prim_w, int64_t n_prim,
                        const tpcf_config *cfg, double monopole_weight,
                        float *alm, int32_t *counts, double *diag, double *wsp, int64_t *pair_counts,
                        void *stream);

/* Integer pair counts only (the random-only pass behind RRR_00^0, the R^3 term
 * of Eq. ssest, with unit random weights): the same neighbour search and exact
 * binning as tpcf_accumulate_alm, without harmonics.
 *   prim_xyz: dev primaries [n_prim][3] (NULL: the grid's own points in grid
 *     order, n_prim equal to the grid's point count);
 *   counts: dev int32 [n_prim][n_bins] pair counts per primary (or NULL);
 *   pair_counts: dev int64 [n_bins], += total pairs per bin (or NULL).
 * Errors: TPCF_ERR_ARG for a NULL grid, n_prim < 0 or a mismatched n_prim. */
int tpcf_pair_counts(tpcf_grid grid, const uint32_t *prim_xyz, int64_t n_prim, const tpcf_config *cfg,
                     int32_t *counts, int64_t *pair_counts, void *stream);

/* Coupling over primaries (Eq. measured_mult summed over x): with the outputs of
 * tpcf_accumulate_alm for the same primaries (dev alm, dev prim_w or NULL for
 * unit weights, dev counts or NULL, dev diag, dev wsp), writes
 *   nnn[m][l1][l2][n_bins][n_bins]  (m, l1, l2 = 0..l_max; zero where l < m)
 *       = Re NNN^m_{l1 l2}, with the j = k term removed per cfg->remove_self;
 *   triplet_counts[n_bins][n_bins] = sum_i n_b1(i) (n_b2(i) - delta_b1b2)  (if counts given).
 * Outputs are overwritten (not accumulated).  cfg->precision selects the Gram
 * arithmetic. */
int tpcf_couple_multipoles(const float *alm, const float *prim_w, const int32_t *counts, int64_t n_prim,
                           const tpcf_config *cfg, const double *diag, const double *wsp,
                           double *nnn, int64_t *triplet_counts, void *stream);

/* The paper has no counterpart to this entry point: it exists for callers that
 * must not allocate GPU memory while they run (an application whose device
 * memory is fully reserved by its own pool, a process that may not grow its
 * footprint after start-up, or code running where calls into the CUDA
 * allocator are not allowed).  Same arguments, results and output layout as
 * tpcf_couple_multipoles with cfg->precision = TPCF_PREC_FP32, but its scratch
 * (the FP64 Gram blocks, a tile table, the triplet-count accumulator and the
 * j = k coefficient tables) lives in one fixed block of device memory that the
 * library declares, about 560 KiB held by every GPU that loads the library
 * until the process exits; it makes no allocation of any kind on the device.
 * Limit: the packed Gram blocks, sum over m of (n_bins (l_max - m + 1))^2, must
 * fit in 65,536 doubles (l_max <= 4 with up to 32 bins; l_max = 6 with up to 21
 * bins); larger requests return TPCF_ERR_ARG.  The first call on each device
 * sets the block up with a synchronous copy, so make it before any stream
 * capture; the set-up belongs to the device's CUDA context, and the first call
 * after a cudaDeviceReset repeats it.  All calls on a device share the block (the parts that must start
 * at zero are cleared by each call): calls whose work overlaps on the GPU race
 * and must be serialised by the caller. */
int tpcf_couple_multipoles_static(const float *alm, const float *prim_w, const int32_t *counts, int64_t n_prim,
                                  const tpcf_config *cfg, const double *diag, const double *wsp,
                                  double *nnn, int64_t *triplet_counts, void *stream);

/* Sharded form, for several ranks (one GPU each) sharing one catalogue.  The
 * estimator is a sum over primaries (Sec. 4.2: the average over positions x of
 * the local products of Eq. measured_mult), so a rank can compute the part of
 * every sum that its primaries contribute; the parts are added over the ranks
 * (one sum reduction, e.g. an NCCL all-reduce) and then finished.
 *
 * tpcf_partial_sizes: the lengths of one rank's partial results: n_double
 * doubles (NNN^m [m][l1][l2][b1][b2], the 2PCF sums, the randoms' l = 0
 * coupling and 2PCF sums) and n_int64 counts (pair counts, triplet counts, the
 * randoms' triplet and pair counts).
 *
 * tpcf_estimate_3pcf_partial: one rank's partials (dev part_f[n_double],
 * dev part_i[n_int64], overwritten).
 *   d_xyz/d_w (nd), r_xyz/r_w (nr): the data and random points within r_max of
 *     any of this rank's primaries (its secondaries, primaries included);
 *     nr = nrp = 0: periodic analytic randoms;
 *   dp_xyz/dp_w (ndp), rp_xyz/rp_w (nrp): this rank's primaries; every primary of
 *     the catalogue belongs to exactly one rank;
 *   w_d_total, w_r_total: the weight totals of the whole catalogue (they set the
 *     periodic offset and the D - R weights -(W_D / W_R) w of the randoms);
 *   weighted_randoms: nonzero if any random weight of the catalogue is not 1
 *     (RRR_00^0 then comes from the randoms' l = 0 coupling, else from integer
 *     random triplet counts); the same on every rank.
 *   Weights NULL: unit weights.  Arrays are device arrays, layout as in
 *   tpcf_estimate_3pcf.  Synchronises the stream before returning.
 *
 * tpcf_estimate_3pcf_finish: from the partials summed over every rank, the
 * estimate: dev zeta[n_mult][n_bins][n_bins] (required), and, if not NULL, dev
 * nnn, rrr, pair_counts, triplet_counts and xi as tpcf_estimate_3pcf_xi gives
 * them.  explicit_randoms: 0 for periodic analytic randoms.  Synchronises the
 * stream before returning.
 * Errors: TPCF_ERR_ARG for missing buffers or totals, analytic randoms in an open
 * volume, or a bad configuration. */
int tpcf_partial_sizes(const tpcf_config *cfg, int64_t *n_double, int64_t *n_int64);
int tpcf_estimate_3pcf_partial(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                               const uint32_t *r_xyz, const float *r_w, int64_t nr, const uint32_t *dp_xyz,
                               const float *dp_w, int64_t ndp, const uint32_t *rp_xyz, const float *rp_w, int64_t nrp,
                               double w_d_total, double w_r_total, int32_t weighted_randoms, double *part_f,
                               int64_t *part_i, void *stream);
int tpcf_estimate_3pcf_finish(const tpcf_config *cfg, double w_d_total, double w_r_total, int32_t explicit_randoms,
                              int32_t weighted_randoms, const double *part_f, const int64_t *part_i, double *zeta,
                              double *nnn, double *rrr, int64_t *pair_counts, int64_t *triplet_counts, double *xi,
                              void *stream);

/* TripoSH projection (Eq. slep2sugy) of dev nnn (layout as above) divided bin
 * by bin by dev rrr[n_bins][n_bins]; writes dev zeta[n_mult][n_bins][n_bins]. */
int tpcf_project(const tpcf_config *cfg, const double *nnn, const double *rrr, double *zeta, void *stream);

/* Full estimator, Eq. ssest with Eq. slep2sugy.
 *   Periodic box with analytic randoms: r_xyz = NULL, nr = 0 (cfg->periodic = 1).
 *   Explicit randoms (any geometry): the neighbour field is D - (W_D/W_R) R for
 *   primaries and secondaries, and RRR_00^0 comes from the randoms alone.
 * Inputs dev d_xyz[nd][3], d_w[nd] (NULL: unit), r_xyz[nr][3], r_w[nr] (NULL: unit).
 * Outputs dev: zeta[n_mult][n_bins][n_bins] (required), and optionally
 *   nnn (as tpcf_couple_multipoles), rrr[n_bins][n_bins], pair_counts[n_bins]
 *   (pairs of the neighbour field), triplet_counts[n_bins][n_bins].
 * RRR_00^0 with explicit randoms: with unit random weights (r_w NULL or all
 * ones, checked on the device with one 4-byte read back) it is
 * (W_D/W_R)^3 T_RR / (4 pi) from the integer random triplet counts T_RR (a
 * lean count-only pass); otherwise it is (W_D/W_R)^3 times the l = 0 coupling
 * of the randoms with their own weights (one l = 0 harmonic pass). */
int tpcf_estimate_3pcf(const tpcf_config *cfg,
                       const uint32_t *d_xyz, const float *d_w, int64_t nd,
                       const uint32_t *r_xyz, const float *r_w, int64_t nr,
                       double *zeta, double *nnn, double *rrr,
                       int64_t *pair_counts, int64_t *triplet_counts, void *stream);

/* tpcf_estimate_3pcf plus the even anisotropic 2PCF multipoles of the same
 * field and radial bins (Eq. xi_meas_leg with the natural estimator of
 * Eq. xi_natest, which the D - R field turns into (DD - 2DR + RR) / RR):
 *   xi[e][b] = (2l + 1) sum_{pairs in b} w_i w_j P_l(mu_ij) / RR_b,  l = 2e,
 *   e = 0 .. l_max / 2, mu the cosine of the pair separation to the z axis
 *   (the fixed line of sight), every pair's P_l taken exactly (the limit of
 *   vanishing mu bins).  RR_b is W_D (W_D - 1) V_b / L^3 with analytic randoms,
 *   else (W_D/W_R)^2 times the weighted ordered random pair sum of bin b.
 *   The l = 0 term carries the -1 of Eq. xi_natest through the random
 *   subtraction.  dev xi[l_max/2 + 1][n_bins] (NULL: as tpcf_estimate_3pcf).
 *   The sums come from the m = 0 harmonics of the pair stage: no extra pass. */
int tpcf_estimate_3pcf_xi(const tpcf_config *cfg,
                          const uint32_t *d_xyz, const float *d_w, int64_t nd,
                          const uint32_t *r_xyz, const float *r_w, int64_t nr,
                          double *zeta, double *nnn, double *rrr,
                          int64_t *pair_counts, int64_t *triplet_counts, double *xi, void *stream);

/* The estimator with the full anisotropic edge correction (explicit randoms,
 * nr >= 1; any geometry).  Instead of dividing NNN^m bin-wise by RRR_00^0 it
 * computes every RRR^m_{l1 l2} of the randoms (weights (W_D/W_R) r_w, the
 * same pair and coupling kernels at l_max) and, for every bin pair, solves
 * N = zeta R, the product of functions of (r_hat_1, r_hat_2) about the fixed
 * line of sight expanded in Y_l1^m(r_hat_1) Y_l2^m*(r_hat_2) (Eq. zeta_meas),
 * whose coefficients couple through one Gaunt integral per direction:
 *   Re NNN^m_{l1 l2} = sum 4 pi RRR^{m - m'}_{l1'' l2''} G(l1' m', l1'' m-m'; l1)
 *                      G(l2' m', l2'' m-m'; l2) zeta_hat^m'_{l1' l2'},
 * truncated at l_max, on the real coefficients with l1 + l2 even (the ones
 * the L-even multipoles use; the imaginary and odd-parity parts of RRR, zero
 * for a mirror-symmetric random catalogue, are dropped).  zeta_hat is then
 * projected with Eq. slep2sugy.  For isotropic randoms it equals the bin-wise
 * tpcf_estimate_3pcf.  Outputs dev: zeta[n_mult][n_bins][n_bins] (required),
 * nnn (the D - R field's, as tpcf_couple_multipoles), rrr_multipoles
 * [l_max+1]^3[n_bins][n_bins] (RRR^m_{l1 l2} in the nnn layout) and
 * xi[l_max/2 + 1][n_bins] (as tpcf_estimate_3pcf_xi), each optional.  A
 * singular system (no random triangles in a bin pair) gives NaN there and
 * TPCF_ERR_DATA from tpcf_stream_status. */
int tpcf_estimate_3pcf_full_edge(const tpcf_config *cfg,
                                 const uint32_t *d_xyz, const float *d_w, int64_t nd,
                                 const uint32_t *r_xyz, const float *r_w, int64_t nr,
                                 double *zeta, double *nnn, double *rrr_multipoles, double *xi, void *stream);

/* As tpcf_estimate_3pcf, but every pointer is HOST memory (pinned memory gives
 * the fastest copies).  Copies in, runs, copies out, and synchronises the
 * stream before returning. */
int tpcf_estimate_3pcf_host(const tpcf_config *cfg,
                            const uint32_t *d_xyz, const float *d_w, int64_t nd,
                            const uint32_t *r_xyz, const float *r_w, int64_t nr,
                            double *zeta, double *nnn, double *rrr,
                            int64_t *pair_counts, int64_t *triplet_counts, void *stream);

/* ----------------------------------------------------------------- batches
 * Many periodic catalogues of uneven sizes (mocks for a covariance matrix, the
 * use Sec. 4.3 motivates), each estimated with analytic randoms.  The points of
 * all mocks are concatenated: mock k is points [offsets[k], offsets[k+1]).  The
 * pair stage of a whole group of mocks is one persistent launch whose tiles may
 * come from any mock (each tile holds primaries of one mock only: up to
 * cfg->tile_primaries of them, or, for 0, the single-catalogue rule of about
 * 3000 pairs per tile at the mean mock density), and so is the coupling (every
 * mock's Gram in one launch whose slices never cross a mock); all mocks fit one
 * group unless the per-point buffers would take more than half of the free
 * device memory. */
typedef struct tpcf_batch_s *tpcf_batch;

/* Plans a batch: host offsets[n_mocks + 1] (offsets[0] = 0, non-decreasing,
 * total < 2^28), cfg->periodic = 1.  group_points > 0 caps the points of one
 * group (0: the memory rule above); a single mock larger than the cap is an
 * error.  Allocates every buffer and uploads every table now, so
 * tpcf_batch_run only enqueues device work. */
int tpcf_batch_create(const tpcf_config *cfg, const int64_t *offsets, int32_t n_mocks, int64_t group_points,
                      tpcf_batch *out);

/* Number of groups (persistent pair-stage launches per run) and cells per axis. */
int tpcf_batch_info(tpcf_batch batch, int32_t *n_groups, int32_t *cells_per_axis);

/* Runs the batch: dev xyz[total][3], dev w[total] (NULL: unit weights);
 * writes dev zeta[n_mocks][n_mult][n_bins][n_bins] and, if not NULL, dev
 * triplet_counts[n_mocks][n_bins][n_bins].  Makes no host synchronisation and no
 * host-to-device copy, so it can be captured into a CUDA graph (its scratch
 * comes from stream-ordered allocations, which capture as graph memory nodes). */
int tpcf_batch_run(tpcf_batch batch, const uint32_t *xyz, const float *w, double *zeta, int64_t *triplet_counts,
                   void *stream);

/* Same work as tpcf_batch_run, as one CUDA graph launch.  The first call with a
 * given set of buffers runs the batch eagerly on `stream` and captures the same
 * work (on a private stream, thread-local capture mode) into a graph kept in the
 * batch; later calls with the same four pointers launch that graph on `stream`.
 * New pointers replace the graph.  Calls on one batch must not overlap. */
int tpcf_batch_run_graph(tpcf_batch batch, const uint32_t *xyz, const float *w, double *zeta,
                         int64_t *triplet_counts, void *stream);

/* Releases a batch (synchronises the device first). NULL is accepted. */
int tpcf_batch_destroy(tpcf_batch batch);

/* Status of every mock in the batch's last run (host status[n_mocks]; synchronises
 * the stream): TPCF_OK, TPCF_ERR_DATA (a non-finite weight in that mock: its own
 * multipoles are not finite, the other mocks are unaffected) or TPCF_ERR_ARG
 * (fewer than two points: no pair to estimate from). */
int tpcf_batch_status(tpcf_batch batch, int32_t *status, void *stream);

/* create + run + tpcf_stream_status + destroy; status_per_mock (host
 * [n_mocks], or NULL) as tpcf_batch_status gives it.  A bad mock does not fail
 * the call: only whole-batch failures are returned. */
int tpcf_estimate_3pcf_batched(const tpcf_config *cfg, const uint32_t *xyz, const float *w, const int64_t *offsets,
                               int32_t n_mocks, double *zeta, int64_t *triplet_counts, int32_t *status_per_mock,
                               void *stream);

/* Chooses cell_div (2..6), tile_primaries (1, 2, 4) and chunk (12288, 15360,
 * 24576) for a catalogue like this one by timing the pair stage on a strided
 * sample of at most 32768 of its primaries (dev xyz[n][3], dev w[n] or NULL) for
 * every valid combination (best of three runs after a warm-up run); *tuned =
 * *cfg with the fastest choice.  A nonzero
 * cfg->tile_primaries is kept fixed.  Synchronises the stream. */
int tpcf_autotune(const tpcf_config *cfg, const uint32_t *xyz, const float *w, int64_t n, void *stream,
                  tpcf_config *tuned);

/* -------------------------------------------------------------- covariance
 * Covariant errors from mocks (Sec. 4.3).  The data vector of mock k is
 * d_i^k = src[k * stride + idx[i]], i = 0 .. n_dv-1 (dev idx, or NULL for
 * d_i^k = src[k * stride + i]); with the batch's zeta array
 * [n_mocks][n_mult][n_bins][n_bins], stride = n_mult n_bins^2 and idx from
 * tpcf_data_vector_index select multipoles and triangles in place.
 * Writes dev mean[n_dv] and dev cov[n_dv][n_dv] (row-major, symmetric):
 *   cov_ij = sum_k (d_i^k - mean_i)(d_j^k - mean_j) / (n_mocks - 1)
 * (Eq. covariance), in FP64.  n_mocks >= 2, n_dv <= 2^20.  An idx entry
 * outside [0, stride) is reported as TPCF_ERR_DATA by tpcf_stream_status and
 * turns its row and column into NaN. */
int tpcf_covariance(const double *src, int64_t n_mocks, int64_t stride, const int64_t *idx, int64_t n_dv,
                    double *mean, double *cov, void *stream);

/* Host arithmetic for a covariance from n_mocks mocks of an n_dv-long data
 * vector and n_params fitted parameters: *hartlap = (n_mocks - n_dv - 2) /
 * (n_mocks - 1), the factor on the inverse covariance (Eq. Hartlap), and *m1,
 * the factor on the parameters' variance (Eqs. Perc1, Perc).  Either output
 * may be NULL.  Needs n_mocks > n_dv + 4 (TPCF_ERR_ARG otherwise). */
int tpcf_covariance_factors(int64_t n_mocks, int64_t n_dv, int64_t n_params, double *hartlap, double *m1);

/* Host: flat indices into a zeta array [n_mult][n_bins][n_bins] of cfg (the
 * order of tpcf_multipole_index) for the n_sel multipoles host
 * l1l2L[n_sel][3], in that order, each over the triangles b1 <= b2 with
 * b2 - b1 >= eta (|r1 - r2| >= eta dr, the selection of Sec. 4.3), b1 then b2
 * ascending.  *n_out = entries needed; host idx (cap entries, may be NULL to
 * query the count).  A multipole cfg does not measure is TPCF_ERR_ARG. */
int tpcf_data_vector_index(const tpcf_config *cfg, const int32_t *l1l2L, int32_t n_sel, int32_t eta,
                           int64_t *idx, int64_t cap, int64_t *n_out);

/* Diagnostic (no counterpart in the paper): compares the pair stage's
 * reciprocal square root (the hardware estimate refined by one Newton-Raphson
 * step) with CUDA's correctly rounded __frsqrt_rn on n log-uniform inputs in
 * [1, 2^62) drawn from seed.  Host stats[5]: max |difference| in units in the
 * last place, mean relative difference, mean of x y^2 - 1 for the pair stage's
 * y, the same for the correctly rounded y, fraction of inputs that differ.
 * Synchronises the stream. */
int tpcf_check_rsqrt(int64_t n, uint64_t seed, double *stats, void *stream);

/* Measured FP32 FMA throughput of this GPU, the denominator beside the nominal
 * 2 x 128 x SMs x clock peak of the pair stage's roofline: host tflops[0] with
 * scalar FMAs, tflops[1] with paired FFMA2 instructions (8 CTAs of 256 threads
 * per SM, 8 independent chains per thread, best of three timed runs after a
 * warm-up).  Synchronises the stream. */
int tpcf_measure_fp32_peak(double *tflops, void *stream);

/* Synchronises the stream and reports any latched device-side error
 * (TPCF_ERR_DATA, TPCF_ERR_TIMEOUT) or CUDA error; clears the latch. */
int tpcf_stream_status(void *stream);

/* Memory housekeeping (the paper has no counterpart).  Device scratch and grids
 * come, outside stream capture, from a memory pool that the library owns on each
 * device; freed blocks stay cached there for the next call instead of going back
 * to the driver at every synchronisation (for the clustered D - R field that is
 * the 3.2 GB of per-primary harmonic sums of every estimate).  This call hands
 * the cached blocks of the current device back to the driver: blocks whose
 * stream-ordered release has completed (synchronise the streams that used the
 * library first to return all of them).  Blocks still in use, and grids not yet
 * destroyed, are kept.  Host only; no stream work; TPCF_OK when the device has no
 * pool yet. */
int tpcf_trim_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* TPCF_H */
