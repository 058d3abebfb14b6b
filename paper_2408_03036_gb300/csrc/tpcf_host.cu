// Host side of libtpcf: argument checks, exact bin edges, constant tables
// (harmonic polynomials, 3j / Gaunt coefficients, projection weights), scratch
// management and the C-ABI entry points declared in include/tpcf.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <atomic>

#include <cuda_runtime.h>

#include "internal.h"
#include "k_pairs.cuh"

namespace tpcf {
cudaError_t launch_pairs_l0(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
cudaError_t launch_pairs_l1(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
cudaError_t launch_pairs_l2(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
cudaError_t launch_pairs_l3(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
cudaError_t launch_pairs_l4(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
cudaError_t launch_pairs_l5(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
cudaError_t launch_pairs_l6(bool, const PairParams &, const HarmTables &, int, int, size_t, cudaStream_t);
size_t pairs_smem_l0(bool, int, int, int, int, int);
size_t pairs_smem_l1(bool, int, int, int, int, int);
size_t pairs_smem_l2(bool, int, int, int, int, int);
size_t pairs_smem_l3(bool, int, int, int, int, int);
size_t pairs_smem_l4(bool, int, int, int, int, int);
size_t pairs_smem_l5(bool, int, int, int, int, int);
size_t pairs_smem_l6(bool, int, int, int, int, int);
int pairs_per_sm_l0(bool, bool, int, size_t);
int pairs_per_sm_l1(bool, bool, int, size_t);
int pairs_per_sm_l2(bool, bool, int, size_t);
int pairs_per_sm_l3(bool, bool, int, size_t);
int pairs_per_sm_l4(bool, bool, int, size_t);
int pairs_per_sm_l5(bool, bool, int, size_t);
int pairs_per_sm_l6(bool, bool, int, size_t);
}  // namespace tpcf

using namespace tpcf;

namespace {
std::atomic<long long> g_launches{0};
}

void tpcf::note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
std::atomic<long long> g_wait_limit{0};
std::atomic<int> g_wait_unmet{0};
}
long long tpcf::device_wait_limit()
{
    const long long v = g_wait_limit.load(std::memory_order_relaxed);
    return v > 0 ? v : (1ll << 26);
}
int tpcf::device_wait_unmet() { return g_wait_unmet.load(std::memory_order_relaxed); }

struct tpcf_grid_s {
    GridDev g;
    cudaStream_t stream;
    int device;
};

// A planned batch of periodic catalogues (analytic randoms): device tables and
// every buffer are made at creation, so a run only enqueues kernels, copies and
// stream-ordered allocations (it can be captured in a CUDA graph).
struct tpcf_batch_s {
    tpcf_config cfg;
    int n_mocks = 0;
    std::vector<int64_t> off;            // host offsets [n_mocks + 1]
    std::vector<int> group;              // first mock of every group, then n_mocks
    int device = 0;
    int nc = 0;
    int64_t max_group_points = 0;
    int n_mult = 0;
    // device tables and buffers
    int64_t *d_off = nullptr;            // [n_mocks + 1]
    int64_t *d_goff = nullptr;           // rebased offsets per group (concatenated)
    double *d_gaunt = nullptr, *d_coef = nullptr, *d_mono = nullptr;
    int *d_mults = nullptr, *d_tiles = nullptr;
    int32_t *rec_mock = nullptr;
    float *alm = nullptr, *wprim = nullptr;
    int32_t *counts = nullptr;
    double *wsum = nullptr, *diag = nullptr, *wsp = nullptr, *G = nullptr, *nnn = nullptr, *rrr = nullptr;
    unsigned long long *pairs = nullptr, *T = nullptr;
    int *d_status = nullptr;             // [n_mocks] DEV_ERR_* of every mock's last run
    // the one-launch Gram of every group: slice boundaries (primaries from the
    // group's first) and every mock's first slice, concatenated over groups
    int64_t *d_slice_k = nullptr;
    int *d_mslice = nullptr;
    std::vector<size_t> gs_at, gm_at;    // per group: offsets into d_slice_k and d_mslice
    std::vector<int> gs_n;               // per group: slices
    int max_group_mocks = 0;
    // pair-stage tiles of up to tile_p primaries of one mock (tile_p > 1), starts
    // relative to the group's first primary, concatenated over groups
    int tile_p = 1;
    int64_t *d_tile_start = nullptr;
    std::vector<size_t> gt_at;           // per group: offset into d_tile_start
    std::vector<int64_t> gt_n;           // per group: tiles
    // graph of one run, captured for the buffers in gp
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *gp[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwo32 = 4294967296.0;
constexpr int64_t kMaxPoints = (int64_t)1 << 28;   // staged pairs carry the candidate index in 28 bits

thread_local char g_msg[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    if (e == cudaErrorMemoryAllocation) return fail(TPCF_ERR_OOM, "%s: out of device memory", where);
    return fail(TPCF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                           \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
    } while (0)

// ---------------------------------------------------------------- config

int check_config(const tpcf_config *c)
{
    if (!c) return fail(TPCF_ERR_ARG, "config is NULL");
    if (c->n_bins < 1 || c->n_bins > TPCF_MAX_BINS) return fail(TPCF_ERR_ARG, "n_bins must be 1..%d", TPCF_MAX_BINS);
    if (c->l_max < 0 || c->l_max > TPCF_MAX_LMAX) return fail(TPCF_ERR_ARG, "l_max must be 0..%d", TPCF_MAX_LMAX);
    if (!(c->box > 0.0) || !std::isfinite(c->box)) return fail(TPCF_ERR_ARG, "box must be positive");
    if (!(c->r_min > 0.0)) return fail(TPCF_ERR_ARG, "r_min must be > 0");
    if (!(c->r_max > c->r_min)) return fail(TPCF_ERR_ARG, "r_max must exceed r_min");
    if (!(2.0 * c->r_max < c->box)) return fail(TPCF_ERR_ARG, "r_max must be below box/2");
    if (c->n_L < 1 || c->n_L > 8) return fail(TPCF_ERR_ARG, "n_L must be 1..8");
    for (int i = 0; i < c->n_L; ++i)
        if (c->L[i] < 0 || c->L[i] > 2 * c->l_max || (c->L[i] & 1))
            return fail(TPCF_ERR_ARG, "L values must be even and in 0..2*l_max");
    if (c->precision < TPCF_PREC_FP32 || c->precision > TPCF_PREC_TF32X3)
        return fail(TPCF_ERR_ARG, "unknown precision");
    if (c->convention != TPCF_CONV_S_COEFF && c->convention != TPCF_CONV_PAPER_EQ)
        return fail(TPCF_ERR_ARG, "unknown convention");
    if (c->remove_self != 0 && c->remove_self != 1) return fail(TPCF_ERR_ARG, "remove_self must be 0 or 1");
    if (c->cell_div < 0 || c->cell_div > 6) return fail(TPCF_ERR_ARG, "cell_div must be 0..6");
    if (c->tile_primaries < 0 || c->tile_primaries > TPCF_MAX_TILE) return fail(TPCF_ERR_ARG, "tile_primaries must be 0..8");
    if (c->los != 0 && c->los != 1) return fail(TPCF_ERR_ARG, "los must be 0 (z) or 1 (observer)");
    if (c->los == 1)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(c->observer[k]) || std::fabs(c->observer[k]) > 1e6 * c->box)
                return fail(TPCF_ERR_ARG, "observer coordinates must be finite and within 1e6 box lengths");
    if (c->chunk != 0 && (c->chunk < 512 || (c->chunk % 256) != 0 || c->chunk > 49152))
        return fail(TPCF_ERR_ARG, "chunk must be 0 or a multiple of 256 in 512..49152");
    return TPCF_OK;
}

// Exact ceil(s^2) of a finite double s >= 0 from its IEEE-754 fields.
unsigned long long ceil_sq(double s)
{
    if (!(s > 0.0)) return 0ull;
    uint64_t bits;
    std::memcpy(&bits, &s, 8);
    const int ex = (int)((bits >> 52) & 0x7ff);
    uint64_t mant = bits & ((1ull << 52) - 1);
    int e2;
    if (ex == 0) { e2 = -1074; } else { mant |= (1ull << 52); e2 = ex - 1075; }
    const unsigned __int128 sq = (unsigned __int128)mant * mant;   // s^2 = sq * 2^(2 e2)
    const int sh = -2 * e2;
    if (sh <= 0) return (unsigned long long)(sq << (-sh));
    if (sh >= 128) return 1ull;
    const unsigned __int128 q = sq >> sh;
    const unsigned __int128 rem = sq - (q << sh);
    return (unsigned long long)(q + (rem != 0 ? 1 : 0));
}

void edge_tables(const tpcf_config *c, unsigned long long *E, double *r)
{
    for (int b = 0; b <= c->n_bins; ++b) {
        const double rb = c->r_min + ((c->r_max - c->r_min) * (double)b) / (double)c->n_bins;
        const double sb = (rb * kTwo32) / c->box;
        E[b] = ceil_sq(sb);
        if (r) r[b] = rb;
    }
}

// ------------------------------------------------------------- 3j symbols

double factd(int n)
{
    static double tab[64];
    static bool init = false;
    if (!init) {
        tab[0] = 1.0;
        for (int i = 1; i < 64; ++i) tab[i] = tab[i - 1] * (double)i;
        init = true;
    }
    return (n >= 0 && n < 64) ? tab[n] : NAN;
}

// Wigner 3j symbol for integer arguments (Racah's closed form).
double w3j(int a, int b, int c, int ma, int mb, int mc)
{
    if (ma + mb + mc != 0 || c < std::abs(a - b) || c > a + b) return 0.0;
    if (std::abs(ma) > a || std::abs(mb) > b || std::abs(mc) > c) return 0.0;
    const double delta = factd(a + b - c) * factd(a - b + c) * factd(b + c - a) / factd(a + b + c + 1);
    const double norm = std::sqrt(delta * factd(a + ma) * factd(a - ma) * factd(b + mb) * factd(b - mb)
                                  * factd(c + mc) * factd(c - mc));
    int tlo = std::max(0, std::max(b - c - ma, a - c + mb));
    int thi = std::min(a + b - c, std::min(a - ma, b + mb));
    double sum = 0.0;
    for (int t = tlo; t <= thi; ++t) {
        const double d = factd(t) * factd(c - b + t + ma) * factd(c - a + t - mb) * factd(a + b - c - t)
                       * factd(a - t - ma) * factd(b - t + mb);
        sum += ((t % 2) ? -1.0 : 1.0) / d;
    }
    const int ph = a - b - mc;
    return (((ph % 2) + 2) % 2 ? -1.0 : 1.0) * norm * sum;
}

double nlm(int l, int m)
{
    return std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factd(l - m) / factd(l + m));
}

// Polynomials with double coefficients (index = power of the variable).
using Poly = std::vector<double>;

Poly pmul(const Poly &a, const Poly &b)
{
    Poly r(a.size() + b.size() - 1, 0.0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
    return r;
}

// V_l^m(z) in powers of z: V_m = 1, V_{m+1} = (2m+1) z,
// V_l = (2l-1) z V_{l-1} - (l+m-1)(l-m-1) V_{l-2}; integer coefficients, exact in double.
Poly v_poly(int l, int m)
{
    Poly vm2{1.0}, vm1{0.0, (double)(2 * m + 1)};
    if (l == m) return vm2;
    if (l == m + 1) return vm1;
    Poly v;
    for (int k = m + 2; k <= l; ++k) {
        v.assign(k - m + 1, 0.0);
        for (size_t i = 0; i < vm1.size(); ++i) v[i + 1] += (2.0 * k - 1.0) * vm1[i];
        const double c = (double)((k + m - 1) * (k - m - 1));
        for (size_t i = 0; i < vm2.size(); ++i) v[i] -= c * vm2[i];
        vm2 = vm1;
        vm1 = v;
    }
    return vm1;
}

// Even polynomial in z -> polynomial in y = z^2.
Poly even_to_y(const Poly &p)
{
    Poly r((p.size() + 1) / 2, 0.0);
    for (size_t i = 0; i < p.size(); i += 2) r[i / 2] = p[i];
    return r;
}

// Y_l^m = K_lm V_l^m(z) (x + i y)^m
double k_scale(int l, int m)
{
    double dfact = 1.0;
    for (int i = 1; i <= 2 * m - 1; i += 2) dfact *= (double)i;
    return ((m % 2) ? -1.0 : 1.0) * nlm(l, m) * dfact / factd(l - m);
}

// f_j(y) of the device's self accumulators: f_0 = 1, f_j = V_{2j}^0.
Poly f_poly(int j) { return j == 0 ? Poly{1.0} : even_to_y(v_poly(2 * j, 0)); }

// g_j with V_l1^m V_l2^m (1 - y)^m = sum_j g_j f_j(y)   (l1 + l2 even), exactly
// (integer polynomials; the solve is a triangular back-substitution in double).
std::vector<double> self_coefs(int lmax, int l1, int l2, int m)
{
    Poly t = even_to_y(pmul(v_poly(l1, m), v_poly(l2, m)));
    for (int k = 0; k < m; ++k) t = pmul(t, Poly{1.0, -1.0});
    std::vector<double> g(lmax + 1, 0.0);
    for (int j = (int)t.size() - 1; j >= 0; --j) {
        if (j > lmax) continue;   // degree <= max(l1, l2) <= lmax
        const Poly f = f_poly(j);
        const double c = t[j] / f[j];
        g[j] = c;
        for (int k = 0; k <= j; ++k) t[k] -= c * f[k];
    }
    return g;
}

HarmTables make_tables(int lmax)
{
    HarmTables h;
    std::memset(&h, 0, sizeof(h));
    for (int l = 0; l <= TPCF_MAX_LMAX; ++l)
        for (int m = 0; m <= l; ++m) {
            const double k = k_scale(l, m);
            h.K[l][m] = k;
            h.k2[l * (l + 1) / 2 + m] = (float)(k * k);
            const float hi = (float)k, lo = (float)(k - (double)hi);
            for (int part = 0; part < (m ? 2 : 1); ++part) {
                const int idx = l * l + (m ? 2 * m - 1 + part : 0);
                h.kout[idx][0] = hi;
                h.kout[idx][1] = lo;
            }
        }
    int jd = 0;
    for (int l = 0; l <= lmax; ++l)
        for (int m = 0; m <= l; ++m, ++jd) {
            const std::vector<double> g = self_coefs(lmax, l, l, m);
            for (int j = 0; j <= lmax; ++j) {
                const float hi = (float)g[j];
                h.gd_hi[jd][j] = hi;
                h.gd_lo[jd][j] = (float)(g[j] - (double)hi);
            }
        }
    return h;
}

void multipole_list(const tpcf_config *c, std::vector<int> &out)
{
    out.clear();
    for (int i = 0; i < c->n_L; ++i) {
        const int L = c->L[i];
        for (int l1 = 0; l1 <= c->l_max; ++l1)
            for (int l2 = 0; l2 <= c->l_max; ++l2)
                if (std::abs(l1 - l2) <= L && L <= l1 + l2 && ((l1 + l2 + L) % 2) == 0) {
                    out.push_back(l1); out.push_back(l2); out.push_back(L);
                }
    }
}

// ------------------------------------------------------------ device state

struct DevState {
    int *err = nullptr;
    int sms = 0;
    // device copies of the harmonic tables, one per l_max (read by the pair
    // stage's tile epilogue with lane-dependent indices)
    HarmTables *harm[TPCF_MAX_LMAX + 1] = {};
};
std::mutex g_mu;
DevState g_dev[64];

// Per-device scratch pools (scratch_malloc), each tagged with the context it was
// made in: cudaDeviceReset ends the context and its pools with it.
struct ScratchPool {
    cudaMemPool_t pool = nullptr;
    unsigned long long ctx = 0;
};
std::mutex g_pool_mu;
ScratchPool g_pool[64];

int dev_state(DevState **out)
{
    int d = 0;
    CK(cudaGetDevice(&d));
    if (d < 0 || d >= 64) return fail(TPCF_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &s = g_dev[d];
    if (!s.err) {
        CK(cudaMalloc((void **)&s.err, sizeof(int)));
        CK(cudaMemset(s.err, 0, sizeof(int)));
        CK(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, d));
    }
    *out = &s;
    return TPCF_OK;
}

// ------------------------------------------------------------ scheduling

struct Plan {
    int s;      // cells scanned on each side
    int nc;     // cells per axis
    int P;      // primaries per tile
    int chunk;
};

Plan make_plan(const tpcf_config *c, int64_t n_sec, int64_t n_prim_hint)
{
    Plan p;
    const double nbar = (double)(n_sec > 0 ? n_sec : 1) / (c->box * c->box * c->box);
    int s = c->cell_div;
    if (s == 0) {
        // about 24 points per cell, cells no smaller than r_max / 6
        const double h_want = std::cbrt(24.0 / nbar);
        s = (int)std::floor(c->r_max / h_want);
        s = std::max(1, std::min(6, s));
    }
    for (;;) {
        int nc = (int)std::floor((double)s * c->box / c->r_max);
        nc = std::min(nc, 256);
        const int need = c->periodic ? 2 * s + 1 : 2 * s + 3;
        if (nc >= need || s == 1) { p.s = s; p.nc = std::max(nc, 1); break; }
        --s;
    }
    const double vol = 4.0 / 3.0 * kPi * (c->r_max * c->r_max * c->r_max - c->r_min * c->r_min * c->r_min);
    const double pairs = nbar * vol;
    int P = c->tile_primaries;
    if (P == 0) {
        P = (int)std::lround(3000.0 / std::max(pairs, 1.0));
        P = std::max(1, std::min(TPCF_MAX_TILE, P));
    }
    // the chunk's lane groups need P * n_bins <= 128 keys (half the CTA's lanes)
    P = std::min(P, std::max(1, 128 / c->n_bins));
    p.P = P;
    // queue entries (4 bytes each) per CTA: three CTAs per SM up to l_max 4, one above
    p.chunk = c->chunk ? c->chunk : (c->l_max <= 4 ? 15360 : 49152);
    (void)n_prim_hint;
    return p;
}

size_t pair_smem(int lmax, bool counts, const Plan &pl, int nb)
{
    switch (counts ? 0 : lmax) {
    case 0: return pairs_smem_l0(counts, pl.P, nb, pl.s, pl.chunk, 256);
    case 1: return pairs_smem_l1(counts, pl.P, nb, pl.s, pl.chunk, 256);
    case 2: return pairs_smem_l2(counts, pl.P, nb, pl.s, pl.chunk, 256);
    case 3: return pairs_smem_l3(counts, pl.P, nb, pl.s, pl.chunk, 256);
    case 4: return pairs_smem_l4(counts, pl.P, nb, pl.s, pl.chunk, 256);
    case 5: return pairs_smem_l5(counts, pl.P, nb, pl.s, pl.chunk, 256);
    default: return pairs_smem_l6(counts, pl.P, nb, pl.s, pl.chunk, 256);
    }
}

int pair_per_sm(int lmax, bool counts, bool vlos, size_t smem)
{
    switch (counts ? 0 : lmax) {
    case 0: return pairs_per_sm_l0(counts, vlos, 256, smem);
    case 1: return pairs_per_sm_l1(counts, vlos, 256, smem);
    case 2: return pairs_per_sm_l2(counts, vlos, 256, smem);
    case 3: return pairs_per_sm_l3(counts, vlos, 256, smem);
    case 4: return pairs_per_sm_l4(counts, vlos, 256, smem);
    case 5: return pairs_per_sm_l5(counts, vlos, 256, smem);
    default: return pairs_per_sm_l6(counts, vlos, 256, smem);
    }
}

cudaError_t pair_launch(int lmax, bool counts, const PairParams &p, const HarmTables &h, int grid, size_t smem,
                        cudaStream_t st)
{
    switch (counts ? 0 : lmax) {
    case 0: return launch_pairs_l0(counts, p, h, grid, 256, smem, st);
    case 1: return launch_pairs_l1(counts, p, h, grid, 256, smem, st);
    case 2: return launch_pairs_l2(counts, p, h, grid, 256, smem, st);
    case 3: return launch_pairs_l3(counts, p, h, grid, 256, smem, st);
    case 4: return launch_pairs_l4(counts, p, h, grid, 256, smem, st);
    case 5: return launch_pairs_l5(counts, p, h, grid, 256, smem, st);
    default: return launch_pairs_l6(counts, p, h, grid, 256, smem, st);
    }
}

}  // namespace

// Unique id of the current CUDA context (the driver's cuCtxGetId, reached through
// the runtime's entry-point query so the library does not link libcuda); 0 if
// unavailable.  cudaDeviceReset replaces the primary context, and its id.
unsigned long long tpcf::context_id()
{
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

cudaError_t tpcf::scratch_malloc(void **p, size_t bytes, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaMallocAsync(p, bytes, st);
    int d = 0;
    if ((e = cudaGetDevice(&d)) != cudaSuccess) return e;
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool = nullptr;
    {
        const unsigned long long ctx = context_id();
        std::lock_guard<std::mutex> lk(g_pool_mu);
        ScratchPool &sp = g_pool[d];
        if (!sp.pool || sp.ctx != ctx) {
            // a pool left from an earlier context went with that context
            cudaMemPoolProps props;
            std::memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = d;
            cudaMemPool_t np = nullptr;
            if ((e = cudaMemPoolCreate(&np, &props)) != cudaSuccess) return e;
            uint64_t keep = ~0ull;
            if ((e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
                cudaMemPoolDestroy(np);
                return e;
            }
            sp.pool = np;
            sp.ctx = ctx;
        }
        pool = sp.pool;
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

namespace {

// Runs the pair stage over `n_prim` primary records against grid g.
template <class T>
int dalloc(T **p, size_t n, cudaStream_t st, bool zero)
{
    CK(scratch_malloc((void **)p, (n ? n : 1) * sizeof(T), st));
    if (zero) CK(cudaMemsetAsync(*p, 0, (n ? n : 1) * sizeof(T), st));
    return TPCF_OK;
}

// Device buffers and grids a host function allocates for itself, released in
// stream order on every return path (success or error).
class Scratch {
public:
    explicit Scratch(cudaStream_t st) : st_(st) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch()
    {
        for (void *q : ptrs_) cudaFreeAsync(q, st_);
        for (GridDev *g : grids_) free_grid_dev(*g, st_);
    }
    template <class T>
    int alloc(T **p, size_t n, bool zero)
    {
        const int rc = dalloc(p, n, st_, zero);
        keep(*p);
        return rc;
    }
    void keep(void *q)
    {
        if (q) ptrs_.push_back(q);
    }
    void own(GridDev &g) { grids_.push_back(&g); }

private:
    cudaStream_t st_;
    std::vector<void *> ptrs_;
    std::vector<GridDev *> grids_;
};

struct BatchInfo {
    const int *prim_mock;       // mock of every primary
    int64_t ncell_mock;         // cells per mock
    const double *mono_w_mock;  // W per mock
    int *mock_status;           // per-mock device status (the group's first mock at index 0)
    int P = 1;                  // primaries per tile of tile_start (1: no table)
    const int64_t *tile_start = nullptr;   // [n_tiles + 1] tiles within single mocks, or null
    int64_t n_tiles = 0;
};

// Random-random pair counts taken during a D - R pass (PairParams::counts_r):
// per primary and bin, and their sum per bin (either may be null).
struct RRCounts {
    int32_t *counts;
    unsigned long long *pairs;
};

int run_pairs(const tpcf_config *c, const GridDev &g, const int4 *prim, int64_t n_prim, bool counts_only,
              double mono_w, const double *mono_w_dev, bool use_mono, float *alm, int32_t *counts, double *diag,
              double *wsp, unsigned long long *pair_counts, cudaStream_t st, const BatchInfo *bi = nullptr,
              const RRCounts *rrc = nullptr)
{
    DevState *ds;
    int rc = dev_state(&ds);
    if (rc) return rc;
    if (n_prim <= 0) return TPCF_OK;
    Plan pl = make_plan(c, g.n, n_prim);
    // the grid's cell count was fixed when it was built; recover s for it
    pl.nc = g.nc;
    int s = std::max(1, (int)std::ceil(c->r_max * g.nc / c->box - 1e-9));
    pl.s = s;
    if (c->periodic && 2 * s + 1 > g.nc) return fail(TPCF_ERR_ARG, "grid too coarse for r_max (periodic)");
    if (!c->periodic && 2 * s + 2 >= g.nc) return fail(TPCF_ERR_ARG, "grid too coarse for r_max (open volume)");

    PairParams p;
    std::memset(&p, 0, sizeof(p));
    p.rec = g.rec;
    p.cell_start = g.cell_start;
    p.nc = g.nc;
    p.s = pl.s;
    p.periodic = c->periodic;
    p.prim = prim;
    p.n_prim = n_prim;
    p.nb = c->n_bins;
    p.P = pl.P;
    double r[TPCF_MAX_BINS + 1];
    edge_tables(c, p.E, r);
    for (int b = 0; b <= c->n_bins; ++b) p.Ef[b] = (float)(double)p.E[b];
    const double u = kTwo32 / c->box;   // units per length
    p.rmin_u = (float)(c->r_min * u);
    p.inv_dr_u = (float)((double)c->n_bins / ((c->r_max - c->r_min) * u));
    {
        // float bin coordinate t = (r - r_min) / dr from the float r^2: relative error of r
        // below 5.1e-7 (r^2 from rounded separations 3e-7, rsqrt 2.4e-7, products), of the
        // constants below 6e-8; a margin of four times the resulting bound
        const double dr = (c->r_max - c->r_min) / c->n_bins;
        p.t_off = (float)(-(double)p.rmin_u * (double)p.inv_dr_u);
        p.tdelta = (float)(4.0 * (((c->r_max + dr) / dr) * 5.1e-7 + (c->r_min / dr) * 6e-8
                                  + (c->n_bins + 1.0) * 6e-8));
    }
    p.rmax_trim = (float)(c->r_max * u * (1.0 + 1e-5) + 4096.0);
    p.h_u = (float)(kTwo32 / (double)g.nc);
    for (int b = 0; b < c->n_bins; ++b) {
        const double vb = 4.0 * kPi / 3.0 * (r[b + 1] * r[b + 1] * r[b + 1] - r[b] * r[b] * r[b]);
        p.mono_coef[b] = vb / (c->box * c->box * c->box) / std::sqrt(4.0 * kPi);
    }
    p.use_mono = use_mono ? 1 : 0;
    p.vlos = (c->los && !counts_only) ? 1 : 0;
    for (int k = 0; k < 3; ++k) p.obs[k] = c->observer[k] / c->box * kTwo32;
    p.mono_w = mono_w;
    p.mono_w_dev = mono_w_dev;
    p.remove_self = c->remove_self;
    p.alm = alm;
    p.counts = counts;
    p.diag = diag;
    p.wsp = wsp;
    p.pair_counts = pair_counts;
    if (rrc && !counts_only) {
        p.counts_r = rrc->counts;
        p.pair_counts_r = rrc->pairs;
    }
    p.err = ds->err;
    const HarmTables h = make_tables(counts_only ? 0 : c->l_max);
    {
        const int hl = counts_only ? 0 : c->l_max;
        std::lock_guard<std::mutex> lk(g_mu);
        if (!ds->harm[hl]) {
            // once per device and l_max, before any capture: a synchronous upload
            CK(cudaMalloc((void **)&ds->harm[hl], sizeof(HarmTables)));
            CK(cudaMemcpy(ds->harm[hl], &h, sizeof(HarmTables), cudaMemcpyHostToDevice));
        }
        p.harm = ds->harm[hl];
    }

    size_t smem = pair_smem(c->l_max, counts_only, pl, c->n_bins);
    // the varying-line-of-sight kernel keeps its tile's frames in static shared memory
    const size_t smem_cap = 227 * 1024 - (counts_only ? 0 : kPairsStaticSmem)
                          - ((c->los && !counts_only) ? kVlosStaticSmem : 0);
    while (smem > smem_cap && pl.chunk > 512) {
        pl.chunk -= 256;
        smem = pair_smem(c->l_max, counts_only, pl, c->n_bins);
    }
    while (smem > smem_cap && pl.P > 1) {
        --pl.P;
        smem = pair_smem(c->l_max, counts_only, pl, c->n_bins);
    }
    if (smem > smem_cap) return fail(TPCF_ERR_UNSUPPORTED, "pair stage needs %zu bytes of shared memory", smem);
    if (!counts_only) {
        // the harmonic kernel gives every key at least 32 queue entries
        while (pl.P > 1 && pl.chunk < 32 * (pl.P * c->n_bins + 1)) --pl.P;
        if (pl.chunk < 32 * (pl.P * c->n_bins + 1))
            return fail(TPCF_ERR_ARG, "chunk %d is below 32 entries per bin (%d bins)", pl.chunk, c->n_bins);
        smem = pair_smem(c->l_max, counts_only, pl, c->n_bins);
    }
    if (bi) {
        // a tile never straddles two catalogues: the batch's own tiles (at most
        // bi->P primaries of one mock) when the plan allows that many, else one
        // primary per tile
        bool table = false;
        if (bi->tile_start && bi->P > 1 && !counts_only) {
            Plan q = pl;
            q.P = bi->P;
            table = pair_smem(c->l_max, counts_only, q, c->n_bins) <= smem_cap &&
                    (counts_only || q.chunk >= 32 * (q.P * c->n_bins + 1));
        }
        pl.P = table ? bi->P : 1;
        smem = pair_smem(c->l_max, counts_only, pl, c->n_bins);
        if (table) {
            p.tile_start = bi->tile_start;
            p.n_tiles = bi->n_tiles;
        }
        p.prim_mock = bi->prim_mock;
        p.ncell_mock = bi->ncell_mock;
        p.mono_w_mock = bi->mono_w_mock;
        p.mock_status = bi->mock_status;
    }
    p.P = pl.P;
    p.chunk = pl.chunk;
    Scratch sc(st);
    int *work = nullptr;
    if ((rc = sc.alloc(&work, 1, true))) return rc;
    p.work = work;
    // resident CTAs per SM from the occupancy calculator (registers and shared memory)
    const int per_sm = pair_per_sm(c->l_max, counts_only, p.vlos != 0, smem);
    int grid = ds->sms * per_sm;
    const int64_t tiles = p.tile_start ? p.n_tiles : (n_prim + pl.P - 1) / pl.P;
    if (grid > tiles) grid = (int)tiles;
    cudaError_t e = pair_launch(c->l_max, counts_only, p, h, grid, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "pair stage launch");
    return TPCF_OK;
}

int couple(const tpcf_config *c, const float *alm, const float *w, const int32_t *counts, int64_t K,
           const double *diag, const double *wsp, double *nnn, unsigned long long *trip_u64, cudaStream_t st)
{
    const int nb = c->n_bins, L = c->l_max;
    DevState *ds;
    int rc0 = dev_state(&ds);
    if (rc0) return rc0;
    int64_t gsz = gram_offset(nb, L, L + 1);
    Scratch sc(st);
    double *G = nullptr, *gaunt = nullptr;
    if ((rc0 = sc.alloc(&G, (size_t)gsz, true))) return rc0;
    const int L1 = L + 1;
    std::vector<double> hg((size_t)L1 * L1 * L1 * L1, 0.0);
    for (int m = 0; m <= L; ++m)
        for (int l1 = m; l1 <= L; ++l1)
            for (int l2 = m; l2 <= L; ++l2) {
                if ((l1 + l2) & 1) continue;
                const std::vector<double> g = self_coefs(L, l1, l2, m);
                const double kk = k_scale(l1, m) * k_scale(l2, m);
                for (int j = 0; j <= L; ++j) hg[(((size_t)m * L1 + l1) * L1 + l2) * L1 + j] = kk * g[j];
            }
    if ((rc0 = sc.alloc(&gaunt, hg.size(), false))) return rc0;
    CK(cudaMemcpyAsync(gaunt, hg.data(), hg.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    if (c->precision == TPCF_PREC_FP32) {
        CK(couple_gram_simt(alm, w, K, nb, L, G, ds->sms, st));
    } else {
        cudaError_t e = couple_gram_tc(alm, w, K, nb, L, c->precision == TPCF_PREC_TF32X3, G, ds->err, ds->sms, st);
        if (e == cudaErrorInvalidValue)
            return fail(TPCF_ERR_UNSUPPORTED, "tensor-core Gram: no tile plan for this shape");
        CK(e);
    }
    CK(assemble_nnn(G, diag, wsp, nb, L, c->remove_self, gaunt, nnn, st));
    if (counts && trip_u64) CK(tpcf::triplet_counts(counts, K, nb, trip_u64, st));
    // the host vector must outlive the asynchronous copy
    CK(cudaStreamSynchronize(st));
    return TPCF_OK;
}

void projection_tables(const tpcf_config *c, std::vector<double> &coef, std::vector<int> &ml)
{
    multipole_list(c, ml);
    const int nm = (int)ml.size() / 3, L1 = c->l_max + 1;
    coef.assign((size_t)nm * L1, 0.0);
    for (int k = 0; k < nm; ++k) {
        const int l1 = ml[3 * k], l2 = ml[3 * k + 1], L = ml[3 * k + 2];
        const double H = w3j(l1, l2, L, 0, 0, 0);
        const double conv = (c->convention == TPCF_CONV_S_COEFF) ? std::sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0)) : 1.0;
        for (int m = 0; m <= std::min(l1, l2); ++m) {
            const double t = w3j(l1, l2, L, m, -m, 0) * ((m % 2) ? -1.0 : 1.0);
            coef[(size_t)k * L1 + m] = conv * (2.0 * L + 1.0) * H * (m == 0 ? t : 2.0 * t);
        }
    }
}

// Gaunt coefficient: int Y_l1^m1 Y_l2^m2 (Y_l3^(m1+m2))* dOmega.
double gaunt(int l1, int m1, int l2, int m2, int l3)
{
    const int m3 = m1 + m2;
    if (std::abs(m1) > l1 || std::abs(m2) > l2 || std::abs(m3) > l3) return 0.0;
    const double pre = std::sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * (2.0 * l3 + 1.0) / (4.0 * kPi));
    return pre * w3j(l1, l2, l3, 0, 0, 0) * w3j(l1, l2, l3, m1, m2, -m3) * ((m3 & 1) ? -1.0 : 1.0);
}

// The unknowns of the edge-correction system and the sparse terms of its matrix:
// entry (r, c) = sum over t in [tstart[r nu + c], tstart[r nu + c + 1]) of
// tcoef[t] * RRR block tridx[t] (block (m * L1 + l1) * L1 + l2 of the [m][l1][l2]
// layout), with the +m' and -m' columns of a real, m-symmetric unknown added.
struct EdgeTables {
    std::vector<int> modes, tstart, tridx;
    std::vector<double> tcoef;
    int nu = 0;
};

void edge_corr_tables(int L, EdgeTables &t)
{
    const int L1 = L + 1;
    t.modes.clear();
    for (int m = 0; m <= L; ++m)
        for (int l1 = m; l1 <= L; ++l1)
            for (int l2 = m; l2 <= L; ++l2)
                if (((l1 + l2) & 1) == 0) {
                    t.modes.push_back(l1);
                    t.modes.push_back(l2);
                    t.modes.push_back(m);
                }
    t.nu = (int)t.modes.size() / 3;
    t.tstart.assign(1, 0);
    t.tridx.clear();
    t.tcoef.clear();
    for (int r = 0; r < t.nu; ++r) {
        const int l1 = t.modes[3 * r], l2 = t.modes[3 * r + 1], m = t.modes[3 * r + 2];
        for (int c = 0; c < t.nu; ++c) {
            const int p1 = t.modes[3 * c], p2 = t.modes[3 * c + 1], mp = t.modes[3 * c + 2];
            for (int sgn = 0; sgn < (mp > 0 ? 2 : 1); ++sgn) {
                const int mq = sgn ? -mp : mp, mr = m - mq, ar = std::abs(mr);
                if (ar > L) continue;
                for (int q1 = ar; q1 <= L; ++q1)
                    for (int q2 = ar; q2 <= L; ++q2) {
                        if ((q1 + q2) & 1) continue;
                        const double g = gaunt(p1, mq, q1, mr, l1) * gaunt(p2, mq, q2, mr, l2);
                        if (g == 0.0) continue;
                        t.tridx.push_back((ar * L1 + q1) * L1 + q2);
                        t.tcoef.push_back(4.0 * kPi * g);
                    }
            }
            t.tstart.push_back((int)t.tridx.size());
        }
    }
}

int project(const tpcf_config *c, const double *nnn, const double *rrr, double *zeta, cudaStream_t st)
{
    std::vector<int> ml;
    multipole_list(c, ml);
    const int nm = (int)ml.size() / 3, L1 = c->l_max + 1;
    std::vector<double> coef((size_t)nm * L1, 0.0);
    for (int k = 0; k < nm; ++k) {
        const int l1 = ml[3 * k], l2 = ml[3 * k + 1], L = ml[3 * k + 2];
        const double H = w3j(l1, l2, L, 0, 0, 0);
        double conv = (c->convention == TPCF_CONV_S_COEFF) ? std::sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0)) : 1.0;
        for (int m = 0; m <= std::min(l1, l2); ++m) {
            const double t = w3j(l1, l2, L, m, -m, 0) * ((m % 2) ? -1.0 : 1.0);
            coef[(size_t)k * L1 + m] = conv * (2.0 * L + 1.0) * H * (m == 0 ? t : 2.0 * t);
        }
    }
    Scratch sc(st);
    double *dcoef = nullptr;
    int *dml = nullptr;
    int rc = sc.alloc(&dcoef, coef.size() + 1, false);
    if (!rc) rc = sc.alloc(&dml, ml.size() + 1, false);
    if (rc) return rc;
    CK(cudaMemcpyAsync(dcoef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dml, ml.data(), ml.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(project_zeta(nnn, rrr, c->n_bins, c->l_max, nm, dcoef, dml, zeta, st));
    CK(cudaStreamSynchronize(st));
    return TPCF_OK;
}

int choose_nc(const tpcf_config *c, int64_t n)
{
    return make_plan(c, n, n).nc;
}

int mono_coef_dev(const tpcf_config *c, double **out, cudaStream_t st)
{
    double r[TPCF_MAX_BINS + 1];
    unsigned long long E[TPCF_MAX_BINS + 1];
    edge_tables(c, E, r);
    std::vector<double> coef(c->n_bins);
    for (int b = 0; b < c->n_bins; ++b) {
        const double vb = 4.0 * kPi / 3.0 * (r[b + 1] * r[b + 1] * r[b + 1] - r[b] * r[b] * r[b]);
        coef[b] = vb / (c->box * c->box * c->box) / std::sqrt(4.0 * kPi);
    }
    CK(scratch_malloc((void **)out, c->n_bins * sizeof(double), st));
    CK(cudaMemcpyAsync(*out, coef.data(), c->n_bins * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return TPCF_OK;
}


// Whether the randoms of a D - R field are exactly its records whose weight has the
// sign bit set, so that the harmonic pass can count random-random pairs: true when
// no data weight has its sign bit set and one is positive (then W_D > 0 and every
// random's weight -(W_D / W_R) w is negative for w > 0).  Null weights are ones.
// Synchronises the stream.
int randoms_are_negative(const float *w1, int64_t n1, const float *w2, int64_t n2, bool *ok, cudaStream_t st)
{
    *ok = false;
    if (!w1 && !w2) {
        *ok = (n1 + n2) > 0;
        return TPCF_OK;
    }
    int *d = nullptr;
    CK(scratch_malloc((void **)&d, 2 * sizeof(int), st));
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess && w1) e = weight_signs(w1, n1, d, st);
    if (e == cudaSuccess && w2) e = weight_signs(w2, n2, d, st);
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    CK(e);
    const int64_t pos_unit = (w1 ? 0 : n1) + (w2 ? 0 : n2);   // null weights are ones
    *ok = h[0] == 0 && (h[1] > 0 || pos_unit > 0);
    return TPCF_OK;
}

int estimate_impl(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                  const uint32_t *r_xyz, const float *r_w, int64_t nr, double *zeta, double *nnn_out,
                  double *rrr_out, int64_t *pair_counts, int64_t *triplet_counts, double *xi, bool edge_full,
                  double *rfull_out, cudaStream_t st)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!zeta) return fail(TPCF_ERR_ARG, "zeta is required");
    if (nd < 1 || !d_xyz) return fail(TPCF_ERR_ARG, "need at least one data point");
    if (nr < 0 || (nr > 0 && !r_xyz)) return fail(TPCF_ERR_ARG, "bad randoms");
    const bool analytic = (nr == 0);
    if (analytic && !cfg->periodic) return fail(TPCF_ERR_ARG, "analytic randoms need a periodic box");
    if (nd + nr >= kMaxPoints) return fail(TPCF_ERR_ARG, "catalogue too large (nd + nr < 2^28)");
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    GridDev gf, gr;   // declared before the guard that releases them
    Scratch sc(st);
    sc.own(gf);
    sc.own(gr);
    const int nb = cfg->n_bins, L = cfg->l_max;
    const int nlm = (L + 1) * (L + 1), ndiag = (L + 1) * (L + 2) / 2;
    const int L1 = L + 1;
    const int n_ell = L / 2 + 1;   // even multipoles 0, 2, ..., l_max
    // weighted randoms: RRR_00^0 and the pair normaliser come from the l = 0 harmonic
    // sums of the randoms; unit randoms (r_w NULL or all ones): from integer counts
    bool weighted_r = false;
    if (!analytic && r_w) {
        int *d_n = nullptr, h_n = 0;
        if ((rc = sc.alloc(&d_n, 1, true))) return rc;
        CK(count_not_one(r_w, nr, d_n, st));
        CK(cudaMemcpyAsync(&h_n, d_n, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        weighted_r = h_n != 0;
    }
    // open volume, unit randoms, the l = 0 normaliser: the random-random counts come
    // with the D - R pass when the randoms are its only negative weights
    bool rr_fused = false;
    if (!analytic && !weighted_r && !edge_full)
        if ((rc = randoms_are_negative(d_w, nd, nullptr, 0, &rr_fused, st))) return rc;

    double *wsums = nullptr, *diag = nullptr, *wsp = nullptr, *nnn = nnn_out, *rrr = rrr_out, *mono = nullptr;
    double *S = nullptr, *s0 = nullptr, *rr = nullptr;
    float *alm = nullptr;
    int32_t *cnt = nullptr, *cnt_r = nullptr;
    unsigned long long *pairs = nullptr, *T = nullptr, *TR = nullptr, *pairs_r = nullptr;
    float *alm_r = nullptr, *wprim_r = nullptr;
    double *diag_r = nullptr, *wsp_r = nullptr, *nnn_r = nullptr;
    if ((rc = sc.alloc(&wsums, 2, true))) return rc;
    CK(weight_sums(d_w, nd, r_w, nr, wsums, st));
    const int64_t K = nd + nr;
    // neighbour field grid: D, or D - (W_D/W_R) R
    CK(build_grid_dev(d_xyz, d_w, nd, r_xyz, r_w, nr, analytic ? nullptr : wsums, choose_nc(cfg, K), gf, ds->err, st));
    if ((rc = sc.alloc(&alm, (size_t)K * nb * nlm, false))) return rc;
    if ((rc = sc.alloc(&cnt, (size_t)K * nb, false))) return rc;
    if ((rc = sc.alloc(&diag, (size_t)ndiag * nb, true))) return rc;
    if ((rc = sc.alloc(&wsp, (size_t)L1 * nb, true))) return rc;
    if ((rc = sc.alloc(&pairs, (size_t)nb, true))) return rc;
    if ((rc = sc.alloc(&T, (size_t)nb * nb, true))) return rc;
    if (!nnn && (rc = sc.alloc(&nnn, (size_t)L1 * L1 * L1 * nb * nb, false))) return rc;
    if (!rrr && (rc = sc.alloc(&rrr, (size_t)nb * nb, false))) return rc;
    RRCounts rrc = {nullptr, nullptr};
    if (rr_fused) {
        if ((rc = sc.alloc(&cnt_r, (size_t)K * nb, false))) return rc;
        if ((rc = sc.alloc(&TR, (size_t)nb * nb, true))) return rc;
        if (xi && (rc = sc.alloc(&pairs_r, (size_t)nb, true))) return rc;
        rrc.counts = cnt_r;
        rrc.pairs = pairs_r;
    }
    rc = run_pairs(cfg, gf, gf.rec, K, false, 0.0, analytic ? wsums : nullptr, analytic, alm, cnt, diag, wsp, pairs,
                   st, nullptr, rr_fused ? &rrc : nullptr);
    if (rc) return rc;
    // primary weights in grid order are the records' w fields: pass them through a strided copy
    float *wprim = nullptr;
    if ((rc = sc.alloc(&wprim, (size_t)K, false))) return rc;
    CK(cudaMemcpy2DAsync(wprim, 4, (const char *)gf.rec + 12, 16, 4, K, cudaMemcpyDeviceToDevice, st));
    if ((rc = couple(cfg, alm, wprim, cnt, K, diag, wsp, nnn, T, st))) return rc;
    if (xi) {
        if ((rc = sc.alloc(&S, (size_t)n_ell * nb, true))) return rc;
        if ((rc = sc.alloc(&rr, (size_t)nb, false))) return rc;
        CK(m0_sums(alm, wprim, K, nb, L, n_ell, 2, S, st));
    }
    int rr_mode = 0;
    if (analytic) {
        rc = mono_coef_dev(cfg, &mono, st);
        sc.keep(mono);
        if (rc) return rc;
        CK(rrr_analytic(wsums, mono, nb, rrr, st));
    } else if (!weighted_r && !edge_full) {
        if (rr_fused) {
            // counted by the D - R pass: rows of data primaries are zero
            CK(tpcf::triplet_counts(cnt_r, K, nb, TR, st));
        } else {
            CK(build_grid_dev(r_xyz, r_w, nr, nullptr, nullptr, 0, nullptr, choose_nc(cfg, nr), gr, ds->err, st));
            if ((rc = sc.alloc(&cnt_r, (size_t)nr * nb, false))) return rc;
            if ((rc = sc.alloc(&TR, (size_t)nb * nb, true))) return rc;
            if (xi && (rc = sc.alloc(&pairs_r, (size_t)nb, true))) return rc;
            rc = run_pairs(cfg, gr, gr.rec, nr, true, 0.0, nullptr, false, nullptr, cnt_r, nullptr, nullptr,
                           pairs_r, st);
            if (rc) return rc;
            CK(tpcf::triplet_counts(cnt_r, nr, nb, TR, st));
        }
        CK(rrr_from_counts(TR, wsums, nb, rrr, st));
        rr_mode = 1;
    } else {
        // a harmonic pass over the randoms with their own weights, then its coupling:
        // l = 0 only (RRR_00^0 of weighted randoms) or every l (the full edge correction)
        tpcf_config cr = *cfg;
        if (!edge_full) {
            cr.l_max = 0;
            cr.n_L = 1;
            cr.L[0] = 0;
        }
        const int Lr = cr.l_max, L1r = Lr + 1;
        const size_t nfull = (size_t)L1r * L1r * L1r * nb * nb;
        CK(build_grid_dev(r_xyz, r_w, nr, nullptr, nullptr, 0, nullptr, choose_nc(cfg, nr), gr, ds->err, st));
        if ((rc = sc.alloc(&alm_r, (size_t)nr * nb * L1r * L1r, false))) return rc;
        if ((rc = sc.alloc(&cnt_r, (size_t)nr * nb, false))) return rc;
        if ((rc = sc.alloc(&diag_r, (size_t)nb * L1r * (Lr + 2) / 2, true))) return rc;
        if ((rc = sc.alloc(&wsp_r, (size_t)nb * L1r, true))) return rc;
        if (rfull_out) nnn_r = rfull_out;
        else if ((rc = sc.alloc(&nnn_r, nfull, false))) return rc;
        if ((rc = sc.alloc(&wprim_r, (size_t)nr, false))) return rc;
        rc = run_pairs(&cr, gr, gr.rec, nr, false, 0.0, nullptr, false, alm_r, cnt_r, diag_r, wsp_r, nullptr, st);
        if (rc) return rc;
        CK(cudaMemcpy2DAsync(wprim_r, 4, (const char *)gr.rec + 12, 16, 4, nr, cudaMemcpyDeviceToDevice, st));
        if ((rc = couple(&cr, alm_r, wprim_r, nullptr, nr, diag_r, wsp_r, nnn_r, nullptr, st))) return rc;
        // RRR = alpha^3 times the randoms' own coupling; its m = 0, l1 = l2 = 0 block is RRR_00^0
        CK(scale_alpha3(nnn_r, (int64_t)nfull, wsums, st));
        CK(cudaMemcpyAsync(rrr, nnn_r, (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (xi) {
            if ((rc = sc.alloc(&s0, (size_t)nb, true))) return rc;
            CK(m0_sums(alm_r, wprim_r, nr, nb, Lr, 1, 2, s0, st));
        }
        rr_mode = 2;
    }
    if (edge_full) {
        EdgeTables et;
        edge_corr_tables(L, et);
        int *d_modes = nullptr, *d_ts = nullptr, *d_ti = nullptr;
        double *d_tc = nullptr, *zhat = nullptr;
        if ((rc = sc.alloc(&d_modes, et.modes.size(), false))) return rc;
        if ((rc = sc.alloc(&d_ts, et.tstart.size(), false))) return rc;
        if ((rc = sc.alloc(&d_ti, et.tridx.size() + 1, false))) return rc;
        if ((rc = sc.alloc(&d_tc, et.tcoef.size() + 1, false))) return rc;
        if ((rc = sc.alloc(&zhat, (size_t)L1 * L1 * L1 * nb * nb, false))) return rc;
        CK(cudaMemcpyAsync(d_modes, et.modes.data(), et.modes.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_ts, et.tstart.data(), et.tstart.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_ti, et.tridx.data(), et.tridx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_tc, et.tcoef.data(), et.tcoef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(edge_solve(nnn, nnn_r, nb, L, et.nu, d_modes, d_ts, d_ti, d_tc, zhat, ds->err, st));
        if ((rc = project(cfg, zhat, nullptr, zeta, st))) return rc;   // synchronises: the host tables outlive the copies
    } else if ((rc = project(cfg, nnn, rrr, zeta, st))) {
        return rc;
    }
    if (xi) CK(xi_from_sums(rr_mode, wsums, mono, pairs_r, s0, S, n_ell, 2, nb, rr, xi, st));
    if (pair_counts) CK(i64_from_u64(pairs, pair_counts, nb, st));
    if (triplet_counts) CK(i64_from_u64(T, triplet_counts, nb * nb, st));
    CK(cudaGetLastError());
    return TPCF_OK;
}

// ----------------------------------------------------------- sharded form
// Sizes of the additive partial results of one shard (doubles, int64 counts).
// doubles: nnn [L1^3 nb^2], S [n_ell nb] (2PCF sums), R00 [nb^2] and s0 [nb] (the
// randoms' l = 0 coupling and 2PCF sums, weighted randoms);
// int64: pair counts [nb], triplet counts [nb^2], random triplet counts [nb^2],
// random pair counts [nb].
struct PartLayout {
    int64_t nnn, S, R00, s0, nf;
    int64_t pairs, T, TR, pairs_r, ni;
};

PartLayout part_layout(const tpcf_config *c)
{
    PartLayout P;
    const int64_t nb = c->n_bins, L1 = c->l_max + 1, n_ell = c->l_max / 2 + 1;
    P.nnn = 0;
    P.S = P.nnn + L1 * L1 * L1 * nb * nb;
    P.R00 = P.S + n_ell * nb;
    P.s0 = P.R00 + nb * nb;
    P.nf = P.s0 + nb;
    P.pairs = 0;
    P.T = P.pairs + nb;
    P.TR = P.T + nb * nb;
    P.pairs_r = P.TR + nb * nb;
    P.ni = P.pairs_r + nb;
    return P;
}

// One shard's additive partials: primaries dp (data, weights as given) and rp
// (randoms, weights -(W_D / W_R) w in the D - R field) against the secondaries
// d, r given (every point within r_max of a primary), with the weight totals of
// the whole catalogue.  Periodic analytic randoms when nr = nrp = 0.
int partial_impl(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd, const uint32_t *r_xyz,
                 const float *r_w, int64_t nr, const uint32_t *dp_xyz, const float *dp_w, int64_t ndp,
                 const uint32_t *rp_xyz, const float *rp_w, int64_t nrp, double w_d, double w_r, int weighted_r,
                 double *part_f, int64_t *part_i, cudaStream_t st)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!part_f || !part_i) return fail(TPCF_ERR_ARG, "the partial outputs are required");
    const bool analytic = (nr == 0 && nrp == 0);
    if (analytic && !cfg->periodic) return fail(TPCF_ERR_ARG, "analytic randoms need a periodic box");
    if (nd < 0 || nr < 0 || ndp < 0 || nrp < 0) return fail(TPCF_ERR_ARG, "negative point count");
    if ((nd > 0 && !d_xyz) || (nr > 0 && !r_xyz) || (ndp > 0 && !dp_xyz) || (nrp > 0 && !rp_xyz))
        return fail(TPCF_ERR_ARG, "coordinates are required for every non-empty set");
    if (!(w_d > 0.0) || (!analytic && !(w_r != 0.0)))
        return fail(TPCF_ERR_ARG, "the catalogue's weight totals are required");
    if (nd + nr >= kMaxPoints) return fail(TPCF_ERR_ARG, "catalogue too large (nd + nr < 2^28)");
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    const PartLayout PL = part_layout(cfg);
    CK(cudaMemsetAsync(part_f, 0, PL.nf * sizeof(double), st));
    CK(cudaMemsetAsync(part_i, 0, PL.ni * sizeof(int64_t), st));
    const int nb = cfg->n_bins, L = cfg->l_max;
    const int nlm = (L + 1) * (L + 1), ndiag = (L + 1) * (L + 2) / 2, L1 = L + 1, n_ell = L / 2 + 1;
    GridDev gf, gr;
    Scratch sc(st);
    sc.own(gf);
    sc.own(gr);
    double *wsums = nullptr;
    if ((rc = sc.alloc(&wsums, 2, false))) return rc;
    const double hw[2] = {w_d, w_r};
    CK(cudaMemcpyAsync(wsums, hw, sizeof(hw), cudaMemcpyHostToDevice, st));
    const int64_t K = ndp + nrp;
    // unit randoms: their pair counts come with the D - R pass when they are its only
    // negative weights (as in the one-catalogue estimate)
    bool rr_fused = false;
    const bool rr_counts = !analytic && nr > 0 && nrp > 0 && !weighted_r;
    if (rr_counts && nd + nr > 0 && K > 0)
        if ((rc = randoms_are_negative(d_w, nd, dp_w, ndp, &rr_fused, st))) return rc;
    if (nd + nr > 0 && K > 0) {
        CK(build_grid_dev(d_xyz, d_w, nd, r_xyz, r_w, nr, analytic ? nullptr : wsums, choose_nc(cfg, nd + nr), gf,
                          ds->err, st));
        int4 *prim = nullptr;
        float *alm = nullptr, *wprim = nullptr;
        int32_t *cnt = nullptr;
        double *diag = nullptr, *wsp = nullptr;
        unsigned long long *pairs = nullptr, *T = nullptr;
        if ((rc = sc.alloc(&prim, (size_t)K, false))) return rc;
        CK(pack_records(dp_xyz, dp_w, ndp, prim, ds->err, st));
        CK(pack_records(rp_xyz, rp_w, nrp, prim + ndp, ds->err, st, wsums));
        if ((rc = sc.alloc(&alm, (size_t)K * nb * nlm, false))) return rc;
        if ((rc = sc.alloc(&cnt, (size_t)K * nb, false))) return rc;
        if ((rc = sc.alloc(&diag, (size_t)ndiag * nb, true))) return rc;
        if ((rc = sc.alloc(&wsp, (size_t)L1 * nb, true))) return rc;
        if ((rc = sc.alloc(&pairs, (size_t)nb, true))) return rc;
        if ((rc = sc.alloc(&T, (size_t)nb * nb, true))) return rc;
        if ((rc = sc.alloc(&wprim, (size_t)K, false))) return rc;
        RRCounts rrc = {nullptr, nullptr};
        unsigned long long *TR = nullptr;
        if (rr_fused) {
            if ((rc = sc.alloc(&rrc.counts, (size_t)K * nb, false))) return rc;
            if ((rc = sc.alloc(&rrc.pairs, (size_t)nb, true))) return rc;
            if ((rc = sc.alloc(&TR, (size_t)nb * nb, true))) return rc;
        }
        rc = run_pairs(cfg, gf, prim, K, false, 0.0, analytic ? wsums : nullptr, analytic, alm, cnt, diag, wsp,
                       pairs, st, nullptr, rr_fused ? &rrc : nullptr);
        if (rc) return rc;
        if (rr_fused) {
            // rows of data primaries are zero
            CK(tpcf::triplet_counts(rrc.counts, K, nb, TR, st));
            CK(i64_from_u64(TR, part_i + PL.TR, nb * nb, st));
            CK(i64_from_u64(rrc.pairs, part_i + PL.pairs_r, nb, st));
        }
        CK(cudaMemcpy2DAsync(wprim, 4, (const char *)prim + 12, 16, 4, K, cudaMemcpyDeviceToDevice, st));
        if ((rc = couple(cfg, alm, wprim, cnt, K, diag, wsp, part_f + PL.nnn, T, st))) return rc;
        CK(m0_sums(alm, wprim, K, nb, L, n_ell, 2, part_f + PL.S, st));
        CK(i64_from_u64(pairs, part_i + PL.pairs, nb, st));
        CK(i64_from_u64(T, part_i + PL.T, nb * nb, st));
    }
    if (!analytic && nr > 0 && nrp > 0 && !rr_fused) {
        if (!weighted_r) {
            // integer random triplet counts of the shard's random primaries
            int4 *rprim = nullptr;
            int32_t *cnt_r = nullptr;
            unsigned long long *TR = nullptr, *pairs_r = nullptr;
            CK(build_grid_dev(r_xyz, r_w, nr, nullptr, nullptr, 0, nullptr, choose_nc(cfg, nr), gr, ds->err, st));
            if ((rc = sc.alloc(&rprim, (size_t)nrp, false))) return rc;
            CK(pack_records(rp_xyz, rp_w, nrp, rprim, ds->err, st));
            if ((rc = sc.alloc(&cnt_r, (size_t)nrp * nb, false))) return rc;
            if ((rc = sc.alloc(&TR, (size_t)nb * nb, true))) return rc;
            if ((rc = sc.alloc(&pairs_r, (size_t)nb, true))) return rc;
            rc = run_pairs(cfg, gr, rprim, nrp, true, 0.0, nullptr, false, nullptr, cnt_r, nullptr, nullptr, pairs_r,
                           st);
            if (rc) return rc;
            CK(tpcf::triplet_counts(cnt_r, nrp, nb, TR, st));
            CK(i64_from_u64(TR, part_i + PL.TR, nb * nb, st));
            CK(i64_from_u64(pairs_r, part_i + PL.pairs_r, nb, st));
        } else {
            // the randoms' own l = 0 coupling with their weights (alpha^3 applied at the end)
            tpcf_config cr = *cfg;
            cr.l_max = 0;
            cr.n_L = 1;
            cr.L[0] = 0;
            int4 *rprim = nullptr;
            float *alm_r = nullptr, *wprim_r = nullptr;
            int32_t *cnt_r = nullptr;
            double *diag_r = nullptr, *wsp_r = nullptr, *nnn_r = nullptr;
            CK(build_grid_dev(r_xyz, r_w, nr, nullptr, nullptr, 0, nullptr, choose_nc(cfg, nr), gr, ds->err, st));
            if ((rc = sc.alloc(&rprim, (size_t)nrp, false))) return rc;
            CK(pack_records(rp_xyz, rp_w, nrp, rprim, ds->err, st));
            if ((rc = sc.alloc(&alm_r, (size_t)nrp * nb, false))) return rc;
            if ((rc = sc.alloc(&cnt_r, (size_t)nrp * nb, false))) return rc;
            if ((rc = sc.alloc(&diag_r, (size_t)nb, true))) return rc;
            if ((rc = sc.alloc(&wsp_r, (size_t)nb, true))) return rc;
            if ((rc = sc.alloc(&nnn_r, (size_t)nb * nb, false))) return rc;
            if ((rc = sc.alloc(&wprim_r, (size_t)nrp, false))) return rc;
            rc = run_pairs(&cr, gr, rprim, nrp, false, 0.0, nullptr, false, alm_r, cnt_r, diag_r, wsp_r, nullptr, st);
            if (rc) return rc;
            CK(cudaMemcpy2DAsync(wprim_r, 4, (const char *)rprim + 12, 16, 4, nrp, cudaMemcpyDeviceToDevice, st));
            if ((rc = couple(&cr, alm_r, wprim_r, nullptr, nrp, diag_r, wsp_r, nnn_r, nullptr, st))) return rc;
            CK(cudaMemcpyAsync(part_f + PL.R00, nnn_r, (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToDevice,
                               st));
            CK(m0_sums(alm_r, wprim_r, nrp, nb, 0, 1, 2, part_f + PL.s0, st));
        }
    }
    CK(cudaStreamSynchronize(st));   // the host copy of the totals outlives the upload
    CK(cudaGetLastError());
    return TPCF_OK;
}

// zeta (and NNN, RRR, counts, xi) from the summed partials of every shard.
int finish_impl(const tpcf_config *cfg, double w_d, double w_r, int explicit_randoms, int weighted_r,
                const double *part_f, const int64_t *part_i, double *zeta, double *nnn_out, double *rrr_out,
                int64_t *pair_counts, int64_t *triplet_counts, double *xi, cudaStream_t st)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!part_f || !part_i || !zeta) return fail(TPCF_ERR_ARG, "partials and zeta are required");
    const bool analytic = !explicit_randoms;
    if (analytic && !cfg->periodic) return fail(TPCF_ERR_ARG, "analytic randoms need a periodic box");
    if (!(w_d > 0.0) || (!analytic && !(w_r != 0.0)))
        return fail(TPCF_ERR_ARG, "the catalogue's weight totals are required");
    const PartLayout PL = part_layout(cfg);
    const int nb = cfg->n_bins, L = cfg->l_max, L1 = L + 1, n_ell = L / 2 + 1;
    Scratch sc(st);
    double *wsums = nullptr, *rrr = rrr_out, *mono = nullptr, *r00 = nullptr, *rr = nullptr;
    unsigned long long *TRu = nullptr, *pr = nullptr;
    if ((rc = sc.alloc(&wsums, 2, false))) return rc;
    const double hw[2] = {w_d, w_r};
    CK(cudaMemcpyAsync(wsums, hw, sizeof(hw), cudaMemcpyHostToDevice, st));
    if (!rrr && (rc = sc.alloc(&rrr, (size_t)nb * nb, false))) return rc;
    int rr_mode = 0;
    if (analytic) {
        rc = mono_coef_dev(cfg, &mono, st);
        sc.keep(mono);
        if (rc) return rc;
        CK(rrr_analytic(wsums, mono, nb, rrr, st));
    } else if (!weighted_r) {
        if ((rc = sc.alloc(&TRu, (size_t)nb * nb, false))) return rc;
        if ((rc = sc.alloc(&pr, (size_t)nb, false))) return rc;
        CK(cudaMemcpyAsync(TRu, part_i + PL.TR, (size_t)nb * nb * 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(pr, part_i + PL.pairs_r, (size_t)nb * 8, cudaMemcpyDeviceToDevice, st));
        CK(rrr_from_counts(TRu, wsums, nb, rrr, st));
        rr_mode = 1;
    } else {
        if ((rc = sc.alloc(&r00, (size_t)nb * nb, false))) return rc;
        CK(cudaMemcpyAsync(r00, part_f + PL.R00, (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(scale_alpha3(r00, (int64_t)nb * nb, wsums, st));
        CK(cudaMemcpyAsync(rrr, r00, (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
        rr_mode = 2;
    }
    if (nnn_out)
        CK(cudaMemcpyAsync(nnn_out, part_f + PL.nnn, (size_t)L1 * L1 * L1 * nb * nb * sizeof(double),
                           cudaMemcpyDeviceToDevice, st));
    if ((rc = project(cfg, part_f + PL.nnn, rrr, zeta, st))) return rc;
    if (xi) {
        if ((rc = sc.alloc(&rr, (size_t)nb, false))) return rc;
        CK(xi_from_sums(rr_mode, wsums, mono, pr, part_f + PL.s0, part_f + PL.S, n_ell, 2, nb, rr, xi, st));
    }
    if (pair_counts)
        CK(cudaMemcpyAsync(pair_counts, part_i + PL.pairs, (size_t)nb * 8, cudaMemcpyDeviceToDevice, st));
    if (triplet_counts)
        CK(cudaMemcpyAsync(triplet_counts, part_i + PL.T, (size_t)nb * nb * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return TPCF_OK;
}

}  // namespace

void tpcf::self_term_table(int lmax, double *out)
{
    const int L1 = lmax + 1;
    for (int i = 0; i < L1 * L1 * L1 * L1; ++i) out[i] = 0.0;
    for (int m = 0; m <= lmax; ++m)
        for (int l1 = m; l1 <= lmax; ++l1)
            for (int l2 = m; l2 <= lmax; ++l2) {
                if ((l1 + l2) & 1) continue;
                const std::vector<double> g = self_coefs(lmax, l1, l2, m);
                const double kk = k_scale(l1, m) * k_scale(l2, m);
                for (int j = 0; j <= lmax; ++j) out[(((size_t)m * L1 + l1) * L1 + l2) * L1 + j] = kk * g[j];
            }
}

int tpcf::check_config_public(const tpcf_config *c) { return check_config(c); }

int *tpcf::device_error_flag()
{
    DevState *ds = nullptr;
    return dev_state(&ds) == TPCF_OK ? ds->err : nullptr;
}

int tpcf::set_error(int code, const char *msg) { return fail(code, "%s", msg); }

// ===================================================================== C ABI

extern "C" {

const char *tpcf_last_error(void) { return g_msg; }

int tpcf_version(void) { return 100; }

int tpcf_set_wait_limit(int64_t polls, int32_t unmet_wait)
{
    if (polls < 0) return fail(TPCF_ERR_ARG, "polls < 0");
    g_wait_limit.store((long long)polls, std::memory_order_relaxed);
    g_wait_unmet.store(unmet_wait ? 1 : 0, std::memory_order_relaxed);
    return TPCF_OK;
}

int64_t tpcf_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

int tpcf_quantize_host(const float *x, int64_t n, double box, uint32_t *u)
{
    if (!(box > 0.0) || n < 0 || (n > 0 && (!x || !u))) return fail(TPCF_ERR_ARG, "box > 0 and both arrays are required");
    const double scale = kTwo32 / box;
    for (int64_t i = 0; i < n; ++i) {
        const double v = (double)x[i];
        if (!(v >= 0.0 && v < box))
            return fail(TPCF_ERR_DATA, "position %lld (%g) outside [0, %g)", (long long)i, v, box);
        const double q = std::floor(v * scale);
        u[i] = q >= kTwo32 ? 0xFFFFFFFFu : (uint32_t)q;   // v < box, so q < 2^32 up to the product's rounding
    }
    return TPCF_OK;
}

int tpcf_multipole_count(const tpcf_config *cfg, int32_t *n_mult)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!n_mult) return fail(TPCF_ERR_ARG, "n_mult is NULL");
    std::vector<int> ml;
    multipole_list(cfg, ml);
    *n_mult = (int32_t)(ml.size() / 3);
    return TPCF_OK;
}

int tpcf_multipole_index(const tpcf_config *cfg, int32_t *l1l2L, int32_t cap)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    std::vector<int> ml;
    multipole_list(cfg, ml);
    if (!l1l2L || cap < (int32_t)(ml.size() / 3)) return fail(TPCF_ERR_ARG, "output too small");
    for (size_t i = 0; i < ml.size(); ++i) l1l2L[i] = ml[i];
    return TPCF_OK;
}

int tpcf_bin_edges(const tpcf_config *cfg, uint64_t *E)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!E) return fail(TPCF_ERR_ARG, "E is NULL");
    unsigned long long e[TPCF_MAX_BINS + 1];
    edge_tables(cfg, e, nullptr);
    for (int b = 0; b <= cfg->n_bins; ++b) E[b] = e[b];
    return TPCF_OK;
}

int tpcf_build_grid(const uint32_t *xyz, const float *w, int64_t n, const tpcf_config *cfg, tpcf_grid *out,
                    void *stream)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!out) return fail(TPCF_ERR_ARG, "out is NULL");
    if (n < 0 || n >= kMaxPoints) return fail(TPCF_ERR_ARG, "n out of range (0 <= n < 2^28)");
    if (n > 0 && !xyz) return fail(TPCF_ERR_ARG, "xyz is NULL");
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    tpcf_grid g = new tpcf_grid_s();
    g->stream = st;
    cudaGetDevice(&g->device);
    cudaError_t e = build_grid_dev(xyz, w, n, nullptr, nullptr, 0, nullptr, choose_nc(cfg, n), g->g, ds->err, st);
    if (e != cudaSuccess) {
        free_grid_dev(g->g, st);
        delete g;
        return cuda_fail(e, "build_grid");
    }
    *out = g;
    return TPCF_OK;
}

int tpcf_grid_destroy(tpcf_grid grid)
{
    if (!grid) return TPCF_OK;
    free_grid_dev(grid->g, grid->stream);
    cudaError_t e = cudaStreamSynchronize(grid->stream);
    delete grid;
    if (e != cudaSuccess) return cuda_fail(e, "grid_destroy");
    return TPCF_OK;
}

int tpcf_grid_info(tpcf_grid grid, int64_t *n_points, int32_t *cells_per_axis)
{
    if (!grid) return fail(TPCF_ERR_ARG, "grid is NULL");
    if (n_points) *n_points = grid->g.n;
    if (cells_per_axis) *cells_per_axis = grid->g.nc;
    return TPCF_OK;
}

int tpcf_grid_points(tpcf_grid grid, uint32_t *xyz, float *w, int64_t *order, void *stream)
{
    if (!grid) return fail(TPCF_ERR_ARG, "grid is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = grid->g.n;
    if (n == 0) return TPCF_OK;
    if (xyz) CK(cudaMemcpy2DAsync(xyz, 12, grid->g.rec, 16, 12, n, cudaMemcpyDeviceToDevice, st));
    if (w) CK(cudaMemcpy2DAsync(w, 4, (const char *)grid->g.rec + 12, 16, 4, n, cudaMemcpyDeviceToDevice, st));
    if (order) CK(cudaMemcpyAsync(order, grid->g.order, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    return TPCF_OK;
}

int tpcf_accumulate_alm(tpcf_grid grid, const uint32_t *prim_xyz, const float *prim_w, int64_t n_prim,
                        const tpcf_config *cfg, double monopole_weight, float *alm, int32_t *counts, double *diag,
                        double *wsp, int64_t *pair_counts, void *stream)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!grid) return fail(TPCF_ERR_ARG, "grid is NULL");
    if (n_prim < 0) return fail(TPCF_ERR_ARG, "n_prim < 0");
    cudaStream_t st = (cudaStream_t)stream;
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    const int4 *prim = grid->g.rec;
    Scratch sc(st);
    int4 *packed = nullptr;
    if (prim_xyz) {
        if ((rc = sc.alloc(&packed, (size_t)n_prim, false))) return rc;
        CK(pack_records(prim_xyz, prim_w, n_prim, packed, ds->err, st));
        prim = packed;
    } else if (n_prim != grid->g.n) {
        return fail(TPCF_ERR_ARG, "n_prim must equal the grid size when prim_xyz is NULL");
    }
    rc = run_pairs(cfg, grid->g, prim, n_prim, false, monopole_weight, nullptr, monopole_weight >= 0.0, alm, counts,
                   diag, wsp, (unsigned long long *)pair_counts, st);
    return rc;
}

int tpcf_pair_counts(tpcf_grid grid, const uint32_t *prim_xyz, int64_t n_prim, const tpcf_config *cfg,
                     int32_t *counts, int64_t *pair_counts, void *stream)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!grid) return fail(TPCF_ERR_ARG, "grid is NULL");
    if (n_prim < 0) return fail(TPCF_ERR_ARG, "n_prim < 0");
    cudaStream_t st = (cudaStream_t)stream;
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    const int4 *prim = grid->g.rec;
    Scratch sc(st);
    int4 *packed = nullptr;
    if (prim_xyz) {
        if ((rc = sc.alloc(&packed, (size_t)n_prim, false))) return rc;
        CK(pack_records(prim_xyz, nullptr, n_prim, packed, ds->err, st));
        prim = packed;
    } else if (n_prim != grid->g.n) {
        return fail(TPCF_ERR_ARG, "n_prim must equal the grid size when prim_xyz is NULL");
    }
    return run_pairs(cfg, grid->g, prim, n_prim, true, -1.0, nullptr, false, nullptr, counts, nullptr, nullptr,
                     (unsigned long long *)pair_counts, st);
}

int tpcf_couple_multipoles(const float *alm, const float *prim_w, const int32_t *counts, int64_t n_prim,
                           const tpcf_config *cfg, const double *diag, const double *wsp, double *nnn,
                           int64_t *triplet_counts, void *stream)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!alm || !diag || !wsp || !nnn) return fail(TPCF_ERR_ARG, "alm, diag, wsp and nnn are required");
    if (n_prim < 0) return fail(TPCF_ERR_ARG, "n_prim < 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = cfg->n_bins;
    Scratch sc(st);
    unsigned long long *T = nullptr;
    if (triplet_counts && counts) {
        if ((rc = sc.alloc(&T, (size_t)nb * nb, true))) return rc;
    }
    rc = couple(cfg, alm, prim_w, counts, n_prim, diag, wsp, nnn, T, st);
    if (!rc && T) {
        cudaError_t e = i64_from_u64(T, triplet_counts, nb * nb, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "triplet counts");
    }
    return rc;
}

int tpcf_project(const tpcf_config *cfg, const double *nnn, const double *rrr, double *zeta, void *stream)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!nnn || !rrr || !zeta) return fail(TPCF_ERR_ARG, "nnn, rrr and zeta are required");
    return project(cfg, nnn, rrr, zeta, (cudaStream_t)stream);
}

int tpcf_estimate_3pcf(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                       const uint32_t *r_xyz, const float *r_w, int64_t nr, double *zeta, double *nnn_out,
                       double *rrr_out, int64_t *pair_counts, int64_t *triplet_counts, void *stream)
{
    return tpcf_estimate_3pcf_xi(cfg, d_xyz, d_w, nd, r_xyz, r_w, nr, zeta, nnn_out, rrr_out, pair_counts,
                                 triplet_counts, nullptr, stream);
}

int tpcf_estimate_3pcf_xi(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                          const uint32_t *r_xyz, const float *r_w, int64_t nr, double *zeta, double *nnn_out,
                          double *rrr_out, int64_t *pair_counts, int64_t *triplet_counts, double *xi,
                          void *stream)
{
    return estimate_impl(cfg, d_xyz, d_w, nd, r_xyz, r_w, nr, zeta, nnn_out, rrr_out, pair_counts, triplet_counts,
                         xi, false, nullptr, (cudaStream_t)stream);
}

int tpcf_estimate_3pcf_full_edge(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                                 const uint32_t *r_xyz, const float *r_w, int64_t nr, double *zeta, double *nnn,
                                 double *rrr_multipoles, double *xi, void *stream)
{
    if (nr < 1 || !r_xyz) return fail(TPCF_ERR_ARG, "the full edge correction needs explicit randoms");
    return estimate_impl(cfg, d_xyz, d_w, nd, r_xyz, r_w, nr, zeta, nnn, nullptr, nullptr, nullptr, xi, true,
                         rrr_multipoles, (cudaStream_t)stream);
}

int tpcf_partial_sizes(const tpcf_config *cfg, int64_t *n_double, int64_t *n_int64)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!n_double || !n_int64) return fail(TPCF_ERR_ARG, "outputs are required");
    const PartLayout PL = part_layout(cfg);
    *n_double = PL.nf;
    *n_int64 = PL.ni;
    return TPCF_OK;
}

int tpcf_estimate_3pcf_partial(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                               const uint32_t *r_xyz, const float *r_w, int64_t nr, const uint32_t *dp_xyz,
                               const float *dp_w, int64_t ndp, const uint32_t *rp_xyz, const float *rp_w, int64_t nrp,
                               double w_d_total, double w_r_total, int32_t weighted_randoms, double *part_f,
                               int64_t *part_i, void *stream)
{
    return partial_impl(cfg, d_xyz, d_w, nd, r_xyz, r_w, nr, dp_xyz, dp_w, ndp, rp_xyz, rp_w, nrp, w_d_total,
                        w_r_total, weighted_randoms, part_f, part_i, (cudaStream_t)stream);
}

int tpcf_estimate_3pcf_finish(const tpcf_config *cfg, double w_d_total, double w_r_total, int32_t explicit_randoms,
                              int32_t weighted_randoms, const double *part_f, const int64_t *part_i, double *zeta,
                              double *nnn, double *rrr, int64_t *pair_counts, int64_t *triplet_counts, double *xi,
                              void *stream)
{
    return finish_impl(cfg, w_d_total, w_r_total, explicit_randoms, weighted_randoms, part_f, part_i, zeta, nnn, rrr,
                       pair_counts, triplet_counts, xi, (cudaStream_t)stream);
}

int tpcf_estimate_3pcf_host(const tpcf_config *cfg, const uint32_t *d_xyz, const float *d_w, int64_t nd,
                            const uint32_t *r_xyz, const float *r_w, int64_t nr, double *zeta, double *nnn,
                            double *rrr, int64_t *pair_counts, int64_t *triplet_counts, void *stream)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!zeta || !d_xyz || nd < 1) return fail(TPCF_ERR_ARG, "zeta and data are required");
    if (nr < 0 || (nr > 0 && !r_xyz)) return fail(TPCF_ERR_ARG, "bad randoms");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    int32_t nm = 0;
    tpcf_multipole_count(cfg, &nm);
    const int nb = cfg->n_bins, L1 = cfg->l_max + 1;
    uint32_t *dx = nullptr, *rx = nullptr;
    float *dw = nullptr, *rw = nullptr;
    double *z = nullptr, *n3 = nullptr, *r3 = nullptr;
    int64_t *pc = nullptr, *tc = nullptr;
    if ((rc = sc.alloc(&dx, (size_t)nd * 3, false))) return rc;
    CK(cudaMemcpyAsync(dx, d_xyz, (size_t)nd * 12, cudaMemcpyHostToDevice, st));
    if (d_w) {
        if ((rc = sc.alloc(&dw, (size_t)nd, false))) return rc;
        CK(cudaMemcpyAsync(dw, d_w, (size_t)nd * 4, cudaMemcpyHostToDevice, st));
    }
    if (nr > 0) {
        if ((rc = sc.alloc(&rx, (size_t)nr * 3, false))) return rc;
        CK(cudaMemcpyAsync(rx, r_xyz, (size_t)nr * 12, cudaMemcpyHostToDevice, st));
        if (r_w) {
            if ((rc = sc.alloc(&rw, (size_t)nr, false))) return rc;
            CK(cudaMemcpyAsync(rw, r_w, (size_t)nr * 4, cudaMemcpyHostToDevice, st));
        }
    }
    if ((rc = sc.alloc(&z, (size_t)nm * nb * nb, false))) return rc;
    if (nnn && (rc = sc.alloc(&n3, (size_t)L1 * L1 * L1 * nb * nb, false))) return rc;
    if (rrr && (rc = sc.alloc(&r3, (size_t)nb * nb, false))) return rc;
    if (pair_counts && (rc = sc.alloc(&pc, (size_t)nb, false))) return rc;
    if (triplet_counts && (rc = sc.alloc(&tc, (size_t)nb * nb, false))) return rc;
    rc = tpcf_estimate_3pcf(cfg, dx, dw, nd, rx, rw, nr, z, n3, r3, pc, tc, stream);
    if (rc) return rc;
    CK(cudaMemcpyAsync(zeta, z, (size_t)nm * nb * nb * 8, cudaMemcpyDeviceToHost, st));
    if (nnn) CK(cudaMemcpyAsync(nnn, n3, (size_t)L1 * L1 * L1 * nb * nb * 8, cudaMemcpyDeviceToHost, st));
    if (rrr) CK(cudaMemcpyAsync(rrr, r3, (size_t)nb * nb * 8, cudaMemcpyDeviceToHost, st));
    if (pair_counts) CK(cudaMemcpyAsync(pair_counts, pc, (size_t)nb * 8, cudaMemcpyDeviceToHost, st));
    if (triplet_counts) CK(cudaMemcpyAsync(triplet_counts, tc, (size_t)nb * nb * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return tpcf_stream_status(stream);
}

int tpcf_batch_create(const tpcf_config *cfg, const int64_t *offsets, int32_t n_mocks, int64_t group_points,
                      tpcf_batch *out)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!out || !offsets || n_mocks < 1) return fail(TPCF_ERR_ARG, "need offsets and at least one mock");
    if (!cfg->periodic) return fail(TPCF_ERR_UNSUPPORTED, "batches use periodic boxes with analytic randoms");
    for (int k = 0; k < n_mocks; ++k)
        if (offsets[k + 1] < offsets[k] || offsets[0] != 0) return fail(TPCF_ERR_ARG, "offsets must start at 0 and not decrease");
    const int64_t n_total = offsets[n_mocks];
    if (n_total >= kMaxPoints) return fail(TPCF_ERR_ARG, "batch too large (total points < 2^28)");
    if (group_points < 0) return fail(TPCF_ERR_ARG, "group_points < 0");
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    tpcf_batch b = new tpcf_batch_s();
    b->cfg = *cfg;
    b->n_mocks = n_mocks;
    b->off.assign(offsets, offsets + n_mocks + 1);
    cudaGetDevice(&b->device);
    b->nc = choose_nc(cfg, std::max<int64_t>(1, n_total / n_mocks));
    const int nb = cfg->n_bins, L = cfg->l_max, L1 = L + 1;
    const int nlm = L1 * L1, ndiag = L1 * (L1 + 1) / 2;
    const int64_t ncell1 = (int64_t)b->nc * b->nc * b->nc;
    // groups of whole mocks: the per-point buffers of one group use at most half the free memory
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double per_point = (double)nb * nlm * 4 + nb * 4 + 4 + 4 + 64 * 2;
    int64_t cap = (int64_t)(0.5 * (double)free_b / per_point);
    if (group_points > 0) cap = std::min(cap, group_points);
    cap = std::max<int64_t>(cap, 1);
    b->group.push_back(0);
    int64_t gstart = 0;
    for (int k = 0; k < n_mocks; ++k) {
        const int64_t nk = offsets[k + 1] - offsets[k];
        if (nk > cap) {
            delete b;
            if (group_points > 0 && nk > group_points) return fail(TPCF_ERR_ARG, "mock %d exceeds group_points", k);
            return fail(TPCF_ERR_OOM, "mock %d does not fit in device memory", k);
        }
        if (offsets[k + 1] - gstart > cap || (int64_t)(k - b->group.back() + 1) * ncell1 >= ((int64_t)1 << 31)) {
            b->group.push_back(k);
            gstart = offsets[k];
        }
    }
    b->group.push_back(n_mocks);
    for (size_t g = 0; g + 1 < b->group.size(); ++g)
        b->max_group_points = std::max(b->max_group_points, offsets[b->group[g + 1]] - offsets[b->group[g]]);
    std::vector<int64_t> goff;
    for (size_t g = 0; g + 1 < b->group.size(); ++g)
        for (int k = b->group[g]; k <= b->group[g + 1]; ++k) goff.push_back(offsets[k] - offsets[b->group[g]]);
    std::vector<int64_t> all_sk;
    std::vector<int> all_ms;
    for (size_t g = 0; g + 1 < b->group.size(); ++g) {
        const int m0 = b->group[g], m1 = b->group[g + 1];
        std::vector<int64_t> sk;
        std::vector<int> ms;
        gram_batch_slices(offsets + m0, m1 - m0, nb, L, cfg->precision == TPCF_PREC_FP32, ds->sms, sk, ms);
        if (sk.empty()) {
            delete b;
            return fail(TPCF_ERR_UNSUPPORTED, "Gram: no tile plan for this shape");
        }
        b->gs_at.push_back(all_sk.size());
        b->gm_at.push_back(all_ms.size());
        b->gs_n.push_back((int)sk.size() - 1);
        all_sk.insert(all_sk.end(), sk.begin(), sk.end());
        all_ms.insert(all_ms.end(), ms.begin(), ms.end());
        b->max_group_mocks = std::max(b->max_group_mocks, m1 - m0);
    }
    // pair-stage tiles: the plan's primaries per tile at the mean mock density
    // (about 3000 pairs per tile), never straddling two mocks
    std::vector<int64_t> all_ts;
    {
        const double nbar = (double)n_total / n_mocks / (cfg->box * cfg->box * cfg->box);
        const double vol =
            4.0 / 3.0 * kPi * (cfg->r_max * cfg->r_max * cfg->r_max - cfg->r_min * cfg->r_min * cfg->r_min);
        int P = cfg->tile_primaries;
        if (P == 0) P = (int)std::lround(3000.0 / std::max(nbar * vol, 1.0));
        P = std::max(1, std::min(P, std::min(TPCF_MAX_TILE, std::max(1, 128 / nb))));
        b->tile_p = P;
        for (size_t g = 0; g + 1 < b->group.size(); ++g) {
            const int m0 = b->group[g], m1 = b->group[g + 1];
            const int64_t p0 = offsets[m0];
            b->gt_at.push_back(all_ts.size());
            if (P > 1) {
                const size_t first = all_ts.size();
                for (int k = m0; k < m1; ++k)
                    for (int64_t t = offsets[k]; t < offsets[k + 1]; t += P) all_ts.push_back(t - p0);
                all_ts.push_back(offsets[m1] - p0);
                b->gt_n.push_back((int64_t)(all_ts.size() - first) - 1);
            } else {
                b->gt_n.push_back(0);
            }
        }
    }
    std::vector<double> coef;
    std::vector<int> ml;
    projection_tables(cfg, coef, ml);
    b->n_mult = (int)ml.size() / 3;
    std::vector<double> gaunt((size_t)L1 * L1 * L1 * L1);
    self_term_table(L, gaunt.data());
    double r[TPCF_MAX_BINS + 1];
    unsigned long long E[TPCF_MAX_BINS + 1];
    edge_tables(cfg, E, r);
    std::vector<double> mono(nb);
    for (int q = 0; q < nb; ++q)
        mono[q] = 4.0 * kPi / 3.0 * (r[q + 1] * r[q + 1] * r[q + 1] - r[q] * r[q] * r[q]) / (cfg->box * cfg->box * cfg->box)
                  / std::sqrt(4.0 * kPi);
    const int64_t P = b->max_group_points;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes ? bytes : 8);
    };
    A((void **)&b->d_off, (n_mocks + 1) * sizeof(int64_t));
    A((void **)&b->d_goff, goff.size() * sizeof(int64_t));
    A((void **)&b->d_gaunt, gaunt.size() * sizeof(double));
    A((void **)&b->d_coef, coef.size() * sizeof(double));
    A((void **)&b->d_mults, ml.size() * sizeof(int));
    A((void **)&b->d_mono, nb * sizeof(double));
    A((void **)&b->d_tiles, 3 * (size_t)gram_tile_count(nb, L) * sizeof(int));
    A((void **)&b->rec_mock, P * sizeof(int32_t));
    A((void **)&b->alm, (size_t)P * nb * nlm * sizeof(float));
    A((void **)&b->wprim, P * sizeof(float));
    A((void **)&b->counts, (size_t)P * nb * sizeof(int32_t));
    A((void **)&b->wsum, n_mocks * sizeof(double));
    A((void **)&b->diag, (size_t)n_mocks * ndiag * nb * sizeof(double));
    A((void **)&b->wsp, (size_t)n_mocks * L1 * nb * sizeof(double));
    A((void **)&b->G, (size_t)b->max_group_mocks * gram_offset(nb, L, L + 1) * sizeof(double));
    A((void **)&b->d_slice_k, all_sk.size() * sizeof(int64_t));
    A((void **)&b->d_mslice, all_ms.size() * sizeof(int));
    A((void **)&b->d_tile_start, all_ts.size() * sizeof(int64_t));
    A((void **)&b->nnn, (size_t)L1 * L1 * L1 * nb * nb * sizeof(double));
    A((void **)&b->rrr, (size_t)nb * nb * sizeof(double));
    A((void **)&b->pairs, (size_t)n_mocks * nb * sizeof(unsigned long long));
    A((void **)&b->T, (size_t)n_mocks * nb * nb * sizeof(unsigned long long));
    A((void **)&b->d_status, (size_t)n_mocks * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, (size_t)n_mocks * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_off, offsets, (n_mocks + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_goff, goff.data(), goff.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_gaunt, gaunt.data(), gaunt.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_mults, ml.data(), ml.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_mono, mono.data(), nb * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_slice_k, all_sk.data(), all_sk.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_mslice, all_ms.data(), all_ms.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !all_ts.empty())
        e = cudaMemcpy(b->d_tile_start, all_ts.data(), all_ts.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        tpcf_batch_destroy(b);
        return cuda_fail(e, "batch buffers");
    }
    *out = b;
    return TPCF_OK;
}

int tpcf_batch_destroy(tpcf_batch b)
{
    if (!b) return TPCF_OK;
    cudaDeviceSynchronize();
    for (void *ptr : {(void *)b->d_off, (void *)b->d_goff, (void *)b->d_gaunt, (void *)b->d_coef, (void *)b->d_mults,
                      (void *)b->d_mono, (void *)b->d_tiles, (void *)b->rec_mock, (void *)b->alm, (void *)b->wprim,
                      (void *)b->counts, (void *)b->wsum, (void *)b->diag, (void *)b->wsp, (void *)b->G,
                      (void *)b->nnn, (void *)b->rrr, (void *)b->pairs, (void *)b->T, (void *)b->d_status,
                      (void *)b->d_slice_k, (void *)b->d_mslice, (void *)b->d_tile_start})
        if (ptr) cudaFree(ptr);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return TPCF_OK;
}

int tpcf_batch_info(tpcf_batch b, int32_t *n_groups, int32_t *cells_per_axis)
{
    if (!b) return fail(TPCF_ERR_ARG, "batch is NULL");
    if (n_groups) *n_groups = (int32_t)b->group.size() - 1;
    if (cells_per_axis) *cells_per_axis = b->nc;
    return TPCF_OK;
}

int tpcf_batch_run(tpcf_batch b, const uint32_t *xyz, const float *w, double *zeta, int64_t *triplet_counts,
                   void *stream)
{
    if (!b) return fail(TPCF_ERR_ARG, "batch is NULL");
    if (!xyz || !zeta) return fail(TPCF_ERR_ARG, "xyz and zeta are required");
    cudaStream_t st = (cudaStream_t)stream;
    DevState *ds;
    int rc = dev_state(&ds);
    if (rc) return rc;
    const tpcf_config *c = &b->cfg;
    const int nb = c->n_bins, L = c->l_max, L1 = L + 1;
    const int ndiag = L1 * (L1 + 1) / 2;
    const int64_t ncell1 = (int64_t)b->nc * b->nc * b->nc;
    CK(cudaMemsetAsync(b->diag, 0, (size_t)b->n_mocks * ndiag * nb * sizeof(double), st));
    CK(cudaMemsetAsync(b->wsp, 0, (size_t)b->n_mocks * L1 * nb * sizeof(double), st));
    CK(cudaMemsetAsync(b->pairs, 0, (size_t)b->n_mocks * nb * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(b->T, 0, (size_t)b->n_mocks * nb * nb * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(b->d_status, 0, (size_t)b->n_mocks * sizeof(int), st));
    size_t goff_at = 0;
    for (size_t g = 0; g + 1 < b->group.size(); ++g) {
        const int m0 = b->group[g], m1 = b->group[g + 1], nm = m1 - m0;
        const int64_t p0 = b->off[m0], np = b->off[m1] - p0;
        const int64_t *d_goff = b->d_goff + goff_at;
        goff_at += (size_t)nm + 1;
        const float *wg = w ? w + p0 : nullptr;
        CK(weight_sums_mocks(wg, d_goff, nm, b->wsum + m0, st));
        GridDev grid;
        CK(build_grid_batched_dev(xyz + 3 * p0, wg, np, d_goff, nm, b->nc, grid, b->rec_mock, ds->err, st,
                                  b->d_status + m0));
        BatchInfo bi{b->rec_mock, ncell1, b->wsum + m0, b->d_status + m0};
        if (b->tile_p > 1) {
            bi.P = b->tile_p;
            bi.tile_start = b->d_tile_start + b->gt_at[g];
            bi.n_tiles = b->gt_n[g];
        }
        rc = run_pairs(c, grid, grid.rec, np, false, 0.0, nullptr, true, b->alm, b->counts,
                       b->diag + (size_t)m0 * ndiag * nb, b->wsp + (size_t)m0 * L1 * nb, b->pairs + (size_t)m0 * nb,
                       st, &bi);
        if (rc) return rc;
        if (np > 0)
            CK(cudaMemcpy2DAsync(b->wprim, 4, (const char *)grid.rec + 12, 16, 4, np, cudaMemcpyDeviceToDevice, st));
        // every mock's Gram in one launch (slices never straddle two mocks)
        const int64_t gsz = gram_offset(nb, L, L + 1);
        CK(couple_gram_batched(b->alm, b->wprim, nm, b->d_slice_k + b->gs_at[g], b->gs_n[g], b->d_mslice + b->gm_at[g],
                               nb, L, c->precision, b->G, ds->err, ds->sms, st));
        for (int k = m0; k < m1; ++k) {
            const int64_t r0 = b->off[k] - p0, K = b->off[k + 1] - b->off[k];
            CK(assemble_nnn(b->G + (size_t)(k - m0) * gsz, b->diag + (size_t)k * ndiag * nb, b->wsp + (size_t)k * L1 * nb, nb, L,
                            c->remove_self, b->d_gaunt, b->nnn, st));
            CK(tpcf::triplet_counts(b->counts + (size_t)r0 * nb, K, nb, b->T + (size_t)k * nb * nb, st));
            CK(rrr_analytic(b->wsum + k, b->d_mono, nb, b->rrr, st));
            CK(project_zeta(b->nnn, b->rrr, nb, L, b->n_mult, b->d_coef, b->d_mults,
                            zeta + (size_t)k * b->n_mult * nb * nb, st));
        }
        free_grid_dev(grid, st);
    }
    if (triplet_counts) CK(i64_from_u64(b->T, triplet_counts, b->n_mocks * nb * nb, st));
    return TPCF_OK;
}

int tpcf_batch_run_graph(tpcf_batch b, const uint32_t *xyz, const float *w, double *zeta, int64_t *triplet_counts,
                         void *stream)
{
    if (!b) return fail(TPCF_ERR_ARG, "batch is NULL");
    const void *key[4] = {xyz, w, zeta, triplet_counts};
    if (b->exec && std::memcmp(key, b->gp, sizeof(key)) == 0) {
        CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
        return TPCF_OK;
    }
    // first use with these buffers: run eagerly (this also finishes every one-time
    // set-up), then record the same work on a private stream
    int rc = tpcf_batch_run(b, xyz, w, zeta, triplet_counts, stream);
    if (rc) return rc;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (!b->cap) CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    rc = tpcf_batch_run(b, xyz, w, zeta, triplet_counts, b->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch capture");
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(e2, "batch graph instantiation");
    }
    std::memcpy(b->gp, key, sizeof(key));
    return TPCF_OK;
}

int tpcf_batch_status(tpcf_batch b, int32_t *status, void *stream)
{
    if (!b || !status) return fail(TPCF_ERR_ARG, "batch and status are required");
    std::vector<int> h(b->n_mocks, 0);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMemcpy(h.data(), b->d_status, (size_t)b->n_mocks * sizeof(int), cudaMemcpyDeviceToHost));
    for (int k = 0; k < b->n_mocks; ++k) {
        int v = TPCF_OK;
        if (b->off[k + 1] - b->off[k] < 2) v = TPCF_ERR_ARG;   // no pair: the estimate is 0 / 0
        else if (h[k] == DEV_ERR_DATA) v = TPCF_ERR_DATA;
        else if (h[k]) v = TPCF_ERR_CUDA;
        status[k] = v;
    }
    return TPCF_OK;
}

int tpcf_estimate_3pcf_batched(const tpcf_config *cfg, const uint32_t *xyz, const float *w, const int64_t *offsets,
                               int32_t n_mocks, double *zeta, int64_t *triplet_counts, int32_t *status_per_mock,
                               void *stream)
{
    tpcf_batch b = nullptr;
    int rc = tpcf_batch_create(cfg, offsets, n_mocks, 0, &b);
    if (rc) return rc;
    rc = tpcf_batch_run(b, xyz, w, zeta, triplet_counts, stream);
    if (!rc) rc = tpcf_stream_status(stream);
    if (!rc && status_per_mock) rc = tpcf_batch_status(b, status_per_mock, stream);
    tpcf_batch_destroy(b);
    return rc;
}

int tpcf_autotune(const tpcf_config *cfg, const uint32_t *xyz, const float *w, int64_t n, void *stream,
                  tpcf_config *tuned)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (!tuned || !xyz || n < 1 || n >= kMaxPoints) return fail(TPCF_ERR_ARG, "autotune needs a catalogue and an output");
    cudaStream_t st = (cudaStream_t)stream;
    DevState *ds;
    if ((rc = dev_state(&ds))) return rc;
    *tuned = *cfg;
    const int nb = cfg->n_bins, L1 = cfg->l_max + 1;
    // sampled primaries per trial: enough tiles per CTA (a few dozen at the
    // catalogue sizes of a covariance batch) that the launch's ramp and tail do
    // not decide the timing
    const int64_t ns = std::min<int64_t>(n, 32768);
    const int64_t stride = std::max<int64_t>(1, n / ns);
    Scratch sc(st);
    float *alm = nullptr;
    int32_t *cnt = nullptr;
    double *diag = nullptr, *wsp = nullptr;
    unsigned long long *pc = nullptr;
    int4 *prim = nullptr;
    if ((rc = sc.alloc(&alm, (size_t)ns * nb * L1 * L1, false)) || (rc = sc.alloc(&cnt, (size_t)ns * nb, false)) ||
        (rc = sc.alloc(&diag, (size_t)L1 * (L1 + 1) / 2 * nb, false)) || (rc = sc.alloc(&wsp, (size_t)L1 * nb, false)) ||
        (rc = sc.alloc(&pc, (size_t)nb, false)) || (rc = sc.alloc(&prim, (size_t)ns, false)))
        return rc;
    // timing events, destroyed on every return path
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    float best = 1e30f;
    const int divs[] = {2, 3, 4, 5, 6};
    const int tiles_all[] = {1, 2, 4};
    const int tiles_fixed[] = {cfg->tile_primaries};
    const bool fixed_tile = cfg->tile_primaries > 0;   // the caller fixed the tile size
    const int chunks[] = {12288, 15360, 24576};
    for (int dv : divs) {
        tpcf_config t = *cfg;
        t.cell_div = dv;
        const Plan pl = make_plan(&t, n, n);
        if (pl.s != dv) continue;   // the box cannot hold this many cells per r_max
        GridDev g;
        Scratch gs(st);   // releases this cell size's grid on every path
        gs.own(g);
        CK(build_grid_dev(xyz, w, n, nullptr, nullptr, 0, nullptr, pl.nc, g, ds->err, st));
        CK(cudaMemcpy2DAsync(prim, 16, g.rec, 16 * stride, 16, ns, cudaMemcpyDeviceToDevice, st));
        for (int ti = 0; ti < (fixed_tile ? 1 : 3); ++ti) {
            const int tp = fixed_tile ? tiles_fixed[0] : tiles_all[ti];
            if (tp * nb > 128) continue;
            for (int ch : chunks) {
                t.tile_primaries = tp;
                t.chunk = ch;
                float ms = 1e30f;
                for (int rep = 0; rep < 4; ++rep) {   // the first run warms up; best of three
                    cudaEventRecord(e0, st);
                    rc = run_pairs(&t, g, prim, ns, false, -1.0, nullptr, false, alm, cnt, diag, wsp, pc, st);
                    cudaEventRecord(e1, st);
                    if (rc) break;
                    cudaEventSynchronize(e1);
                    float x = 0.f;
                    cudaEventElapsedTime(&x, e0, e1);
                    if (rep > 0) ms = std::min(ms, x);
                }
                if (rc) break;
                if (ms < best) {
                    best = ms;
                    tuned->cell_div = dv;
                    tuned->tile_primaries = tp;
                    tuned->chunk = ch;
                }
            }
            if (rc) break;
        }
        if (rc) break;
    }
    cudaStreamSynchronize(st);
    return rc;
}

int tpcf_covariance(const double *src, int64_t n_mocks, int64_t stride, const int64_t *idx, int64_t n_dv,
                    double *mean, double *cov, void *stream)
{
    if (!src || !mean || !cov) return fail(TPCF_ERR_ARG, "src, mean and cov are required");
    if (n_mocks < 2) return fail(TPCF_ERR_ARG, "need at least two mocks (got %lld)", (long long)n_mocks);
    if (n_dv < 1 || stride < 1) return fail(TPCF_ERR_ARG, "n_dv and stride must be positive");
    if (!idx && n_dv > stride) return fail(TPCF_ERR_ARG, "without idx, n_dv must not exceed stride");
    if (n_dv > (int64_t)1 << 20) return fail(TPCF_ERR_ARG, "data vector longer than 2^20");
    DevState *ds;
    int rc = dev_state(&ds);
    if (rc) return rc;
    CK(covariance(src, n_mocks, stride, idx, n_dv, mean, cov, ds->err, (cudaStream_t)stream));
    return TPCF_OK;
}

int tpcf_covariance_factors(int64_t n_mocks, int64_t n_dv, int64_t n_params, double *hartlap, double *m1)
{
    if (n_dv < 1 || n_params < 0) return fail(TPCF_ERR_ARG, "n_dv >= 1 and n_params >= 0 required");
    if (n_mocks <= n_dv + 4)
        return fail(TPCF_ERR_ARG, "need n_mocks > n_dv + 4 (got %lld mocks for %lld entries)", (long long)n_mocks,
                    (long long)n_dv);
    const double nm = (double)n_mocks, nd = (double)n_dv, np = (double)n_params;
    if (hartlap) *hartlap = (nm - nd - 2.0) / (nm - 1.0);
    const double q = (nm - nd - 1.0) * (nm - nd - 4.0);
    const double A = 2.0 / q, B = (nm - nd - 2.0) / q;
    if (m1) *m1 = (1.0 + B * (nd - np)) / (1.0 + A + B * (np + 1.0));
    return TPCF_OK;
}

int tpcf_data_vector_index(const tpcf_config *cfg, const int32_t *l1l2L, int32_t n_sel, int32_t eta, int64_t *idx,
                           int64_t cap, int64_t *n_out)
{
    int rc = check_config(cfg);
    if (rc) return rc;
    if (n_sel < 0 || (n_sel > 0 && !l1l2L) || eta < 0 || !n_out)
        return fail(TPCF_ERR_ARG, "bad selection arguments");
    std::vector<int> ml;
    multipole_list(cfg, ml);
    const int nm = (int)ml.size() / 3, nb = cfg->n_bins;
    int64_t n = 0;
    for (int s = 0; s < n_sel; ++s) {
        int k = -1;
        for (int q = 0; q < nm; ++q)
            if (ml[3 * q] == l1l2L[3 * s] && ml[3 * q + 1] == l1l2L[3 * s + 1] && ml[3 * q + 2] == l1l2L[3 * s + 2])
                k = q;
        if (k < 0)
            return fail(TPCF_ERR_ARG, "multipole (%d %d %d) is not measured by this configuration", l1l2L[3 * s],
                        l1l2L[3 * s + 1], l1l2L[3 * s + 2]);
        for (int b1 = 0; b1 < nb; ++b1)
            for (int b2 = b1 + eta; b2 < nb; ++b2) {
                if (idx && n < cap) idx[n] = ((int64_t)k * nb + b1) * nb + b2;
                ++n;
            }
    }
    *n_out = n;
    if (idx && n > cap) return fail(TPCF_ERR_ARG, "idx holds %lld entries, %lld needed", (long long)cap, (long long)n);
    return TPCF_OK;
}

int tpcf_check_rsqrt(int64_t n, uint64_t seed, double *stats, void *stream)
{
    if (n < 1 || !stats) return fail(TPCF_ERR_ARG, "n >= 1 and host stats[5] required");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    double *d = nullptr;
    unsigned long long *mu = nullptr;
    int rc;
    if ((rc = sc.alloc(&d, 5, true))) return rc;
    if ((rc = sc.alloc(&mu, 1, true))) return rc;
    CK(check_rsqrt(n, (unsigned long long)seed, d, mu, st));
    double h[5];
    unsigned long long hm = 0;
    CK(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hm, mu, sizeof(hm), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    stats[0] = (double)hm;
    stats[1] = h[1] / (double)n;
    stats[2] = h[2] / (double)n;
    stats[3] = h[3] / (double)n;
    stats[4] = h[4] / (double)n;
    return TPCF_OK;
}

int tpcf_measure_fp32_peak(double *tflops, void *stream)
{
    if (!tflops) return fail(TPCF_ERR_ARG, "host tflops[2] required");
    cudaStream_t st = (cudaStream_t)stream;
    DevState *ds;
    int rc = dev_state(&ds);
    if (rc) return rc;
    Scratch sc(st);
    float *sink = nullptr;
    if ((rc = sc.alloc(&sink, 256, false))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    const int blocks = ds->sms * 8, iters = 16384;
    for (int paired = 0; paired < 2 && e == cudaSuccess; ++paired) {
        float best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms up
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = ffma_peak(paired != 0, blocks, iters, sink, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        tflops[paired] = 16.0 * iters * 256.0 * blocks / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    CK(e);
    return TPCF_OK;
}

int tpcf_trim_memory(void)
{
    int d = 0;
    CK(cudaGetDevice(&d));
    if (d < 0 || d >= 64) return fail(TPCF_ERR_CUDA, "device index out of range");
    const unsigned long long ctx = context_id();
    std::lock_guard<std::mutex> lk(g_pool_mu);
    ScratchPool &sp = g_pool[d];
    if (!sp.pool || sp.ctx != ctx) return TPCF_OK;
    CK(cudaMemPoolTrimTo(sp.pool, 0));
    return TPCF_OK;
}

int tpcf_stream_status(void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    DevState *ds;
    int rc = dev_state(&ds);
    if (rc) return rc;
    int h = 0;
    CK(cudaMemcpy(&h, ds->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CK(cudaMemset(ds->err, 0, sizeof(int)));
        if (h == DEV_ERR_DATA) return fail(TPCF_ERR_DATA, "non-finite weight in the input");
        if (h == DEV_ERR_TIMEOUT) return fail(TPCF_ERR_TIMEOUT, "a bounded device wait ran out");
        if (h == DEV_ERR_INDEX) return fail(TPCF_ERR_DATA, "a data-vector index is outside the source row");
        return fail(TPCF_ERR_CUDA, "device error code %d", h);
    }
    return TPCF_OK;
}

}  // extern "C"
