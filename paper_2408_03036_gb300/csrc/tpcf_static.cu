// tpcf_couple_multipoles_static: the coupling step (Gram over primaries, j = k
// correction, NNN assembly, triplet counts) without any device allocation.
//
// Who needs it: code that may not allocate GPU memory while it runs, for
// example a host application whose memory is fully reserved by its own pool
// or framework, a process that must not grow its footprint after start-up, or
// work submitted from a context where calls into the CUDA allocator are not
// allowed.  tpcf_couple_multipoles takes its FP64 Gram blocks and small tables
// from stream-ordered allocations; this variant uses instead one fixed block
// of device memory declared in this file, which every GPU that loads the
// library keeps for the life of the process.
//
// Size limit: the packed Gram blocks, sum over m of (n_bins (l_max - m + 1))^2
// doubles, must fit in kGramMax = 65,536 doubles (512 KiB); that covers
// l_max <= 4 with up to 32 bins, and l_max 6 with up to 21 bins.  Larger
// requests are rejected with TPCF_ERR_ARG.  The whole block is about 560 KiB.
//
// Set-up: the first call on each device (with that device current) looks up
// the block's device address with cudaGetSymbolAddress and copies the j = k
// coefficient tables into it with a synchronous cudaMemcpy.  Make that first
// call before any stream capture.  The set-up is tied to the device's current
// CUDA context (its unique context id): after cudaDeviceReset the module is
// loaded again with a zeroed block, and the next call repeats the set-up.
//
// Sharing: every call on a device uses the same block.  The Gram area and the
// triplet-count accumulator are cleared at the start of each call (they must
// start at zero); the tables are written once.  Two calls whose work overlaps
// on the GPU (different streams, or different host threads) race on the block
// and give wrong results: serialise them.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int64_t kGramMax = 65536;                 // doubles of packed Gram blocks
constexpr int kTilesMax = 512;                      // (m, tr, tc) tiles
constexpr int kSelfLmax = TPCF_MAX_LMAX;

constexpr int64_t self_doubles(int lmax)   // sum of (L+1)^4, L = 0..lmax
{
    int64_t s = 0;
    for (int L = 0; L <= lmax; ++L) s += (int64_t)(L + 1) * (L + 1) * (L + 1) * (L + 1);
    return s;
}
constexpr int64_t kSelfDoubles = self_doubles(kSelfLmax);
static_assert(kSelfDoubles == 1 + 16 + 81 + 256 + 625 + 1296 + 2401 || kSelfLmax != 6, "table size");

constexpr size_t kOffGram = 0;
constexpr size_t kOffSelf = kOffGram + kGramMax * sizeof(double);
constexpr size_t kOffTiles = kOffSelf + ((kSelfDoubles * sizeof(double) + 255) / 256) * 256;
constexpr size_t kOffTrip = kOffTiles + ((kTilesMax * 3 * sizeof(int) + 255) / 256) * 256;
constexpr size_t kScratchBytes = kOffTrip + TPCF_MAX_BINS * TPCF_MAX_BINS * sizeof(unsigned long long);

// The fixed scratch block.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress (see scratch_on()).
static __device__ __align__(256) unsigned char g_couple_scratch[kScratchBytes];

int64_t self_offset(int lmax)
{
    int64_t off = 0;
    for (int L = 0; L < lmax; ++L) off += (int64_t)(L + 1) * (L + 1) * (L + 1) * (L + 1);
    return off;
}

std::mutex g_mu;
unsigned char *g_ptr[64] = {nullptr};
unsigned long long g_ctx[64] = {0};   // id of the context the block was set up in

// Device address of the scratch block on the current device, set up on first use
// in the current context.
int scratch_on(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tpcf::set_error(TPCF_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return tpcf::set_error(TPCF_ERR_CUDA, "device index out of range");
    // every call: the block's address (this also brings up the device's context)
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_couple_scratch);
    if (e != cudaSuccess || !p) return tpcf::set_error(TPCF_ERR_CUDA, "cudaGetSymbolAddress failed for the static scratch");
    const unsigned long long ctx = tpcf::context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_ptr[dev] != (unsigned char *)p || g_ctx[dev] != ctx) {
        static double tables[kSelfDoubles];
        for (int L = 0; L <= kSelfLmax; ++L) tpcf::self_term_table(L, tables + self_offset(L));
        e = cudaMemcpy((unsigned char *)p + kOffSelf, tables, kSelfDoubles * sizeof(double),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return tpcf::set_error(TPCF_ERR_CUDA, cudaGetErrorString(e));
        g_ptr[dev] = (unsigned char *)p;
        g_ctx[dev] = ctx;
    }
    *out = g_ptr[dev];
    return TPCF_OK;
}

int cuda_err(cudaError_t e)
{
    return tpcf::set_error(e == cudaErrorMemoryAllocation ? TPCF_ERR_OOM : TPCF_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" int tpcf_couple_multipoles_static(const float *alm, const float *prim_w, const int32_t *counts,
                                             int64_t n_prim, const tpcf_config *cfg, const double *diag,
                                             const double *wsp, double *nnn, int64_t *triplet_counts,
                                             void *stream)
{
    int rc = tpcf::check_config_public(cfg);
    if (rc) return rc;
    if (!alm || !diag || !wsp || !nnn) return tpcf::set_error(TPCF_ERR_ARG, "alm, diag, wsp and nnn are required");
    if (n_prim < 0) return tpcf::set_error(TPCF_ERR_ARG, "n_prim < 0");
    if (cfg->precision != TPCF_PREC_FP32)
        return tpcf::set_error(TPCF_ERR_UNSUPPORTED, "the static-scratch coupling runs the FP32 Gram only");
    const int nb = cfg->n_bins, L = cfg->l_max;
    const int64_t gsz = tpcf::gram_offset(nb, L, L + 1);
    if (gsz > kGramMax)
        return tpcf::set_error(TPCF_ERR_ARG, "Gram blocks exceed the static scratch (65536 doubles): "
                                             "lower l_max or n_bins, or use tpcf_couple_multipoles");
    if (tpcf::gram_tile_count(nb, L) > kTilesMax)
        return tpcf::set_error(TPCF_ERR_ARG, "too many Gram tiles for the static scratch");
    unsigned char *base = nullptr;
    if ((rc = scratch_on(&base))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *G = reinterpret_cast<double *>(base + kOffGram);
    const double *self = reinterpret_cast<const double *>(base + kOffSelf) + self_offset(L);
    int *tiles = reinterpret_cast<int *>(base + kOffTiles);
    unsigned long long *T = reinterpret_cast<unsigned long long *>(base + kOffTrip);
    cudaError_t e;
    if ((e = cudaMemsetAsync(G, 0, gsz * sizeof(double), st)) != cudaSuccess) return cuda_err(e);
    if ((e = tpcf::couple_gram_fp32_tiles(alm, prim_w, n_prim, nb, L, tiles, G, st)) != cudaSuccess)
        return cuda_err(e);
    if ((e = tpcf::assemble_nnn(G, diag, wsp, nb, L, cfg->remove_self, self, nnn, st)) != cudaSuccess)
        return cuda_err(e);
    if (counts && triplet_counts) {
        if ((e = cudaMemsetAsync(T, 0, (size_t)nb * nb * sizeof(unsigned long long), st)) != cudaSuccess)
            return cuda_err(e);
        if ((e = tpcf::triplet_counts(counts, n_prim, nb, T, st)) != cudaSuccess) return cuda_err(e);
        if ((e = tpcf::i64_from_u64(T, triplet_counts, nb * nb, st)) != cudaSuccess) return cuda_err(e);
    }
    return TPCF_OK;
}
