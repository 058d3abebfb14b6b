// Instantiation of the pair-stage kernels for one l_max, given at compile time
// as TPCF_LMAX (the build compiles this file once per l_max, 0..6, so the
// unrolled variants compile in parallel).  l_max = 0 also carries the integer
// count kernel of the random-only pass.
#include "k_pairs.cuh"

#ifndef TPCF_LMAX
#error "compile once per l_max with -DTPCF_LMAX=<0..6>"
#endif
#define TPCF_CAT2(a, b) a##b
#define TPCF_CAT(a, b) TPCF_CAT2(a, b)

namespace tpcf {

namespace {

constexpr int kL = TPCF_LMAX;

// COUNTS: integer pair counts only (k_counts); otherwise the queued harmonic kernel,
// with the line of sight along z or (VLOS) from the observer to each primary.
template <bool COUNTS, bool VLOS>
cudaError_t prepare()
{
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const unsigned long long bit = device_bit();
    if (attr_done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    // the largest dynamic shared memory, and the carveout that gives shared memory
    // all of the unified L1 / shared storage, so that as many CTAs are resident as
    // registers and shared memory allow (the driver's default carveout choice can
    // leave room for fewer)
    cudaError_t e;
    if constexpr (COUNTS) {
        e = cudaFuncSetAttribute(k_counts<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_counts<0>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
    } else {
        e = cudaFuncSetAttribute(k_pairs_q<kL, VLOS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024 - kPairsStaticSmem - (VLOS ? kVlosStaticSmem : 0));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_pairs_q<kL, VLOS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
    }
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit, std::memory_order_acq_rel);
    return cudaSuccess;
}

template <bool COUNTS, bool VLOS = false>
cudaError_t launch_one(const PairParams &p, const HarmTables &h, int grid, int block, size_t smem, cudaStream_t st)
{
    cudaError_t e = prepare<COUNTS, VLOS>();
    if (e != cudaSuccess) return e;
    if constexpr (COUNTS) k_counts<0><<<grid, block, smem, st>>>(p);
    else k_pairs_q<kL, VLOS><<<grid, block, smem, st>>>(p, h);
    note_launch();
    return cudaGetLastError();
}

template <bool COUNTS, bool VLOS = false>
int per_sm_one(int block, size_t smem)
{
    if (prepare<COUNTS, VLOS>() != cudaSuccess) return 1;
    int n = 0;
    cudaError_t e;
    if constexpr (COUNTS) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_counts<0>, block, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pairs_q<kL, VLOS>, block, smem);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace

cudaError_t TPCF_CAT(launch_pairs_l, TPCF_LMAX)(bool counts_only, const PairParams &p, const HarmTables &h,
                                                 int grid, int block, size_t smem, cudaStream_t st)
{
    if (counts_only) {
        if constexpr (kL == 0) return launch_one<true>(p, h, grid, block, smem, st);
        return cudaErrorInvalidValue;
    }
    if (p.vlos) return launch_one<false, true>(p, h, grid, block, smem, st);
    return launch_one<false>(p, h, grid, block, smem, st);
}

size_t TPCF_CAT(pairs_smem_l, TPCF_LMAX)(bool counts_only, int P, int nb, int s, int chunk, int block)
{
    if (counts_only) return (size_t)make_cmap(P, nb, s).total;
    return (size_t)make_qmap<kL>(P, nb, s, chunk, block).total;
}

// Resident CTAs per SM for a launch with `smem` bytes of dynamic shared memory
// (the occupancy calculator on the kernel's registers and shared memory).
int TPCF_CAT(pairs_per_sm_l, TPCF_LMAX)(bool counts_only, bool vlos, int block, size_t smem)
{
    if (counts_only) return kL == 0 ? per_sm_one<true>(block, smem) : 1;
    return vlos ? per_sm_one<false, true>(block, smem) : per_sm_one<false>(block, smem);
}

}  // namespace tpcf
