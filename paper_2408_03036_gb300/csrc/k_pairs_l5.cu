// Instantiation of the pair-stage kernel for l_max = 5 (one translation unit
// per l_max so the unrolled variants compile in parallel).
#include "k_pairs.cuh"

namespace tpcf {

// COUNTS: integer pair counts only (k_counts); otherwise the queued harmonic kernel,
// with the line of sight along z or (VLOS) from the observer to each primary.
template <int LMAX, bool COUNTS, bool VLOS = false>
static cudaError_t launch_one(const PairParams &p, const HarmTables &h, int grid, int block,
                              size_t smem, cudaStream_t st)
{
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const unsigned long long bit = device_bit();
    if (!(attr_done.load(std::memory_order_acquire) & bit)) {
        cudaError_t e;
        if constexpr (COUNTS)
            e = cudaFuncSetAttribute(k_counts<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        else
            e = cudaFuncSetAttribute(k_pairs_q<LMAX, VLOS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024 - (VLOS ? kVlosStaticSmem : 0));
        if (e != cudaSuccess) return e;
        attr_done.fetch_or(bit, std::memory_order_acq_rel);
    }
    if constexpr (COUNTS) k_counts<0><<<grid, block, smem, st>>>(p);
    else k_pairs_q<LMAX, VLOS><<<grid, block, smem, st>>>(p, h);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_pairs_l5(bool counts_only, const PairParams &p, const HarmTables &h, int grid,
                             int block, size_t smem, cudaStream_t st)
{
    if (counts_only) return cudaErrorInvalidValue;
    if (p.vlos) return launch_one<5, false, true>(p, h, grid, block, smem, st);
    return launch_one<5, false>(p, h, grid, block, smem, st);
}

size_t pairs_smem_l5(bool counts_only, int P, int nb, int s, int chunk, int block)
{
    if (counts_only) return (size_t)make_cmap(P, nb, s).total;
    return (size_t)make_qmap<5>(P, nb, s, chunk, block).total;
}

}  // namespace tpcf
