// Coupling over primaries on the 5th-generation tensor cores (tcgen05, TMEM).
//
// G_m = sum_i w_i (Re v_i Re v_i^T + Im v_i Im v_i^T) for every azimuthal m
// (Eq. measured_mult summed over primaries, Sec. 4.2 of arXiv:2408.03036), with
// v_i the per-primary harmonic sums a_l^m[b], l = m..l_max, b = 0..n_b-1.  As a
// matrix product D = A B^T with K running over (primary, real/imaginary part):
// A = (w v)^T rows, B = v^T rows, both K-major.
//
// Split precision: every operand value x is written as hi + lo in the MMA type
// (bf16 or tf32) and D accumulates hi_A hi_B + hi_A lo_B + lo_A hi_B in FP32 in
// tensor memory; the dropped lo_A lo_B term is below 2^-16 (bf16) or 2^-22 (tf32)
// of each product.  Partial sums are moved to FP64 every kFlushK K-rows.
//
// One CTA owns one m block (one or two 128-row tiles of D, N = n_m padded to a
// multiple of 16 columns) for one slice of primaries.  Operand tiles of 16 K
// entries (bf16) or 8 (tf32) are staged in shared memory in the canonical
// no-swizzle K-major layout (core matrices of 8 rows x 16 bytes; core matrices
// adjacent in K are 128 bytes apart, adjacent 8-row groups 256 bytes apart),
// double-buffered; one elected thread issues the MMAs and commits them to an
// mbarrier per stage.  Every wait is bounded; a timeout latches an error flag,
// releases tensor memory and returns.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

namespace {

constexpr int kThreads = 256;
constexpr int kRowTile = 128;                 // M of every MMA (TMEM lanes)
constexpr int kStageBytesRow = 32;            // one K step = 32 bytes per operand row
constexpr long long kWaitLimit = 1ll << 26;   // polls of an mbarrier before giving up
constexpr int kFlushK = 1024;                 // K rows accumulated in FP32 per flush

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start, leading (K) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B type code `ab` (bf16 = 1 in
// kind::f16, tf32 = 2 in kind::tf32), both K-major, N and M.
__device__ __forceinline__ uint32_t make_idesc(uint32_t ab, int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;                 // D format: F32
    d |= ab << 7;                 // A format
    d |= ab << 10;                // B format
    d |= (uint32_t)(N >> 3) << 17;
    d |= (uint32_t)(M >> 4) << 24;
    return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Splits x into hi + lo in the MMA type, returned as the 16-bit (bf16) or
// 32-bit (tf32, low 13 mantissa bits zero) storage words.
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

// Byte offset of element (row, k) of a staged tile (k < 16 for bf16, < 8 for tf32).
template <bool TF32>
__device__ __forceinline__ uint32_t tile_off(int row, int k)
{
    const int per = TF32 ? 4 : 8;   // elements per 16-byte core-matrix row
    const int esz = TF32 ? 4 : 2;
    return (uint32_t)(((row >> 3) * 2 + k / per) * 128 + (row & 7) * 16 + (k % per) * esz);
}

struct TcParams {
    const float *alm;
    const float *w;
    int64_t K;            // primaries
    int nb, lmax;
    int64_t per_slice;    // primaries per slice
    int n_slices;
    double *partial;      // [n_slices][sum over m of rt_m * 128 * N_m]
    int *err;
};

__device__ __forceinline__ int harm_index(int l, int m, int part)
{
    return l * l + (m == 0 ? 0 : 2 * m - 1 + part);
}

__host__ __device__ inline int pad16(int n) { return (n + 15) / 16 * 16; }

__host__ __device__ inline int64_t partial_offset(int nb, int lmax, int m)
{
    int64_t off = 0;
    for (int k = 0; k < m; ++k) {
        const int n = nb * (lmax - k + 1);
        off += (int64_t)((n + kRowTile - 1) / kRowTile) * kRowTile * pad16(n);
    }
    return off;
}

template <bool TF32>
__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(const TcParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int m = blockIdx.x;
    const int slice = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nb = p.nb, lmax = p.lmax;
    const int nlm = (lmax + 1) * (lmax + 1);
    const int n_m = nb * (lmax - m + 1);
    const int RT = (n_m + kRowTile - 1) / kRowTile;   // row tiles (1 or 2)
    const int N = pad16(n_m);
    const int parts = m == 0 ? 1 : 2;
    const int KS = TF32 ? 8 : 16;                      // K entries per MMA step
    const int64_t i0 = (int64_t)slice * p.per_slice;
    const int64_t i1 = min(p.K, i0 + p.per_slice);
    const int64_t krows = (i1 > i0) ? (i1 - i0) * parts : 0;
    const int64_t nsteps = (krows + KS - 1) / KS;

    // stage layout: A_hi, A_lo (RT*128 rows), B_hi, B_lo (N rows); 32 bytes per row
    const uint32_t a_bytes = (uint32_t)RT * kRowTile * kStageBytesRow;
    const uint32_t b_bytes = (uint32_t)N * kStageBytesRow;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    unsigned char *stage0 = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);   // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 2 * stage_bytes + 16);
    int *s_abort = reinterpret_cast<int *>(smem + 2 * stage_bytes + 20);

    uint32_t ncols = 32;
    while (ncols < (uint32_t)(RT * N)) ncols <<= 1;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, kRowTile, N);
    double *part_out = p.partial + (int64_t)slice * partial_offset(nb, lmax, lmax + 1) + partial_offset(nb, lmax, m);

    uint32_t phase[2] = {0u, 0u};
    bool used[2] = {false, false};
    bool ok = true;
    int64_t since_flush = 0;
    bool acc_on = false;

    // FP32 tensor-memory partials -> this slice's FP64 partial block, then restart accumulation
    auto flush = [&](bool first) {
        // all MMAs committed so far must have landed
        for (int s = 0; s < 2; ++s)
            if (used[s]) {
                if (tid == 0 && !mbar_wait(&bars[s], phase[s] ^ 1u)) *s_abort = 1;
            }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (*s_abort) return;
        if (warp < 4) {
            const int lane_base = 32 * warp;
            const int row_in_tile = lane_base + (tid & 31);
            for (int rt = 0; rt < RT; ++rt) {
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(rt * N + c0), v);
                    double *dst = part_out + ((int64_t)(rt * kRowTile + row_in_tile)) * N + c0;
#pragma unroll
                    for (int q = 0; q < 16; ++q) dst[q] = first ? (double)v[q] : dst[q] + (double)v[q];
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };

    bool first_flush = true;
    for (int64_t st = 0; st < nsteps && ok; ++st) {
        const int s = (int)(st & 1);
        unsigned char *stg = stage0 + s * stage_bytes;
        // the MMAs that last read this stage must be done before it is rewritten
        if (used[s]) {
            if (tid == 0 && !mbar_wait(&bars[s], phase[s] ^ 1u)) *s_abort = 1;
        }
        __syncthreads();
        if (*s_abort) { ok = false; break; }
        // stage KS K-entries: element (row, k) for rows < RT*128 (A) and < N (B)
        const int64_t k0 = st * KS;
        const int rows_a = RT * kRowTile;
        for (int e = tid; e < rows_a * KS; e += kThreads) {
            const int row = e / KS, k = e % KS;
            const int64_t kk = k0 + k;
            float x = 0.f, wx = 0.f;
            if (row < n_m && kk < krows) {
                const int64_t i = i0 + kk / parts;
                const int part = (int)(kk % parts);
                const int l = m + row / nb, b = row % nb;
                x = p.alm[(i * nb + b) * nlm + harm_index(l, m, part)];
                wx = p.w ? p.w[i] * x : x;
            }
            const uint32_t off = tile_off<TF32>(row, k);
            if (TF32) {
                uint32_t h, lo;
                split_tf32(wx, h, lo);
                *reinterpret_cast<uint32_t *>(stg + off) = h;
                *reinterpret_cast<uint32_t *>(stg + a_bytes + off) = lo;
                if (row < N) {
                    split_tf32(x, h, lo);
                    *reinterpret_cast<uint32_t *>(stg + 2 * a_bytes + off) = h;
                    *reinterpret_cast<uint32_t *>(stg + 2 * a_bytes + b_bytes + off) = lo;
                }
            } else {
                uint16_t h, lo;
                split_bf16(wx, h, lo);
                *reinterpret_cast<uint16_t *>(stg + off) = h;
                *reinterpret_cast<uint16_t *>(stg + a_bytes + off) = lo;
                if (row < N) {
                    split_bf16(x, h, lo);
                    *reinterpret_cast<uint16_t *>(stg + 2 * a_bytes + off) = h;
                    *reinterpret_cast<uint16_t *>(stg + 2 * a_bytes + b_bytes + off) = lo;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(stg);
            const uint64_t bhi = make_desc(base + 2 * a_bytes, 128, 256);
            const uint64_t blo = make_desc(base + 2 * a_bytes + b_bytes, 128, 256);
            for (int rt = 0; rt < RT; ++rt) {
                const uint32_t aoff = (uint32_t)rt * kRowTile * kStageBytesRow;
                const uint64_t ahi = make_desc(base + aoff, 128, 256);
                const uint64_t alo = make_desc(base + a_bytes + aoff, 128, 256);
                const uint32_t d = tmem + (uint32_t)(rt * N);
                mma_issue<TF32>(d, ahi, bhi, idesc, acc_on ? 1u : 0u);
                mma_issue<TF32>(d, ahi, blo, idesc, 1u);
                mma_issue<TF32>(d, alo, bhi, idesc, 1u);
            }
            mma_commit(&bars[s]);
        }
        used[s] = true;
        phase[s] ^= 1u;
        acc_on = true;
        since_flush += KS;
        if (since_flush >= kFlushK) {
            flush(first_flush);
            first_flush = false;
            since_flush = 0;
            acc_on = false;
            used[0] = used[1] = false;
            if (*s_abort) { ok = false; break; }
        }
    }
    if (ok && acc_on) {
        flush(first_flush);
        first_flush = false;
    }
    if (first_flush && ok) {   // empty slice: the partial block must still read as zero
        for (int64_t q = tid; q < (int64_t)RT * kRowTile * N; q += kThreads) part_out[q] = 0.0;
    }
    if (*s_abort || !ok) {
        if (tid == 0) atomicCAS(p.err, 0, DEV_ERR_TIMEOUT);
        // wait (bounded) for anything still in flight before releasing TMEM
        for (int s = 0; s < 2; ++s)
            if (used[s] && tid == 0) mbar_wait(&bars[s], phase[s] ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// G_m[row][col] = sum over slices of the partial blocks (rows/cols < n_m).
__global__ void k_gram_tc_reduce(const double *partial, int n_slices, int nb, int lmax, double *G)
{
    const int64_t per_slice = partial_offset(nb, lmax, lmax + 1);
    const int64_t total = gram_offset(nb, lmax, lmax + 1);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int m = 0;
        while (m < lmax && idx >= gram_offset(nb, lmax, m + 1)) ++m;
        const int n_m = nb * (lmax - m + 1);
        const int64_t r = idx - gram_offset(nb, lmax, m);
        const int row = (int)(r / n_m), col = (int)(r % n_m);
        const int64_t src = partial_offset(nb, lmax, m) + (int64_t)row * pad16(n_m) + col;
        double s = 0.0;
        for (int sl = 0; sl < n_slices; ++sl) s += partial[sl * per_slice + src];
        G[idx] = s;
    }
}

}  // namespace

size_t gram_tc_smem(int nb, int lmax)
{
    size_t best = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int n_m = nb * (lmax - m + 1);
        const int RT = (n_m + kRowTile - 1) / kRowTile;
        const size_t stage = 2 * (size_t)RT * kRowTile * kStageBytesRow + 2 * (size_t)pad16(n_m) * kStageBytesRow;
        best = stage > best ? stage : best;
    }
    return 2 * best + 64;
}

cudaError_t couple_gram_tc(const float *alm, const float *w, int64_t K, int nb, int lmax, bool tf32, double *G,
                           int *err, int sms, cudaStream_t st)
{
    // TMEM columns: RT * N per CTA must fit 512; two 128-row tiles of N <= 256
    for (int m = 0; m <= lmax; ++m) {
        const int n_m = nb * (lmax - m + 1);
        const int RT = (n_m + kRowTile - 1) / kRowTile;
        if (RT > 2 || RT * pad16(n_m) > 512 || pad16(n_m) > 256) return cudaErrorInvalidValue;
    }
    if (K <= 0) return cudaMemsetAsync(G, 0, gram_offset(nb, lmax, lmax + 1) * sizeof(double), st);
    int slices = (sms + lmax) / (lmax + 1);
    if (slices < 1) slices = 1;
    const int64_t min_per = 1024;
    if ((K + slices - 1) / slices < min_per) slices = (int)((K + min_per - 1) / min_per);
    if (slices < 1) slices = 1;
    TcParams p;
    p.alm = alm;
    p.w = w;
    p.K = K;
    p.nb = nb;
    p.lmax = lmax;
    p.per_slice = (K + slices - 1) / slices;
    p.n_slices = slices;
    p.err = err;
    const int64_t per = partial_offset(nb, lmax, lmax + 1);
    // at least 116 KB so that one CTA owns an SM: tensor-memory allocations never wait
    size_t smem = gram_tc_smem(nb, lmax);
    if (smem < 116 * 1024) smem = 116 * 1024;
    static std::atomic<unsigned long long> attr_done[2];   // devices whose attribute is set
    const unsigned long long bit = device_bit();
    cudaError_t e;
    if (!(attr_done[tf32].load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(tf32 ? k_gram_tc<true> : k_gram_tc<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr_done[tf32].fetch_or(bit, std::memory_order_acq_rel);
    }
    e = cudaMallocAsync((void **)&p.partial, (size_t)slices * per * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const dim3 grid(lmax + 1, slices);
    if (tf32) k_gram_tc<true><<<grid, kThreads, smem, st>>>(p);
    else k_gram_tc<false><<<grid, kThreads, smem, st>>>(p);
    note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const int64_t tot = gram_offset(nb, lmax, lmax + 1);
        int g = (int)((tot + 255) / 256);
        if (g > 4096) g = 4096;
        k_gram_tc_reduce<<<g, 256, 0, st>>>(p.partial, slices, nb, lmax, G);
        note_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(p.partial, st);
    return e;
}

}  // namespace tpcf
