// Cell list of a catalogue (the linked-list partition of arXiv:2408.03036,
// Sec. 4.1, built on the GPU as a counting sort by cell).
//
// cell(u) = floor(u * nc / 2^32) per axis, linear cell index
// (cz * nc + cy) * nc + cx.  Points are stored as 16-byte records
// {x, y, z, float_as_int(w)}, grouped by cell, with cell_start[c] the first
// record of cell c.  Within a cell, records keep their input order (a stable
// rank computed from per-cell atomic counters followed by a per-cell sort of
// the input indices), so a grid is bit-identical from run to run.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace tpcf {

namespace {

__device__ __forceinline__ int cell1(uint32_t u, int nc)
{
    return (int)(((unsigned long long)u * (unsigned long long)nc) >> 32);
}

// Per-point cell index and cell histogram.  Points [0, n) come from (xyz, w),
// points [n, n + n2) from (xyz2, w2) with weights scaled by -W_D/W_R
// (the data-minus-random field) when wsums = {W_D, W_R} is given.
__global__ void k_cell_hist(const uint32_t *__restrict__ xyz, const float *__restrict__ w, int64_t n,
                            const uint32_t *__restrict__ xyz2, const float *__restrict__ w2, int64_t n2,
                            const double *__restrict__ wsums, int nc, int32_t *__restrict__ cid,
                            int32_t *__restrict__ hist, int4 *__restrict__ tmp, int *err)
{
    const int64_t tot = n + n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x, y, z;
        float wt;
        if (i < n) {
            x = xyz[3 * i]; y = xyz[3 * i + 1]; z = xyz[3 * i + 2];
            wt = w ? w[i] : 1.0f;
        } else {
            const int64_t j = i - n;
            x = xyz2[3 * j]; y = xyz2[3 * j + 1]; z = xyz2[3 * j + 2];
            wt = w2 ? w2[j] : 1.0f;
            if (wsums) wt = (float)(-(wsums[0] / wsums[1]) * (double)wt);
        }
        if (!(wt == wt) || isinf(wt)) atomicCAS(err, 0, DEV_ERR_DATA);
        const int c = (cell1(z, nc) * nc + cell1(y, nc)) * nc + cell1(x, nc);
        cid[i] = c;
        tmp[i] = make_int4((int)x, (int)y, (int)z, __float_as_int(wt));
        atomicAdd(&hist[c], 1);
    }
}

// Single-CTA exclusive scan of hist[0..ncell) into start[0..ncell], also
// copying start into cursor.
__global__ void k_scan_cells(const int32_t *__restrict__ hist, int64_t ncell, int32_t *__restrict__ start,
                             int32_t *__restrict__ cursor)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ncell; base += T) {
        const int64_t i = base + tid;
        const int32_t v = i < ncell ? hist[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t y = lane < (T >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t t = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += t;
            }
            wsum[lane] = y;
        }
        __syncthreads();
        const int32_t excl = carry + (warp ? wsum[warp - 1] : 0) + x - v;
        if (i < ncell) {
            start[i] = excl;
            cursor[i] = excl;
        }
        __syncthreads();
        if (tid == T - 1) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) start[ncell] = carry;
}

// Scatter of input indices into cell order (order within a cell is arbitrary here).
__global__ void k_scatter_idx(const int32_t *__restrict__ cid, int64_t tot, int32_t *__restrict__ cursor,
                              int64_t *__restrict__ order)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&cursor[cid[i]], 1);
        order[pos] = i;
    }
}

// Orders every cell's points by x, ties by input index (one warp per cell: each
// point's rank is the number of points of its cell with a smaller key, the keys
// passed round the warp 32 at a time), then gathers the records.  Deterministic
// output; the x order lets the pair stage trim a row of cells to the sphere at
// record granularity.
__global__ void k_sort_cells(const int32_t *__restrict__ start, int64_t ncell, int64_t *__restrict__ order,
                             const int4 *__restrict__ tmp, int4 *__restrict__ rec, int64_t *__restrict__ scratch)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = wid; c < ncell; c += nwarps) {
        const int a = start[c], b = start[c + 1];
        const int n = b - a;
        if (n <= 0) continue;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const int64_t v = i < n ? order[a + i] : 0;
            const uint32_t xv = i < n ? (uint32_t)tmp[v].x : 0u;
            int rank = 0;
            for (int j0 = 0; j0 < n; j0 += 32) {
                const int j = j0 + lane;
                const int64_t u = j < n ? order[a + j] : 0;
                const uint32_t xu = j < n ? (uint32_t)tmp[u].x : 0u;
                const int cnt = min(32, n - j0);
                for (int q = 0; q < cnt; ++q) {
                    const uint32_t xq = __shfl_sync(FULL, xu, q);
                    const int64_t uq = __shfl_sync(FULL, u, q);
                    rank += (xq < xv || (xq == xv && uq < v)) ? 1 : 0;
                }
            }
            if (i < n) scratch[a + rank] = v;
        }
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const int64_t v = scratch[a + i];
            order[a + i] = v;
            rec[a + i] = tmp[v];
        }
        __syncwarp();
    }
}

// records (x, y, z, w) of n points; with wsums = {W_D, W_R} the weights become
// -(W_D / W_R) w, the random part of the data-minus-random field (as in the grid)
__global__ void k_pack(const uint32_t *__restrict__ xyz, const float *__restrict__ w, int64_t n,
                       const double *__restrict__ wsums, int4 *__restrict__ out, int *err)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float wt = w ? w[i] : 1.0f;
        if (wsums) wt = (float)(-(wsums[0] / wsums[1]) * (double)wt);
        if (!(wt == wt) || isinf(wt)) atomicCAS(err, 0, DEV_ERR_DATA);
        out[i] = make_int4((int)xyz[3 * i], (int)xyz[3 * i + 1], (int)xyz[3 * i + 2], __float_as_int(wt));
    }
}

__global__ void k_wsum(const float *__restrict__ w1, int64_t n1, const float *__restrict__ w2, int64_t n2,
                       double *out)
{
    __shared__ double red[2][32];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1 + n2;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n1) s1 += w1 ? (double)w1[i] : 1.0;
        else s2 += w2 ? (double)w2[i - n1] : 1.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) { red[0][warp] = s1; red[1][warp] = s2; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s1 = lane < nw ? red[0][lane] : 0.0;
        s2 = lane < nw ? red[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            atomicAdd(out, s1);
            atomicAdd(out + 1, s2);
        }
    }
}

// Mock of every point from the offsets (binary search), cell index offset by
// mock * ncell, histogram; weights copied as given.
__global__ void k_cell_hist_batched(const uint32_t *__restrict__ xyz, const float *__restrict__ w, int64_t n,
                                    const int64_t *__restrict__ offsets, int n_mocks, int nc, int64_t ncell,
                                    int32_t *__restrict__ cid, int32_t *__restrict__ mock_of,
                                    int32_t *__restrict__ hist, int4 *__restrict__ tmp, int *err,
                                    int *__restrict__ mock_status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_mocks - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const uint32_t x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        const float wt = w ? w[i] : 1.0f;
        if (!(wt == wt) || isinf(wt)) atomicCAS(mock_status ? mock_status + lo : err, 0, DEV_ERR_DATA);
        const int64_t c = (int64_t)lo * ncell + (cell1(z, nc) * nc + cell1(y, nc)) * nc + cell1(x, nc);
        cid[i] = (int32_t)c;
        mock_of[i] = lo;
        tmp[i] = make_int4((int)x, (int)y, (int)z, __float_as_int(wt));
        atomicAdd(&hist[c], 1);
    }
}

// Mock id of every record in grid order.
__global__ void k_mock_of_rec(const int64_t *__restrict__ order, const int32_t *__restrict__ mock_of, int64_t n,
                              int32_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mock_of[order[i]];
}

// W per mock: one block per mock.
// *out += number of weights that differ from 1.
__global__ void k_count_not_one(const float *__restrict__ w, int64_t n, int *out)
{
    int c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += w[i] != 1.0f;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// out[0] += weights with the sign bit set (negative, -0, negative NaN), out[1] += weights > 0
__global__ void k_weight_signs(const float *__restrict__ w, int64_t n, int *out)
{
    int neg = 0, pos = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = w[i];
        neg += (int)(__float_as_uint(v) >> 31);
        pos += v > 0.0f;
    }
    neg = __reduce_add_sync(0xffffffffu, neg);
    pos = __reduce_add_sync(0xffffffffu, pos);
    if ((threadIdx.x & 31) == 0) {
        if (neg) atomicAdd(out, neg);
        if (pos) atomicAdd(out + 1, pos);
    }
}

__global__ void k_wsum_mocks(const float *__restrict__ w, const int64_t *__restrict__ offsets, double *out)
{
    __shared__ double red[32];
    const int mk = blockIdx.x;
    double s = 0.0;
    for (int64_t i = offsets[mk] + threadIdx.x; i < offsets[mk + 1]; i += blockDim.x) s += w ? (double)w[i] : 1.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (warp == 0) {
        s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[mk] = s;
    }
}

int grid_blocks(int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > sm_count() * 16) b = sm_count() * 16;
    return (int)b;
}

}  // namespace

namespace {

// Temporaries of a grid build, released in stream order on every return path.
struct Temps {
    cudaStream_t st;
    void *p[8] = {};
    int n = 0;
    explicit Temps(cudaStream_t s) : st(s) {}
    Temps(const Temps &) = delete;
    Temps &operator=(const Temps &) = delete;
    template <class T>
    cudaError_t alloc(T **q, size_t bytes)
    {
        const cudaError_t e = scratch_malloc((void **)q, bytes, st);
        if (e == cudaSuccess) p[n++] = *q;
        return e;
    }
    ~Temps()
    {
        for (int i = 0; i < n; ++i) cudaFreeAsync(p[i], st);
    }
};

}  // namespace

cudaError_t build_grid_dev(const uint32_t *xyz, const float *w, int64_t n,
                           const uint32_t *xyz2, const float *w2, int64_t n2, const double *wsums,
                           int nc, GridDev &g, int *err, cudaStream_t st)
{
    const int64_t tot = n + n2;
    const int64_t ncell = (int64_t)nc * nc * nc;
    g.n = tot;
    g.nc = nc;
    g.ncell = ncell;
    cudaError_t e;
    Temps tmps(st);
    int32_t *cid = nullptr, *hist = nullptr, *cursor = nullptr;
    int4 *tmp = nullptr;
    int64_t *scratch = nullptr;
    const int64_t alloc_n = tot > 0 ? tot : 1;
    if ((e = scratch_malloc((void **)&g.rec, alloc_n * sizeof(int4), st)) != cudaSuccess) return e;
    if ((e = scratch_malloc((void **)&g.order, alloc_n * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = scratch_malloc((void **)&g.cell_start, (ncell + 1) * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = tmps.alloc(&cid, alloc_n * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&tmp, alloc_n * sizeof(int4))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&scratch, alloc_n * sizeof(int64_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&hist, ncell * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&cursor, ncell * sizeof(int32_t))) != cudaSuccess) return e;
    cudaMemsetAsync(hist, 0, ncell * sizeof(int32_t), st);
    const int B = 256;
    if (tot > 0) {
        k_cell_hist<<<grid_blocks(tot, B), B, 0, st>>>(xyz, w, n, xyz2, w2, n2, wsums, nc, cid, hist, tmp, err);
        note_launch();
    }
    k_scan_cells<<<1, 1024, 0, st>>>(hist, ncell, g.cell_start, cursor);
    note_launch();
    if (tot > 0) {
        k_scatter_idx<<<grid_blocks(tot, B), B, 0, st>>>(cid, tot, cursor, g.order);
        k_sort_cells<<<grid_blocks(ncell * 32, B), B, 0, st>>>(g.cell_start, ncell, g.order, tmp, g.rec, scratch);
        note_launch(2);
    }
    e = cudaGetLastError();
    return e;
}

cudaError_t build_grid_batched_dev(const uint32_t *xyz, const float *w, int64_t n, const int64_t *d_offsets,
                                   int n_mocks, int nc, GridDev &g, int32_t *rec_mock, int *err, cudaStream_t st,
                                   int *mock_status)
{
    const int64_t ncell1 = (int64_t)nc * nc * nc;
    const int64_t ncell = ncell1 * n_mocks;
    g.n = n;
    g.nc = nc;
    g.ncell = ncell;
    cudaError_t e;
    Temps tmps(st);
    int32_t *cid = nullptr, *hist = nullptr, *cursor = nullptr, *mock_of = nullptr;
    int4 *tmp = nullptr;
    int64_t *scratch = nullptr;
    const int64_t alloc_n = n > 0 ? n : 1;
    if ((e = scratch_malloc((void **)&g.rec, alloc_n * sizeof(int4), st)) != cudaSuccess) return e;
    if ((e = scratch_malloc((void **)&g.order, alloc_n * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = scratch_malloc((void **)&g.cell_start, (ncell + 1) * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = tmps.alloc(&cid, alloc_n * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&mock_of, alloc_n * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&tmp, alloc_n * sizeof(int4))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&scratch, alloc_n * sizeof(int64_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&hist, ncell * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = tmps.alloc(&cursor, ncell * sizeof(int32_t))) != cudaSuccess) return e;
    cudaMemsetAsync(hist, 0, ncell * sizeof(int32_t), st);
    const int B = 256;
    if (n > 0) {
        k_cell_hist_batched<<<grid_blocks(n, B), B, 0, st>>>(xyz, w, n, d_offsets, n_mocks, nc, ncell1, cid, mock_of,
                                                            hist, tmp, err, mock_status);
        note_launch();
    }
    k_scan_cells<<<1, 1024, 0, st>>>(hist, ncell, g.cell_start, cursor);
    note_launch();
    if (n > 0) {
        k_scatter_idx<<<grid_blocks(n, B), B, 0, st>>>(cid, n, cursor, g.order);
        k_sort_cells<<<grid_blocks(ncell * 32, B), B, 0, st>>>(g.cell_start, ncell, g.order, tmp, g.rec, scratch);
        k_mock_of_rec<<<grid_blocks(n, B), B, 0, st>>>(g.order, mock_of, n, rec_mock);
        note_launch(3);
    }
    e = cudaGetLastError();
    return e;
}

cudaError_t count_not_one(const float *w, int64_t n, int *out, cudaStream_t st)
{
    if (n > 0) {
        k_count_not_one<<<grid_blocks(n, 256), 256, 0, st>>>(w, n, out);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t weight_signs(const float *w, int64_t n, int *out, cudaStream_t st)
{
    if (n > 0) {
        k_weight_signs<<<grid_blocks(n, 256), 256, 0, st>>>(w, n, out);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t weight_sums_mocks(const float *w, const int64_t *d_offsets, int n_mocks, double *out, cudaStream_t st)
{
    if (n_mocks > 0) {
        k_wsum_mocks<<<n_mocks, 256, 0, st>>>(w, d_offsets, out);
        note_launch();
    }
    return cudaGetLastError();
}

void free_grid_dev(GridDev &g, cudaStream_t st)
{
    if (g.rec) cudaFreeAsync(g.rec, st);
    if (g.order) cudaFreeAsync(g.order, st);
    if (g.cell_start) cudaFreeAsync(g.cell_start, st);
    g.rec = nullptr;
    g.order = nullptr;
    g.cell_start = nullptr;
}

cudaError_t pack_records(const uint32_t *xyz, const float *w, int64_t n, int4 *out, int *err, cudaStream_t st,
                         const double *wsums)
{
    if (n > 0) {
        k_pack<<<grid_blocks(n, 256), 256, 0, st>>>(xyz, w, n, wsums, out, err);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t weight_sums(const float *w1, int64_t n1, const float *w2, int64_t n2, double *out2, cudaStream_t st)
{
    cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    if (n1 + n2 > 0) {
        k_wsum<<<grid_blocks(n1 + n2, 256), 256, 0, st>>>(w1, n1, w2, n2, out2);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace tpcf
