// Nodes sorted by grid cell, per term of order <= 2 (built once per plan).
//
// The adjoint spreads y_j psi(n x_j - l) onto the oversampled grid of every
// term (stacked adjoint after the error remark, Sec. 3).  Nodes whose grid
// position has the same integer part (the same cell) touch the same window
// footprint, so with the nodes of a term in cell order the spread sums a
// cell's contributions in registers and adds them to the grid once per cell.
// This file builds that order: a counting sort of the node indices by cell,
// one term per blockIdx.y, and per sorted node a 16-byte record with the
// window arguments, the grid offset of its cell and its original index.
// The order inside a cell is left to the atomics of the scatter; it changes
// only the rounding order of the sums.  FP64 plans sort by the bases of their
// window tables (records carry only the cell offset and the node index).
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

__device__ __forceinline__ int cell_bins(const Term &T) {
    return T.order == 3 ? T.n * T.n * T.n : (T.order == 2 ? T.n * T.n : T.n);
}

// cell of a node: (i_row0 * n + i_row1) * n + i_col over the term's coordinates
__device__ __forceinline__ int cell_of(const Term &T, float xr, float xr1, float xc) {
    float t;
    const int fc = grid_pos(xc, T.n, t);
    if (T.order == 1) return fc;
    const int fr = grid_pos(xr, T.n, t);
    if (T.order == 2) return fr * T.n + fc;
    const int fr1 = grid_pos(xr1, T.n, t);
    return (fr * T.n + fr1) * T.n + fc;
}

// counts[slot][cell] += nodes of the block's range in that cell
__global__ void k_cell_count(const Term *terms, const float *x, long long M, int *counts, int max_bins) {
    extern __shared__ int hist[];
    const Term &T = terms[blockIdx.y];
    if (T.sort_slot < 0) return;
    const int nb = cell_bins(T);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const float *xr = x + (long long)(T.order >= 2 ? T.row0 : T.col) * M;
    const float *xr1 = x + (long long)(T.order == 3 ? T.row1 : T.col) * M;
    const float *xc = x + (long long)T.col * M;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M; j += (long long)gridDim.x * blockDim.x)
        atomicAdd(&hist[cell_of(T, xr[j], xr1[j], xc[j])], 1);
    __syncthreads();
    int *cnt = counts + (long long)T.sort_slot * max_bins;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (hist[b]) atomicAdd(&cnt[b], hist[b]);
}

// exclusive prefix sum of counts[slot][0..bins) in place, one block per term
__global__ void k_cell_scan(const Term *terms, int *counts, int max_bins) {
    __shared__ int wsum[32];
    const Term &T = terms[blockIdx.x];
    if (T.sort_slot < 0) return;
    const int nb = cell_bins(T);
    int *c = counts + (long long)T.sort_slot * max_bins;
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += c[b];
    // inclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = v - local + (wid > 0 ? wsum[wid - 1] : 0);   // exclusive prefix of this thread's range
    for (int b = b0; b < b1; ++b) {
        const int t = c[b];
        c[b] = run;
        run += t;
    }
}

// scatter: every node goes to the next free place of its cell, as a record.
// Order <= 2: (2 tau_row - 1, 2 tau_col - 1, first-tap grid offset, original
// index).  Order 3, two records: (2 tau_row0 - 1, 2 tau_row1 - 1, 2 tau_col - 1,
// original index) and the cell's grid indices and cell number (i_row0, i_row1,
// i_col, (i_row0 n + i_row1) n + i_col).
__global__ void k_cell_scatter(const Term *terms, const float *x, long long M, int *cursor, int max_bins,
                               float4 *srec) {
    const Term &T = terms[blockIdx.y];
    if (T.sort_slot < 0) return;
    const float *xr = x + (long long)(T.order >= 2 ? T.row0 : T.col) * M;
    const float *xr1 = x + (long long)(T.order == 3 ? T.row1 : T.col) * M;
    const float *xc = x + (long long)T.col * M;
    int *cur = cursor + (long long)T.sort_slot * max_bins;
    float4 *dst = srec + (long long)T.sort_slot * M;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M;
         j += (long long)gridDim.x * blockDim.x) {
        float tc, tr = 0.f, tr1 = 0.f;
        const int fc = grid_pos(xc[j], T.n, tc);
        int fr = 0, fr1 = 0;
        if (T.order >= 2) fr = grid_pos(xr[j], T.n, tr);
        if (T.order == 3) fr1 = grid_pos(xr1[j], T.n, tr1);
        if (T.order == 3) {
            const int pos = atomicAdd(&cur[(fr * T.n + fr1) * T.n + fc], 1);
            dst[2 * pos] = make_float4(2.f * tr - 1.f, 2.f * tr1 - 1.f, 2.f * tc - 1.f, __int_as_float((int)j));
            dst[2 * pos + 1] = make_float4(__int_as_float(fr), __int_as_float(fr1), __int_as_float(fc),
                                           __int_as_float((fr * T.n + fr1) * T.n + fc));
        } else {
            const int pos = atomicAdd(&cur[fr * (T.order == 2 ? T.n : 0) + fc], 1);
            const int off = fr * T.stride + fc;
            dst[pos] = make_float4(T.order == 2 ? 2.f * tr - 1.f : 0.f, 2.f * tc - 1.f, __int_as_float(off),
                                   __int_as_float((int)j));
        }
    }
}

// FP64 plans: the cell of a node is that of its window-table bases (the
// spread adds at exactly those bases); records (0, 0, offset, index)
__device__ __forceinline__ int cell_of64(const Term &T, const int *wb, long long M, long long j, int &off) {
    const int fc = wb[(long long)T.slot_c * M + j];
    if (T.order != 2) {
        off = fc;
        return fc;
    }
    const int fr = wb[(long long)T.slot_r0 * M + j];
    off = fr * T.stride + fc;
    return fr * T.n + fc;
}

__global__ void k_cell_count64(const Term *terms, const int *wb, long long M, int *counts, int max_bins) {
    extern __shared__ int hist[];
    const Term &T = terms[blockIdx.y];
    if (T.sort_slot < 0) return;
    const int nb = cell_bins(T);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M; j += (long long)gridDim.x * blockDim.x) {
        int off;
        atomicAdd(&hist[cell_of64(T, wb, M, j, off)], 1);
    }
    __syncthreads();
    int *cnt = counts + (long long)T.sort_slot * max_bins;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (hist[b]) atomicAdd(&cnt[b], hist[b]);
}

__global__ void k_cell_scatter64(const Term *terms, const int *wb, long long M, int *cursor, int max_bins,
                                 float4 *srec) {
    const Term &T = terms[blockIdx.y];
    if (T.sort_slot < 0) return;
    int *cur = cursor + (long long)T.sort_slot * max_bins;
    float4 *dst = srec + (long long)T.sort_slot * M;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M;
         j += (long long)gridDim.x * blockDim.x) {
        int off;
        const int pos = atomicAdd(&cur[cell_of64(T, wb, M, j, off)], 1);
        dst[pos] = make_float4(0.f, 0.f, __int_as_float(off), __int_as_float((int)j));
    }
}

int sort_nodes_by_cell(Plan &p) {
    if (!p.srec || p.n_sorted == 0 || p.M == 0) return ANOVA_OK;
    int max_bins = 1;
    for (int s = 0; s < p.n_terms; ++s) {
        const Term &T = p.h_terms[s];
        if (T.sort_slot >= 0)
            max_bins = std::max(max_bins, T.order == 3 ? T.n * T.n * T.n : (T.order == 2 ? T.n * T.n : T.n));
    }
    int *counts = nullptr;
    cudaError_t e = plan_malloc(&counts, sizeof(int) * (size_t)p.n_sorted * max_bins);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t hist_bytes = sizeof(int) * (size_t)max_bins;
    const bool f64 = p.precision == ANOVA_PREC_F64;
    if (hist_bytes > 48 * 1024)
        e = cudaFuncSetAttribute(f64 ? (const void *)k_cell_count64 : (const void *)k_cell_count,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_bytes);
    const int bx = (int)std::max<long long>(1, std::min<long long>(64, (p.M + 4095) / 4096));
    const dim3 grid(bx, p.n_terms);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)p.n_sorted * max_bins, p.stream);
    if (e == cudaSuccess) {
        if (f64)
            k_cell_count64<<<grid, 256, hist_bytes, p.stream>>>(p.terms, p.wb64, p.M, counts, max_bins);
        else
            k_cell_count<<<grid, 256, hist_bytes, p.stream>>>(p.terms, (const float *)p.x, p.M, counts, max_bins);
        k_cell_scan<<<p.n_terms, 1024, 0, p.stream>>>(p.terms, counts, max_bins);
        if (f64)
            k_cell_scatter64<<<grid, 256, 0, p.stream>>>(p.terms, p.wb64, p.M, counts, max_bins, p.srec);
        else
            k_cell_scatter<<<grid, 256, 0, p.stream>>>(p.terms, (const float *)p.x, p.M, counts, max_bins,
                                                       p.srec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    cudaFree(counts);
    return cuda_status(e);
}

}  // namespace agft
