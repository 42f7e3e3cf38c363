// Adjoint grouped transform fhat = F^H y (stacked adjoint after the error
// remark, Sec. 3), FP32.
//
//   1. spread: work items (term, node chunk) from a global queue.  An item
//      accumulates y_j times the window into a shared-memory copy of the
//      term's stored grid (halos included), then writes it to partial grid z
//      of the term (z = chunk index).  With cell-sorted node records the sums
//      of one grid cell's nodes are formed first -- on the tensor cores
//      (spread_mma_f32, spread3_mma_f32) or in registers on the CUDA cores
//      (spread_f32 sorted items, spread3_f32) -- and added to the shared grid
//      once per cell; without records every node's window is added with
//      shared-memory atomics.
//   2. reduce_partials: grid = sum_z partials[z] in a fixed order.
//   3. adjoint_post: per term, fold the halos back onto the periodic grid, FFT
//      with sign -, multiply by the deconvolution factors and crop the block
//      (I_N minus {0})^{|u|}.
//   4. empty-set terms: sum_j y_j by a two-stage reduction.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

// shared-memory float reduction without a returned value
__device__ __forceinline__ void red_add(float *addr, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(smem_addr(addr)), "f"(v) : "memory");
}

__device__ __forceinline__ int freq_index_a(int q, int N) { return q < N / 2 ? q - N / 2 : q - N / 2 + 1; }

enum { SK_STAGED = 0, SK_ORDER3 = 1, SK_MMA = 2, SK_MMA3 = 3 };
// the order-1/2 tensor-core spread: 12 warps per CTA, 2 CTAs per SM (80
// registers); two grid copies per SM leave each warp room for deep rings
constexpr int SPREAD_MMA_THREADS = 384;
constexpr int SPREAD_MMA_CTAS_PER_SM = 2;

constexpr int SP_CH = 512;   // nodes staged per block of a work item (order 1/2: SP_CH or SP_CH / 2)

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// staging area after the grid: the larger of the unsorted layout
// (float4 [2][SP]) and the sorted one (float4 [3][SP] node records, float2
// [2][SP] values of y), SP nodes per block
__host__ __device__ constexpr size_t sp_stage_bytes(int sp) { return (size_t)sp * (3 * 16 + 2 * 8); }
// third-order items (spread3_f32): 8 warp runs of 32 nodes, two records each
constexpr size_t SP3_STAGE_BYTES = 3 * 256 * 32 + 2 * 256 * 8;


// shared memory of spread_f32 (o3 = false, sp nodes per block) or spread3_f32:
// grid, node blocks, item slot
size_t spread_smem_bytes(long long max_grid_bytes, bool o3, int sp) {
    return (size_t)max_grid_bytes + (o3 ? SP3_STAGE_BYTES : sp_stage_bytes(sp)) + 16;
}

// CTAs per SM that shared memory allows for spread_f32 with sp-node blocks
static size_t smem_ctas(long long max_grid_bytes, int sp) {
    const size_t per = spread_smem_bytes(max_grid_bytes, false, sp) + 1024;   // + the per-CTA reserve
    return (size_t)(MAX_SMEM + 1024) / per;
}

// CTAs per SM of spread_f32 with sp-node blocks: at most 4 (64 registers) for
// SP_CH / 2, 3 (80 registers) for SP_CH
static int ctas_for(long long max_grid_bytes, int sp) {
    const size_t cap = sp == SP_CH ? 3 : SPREAD_MAX_CTAS_PER_SM;
    return (int)std::max<size_t>(1, std::min(cap, smem_ctas(max_grid_bytes, sp)));
}

// nodes per staging block.  The larger block runs best where registers, not
// shared memory, hold it at 3 CTAs per SM (small grids); where the grids fill
// shared memory, the smaller block gains a fourth CTA per SM (measured on the
// d = 20 workloads: bandwidths 64/32 gain, 32/16 lose with the smaller block).
int spread_block_nodes(long long max_grid_bytes) {
    const bool smem_bound = smem_ctas(max_grid_bytes, SP_CH) < (size_t)SPREAD_MAX_CTAS_PER_SM;
    return smem_bound && ctas_for(max_grid_bytes, SP_CH / 2) > ctas_for(max_grid_bytes, SP_CH) ? SP_CH / 2 : SP_CH;
}

// the tensor-core kernel: grid, one ring per warp, item slot
static size_t spread_mma_smem_bytes(long long max_grid_bytes);

int spread_ctas_per_sm(long long max_grid_bytes, bool tc) {
    if (tc) {
        const size_t per = spread_mma_smem_bytes(max_grid_bytes) + 1024;
        return (int)std::max<size_t>(1, std::min<size_t>(SPREAD_MMA_CTAS_PER_SM, (size_t)(MAX_SMEM + 1024) / per));
    }
    return ctas_for(max_grid_bytes, spread_block_nodes(max_grid_bytes));
}

int spread_chunks_for(long long M, int n_act_total, int kmax, long long max_grid_bytes, int sm_count, bool tc,
                      bool order3) {
    // third-order items cost several times an order-1/2 item per node: with
    // them, finer chunks (three per CTA of 3 per SM, the forward gather's
    // count) keep the last wave of both kernels short
    const int per_sm = spread_ctas_per_sm(max_grid_bytes, tc);
    const long long resident = (long long)(order3 ? std::max(3, per_sm) : per_sm) * sm_count;
    long long K = (3 * resident + std::max(1, n_act_total) - 1) / std::max(1, n_act_total);
    K = std::min<long long>(K, (M + 2047) / 2048);
    K = std::min<long long>(K, kmax);
    return (int)std::max<long long>(1, K);
}

int append_spread_items(const Plan &p, int prob, int K, int4 *out, int sel) {
    int n = 0;
    for (int order = sel == 3 ? 3 : 2; order >= (sel == 3 ? 3 : 1); --order)
        for (int s = 0; s < p.n_act; ++s) {
            if (p.h_terms[p.h_act[s]].order != order) continue;
            for (int z = 0; z < K; ++z) out[n++] = make_int4(prob, s, z, K);
        }
    return n;
}

// Window weights of one node for a half-warp, lane (r, k): lanes r = 0
// evaluate the column tap k, lanes r = 1 the row tap k (clamped to the
// window), each from its own coefficients wcf; shuffles hand every lane the
// column weight of its tap and the row weights of rows r, r + 2, ...
template <int MR>
__device__ __forceinline__ void node_weights(const float wcf[NCOEF], float vrow, float vcol, int half, int r, int k,
                                             float &cw, float w[MR]) {
    const float wt = horner8(wcf, r ? vrow : vcol);
    cw = __shfl_sync(0xffffffffu, wt, (half << 4) | k);
#pragma unroll
    for (int j = 0; j < MR; ++j) w[j] = __shfl_sync(0xffffffffu, wt, (half << 4) | 8 | (r + 2 * j));
}

// Sorted item: the item's nodes in cell order of its term, as records
// (window arguments, first-tap grid offset, original index).  The item's node
// range is cut into 16 contiguous runs, one per half-warp; block c of the
// staging holds records c*RUN .. c*RUN+RUN-1 of every run.  Records pass
// through shared memory by cp.async two blocks ahead, the values y[index] one
// block ahead (their addresses come from the staged records).  A half-warp
// sums the contributions of a cell in registers (lane (r, k): column tap k,
// rows r, r + 2, ..), two nodes per step, and adds the sums to the shared
// grid when the cell changes and at the end of its run.  Order 1: the lane
// groups r = 0, 1 take alternate nodes of the run.
template <int MR, int SP>
__device__ __forceinline__ void spread_sorted_item(const DevPlan &P, const Term &T, const float2 *__restrict__ y,
                                                   long long j0, long long j1, float2 *S, unsigned char *stg_raw,
                                                   const float wcf[NCOEF]) {
    constexpr int RUN = SP / 16;
    const int tid = threadIdx.x;
    const int lane = tid & 31, half = lane >> 4, sub = lane & 15;
    const int r = sub >> 3, k = sub & 7;
    const int hw = (tid >> 5) * 2 + half;
    const int stride = T.stride;
    const float4 *src = P.srec + (long long)T.sort_slot * P.M + j0;
    float4 *rbuf = (float4 *)stg_raw;            // [3][SP]
    float2 *ybuf = (float2 *)(rbuf + 3 * SP); // [2][SP]
    const long long len = j1 - j0;
    const long long L = (len + 15) / 16;           // run length
    const long long nblk = (L + RUN - 1) / RUN;
    // records of run h: [h L, min((h+1) L, len))
    auto run_len = [&](int h) { return max(0LL, min(L, len - (long long)h * L)); };
    auto stage_a = [&](long long c) {
        const int b = (int)(c % 3) * SP;
        for (int e = tid; e < SP; e += SPREAD_THREADS) {
            const int h = e / RUN, t = e % RUN;
            const long long q = c * RUN + t;
            if (q < run_len(h)) cp_async16(&rbuf[b + e], src + (long long)h * L + q);
        }
    };
    // reads records this thread staged itself (same e), so its own wait suffices
    auto stage_b = [&](long long c) {
        const int b = (int)(c % 3) * SP, yb = (int)(c & 1) * SP;
        for (int e = tid; e < SP; e += SPREAD_THREADS) {
            const int h = e / RUN, t = e % RUN;
            if (c * RUN + t < run_len(h)) cp_async8(&ybuf[yb + e], y + __float_as_int(rbuf[b + e].w));
        }
    };
    const long long my_len = run_len(hw);
    int cur = -1;   // grid offset of the cell being summed
    float ax[MR], ay[MR];
#pragma unroll
    for (int j = 0; j < MR; ++j) ax[j] = ay[j] = 0.f;
    auto flush2 = [&]() {
        float *base = (float *)(S + cur + r * stride + k);
#pragma unroll
        for (int j = 0; j < MR; ++j) {
            red_add(base + 4 * j * stride, ax[j]);
            red_add(base + 4 * j * stride + 1, ay[j]);
            ax[j] = ay[j] = 0.f;
        }
    };
    auto flush1 = [&]() {
        float *base = (float *)(S + cur + k);
        red_add(base, ax[0]);
        red_add(base + 1, ay[0]);
        ax[0] = ay[0] = 0.f;
    };
    const int col_src = (half << 4) | k, row_src = (half << 4) | 8 | r;
    if (nblk > 0) stage_a(0);
    cp_async_commit();
    if (nblk > 1) stage_a(1);
    cp_async_commit();
    cp_async_wait1();
    if (nblk > 0) stage_b(0);
    cp_async_commit();
    for (long long c = 0; c < nblk; ++c) {
        cp_async_wait0();
        __syncthreads();
        if (c + 1 < nblk) stage_b(c + 1);
        cp_async_commit();
        if (c + 2 < nblk) stage_a(c + 2);
        cp_async_commit();
        const float4 *rb = rbuf + (int)(c % 3) * SP + hw * RUN;
        const float2 *yb = ybuf + (int)(c & 1) * SP + hw * RUN;
        const long long left = my_len - c * RUN;   // records of this run still to come
        if (T.order == 2) {
            // both half-warps of a warp run all steps (shuffles); a node past
            // the run's end computes on record 0, adds zero and keeps the cell
            for (int t = 0; t < RUN; t += 2) {
                const bool ok0 = t < left, ok1 = t + 1 < left;
                const float4 q0 = rb[ok0 ? t : 0], q1 = rb[ok1 ? t + 1 : 0];
                const float wt0 = horner8(wcf, r ? q0.x : q0.y);
                const float wt1 = horner8(wcf, r ? q1.x : q1.y);
                const float cw0 = __shfl_sync(0xffffffffu, wt0, col_src);
                const float cw1 = __shfl_sync(0xffffffffu, wt1, col_src);
                float w0[MR], w1[MR];
#pragma unroll
                for (int j = 0; j < MR; ++j) {
                    w0[j] = __shfl_sync(0xffffffffu, wt0, row_src + 2 * j);
                    w1[j] = __shfl_sync(0xffffffffu, wt1, row_src + 2 * j);
                }
                const float2 y0 = ok0 ? yb[t] : make_float2(0.f, 0.f);
                const float2 y1 = ok1 ? yb[t + 1] : make_float2(0.f, 0.f);
                const int off0 = ok0 ? __float_as_int(q0.z) : cur;
                const int off1 = ok1 ? __float_as_int(q1.z) : off0;
                if (off0 != cur) {
                    if (cur >= 0) flush2();
                    cur = off0;
                }
                const float y0x = y0.x * cw0, y0y = y0.y * cw0;
#pragma unroll
                for (int j = 0; j < MR; ++j) {
                    ax[j] = fmaf(y0x, w0[j], ax[j]);
                    ay[j] = fmaf(y0y, w0[j], ay[j]);
                }
                if (off1 != cur) {
                    flush2();
                    cur = off1;
                }
                const float y1x = y1.x * cw1, y1y = y1.y * cw1;
#pragma unroll
                for (int j = 0; j < MR; ++j) {
                    ax[j] = fmaf(y1x, w1[j], ax[j]);
                    ay[j] = fmaf(y1y, w1[j], ay[j]);
                }
            }
        } else {
            for (int t = r; t < RUN; t += 2) {
                if (t >= left) break;
                const float4 q = rb[t];
                const int off = __float_as_int(q.z);
                if (off != cur) {
                    if (cur >= 0) flush1();
                    cur = off;
                }
                const float cw = horner8(wcf, q.y);
                const float2 yv = yb[t];
                ax[0] = fmaf(yv.x, cw, ax[0]);
                ay[0] = fmaf(yv.y, cw, ay[0]);
            }
        }
        __syncthreads();
    }
    cp_async_wait0();
    if (cur >= 0) {
        if (T.order == 2)
            flush2();
        else
            flush1();
    }
}

// Sorted third-order item: two records per node (window arguments and
// original index; the cell's grid indices).  The item's nodes are cut into 8
// runs, one per warp; blocks of 32 nodes per run are staged like the order-2
// path (records two blocks ahead, y one block ahead).  A warp takes one node
// at a time: lane (g, k), g = lane / 8, owns column tap k and the row pairs
// (ia, ib) with ib in {g, g + 4}, keeps their sums for the current cell in
// registers and adds them to the shared grid (indices modulo n) when the cell
// changes and at the end of its run.  Lanes 0..7 evaluate the first row
// coordinate's taps, lanes 8..15 the second's; shuffles hand them round.
constexpr int SP3_RUN = 32;                     // nodes per warp and block
constexpr int SP3_BLK = SP3_RUN * (SPREAD_THREADS / 32);
static_assert(3 * SP3_BLK * 32 + 2 * SP3_BLK * 8 <= SP3_STAGE_BYTES, "third-order staging");

template <int MR>
__device__ __forceinline__ void spread_sorted_item3(const DevPlan &P, const Term &T, const float2 *__restrict__ y,
                                                    long long j0, long long j1, float2 *S, unsigned char *stg_raw,
                                                    const float cc[NCOEF]) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 3, k = lane & 7;
    const int n = T.n, stride = T.stride, mc = T.mc;
    const float4 *src = P.srec + (long long)T.sort_slot * P.M + 2 * j0;
    float4 *rbuf = (float4 *)stg_raw;                   // [3][SP3_BLK][2]
    float2 *ybuf = (float2 *)(rbuf + 3 * 2 * SP3_BLK);  // [2][SP3_BLK]
    float rcf[NCOEF];
    {
        const float *c = P.windows[T.wr].c[min(k, 2 * MR - 1)];
#pragma unroll
        for (int q = 0; q < NCOEF; ++q) rcf[q] = __ldg(c + q);
    }
    const long long len = j1 - j0;
    const long long L = (len + 7) / 8;   // run length
    const long long nblk = (L + SP3_RUN - 1) / SP3_RUN;
    auto run_len = [&](int h) { return max(0LL, min(L, len - (long long)h * L)); };
    // thread tid stages node t_s of run h_s in every block
    const int h_s = tid / SP3_RUN, t_s = tid % SP3_RUN;
    const long long len_s = run_len(h_s);
    auto stage_a = [&](long long c) {
        const long long q = c * SP3_RUN + t_s;
        if (q < len_s) {
            float4 *d = rbuf + ((int)(c % 3) * SP3_BLK + tid) * 2;
            const float4 *gsrc = src + 2 * ((long long)h_s * L + q);
            cp_async16(d, gsrc);
            cp_async16(d + 1, gsrc + 1);
        }
    };
    auto stage_b = [&](long long c) {   // reads this thread's own staged record
        if (c * SP3_RUN + t_s < len_s)
            cp_async8(&ybuf[(int)(c & 1) * SP3_BLK + tid],
                      y + __float_as_int(rbuf[((int)(c % 3) * SP3_BLK + tid) * 2].w));
    };
    const long long my_len = run_len(warp);
    const bool ib1_ok = g + 4 < 2 * MR;
    int cfa = -1, cfb = 0, cfc = 0;
    float ax[2 * MR][2], ay[2 * MR][2];
#pragma unroll
    for (int a = 0; a < 2 * MR; ++a) ax[a][0] = ax[a][1] = ay[a][0] = ay[a][1] = 0.f;
    auto flush = [&]() {
        const int col = wrap(cfc - mc + 1 + k, n);
        const int rb0 = wrap(cfb - MR + 1 + g, n), rb1 = wrap(cfb - MR + 1 + g + 4, n);
#pragma unroll
        for (int a = 0; a < 2 * MR; ++a) {
            const int ra = wrap(cfa - MR + 1 + a, n) * n;
            if (g < 2 * MR) {
                float *cp = (float *)(S + (ra + rb0) * stride + col);
                red_add(cp, ax[a][0]);
                red_add(cp + 1, ay[a][0]);
            }
            if (ib1_ok) {
                float *cp = (float *)(S + (ra + rb1) * stride + col);
                red_add(cp, ax[a][1]);
                red_add(cp + 1, ay[a][1]);
            }
            ax[a][0] = ax[a][1] = ay[a][0] = ay[a][1] = 0.f;
        }
    };
    if (nblk > 0) stage_a(0);
    cp_async_commit();
    if (nblk > 1) stage_a(1);
    cp_async_commit();
    cp_async_wait1();
    if (nblk > 0) stage_b(0);
    cp_async_commit();
    for (long long c = 0; c < nblk; ++c) {
        cp_async_wait0();
        __syncthreads();
        if (c + 1 < nblk) stage_b(c + 1);
        cp_async_commit();
        if (c + 2 < nblk) stage_a(c + 2);
        cp_async_commit();
        const float4 *rb = rbuf + ((int)(c % 3) * SP3_BLK + warp * SP3_RUN) * 2;
        const float2 *yb = ybuf + (int)(c & 1) * SP3_BLK + warp * SP3_RUN;
        const long long left = my_len - c * SP3_RUN;
        for (int t = 0; t < SP3_RUN; ++t) {
            if (t >= left) break;   // warp-uniform
            const float4 q = rb[2 * t], qc = rb[2 * t + 1];
            const float cw = horner8(cc, q.z);
            const float wt = horner8(rcf, g == 0 ? q.x : q.y);   // lanes 0..7: first row, 8..15: second
            float wa[2 * MR];
#pragma unroll
            for (int a = 0; a < 2 * MR; ++a) wa[a] = __shfl_sync(0xffffffffu, wt, a);
            const float wb0 = __shfl_sync(0xffffffffu, wt, 8 + min(g, 2 * MR - 1));
            const float wb1 = __shfl_sync(0xffffffffu, wt, 8 + min(g + 4, 2 * MR - 1));
            const int fa = __float_as_int(qc.x), fb = __float_as_int(qc.y), fc = __float_as_int(qc.z);
            if (fa != cfa || fb != cfb || fc != cfc) {
                if (cfa >= 0) flush();
                cfa = fa;
                cfb = fb;
                cfc = fc;
            }
            const float2 yv = yb[t];
            const float yx = yv.x * cw, yy = yv.y * cw;
            const float u0x = yx * wb0, u0y = yy * wb0, u1x = yx * wb1, u1y = yy * wb1;
#pragma unroll
            for (int a = 0; a < 2 * MR; ++a) {
                ax[a][0] = fmaf(u0x, wa[a], ax[a][0]);
                ay[a][0] = fmaf(u0y, wa[a], ay[a][0]);
                ax[a][1] = fmaf(u1x, wa[a], ax[a][1]);
                ay[a][1] = fmaf(u1y, wa[a], ay[a][1]);
            }
        }
        __syncthreads();
    }
    cp_async_wait0();
    if (cfa >= 0) flush();
}

// Unsorted item (order 3, or a plan without sorted copies): the item's nodes
// in their original order, staged as float4 (first-row coordinate, last
// coordinate, y) one block ahead; every node adds its window to the shared
// grid with shared-memory atomics.
template <int MR, bool O3, int SP>
__device__ __forceinline__ void spread_unsorted_item(const DevPlan &P, const Term &T, const float2 *__restrict__ y,
                                                     long long j0, long long j1, float2 *S, unsigned char *stg_raw,
                                                     const float wcf[NCOEF]) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, half = lane >> 4, sub = lane & 15;
    const int r = sub >> 3, k = sub & 7;
    const int warp = tid >> 5;
    constexpr int NW = SPREAD_THREADS / 32;
    const int order = T.order, n = T.n, stride = T.stride;
    const long long M = P.M;
    float4 *stage = (float4 *)stg_raw;   // [2][SP]
    const float *__restrict__ X = P.x;
    const float *xr = X + (long long)(order >= 2 ? T.row0 : T.col) * M;
    const float *xc = X + (long long)T.col * M;
    const float *xr1 = order == 3 ? X + (long long)T.row1 * M : nullptr;
    const long long nblk = (j1 - j0 + SP - 1) / SP;
    auto stage_block = [&](long long c, int buf) {
        const long long a = j0 + c * SP;
        const int cnt = (int)min((long long)SP, j1 - a);
        float4 *dst = stage + buf * SP;
        for (int e = tid; e < cnt; e += SPREAD_THREADS) {
            const long long j = a + e;
            cp_async4(&dst[e].x, xr + j);
            cp_async4(&dst[e].y, xc + j);
            cp_async8(&dst[e].z, y + j);
        }
    };
    if (nblk > 0) stage_block(0, 0);
    cp_async_commit();
    for (long long c = 0; c < nblk; ++c) {
        if (c + 1 < nblk) stage_block(c + 1, (int)((c + 1) & 1));
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const float4 *stg = stage + (int)(c & 1) * SP;
        const long long a = j0 + c * SP;
        const int cnt = (int)min((long long)SP, j1 - a);
        if (order == 2) {
            for (int i0 = 2 * warp; i0 < cnt; i0 += 2 * NW) {
                const int i = i0 + half;
                const bool ok = i < cnt;
                const float4 q = stg[ok ? i : i0];
                float ta, tb;
                const int fa = grid_pos(q.x, n, ta);
                const int fb = grid_pos(q.y, n, tb);
                float cw, w[MR];
                node_weights<MR>(wcf, 2.f * ta - 1.f, 2.f * tb - 1.f, half, r, k, cw, w);
                const float yx = q.z * cw, yy = q.w * cw;
                float *base = (float *)(S + (fa + r) * stride + fb + k);
                if (ok) {
#pragma unroll
                    for (int j = 0; j < MR; ++j) {
                        red_add(base + 4 * j * stride, yx * w[j]);
                        red_add(base + 4 * j * stride + 1, yy * w[j]);
                    }
                }
            }
        } else if (order == 1) {
            const int g = tid >> 3;
            for (int i = g; i < cnt; i += SPREAD_THREADS / 8) {
                const float4 q = stg[i];
                float tb;
                const int fb = grid_pos(q.y, n, tb);
                const float cw = horner8(wcf, 2.f * tb - 1.f);
                float *base = (float *)(S + fb + k);
                red_add(base, q.z * cw);
                red_add(base + 1, q.w * cw);
            }
        } else if constexpr (O3) {
            // order 3: rows wrap modulo n; row weights from the per-tap
            // polynomials, lane (0, k) the first row coordinate's tap k, lane
            // (1, k) the second's, handed round by shuffles (the whole warp
            // iterates together; a half-warp past the end adds nothing)
            float rcf[NCOEF];
            {
                const float *src = P.windows[T.wr].c[min(k, 2 * MR - 1)];
#pragma unroll
                for (int q = 0; q < NCOEF; ++q) rcf[q] = __ldg(src + q);
            }
            const int mc = T.mc;
            for (int i0 = 2 * warp; i0 < cnt; i0 += 2 * NW) {
                const int i = i0 + half;
                const bool ok = i < cnt;
                const int ii = ok ? i : i0;
                const float4 q = stg[ii];
                float ta, tb, tc;
                const int fa = grid_pos(q.x, n, ta);
                const int fb = grid_pos(__ldg(xr1 + a + ii), n, tb);
                const int fc = grid_pos(q.y, n, tc);
                const float cw = horner8(wcf, 2.f * tc - 1.f);
                const float wrow = horner8(rcf, r ? 2.f * tb - 1.f : 2.f * ta - 1.f);
                float wa[2 * MR], wb[MR];
#pragma unroll
                for (int t = 0; t < 2 * MR; ++t) wa[t] = __shfl_sync(0xffffffffu, wrow, (half << 4) | t);
#pragma unroll
                for (int j = 0; j < MR; ++j) wb[j] = __shfl_sync(0xffffffffu, wrow, (half << 4) | 8 | (r + 2 * j));
                if (!ok) continue;
                const int cidx = wrap(fc - mc + 1 + k, n);
                const float yx = q.z * cw, yy = q.w * cw;
#pragma unroll
                for (int ia = 0; ia < 2 * MR; ++ia) {
                    const int row = wrap(fa - MR + 1 + ia, n) * n;
                    const float ax = yx * wa[ia], ay = yy * wa[ia];
#pragma unroll
                    for (int j = 0; j < MR; ++j) {
                        const int rbj = wrap(fb - MR + 1 + r + 2 * j, n);
                        float *cp = (float *)(S + (row + rbj) * stride + cidx);
                        red_add(cp, ax * wb[j]);
                        red_add(cp + 1, ay * wb[j]);
                    }
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait0();
}

// ---- Tensor-core cell sums (order 1/2 terms with cell-sorted records) ----
//
// For the nodes j of one cell the contributions to its window block are
//     G[r][k] += sum_j y_j psi_row,r(j) psi_col,k(j)   (r < 2 m_row, k < 8).
// Every tap weight is a degree-7 polynomial in the node's cell offset v, kept
// in the Chebyshev basis X_i (Window::ch): psi_k = sum_i C[k][i] X_i.  So
//     G = C_col Mo C_row^T,   Mo[(re/im, i)][l] = sum_j y_j X_i(v_col,j) X_l(v_row,j),
// and the nodes of a cell only build the 16 x 8 moment matrix Mo: a product
// A B with A[(re/im, i)][j] = y_j X_i(v_col,j) (16 x n) and B[j][l] =
// X_l(v_row,j) (n x 8), one mma.m16n8k8 per group of 8 cell-sorted nodes.  A
// node's 2 x 8 basis values come from one lane (the recurrence: 8 packed FP32
// operations for both coordinates) through shared memory, where lane (g, t) =
// (lane / 4, lane % 4) picks up X_g of nodes t and t + 4 (the fragment layout
// of the PTX ISA for tf32 m16n8k8).  Instead of 16 polynomial evaluations
// per node (one per lane that holds a tap of it), each node's basis is
// computed once.  When the cell changes, two more products turn Mo into G,
// with the contraction index permuted (2t, 2t + 1 -> t, t + 4) so that each
// D fragment is the next product's operand as it stands, and G goes to the
// shared grid by shared-memory additions.  Each operand is split x = hi + lo
// into TF32 parts and a product is hi*hi + hi*lo + lo*hi (relative error near
// 2^-21); the three products of a group are summed by the tensor core, the
// groups in FP32 registers.  A group holding nodes of several cells is run
// once per cell with the other nodes masked.

// Records rec[0, n) of one term for one warp, in steps of STEP = 32 nodes (4
// groups of 8 for the tensor core; a step lying in one cell takes one test),
// lane u holding node u of a step.  The warp's ring in shared memory (RING
// steps of records) is filled by its lanes with cp.async DR steps ahead, and
// records PF steps ahead are prefetched into L2 (one bulk prefetch per step),
// so that the ring's copies find them there.  The value y[index] of a node is
// loaded by its lane into registers DY steps ahead, through L2 only
// (ld.global.cg: the scattered reads allocate no L1 lines, whose few hundred
// per SM would otherwise bound the reads in flight, and they cost no
// shared-memory writes); the lane then computes the node's basis and leaves
// it, with the value, in shared memory: the basis rows X_0..X_7 of the
// current step XROW words apart (= 8 mod 32: the four rows a half-warp reads
// lie in distinct banks), then the step's values.
// Order 1: B = e_0 (the single grid row), exact in TF32.
template <int STEP>
struct MmaRing {
    static constexpr int RING = 4, DR = 3, DY = 2, PF = 7;   // PF: L2 prefetch distance
    static constexpr int XROW = 2 * STEP + 8;   // words per basis row (STEP float2 + pad)
    static constexpr size_t REC_BYTES = (size_t)RING * STEP * 16;                    // float4 records
    static constexpr size_t X_OFF = REC_BYTES;                                       // basis rows
    static constexpr size_t YC_OFF = X_OFF + (size_t)NCOEF * XROW * 4;               // + values
    static constexpr size_t BYTES = YC_OFF + (size_t)STEP * 8;                       // per warp
    static_assert(DY < DR && DR < RING && STEP == 32 && XROW % 32 == 8, "ring layout");
};

constexpr int MMA_STEP = 32;   // nodes per ring step of the order-1/2 tensor-core spread

static size_t spread_mma_smem_bytes(long long max_grid_bytes) {
    return (size_t)max_grid_bytes + MmaRing<MMA_STEP>::BYTES * (SPREAD_MMA_THREADS / 32) + 16;
}

template <int MR, bool ORD2>
__device__ __forceinline__ void spread_mma_run(const float4 *__restrict__ rec, const float2 *__restrict__ y, int n,
                                               float2 *S, int stride, const float *__restrict__ chr,
                                               const float *__restrict__ chc, float4 *rring, float2 *xs,
                                               float2 *yc) {
    using R = MmaRing<MMA_STEP>;
    constexpr unsigned MMA_RING = R::RING;
    constexpr int MMA_DR = R::DR, MMA_DY = R::DY, XR = R::XROW / 2;   // basis row stride in float2
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ns = (n + MMA_STEP - 1) / MMA_STEP;
    int cur = -1;   // grid offset of the cell being summed
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    // d = Mo (re i = g, l = 2t), (re g, 2t + 1), (im g, 2t), (im g, 2t + 1)
    auto flush = [&]() {
        // this lane's window coefficients of the two products, split into TF32
        // parts: the row window's C_row[g][2t], C_row[g][2t + 1] (zero for g >=
        // 2 m_row; order 1: e_0 e_0^T) and the column window's C_col[g][2t],
        // C_col[g][2t + 1] (Window::ch rows are taps)
        unsigned ah[4], al[4], ch0, cl0, ch1, cl1;
        {
            float r0 = 0.f, r1 = 0.f;
            if (ORD2) {
                if (g < 2 * MR) {
                    r0 = __ldg(chr + g * NCOEF + 2 * t);
                    r1 = __ldg(chr + g * NCOEF + 2 * t + 1);
                }
            } else {
                r0 = g == 0 && t == 0 ? 1.f : 0.f;
            }
            split_tf32_x2(pk2(r0, r1), ah[0], al[0], ah[2], al[2]);
            ah[1] = ah[3] = al[1] = al[3] = 0u;
            split_tf32_x2(pk2(__ldg(chc + g * NCOEF + 2 * t), __ldg(chc + g * NCOEF + 2 * t + 1)), ch0, cl0, ch1,
                          cl1);
        }
        // Q_x[j][i] = sum_l C_row[j][l] Mo_x[i][l]: A = C_row (rows 8..15 zero),
        // B[k][i] = Mo_x[i][l(k)] with l(t) = 2t, l(t + 4) = 2t + 1
        unsigned mh[4], ml[4];
        split_tf32_x2(pk2(d[0], d[1]), mh[0], ml[0], mh[1], ml[1]);
        split_tf32_x2(pk2(d[2], d[3]), mh[2], ml[2], mh[3], ml[3]);
        float qr[4] = {0.f, 0.f, 0.f, 0.f}, qi[4] = {0.f, 0.f, 0.f, 0.f};
        mma_tf32(qr, al, mh[0], mh[1]);
        mma_tf32(qr, ah, ml[0], ml[1]);
        mma_tf32(qr, ah, mh[0], mh[1]);
        mma_tf32(qi, al, mh[2], mh[3]);
        mma_tf32(qi, ah, ml[2], ml[3]);
        mma_tf32(qi, ah, mh[2], mh[3]);
        // q = Q_x[j = g][i = 2t], Q_x[g][2t + 1] (entries 2, 3: zero rows).
        // G_x^T[j][k] = sum_i Q_x[j][i] C_col[k][i]: A[(x, j)][k'] = Q_x[j][i(k')],
        // B[k'][k] = C_col[k][i(k')]
        unsigned qh[4], ql[4];
        split_tf32_x2(pk2(qr[0], qi[0]), qh[0], ql[0], qh[1], ql[1]);
        split_tf32_x2(pk2(qr[1], qi[1]), qh[2], ql[2], qh[3], ql[3]);
        float G[4] = {0.f, 0.f, 0.f, 0.f};
        mma_tf32(G, ql, ch0, ch1);
        mma_tf32(G, qh, cl0, cl1);
        mma_tf32(G, qh, ch0, ch1);
        // G = (re, row tap g, column tap 2t), (re, g, 2t + 1), (im, g, 2t), (im, g, 2t + 1)
        if (ORD2 ? g < 2 * MR : g == 0) {
            float *c = (float *)(S + cur + g * stride + 2 * t);
            red_add(c, G[0]);
            red_add(c + 1, G[2]);
            red_add(c + 2, G[1]);
            red_add(c + 3, G[3]);
        }
        d[0] = d[1] = d[2] = d[3] = 0.f;
    };
    // tensor-core products of one group added to e (hi*lo terms first); a01 =
    // (A[g][t], A[g + 8][t]), a23 = (A[g][t + 4], A[g + 8][t + 4])
    auto group_mma = [&](float (&e)[4], f32x2 a01, f32x2 a23, unsigned bh0, unsigned bl0, unsigned bh1,
                         unsigned bl1) {
        unsigned ah[4], al[4];
        split_tf32_x2(a01, ah[0], al[0], ah[1], al[1]);
        split_tf32_x2(a23, ah[2], al[2], ah[3], al[3]);
        mma_tf32(e, al, bh0, bh1);
        if (ORD2) mma_tf32(e, ah, bl0, bl1);
        mma_tf32(e, ah, bh0, bh1);
    };
    // basis row 0 is X_0 = 1 for every node
    xs[lane] = make_float2(1.f, 1.f);
    float2 y_mid = make_float2(0.f, 0.f), y_cur = y_mid;   // values of steps i + 1, i (DY = 2 in flight)
    static_assert(MmaRing<MMA_STEP>::DY == 2, "two values in flight");
    // A fresh tensor-core sum per step (at most eight groups), added to d in
    // FP32 with rounding to nearest: the tensor core's own accumulation is
    // not rounded to nearest, and its bias would grow with the cell's node
    // count.
    for (int i = -MMA_DR; i < ns; ++i) {
        // iteration i commits one cp.async group, the records of step i + DR,
        // and loads the values of step i + DY; steps i < 0 fill the pipeline
        const int qr = i + MMA_DR, qy = i + MMA_DY, qp = i + R::PF;
        // the records of step qp into L2 (whole records of the run only)
        if (lane == 0 && qp < ns && qp >= MMA_DR)
            prefetch_l2_bulk(rec + MMA_STEP * qp, 16u * (unsigned)min(MMA_STEP, n - MMA_STEP * qp));
        if (qr < ns) cp_async16(&rring[((unsigned)qr % MMA_RING) * MMA_STEP + lane], rec + min(MMA_STEP * qr + lane, n - 1));
        cp_async_commit();
        // this lane's records of steps <= i + DR - 1 (the groups before this one) have landed
        cp_async_wait_n<1>();
        // the value of this lane's node of step qy, into registers
        float2 y_next = make_float2(0.f, 0.f);
        if (qy >= 0 && qy < ns) y_next = __ldcg(y + __float_as_int(rring[((unsigned)qy % MMA_RING) * MMA_STEP + lane].w));
        const float2 y_now = y_cur;   // the value of this lane's node of step i
        y_cur = y_mid;
        y_mid = y_next;
        if (i < 0) continue;
        const int sl0 = ((unsigned)i % MMA_RING) * MMA_STEP;
        // value and basis values X_1..X_7 of node `lane` of the step, (row,
        // column) coordinate pairs: X_{k+1} = X_{k-1} + (-1)^k 2 v X_k
        {
            const int u = lane;
            const float4 r = rring[sl0 + u];
            yc[u] = y_now;
            const f32x2 v = pk2(r.x, r.y);
            const f32x2 up = mul2(v, pk2(2.f, 2.f)), um = mul2(v, pk2(-2.f, -2.f));
            f32x2 xm = pk2(1.f, 1.f), x = v;
            f32x2 *row = (f32x2 *)(xs + u);
            row[XR] = x;
#pragma unroll
            for (int k = 2; k < NCOEF; ++k) {
                const f32x2 xn = fma2((k & 1) ? up : um, x, xm);
                row[k * XR] = xn;
                xm = x;
                x = xn;
            }
        }
        __syncwarp();   // records, values and basis rows of step i visible to the warp
        // two tensor-core sums (even and odd groups), so that two chains of
        // dependent products are in flight
        float e[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
        const bool whole = MMA_STEP * (i + 1) <= n;   // no group of this step runs past the end
        // the records are in cell order: if the step's first and last nodes lie in
        // the cell being summed, all of them do (the same test in every lane)
        const bool step_in_cell = whole && __float_as_int(rring[sl0].z) == cur &&
                                  __float_as_int(rring[sl0 + MMA_STEP - 1].z) == cur;
        // operands of group h: A = y times X_g of the column coordinate of nodes
        // t, t + 4, B = X_g of their row coordinate
        struct GroupOp {
            f32x2 a01, a23;
            unsigned bh0, bl0, bh1, bl1;
        };
        auto operands = [&](int h) {
            GroupOp o;
            const float2 x0 = xs[g * XR + 8 * h + t], x1 = xs[g * XR + 8 * h + t + 4];
            const float2 y0 = yc[8 * h + t], y1 = yc[8 * h + t + 4];
            o.a01 = pk2(y0.x * x0.y, y0.y * x0.y);
            o.a23 = pk2(y1.x * x1.y, y1.y * x1.y);
            if (ORD2) {
                split_tf32_x2(pk2(x0.x, x1.x), o.bh0, o.bl0, o.bh1, o.bl1);
            } else {
                o.bh0 = o.bh1 = g == 0 ? 0x3f800000u : 0u;
                o.bl0 = o.bl1 = 0u;
            }
            return o;
        };
        if (step_in_cell) {
            // every group of the step lies in the cell being summed
#pragma unroll
            for (int h = 0; h < MMA_STEP / 8; ++h) {
                const GroupOp o = operands(h);
                group_mma((h & 1) ? e2 : e, o.a01, o.a23, o.bh0, o.bl0, o.bh1, o.bl1);
            }
        } else {
#pragma unroll
            for (int h = 0; h < MMA_STEP / 8; ++h) {
                const int base = MMA_STEP * i + 8 * h;   // first node of this group (may be past the end)
                const GroupOp o = operands(h);
                const int off0 = __float_as_int(rring[sl0 + 8 * h + t].z);
                const int off1 = __float_as_int(rring[sl0 + 8 * h + t + 4].z);
                if (__all_sync(0xffffffffu, (whole || base + 8 <= n) && off0 == cur && off1 == cur)) {
                    // the whole group lies in the cell being summed
                    group_mma((h & 1) ? e2 : e, o.a01, o.a23, o.bh0, o.bl0, o.bh1, o.bl1);
                    continue;
                }
                // past the end the ring holds the last record again: masked here
                bool p0 = base + t < n, p1 = base + t + 4 < n;   // nodes t, t + 4 not yet added
                for (;;) {
                    const unsigned pm =
                        (__ballot_sync(0xffffffffu, p0) & 0xfu) | ((__ballot_sync(0xffffffffu, p1) & 0xfu) << 4);
                    if (!pm) break;
                    const int f = __ffs(pm) - 1;   // first node not yet added; its cell is next
                    const int oc = __shfl_sync(0xffffffffu, f < 4 ? off0 : off1, f & 3);
                    const bool e0 = p0 && off0 == oc, e1 = p1 && off1 == oc;
                    if (oc != cur) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            d[q] += e[q] + e2[q];
                            e[q] = e2[q] = 0.f;
                        }
                        if (cur >= 0) flush();
                        cur = oc;
                    }
                    group_mma(e, e0 ? o.a01 : pk2(0.f, 0.f), e1 ? o.a23 : pk2(0.f, 0.f), o.bh0, o.bl0, o.bh1,
                              o.bl1);
                    p0 = p0 && !e0;
                    p1 = p1 && !e1;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] += e[q] + e2[q];
        __syncwarp();   // ring slot i and the basis rows are read before later iterations refill them
    }
    cp_async_wait0();
    if (cur >= 0) flush();
}

// Sorted item of order 1/2 on the tensor cores: the item's records are cut
// into 8 contiguous runs (multiples of 8 nodes), one per warp.
template <int MR>
__device__ __forceinline__ void spread_mma_item(const DevPlan &P, const Term &T, const float2 *__restrict__ y,
                                                long long j0, long long j1, float2 *S, unsigned char *stg_raw) {
    const int warp = threadIdx.x >> 5;
    constexpr int NW = SPREAD_MMA_THREADS / 32;
    const long long len = j1 - j0, per = (len + 8 * NW - 1) / (8 * NW) * 8;
    const long long a = j0 + warp * per, b = min(j1, a + per);
    if (a >= b) return;
    const float4 *rec = P.srec + (long long)T.sort_slot * P.M + a;
    using R = MmaRing<MMA_STEP>;
    unsigned char *ring = stg_raw + warp * R::BYTES;
    float4 *rring = (float4 *)ring;
    float2 *xs = (float2 *)(ring + R::X_OFF);
    float2 *yc = (float2 *)(ring + R::YC_OFF);
    const float *chc = &P.windows[T.wc].ch[0][0];
    if (T.order == 2)
        spread_mma_run<MR, true>(rec, y, (int)(b - a), S, T.stride, &P.windows[T.wr].ch[0][0], chc, rring, xs, yc);
    else
        spread_mma_run<MR, false>(rec, y, (int)(b - a), S, T.stride, nullptr, chc, rring, xs, yc);
}

// ---- Third-order cell sums on the tensor cores ----
//
// For the nodes j of one cell of a term (a, b, c) the window sums are
//     G[ia][ib][k] += sum_j psi_a,ia(j) psi_b,ib(j) y_j psi_c,k(j).
// For each row tap ia this is one product A B_ia: A[(k, re/im)][j] =
// y_j psi_c,k(j) as in the order-2 kernel (shared by all ia) and
// B_ia[j][ib] = psi_a,ia(j) psi_b,ib(j), 2 m_row mma.m16n8k8 (three TF32
// products each) per group of 8 nodes.  Column n of B_ia holds second-row tap
// ib = n / 2 (n even) or n / 2 + 4 (n odd), so the two taps a lane's D
// fragment covers, t and t + 4, are 4 grid rows apart, which spreads its
// shared-memory additions over more banks.  Lane (g, t) evaluates column tap
// g, second-row tap ib(g) and first-row tap g of nodes t, t + 4; shuffles hand
// each lane the first coordinate's taps of its nodes.  The sums stay in the D
// fragments (4 per ia) and go to the shared grid (indices modulo n) when the
// cell changes and after 8 steps of 16 nodes in one cell, which keeps the
// tensor core's own accumulation chains short.
constexpr int MMA3_STEP = 16, MMA3_RING = 4, MMA3_DR = 3, MMA3_DY = 1;
constexpr size_t MMA3_REC_BYTES = (size_t)MMA3_RING * MMA3_STEP * 32;              // two float4 per node
constexpr size_t MMA3_RING_BYTES = MMA3_REC_BYTES + (size_t)MMA3_RING * MMA3_STEP * 8;  // + float2 values
static_assert(MMA3_DY < MMA3_DR && MMA3_DR < MMA3_RING && (MMA3_RING & (MMA3_RING - 1)) == 0, "ring depths");

static size_t spread3_mma_smem_bytes(long long max_grid_bytes) {
    return (size_t)max_grid_bytes + MMA3_RING_BYTES * (SPREAD_THREADS / 32) + 16;
}

template <int MR>
__device__ __forceinline__ void spread3_mma_run(const float4 *__restrict__ rec, const float2 *__restrict__ y, int n,
                                                float2 *S, const Term &T, const f32x2 cbp[NCOEF],
                                                const float rcf[NCOEF], float4 *rring, float2 *yring) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ib_g = (g >> 1) + 4 * (g & 1);   // second-row tap of B column g
    const int nn = T.n, stride = T.stride, mc = T.mc;
    const int ns = (n + MMA3_STEP - 1) / MMA3_STEP;
    int cur = -1, cfa = 0, cfb = 0, cfc = 0;   // the cell being summed: number and grid indices
    float d[2 * MR][4];
#pragma unroll
    for (int a = 0; a < 2 * MR; ++a) d[a][0] = d[a][1] = d[a][2] = d[a][3] = 0.f;
    // d[ia] = (re ib t, re ib t + 4, im ib t, im ib t + 4) of column tap g
    int chain = 0;   // steps summed into d since the last flush
    auto flush = [&]() {
        const int col = wrap(cfc - mc + 1 + g, nn);
        const int rb0 = wrap(cfb - MR + 1 + t, nn), rb1 = wrap(cfb - MR + 1 + t + 4, nn);
#pragma unroll
        for (int a = 0; a < 2 * MR; ++a) {
            const int ra = wrap(cfa - MR + 1 + a, nn) * nn;
            float *c0 = (float *)(S + (ra + rb0) * stride + col);
            red_add(c0, d[a][0]);
            red_add(c0 + 1, d[a][2]);
            if (t + 4 < 2 * MR) {
                float *c1 = (float *)(S + (ra + rb1) * stride + col);
                red_add(c1, d[a][1]);
                red_add(c1 + 1, d[a][3]);
            }
            d[a][0] = d[a][1] = d[a][2] = d[a][3] = 0.f;
        }
        chain = 0;
    };
    for (int i = -MMA3_DR; i < ns; ++i) {
        // iteration i commits one cp.async group: the records of step i + MMA3_DR
        // and the values of step i + MMA3_DY; lanes 0..15 copy one node each
        if (lane < MMA3_STEP) {
            const int qr = i + MMA3_DR, qy = i + MMA3_DY;
            if (qr < ns) {
                const float4 *src = rec + 2 * min(MMA3_STEP * qr + lane, n - 1);
                float4 *dst = &rring[((qr & (MMA3_RING - 1)) * MMA3_STEP + lane) * 2];
                cp_async16(dst, src);
                cp_async16(dst + 1, src + 1);
            }
            if (qy >= 0 && qy < ns) {
                cp_async_wait_n<MMA3_DR - MMA3_DY - 1>();
                const int j = __float_as_int(rring[((qy & (MMA3_RING - 1)) * MMA3_STEP + lane) * 2].w);
                cp_async8(&yring[(qy & (MMA3_RING - 1)) * MMA3_STEP + lane], y + j);
            }
        }
        cp_async_commit();
        if (i < 0) continue;
        cp_async_wait_n<MMA3_DY>();
        __syncwarp();
#pragma unroll
        for (int h = 0; h < MMA3_STEP / 8; ++h) {
            const int base = MMA3_STEP * i + 8 * h;   // first node of this group (may be past the end)
            const int sl = (i & (MMA3_RING - 1)) * MMA3_STEP + 8 * h;
            const float4 q0 = rring[2 * (sl + t)], c0 = rring[2 * (sl + t) + 1];
            const float4 q1 = rring[2 * (sl + t + 4)], c1 = rring[2 * (sl + t + 4) + 1];
            const float2 y0 = yring[sl + t], y1 = yring[sl + t + 4];
            // column tap g and second-row tap ib(g) (the B column) of nodes t,
            // t + 4, one packed Horner per node; first-row tap g here, handed
            // round below
            const bool gok = ib_g < 2 * MR;
            float wc0, wc1, wb0, wb1;
            horner8_x2(cbp, q0.z, q0.y, wc0, wb0);
            horner8_x2(cbp, q1.z, q1.y, wc1, wb1);
            wb0 = gok ? wb0 : 0.f;
            wb1 = gok ? wb1 : 0.f;
            const float wa0 = horner8(rcf, q0.x), wa1 = horner8(rcf, q1.x);
            const int key0 = __float_as_int(c0.w), key1 = __float_as_int(c1.w);
            bool p0 = base + t < n, p1 = base + t + 4 < n;   // nodes t, t + 4 not yet added
            const bool fast = __all_sync(0xffffffffu, p0 && p1 && key0 == cur && key1 == cur);
            for (;;) {
                bool e0 = p0, e1 = p1;
                if (!fast) {
                    const unsigned pm =
                        (__ballot_sync(0xffffffffu, p0) & 0xfu) | ((__ballot_sync(0xffffffffu, p1) & 0xfu) << 4);
                    if (!pm) break;
                    const int f = __ffs(pm) - 1;   // first node not yet added; its cell is next
                    const int src = f & 3;
                    const bool second = f >= 4;
                    const int oc = __shfl_sync(0xffffffffu, second ? key1 : key0, src);
                    e0 = p0 && key0 == oc;
                    e1 = p1 && key1 == oc;
                    if (oc != cur) {
                        if (cur >= 0) flush();
                        cur = oc;
                        cfa = __shfl_sync(0xffffffffu, __float_as_int(second ? c1.x : c0.x), src);
                        cfb = __shfl_sync(0xffffffffu, __float_as_int(second ? c1.y : c0.y), src);
                        cfc = __shfl_sync(0xffffffffu, __float_as_int(second ? c1.z : c0.z), src);
                    }
                }
                unsigned ah[4], al[4];
                split_tf32_x2(e0 ? mul2(pk2(y0.x, y0.y), pk2(wc0, wc0)) : pk2(0.f, 0.f), ah[0], al[0], ah[1], al[1]);
                split_tf32_x2(e1 ? mul2(pk2(y1.x, y1.y), pk2(wc1, wc1)) : pk2(0.f, 0.f), ah[2], al[2], ah[3], al[3]);
                const f32x2 wb = pk2(wb0, wb1);
#pragma unroll
                for (int a = 0; a < 2 * MR; ++a) {
                    // first coordinate's tap a of nodes t, t + 4 from lane (a, t)
                    const float va0 = __shfl_sync(0xffffffffu, wa0, 4 * a + t);
                    const float va1 = __shfl_sync(0xffffffffu, wa1, 4 * a + t);
                    unsigned bh0, bl0, bh1, bl1;
                    split_tf32_x2(mul2(pk2(va0, va1), wb), bh0, bl0, bh1, bl1);
                    mma_tf32(d[a], al, bh0, bh1);
                    mma_tf32(d[a], ah, bl0, bl1);
                    mma_tf32(d[a], ah, bh0, bh1);
                }
                if (fast) break;
                p0 = p0 && !e0;
                p1 = p1 && !e1;
            }
        }
        // at most 8 steps per tensor-core chain
        if (cur >= 0 && ++chain == 8) flush();
        __syncwarp();   // ring slot i is read before a later iteration refills it
    }
    cp_async_wait0();
    if (cur >= 0) flush();
}

template <int MR>
__device__ __forceinline__ void spread3_mma_item(const DevPlan &P, const Term &T, const float2 *__restrict__ y,
                                                 long long j0, long long j1, float2 *S, unsigned char *stg_raw) {
    const int warp = threadIdx.x >> 5, g = (threadIdx.x & 31) >> 2;
    // (column tap g, second-row tap of B column g) pairs, first-row tap g
    f32x2 cbp[NCOEF];
    float rcf[NCOEF];
    {
        const int ib = (g >> 1) + 4 * (g & 1);
        const float *cs = P.windows[T.wc].c[g];
        const float *rs = P.windows[T.wr].c[min(g, 2 * MR - 1)];
        const float *bs = P.windows[T.wr].c[min(ib, 2 * MR - 1)];
#pragma unroll
        for (int q = 0; q < NCOEF; ++q) {
            cbp[q] = pk2(__ldg(cs + q), __ldg(bs + q));
            rcf[q] = __ldg(rs + q);
        }
    }
    constexpr int NW = SPREAD_THREADS / 32;
    const long long len = j1 - j0, per = (len + 8 * NW - 1) / (8 * NW) * 8;
    const long long a = j0 + warp * per, b = min(j1, a + per);
    if (a >= b) return;
    unsigned char *ring = stg_raw + warp * MMA3_RING_BYTES;
    spread3_mma_run<MR>(P.srec + (long long)T.sort_slot * P.M + 2 * a, y, (int)(b - a), S, T, cbp, rcf,
                        (float4 *)ring, (float2 *)(ring + MMA3_REC_BYTES));
}

// One work item (x = problem, y = active term, z = node chunk, w = chunks per
// term) spreads nodes [M z / w, M (z+1) / w) of one term (in the term's cell
// order if the plan keeps sorted copies and the term has order <= 2, else in
// the original order) into a shared-memory copy of the term's stored grid
// (halos included) and writes it to partial grid z of its problem.  CTAs take
// items from a global counter.
// KIND: SK_STAGED (order 1/2 on the CUDA cores), SK_ORDER3, SK_MMA (order 1/2
// with records on the tensor cores; no staging area)
template <int MR, typename G, int KIND, int SP, int NT = SPREAD_THREADS>
__device__ __forceinline__ void spread_items(const DevPlan &single, const BatchArgs &B,
                                             const float2 *__restrict__ y_base, int item_begin, int item_end,
                                             int *counter, long long max_grid_bytes) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *S = (float2 *)smem_raw;
    unsigned char *stg_raw = smem_raw + max_grid_bytes;
    constexpr bool O3 = KIND == SK_ORDER3;
    int &s_item = *(int *)(stg_raw + (KIND == SK_MMA    ? MmaRing<MMA_STEP>::BYTES * (NT / 32)
                                      : KIND == SK_MMA3 ? MMA3_RING_BYTES * (NT / 32)
                                      : O3              ? SP3_STAGE_BYTES
                                                        : sp_stage_bytes(SP)));
    const int tid = threadIdx.x;
    const int k = tid & 7;
    for (;;) {
        if (tid == 0) s_item = item_begin + atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= item_end) break;
        const int4 itm = B.items[item];
        const DevPlan &P = B.plans ? B.plans[itm.x] : single;
        if (P.skip && *P.skip) continue;
        const Term &T = P.terms[P.act[itm.y]];
        const long long M = P.M;
        const long long j0 = M * itm.z / itm.w, j1 = M * (itm.z + 1) / itm.w;
        const long long elems = T.grid_bytes / (long long)sizeof(G);   // shared copy is FP32 complex
        float4 *S4 = (float4 *)S;
        for (long long e = tid; e < elems / 2; e += NT) S4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 *y = y_base + P.vec_node_off;
        // window coefficients of this lane: row tap k for lanes r = 1 of an
        // order-2 term (see node_weights), column tap k otherwise
        float wcf[NCOEF];
        if constexpr (KIND != SK_MMA && KIND != SK_MMA3) {
            const bool row = T.order == 2 && (tid & 8);
            const float *wsrc = row ? P.windows[T.wr].c[min(k, 2 * MR - 1)] : P.windows[T.wc].c[k];
#pragma unroll
            for (int i = 0; i < NCOEF; ++i) wcf[i] = __ldg(wsrc + i);
        }
        __syncthreads();   // grid zeroed before any addition
        if constexpr (KIND == SK_MMA) {
            spread_mma_item<MR>(P, T, y, j0, j1, S, stg_raw);
        } else if constexpr (KIND == SK_MMA3) {
            spread3_mma_item<MR>(P, T, y, j0, j1, S, stg_raw);
        } else if constexpr (O3) {
            if (T.sort_slot >= 0 && P.srec)
                spread_sorted_item3<MR>(P, T, y, j0, j1, S, stg_raw, wcf);
            else
                spread_unsorted_item<MR, true, SP>(P, T, y, j0, j1, S, stg_raw, wcf);
        } else {
            if (T.sort_slot >= 0 && P.srec)
                spread_sorted_item<MR, SP>(P, T, y, j0, j1, S, stg_raw, wcf);
            else
                spread_unsorted_item<MR, false, SP>(P, T, y, j0, j1, S, stg_raw, wcf);
        }
        __syncthreads();
        if constexpr (std::is_same<G, float2>::value) {
            float4 *dst = (float4 *)(P.partials + (long long)itm.z * P.grid_elems + T.grid_off);
            for (long long e = tid; e < elems / 2; e += NT) dst[e] = S4[e];
        } else {
            G *dst = (G *)P.partials + (long long)itm.z * P.grid_elems + T.grid_off;
            for (long long e = tid; e < elems; e += NT) dst[e] = GridEl<G>::store(S[e].x, S[e].y);
        }
        __syncthreads();
    }
}

// the order-1/2 items (3 CTAs per SM) and the third-order items (more
// registers for the 2 x 2 m_row row-pair sums, 2 CTAs per SM)
template <int MR, typename G, int SP>
__global__ void __launch_bounds__(SPREAD_THREADS, SP == SP_CH ? 3 : SPREAD_MAX_CTAS_PER_SM)
spread_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ y_base, int item_begin, int item_end,
           int *counter, long long max_grid_bytes) {
    spread_items<MR, G, SK_STAGED, SP>(single, B, y_base, item_begin, item_end, counter, max_grid_bytes);
}

// order-1/2 items of plans with cell-sorted records, on the tensor cores, in
// steps of STEP nodes
template <int MR, typename G>
__global__ void __launch_bounds__(SPREAD_MMA_THREADS, SPREAD_MMA_CTAS_PER_SM)
spread_mma_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ y_base, int item_begin, int item_end,
               int *counter, long long max_grid_bytes) {
    spread_items<MR, G, SK_MMA, MMA_STEP, SPREAD_MMA_THREADS>(single, B, y_base, item_begin, item_end, counter,
                                                              max_grid_bytes);
}

// third-order items of plans with cell-sorted records, on the tensor cores
template <int MR, typename G>
__global__ void __launch_bounds__(SPREAD_THREADS, 2)
spread3_mma_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ y_base, int item_begin, int item_end,
                int *counter, long long max_grid_bytes) {
    spread_items<MR, G, SK_MMA3, 0>(single, B, y_base, item_begin, item_end, counter, max_grid_bytes);
}

template <int MR, typename G>
__global__ void __launch_bounds__(SPREAD_THREADS, 2)
spread3_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ y_base, int item_begin, int item_end,
            int *counter, long long max_grid_bytes) {
    spread_items<MR, G, SK_ORDER3, SP_CH / 2>(single, B, y_base, item_begin, item_end, counter, max_grid_bytes);
}

template <typename G>
__global__ void reduce_partials_f32(DevPlan single, BatchArgs B) {
    const DevPlan &P = B.plans ? B.plans[blockIdx.y] : single;
    if (P.skip && *P.skip) return;
    const int nparts = P.spread_chunks;
    if constexpr (std::is_same<G, float2>::value) {
        const float4 *__restrict__ partials = (const float4 *)P.partials;
        float4 *__restrict__ out = (float4 *)P.grids;
        const long long n4 = P.grid_elems / 2, pstride4 = n4;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
             i += (long long)gridDim.x * blockDim.x) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int c = 0; c < nparts; ++c) {
                float4 v = __ldg(partials + (long long)c * pstride4 + i);
                a.x += v.x;
                a.y += v.y;
                a.z += v.z;
                a.w += v.w;
            }
            out[i] = a;
        }
    } else {
        // 16-bit partials and grid: widen, sum in FP32, round once
        const G *__restrict__ partials = (const G *)P.partials;
        G *__restrict__ out = (G *)P.grids;
        const long long ne = P.grid_elems;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ne;
             i += (long long)gridDim.x * blockDim.x) {
            float ax = 0.f, ay = 0.f;
            for (int c = 0; c < nparts; ++c) {
                const float2 v = GridEl<G>::load(partials[(long long)c * ne + i]);
                ax += v.x;
                ay += v.y;
            }
            out[i] = GridEl<G>::store(ax, ay);
        }
    }
}

template <typename G>
__global__ void adjoint_post_f32(DevPlan single, BatchArgs B, float2 *__restrict__ fhat_base) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int pb = B.plans ? B.blk_prob[blockIdx.x] : 0;
    const DevPlan &P = B.plans ? B.plans[pb] : single;
    const int sblk = B.plans ? (int)blockIdx.x - B.blk0[pb] : (int)blockIdx.x;
    if (P.skip && *P.skip) return;
    const G *__restrict__ grids = (const G *)P.grids;
    float2 *__restrict__ fhat = fhat_base + P.vec_coef_off;
    const Term T = P.terms[P.act[sblk]];
    const int n = T.n, s = T.order, N = T.N;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    float2 *a = (float2 *)smem_raw;
    float2 *b = a + fe;
    const G *g = grids + T.grid_off;
    // fold the stored (halo) grid onto the periodic grid
    for (int e = threadIdx.x; e < fe; e += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (s <= 2) {
            int qc = e % n, qr = s == 2 ? e / n : 0;
            int ecw = n + 2 * T.hc + 1;
            for (int dr = -1; dr <= 1; ++dr) {
                int er = s == 2 ? qr + T.hr + dr * n : 0;
                if (s == 1 && dr != 0) continue;
                if (er < 0 || er >= T.erows) continue;
                for (int dc = -1; dc <= 1; ++dc) {
                    int ec = qc + T.hc + dc * n;
                    if (ec < 0 || ec >= ecw) continue;
                    const float2 u = GridEl<G>::load(g[(long long)er * T.stride + ec]);
                    v.x += u.x;
                    v.y += u.y;
                }
            }
        } else {
            int row = e / n, c = e % n;
            v = GridEl<G>::load(g[(long long)row * T.stride + c]);
        }
        a[e] = v;
    }
    __syncthreads();
    // FFT along every axis, sign -
    float2 *cur = a, *oth = b;
    int inner = 1;
    for (int ax = s - 1; ax >= 0; --ax) {
        int rad[24];
        int ns = fft_radices(n, rad);
        const int nlines = fe / n;
        float2 *src = cur, *dst = oth;
        int which = 0, Ns = 1;
        for (int st = 0; st < ns; ++st) {
            const int Rr = rad[st];
            const int nb = n / Rr;
            for (int w = threadIdx.x; w < nlines * nb; w += blockDim.x) {
                const int l = w / nb, j = w - l * nb;
                const int base = (l / inner) * inner * n + (l % inner);
                const float2 *in = src + base;
                float2 *out = dst + base;
                float2 v[5];
                const int jm = j % Ns;
                for (int r = 0; r < Rr; ++r) {
                    float2 x = in[(j + r * nb) * inner];
                    if (r && jm) {
                        float sn, cs;
                        sincospif(-(float)(2 * r * jm) / (float)(Ns * Rr), &sn, &cs);
                        x = cmul(x, make_float2(cs, sn));
                    }
                    v[r] = x;
                }
                float2 V[5];
                if (Rr == 2) {
                    V[0] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
                    V[1] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
                } else if (Rr == 4) {
                    float2 s0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
                    float2 d0 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
                    float2 s1 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
                    float2 d1 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
                    float2 jd1 = make_float2(d1.y, -d1.x);   // -i d1
                    V[0] = make_float2(s0.x + s1.x, s0.y + s1.y);
                    V[2] = make_float2(s0.x - s1.x, s0.y - s1.y);
                    V[1] = make_float2(d0.x + jd1.x, d0.y + jd1.y);
                    V[3] = make_float2(d0.x - jd1.x, d0.y - jd1.y);
                } else {
                    for (int q = 0; q < Rr; ++q) {
                        float2 acc = v[0];
                        for (int r = 1; r < Rr; ++r) {
                            float sn, cs;
                            sincospif(-(float)(2 * ((r * q) % Rr)) / (float)Rr, &sn, &cs);
                            float2 t = cmul(v[r], make_float2(cs, sn));
                            acc.x += t.x;
                            acc.y += t.y;
                        }
                        V[q] = acc;
                    }
                }
                const int idxD = (j / Ns) * Ns * Rr + jm;
                for (int r = 0; r < Rr; ++r) out[(idxD + r * Ns) * inner] = V[r];
            }
            __syncthreads();
            float2 *t = src;
            src = dst;
            dst = t;
            which ^= 1;
            Ns *= Rr;
        }
        if (which) {
            float2 *t = cur;
            cur = oth;
            oth = t;
        }
        inner *= n;
    }
    // crop and deconvolve
    const int Nm = N - 1;
    for (long long q = threadIdx.x; q < T.coef_len && T.basis == ANOVA_BASIS_COS; q += blockDim.x) {
        // cosine term: 2^{-s/2} times the sum over its 2^s mirrored frequencies
        int k[3];
        cos_decode(q, s, N, k);
        float sx = 0.f, sy = 0.f;
        for (int sg = 0; sg < (1 << s); ++sg) {
            float D = (float)cos_amp(s);
            const float2 v = cur[cos_mirror(k, s, sg, N, n, P.deconv, T.dc_off, T.dr_off, D)];
            sx = fmaf(v.x, D, sx);
            sy = fmaf(v.y, D, sy);
        }
        fhat[T.coef_off + q] = make_float2(sx, sy);
    }
    for (long long q = threadIdx.x; q < T.coef_len && T.basis != ANOVA_BASIS_COS; q += blockDim.x) {
        long long rr = q;
        int pos = 0, mul = 1;
        float D = 1.f;
        for (int t = s - 1; t >= 0; --t) {
            int it = (int)(rr % Nm);
            rr /= Nm;
            int kk = freq_index_a(it, N);
            pos += (kk < 0 ? kk + n : kk) * mul;
            mul *= n;
            D *= (t == s - 1) ? P.deconv[T.dc_off + it] : P.deconv[T.dr_off + it];
        }
        float2 v = cur[pos];
        fhat[T.coef_off + q] = make_float2(v.x * D, v.y * D);
    }
}

// two-stage sum of y for the empty-set coefficients
__global__ void sum_y_stage1(DevPlan single, BatchArgs B, const float2 *__restrict__ y_base, double2 *part_base) {
    const DevPlan &P = B.plans ? B.plans[blockIdx.y] : single;
    if (P.skip && *P.skip) return;
    if (P.n_empty == 0) return;
    const float2 *__restrict__ y = y_base + P.vec_node_off;
    const long long M = P.M;
    double2 *part = part_base + (long long)blockIdx.y * gridDim.x;
    __shared__ double2 red[256];
    double sx = 0, sy = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        float2 v = y[i];
        sx += v.x;
        sy += v.y;
    }
    red[threadIdx.x] = make_double2(sx, sy);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[threadIdx.x].x += red[threadIdx.x + o].x;
            red[threadIdx.x].y += red[threadIdx.x + o].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_y_stage2(DevPlan single, BatchArgs B, const double2 *part_base, int nparts, float2 *fhat_base) {
    const DevPlan &P = B.plans ? B.plans[blockIdx.x] : single;
    if (threadIdx.x != 0 || (P.skip && *P.skip) || P.n_empty == 0) return;
    const double2 *part = part_base + (long long)blockIdx.x * nparts;
    float2 *fhat = fhat_base + P.vec_coef_off;
    const long long *eoff = P.empty_off;
    const int n_empty = P.n_empty;
    double sx = 0, sy = 0;
    for (int i = 0; i < nparts; ++i) {
        sx += part[i].x;
        sy += part[i].y;
    }
    for (int e = 0; e < n_empty; ++e) fhat[eoff[e]] = make_float2((float)sx, (float)sy);
}

template <typename G>
static void adjoint_attrs() {
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(adjoint_post_f32<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(spread_f32<3, G, SP_CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread_f32<4, G, SP_CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread_f32<3, G, SP_CH / 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread_f32<4, G, SP_CH / 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread3_f32<3, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread3_mma_f32<3, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread3_mma_f32<4, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread_mma_f32<3, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread_mma_f32<4, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread3_f32<4, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
    });
}

// spread + reduce + post for grids stored as G; sgrid = bytes of the largest
// grid in FP32 (the spread's shared-memory copy)
template <typename G>
static void adjoint_kernels(Plan *prof, cudaStream_t st, const DevPlan &v, const BatchArgs &B, int P,
                            const float2 *y, float2 *fhat, int n_items, int n_items3, int *counter, int n_blocks,
                            int mr, long long sgrid, int max_fft_elems, int sm_count, long long max_grid_elems,
                            bool tc) {
    adjoint_attrs<G>();
    const int sp = spread_block_nodes(sgrid);
    const size_t ssm = spread_smem_bytes(sgrid, false, sp), ssm3 = spread_smem_bytes(sgrid, true, sp);
    const int per_sm = spread_ctas_per_sm(sgrid, false);
    if (prof) stage_begin(*prof, ST_SPREAD);
    cudaMemsetAsync(counter, 0, 2 * sizeof(int), st);
    if (n_items3 > 0 && tc) {
        const size_t sm3 = spread3_mma_smem_bytes(sgrid);
        const int per3 = (int)std::max<size_t>(1, std::min<size_t>(2, (size_t)(MAX_SMEM + 1024) / (sm3 + 1024)));
        const int c3 = std::max(1, std::min(n_items3, per3 * sm_count));
        auto k = mr <= 3 ? spread3_mma_f32<3, G> : spread3_mma_f32<4, G>;
        k<<<c3, SPREAD_THREADS, sm3, st>>>(v, B, y, 0, n_items3, counter, sgrid);
    } else if (n_items3 > 0) {
        const int c3 = std::max(1, std::min(n_items3, std::min(per_sm, 2) * sm_count));
        if (mr <= 3)
            spread3_f32<3, G><<<c3, SPREAD_THREADS, ssm3, st>>>(v, B, y, 0, n_items3, counter, sgrid);
        else
            spread3_f32<4, G><<<c3, SPREAD_THREADS, ssm3, st>>>(v, B, y, 0, n_items3, counter, sgrid);
    }
    if (n_items > n_items3 && tc) {
        const size_t sm = spread_mma_smem_bytes(sgrid);
        const int per = (int)std::max<size_t>(
            1, std::min<size_t>(SPREAD_MMA_CTAS_PER_SM, (size_t)(MAX_SMEM + 1024) / (sm + 1024)));
        const int c = std::max(1, std::min(n_items - n_items3, per * sm_count));
        auto k = mr <= 3 ? spread_mma_f32<3, G> : spread_mma_f32<4, G>;
        k<<<c, SPREAD_MMA_THREADS, sm, st>>>(v, B, y, n_items3, n_items, counter + 1, sgrid);
    } else if (n_items > n_items3) {
        const int c = std::max(1, std::min(n_items - n_items3, per_sm * sm_count));
        auto k = mr <= 3 ? (sp == SP_CH ? spread_f32<3, G, SP_CH> : spread_f32<3, G, SP_CH / 2>)
                         : (sp == SP_CH ? spread_f32<4, G, SP_CH> : spread_f32<4, G, SP_CH / 2>);
        k<<<c, SPREAD_THREADS, ssm, st>>>(v, B, y, n_items3, n_items, counter + 1, sgrid);
    }
    if (prof) stage_end(*prof, ST_SPREAD);
    const long long n4 = max_grid_elems / 2;
    const int rb = (int)std::max<long long>(1, std::min<long long>(sm_count * 8LL / std::max(1, P) + 1, (n4 + 255) / 256));
    if (prof) stage_begin(*prof, ST_REDUCE);
    reduce_partials_f32<G><<<dim3(rb, P), 256, 0, st>>>(v, B);
    if (prof) stage_end(*prof, ST_REDUCE);
    const size_t post_smem = (size_t)max_fft_elems * 2 * sizeof(float2);
    if (prof) stage_begin(*prof, ST_POST);
    adjoint_post_f32<G><<<n_blocks, 256, post_smem, st>>>(v, B, fhat);
    if (prof) stage_end(*prof, ST_POST);
}

// The adjoint kernels for one problem (B.plans == null) or a batch of P problems.
int adjoint_launch(Plan *prof, cudaStream_t st, const DevPlan &v, const BatchArgs &B, int P, const float2 *y,
                   float2 *fhat, int n_items, int n_items3, int *counter, int n_blocks, int mr,
                   long long max_grid_bytes, int max_fft_elems, int sm_count, long long max_grid_elems,
                   bool any_empty, double2 *scratch, int prec, bool tc) {
    if (any_empty) {
        const int nb = 256;
        if (prof) stage_begin(*prof, ST_SUMY);
        sum_y_stage1<<<dim3(nb, P), 256, 0, st>>>(v, B, y, scratch);
        sum_y_stage2<<<P, 32, 0, st>>>(v, B, scratch, nb, fhat);
        if (prof) stage_end(*prof, ST_SUMY);
    }
    if (n_blocks == 0) return cuda_status(cudaGetLastError());
    if (prec == ANOVA_PREC_F16)
        adjoint_kernels<__half2>(prof, st, v, B, P, y, fhat, n_items, n_items3, counter, n_blocks, mr,
                                 2 * max_grid_bytes, max_fft_elems, sm_count, max_grid_elems, tc);
    else if (prec == ANOVA_PREC_BF16)
        adjoint_kernels<__nv_bfloat162>(prof, st, v, B, P, y, fhat, n_items, n_items3, counter, n_blocks, mr,
                                        2 * max_grid_bytes, max_fft_elems, sm_count, max_grid_elems, tc);
    else
        adjoint_kernels<float2>(prof, st, v, B, P, y, fhat, n_items, n_items3, counter, n_blocks, mr,
                                max_grid_bytes, max_fft_elems, sm_count, max_grid_elems, tc);
    return cuda_status(cudaGetLastError());
}

int launch_adjoint_f32(Plan &p, const float2 *y, float2 *fhat) {
    DevPlan v = dev_view(p);
    BatchArgs B;
    std::memset(&B, 0, sizeof(B));
    B.items = p.items;
    if (p.M == 0) {
        cudaMemsetAsync(fhat, 0, sizeof(float2) * p.n_coeffs, p.stream);
        return cuda_status(cudaGetLastError());
    }
    int mr = 3;
    for (int s = 0; s < p.n_terms; ++s) mr = p.h_terms[s].mr > 0 ? p.h_terms[s].mr : mr;
    return adjoint_launch(&p, p.stream, v, B, 1, y, fhat, p.n_items, p.n_items3, p.counter, p.n_act, mr,
                          p.max_grid_bytes, p.max_fft_elems, p.sm_count, p.grid_elems, p.n_empty > 0,
                          (double2 *)p.scratch, p.precision, p.srec && p.cell_tc);
}

}  // namespace agft
