// Forward gather over the cell-sorted node records (every term with records:
// all terms of an FP32 plan that keeps them) (the window interpolation step of the NFFT behind eq. (somafm),
// Sec. 3), FP32.
//
// Work items are the adjoint's (active term, node chunk) pairs.  A CTA copies
// the term's stored grid into shared memory and gives each thread one node at
// a time (two in flight): the thread evaluates the node's 8 column and 2 m_row
// row window weights from the per-tap polynomials (coefficients broadcast from
// shared memory, 16 bytes at a time), reads the 6 x 8 grid values around the
// node's cell (the nodes of a warp mostly share a cell, so the reads are
// broadcasts) and adds sum_i w_row[i] sum_t w_col[t] g[i][t] into node j's
// accumulator.  The accumulators are 64-bit integers holding the values in
// fixed point, v * 2^e with 2^e chosen from ||fhat||_1 (a bound on every
// partial sum), so the additions are exact and their order, which the
// hardware does not fix, cannot change the result: the forward is bitwise
// reproducible.  A last pass adds acc * 2^-e to f, which already holds the
// empty set's coefficient and the third-order terms.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

constexpr int GS_THREADS = 256;

__device__ __forceinline__ void red_add_u64(unsigned long long *addr, long long v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(addr), "l"(v) : "memory");
}

// fixed-point exponent e for the accumulators: 2^e * 2 sum |fhat| <= 2^62
// (every partial sum of a node's terms is bounded by sum_k |fhat_k| up to the
// window error), clamped so that 2^e stays a normal float.  Two passes with
// a fixed block count, so the sum (and e) never depends on timing.
constexpr int FPE_BLOCKS = 128;

__global__ void k_fixed_point_partial(const float2 *__restrict__ fhat, long long n, double *part) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = fhat[i];
        a += fabs((double)v.x) + fabs((double)v.y);
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_fixed_point_exponent(const double *part, int *e_out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < FPE_BLOCKS; ++b) s += part[b];
    int e = 100;
    if (s > 0) e = 61 - (int)ceil(log2(s));
    *e_out = max(-100, min(100, e));
}

// f[j] += acc[j] * 2^-e
__global__ void k_fixed_point_finish(float2 *f, const long long *acc, const int *e_in, long long M, const int *skip) {
    if (skip && *skip) return;
    const double sc = ldexp(1.0, -*e_in);
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M; j += (long long)gridDim.x * blockDim.x) {
        float2 v = f[j];
        v.x += (float)((double)acc[2 * j] * sc);
        v.y += (float)((double)acc[2 * j + 1] * sc);
        f[j] = v;
    }
}

// polynomial of tap t from the shared coefficient table (two float4 per tap)
__device__ __forceinline__ void horner_pair(const float4 *c, float v0, float v1, float &w0, float &w1) {
    const float4 lo = c[0], hi = c[1];
    float a = hi.w, b = hi.w;
    a = fmaf(a, v0, hi.z);
    b = fmaf(b, v1, hi.z);
    a = fmaf(a, v0, hi.y);
    b = fmaf(b, v1, hi.y);
    a = fmaf(a, v0, hi.x);
    b = fmaf(b, v1, hi.x);
    a = fmaf(a, v0, lo.w);
    b = fmaf(b, v1, lo.w);
    a = fmaf(a, v0, lo.z);
    b = fmaf(b, v1, lo.z);
    a = fmaf(a, v0, lo.y);
    b = fmaf(b, v1, lo.y);
    w0 = fmaf(a, v0, lo.x);
    w1 = fmaf(b, v1, lo.x);
}

template <int MR>
__global__ void __launch_bounds__(GS_THREADS, 3)
gather_sorted_f32(DevPlan P, const int4 *__restrict__ items, unsigned long long *__restrict__ acc, const int *e_in,
                  int item_begin, int item_end, int *counter, long long max_grid_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *S = (float2 *)smem;
    float4 *coef = (float4 *)(smem + max_grid_bytes);   // [8 column taps + 8 row taps][2]
    int &s_item = *(int *)(coef + 32);
    const int tid = threadIdx.x;
    const long long M = P.M;
    const float sc = __int_as_float((127 + *e_in) << 23);   // 2^e, exact scaling
    for (;;) {
        if (tid == 0) s_item = item_begin + atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= item_end) break;
        if (P.skip && *P.skip) continue;
        const int4 itm = items[item];
        const Term &T = P.terms[P.act[itm.y]];
        if (T.sort_slot < 0) continue;   // no records: the point-major gather has the term
        const long long j0 = M * itm.z / itm.w, j1 = M * (itm.z + 1) / itm.w;
        // the term's grid and window coefficients into shared memory
        {
            const float4 *g = (const float4 *)(P.grids + T.grid_off);
            float4 *S4 = (float4 *)S;
            const long long n4 = T.grid_bytes / 16;
            for (long long e = tid; e < n4; e += GS_THREADS) S4[e] = __ldg(g + e);
            if (tid < 32) {
                const int tap = tid >> 1, h = tid & 1;
                const float *src = tap < 8 ? P.windows[T.wc].c[tap] : P.windows[T.wr].c[min(tap - 8, 2 * MR - 1)];
                coef[tid] = make_float4(__ldg(src + 4 * h), __ldg(src + 4 * h + 1), __ldg(src + 4 * h + 2),
                                        __ldg(src + 4 * h + 3));
            }
        }
        __syncthreads();
        const float4 *rec = P.srec + (long long)T.sort_slot * M;
        const int stride = T.stride;
        const bool two = T.order == 2;
        if (T.order == 3) {
            // one node per thread: two records (window arguments and index; the
            // cell's grid indices), 2 MR x 2 MR rows of 8 taps, indices modulo n
            const int n = T.n;
            for (long long p = j0 + tid; p < j1; p += GS_THREADS) {
                const float4 q = __ldg(rec + 2 * p), qc = __ldg(rec + 2 * p + 1);
                const int fa = __float_as_int(qc.x), fb = __float_as_int(qc.y), fc = __float_as_int(qc.z);
                float wc[8], wb[2 * MR], dummy;
                int col[8], rb[2 * MR];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    horner_pair(coef + 2 * t, q.z, q.z, wc[t], dummy);
                    col[t] = wrap(fc - T.mc + 1 + t, n);
                }
#pragma unroll
                for (int i = 0; i < 2 * MR; ++i) {
                    horner_pair(coef + 16 + 2 * i, q.y, q.y, wb[i], dummy);
                    rb[i] = wrap(fb - MR + 1 + i, n);
                }
                float sx = 0.f, sy = 0.f;
#pragma unroll 1
                for (int ia = 0; ia < 2 * MR; ++ia) {
                    float wa;
                    horner_pair(coef + 16 + 2 * ia, q.x, q.x, wa, dummy);
                    const int ra = wrap(fa - MR + 1 + ia, n) * n;
                    float ux = 0.f, uy = 0.f;
#pragma unroll
                    for (int ib = 0; ib < 2 * MR; ++ib) {
                        const float2 *row = S + (ra + rb[ib]) * stride;
                        float tx = 0.f, ty = 0.f;
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const float2 g = row[col[t]];
                            tx = fmaf(wc[t], g.x, tx);
                            ty = fmaf(wc[t], g.y, ty);
                        }
                        ux = fmaf(wb[ib], tx, ux);
                        uy = fmaf(wb[ib], ty, uy);
                    }
                    sx = fmaf(wa, ux, sx);
                    sy = fmaf(wa, uy, sy);
                }
                unsigned long long *a0 = acc + 2 * (long long)__float_as_int(q.w);
                red_add_u64(a0, __float2ll_rn(sx * sc));
                red_add_u64(a0 + 1, __float2ll_rn(sy * sc));
            }
            __syncthreads();
            continue;
        }
        for (long long p = j0 + tid; p < j1; p += 2 * GS_THREADS) {
            const long long p1 = p + GS_THREADS;
            const bool ok1 = p1 < j1;
            const float4 q0 = __ldg(rec + p), q1 = __ldg(rec + (ok1 ? p1 : p));
            float wc0[8], wc1[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) horner_pair(coef + 2 * t, q0.y, q1.y, wc0[t], wc1[t]);
            const int off0 = __float_as_int(q0.z), off1 = __float_as_int(q1.z);
            float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f;
            if (two) {
#pragma unroll
                for (int i = 0; i < 2 * MR; ++i) {
                    float wr0, wr1;
                    horner_pair(coef + 16 + 2 * i, q0.x, q1.x, wr0, wr1);
                    const float2 *r0 = S + off0 + i * stride, *r1 = S + off1 + i * stride;
                    float tx0 = 0.f, ty0 = 0.f, tx1 = 0.f, ty1 = 0.f;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float2 a = r0[t], b = r1[t];
                        tx0 = fmaf(wc0[t], a.x, tx0);
                        ty0 = fmaf(wc0[t], a.y, ty0);
                        tx1 = fmaf(wc1[t], b.x, tx1);
                        ty1 = fmaf(wc1[t], b.y, ty1);
                    }
                    sx0 = fmaf(wr0, tx0, sx0);
                    sy0 = fmaf(wr0, ty0, sy0);
                    sx1 = fmaf(wr1, tx1, sx1);
                    sy1 = fmaf(wr1, ty1, sy1);
                }
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 a = S[off0 + t], b = S[off1 + t];
                    sx0 = fmaf(wc0[t], a.x, sx0);
                    sy0 = fmaf(wc0[t], a.y, sy0);
                    sx1 = fmaf(wc1[t], b.x, sx1);
                    sy1 = fmaf(wc1[t], b.y, sy1);
                }
            }
            unsigned long long *a0 = acc + 2 * (long long)__float_as_int(q0.w);
            red_add_u64(a0, __float2ll_rn(sx0 * sc));
            red_add_u64(a0 + 1, __float2ll_rn(sy0 * sc));
            if (ok1) {
                unsigned long long *a1 = acc + 2 * (long long)__float_as_int(q1.w);
                red_add_u64(a1, __float2ll_rn(sx1 * sc));
                red_add_u64(a1 + 1, __float2ll_rn(sy1 * sc));
            }
        }
        __syncthreads();   // the grid is read by every thread before the next item replaces it
    }
}

int launch_gather_sorted_f32(Plan &p, const float2 *fhat, float2 *f) {
    DevPlan v = dev_view(p);
    double *part = (double *)p.scratch;   // FPE_BLOCKS partial sums
    k_fixed_point_partial<<<FPE_BLOCKS, 256, 0, p.stream>>>(fhat, p.n_coeffs, part);
    k_fixed_point_exponent<<<1, 32, 0, p.stream>>>(part, p.fexp);
    cudaMemsetAsync(p.facc, 0, sizeof(unsigned long long) * 2 * p.M, p.stream);
    int mr = 3;
    for (int s = 0; s < p.n_terms; ++s)
        if (p.h_terms[s].mr > 0) mr = p.h_terms[s].mr;
    const size_t smem = (size_t)p.max_grid_bytes + 32 * sizeof(float4) + 16;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gather_sorted_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(gather_sorted_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        attr = true;
    }
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(3, (size_t)(MAX_SMEM + 1024) / (smem + 1024)));
    // the order-1/2 items, and the third-order ones (the first n_items3) when they have records
    const int first = p.n_act3 > 0 ? p.n_items3 : 0;
    const int ctas = std::max(1, std::min(p.n_items - first, per_sm * p.sm_count));
    cudaMemsetAsync(p.counter, 0, sizeof(int), p.stream);
    if (mr <= 3)
        gather_sorted_f32<3><<<ctas, GS_THREADS, smem, p.stream>>>(v, p.items, p.facc, p.fexp, first,
                                                                  p.n_items, p.counter, p.max_grid_bytes);
    else
        gather_sorted_f32<4><<<ctas, GS_THREADS, smem, p.stream>>>(v, p.items, p.facc, p.fexp, first,
                                                                  p.n_items, p.counter, p.max_grid_bytes);
    const int fb = (int)std::min<long long>(4LL * p.sm_count, (p.M + 255) / 256);
    k_fixed_point_finish<<<fb, 256, 0, p.stream>>>(f, (const long long *)p.facc, p.fexp, p.M, p.skip);
    return cuda_status(cudaGetLastError());
}

}  // namespace agft
