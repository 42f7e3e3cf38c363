// Forward gather over the cell-sorted node records (every term with records:
// all terms of an FP32 plan that keeps them), the window interpolation step
// of the NFFT behind eq. (somafm), Sec. 3, FP32.
//
// Work items are the adjoint's (active term, node chunk) pairs.  A CTA copies
// the term's stored grid into shared memory.  gather_sorted_f32 gives each
// thread two consecutive records: the thread evaluates each node's 8 column
// and 2 m_row row window weights from the per-tap polynomials (coefficients
// broadcast from shared memory, 16 bytes at a time), reads the 6 x 8 grid
// values around the cell (the nodes of a warp mostly share a cell, so the
// reads are broadcasts, and one read serves both nodes when the pair shares a
// cell) and adds sum_i w_row[i] sum_t w_col[t] g[i][t] into node j's
// accumulator.  gather_mma_f32 (below) forms the same sums on the tensor
// cores.  The accumulators are 64-bit integers holding the values in
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

__device__ __forceinline__ const DevPlan &plan_of(const DevPlan &single, const BatchArgs &B, int prob) {
    return B.plans ? B.plans[prob] : single;
}

// per problem (blockIdx.y): partial sums of |Re| + |Im| of its coefficients
__global__ void k_fixed_point_partial(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base,
                                      double *part_base) {
    __shared__ double sh[32];
    const DevPlan &P = plan_of(single, B, blockIdx.y);
    if (P.skip && *P.skip) return;
    const float2 *fhat = fhat_base + P.vec_coef_off;
    const long long n = P.n_coeffs;
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
        part_base[(long long)blockIdx.y * FPE_BLOCKS + blockIdx.x] = s;
    }
}

// per problem (blockIdx.x): the exponent from its partial sums
__global__ void k_fixed_point_exponent(DevPlan single, BatchArgs B, const double *part_base) {
    const DevPlan &P = plan_of(single, B, blockIdx.x);
    if (threadIdx.x != 0 || (P.skip && *P.skip)) return;
    const double *part = part_base + (long long)blockIdx.x * FPE_BLOCKS;
    double s = 0.0;
    for (int b = 0; b < FPE_BLOCKS; ++b) s += part[b];
    int e = 100;
    // a cosine coefficient stands for 2^s exponential ones of 2^{-s/2} its size
    // (s <= 3): their absolute sum is at most 2^{3/2} = 2.83 times larger
    if (s > 0) e = 61 - (int)ceil(log2(s)) - (P.basis == ANOVA_BASIS_COS ? 2 : 0);
    *P.fexp = max(-100, min(100, e));
}

// per problem (blockIdx.y): f = empty-set coefficient, accumulators = 0
__global__ void k_sorted_forward_init(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base,
                                      float2 *f_base) {
    const DevPlan &P = plan_of(single, B, blockIdx.y);
    if (P.skip && *P.skip) return;
    const float2 *fhat = fhat_base + P.vec_coef_off;
    float2 c0 = make_float2(0.f, 0.f);
    for (int e = 0; e < P.n_empty; ++e) {
        const float2 c = fhat[P.empty_off[e]];
        c0.x += c.x;
        c0.y += c.y;
    }
    float2 *f = f_base + P.vec_node_off;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < P.M; j += (long long)gridDim.x * blockDim.x) {
        f[j] = c0;
        P.facc[2 * j] = 0ULL;
        P.facc[2 * j + 1] = 0ULL;
    }
}

// per problem (blockIdx.y): f[j] += acc[j] * 2^-e
__global__ void k_fixed_point_finish(DevPlan single, BatchArgs B, float2 *f_base) {
    const DevPlan &P = plan_of(single, B, blockIdx.y);
    if (P.skip && *P.skip) return;
    const double sc = ldexp(1.0, -*P.fexp);
    float2 *f = f_base + P.vec_node_off;
    const long long *acc = (const long long *)P.facc;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < P.M; j += (long long)gridDim.x * blockDim.x) {
        float2 v = f[j];
        v.x += (float)((double)acc[2 * j] * sc);
        v.y += (float)((double)acc[2 * j + 1] * sc);
        f[j] = v;
    }
}

// polynomial of tap t from the shared coefficient table (two float4 per tap),
// at two arguments; the same operations as horner8
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
gather_sorted_f32(DevPlan single, BatchArgs B, const int4 *__restrict__ items, int item_begin, int item_end,
                  int *counter, long long max_grid_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *S = (float2 *)smem;
    float4 *coef = (float4 *)(smem + max_grid_bytes);   // [8 column taps + 8 row taps][2]
    int &s_item = *(int *)(coef + 32);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = item_begin + atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= item_end) break;
        const int4 itm = items[item];
        const DevPlan &P = plan_of(single, B, itm.x);
        if (P.skip && *P.skip) continue;
        const long long M = P.M;
        unsigned long long *__restrict__ acc = P.facc;
        const float sc = __int_as_float((127 + *P.fexp) << 23);   // 2^e, exact scaling
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
        // a thread takes two consecutive records (mostly of one cell: then
        // every grid value read serves both); the warp iterates as a whole
        const int lane = tid & 31;
        for (long long wb = j0 + 2 * (tid - lane); wb < j1; wb += 2 * GS_THREADS) {
            const long long p = wb + 2 * lane;
            const bool ok0 = p < j1, ok1 = p + 1 < j1;
            const float4 q0 = __ldg(rec + (ok0 ? p : j1 - 1)), q1 = __ldg(rec + (ok1 ? p + 1 : j1 - 1));
            float wc0[8], wc1[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) horner_pair(coef + 2 * t, q0.y, q1.y, wc0[t], wc1[t]);
            const int off0 = __float_as_int(q0.z), off1 = __float_as_int(q1.z);
            const bool same = __all_sync(0xffffffffu, off0 == off1);
            float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f;
            if (two) {
#pragma unroll
                for (int i = 0; i < 2 * MR; ++i) {
                    float wr0, wr1;
                    horner_pair(coef + 16 + 2 * i, q0.x, q1.x, wr0, wr1);
                    const float2 *r0 = S + off0 + i * stride, *r1 = S + off1 + i * stride;
                    float tx0 = 0.f, ty0 = 0.f, tx1 = 0.f, ty1 = 0.f;
                    if (same) {
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const float2 a = r0[t];
                            tx0 = fmaf(wc0[t], a.x, tx0);
                            ty0 = fmaf(wc0[t], a.y, ty0);
                            tx1 = fmaf(wc1[t], a.x, tx1);
                            ty1 = fmaf(wc1[t], a.y, ty1);
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const float2 a = r0[t], c = r1[t];
                            tx0 = fmaf(wc0[t], a.x, tx0);
                            ty0 = fmaf(wc0[t], a.y, ty0);
                            tx1 = fmaf(wc1[t], c.x, tx1);
                            ty1 = fmaf(wc1[t], c.y, ty1);
                        }
                    }
                    sx0 = fmaf(wr0, tx0, sx0);
                    sy0 = fmaf(wr0, ty0, sy0);
                    sx1 = fmaf(wr1, tx1, sx1);
                    sy1 = fmaf(wr1, ty1, sy1);
                }
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 a = S[off0 + t], c = same ? a : S[off1 + t];
                    sx0 = fmaf(wc0[t], a.x, sx0);
                    sy0 = fmaf(wc0[t], a.y, sy0);
                    sx1 = fmaf(wc1[t], c.x, sx1);
                    sy1 = fmaf(wc1[t], c.y, sy1);
                }
            }
            if (ok0) {
                unsigned long long *a0 = acc + 2 * (long long)__float_as_int(q0.w);
                red_add_u64(a0, __float2ll_rn(sx0 * sc));
                red_add_u64(a0 + 1, __float2ll_rn(sy0 * sc));
            }
            if (ok1) {
                unsigned long long *a1 = acc + 2 * (long long)__float_as_int(q1.w);
                red_add_u64(a1, __float2ll_rn(sx1 * sc));
                red_add_u64(a1 + 1, __float2ll_rn(sy1 * sc));
            }
        }
        __syncthreads();   // the grid is read by every thread before the next item replaces it
    }
}

// ---- Forward gather of order-1/2 terms on the tensor cores ----
//
// Every tap weight is a degree-7 polynomial in the node's cell offset v, kept
// in the Chebyshev basis X_i (Window::ch): psi_k = sum_i C[k][i] X_i.  For the
// nodes j of one cell with grid window G (m_row x 8, complex)
//     f_j = sum_{r,k} G[r][k] psi_row,r(j) psi_col,k(j)
//         = sum_{l,i} X_l(v_row,j) H[l][i] X_i(v_col,j),   H = C_row^T G C_col,
// so a cell change costs two small products that turn G into H (8 x 8,
// complex), and each node only needs its 2 x 8 basis values: one lane
// computes them (the recurrence, 8 packed FP32 operations) and leaves them in
// shared memory.  A tile of 16 cell-sorted nodes takes P = X_col H^T (16 x 8,
// real and imaginary parts one mma.m16n8k8 each, three TF32 products) and
// f_j = sum_l X_l(v_row,j) P[j][l]: two FMAs per lane and a reduce-scatter
// over the 4 lanes that hold node j's columns.  The contraction index of every
// product is permuted (2t, 2t + 1 -> t, t + 4), so that lane (g, t) needs
// X_2t and X_2t+1 of both coordinates of nodes g, g + 8, one 16-byte read per
// node, and so that each accumulator fragment is the next product's operand
// as it stands.  A warp takes two tiles per step.  A tile holding nodes of
// several cells is run once per cell with the other nodes' rows of A zeroed.
// The sums go to the 64-bit fixed-point accumulators as in gather_sorted_f32,
// one (node, real or imaginary part) per lane.
//
// Records arrive in a per-warp ring (cp.async, DR steps ahead; L2 bulk
// prefetch PF steps ahead); the basis of a node lies in 4 chunks of 16 bytes
// (X_2c(v_row), X_2c+1(v_row), X_2c(v_col), X_2c+1(v_col)), chunk c of node
// u at position c ^ ((u / 2) mod 4), which keeps the writes (a lane per node)
// and the reads (a lane per chunk) free of bank conflicts.
constexpr int GM_TILE = 16, GM_STEP = 2 * GM_TILE;
struct GmRing {
    static constexpr int RING = 4, DR = 3, PF = 7;
    static constexpr size_t REC_BYTES = (size_t)RING * GM_STEP * 16;
    static constexpr size_t BYTES = REC_BYTES + (size_t)GM_STEP * 64;   // + basis chunks, per warp
    static_assert(DR < RING, "ring depth");
};
constexpr int GM_CTAS_PER_SM = 3;

__device__ __forceinline__ void mma3_tf32(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4],
                                          unsigned bh0, unsigned bh1, unsigned bl0, unsigned bl1) {
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, ah, bh0, bh1);
}

template <int MR>
__device__ __forceinline__ void gather_mma_run(const float4 *__restrict__ rec, int n, const float2 *S, int stride,
                                               bool ord2, const float *__restrict__ chr, const float *__restrict__ chc,
                                               unsigned long long *__restrict__ acc, float sc, float4 *rring,
                                               float4 *xs) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ns = (n + GM_STEP - 1) / GM_STEP;
    int cur = -1;            // cell whose H is in bh, bl
    unsigned bh[4], bl[4];   // B fragments of H: real part (b0, b1), imaginary part (b0, b1)
    // H = C_row^T G C_col for the cell at grid offset off.  Stage 1: D1_x[i][r]
    // = sum_k C_col[k][i] G_x[r][k] (A = C_col^T, rows 8..15 zero; B[k][r] =
    // G_x[r][k]); stage 2: H_x[l][i] = sum_r C_row[r][l] D1_x[i][r] (A[l][k] =
    // C_row[r(k)][l], B[k][i] = D1_x[i][r(k)], r(t) = 2t, r(t + 4) = 2t + 1).
    // Order 1: C_row = e_0 e_0^T and only grid row 0 exists.
    auto load_h = [&](int off) {
        const bool row_ok = ord2 ? g < 2 * MR : g == 0;   // grid row g of the window exists
        float2 g0 = make_float2(0.f, 0.f), g1 = g0;
        if (row_ok) {
            g0 = S[off + g * stride + t];
            g1 = S[off + g * stride + t + 4];
        }
        unsigned c1h[4], c1l[4], c2h[4], c2l[4];
        split_tf32_x2(pk2(__ldg(chc + t * NCOEF + g), __ldg(chc + (t + 4) * NCOEF + g)), c1h[0], c1l[0], c1h[2],
                      c1l[2]);
        float r0 = 0.f, r1 = 0.f;
        if (ord2) {
            r0 = __ldg(chr + 2 * t * NCOEF + g);
            r1 = __ldg(chr + (2 * t + 1) * NCOEF + g);
        } else {
            r0 = g == 0 && t == 0 ? 1.f : 0.f;
        }
        split_tf32_x2(pk2(r0, r1), c2h[0], c2l[0], c2h[2], c2l[2]);
        c1h[1] = c1h[3] = c1l[1] = c1l[3] = c2h[1] = c2h[3] = c2l[1] = c2l[3] = 0u;
        unsigned gh[4], gl[4];   // B of stage 1: (re k = t, re k = t + 4, im t, im t + 4)
        split_tf32_x2(pk2(g0.x, g1.x), gh[0], gl[0], gh[1], gl[1]);
        split_tf32_x2(pk2(g0.y, g1.y), gh[2], gl[2], gh[3], gl[3]);
        float ur[4] = {0.f, 0.f, 0.f, 0.f}, ui[4] = {0.f, 0.f, 0.f, 0.f};
        mma3_tf32(ur, c1h, c1l, gh[0], gh[1], gl[0], gl[1]);
        mma3_tf32(ui, c1h, c1l, gh[2], gh[3], gl[2], gl[3]);
        // ur = (D1_re[i = g][r = 2t], D1_re[g][2t + 1], 0, 0): the B fragment of stage 2
        unsigned uh[4], ul[4];
        split_tf32_x2(pk2(ur[0], ur[1]), uh[0], ul[0], uh[1], ul[1]);
        split_tf32_x2(pk2(ui[0], ui[1]), uh[2], ul[2], uh[3], ul[3]);
        float hr[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
        mma3_tf32(hr, c2h, c2l, uh[0], uh[1], ul[0], ul[1]);
        mma3_tf32(hi, c2h, c2l, uh[2], uh[3], ul[2], ul[3]);
        // hr = (H_re[l = g][i = 2t], H_re[g][2t + 1], 0, 0): B of the tile product
        split_tf32_x2(pk2(hr[0], hr[1]), bh[0], bl[0], bh[1], bl[1]);
        split_tf32_x2(pk2(hi[0], hi[1]), bh[2], bl[2], bh[3], bl[3]);
    };
    // tile h: A rows from the basis of nodes g, g + 8 (q0, q1 = their chunk t)
    auto tile_slow = [&](const unsigned (&ah)[4], const unsigned (&al)[4], int off0, int off1, float (&dre)[4],
                         float (&dim)[4]) {
        bool p0 = true, p1 = true;   // nodes g, g + 8 not yet covered
        for (;;) {
            // lanes t = 0 speak for their nodes
            const unsigned m0 = __ballot_sync(0xffffffffu, p0) & 0x11111111u;
            const unsigned m1 = __ballot_sync(0xffffffffu, p1) & 0x11111111u;
            if (!(m0 | m1)) break;
            const int src = __ffs(m0 ? m0 : m1) - 1;
            const int oc = __shfl_sync(0xffffffffu, m0 ? off0 : off1, src);
            const bool e0 = p0 && off0 == oc, e1 = p1 && off1 == oc;
            if (oc != cur) {
                load_h(oc);
                cur = oc;
            }
            const unsigned mh[4] = {e0 ? ah[0] : 0u, e1 ? ah[1] : 0u, e0 ? ah[2] : 0u, e1 ? ah[3] : 0u};
            const unsigned ml[4] = {e0 ? al[0] : 0u, e1 ? al[1] : 0u, e0 ? al[2] : 0u, e1 ? al[3] : 0u};
            mma3_tf32(dre, mh, ml, bh[0], bh[1], bl[0], bl[1]);
            mma3_tf32(dim, mh, ml, bh[2], bh[3], bl[2], bl[3]);
            p0 = p0 && !e0;
            p1 = p1 && !e1;
        }
    };
    const int sw = (g >> 1) & 3;   // chunk swizzle of nodes g, g + 8 (of every tile)
    const float4 *xq0 = xs + g * 4 + (t ^ sw);   // chunk t of node g of tile 0 (+ 8 nodes: + 32)
    float4 *xw = xs + lane * 4;                  // this lane's node's chunks
    const int msw = (lane >> 1) & 3;
    unsigned long long *acc_t = acc + (t & 1);   // this lane's part (real or imaginary)
    for (int i = -GmRing::DR; i < ns; ++i) {
        {
            const int qr = i + GmRing::DR, qp = i + GmRing::PF;
            // the records of step qp into L2 (whole records of the run only)
            if (lane == 0 && qp < ns && qp >= GmRing::DR)
                prefetch_l2_bulk(rec + GM_STEP * qp, 16u * (unsigned)min(GM_STEP, n - GM_STEP * qp));
            // record u of step qr; past the end the last record again (not written back)
            if (qr < ns)
                cp_async16(&rring[((unsigned)qr % GmRing::RING) * GM_STEP + lane], rec + min(GM_STEP * qr + lane, n - 1));
            cp_async_commit();
        }
        if (i < 0) continue;
        cp_async_wait_n<GmRing::DR>();   // the records of step i (this lane's own copy) have landed
        // the basis of node `lane`, (row, column) pairs: X_{k+1} = X_{k-1} + (-1)^k 2 v X_k
        const float4 r = rring[((unsigned)i % GmRing::RING) * GM_STEP + lane];
        const int my_cell = __float_as_int(r.z), my_j = __float_as_int(r.w);
        {
            const f32x2 v = pk2(r.x, r.y);
            const f32x2 up = mul2(v, pk2(2.f, 2.f)), um = mul2(v, pk2(-2.f, -2.f));
            f32x2 x[NCOEF];
            x[0] = pk2(1.f, 1.f);
            x[1] = v;
#pragma unroll
            for (int k = 2; k < NCOEF; ++k) x[k] = fma2((k & 1) ? up : um, x[k - 1], x[k - 2]);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float a0, b0, a1, b1;   // (row, column) of X_2c and X_2c+1
                upk2(x[2 * c], a0, b0);
                upk2(x[2 * c + 1], a1, b1);
                xw[c ^ msw] = make_float4(a0, a1, b0, b1);
            }
        }
        __syncwarp();   // the step's basis chunks visible to the warp
        const bool fast = __all_sync(0xffffffffu, my_cell == cur);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n0 = GM_TILE * h + g, n1 = n0 + 8;   // nodes of this lane's A rows
            const float4 q0 = xq0[GM_TILE * 4 * h], q1 = xq0[GM_TILE * 4 * h + 32];
            // A: a0 = X_2t(v_col) of node g, a1 = of node g + 8, a2 = X_2t+1(v_col) of g, a3 = of g + 8
            unsigned ah[4], al[4];
            split_tf32_x2(pk2(q0.z, q0.w), ah[0], al[0], ah[2], al[2]);
            split_tf32_x2(pk2(q1.z, q1.w), ah[1], al[1], ah[3], al[3]);
            float dre[4] = {0.f, 0.f, 0.f, 0.f}, dim[4] = {0.f, 0.f, 0.f, 0.f};
            if (fast) {
                mma3_tf32(dre, ah, al, bh[0], bh[1], bl[0], bl[1]);
                mma3_tf32(dim, ah, al, bh[2], bh[3], bl[2], bl[3]);
            } else {
                tile_slow(ah, al, __shfl_sync(0xffffffffu, my_cell, n0), __shfl_sync(0xffffffffu, my_cell, n1), dre,
                          dim);
            }
            // d0, d1: node g, l = 2t, 2t + 1; d2, d3: node g + 8.  Row basis X_2t, X_2t+1 = q.x, q.y
            const float fx0 = fmaf(q0.y, dre[1], q0.x * dre[0]), fy0 = fmaf(q0.y, dim[1], q0.x * dim[0]);
            const float fx1 = fmaf(q1.y, dre[3], q1.x * dre[2]), fy1 = fmaf(q1.y, dim[3], q1.x * dim[2]);
            // reduce-scatter over the 4 lanes of nodes g, g + 8: lane t ends with
            // value t of (node g: re, im; node g + 8: re, im) summed over the lanes
            const bool hi2 = t & 2, hi1 = t & 1;
            float k0 = hi2 ? fx1 : fx0, k1 = hi2 ? fy1 : fy0;   // the pair this lane keeps
            k0 += __shfl_xor_sync(0xffffffffu, hi2 ? fx0 : fx1, 2);
            k1 += __shfl_xor_sync(0xffffffffu, hi2 ? fy0 : fy1, 2);
            const float v = (hi1 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, hi1 ? k0 : k1, 1);
            const int nl = t < 2 ? n0 : n1;
            const int j = __shfl_sync(0xffffffffu, my_j, nl);
            if (GM_STEP * i + nl < n) red_add_u64(acc_t + 2 * (long long)j, __float2ll_rn(v * sc));
        }
        __syncwarp();   // ring slot i and the basis chunks are read before later steps refill them
    }
    cp_async_wait0();
}

template <int MR>
__global__ void __launch_bounds__(GS_THREADS, GM_CTAS_PER_SM)
gather_mma_f32(DevPlan single, BatchArgs B, const int4 *__restrict__ items, int item_begin, int item_end,
               int *counter, long long max_grid_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *S = (float2 *)smem;
    unsigned char *rings = smem + max_grid_bytes;
    constexpr int NW = GS_THREADS / 32;
    int &s_item = *(int *)(rings + NW * GmRing::BYTES);
    const int tid = threadIdx.x, warp = tid >> 5;
    float4 *rring = (float4 *)(rings + warp * GmRing::BYTES);
    float4 *xs = (float4 *)(rings + warp * GmRing::BYTES + GmRing::REC_BYTES);
    for (;;) {
        if (tid == 0) s_item = item_begin + atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= item_end) break;
        const int4 itm = items[item];
        const DevPlan &P = plan_of(single, B, itm.x);
        if (P.skip && *P.skip) continue;
        const long long M = P.M;
        const float sc = __int_as_float((127 + *P.fexp) << 23);   // 2^e, exact scaling
        const Term &T = P.terms[P.act[itm.y]];
        const long long j0 = M * itm.z / itm.w, j1 = M * (itm.z + 1) / itm.w;
        {
            const float4 *gsrc = (const float4 *)(P.grids + T.grid_off);
            float4 *S4 = (float4 *)S;
            const long long n4 = T.grid_bytes / 16;
            for (long long e = tid; e < n4; e += GS_THREADS) S4[e] = __ldg(gsrc + e);
        }
        __syncthreads();
        // warp w takes a contiguous run of the item's records (whole steps of two tiles)
        const long long len = j1 - j0, per = (len + GM_STEP * NW - 1) / (GM_STEP * NW) * GM_STEP;
        const long long a = j0 + warp * per, b = min(j1, a + per);
        if (a < b)
            gather_mma_run<MR>(P.srec + (long long)T.sort_slot * M + a, (int)(b - a), S, T.stride, T.order == 2,
                               T.order == 2 ? &P.windows[T.wr].ch[0][0] : nullptr, &P.windows[T.wc].ch[0][0],
                               P.facc, sc, rring, xs);
        __syncthreads();   // the grid is read by every warp before the next item replaces it
    }
}

int gather_sorted_launch(cudaStream_t st, const DevPlan &v, const BatchArgs &B, int P, const float2 *fhat,
                         float2 *f, const int4 *items, int n_items3, int item_end, int *counter,
                         long long max_grid_bytes, long long max_M, int sm_count, int mr, double *part, bool tc) {
    const int item_begin = 0;
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(gather_sorted_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(gather_sorted_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(gather_mma_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(gather_mma_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
    });
    // Order-1/2 items on the tensor cores only where no third-order item (the
    // first n_items3, always on the CUDA cores) precedes them: two launches in
    // a row idle the GPU at the seam, which costs more than the tensor cores
    // gain (10 % on the d = 10, |u| <= 3 workload).
    const int cuda_end = tc && n_items3 == 0 ? 0 : item_end;
    const int nb = (int)std::max<long long>(1, std::min<long long>(4LL * sm_count / std::max(1, P) + 1,
                                                                   (max_M + 255) / 256));
    k_fixed_point_partial<<<dim3(FPE_BLOCKS, P), 256, 0, st>>>(v, B, fhat, part);
    k_fixed_point_exponent<<<P, 32, 0, st>>>(v, B, part);
    k_sorted_forward_init<<<dim3(nb, P), 256, 0, st>>>(v, B, fhat, f);
    const size_t smem = (size_t)max_grid_bytes + 32 * sizeof(float4) + 16;
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(3, (size_t)(MAX_SMEM + 1024) / (smem + 1024)));
    const size_t smem_mma = (size_t)max_grid_bytes + (GS_THREADS / 32) * GmRing::BYTES + 16;
    const int per_sm_mma = (int)std::max<size_t>(
        1, std::min<size_t>(GM_CTAS_PER_SM, (size_t)(MAX_SMEM + 1024) / (smem_mma + 1024)));
    if (item_end > item_begin) cudaMemsetAsync(counter, 0, 2 * sizeof(int), st);
    if (cuda_end > item_begin) {
        const int ctas = std::max(1, std::min(cuda_end - item_begin, per_sm * sm_count));
        if (mr <= 3)
            gather_sorted_f32<3><<<ctas, GS_THREADS, smem, st>>>(v, B, items, item_begin, cuda_end, counter,
                                                                 max_grid_bytes);
        else
            gather_sorted_f32<4><<<ctas, GS_THREADS, smem, st>>>(v, B, items, item_begin, cuda_end, counter,
                                                                 max_grid_bytes);
    }
    if (item_end > cuda_end) {
        const int ctas = std::max(1, std::min(item_end - cuda_end, per_sm_mma * sm_count));
        if (mr <= 3)
            gather_mma_f32<3><<<ctas, GS_THREADS, smem_mma, st>>>(v, B, items, cuda_end, item_end, counter + 1,
                                                                  max_grid_bytes);
        else
            gather_mma_f32<4><<<ctas, GS_THREADS, smem_mma, st>>>(v, B, items, cuda_end, item_end, counter + 1,
                                                                  max_grid_bytes);
    }
    k_fixed_point_finish<<<dim3(nb, P), 256, 0, st>>>(v, B, f);
    return cuda_status(cudaGetLastError());
}

// single plan: every term has records (third-order ones without records were
// handled by the point-major gather, which then wrote f; see trafo.cu)
int launch_gather_sorted_f32(Plan &p, const float2 *fhat, float2 *f) {
    DevPlan v = dev_view(p);
    BatchArgs B;
    std::memset(&B, 0, sizeof(B));
    int mr = 3;
    for (int s = 0; s < p.n_terms; ++s)
        if (p.h_terms[s].mr > 0) mr = p.h_terms[s].mr;
    return gather_sorted_launch(p.stream, v, B, 1, fhat, f, p.items, p.n_items3, p.n_items, p.counter,
                                p.max_grid_bytes, p.M, p.sm_count, mr, (double *)p.scratch, p.cell_tc);
}

}  // namespace agft
