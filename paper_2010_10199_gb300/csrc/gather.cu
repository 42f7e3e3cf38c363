// Forward gather over all terms, f_j = c_empty + sum_u sum_taps g_u[tap] psi(...)
// (the window interpolation step of the NFFT behind eq. (somafm), Sec. 3), FP32.
//
// Point-major and persistent: a CTA owns a tile of 128 nodes whose coordinates
// it stages in shared memory, and walks the term schedule; each term's stored
// grid arrives in shared memory by a bulk async copy into one of two buffers,
// tracked by an mbarrier.  There is no block-wide barrier per term: every warp
// counts itself out of a buffer when done with it, and the last warp out
// issues the copy of the term two steps ahead into it, so warps drift freely
// within that window.  A half-warp owns 8 nodes and evaluates one node at a
// time with 16 lanes = 2 grid rows x 8 grid columns, so a warp instruction
// reads 2 nodes x 2 rows x 8 columns; the row pitch = 8 (mod 16) complex
// elements puts the two rows of a node in complementary bank halves.  The
// window polynomials are evaluated once per (node, tap): order-2 terms share
// the row weights of their first coordinate across the row group (lane (r, k)
// evaluates rows r, r+2, .. of node k and shuffles hand them round), and the
// column weights of two nodes come from the two lane groups r = 0, 1.  Lanes
// accumulate over all terms in registers; a transposed reduce-scatter per tile
// finishes each node.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

constexpr int G2_THREADS = 256;
constexpr int G2_WARPS = G2_THREADS / 32;
constexpr int G2_PTS = 8;                              // nodes per half-warp
constexpr int G2_TILE = (G2_THREADS / 16) * G2_PTS;    // 128 nodes per CTA tile
static_assert(G2_PTS == 8, "coordinate loads read a half-warp's nodes as two float4");
static_assert(G2_TILE == GATHER_TILE, "tile size shared with the batch tables");

// Problem of a tile and the number of its terms still to run (0 when the
// problem's skip flag is set).
__device__ __forceinline__ const DevPlan &tile_plan(const DevPlan &single, const BatchArgs &B, int tile, int &lt) {
    if (!B.plans) {
        lt = tile;
        return single;
    }
    const int p = B.tile_prob[tile];
    lt = tile - B.tile0[p];
    return B.plans[p];
}

__device__ __forceinline__ int tile_terms(const DevPlan &D) { return (D.skip && *D.skip) ? 0 : D.n_act; }

// this CTA's first tile at or after t (stride gridDim.x) with terms to run
__device__ __forceinline__ int next_busy_tile(const DevPlan &single, const BatchArgs &B, int t, int n_tiles) {
    int lt;
    while (t < n_tiles && tile_terms(tile_plan(single, B, t, lt)) == 0) t += gridDim.x;
    return t;
}

// Moves (t, s) = (tile, term of that tile) `steps` terms ahead in this CTA's
// stream; t >= n_tiles when the stream ends first.
__device__ __forceinline__ void stream_ahead(const DevPlan &single, const BatchArgs &B, int n_tiles, int &t, int &s,
                                             int steps) {
    s += steps;
    while (t < n_tiles) {
        int lt;
        const int nt = tile_terms(tile_plan(single, B, t, lt));
        if (s < nt) return;
        s -= nt;
        t = next_busy_tile(single, B, t + gridDim.x, n_tiles);
    }
}

// One thread: copy the stored grid of term s of tile t into buffer buf.
template <typename G>
__device__ __forceinline__ void issue_grid(const DevPlan &single, const BatchArgs &B, int t, int s, int buf,
                                           G *sm2, int gb_el, uint64_t *bars) {
    int lt;
    const DevPlan &D = tile_plan(single, B, t, lt);
    const ActRec &R = D.act_rec[s];
    fence_proxy_async();
    mbar_expect_tx(&bars[buf], (uint32_t)R.grid_bytes);
    bulk_g2s(sm2 + (buf ? gb_el : 0), (const G *)D.grids + R.grid_off, (uint32_t)R.grid_bytes, &bars[buf]);
}

template <int MR, int PITCH, typename G>
__global__ void __launch_bounds__(G2_THREADS, 2)
gather2_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base, float2 *__restrict__ f_base,
            int n_tiles, int pitch_rt, long long max_grid_bytes, int dmax) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    G *sm2 = (G *)sm_raw;   // two grid buffers, grid elements of the plan's storage type
    const int gb_el = (int)(max_grid_bytes / sizeof(G));
    float *xs = (float *)(sm2 + 2 * gb_el);                     // [d][G2_TILE]
    uint64_t *bars = (uint64_t *)(xs + dmax * G2_TILE);         // full barriers of the two buffers
    unsigned int *outs = (unsigned int *)(bars + 2);            // warps done with each buffer (running count)
    (void)pitch_rt;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int half = lane >> 4;
    const int sub = lane & 15;
    const int r = sub >> 3, k = sub & 7;
    const int hw = (tid >> 5) * 2 + half;
    const int pbase = hw * G2_PTS;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        outs[0] = outs[1] = 0;
        fence_barrier_init();
    }
    __syncthreads();

    int tile = next_busy_tile(single, B, blockIdx.x, n_tiles);
    if (tile < n_tiles && tid == 0) {
        int t1 = tile, s1 = 0;
        issue_grid(single, B, t1, s1, 0, sm2, gb_el, bars);
        stream_ahead(single, B, n_tiles, t1, s1, 1);
        if (t1 < n_tiles) issue_grid(single, B, t1, s1, 1, sm2, gb_el, bars);
    }

    long long it = 0;
    while (tile < n_tiles) {
        int lt;
        const DevPlan &D = tile_plan(single, B, tile, lt);
        const int nt = tile_terms(D);
        const int next_tile = next_busy_tile(single, B, tile + gridDim.x, n_tiles);
        const long long M = D.M;
        const int d = D.d;
        const float *__restrict__ X = D.x;
        const float2 *fhat = fhat_base + D.vec_coef_off;
        float2 *f = f_base + D.vec_node_off;
        const long long p0 = (long long)lt * G2_TILE;
        float2 c0 = make_float2(0.f, 0.f);
        for (int e = 0; e < D.n_empty; ++e) {
            float2 c = fhat[D.empty_off[e]];
            c0.x += c.x;
            c0.y += c.y;
        }
        // stage the tile's coordinates (the previous tile ended with a barrier)
        for (int e = tid; e < d * G2_TILE; e += G2_THREADS) {
            const int c = e / G2_TILE, i = e - c * G2_TILE;
            const long long pp = p0 + i;
            xs[e] = pp < M ? __ldg(X + (long long)c * M + pp) : 0.f;
        }
        __syncthreads();

        float ax[G2_PTS], ay[G2_PTS];
        float rw[G2_PTS][MR];
        int rbase[G2_PTS];
        float cc[NCOEF];
#pragma unroll
        for (int i = 0; i < G2_PTS; ++i) {
            ax[i] = ay[i] = 0.f;
            rbase[i] = 0;
#pragma unroll
            for (int j = 0; j < MR; ++j) rw[i][j] = 0.f;
        }
        int cur_wc = -1;
        ActRec R = D.act_rec[0];
        for (int s = 0; s < nt; ++s, ++it) {
            ActRec Rn = R;
            if (s + 1 < nt) Rn = D.act_rec[s + 1];   // prefetch the next term's record
            const int b = (int)(it & 1);
            const uint32_t parity = (uint32_t)((it >> 1) & 1);
            const int order = R.order, n = R.n;
            const int pitch = PITCH ? PITCH : R.stride;   // order-2 row pitch of this problem
            const float nf = (float)n, hn = 0.5f * (float)n, nm1 = (float)(n - 1);
            if (R.wc != cur_wc) {
                const float *wsrc = D.windows[R.wc].c[k];
#pragma unroll
                for (int i = 0; i < NCOEF; ++i) cc[i] = __ldg(wsrc + i);
                cur_wc = R.wc;
            }
            if (order == 2 && R.newgroup) {
                // lane (r, k): rows r, r+2, .. of node k; then every lane
                // fetches its rows for all 8 nodes of its half-warp
                float myrw[MR];
                {
                    const float t = fmaf(xs[R.row0 * G2_TILE + pbase + k], nf, hn);
                    const float fl = fminf(floorf(t), nm1);
                    const float v = fmaf(2.f, t - fl, -1.f);
#pragma unroll
                    for (int j = 0; j < MR; ++j) myrw[j] = horner8(D.windows[R.wr].c[r + 2 * j], v);
                }
                const float *xr = xs + R.row0 * G2_TILE + pbase;
#pragma unroll
                for (int i = 0; i < G2_PTS; ++i) {
                    const float t = fmaf(xr[i], nf, hn);
                    const float fl = fminf(floorf(t), nm1);
                    rbase[i] = ((int)fl + r) * pitch + k;   // stored row fl + r (row halo MR - 1)
#pragma unroll
                    for (int j = 0; j < MR; ++j)
                        rw[i][j] = __shfl_sync(0xffffffffu, myrw[j], (half << 4) | (r << 3) | i);
                }
            }
            mbar_wait(&bars[b], parity, D.err, 1);
            const int boff = b ? gb_el : 0;
            const float *xc = xs + R.col * G2_TILE + pbase;
            if (order == 2) {
                // the half-warp's 8 coordinates in two 16-byte loads (broadcast to its lanes)
                float xcv[G2_PTS];
                {
                    const float4 c0 = *(const float4 *)xc, c1 = *(const float4 *)(xc + 4);
                    xcv[0] = c0.x, xcv[1] = c0.y, xcv[2] = c0.z, xcv[3] = c0.w;
                    xcv[4] = c1.x, xcv[5] = c1.y, xcv[6] = c1.z, xcv[7] = c1.w;
                }
#pragma unroll
                for (int i = 0; i < G2_PTS; i += 2) {
                    const float t0 = fmaf(xcv[i], nf, hn), t1 = fmaf(xcv[i + 1], nf, hn);
                    const float fl0 = fminf(floorf(t0), nm1), fl1 = fminf(floorf(t1), nm1);
                    const float wt = horner8(cc, r ? fmaf(2.f, t1 - fl1, -1.f) : fmaf(2.f, t0 - fl0, -1.f));
                    const float cw0 = __shfl_sync(0xffffffffu, wt, (half << 4) | k);
                    const float cw1 = __shfl_sync(0xffffffffu, wt, (half << 4) | 8 | k);
                    const int idx0 = boff + rbase[i] + (int)fl0;
                    const int idx1 = boff + rbase[i + 1] + (int)fl1;
                    float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f;
#pragma unroll
                    for (int j = 0; j < MR; ++j) {
                        const float2 g0 = GridEl<G>::load(sm2[idx0 + 2 * j * pitch]);
                        const float2 g1 = GridEl<G>::load(sm2[idx1 + 2 * j * pitch]);
                        sx0 = fmaf(rw[i][j], g0.x, sx0);
                        sy0 = fmaf(rw[i][j], g0.y, sy0);
                        sx1 = fmaf(rw[i + 1][j], g1.x, sx1);
                        sy1 = fmaf(rw[i + 1][j], g1.y, sy1);
                    }
                    ax[i] = fmaf(cw0, sx0, ax[i]);
                    ay[i] = fmaf(cw0, sy0, ay[i]);
                    ax[i + 1] = fmaf(cw1, sx1, ax[i + 1]);
                    ay[i + 1] = fmaf(cw1, sy1, ay[i + 1]);
                }
            } else if (order == 1) {
                // lane group r takes nodes i + r of each pair
#pragma unroll
                for (int i = 0; i < G2_PTS; i += 2) {
                    const float t = fmaf(xc[i + r], nf, hn);
                    const float fl = fminf(floorf(t), nm1);
                    const float cw = horner8(cc, fmaf(2.f, t - fl, -1.f));
                    const float2 g = GridEl<G>::load(sm2[boff + (int)fl + k]);
                    const float vx = cw * g.x, vy = cw * g.y;
                    ax[i] += r ? 0.f : vx;
                    ay[i] += r ? 0.f : vy;
                    ax[i + 1] += r ? vx : 0.f;
                    ay[i + 1] += r ? vy : 0.f;
                }
            } else {
                // order 3: rows (first, second) wrap modulo n.  The row weights
                // come from the per-tap polynomials: lane (0, k) evaluates tap k of
                // the first row coordinate, lane (1, k) tap k of the second, and
                // shuffles hand them round (all 2 MR first-row taps, rows r, r+2, ..
                // of the second).
                const Term &T = D.terms[R.term];
                const int stride = T.stride;
                const float *xa_p = xs + T.row0 * G2_TILE + pbase;
                const float *xb_p = xs + T.row1 * G2_TILE + pbase;
                const G *Gs = sm2 + boff;
                float rcf[NCOEF];
                {
                    const float *src = D.windows[R.wr].c[min(k, 2 * MR - 1)];
#pragma unroll
                    for (int q = 0; q < NCOEF; ++q) rcf[q] = __ldg(src + q);
                }
#pragma unroll
                for (int i = 0; i < G2_PTS; ++i) {
                    float ta, tb, tc;
                    const int fa = grid_pos(xa_p[i], n, ta);
                    const int fb = grid_pos(xb_p[i], n, tb);
                    const int fc = grid_pos(xc[i], n, tc);
                    const float cw = horner8(cc, 2.f * tc - 1.f);
                    const float wrow = horner8(rcf, r ? 2.f * tb - 1.f : 2.f * ta - 1.f);
                    float wa[2 * MR], wb[MR];
                    int rb[MR];
#pragma unroll
                    for (int q = 0; q < 2 * MR; ++q) wa[q] = __shfl_sync(0xffffffffu, wrow, (half << 4) | q);
#pragma unroll
                    for (int j = 0; j < MR; ++j) {
                        wb[j] = __shfl_sync(0xffffffffu, wrow, (half << 4) | 8 | (r + 2 * j));
                        rb[j] = wrap(fb - MR + 1 + r + 2 * j, n);
                    }
                    const int cidx = wrap(fc - T.mc + 1 + k, n);
                    float sx = 0.f, sy = 0.f;
#pragma unroll
                    for (int ia = 0; ia < 2 * MR; ++ia) {
                        const int row = wrap(fa - MR + 1 + ia, n) * n;
                        float tx = 0.f, ty = 0.f;
#pragma unroll
                        for (int j = 0; j < MR; ++j) {
                            const float2 v = GridEl<G>::load(Gs[(row + rb[j]) * stride + cidx]);
                            tx = fmaf(wb[j], v.x, tx);
                            ty = fmaf(wb[j], v.y, ty);
                        }
                        sx = fmaf(wa[ia], tx, sx);
                        sy = fmaf(wa[ia], ty, sy);
                    }
                    ax[i] = fmaf(cw, sx, ax[i]);
                    ay[i] = fmaf(cw, sy, ay[i]);
                }
            }
            // done with buffer b: the last warp out refills it with the term
            // two steps ahead in this CTA's stream
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const unsigned int prev = atomicAdd(&outs[b], 1u);
                if ((prev + 1) % G2_WARPS == 0) {
                    __threadfence_block();
                    int t2 = tile, s2 = s;
                    stream_ahead(single, B, n_tiles, t2, s2, 2);
                    if (t2 < n_tiles) issue_grid(single, B, t2, s2, b, sm2, gb_el, bars);
                }
            }
            R = Rn;
        }
        // reduce over the 16 lanes of each half-warp: first the two row halves
        // (lane ^ 8), then a transposed reduce-scatter over the 8 nodes
#pragma unroll
        for (int i = 0; i < G2_PTS; ++i) {
            ax[i] += __shfl_xor_sync(0xffffffffu, ax[i], 8);
            ay[i] += __shfl_xor_sync(0xffffffffu, ay[i], 8);
        }
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {
            const bool up = (sub & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const float sx = up ? ax[i] : ax[i + o];
                const float sy = up ? ay[i] : ay[i + o];
                const float kx = up ? ax[i + o] : ax[i];
                const float ky = up ? ay[i + o] : ay[i];
                ax[i] = kx + __shfl_xor_sync(0xffffffffu, sx, o);
                ay[i] = ky + __shfl_xor_sync(0xffffffffu, sy, o);
            }
        }
        const long long pp = p0 + pbase + (sub & 7);
        if (sub < 8 && pp < M) f[pp] = make_float2(ax[0] + c0.x, ay[0] + c0.y);
        __syncthreads();   // every warp is done with xs before the next tile stages it
        tile = next_tile;
    }
}

template <int MR, int PITCH, typename G>
static void launch_one(cudaStream_t st, const DevPlan &v, const BatchArgs &B, const float2 *fhat, float2 *f,
                       int n_tiles, size_t smem, int ctas, int pitch, long long max_grid_bytes, int dmax) {
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(gather2_f32<MR, PITCH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
    });
    gather2_f32<MR, PITCH, G><<<ctas, G2_THREADS, smem, st>>>(v, B, fhat, f, n_tiles, pitch, max_grid_bytes, dmax);
}

template <int MR>
static void launch_mr(cudaStream_t st, const DevPlan &v, const BatchArgs &B, const float2 *fhat, float2 *f,
                      int n_tiles, size_t smem, int ctas, int pitch, long long max_grid_bytes, int dmax, int prec) {
    if (prec == ANOVA_PREC_F16) {
        launch_one<MR, 0, __half2>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax);
        return;
    }
    if (prec == ANOVA_PREC_BF16) {
        launch_one<MR, 0, __nv_bfloat162>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax);
        return;
    }
    switch (pitch) {
        case 40: launch_one<MR, 40, float2>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax); break;
        case 72: launch_one<MR, 72, float2>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax); break;
        default: launch_one<MR, 0, float2>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax); break;
    }
}

int gather_launch(cudaStream_t st, const DevPlan &v, const BatchArgs &B, const float2 *fhat, float2 *f,
                  int n_tiles, int mr, int pitch, long long max_grid_bytes, int dmax, int sm_count, int prec) {
    const size_t smem = (size_t)max_grid_bytes * 2 + (size_t)dmax * G2_TILE * 4 + 64;   // + barriers, counters
    if (smem > (size_t)MAX_SMEM) return ANOVA_ERR_UNSUPPORTED;
    if (n_tiles <= 0) return ANOVA_OK;
    const int per_sm = smem * 2 <= (size_t)MAX_SMEM ? 2 : 1;
    const int ctas = std::max(1, std::min(n_tiles, per_sm * sm_count));
    if (mr <= 3)
        launch_mr<3>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax, prec);
    else
        launch_mr<4>(st, v, B, fhat, f, n_tiles, smem, ctas, pitch, max_grid_bytes, dmax, prec);
    return cuda_status(cudaGetLastError());
}

int launch_gather_f32(Plan &p, const float2 *fhat, float2 *f) {
    DevPlan v = dev_view(p);
    BatchArgs B;
    std::memset(&B, 0, sizeof(B));
    const int n_tiles = (int)((p.M + G2_TILE - 1) / G2_TILE);
    int mr = 3;
    for (int s = 0; s < p.n_terms; ++s)
        if (p.h_terms[s].mr > 0) mr = p.h_terms[s].mr;
    return gather_launch(p.stream, v, B, fhat, f, n_tiles, mr, p.pitch2, p.max_grid_bytes, p.d, p.sm_count,
                         p.precision);
}

}  // namespace agft
