// Forward grouped transform f = F fhat (Definition "grouped Fourier transform"
// and eq. (somafm), Sec. 3), FP32.
//
//   1. trafo_pre: per term, zero-extend the block fhat(u) to ghat(u) on the
//      n^{|u|} grid (the extension before eq. (somafm)), multiply by the
//      deconvolution factors, run the oversampled FFT (sign +) in shared
//      memory and store the grid with its halos.
//   2. gather: all terms fused, point-major.  A CTA owns a tile of 256 nodes;
//      each half-warp owns 16 nodes and evaluates them one at a time with its
//      16 lanes = 2 rows x 8 columns of the window, reading the term's grid from
//      shared memory (double-buffered bulk async copies from L2).  Lanes keep
//      per-node partial sums over all terms in registers; one transposed
//      reduce-scatter per tile leaves node i's value in lane i.
#include <cstdio>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

__device__ __forceinline__ int freq_index(int q, int N) { return q < N / 2 ? q - N / 2 : q - N / 2 + 1; }

// ------------------------------------------------------------ pre-pass ----

__global__ void trafo_pre_f32(DevPlan P, const float2 *__restrict__ fhat, float2 *__restrict__ grids) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Term T = P.terms[blockIdx.x];
    const int n = T.n, s = T.order, N = T.N;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    float2 *a = (float2 *)smem_raw;
    float2 *b = a + fe;
    for (int i = threadIdx.x; i < fe; i += blockDim.x) a[i] = make_float2(0.f, 0.f);
    __syncthreads();
    // zero-extended, deconvolved coefficients at k mod n
    const int Nm = N - 1;
    for (long long q = threadIdx.x; q < T.coef_len; q += blockDim.x) {
        long long r = q;
        int pos = 0, mul = 1;
        float D = 1.f;
        for (int t = s - 1; t >= 0; --t) {
            int it = (int)(r % Nm);
            r /= Nm;
            int k = freq_index(it, N);
            int km = k < 0 ? k + n : k;
            pos += km * mul;
            mul *= n;
            D *= (t == s - 1) ? P.deconv[T.dc_off + it] : P.deconv[T.dr_off + it];
        }
        float2 c = fhat[T.coef_off + q];
        a[pos] = make_float2(c.x * D, c.y * D);
    }
    __syncthreads();
    // FFT along every axis (sign +): g_q = sum_k ghat_k exp(+2 pi i k q / n)
    float2 *cur = a, *oth = b;
    int inner = 1;
    for (int ax = s - 1; ax >= 0; --ax) {
        // lines along axis ax: element stride `inner`
        int rad[24];
        int ns = fft_radices(n, rad);
        (void)ns;
        // smem_fft with generic line bases: handle by looping over outer blocks
        const int nlines = fe / n;
        // express lines as (outer, inner) pairs: base = outer * inner * n + in
        int which;
        {
            // Stockham over all lines at once
            using C = float2;
            C *src = cur, *dst = oth;
            which = 0;
            int Ns = 1;
            for (int st = 0; st < ns; ++st) {
                const int Rr = rad[st];
                const int nb = n / Rr;
                for (int w = threadIdx.x; w < nlines * nb; w += blockDim.x) {
                    const int l = w / nb, j = w - l * nb;
                    const int base = (l / inner) * inner * n + (l % inner);
                    const C *in = src + base;
                    C *out = dst + base;
                    C v[5];
                    const int jm = j % Ns;
                    for (int r = 0; r < Rr; ++r) {
                        C x = in[(j + r * nb) * inner];
                        if (r && jm) {
                            float sn, cs;
                            sincospif((float)(2 * r * jm) / (float)(Ns * Rr), &sn, &cs);
                            x = cmul(x, make_float2(cs, sn));
                        }
                        v[r] = x;
                    }
                    C V[5];
                    if (Rr == 2) {
                        V[0] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
                        V[1] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
                    } else if (Rr == 4) {
                        C s0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
                        C d0 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
                        C s1 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
                        C d1 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
                        C jd1 = make_float2(-d1.y, d1.x);   // +i d1
                        V[0] = make_float2(s0.x + s1.x, s0.y + s1.y);
                        V[2] = make_float2(s0.x - s1.x, s0.y - s1.y);
                        V[1] = make_float2(d0.x + jd1.x, d0.y + jd1.y);
                        V[3] = make_float2(d0.x - jd1.x, d0.y - jd1.y);
                    } else {
                        for (int q = 0; q < Rr; ++q) {
                            C acc = v[0];
                            for (int r = 1; r < Rr; ++r) {
                                float sn, cs;
                                sincospif((float)(2 * ((r * q) % Rr)) / (float)Rr, &sn, &cs);
                                C t = cmul(v[r], make_float2(cs, sn));
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
                C *t = src;
                src = dst;
                dst = t;
                which ^= 1;
                Ns *= Rr;
            }
        }
        if (which) {
            float2 *t = cur;
            cur = oth;
            oth = t;
        }
        inner *= n;
    }
    // store with halos
    float2 *g = grids + T.grid_off;
    const int ecols = T.stride;
    const long long total = (long long)T.erows * ecols;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        int er = (int)(e / ecols), ec = (int)(e % ecols);
        float2 v = make_float2(0.f, 0.f);
        if (s <= 2) {
            if (ec < n + 2 * T.hc + 1) {
                int qc = wrap(ec - T.hc, n);
                int qr = s == 2 ? wrap(er - T.hr, n) : 0;
                v = cur[qr * n + qc];
            }
        } else {
            if (ec < n) v = cur[er * n + ec];
        }
        g[e] = v;
    }
}

// -------------------------------------------------------------- gather ----

struct GatherSmem {
    uint64_t bar[2];
};

template <int MR>
__global__ void __launch_bounds__(GATHER_THREADS, 1)
gather_f32(DevPlan P, const float2 *__restrict__ grids, const float2 *__restrict__ fhat, float2 *__restrict__ f,
           int n_tiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const long long gb = P.max_grid_bytes;
    float2 *const buf0 = (float2 *)smem_raw;
    float2 *const buf1 = (float2 *)(smem_raw + gb);
    uint64_t *bars = (uint64_t *)(smem_raw + 2 * gb);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int sub = lane & 15;
    const int r = sub >> 3, k = sub & 7;
    const int hw = (tid >> 5) * 2 + (lane >> 4);
    const long long M = P.M;
    const int nt = P.n_terms;
    const float *__restrict__ X = P.x;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
    }
    __syncthreads();

    // constant of the empty-set terms
    float2 c0 = make_float2(0.f, 0.f);
    for (int e = 0; e < P.n_empty; ++e) {
        float2 c = fhat[P.empty_off[e]];
        c0.x += c.x;
        c0.y += c.y;
    }

    const int my_tiles = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const long long total_it = (long long)my_tiles * nt;
    if (total_it > 0 && tid == 0) {
        const Term &T0 = P.terms[0];
        mbar_expect_tx(&bars[0], (uint32_t)T0.grid_bytes);
        bulk_g2s(buf0, grids + T0.grid_off, (uint32_t)T0.grid_bytes, &bars[0]);
    }

    long long it = 0;
    for (int ti = 0; ti < my_tiles; ++ti) {
        const long long tile = (long long)blockIdx.x + (long long)ti * gridDim.x;
        const long long p0 = tile * GATHER_TILE + (long long)hw * PTS_PER_HALF;
        float ax[PTS_PER_HALF], ay[PTS_PER_HALF];
        float rw[PTS_PER_HALF][MR];
        int rbase[PTS_PER_HALF];
        float cc[NCOEF];
#pragma unroll
        for (int i = 0; i < PTS_PER_HALF; ++i) {
            ax[i] = 0.f;
            ay[i] = 0.f;
            rbase[i] = 0;
#pragma unroll
            for (int j = 0; j < MR; ++j) rw[i][j] = 0.f;
        }
        int cur_wc = -1;
        for (int s = 0; s < nt; ++s, ++it) {
            const int b = (int)(it & 1);
            const uint32_t parity = (uint32_t)((it >> 1) & 1);
            if (tid == 0 && it + 1 < total_it) {
                const Term &Tn = P.terms[(s + 1) % nt];
                fence_proxy_async();
                mbar_expect_tx(&bars[b ^ 1], (uint32_t)Tn.grid_bytes);
                bulk_g2s(b ? buf0 : buf1, grids + Tn.grid_off, (uint32_t)Tn.grid_bytes, &bars[b ^ 1]);
            }
            const Term &T = P.terms[s];
            const int order = T.order, n = T.n, stride = T.stride, col = T.col;
            if (T.wc != cur_wc) {
                const float *wsrc = P.windows[T.wc].c[k];
#pragma unroll
                for (int i = 0; i < NCOEF; ++i) cc[i] = __ldg(wsrc + i);
                cur_wc = T.wc;
            }
            if (order == 2 && T.new_rowgroup) {
                float rc[MR][NCOEF];
#pragma unroll
                for (int j = 0; j < MR; ++j)
#pragma unroll
                    for (int i = 0; i < NCOEF; ++i) rc[j][i] = __ldg(&P.windows[T.wr].c[r + 2 * j][i]);
                const float *xr = X + (long long)T.row0 * M;
#pragma unroll
                for (int i = 0; i < PTS_PER_HALF; ++i) {
                    long long p = p0 + i;
                    float xa = p < M ? __ldg(xr + p) : 0.f;
                    float tau;
                    int fl = grid_pos(xa, n, tau);
                    float v = 2.f * tau - 1.f;
#pragma unroll
                    for (int j = 0; j < MR; ++j) rw[i][j] = horner8(rc[j], v);
                    rbase[i] = (fl + r) * stride;   // stored row of tap r: fl + r (halo hr = MR - 1)
                }
            }
            mbar_wait(&bars[b], parity, P.err, 1);
            const float2 *G = b ? buf1 : buf0;
            const float *xc = X + (long long)col * M;
            if (order == 2) {
#pragma unroll
                for (int i = 0; i < PTS_PER_HALF; ++i) {
                    long long p = p0 + i;
                    float xb = p < M ? __ldg(xc + p) : 0.f;
                    float tau;
                    int fl = grid_pos(xb, n, tau);
                    float cw = horner8(cc, 2.f * tau - 1.f);
                    const float2 *g = G + rbase[i] + fl + k;
                    float sx = 0.f, sy = 0.f;
#pragma unroll
                    for (int j = 0; j < MR; ++j) {
                        float2 v = g[2 * j * stride];
                        sx = fmaf(rw[i][j], v.x, sx);
                        sy = fmaf(rw[i][j], v.y, sy);
                    }
                    ax[i] = fmaf(cw, sx, ax[i]);
                    ay[i] = fmaf(cw, sy, ay[i]);
                }
            } else if (order == 1) {
                if (r == 0) {
#pragma unroll
                    for (int i = 0; i < PTS_PER_HALF; ++i) {
                        long long p = p0 + i;
                        float xb = p < M ? __ldg(xc + p) : 0.f;
                        float tau;
                        int fl = grid_pos(xb, n, tau);
                        float cw = horner8(cc, 2.f * tau - 1.f);
                        float2 v = G[fl + k];
                        ax[i] = fmaf(cw, v.x, ax[i]);
                        ay[i] = fmaf(cw, v.y, ay[i]);
                    }
                }
            } else {
                // order 3: rows (first, second) wrap modulo n; weights evaluated directly
                const Window &W = P.windows[T.wr];
                const int mr = T.mr, mc = T.mc;
                const float *xa_p = X + (long long)T.row0 * M;
                const float *xb_p = X + (long long)T.row1 * M;
#pragma unroll
                for (int i = 0; i < PTS_PER_HALF; ++i) {
                    long long p = p0 + i;
                    if (p >= M) continue;
                    float ta, tb, tc;
                    int fa = grid_pos(__ldg(xa_p + p), n, ta);
                    int fb = grid_pos(__ldg(xb_p + p), n, tb);
                    int fc = grid_pos(__ldg(xc + p), n, tc);
                    float cw = horner8(cc, 2.f * tc - 1.f);
                    int cidx = wrap(fc - mc + 1 + k, n);
                    float sx = 0.f, sy = 0.f;
                    for (int ia = 0; ia < 2 * mr; ++ia) {
                        float wa = kb_direct(ta + (float)(mr - 1 - ia), mr, W.b, W.inv_psi0);
                        int ra = wrap(fa - mr + 1 + ia, n);
                        for (int jb = r; jb < 2 * mr; jb += 2) {
                            float wb = kb_direct(tb + (float)(mr - 1 - jb), mr, W.b, W.inv_psi0);
                            int rb = wrap(fb - mr + 1 + jb, n);
                            float2 v = G[(ra * n + rb) * stride + cidx];
                            float w = wa * wb;
                            sx = fmaf(w, v.x, sx);
                            sy = fmaf(w, v.y, sy);
                        }
                    }
                    ax[i] = fmaf(cw, sx, ax[i]);
                    ay[i] = fmaf(cw, sy, ay[i]);
                }
            }
            __syncthreads();
        }
        // transposed reduce-scatter over the 16 lanes of the half-warp: after
        // the four steps, lane `sub` holds the full sum of node p0 + sub.
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) {
            const bool up = (sub & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                float sx = up ? ax[i] : ax[i + o];
                float sy = up ? ay[i] : ay[i + o];
                float kx = up ? ax[i + o] : ax[i];
                float ky = up ? ay[i + o] : ay[i];
                sx = __shfl_xor_sync(0xffffffffu, sx, o);
                sy = __shfl_xor_sync(0xffffffffu, sy, o);
                ax[i] = kx + sx;
                ay[i] = ky + sy;
            }
        }
        const long long p = p0 + sub;
        if (p < M) f[p] = make_float2(ax[0] + c0.x, ay[0] + c0.y);
    }
}

// ------------------------------------------------------- empty plan case --

__global__ void fill_const_f32(float2 *f, long long M, const float2 *__restrict__ fhat, const long long *eoff,
                               int n_empty) {
    float2 c0 = make_float2(0.f, 0.f);
    for (int e = 0; e < n_empty; ++e) {
        float2 c = fhat[eoff[e]];
        c0.x += c.x;
        c0.y += c.y;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
        f[i] = c0;
}

int launch_trafo_f32(Plan &p, const float2 *fhat, float2 *f) {
    DevPlan v = dev_view(p);
    if (p.n_terms == 0) {
        int blocks = (int)std::min<long long>(1024, (p.M + 255) / 256);
        fill_const_f32<<<blocks, 256, 0, p.stream>>>(f, p.M, fhat, p.empty_off, p.n_empty);
        return cuda_status(cudaGetLastError());
    }
    size_t pre_smem = (size_t)p.max_fft_elems * 2 * sizeof(float2);
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(trafo_pre_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(gather_f32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(gather_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(gather_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        attr_done = true;
    }
    stage_begin(p, ST_PRE);
    trafo_pre_f32<<<p.n_terms, 256, pre_smem, p.stream>>>(v, fhat, (float2 *)p.grids);
    stage_end(p, ST_PRE);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    int n_tiles = (int)((p.M + GATHER_TILE - 1) / GATHER_TILE);
    size_t gsm = (size_t)p.max_grid_bytes * 2 + 64;
    int mr = p.h_terms[0].mr;
    for (int s = 0; s < p.n_terms; ++s) mr = p.h_terms[s].mr > 0 ? p.h_terms[s].mr : mr;
    stage_begin(p, ST_GATHER);
    if (mr <= 2)
        gather_f32<2><<<p.gather_ctas, GATHER_THREADS, gsm, p.stream>>>(v, (const float2 *)p.grids, fhat, f, n_tiles);
    else if (mr == 3)
        gather_f32<3><<<p.gather_ctas, GATHER_THREADS, gsm, p.stream>>>(v, (const float2 *)p.grids, fhat, f, n_tiles);
    else
        gather_f32<4><<<p.gather_ctas, GATHER_THREADS, gsm, p.stream>>>(v, (const float2 *)p.grids, fhat, f, n_tiles);
    stage_end(p, ST_GATHER);
    return cuda_status(cudaGetLastError());
}

}  // namespace agft
