// Adjoint grouped transform fhat = F^H y (stacked adjoint after the error
// remark, Sec. 3), FP32.
//
//   1. spread: term-outer.  CTA c owns a contiguous range of nodes; for every
//      term it accumulates y_j times the window into a shared-memory copy of
//      the term's stored grid (halos included) with shared-memory atomics,
//      half-warp per node (2 rows x 8 columns of the window per instruction),
//      then writes its partial grid to partials[c].
//   2. reduce_partials: grid = sum_c partials[c] in a fixed order
//      (deterministic across runs for a fixed CTA count).
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

template <int MR>
__global__ void __launch_bounds__(SPREAD_THREADS)
spread_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ y_base, int n_items) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *S = (float2 *)smem_raw;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int sub = lane & 15;
    const int r = sub >> 3, k = sub & 7;
    const int hw = (tid >> 5) * 2 + (lane >> 4);
    const int nhw = SPREAD_THREADS / 16;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int pb = B.plans ? B.item_prob[item] : 0;
    const DevPlan &P = B.plans ? B.plans[pb] : single;
    const int kc = B.plans ? item - B.item0[pb] : item;   // node chunk of this problem
    if (P.skip && *P.skip) continue;
    const long long M = P.M;
    const long long j0 = M * (long long)kc / P.spread_chunks;
    const long long j1 = M * (long long)(kc + 1) / P.spread_chunks;
    const float *__restrict__ X = P.x;
    const float2 *__restrict__ y = y_base + P.vec_node_off;
    float2 *mypart = P.partials + (long long)kc * P.grid_elems;
    for (int s = 0; s < P.n_act; ++s) {
        const Term &T = P.terms[P.act[s]];
        const int order = T.order, n = T.n, stride = T.stride;
        const long long elems = T.grid_bytes / 8;
        float4 *S4 = (float4 *)S;
        for (long long e = tid; e < elems / 2; e += blockDim.x) S4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        float cc[NCOEF];
        const float *wsrc = P.windows[T.wc].c[k];
#pragma unroll
        for (int i = 0; i < NCOEF; ++i) cc[i] = __ldg(wsrc + i);
        __syncthreads();
        const float *xc = X + (long long)T.col * M;
        if (order == 2) {
            float rc[MR][NCOEF];
#pragma unroll
            for (int j = 0; j < MR; ++j)
#pragma unroll
                for (int i = 0; i < NCOEF; ++i) rc[j][i] = __ldg(&P.windows[T.wr].c[r + 2 * j][i]);
            const float *xr = X + (long long)T.row0 * M;
            for (long long p = j0 + hw; p < j1; p += nhw) {
                float2 yv = __ldg(y + p);
                float ta, tb;
                int fa = grid_pos(__ldg(xr + p), n, ta);
                int fb = grid_pos(__ldg(xc + p), n, tb);
                float cw = horner8(cc, 2.f * tb - 1.f);
                float va = 2.f * ta - 1.f;
                float yx = yv.x * cw, yy = yv.y * cw;
                float *base = (float *)(S + (fa + r) * stride + fb + k);
#pragma unroll
                for (int j = 0; j < MR; ++j) {
                    float w = horner8(rc[j], va);
                    red_add(base + 4 * j * stride, yx * w);
                    red_add(base + 4 * j * stride + 1, yy * w);
                }
            }
        } else if (order == 1) {
            if (r == 0) {
                for (long long p = j0 + hw; p < j1; p += nhw) {
                    float2 yv = __ldg(y + p);
                    float tb;
                    int fb = grid_pos(__ldg(xc + p), n, tb);
                    float cw = horner8(cc, 2.f * tb - 1.f);
                    float *base = (float *)(S + fb + k);
                    red_add(base, yv.x * cw);
                    red_add(base + 1, yv.y * cw);
                }
            }
        } else {
            const Window &W = P.windows[T.wr];
            const int mr = T.mr, mc = T.mc;
            const float *xa_p = X + (long long)T.row0 * M;
            const float *xb_p = X + (long long)T.row1 * M;
            for (long long p = j0 + hw; p < j1; p += nhw) {
                float2 yv = __ldg(y + p);
                float ta, tb, tc;
                int fa = grid_pos(__ldg(xa_p + p), n, ta);
                int fb = grid_pos(__ldg(xb_p + p), n, tb);
                int fc = grid_pos(__ldg(xc + p), n, tc);
                float cw = horner8(cc, 2.f * tc - 1.f);
                int cidx = wrap(fc - mc + 1 + k, n);
                float yx = yv.x * cw, yy = yv.y * cw;
                for (int ia = 0; ia < 2 * mr; ++ia) {
                    float wa = kb_direct(ta + (float)(mr - 1 - ia), mr, W.b, W.inv_psi0);
                    int ra = wrap(fa - mr + 1 + ia, n);
                    for (int jb = r; jb < 2 * mr; jb += 2) {
                        float wb = kb_direct(tb + (float)(mr - 1 - jb), mr, W.b, W.inv_psi0);
                        int rb = wrap(fb - mr + 1 + jb, n);
                        float *c = (float *)(S + (ra * n + rb) * stride + cidx);
                        float w = wa * wb;
                        red_add(c, yx * w);
                        red_add(c + 1, yy * w);
                    }
                }
            }
        }
        __syncthreads();
        float4 *dst = (float4 *)(mypart + T.grid_off);
        for (long long e = tid; e < elems / 2; e += blockDim.x) dst[e] = S4[e];
        __syncthreads();
    }
  }
}

__global__ void reduce_partials_f32(DevPlan single, BatchArgs B) {
    const DevPlan &P = B.plans ? B.plans[blockIdx.y] : single;
    if (P.skip && *P.skip) return;
    const float4 *__restrict__ partials = (const float4 *)P.partials;
    float4 *__restrict__ out = (float4 *)P.grids;
    const long long n4 = P.grid_elems / 2, pstride4 = n4;
    const int nparts = P.spread_chunks;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
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
}

__global__ void adjoint_post_f32(DevPlan single, BatchArgs B, float2 *__restrict__ fhat_base) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int pb = B.plans ? B.blk_prob[blockIdx.x] : 0;
    const DevPlan &P = B.plans ? B.plans[pb] : single;
    const int sblk = B.plans ? (int)blockIdx.x - B.blk0[pb] : (int)blockIdx.x;
    if (P.skip && *P.skip) return;
    const float2 *__restrict__ grids = P.grids;
    float2 *__restrict__ fhat = fhat_base + P.vec_coef_off;
    const Term T = P.terms[P.act[sblk]];
    const int n = T.n, s = T.order, N = T.N;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    float2 *a = (float2 *)smem_raw;
    float2 *b = a + fe;
    const float2 *g = grids + T.grid_off;
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
                    float2 u = g[(long long)er * T.stride + ec];
                    v.x += u.x;
                    v.y += u.y;
                }
            }
        } else {
            int row = e / n, c = e % n;
            v = g[(long long)row * T.stride + c];
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
    for (long long q = threadIdx.x; q < T.coef_len; q += blockDim.x) {
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

static void adjoint_attrs() {
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(adjoint_post_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(spread_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(spread_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        attr_done = true;
    }
}

// The adjoint kernels for one problem (B.plans == null) or a batch of P problems.
int adjoint_launch(Plan *prof, cudaStream_t st, const DevPlan &v, const BatchArgs &B, int P, const float2 *y,
                   float2 *fhat, int n_items, int ctas, int n_blocks, int mr, long long max_grid_bytes,
                   int max_fft_elems, int sm_count, long long max_grid_elems, bool any_empty, double2 *scratch) {
    adjoint_attrs();
    if (any_empty) {
        const int nb = 256;
        if (prof) stage_begin(*prof, ST_SUMY);
        sum_y_stage1<<<dim3(nb, P), 256, 0, st>>>(v, B, y, scratch);
        sum_y_stage2<<<P, 32, 0, st>>>(v, B, scratch, nb, fhat);
        if (prof) stage_end(*prof, ST_SUMY);
    }
    if (n_blocks == 0) return cuda_status(cudaGetLastError());
    const size_t ssm = (size_t)max_grid_bytes;
    if (prof) stage_begin(*prof, ST_SPREAD);
    if (mr <= 3)
        spread_f32<3><<<ctas, SPREAD_THREADS, ssm, st>>>(v, B, y, n_items);
    else
        spread_f32<4><<<ctas, SPREAD_THREADS, ssm, st>>>(v, B, y, n_items);
    if (prof) stage_end(*prof, ST_SPREAD);
    const long long n4 = max_grid_elems / 2;
    const int rb = (int)std::max<long long>(1, std::min<long long>(sm_count * 8LL / std::max(1, P) + 1, (n4 + 255) / 256));
    if (prof) stage_begin(*prof, ST_REDUCE);
    reduce_partials_f32<<<dim3(rb, P), 256, 0, st>>>(v, B);
    if (prof) stage_end(*prof, ST_REDUCE);
    const size_t post_smem = (size_t)max_fft_elems * 2 * sizeof(float2);
    if (prof) stage_begin(*prof, ST_POST);
    adjoint_post_f32<<<n_blocks, 256, post_smem, st>>>(v, B, fhat);
    if (prof) stage_end(*prof, ST_POST);
    return cuda_status(cudaGetLastError());
}

int launch_adjoint_f32(Plan &p, const float2 *y, float2 *fhat) {
    DevPlan v = dev_view(p);
    BatchArgs B;
    std::memset(&B, 0, sizeof(B));
    if (p.M == 0) {
        cudaMemsetAsync(fhat, 0, sizeof(float2) * p.n_coeffs, p.stream);
        return cuda_status(cudaGetLastError());
    }
    int mr = 3;
    for (int s = 0; s < p.n_terms; ++s) mr = p.h_terms[s].mr > 0 ? p.h_terms[s].mr : mr;
    return adjoint_launch(&p, p.stream, v, B, 1, y, fhat, p.spread_ctas, p.spread_ctas, p.n_act, mr,
                          p.max_grid_bytes, p.max_fft_elems, p.sm_count, p.grid_elems, p.n_empty > 0,
                          (double2 *)p.scratch);
}

}  // namespace agft
