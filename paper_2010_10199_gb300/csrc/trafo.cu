// Forward grouped transform f = F fhat (Definition "grouped Fourier transform"
// and eq. (somafm), Sec. 3), FP32.
//
//   1. trafo_pre: per term, zero-extend the block fhat(u) to ghat(u) on the
//      n^{|u|} grid (the extension before eq. (somafm)), multiply by the
//      deconvolution factors, run the oversampled FFT (sign +) in shared
//      memory and store the grid with its halos.
//   2. gather: all terms fused, point-major.  A CTA owns a tile of 128 nodes;
//      each half-warp owns 8 nodes and evaluates them one at a time with its
//      16 lanes = 2 rows x 8 columns of the window, reading the term's grid from
//      shared memory (double-buffered bulk async copies from L2).  Lanes keep
//      per-node partial sums over all terms in registers; one transposed
//      reduce-scatter per tile leaves node i's value in lane i.
#include <cstdio>
#include <cstring>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

__device__ __forceinline__ int freq_index(int q, int N) { return q < N / 2 ? q - N / 2 : q - N / 2 + 1; }

// ------------------------------------------------------------ pre-pass ----

// grids stored as G (FP32 complex, or a pair of 16-bit floats rounded from the FP32 FFT)
template <typename G>
__device__ __forceinline__ void trafo_pre_body(const DevPlan &single, const BatchArgs &B,
                                               const float2 *__restrict__ fhat_base) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int pb = B.plans ? B.blk_prob[blockIdx.x] : 0;
    const DevPlan &P = B.plans ? B.plans[pb] : single;
    const int sblk = B.plans ? (int)blockIdx.x - B.blk0[pb] : (int)blockIdx.x;
    if (P.skip && *P.skip) return;
    const float2 *fhat = fhat_base + P.vec_coef_off;
    G *grids = (G *)P.grids;
    const Term T = P.terms[P.act[sblk]];
    const int n = T.n, s = T.order, N = T.N;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    float2 *a = (float2 *)smem_raw;
    float2 *b = a + fe;
    for (int i = threadIdx.x; i < fe; i += blockDim.x) a[i] = make_float2(0.f, 0.f);
    __syncthreads();
    // zero-extended, deconvolved coefficients at k mod n
    const int Nm = N - 1;
    for (long long q = threadIdx.x; q < T.coef_len && T.basis == ANOVA_BASIS_COS; q += blockDim.x) {
        // cosine term: the coefficient at its 2^s mirrored frequencies
        int k[3];
        cos_decode(q, s, N, k);
        const float2 c = fhat[T.coef_off + q];
        for (int sg = 0; sg < (1 << s); ++sg) {
            float D = (float)cos_amp(s);
            const int pos = cos_mirror(k, s, sg, N, n, P.deconv, T.dc_off, T.dr_off, D);
            a[pos] = make_float2(c.x * D, c.y * D);
        }
    }
    for (long long q = threadIdx.x; q < T.coef_len && T.basis != ANOVA_BASIS_COS; q += blockDim.x) {
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
    G *g = grids + T.grid_off;
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
        g[e] = GridEl<G>::store(v.x, v.y);
    }
}

__global__ void trafo_pre_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base) {
    trafo_pre_body<float2>(single, B, fhat_base);
}
__global__ void trafo_pre_f16(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base) {
    trafo_pre_body<__half2>(single, B, fhat_base);
}
__global__ void trafo_pre_bf16(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base) {
    trafo_pre_body<__nv_bfloat162>(single, B, fhat_base);
}

// ------------------------------------------------------- empty plan case --

__global__ void fill_const_f32(float2 *f, long long M, const float2 *__restrict__ fhat, const long long *eoff,
                               int n_empty, const int *skip) {
    if (skip && *skip) return;
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
    if (p.n_act == 0) {
        int blocks = (int)std::min<long long>(1024, (p.M + 255) / 256);
        fill_const_f32<<<blocks, 256, 0, p.stream>>>(f, p.M, fhat, p.empty_off, p.n_empty, p.skip);
        return cuda_status(cudaGetLastError());
    }
    size_t pre_smem = (size_t)p.max_fft_elems * 2 * sizeof(float2);
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(trafo_pre_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(trafo_pre_f16, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(trafo_pre_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    stage_begin(p, ST_PRE);
    BatchArgs B;
    std::memset(&B, 0, sizeof(B));
    auto pre = p.precision == ANOVA_PREC_F16 ? trafo_pre_f16 : p.precision == ANOVA_PREC_BF16 ? trafo_pre_bf16 : trafo_pre_f32;
    pre<<<p.n_act, 256, pre_smem, p.stream>>>(v, B, fhat);
    stage_end(p, ST_PRE);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    stage_begin(p, ST_GATHER);
    int rc;
    if (p.srec && p.facc && p.precision == ANOVA_PREC_F32 && p.n_act3 == 0)
        rc = launch_gather_sorted_f32(p, fhat, f);   // every term over its cell-sorted records
    else
        rc = launch_gather_f32(p, fhat, f);
    stage_end(p, ST_GATHER);
    return rc;
}

}  // namespace agft
