// The grouped transform in FP64 (plans created with ANOVA_PREC_F64): the
// same method as the FP32 path -- deconvolve and zero-extend, oversampled FFT,
// Kaiser--Bessel window gather (forward), window spread, FFT and crop
// (adjoint), Sec. 3 -- with every value and every sum in FP64.  It is the plain
// reference form of the method on the GPU: the window is evaluated directly
// (sinh and sqrt in FP64) once per plan into per-node tables, the way NFFT
// libraries precompute psi, and the kernels are straightforward: one thread
// per node for the gather; for the spread, nodes in cell order (the plan's
// sorted records) summed per cell in registers, FP64 shared-memory atomics
// once per cell.
//
// Window tables: one slot per (window, coordinate) pair that some term uses;
// for node j, slot q holds the weights psi(tau + m - 1 - t) / psi(0) of taps
// t = 0..2m-1 (zero padded to 8) and the first tap's index floor(n x_j + n/2)
// in [0, n).  Orders 1 and 2 keep halos on their grids, so tap t of a node
// sits at stored column (row) base + t; order 3 wraps modulo n.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

__device__ __forceinline__ int freq_index64(int q, int N) { return q < N / 2 ? q - N / 2 : q - N / 2 + 1; }

// ------------------------------------------------------ window tables ----

__global__ void k_wtab_f64(const double *__restrict__ x, long long M, const int4 *slots, const Window *wins,
                           double *wt, int *wb) {
    const int4 sl = slots[blockIdx.y];   // (window, coordinate, n, m)
    const Window &W = wins[sl.x];
    const int n = sl.z, m = sl.w;
    const double b = W.bd, ip0 = W.inv_psi0d;
    const double *xc = x + (long long)sl.y * M;
    double2 *dst = (double2 *)(wt + (long long)blockIdx.y * M * 8);
    int *bdst = wb + (long long)blockIdx.y * M;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M; j += (long long)gridDim.x * blockDim.x) {
        double tau;
        bdst[j] = grid_pos_d(xc[j], n, tau);
        double w[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) w[t] = t < 2 * m ? kb_direct_d(tau + (double)(m - 1 - t), m, b, ip0) : 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t) dst[j * 4 + t] = make_double2(w[2 * t], w[2 * t + 1]);
    }
}

int build_window_tables_f64(Plan &p) {
    if (p.n_slots64 == 0 || p.M == 0) return ANOVA_OK;
    const int bx = (int)std::max<long long>(1, std::min<long long>(256, (p.M + 255) / 256));
    k_wtab_f64<<<dim3(bx, p.n_slots64), 256, 0, p.stream>>>((const double *)p.x, p.M, p.slots64, p.windows, p.wt64,
                                                           p.wb64);
    return cuda_status(cudaGetLastError());
}

__device__ __forceinline__ void load_w8(const double *wt, int slot, long long M, long long j, double w[8], int &base,
                                        const int *wb) {
    const double2 *src = (const double2 *)(wt + ((long long)slot * M + j) * 8);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const double2 v = __ldg(src + t);
        w[2 * t] = v.x;
        w[2 * t + 1] = v.y;
    }
    base = __ldg(wb + (long long)slot * M + j);
}

// ------------------------------------------------------------ forward ----

// per active term: zero-extended, deconvolved block, FFT (sign +), grid with halos
__global__ void trafo_pre_f64(DevPlan P, const double2 *__restrict__ fhat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (P.skip && *P.skip) return;
    const Term T = P.terms[P.act[blockIdx.x]];
    const int n = T.n, s = T.order, N = T.N;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    double2 *a = (double2 *)smem_raw;
    double2 *b = a + fe;
    for (int i = threadIdx.x; i < fe; i += blockDim.x) a[i] = make_double2(0.0, 0.0);
    __syncthreads();
    const int Nm = N - 1;
    for (long long q = threadIdx.x; q < T.coef_len && T.basis == ANOVA_BASIS_COS; q += blockDim.x) {
        int k[3];
        cos_decode(q, s, N, k);
        const double2 c = fhat[T.coef_off + q];
        for (int sg = 0; sg < (1 << s); ++sg) {
            double D = cos_amp(s);
            const int pos = cos_mirror(k, s, sg, N, n, P.deconvd, T.dc_off, T.dr_off, D);
            a[pos] = make_double2(c.x * D, c.y * D);
        }
    }
    for (long long q = threadIdx.x; q < T.coef_len && T.basis != ANOVA_BASIS_COS; q += blockDim.x) {
        long long r = q;
        int pos = 0, mul = 1;
        double D = 1.0;
        for (int t = s - 1; t >= 0; --t) {
            const int it = (int)(r % Nm);
            r /= Nm;
            const int k = freq_index64(it, N);
            pos += (k < 0 ? k + n : k) * mul;
            mul *= n;
            D *= (t == s - 1) ? P.deconvd[T.dc_off + it] : P.deconvd[T.dr_off + it];
        }
        const double2 c = fhat[T.coef_off + q];
        a[pos] = make_double2(c.x * D, c.y * D);
    }
    __syncthreads();
    const double2 *cur = grid_fft<double2, double>(a, b, n, s, +1);
    double2 *g = (double2 *)P.grids + T.grid_off;
    const int ecols = T.stride;
    const long long total = (long long)T.erows * ecols;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const int er = (int)(e / ecols), ec = (int)(e % ecols);
        double2 v = make_double2(0.0, 0.0);
        if (s <= 2) {
            if (ec < n + 2 * T.hc + 1) {
                const int qc = wrap(ec - T.hc, n);
                const int qr = s == 2 ? wrap(er - T.hr, n) : 0;
                v = cur[qr * n + qc];
            }
        } else if (ec < n) {
            v = cur[er * n + ec];
        }
        g[e] = v;
    }
}

// one thread per node, all active terms
__global__ void __launch_bounds__(256) gather_f64(DevPlan P, const double2 *__restrict__ fhat, double2 *f,
                                                  const double *wt, const int *wb) {
    if (P.skip && *P.skip) return;
    const long long M = P.M;
    const long long j = blockIdx.x * 256LL + threadIdx.x;
    if (j >= M) return;
    double ax = 0.0, ay = 0.0;
    for (int e = 0; e < P.n_empty; ++e) {
        const double2 c = fhat[P.empty_off[e]];
        ax += c.x;
        ay += c.y;
    }
    const double2 *G = (const double2 *)P.grids;
    for (int s = 0; s < P.n_act; ++s) {
        const Term &T = P.terms[P.act[s]];
        const double2 *g = G + T.grid_off;
        const int stride = T.stride, n = T.n, mc = T.mc, mr = T.mr;
        double wc[8];
        int fc;
        load_w8(wt, T.slot_c, M, j, wc, fc, wb);
        if (T.order == 1) {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t < 2 * mc) {
                    const double2 v = __ldg(g + fc + t);
                    ax = fma(wc[t], v.x, ax);
                    ay = fma(wc[t], v.y, ay);
                }
        } else if (T.order == 2) {
            double wr[8];
            int fr;
            load_w8(wt, T.slot_r0, M, j, wr, fr, wb);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i >= 2 * mr) break;
                const double2 *row = g + (long long)(fr + i) * stride + fc;
                double sx = 0.0, sy = 0.0;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (t < 2 * mc) {
                        const double2 v = __ldg(row + t);
                        sx = fma(wc[t], v.x, sx);
                        sy = fma(wc[t], v.y, sy);
                    }
                ax = fma(wr[i], sx, ax);
                ay = fma(wr[i], sy, ay);
            }
        } else {
            double wa[8], wb2[8];
            int fa, fb;
            load_w8(wt, T.slot_r0, M, j, wa, fa, wb);
            load_w8(wt, T.slot_r1, M, j, wb2, fb, wb);
            for (int ia = 0; ia < 2 * mr; ++ia) {
                const int ra = wrap(fa - mr + 1 + ia, n);
                for (int ib = 0; ib < 2 * mr; ++ib) {
                    const int rb = wrap(fb - mr + 1 + ib, n);
                    const double2 *row = g + (long long)(ra * n + rb) * stride;
                    double sx = 0.0, sy = 0.0;
                    for (int t = 0; t < 2 * mc; ++t) {
                        const double2 v = __ldg(row + wrap(fc - mc + 1 + t, n));
                        sx = fma(wc[t], v.x, sx);
                        sy = fma(wc[t], v.y, sy);
                    }
                    const double w = wa[ia] * wb2[ib];
                    ax = fma(w, sx, ax);
                    ay = fma(w, sy, ay);
                }
            }
        }
    }
    f[j] = make_double2(ax, ay);
}

__global__ void fill_const_f64(double2 *f, long long M, const double2 *__restrict__ fhat, const long long *eoff,
                               int n_empty, const int *skip) {
    if (skip && *skip) return;
    double2 c0 = make_double2(0.0, 0.0);
    for (int e = 0; e < n_empty; ++e) {
        const double2 c = fhat[eoff[e]];
        c0.x += c.x;
        c0.y += c.y;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
        f[i] = c0;
}

int launch_trafo_f64(Plan &p, const double2 *fhat, double2 *f) {
    if (p.M == 0) return ANOVA_OK;
    DevPlan v = dev_view(p);
    if (p.n_act == 0) {
        const int blocks = (int)std::min<long long>(1024, (p.M + 255) / 256);
        fill_const_f64<<<blocks, 256, 0, p.stream>>>(f, p.M, fhat, p.empty_off, p.n_empty, p.skip);
        return cuda_status(cudaGetLastError());
    }
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(trafo_pre_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
    const size_t pre_smem = (size_t)p.max_fft_elems * 2 * sizeof(double2);
    stage_begin(p, ST_PRE);
    trafo_pre_f64<<<p.n_act, 256, pre_smem, p.stream>>>(v, fhat);
    stage_end(p, ST_PRE);
    stage_begin(p, ST_GATHER);
    gather_f64<<<(int)((p.M + 255) / 256), 256, 0, p.stream>>>(v, fhat, f, p.wt64, p.wb64);
    stage_end(p, ST_GATHER);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------ adjoint ----

// Sorted item (order <= 2, plan with cell-sorted records): the item's nodes in
// the term's cell order, cut into 16 contiguous runs, one per half-warp.  Lane
// (r, k) keeps the sums of column tap k and rows r, r+2, .. of the current
// cell in registers and adds them to the shared grid when the cell changes
// (FP64 atomics, once per cell instead of once per node).  Four nodes are
// loaded ahead of their use.  Order 1: the lane groups r = 0, 1 take
// alternate nodes.
__device__ __forceinline__ void spread_sorted_item_f64(const DevPlan &P, const Term &T, const double2 *__restrict__ y,
                                                       long long j0, long long j1, double2 *S, const double *wt) {
    const int tid = threadIdx.x;
    const int sub = tid & 15, hw = tid >> 4;
    const int r = sub >> 3, k = sub & 7;
    const long long M = P.M;
    const int stride = T.stride, mc = T.mc, mr = T.mr;
    const float4 *rec = P.srec + (long long)T.sort_slot * M;
    const long long len = j1 - j0, L = (len + 15) / 16;
    const long long a = j0 + min((long long)hw * L, len), b = j0 + min((long long)(hw + 1) * L, len);
    const double *wcol = wt + (long long)T.slot_c * M * 8;
    const bool kc = k < 2 * mc;
    int cur = -1;
    if (T.order == 2) {
        const double *wrow = wt + (long long)T.slot_r0 * M * 8;
        double ax[4] = {0.0, 0.0, 0.0, 0.0}, ay[4] = {0.0, 0.0, 0.0, 0.0};
        auto flush = [&]() {
            if (kc) {
                double2 *base = S + cur + r * stride + k;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (r + 2 * q < 2 * mr) {
                        atomicAdd(&base[2 * q * stride].x, ax[q]);
                        atomicAdd(&base[2 * q * stride].y, ay[q]);
                    }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) ax[q] = ay[q] = 0.0;
        };
        for (long long p0 = a; p0 < b; p0 += 4) {
            int off[4], jj[4];
            double wc[4], wr[4][4];
            double2 yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = p0 + u < b;
                const float4 q = __ldg(rec + (ok ? p0 + u : a));
                off[u] = ok ? __float_as_int(q.z) : -2;
                jj[u] = __float_as_int(q.w);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long j = jj[u];
                yv[u] = __ldg(y + j);
                wc[u] = kc ? __ldg(wcol + j * 8 + k) : 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) wr[u][q] = r + 2 * q < 2 * mr ? __ldg(wrow + j * 8 + r + 2 * q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (off[u] == -2) break;
                if (off[u] != cur) {
                    if (cur >= 0) flush();
                    cur = off[u];
                }
                const double yx = yv[u].x * wc[u], yy = yv[u].y * wc[u];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ax[q] = fma(yx, wr[u][q], ax[q]);
                    ay[q] = fma(yy, wr[u][q], ay[q]);
                }
            }
        }
        if (cur >= 0) flush();
    } else {
        double ax = 0.0, ay = 0.0;
        for (long long p = a + r; p < b; p += 2) {
            const float4 q = __ldg(rec + p);
            const int off = __float_as_int(q.z);
            const long long j = __float_as_int(q.w);
            if (off != cur) {
                if (cur >= 0 && kc) {
                    atomicAdd(&S[cur + k].x, ax);
                    atomicAdd(&S[cur + k].y, ay);
                }
                ax = ay = 0.0;
                cur = off;
            }
            const double w = kc ? __ldg(wcol + j * 8 + k) : 0.0;
            const double2 v = __ldg(y + j);
            ax = fma(v.x, w, ax);
            ay = fma(v.y, w, ay);
        }
        if (cur >= 0 && kc) {
            atomicAdd(&S[cur + k].x, ax);
            atomicAdd(&S[cur + k].y, ay);
        }
    }
}

// Work item (problem 0, active term, node chunk z, chunks K): the item's
// nodes add y_j times their window into a shared-memory copy of the term's
// stored grid, which then goes to partial grid z.  Terms with cell-sorted
// records take the sorted path above; the others (order 3, or no records)
// add every tap with FP64 atomics (half-warp per node, lane (r, k): column tap
// k, rows r, r+2, ..), nodes in their original order.
__global__ void __launch_bounds__(256) spread_f64(DevPlan P, const int4 *items, const double2 *__restrict__ y,
                                                  int n_items, int *counter, long long max_grid_bytes,
                                                  const double *wt, const int *wb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *S = (double2 *)smem_raw;
    int &s_item = *(int *)(smem_raw + max_grid_bytes);
    const int tid = threadIdx.x;
    const int sub = tid & 15, hw = tid >> 4;
    const int r = sub >> 3, k = sub & 7;
    const long long M = P.M;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        if (P.skip && *P.skip) continue;
        const int4 itm = items[item];
        const Term &T = P.terms[P.act[itm.y]];
        const long long j0 = M * itm.z / itm.w, j1 = M * (itm.z + 1) / itm.w;
        const long long elems = T.grid_bytes / 16;
        for (long long e = tid; e < elems; e += 256) S[e] = make_double2(0.0, 0.0);
        __syncthreads();
        const int stride = T.stride, n = T.n, mc = T.mc, mr = T.mr;
        if (T.sort_slot >= 0 && P.srec && T.order <= 2) {
            spread_sorted_item_f64(P, T, y, j0, j1, S, wt);
        } else {
            for (long long j = j0 + hw; j < j1; j += 16) {
                const double2 yv = __ldg(y + j);
                const double wck = k < 2 * mc ? __ldg(wt + ((long long)T.slot_c * M + j) * 8 + k) : 0.0;
                const int fc = __ldg(wb + (long long)T.slot_c * M + j);
                const double yx = yv.x * wck, yy = yv.y * wck;
                if (T.order == 1) {
                    if (r == 0 && k < 2 * mc) {
                        atomicAdd(&S[fc + k].x, yx);
                        atomicAdd(&S[fc + k].y, yy);
                    }
                } else if (T.order == 2) {
                    const long long ro = (long long)T.slot_r0 * M + j;
                    const int fr = __ldg(wb + ro);
                    if (k < 2 * mc)
                        for (int i = r; i < 2 * mr; i += 2) {
                            const double w = __ldg(wt + ro * 8 + i);
                            double2 *c = S + (fr + i) * stride + fc + k;
                            atomicAdd(&c->x, yx * w);
                            atomicAdd(&c->y, yy * w);
                        }
                } else if (k < 2 * mc) {
                    const long long ra0 = (long long)T.slot_r0 * M + j, rb0 = (long long)T.slot_r1 * M + j;
                    const int fa = __ldg(wb + ra0), fb = __ldg(wb + rb0);
                    const int col = wrap(fc - mc + 1 + k, n);
                    for (int ia = 0; ia < 2 * mr; ++ia) {
                        const double wa = __ldg(wt + ra0 * 8 + ia);
                        const int ra = wrap(fa - mr + 1 + ia, n);
                        for (int ib = r; ib < 2 * mr; ib += 2) {
                            const double w = wa * __ldg(wt + rb0 * 8 + ib);
                            const int rb = wrap(fb - mr + 1 + ib, n);
                            double2 *c = S + (ra * n + rb) * stride + col;
                            atomicAdd(&c->x, yx * w);
                            atomicAdd(&c->y, yy * w);
                        }
                    }
                }
            }
        }
        __syncthreads();
        double2 *dst = (double2 *)P.partials + (long long)itm.z * P.grid_elems + T.grid_off;
        for (long long e = tid; e < elems; e += 256) dst[e] = S[e];
        __syncthreads();
    }
}

__global__ void reduce_partials_f64(DevPlan P) {
    if (P.skip && *P.skip) return;
    const double2 *__restrict__ part = (const double2 *)P.partials;
    double2 *out = (double2 *)P.grids;
    const long long ne = P.grid_elems;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ne; i += (long long)gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int c = 0; c < P.spread_chunks; ++c) {
            const double2 v = part[(long long)c * ne + i];
            sx += v.x;
            sy += v.y;
        }
        out[i] = make_double2(sx, sy);
    }
}

// per active term: fold the halos, FFT (sign -), deconvolve and crop
__global__ void adjoint_post_f64(DevPlan P, double2 *__restrict__ fhat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (P.skip && *P.skip) return;
    const Term T = P.terms[P.act[blockIdx.x]];
    const int n = T.n, s = T.order, N = T.N;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    double2 *a = (double2 *)smem_raw;
    double2 *b = a + fe;
    const double2 *g = (const double2 *)P.grids + T.grid_off;
    for (int e = threadIdx.x; e < fe; e += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (s <= 2) {
            const int qc = e % n, qr = s == 2 ? e / n : 0;
            const int ecw = n + 2 * T.hc + 1;
            for (int dr = -1; dr <= 1; ++dr) {
                if (s == 1 && dr != 0) continue;
                const int er = s == 2 ? qr + T.hr + dr * n : 0;
                if (er < 0 || er >= T.erows) continue;
                for (int dc = -1; dc <= 1; ++dc) {
                    const int ec = qc + T.hc + dc * n;
                    if (ec < 0 || ec >= ecw) continue;
                    const double2 u = g[(long long)er * T.stride + ec];
                    v.x += u.x;
                    v.y += u.y;
                }
            }
        } else {
            v = g[(long long)(e / n) * T.stride + e % n];
        }
        a[e] = v;
    }
    __syncthreads();
    const double2 *cur = grid_fft<double2, double>(a, b, n, s, -1);
    const int Nm = N - 1;
    for (long long q = threadIdx.x; q < T.coef_len && T.basis == ANOVA_BASIS_COS; q += blockDim.x) {
        int k[3];
        cos_decode(q, s, N, k);
        double sx = 0.0, sy = 0.0;
        for (int sg = 0; sg < (1 << s); ++sg) {
            double D = cos_amp(s);
            const double2 v = cur[cos_mirror(k, s, sg, N, n, P.deconvd, T.dc_off, T.dr_off, D)];
            sx = fma(v.x, D, sx);
            sy = fma(v.y, D, sy);
        }
        fhat[T.coef_off + q] = make_double2(sx, sy);
    }
    for (long long q = threadIdx.x; q < T.coef_len && T.basis != ANOVA_BASIS_COS; q += blockDim.x) {
        long long rr = q;
        int pos = 0, mul = 1;
        double D = 1.0;
        for (int t = s - 1; t >= 0; --t) {
            const int it = (int)(rr % Nm);
            rr /= Nm;
            const int kk = freq_index64(it, N);
            pos += (kk < 0 ? kk + n : kk) * mul;
            mul *= n;
            D *= (t == s - 1) ? P.deconvd[T.dc_off + it] : P.deconvd[T.dr_off + it];
        }
        const double2 v = cur[pos];
        fhat[T.coef_off + q] = make_double2(v.x * D, v.y * D);
    }
}

// sum of y for the empty-set coefficients: partial sums, then one thread
__global__ void sum_y_f64_stage1(DevPlan P, const double2 *__restrict__ y, double2 *part) {
    __shared__ double2 red[256];
    if (P.skip && *P.skip) return;
    double sx = 0.0, sy = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P.M; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = y[i];
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

__global__ void sum_y_f64_stage2(DevPlan P, const double2 *part, int nparts, double2 *fhat) {
    if (threadIdx.x != 0 || (P.skip && *P.skip)) return;
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < nparts; ++i) {
        sx += part[i].x;
        sy += part[i].y;
    }
    for (int e = 0; e < P.n_empty; ++e) fhat[P.empty_off[e]] = make_double2(sx, sy);
}

int launch_adjoint_f64(Plan &p, const double2 *y, double2 *fhat) {
    DevPlan v = dev_view(p);
    cudaStream_t st = p.stream;
    if (p.M == 0) {
        cudaMemsetAsync(fhat, 0, sizeof(double2) * p.n_coeffs, st);
        return cuda_status(cudaGetLastError());
    }
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(spread_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        cudaFuncSetAttribute(adjoint_post_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
    if (p.n_empty > 0) {
        const int nb = 256;
        stage_begin(p, ST_SUMY);
        sum_y_f64_stage1<<<nb, 256, 0, st>>>(v, y, (double2 *)p.scratch);
        sum_y_f64_stage2<<<1, 32, 0, st>>>(v, (const double2 *)p.scratch, nb, fhat);
        stage_end(p, ST_SUMY);
    }
    if (p.n_act == 0) return cuda_status(cudaGetLastError());
    const size_t ssm = (size_t)p.max_grid_bytes + 16;
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(MAX_SMEM + 1024) / (ssm + 1024)));
    const int ctas = std::max(1, std::min(p.n_items, per_sm * p.sm_count));
    stage_begin(p, ST_SPREAD);
    cudaMemsetAsync(p.counter, 0, sizeof(int), st);
    spread_f64<<<ctas, 256, ssm, st>>>(v, p.items, y, p.n_items, p.counter, p.max_grid_bytes, p.wt64, p.wb64);
    stage_end(p, ST_SPREAD);
    stage_begin(p, ST_REDUCE);
    const int rb = (int)std::max<long long>(1, std::min<long long>(p.sm_count * 8LL, (p.grid_elems + 255) / 256));
    reduce_partials_f64<<<rb, 256, 0, st>>>(v);
    stage_end(p, ST_REDUCE);
    stage_begin(p, ST_POST);
    adjoint_post_f64<<<p.n_act, 256, (size_t)p.max_fft_elems * 2 * sizeof(double2), st>>>(v, fhat);
    stage_end(p, ST_POST);
    return cuda_status(cudaGetLastError());
}

}  // namespace agft
