// Solvers around the grouped transform, driven on the device.
//
// * LSQR (Paige and Saunders 1982) for the Tikhonov problem eq. (new_min_prob),
//   Sec. 4.1, on A = F W^{-1/2} with damping sqrt(2 lambda) (the regulariser has
//   no factor 1/2).
// * FISTA, Algorithm "FISTA for group lasso", Sec. 4.2, with the prox p_L of
//   eq. (projection) in the closed form of Theorem "projection": per group zero
//   below the threshold of Lemma (iii), otherwise z / (1 + xi omega) with xi
//   from bisection then Newton (Remark after the Theorem); for omega = 1 this is
//   the group soft threshold.  Constant step (Remark after the Algorithm) or
//   backtracking.
// * KKT check of the group-lasso optimality conditions (Lemma (ii)/(iii)).
//
// Vectors are FP32 complex (the plan's precision); every scalar of the
// bidiagonalisation, every norm and inner product is accumulated and kept in
// FP64 on the device.  One iteration is recorded once into a CUDA graph and
// replayed; when the stopping test fires, a device flag makes every later
// kernel -- transform kernels included -- return at once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "solvers.cuh"

namespace agft {

static void free_work(SolverWork *W) {
    if (!W) return;
    void *b[] = {W->uM, W->tM, W->rM, W->v, W->w, W->x, W->tn, W->h, W->f, W->fp, W->g, W->ws, W->wd,
                 W->part, W->gnorm, W->goff, W->glen, W->gmask, W->st};
    for (void *q : b)
        if (q) cudaFree(q);
    if (W->e0) cudaEventDestroy(W->e0);
    if (W->e1) cudaEventDestroy(W->e1);
    if (W->join) cudaEventDestroy(W->join);
    if (W->stream) cudaStreamDestroy(W->stream);
    delete W;
}

// ------------------------------------------------------------ reductions --

// sum of the RED_BLOCKS partials of slot k into st->red[k]
__global__ void finish_sums(SolverState *st, const double *part, int nslots) {
    __shared__ double sh[32];
    if (st->done) return;
    for (int k = 0; k < nslots; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) v += part[k * RED_BLOCKS + i];
        double s = block_sum(v, sh);
        if (threadIdx.x == 0) st->red[k] = s;
        __syncthreads();
    }
}

#define SKIP_IF_DONE \
    if (st->done) return;

// out = (scale ? scale[i] : 1) * in, |out|^2 partial into slot 0
__global__ void k_scale_copy(const SolverState *st, float2 *out, const float2 *in, const float *scale, long long n,
                             double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 v = in[i];
        if (scale) {
            float s = scale[i];
            v.x *= s;
            v.y *= s;
        }
        out[i] = v;
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = s;
}

// out = a - coef * out (coef = st->red-derived scalar selected by `which`), partial |out|^2
// which: 0 -> alpha, 1 -> beta
__global__ void k_sub_scaled(const SolverState *st, float2 *out, const float2 *a, const float *scale, int which,
                             long long n, double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    const float c = (float)(which == 0 ? st->alpha : st->beta);
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 av = a[i];
        if (scale) {
            float s = scale[i];
            av.x *= s;
            av.y *= s;
        }
        float2 o = out[i];
        o.x = av.x - c * o.x;
        o.y = av.y - c * o.y;
        out[i] = o;
        acc += (double)o.x * o.x + (double)o.y * o.y;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out *= 1/norm where norm = sqrt(st->red[0]); writes the norm to alpha (which 0) or beta (1)
__global__ void k_set_norm(SolverState *st, int which) {
    if (st->done) return;
    double nv = sqrt(st->red[0]);
    if (which == 0)
        st->alpha = nv;
    else
        st->beta = nv;
}

__global__ void k_normalize(const SolverState *st, float2 *v, long long n, int which) {
    SKIP_IF_DONE
    const double nv = which == 0 ? st->alpha : st->beta;
    const float inv = nv > 0 ? (float)(1.0 / nv) : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 a = v[i];
        a.x *= inv;
        a.y *= inv;
        v[i] = a;
    }
}

__global__ void k_lsqr_init(SolverState *st) { lsqr_init_dev(st); }

__global__ void k_lsqr_scalars(SolverState *st) { lsqr_scalars_dev(st); }

// x += phi/rho w ; w = v - theta/rho w ; partial |x|^2
__global__ void k_lsqr_update(const SolverState *st, float2 *x, float2 *w, const float2 *v, long long n,
                              double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    const float a = (float)st->phi_rho, b = (float)st->theta_rho;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 wi = w[i], xi = x[i], vi = v[i];
        xi.x += a * wi.x;
        xi.y += a * wi.y;
        wi.x = vi.x - b * wi.x;
        wi.y = vi.y - b * wi.y;
        x[i] = xi;
        w[i] = wi;
        acc += (double)xi.x * xi.x + (double)xi.y * xi.y;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_lsqr_test(SolverState *st) { lsqr_test_dev(st); }

__global__ void k_weights(const double *w, float *ws, double *wd, long long n, int mode) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double om = w ? w[i] : 1.0;
        wd[i] = om;
        ws[i] = mode == 0 ? (float)(1.0 / sqrt(om)) : (float)om;
    }
}

__global__ void k_zero(float2 *v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = make_float2(0.f, 0.f);
}

// zero the coefficient blocks of masked groups (the adjoint skips inactive terms)
__global__ void k_mask_groups(float2 *v, const long long *goff, const long long *glen, const unsigned char *gmask) {
    const int u = blockIdx.x;
    if (gmask[u]) return;
    const long long o = goff[u], m = glen[u];
    for (long long i = threadIdx.x; i < m; i += blockDim.x) v[o + i] = make_float2(0.f, 0.f);
}

__global__ void k_diff(float2 *out, const float2 *a, const float2 *b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 u = a[i], v = b[i];
        out[i] = make_float2(u.x - v.x, u.y - v.y);
    }
}

__global__ void k_mul(float2 *out, const float2 *in, const float *scale, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 v = in[i];
        float s = scale[i];
        out[i] = make_float2(v.x * s, v.y * s);
    }
}

// ---------------------------------------------------------------- FISTA --

// r = F h - y (in place on r), partial |r|^2 into part slot 0
__global__ void k_residual(const SolverState *st, float2 *r, const float2 *y, long long n, double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 a = r[i], b = y[i];
        a.x -= b.x;
        a.y -= b.y;
        r[i] = a;
        acc += (double)a.x * a.x + (double)a.y * a.y;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = s;
}

// t(xi) = sum_k omega_k |z_k|^2 / (1/xi + omega_k)^2 over a group (block reduction)
__device__ double group_t(const float2 *h, const float2 *g, float invL, const double *wd, long long o, long long m,
                          double xi, double *sh, bool use_s) {
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 hv = h[o + i], gv = g[o + i];
        double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
        double om = wd[o + i];
        double den = use_s ? (xi + om) : (1.0 / xi + om);
        acc += om * (zx * zx + zy * zy) / (den * den);
    }
    double s = block_sum(acc, sh);
    __shared__ double bc;
    if (threadIdx.x == 0) bc = s;
    __syncthreads();
    double r = bc;
    __syncthreads();
    return r;
}

// Prox p_L of eq. (projection), one block per group: f_new = prox(h - g / L).
// Zero when sqrt(sum |z|^2 / omega) <= lam / L (Lemma (iii)); otherwise
// z / (1 + xi omega) with t(xi) = (lam/L)^2 (Theorem "projection"): for
// omega = 1 in closed form, else bisection on [0,1] in xi or in s = 1/xi and
// Newton steps (Remark after the Theorem).  Masked groups are zero.
__global__ void k_prox(const SolverState *st, float2 *fnew, const float2 *h, const float2 *g, const double *wd,
                       const long long *goff, const long long *glen, const unsigned char *gmask, int unit_w) {
    __shared__ double sh[32];
    __shared__ double s_scale, s_xi;
    __shared__ int s_mode;
    if (st->done) return;
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    const double L = st->L, thr = st->lam / L;
    const float invL = (float)(1.0 / L);
    if (gmask && !gmask[u]) {
        for (long long i = threadIdx.x; i < m; i += blockDim.x) fnew[o + i] = make_float2(0.f, 0.f);
        return;
    }
    // zero test
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 hv = h[o + i], gv = g[o + i];
        double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
        acc += (zx * zx + zy * zy) / wd[o + i];
    }
    double z2w = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double zn = sqrt(z2w);
        if (zn <= thr) {
            s_mode = 0;
        } else if (unit_w) {
            s_mode = 1;
            s_scale = 1.0 - thr / zn;
        } else {
            s_mode = 2;
        }
    }
    __syncthreads();
    if (s_mode == 0) {
        for (long long i = threadIdx.x; i < m; i += blockDim.x) fnew[o + i] = make_float2(0.f, 0.f);
        return;
    }
    if (s_mode == 1) {
        const double sc = s_scale;
        for (long long i = threadIdx.x; i < m; i += blockDim.x) {
            float2 hv = h[o + i], gv = g[o + i];
            double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
            fnew[o + i] = make_float2((float)(sc * zx), (float)(sc * zy));
        }
        return;
    }
    // general weights: root of t(xi) = thr^2
    const double lam2 = thr * thr;
    const double t1 = group_t(h, g, invL, wd, o, m, 1.0, sh, false);
    double xi;
    if (t1 >= lam2) {
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 40; ++it) {
            double mid = 0.5 * (lo + hi);
            double tv = mid > 0 ? group_t(h, g, invL, wd, o, m, mid, sh, false) : 0.0;
            if (tv < lam2) lo = mid; else hi = mid;
        }
        xi = 0.5 * (lo + hi);
        for (int it = 0; it < 30; ++it) {
            // d/dxi of omega |z|^2 (1/xi + omega)^-2 = 2 omega |z|^2 (1/xi + omega)^-3 / xi^2
            double f = group_t(h, g, invL, wd, o, m, xi, sh, false) - lam2;
            double acc2 = 0.0;
            for (long long i = threadIdx.x; i < m; i += blockDim.x) {
                float2 hv = h[o + i], gv = g[o + i];
                double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
                double om = wd[o + i], den = 1.0 / xi + om;
                acc2 += 2.0 * om * (zx * zx + zy * zy) / (den * den * den);
            }
            double fp = block_sum(acc2, sh);
            if (threadIdx.x == 0) s_xi = fp;
            __syncthreads();
            fp = s_xi / (xi * xi);
            __syncthreads();
            double nx = fmin(fmax(xi - f / fp, 0.5 * xi), 2.0 * xi);
            if (fabs(nx - xi) <= 1e-15 * xi) {
                xi = nx;
                break;
            }
            xi = nx;
        }
    } else {
        double lo = 0.0, hi = 1.0;   // g(s) = t(1/s) decreasing
        for (int it = 0; it < 40; ++it) {
            double mid = 0.5 * (lo + hi);
            double gv = group_t(h, g, invL, wd, o, m, mid, sh, true);
            if (gv > lam2) lo = mid; else hi = mid;
        }
        double s = 0.5 * (lo + hi);
        for (int it = 0; it < 30; ++it) {
            double f = group_t(h, g, invL, wd, o, m, s, sh, true) - lam2;
            double acc2 = 0.0;
            for (long long i = threadIdx.x; i < m; i += blockDim.x) {
                float2 hv = h[o + i], gv = g[o + i];
                double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
                double om = wd[o + i], den = s + om;
                acc2 += -2.0 * om * (zx * zx + zy * zy) / (den * den * den);
            }
            double fp = block_sum(acc2, sh);
            if (threadIdx.x == 0) s_xi = fp;
            __syncthreads();
            fp = s_xi;
            __syncthreads();
            double ns = s - f / fp;
            ns = s > 0 ? fmin(fmax(ns, 0.5 * s), 2.0 * s) : fmax(ns, 0.0);
            if (fabs(ns - s) <= 1e-15 * fmax(s, 1e-300)) {
                s = ns;
                break;
            }
            s = ns;
        }
        xi = s > 0 ? 1.0 / s : INFINITY;
    }
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 hv = h[o + i], gv = g[o + i];
        double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
        double sc = isfinite(xi) ? 1.0 / (1.0 + xi * wd[o + i]) : 0.0;
        fnew[o + i] = make_float2((float)(sc * zx), (float)(sc * zy));
    }
}

// momentum: t_next = (1 + sqrt(1 + 4 t^2))/2, h = f_new + (t - 1)/t_next (f_new - f);
// f_prev <- f, f <- f_new ; partials: |f_new - f|^2 (slot 0), |f_new|^2 (slot 1)
__global__ void k_momentum(const SolverState *st, float2 *h, float2 *f, float2 *fp, const float2 *fnew, long long n,
                           double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    const double t = st->t, tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const float beta = (float)((t - 1.0) / tn);
    double a0 = 0.0, a1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 fo = f[i], fnv = fnew[i];
        float dx = fnv.x - fo.x, dy = fnv.y - fo.y;
        h[i] = make_float2(fnv.x + beta * dx, fnv.y + beta * dy);
        fp[i] = fo;
        f[i] = fnv;
        a0 += (double)dx * dx + (double)dy * dy;
        a1 += (double)fnv.x * fnv.x + (double)fnv.y * fnv.y;
    }
    double s0 = block_sum(a0, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s0;
    double s1 = block_sum(a1, sh);
    if (threadIdx.x == 0) part[RED_BLOCKS + blockIdx.x] = s1;
}

__global__ void k_fista_step(SolverState *st) {
    if (st->done) return;
    const double t = st->t;
    st->t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    st->diff2 = st->red[0];
    st->fn2 = st->red[1];
    st->iters += 1;
    if (!isfinite(st->diff2) || !isfinite(st->fn2)) {
        st->status = ANOVA_ERR_NOT_FINITE;
        st->done = 1;
    } else if (st->tol > 0 && sqrt(st->diff2) <= st->tol * fmax(sqrt(st->fn2), 1e-300)) {
        st->stop = 1;
        st->done = 1;
    } else if (st->iters >= st->max_it) {
        st->done = 1;
    }
}

// backtracking quantities: slot 0 |F f - y|^2 is finished separately; here
// cross = Re<f - h, g> (slot 2) and |f - h|^2 (slot 3)
__global__ void k_bt_terms(const SolverState *st, const float2 *fnew, const float2 *h, const float2 *g, long long n,
                           double *part) {
    __shared__ double sh[32];
    double a2 = 0.0, a3 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 a = fnew[i], b = h[i], c = g[i];
        double dx = (double)a.x - b.x, dy = (double)a.y - b.y;
        a2 += dx * c.x + dy * c.y;
        a3 += dx * dx + dy * dy;
    }
    double s2 = block_sum(a2, sh);
    if (threadIdx.x == 0) part[2 * RED_BLOCKS + blockIdx.x] = s2;
    double s3 = block_sum(a3, sh);
    if (threadIdx.x == 0) part[3 * RED_BLOCKS + blockIdx.x] = s3;
}

// per-group norms: out[u] = sqrt(sum_k weight_k |v_k|^2) with weight omega (mode 0),
// 1/omega (mode 1) or 1 (mode 2)
__global__ void k_group_norms(const float2 *v, const double *wd, const long long *goff, const long long *glen,
                              double *out, int mode) {
    __shared__ double sh[32];
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 a = v[o + i];
        double q = (double)a.x * a.x + (double)a.y * a.y;
        double om = wd ? wd[o + i] : 1.0;
        acc += mode == 0 ? q * om : (mode == 1 ? q / om : q);
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[u] = sqrt(s);
}

// KKT residual per group, given q = F^H (F f - y) = -F^H r with r = y - F f:
// inactive (f_u = 0) groups (Lemma (iii)): (||W^{-1/2} q_u|| - lam) / lam;
// active groups (stationarity in the proof of Lemma (ii)):
// ||r-part - lam W f_u / ||f_u||_W|| / lam = ||-q_u - lam W f_u / ||f_u||_W|| / lam
__global__ void k_kkt(const float2 *g, const float2 *f, const double *wd, const long long *goff, const long long *glen,
                      double lam, double *viol) {
    __shared__ double sh[32];
    __shared__ double s_fn;
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 a = f[o + i];
        acc += ((double)a.x * a.x + (double)a.y * a.y) * wd[o + i];
    }
    double fn = block_sum(acc, sh);
    if (threadIdx.x == 0) s_fn = sqrt(fn);
    __syncthreads();
    fn = s_fn;
    __syncthreads();
    double acc2 = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 gv = g[o + i], fv = f[o + i];
        double om = wd[o + i];
        if (fn == 0.0) {
            acc2 += ((double)gv.x * gv.x + (double)gv.y * gv.y) / om;
        } else {
            double rx = -gv.x - lam * om * fv.x / fn, ry = -gv.y - lam * om * fv.y / fn;
            acc2 += rx * rx + ry * ry;
        }
    }
    double s = block_sum(acc2, sh);
    if (threadIdx.x == 0) viol[u] = fn == 0.0 ? (sqrt(s) - lam) / lam : sqrt(s) / lam;
}

// ---------------------------------------------------------------- host ----

static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(RED_BLOCKS, (n + 255) / 256)); }

SolverWork *get_work(Plan &p, int &rc) {
    rc = ANOVA_OK;
    SolverWork *W = (SolverWork *)p.solver;
    if (W) return W;
    W = new SolverWork();
    W->M = p.M;
    W->n = p.n_coeffs;
    const size_t bm = sizeof(float2) * std::max<long long>(1, p.M), bn = sizeof(float2) * std::max<long long>(1, p.n_coeffs);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **ptr, size_t b) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, b);
    };
    A((void **)&W->uM, bm);
    A((void **)&W->tM, bm);
    A((void **)&W->rM, bm);
    A((void **)&W->v, bn);
    A((void **)&W->w, bn);
    A((void **)&W->x, bn);
    A((void **)&W->tn, bn);
    A((void **)&W->h, bn);
    A((void **)&W->f, bn);
    A((void **)&W->fp, bn);
    A((void **)&W->g, bn);
    A((void **)&W->ws, sizeof(float) * std::max<long long>(1, p.n_coeffs));
    A((void **)&W->wd, sizeof(double) * std::max<long long>(1, p.n_coeffs));
    A((void **)&W->part, sizeof(double) * 8 * RED_BLOCKS);
    A((void **)&W->gnorm, sizeof(double) * std::max(1, p.n_user_terms));
    A((void **)&W->goff, sizeof(long long) * std::max(1, p.n_user_terms));
    A((void **)&W->glen, sizeof(long long) * std::max(1, p.n_user_terms));
    A((void **)&W->gmask, std::max(1, p.n_user_terms));
    A((void **)&W->st, sizeof(SolverState));
    if (e == cudaSuccess) e = cudaEventCreate(&W->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&W->e1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W->goff, p.h_user_off, sizeof(long long) * p.n_user_terms, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W->glen, p.h_user_len, sizeof(long long) * p.n_user_terms, cudaMemcpyHostToDevice, p.stream);
    if (e != cudaSuccess) {
        free_work(W);
        cudaGetLastError();
        rc = cuda_status(e);
        return nullptr;
    }
    p.solver = W;
    p.solver_free = [](void *q) { free_work((SolverWork *)q); };
    return W;
}

// one graph-recorded unit of work, replayed until the device flag `done` is set
struct Replay {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    ~Replay() {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    }
};

template <typename F>
static int run_loop(Plan &p, SolverWork *W, int max_it, F &&step) {
    // first step uncaptured (sets kernel attributes), then record one step
    int rc = step();
    if (rc) return rc;
    SolverState h;
    cudaError_t e = cudaMemcpyAsync(&h, W->st, sizeof(SolverState), cudaMemcpyDeviceToHost, p.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (h.done || max_it <= 1) return ANOVA_OK;
    Replay R;
    e = cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e);
    rc = step();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p.stream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : cuda_status(e);
    }
    R.g = g;
    e = cudaGraphInstantiate(&R.ge, g, 0);
    if (e != cudaSuccess) return cuda_status(e);
    const int chunk = 16;
    for (int it = 1; it < max_it;) {
        int k = std::min(chunk, max_it - it);
        for (int j = 0; j < k; ++j) {
            e = cudaGraphLaunch(R.ge, p.stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
        it += k;
        e = cudaMemcpyAsync(&h, W->st, sizeof(SolverState), cudaMemcpyDeviceToHost, p.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
        if (e != cudaSuccess) return cuda_status(e);
        if (h.done) break;
    }
    return ANOVA_OK;
}

static int lsqr_impl(Plan &p, const float2 *y, const double *w, double lambda, int max_it, double atol, double btol,
                     float2 *fhat, anova_solve_info *info) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    const long long M = p.M, n = p.n_coeffs;
    const int gM = grid_for(M), gn = grid_for(n);
    cudaStream_t s = p.stream;
    SolverState h0;
    std::memset(&h0, 0, sizeof(h0));
    h0.damp = std::sqrt(2.0 * lambda);
    h0.tiny_rel = std::max(1e-6, p.eps);
    h0.atol = atol;
    h0.btol = btol;
    h0.max_it = max_it;
    cudaMemcpyAsync(W->st, &h0, sizeof(h0), cudaMemcpyHostToDevice, s);
    k_weights<<<gn, 256, 0, s>>>(w, W->ws, W->wd, n, 0);
    const float *ws = w ? W->ws : nullptr;
    int n_tr = 0, n_adj = 0;
    cudaEventRecord(W->e0, s);
    // beta u = y
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->uM, y, nullptr, M, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 1);
    k_normalize<<<gM, 256, 0, s>>>(W->st, W->uM, M, 1);
    // alpha v = A^H u
    rc = launch_adjoint_f32(p, (const float2 *)W->uM, W->tn);
    ++n_adj;
    if (rc) return rc;
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->v, W->tn, ws, n, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 0);
    k_normalize<<<gn, 256, 0, s>>>(W->st, W->v, n, 0);
    cudaMemcpyAsync(W->w, W->v, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
    k_zero<<<gn, 256, 0, s>>>(W->x, n);
    k_lsqr_init<<<1, 1, 0, s>>>(W->st);
    p.skip = &W->st->done;
    auto step = [&]() -> int {
        // u = A v - alpha u ; beta = |u| ; u /= beta
        k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->tn, W->v, ws, n, nullptr);
        int r = launch_trafo_f32(p, (const float2 *)W->tn, W->tM);
        if (r) return r;
        k_sub_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->uM, W->tM, nullptr, 0, M, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_set_norm<<<1, 1, 0, s>>>(W->st, 1);
        k_normalize<<<gM, 256, 0, s>>>(W->st, W->uM, M, 1);
        // v = A^H u - beta v ; alpha = |v| (in the scalar kernel) ; v /= alpha
        r = launch_adjoint_f32(p, (const float2 *)W->uM, W->tn);
        if (r) return r;
        k_sub_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->v, W->tn, ws, 1, n, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_lsqr_scalars<<<1, 1, 0, s>>>(W->st);
        k_normalize<<<gn, 256, 0, s>>>(W->st, W->v, n, 0);
        k_lsqr_update<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->x, W->w, W->v, n, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_lsqr_test<<<1, 1, 0, s>>>(W->st);
        return cuda_status(cudaGetLastError());
    };
    rc = run_loop(p, W, max_it, step);
    p.skip = nullptr;
    if (rc) return rc;
    // fhat = W^{-1/2} x
    if (ws)
        k_mul<<<gn, 256, 0, s>>>(fhat, W->x, W->ws, n);
    else
        cudaMemcpyAsync(fhat, W->x, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
    cudaEventRecord(W->e1, s);
    SolverState h;
    cudaError_t e = cudaMemcpyAsync(&h, W->st, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, W->e0, W->e1);
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = h.iters;
        info->status = h.status;
        info->stop_reason = h.stop;
        info->n_trafo = h.iters;
        info->n_adjoint = h.iters + n_adj;
        info->rnorm = h.rnorm;
        info->arnorm = h.arnorm;
        info->seconds = ms * 1e-3;
    }
    (void)n_tr;
    if (h.status) return h.status;
    return h.stop == 1 ? ANOVA_ERR_BREAKDOWN : ANOVA_OK;
}

// power iteration for ||F||^2 on the active terms (30 steps, FP64 Rayleigh quotient)
static int power_estimate(Plan &p, SolverWork *W, int iters, bool masked, double *out) {
    cudaStream_t s = p.stream;
    const long long n = p.n_coeffs;
    const int gn = grid_for(n);
    std::vector<float2> ones(n, make_float2(1.f, 0.f));
    cudaMemcpyAsync(W->v, ones.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s);
    if (masked) k_mask_groups<<<p.n_user_terms, 256, 0, s>>>(W->v, W->goff, W->glen, W->gmask);
    SolverState h0;
    std::memset(&h0, 0, sizeof(h0));
    cudaMemcpyAsync(W->st, &h0, sizeof(h0), cudaMemcpyHostToDevice, s);
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->v, W->v, nullptr, n, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 0);
    k_normalize<<<gn, 256, 0, s>>>(W->st, W->v, n, 0);
    double lam = 0.0, prev = -1.0;
    for (int it = 0; it < iters; ++it) {
        int rc = launch_trafo_f32(p, (const float2 *)W->v, W->tM);
        if (rc) return rc;
        rc = launch_adjoint_f32(p, (const float2 *)W->tM, W->tn);
        if (rc) return rc;
        if (masked) k_mask_groups<<<p.n_user_terms, 256, 0, s>>>(W->tn, W->goff, W->glen, W->gmask);
        // ||F v||^2 = <v, F^H F v> with |v| = 1
        k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->tM, W->tM, nullptr, p.M, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        SolverState h;
        cudaMemcpyAsync(&h, W->st, sizeof(h), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        lam = h.red[0];
        if (prev > 0 && std::fabs(lam - prev) <= 1e-5 * lam) break;
        prev = lam;
        k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->v, W->tn, nullptr, n, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_set_norm<<<1, 1, 0, s>>>(W->st, 0);
        k_normalize<<<gn, 256, 0, s>>>(W->st, W->v, n, 0);
    }
    *out = lam;
    return cuda_status(cudaGetLastError());
}

int fista_impl(Plan &p, const float2 *y, const double *w, const double *lambdas, int n_lambda, int max_it,
               double tol, int step_mode, double L0, double eta, const uint8_t *mask, const float2 *f0,
               float2 *path, anova_solve_info *info, double *L_out) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    const long long M = p.M, n = p.n_coeffs;
    const int gM = grid_for(M), gn = grid_for(n), G = p.n_user_terms;
    cudaStream_t s = p.stream;
    k_weights<<<gn, 256, 0, s>>>(w, W->ws, W->wd, n, 1);
    std::vector<unsigned char> hm(G, 1);
    if (mask)
        for (int u = 0; u < G; ++u) hm[u] = mask[u] ? 1 : 0;
    cudaMemcpyAsync(W->gmask, hm.data(), G, cudaMemcpyHostToDevice, s);
    rc = set_active_terms(p, mask ? hm.data() : nullptr);
    if (rc) return rc;
    double L = L0;
    if (L <= 0) {
        double est = 0.0;
        rc = power_estimate(p, W, 300, mask != nullptr, &est);
        if (rc) return rc;
        L = 1.05 * est;
        if (!(L > 0)) L = 1.0;
    }
    std::vector<int> ord(n_lambda);
    for (int i = 0; i < n_lambda; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lambdas[a] > lambdas[b]; });
    if (f0) {
        cudaMemcpyAsync(W->f, f0, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
        if (mask) k_mask_groups<<<G, 256, 0, s>>>(W->f, W->goff, W->glen, W->gmask);
    } else {
        k_zero<<<gn, 256, 0, s>>>(W->f, n);
    }
    for (int li = 0; li < n_lambda; ++li) {
        const int idx = ord[li];
        SolverState h0;
        std::memset(&h0, 0, sizeof(h0));
        h0.t = 1.0;
        h0.L = L;
        h0.lam = lambdas[idx];
        h0.tol = tol;
        h0.max_it = max_it;
        h0.eta = eta;
        cudaMemcpyAsync(W->st, &h0, sizeof(h0), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(W->h, W->f, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
        cudaEventRecord(W->e0, s);
        int n_tr = 0, n_adj = 0;
        if (step_mode == 0) {
            p.skip = &W->st->done;
            auto step = [&]() -> int {
                int r = launch_trafo_f32(p, (const float2 *)W->h, W->rM);
                if (r) return r;
                k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->rM, y, M, nullptr);
                r = launch_adjoint_f32(p, (const float2 *)W->rM, W->g);
                if (r) return r;
                if (mask) k_mask_groups<<<G, 256, 0, s>>>(W->g, W->goff, W->glen, W->gmask);
                k_prox<<<G, 256, 0, s>>>(W->st, W->x, W->h, W->g, W->wd, W->goff, W->glen, W->gmask, w ? 0 : 1);
                k_momentum<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->h, W->f, W->fp, W->x, n, W->part);
                finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 2);
                k_fista_step<<<1, 1, 0, s>>>(W->st);
                return cuda_status(cudaGetLastError());
            };
            rc = run_loop(p, W, max_it, step);
            p.skip = nullptr;
            if (rc) return rc;
        } else {
            // backtracking: host checks the sufficient-decrease condition per trial
            SolverState hs;
            for (int it = 0; it < max_it; ++it) {
                rc = launch_trafo_f32(p, (const float2 *)W->h, W->rM);
                ++n_tr;
                if (rc) return rc;
                k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->rM, y, M, nullptr);
                rc = launch_adjoint_f32(p, (const float2 *)W->rM, W->g);
                ++n_adj;
                if (rc) return rc;
                if (mask) k_mask_groups<<<G, 256, 0, s>>>(W->g, W->goff, W->glen, W->gmask);
                for (int trial = 0; trial < 64; ++trial) {
                    // For the quadratic data term the Algorithm's test
                    //   ||y - F f||^2 - ||y - F h||^2 <= 2 Re<f - h, F^H (F h - y)> + L ||f - h||^2
                    // is exactly ||F d||^2 <= L ||d||^2 with d = f - h; that form has no
                    // cancellation of two nearly equal residual norms.
                    k_prox<<<G, 256, 0, s>>>(W->st, W->x, W->h, W->g, W->wd, W->goff, W->glen, W->gmask, w ? 0 : 1);
                    k_diff<<<gn, 256, 0, s>>>(W->tn, W->x, W->h, n);
                    rc = launch_trafo_f32(p, (const float2 *)W->tn, W->tM);
                    ++n_tr;
                    if (rc) return rc;
                    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->tM, W->tM, nullptr, M, W->part);
                    k_bt_terms<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->x, W->h, W->g, n, W->part);
                    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 4);
                    cudaMemcpyAsync(&hs, W->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
                    cudaError_t e = cudaStreamSynchronize(s);
                    if (e != cudaSuccess) return cuda_status(e);
                    if (hs.red[0] <= hs.L * hs.red[3]) break;
                    hs.L *= eta;
                    cudaMemcpyAsync(&W->st->L, &hs.L, sizeof(double), cudaMemcpyHostToDevice, s);
                }
                k_momentum<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->h, W->f, W->fp, W->x, n, W->part);
                finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 2);
                k_fista_step<<<1, 1, 0, s>>>(W->st);
                cudaMemcpyAsync(&hs, W->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return cuda_status(e);
                if (hs.done) break;
            }
        }
        // store the solution and the objective 1/2 ||y - F f||^2 + lam sum_u ||f_u||_W
        cudaMemcpyAsync(path + (long long)idx * n, W->f, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
        SolverState hf;
        cudaMemcpyAsync(&hf, W->st, sizeof(hf), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        L = hf.L;   // a backtracked L carries over to the next lambda
        if (info) {
            anova_solve_info &I = info[idx];
            std::memset(&I, 0, sizeof(I));
            SolverState z;
            std::memset(&z, 0, sizeof(z));
            cudaMemcpyAsync(W->st, &z, sizeof(z), cudaMemcpyHostToDevice, s);
            rc = launch_trafo_f32(p, (const float2 *)W->f, W->tM);
            if (rc) return rc;
            k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->tM, y, M, W->part);
            finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
            k_group_norms<<<G, 256, 0, s>>>(W->f, W->wd, W->goff, W->glen, W->gnorm, 0);
            cudaEventRecord(W->e1, s);
            std::vector<double> gn_h(G);
            SolverState hz;
            cudaMemcpyAsync(gn_h.data(), W->gnorm, sizeof(double) * G, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(&hz, W->st, sizeof(hz), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_status(e);
            double pen = 0.0;
            int act = 0;
            for (int u = 0; u < G; ++u) {
                pen += gn_h[u];
                act += gn_h[u] > 0;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, W->e0, W->e1);
            I.iterations = hf.iters;
            I.status = hf.status;
            I.stop_reason = hf.stop;
            I.n_trafo = step_mode == 0 ? hf.iters : n_tr;
            I.n_adjoint = step_mode == 0 ? hf.iters : n_adj;
            I.active_groups = act;
            I.rnorm = std::sqrt(hz.red[0]);
            I.objective = 0.5 * hz.red[0] + lambdas[idx] * pen;
            I.L = hf.L;
            I.seconds = ms * 1e-3;
        }
        if (hf.status) {
            set_active_terms(p, nullptr);
            return hf.status;
        }
    }
    if (L_out) *L_out = L;
    return set_active_terms(p, nullptr);
}

}  // namespace agft

using namespace agft;

extern "C" {

int lsqr_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, double lambda, int max_it, double atol,
               double btol, void *fhat_dev, anova_solve_info *info) {
    if (!plan || !fhat_dev || lambda < 0 || max_it < 1 || atol < 0 || btol < 0) return ANOVA_ERR_INVALID;
    cudaGetLastError();   // do not report an earlier, unrelated error
    Plan &p = plan->p;
    if (p.M > 0 && !y_dev) return ANOVA_ERR_INVALID;
    if (p.precision != ANOVA_PREC_F32) return ANOVA_ERR_UNSUPPORTED;
    if (p.M == 0) {
        cudaMemsetAsync(fhat_dev, 0, sizeof(float2) * p.n_coeffs, p.stream);
        if (info) std::memset(info, 0, sizeof(*info));
        return cuda_status(cudaStreamSynchronize(p.stream));
    }
    return lsqr_impl(p, (const float2 *)y_dev, w_dev, lambda, max_it, atol, btol, (float2 *)fhat_dev, info);
}

int fista_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, const double *lambdas, int n_lambda,
                int max_it, double tol, int step_mode, double L0, double eta, const uint8_t *group_mask,
                int warm_start, void *fhat_path_dev, anova_solve_info *info) {
    if (!plan || !fhat_path_dev || !lambdas || n_lambda < 1 || max_it < 1 || tol < 0) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    if (step_mode != 0 && step_mode != 1) return ANOVA_ERR_INVALID;
    if (step_mode == 1 && !(eta > 1.0)) return ANOVA_ERR_INVALID;
    for (int i = 0; i < n_lambda; ++i)
        if (!(lambdas[i] >= 0)) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (p.M > 0 && !y_dev) return ANOVA_ERR_INVALID;
    if (p.precision != ANOVA_PREC_F32) return ANOVA_ERR_UNSUPPORTED;
    if (p.M == 0) return ANOVA_ERR_INVALID;
    return fista_impl(p, (const float2 *)y_dev, w_dev, lambdas, n_lambda, max_it, tol, step_mode, L0, eta,
                      group_mask, warm_start ? (const float2 *)fhat_path_dev : nullptr, (float2 *)fhat_path_dev,
                      info, nullptr);
}

// KKT check of a group-lasso solution: viol_out[u] for every user term (host
// array), returns the number of groups above rtol in *n_viol.
int anova_kkt_check(anova_plan_t plan, const void *y_dev, const double *w_dev, const void *fhat_dev, double lambda,
                    double rtol, double *viol_out, int *n_viol) {
    if (!plan || !fhat_dev || !(lambda > 0)) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (p.M > 0 && !y_dev) return ANOVA_ERR_INVALID;
    if (p.precision != ANOVA_PREC_F32) return ANOVA_ERR_UNSUPPORTED;
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    cudaStream_t s = p.stream;
    const long long n = p.n_coeffs, M = p.M;
    const int G = p.n_user_terms;
    k_weights<<<grid_for(n), 256, 0, s>>>(w_dev, W->ws, W->wd, n, 1);
    SolverState z;
    std::memset(&z, 0, sizeof(z));
    cudaMemcpyAsync(W->st, &z, sizeof(z), cudaMemcpyHostToDevice, s);
    rc = set_active_terms(p, nullptr);
    if (rc) return rc;
    rc = launch_trafo_f32(p, (const float2 *)fhat_dev, W->tM);
    if (rc) return rc;
    // F f - y, then q = F^H (F f - y)
    k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, W->tM, (const float2 *)y_dev, M, nullptr);
    rc = launch_adjoint_f32(p, (const float2 *)W->tM, W->g);
    if (rc) return rc;
    k_kkt<<<G, 256, 0, s>>>(W->g, (const float2 *)fhat_dev, W->wd, W->goff, W->glen, lambda, W->gnorm);
    std::vector<double> v(G);
    cudaMemcpyAsync(v.data(), W->gnorm, sizeof(double) * G, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    int cnt = 0;
    for (int u = 0; u < G; ++u) {
        if (viol_out) viol_out[u] = v[u];
        cnt += v[u] > rtol;
    }
    if (n_viol) *n_viol = cnt;
    return ANOVA_OK;
}

}  // extern "C"
