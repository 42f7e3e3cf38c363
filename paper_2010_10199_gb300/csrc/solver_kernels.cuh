// Vector kernels of the solvers, templated on the complex type of the plan's
// vectors (float2 for FP32 plans, double2 for FP64 plans).  Every reduction
// into `part` is accumulated in FP64.  Included by the translation units that
// launch them (each instantiates what it uses).
#pragma once

#include "solvers.cuh"

namespace agft {

template <typename C>
struct CT;
template <>
struct CT<float2> {
    using R = float;
};
template <>
struct CT<double2> {
    using R = double;
};

template <typename C>
__device__ __forceinline__ C mkc(double a, double b);
template <>
__device__ __forceinline__ float2 mkc<float2>(double a, double b) {
    return make_float2((float)a, (float)b);
}
template <>
__device__ __forceinline__ double2 mkc<double2>(double a, double b) {
    return make_double2(a, b);
}

#define SKIP_IF_DONE \
    if (st->done) return;

// out = (scale ? scale[i] : 1) * in, |out|^2 partial into slot 0
template <typename C, typename R = typename CT<C>::R>
__global__ void k_scale_copy(const SolverState *st, C *out, const C *in, const typename CT<C>::R *scale, long long n,
                             double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C v = in[i];
        if (scale) {
            R s = scale[i];
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
template <typename C, typename R = typename CT<C>::R>
__global__ void k_sub_scaled(const SolverState *st, C *out, const C *a, const typename CT<C>::R *scale, int which,
                             long long n, double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    const R c = (R)(which == 0 ? st->alpha : st->beta);
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C av = a[i];
        if (scale) {
            R s = scale[i];
            av.x *= s;
            av.y *= s;
        }
        C o = out[i];
        o.x = av.x - c * o.x;
        o.y = av.y - c * o.y;
        out[i] = o;
        acc += (double)o.x * o.x + (double)o.y * o.y;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename C, typename R = typename CT<C>::R>
__global__ void k_normalize(const SolverState *st, C *v, long long n, int which) {
    SKIP_IF_DONE
    const double nv = which == 0 ? st->alpha : st->beta;
    const R inv = nv > 0 ? (R)(1.0 / nv) : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C a = v[i];
        a.x *= inv;
        a.y *= inv;
        v[i] = a;
    }
}

// x += phi/rho w ; w = v - theta/rho w ; partial |x|^2
template <typename C, typename R = typename CT<C>::R>
__global__ void k_lsqr_update(const SolverState *st, C *x, C *w, const C *v, long long n,
                              double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    const R a = (R)st->phi_rho, b = (R)st->theta_rho;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C wi = w[i], xi = x[i], vi = v[i];
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

template <typename R>
__global__ void k_weights(const double *w, R *ws, double *wd, long long n, int mode) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double om = w ? w[i] : 1.0;
        wd[i] = om;
        ws[i] = mode == 0 ? (R)(1.0 / sqrt(om)) : (R)om;
    }
}

template <typename C, typename R = typename CT<C>::R>
__global__ void k_zero(C *v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = mkc<C>(0.f, 0.f);
}

// zero the coefficient blocks of masked groups (the adjoint skips inactive terms)
template <typename C, typename R = typename CT<C>::R>
__global__ void k_mask_groups(C *v, const long long *goff, const long long *glen, const unsigned char *gmask) {
    const int u = blockIdx.x;
    if (gmask[u]) return;
    const long long o = goff[u], m = glen[u];
    for (long long i = threadIdx.x; i < m; i += blockDim.x) v[o + i] = mkc<C>(0.f, 0.f);
}

template <typename C, typename R = typename CT<C>::R>
__global__ void k_diff(C *out, const C *a, const C *b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C u = a[i], v = b[i];
        out[i] = mkc<C>(u.x - v.x, u.y - v.y);
    }
}

template <typename C, typename R = typename CT<C>::R>
__global__ void k_mul(C *out, const C *in, const typename CT<C>::R *scale, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C v = in[i];
        R s = scale[i];
        out[i] = mkc<C>(v.x * s, v.y * s);
    }
}

// ---------------------------------------------------------------- FISTA --

// r = F h - y (in place on r), partial |r|^2 into part slot 0
template <typename C, typename R = typename CT<C>::R>
__global__ void k_residual(const SolverState *st, C *r, const C *y, long long n, double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C a = r[i], b = y[i];
        a.x -= b.x;
        a.y -= b.y;
        r[i] = a;
        acc += (double)a.x * a.x + (double)a.y * a.y;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = s;
}

// t(xi) = sum_k omega_k |z_k|^2 / (1/xi + omega_k)^2 over a group (block reduction)
template <typename C, typename R = typename CT<C>::R>
__device__ double group_t(const C *h, const C *g, R invL, const double *wd, long long o, long long m,
                          double xi, double *sh, bool use_s) {
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        C hv = h[o + i], gv = g[o + i];
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
template <typename C, typename R = typename CT<C>::R>
__global__ void k_prox(const SolverState *st, C *fnew, const C *h, const C *g, const double *wd,
                       const long long *goff, const long long *glen, const unsigned char *gmask, int unit_w) {
    __shared__ double sh[32];
    __shared__ double s_scale, s_xi;
    __shared__ int s_mode;
    if (st->done) return;
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    const double L = st->L, thr = st->lam / L;
    const R invL = (R)(1.0 / L);
    if (gmask && !gmask[u]) {
        for (long long i = threadIdx.x; i < m; i += blockDim.x) fnew[o + i] = mkc<C>(0.f, 0.f);
        return;
    }
    // zero test
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        C hv = h[o + i], gv = g[o + i];
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
        for (long long i = threadIdx.x; i < m; i += blockDim.x) fnew[o + i] = mkc<C>(0.f, 0.f);
        return;
    }
    if (s_mode == 1) {
        const double sc = s_scale;
        for (long long i = threadIdx.x; i < m; i += blockDim.x) {
            C hv = h[o + i], gv = g[o + i];
            double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
            fnew[o + i] = mkc<C>((R)(sc * zx), (R)(sc * zy));
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
                C hv = h[o + i], gv = g[o + i];
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
                C hv = h[o + i], gv = g[o + i];
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
        C hv = h[o + i], gv = g[o + i];
        double zx = (double)hv.x - (double)gv.x * invL, zy = (double)hv.y - (double)gv.y * invL;
        double sc = isfinite(xi) ? 1.0 / (1.0 + xi * wd[o + i]) : 0.0;
        fnew[o + i] = mkc<C>((R)(sc * zx), (R)(sc * zy));
    }
}

// momentum: t_next = (1 + sqrt(1 + 4 t^2))/2, h = f_new + (t - 1)/t_next (f_new - f);
// f_prev <- f, f <- f_new ; partials: |f_new - f|^2 (slot 0), |f_new|^2 (slot 1)
template <typename C, typename R = typename CT<C>::R>
__global__ void k_momentum(const SolverState *st, C *h, C *f, C *fp, const C *fnew, long long n,
                           double *part) {
    __shared__ double sh[32];
    SKIP_IF_DONE
    const double t = st->t, tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const R beta = (R)((t - 1.0) / tn);
    double a0 = 0.0, a1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C fo = f[i], fnv = fnew[i];
        R dx = fnv.x - fo.x, dy = fnv.y - fo.y;
        h[i] = mkc<C>(fnv.x + beta * dx, fnv.y + beta * dy);
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

// backtracking quantities: slot 0 |F f - y|^2 is finished separately; here
// cross = Re<f - h, g> (slot 2) and |f - h|^2 (slot 3)
template <typename C, typename R = typename CT<C>::R>
__global__ void k_bt_terms(const SolverState *st, const C *fnew, const C *h, const C *g, long long n,
                           double *part) {
    __shared__ double sh[32];
    double a2 = 0.0, a3 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C a = fnew[i], b = h[i], c = g[i];
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
template <typename C, typename R = typename CT<C>::R>
__global__ void k_group_norms(const C *v, const double *wd, const long long *goff, const long long *glen,
                              double *out, int mode) {
    __shared__ double sh[32];
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        C a = v[o + i];
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
template <typename C, typename R = typename CT<C>::R>
__global__ void k_kkt(const C *g, const C *f, const double *wd, const long long *goff, const long long *glen,
                      double lam, double *viol) {
    __shared__ double sh[32];
    __shared__ double s_fn;
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        C a = f[o + i];
        acc += ((double)a.x * a.x + (double)a.y * a.y) * wd[o + i];
    }
    double fn = block_sum(acc, sh);
    if (threadIdx.x == 0) s_fn = sqrt(fn);
    __syncthreads();
    fn = s_fn;
    __syncthreads();
    double acc2 = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        C gv = g[o + i], fv = f[o + i];
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


}  // namespace agft
