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

#include "solver_kernels.cuh"

namespace agft {

static void free_work(SolverWork *W) {
    if (!W) return;
    void *b[] = {W->uM, W->tM, W->rM, W->v, W->w, W->x, W->tn, W->h, W->f, W->fp, W->g, W->ws, W->wd,
                 W->part, W->gnorm, W->goff, W->glen, W->gmask, W->grho, W->gact, W->gorder, W->st};
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

// out *= 1/norm where norm = sqrt(st->red[0]); writes the norm to alpha (which 0) or beta (1)
__global__ void k_set_norm(SolverState *st, int which) {
    if (st->done) return;
    double nv = sqrt(st->red[0]);
    if (which == 0)
        st->alpha = nv;
    else
        st->beta = nv;
}

__global__ void k_lsqr_init(SolverState *st) { lsqr_init_dev(st); }

__global__ void k_lsqr_scalars(SolverState *st) { lsqr_scalars_dev(st); }

__global__ void k_lsqr_test(SolverState *st) { lsqr_test_dev(st); }

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

// ---------------------------------------------------------------- host ----

static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(RED_BLOCKS, (n + 255) / 256)); }

SolverWork *get_work(Plan &p, int &rc) {
    rc = ANOVA_OK;
    SolverWork *W = (SolverWork *)p.solver;
    if (W) return W;
    W = new SolverWork();
    W->M = p.M;
    W->n = p.n_coeffs;
    const size_t es = p.precision == ANOVA_PREC_F64 ? sizeof(double2) : sizeof(float2);   // complex element
    const size_t rs = es / 2;                                                                  // real element
    const size_t bm = es * std::max<long long>(1, p.M), bn = es * std::max<long long>(1, p.n_coeffs);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **ptr, size_t b) {
        if (e == cudaSuccess) e = plan_malloc(ptr, b);
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
    A((void **)&W->ws, rs * std::max<long long>(1, p.n_coeffs));
    A((void **)&W->wd, sizeof(double) * std::max<long long>(1, p.n_coeffs));
    A((void **)&W->part, sizeof(double) * 8 * RED_BLOCKS);
    A((void **)&W->gnorm, sizeof(double) * std::max(1, p.n_user_terms));
    A((void **)&W->goff, sizeof(long long) * std::max(1, p.n_user_terms));
    A((void **)&W->glen, sizeof(long long) * std::max(1, p.n_user_terms));
    A((void **)&W->gmask, std::max(1, p.n_user_terms));
    A((void **)&W->grho, sizeof(double) * std::max(1, p.n_user_terms));
    A((void **)&W->gact, std::max(1, p.n_user_terms));
    A((void **)&W->gorder, sizeof(int) * std::max(1, p.n_user_terms));
    A((void **)&W->st, sizeof(SolverState));
    if (e == cudaSuccess) e = cudaEventCreate(&W->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&W->e1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W->goff, p.h_user_off, sizeof(long long) * p.n_user_terms, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W->glen, p.h_user_len, sizeof(long long) * p.n_user_terms, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W->gorder, p.h_user_order, sizeof(int) * p.n_user_terms, cudaMemcpyHostToDevice, p.stream);
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

// The plan's complex vectors of a solver workspace, typed.
template <typename C>
struct Vecs {
    C *uM, *tM, *rM, *v, *w, *x, *tn, *h, *f, *fp, *g;
    typename CT<C>::R *ws;
    explicit Vecs(const SolverWork *W)
        : uM((C *)W->uM), tM((C *)W->tM), rM((C *)W->rM), v((C *)W->v), w((C *)W->w), x((C *)W->x),
          tn((C *)W->tn), h((C *)W->h), f((C *)W->f), fp((C *)W->fp), g((C *)W->g),
          ws((typename CT<C>::R *)W->ws) {}
};

// the transforms by vector type
static int trafo_c(Plan &p, const float2 *fhat, float2 *f) { return launch_trafo_f32(p, fhat, f); }
static int trafo_c(Plan &p, const double2 *fhat, double2 *f) { return launch_trafo_f64(p, fhat, f); }
static int adjoint_c(Plan &p, const float2 *y, float2 *fhat) { return launch_adjoint_f32(p, y, fhat); }
static int adjoint_c(Plan &p, const double2 *y, double2 *fhat) { return launch_adjoint_f64(p, y, fhat); }

template <typename C>
static int lsqr_impl(Plan &p, const C *y, const double *w, double lambda, int max_it, double atol, double btol,
                     C *fhat, anova_solve_info *info) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    using R = typename CT<C>::R;
    const Vecs<C> V(W);
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
    k_weights<<<gn, 256, 0, s>>>(w, V.ws, W->wd, n, 0);
    const R *ws = w ? V.ws : nullptr;
    int n_tr = 0, n_adj = 0;
    cudaEventRecord(W->e0, s);
    // beta u = y
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.uM, y, nullptr, M, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 1);
    k_normalize<<<gM, 256, 0, s>>>(W->st, V.uM, M, 1);
    // alpha v = A^H u
    rc = adjoint_c(p, (const C *)V.uM, V.tn);
    ++n_adj;
    if (rc) return rc;
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.v, V.tn, ws, n, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 0);
    k_normalize<<<gn, 256, 0, s>>>(W->st, V.v, n, 0);
    cudaMemcpyAsync(V.w, V.v, sizeof(C) * n, cudaMemcpyDeviceToDevice, s);
    k_zero<<<gn, 256, 0, s>>>(V.x, n);
    k_lsqr_init<<<1, 1, 0, s>>>(W->st);
    p.skip = &W->st->done;
    auto step = [&]() -> int {
        // u = A v - alpha u ; beta = |u| ; u /= beta
        k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.tn, V.v, ws, n, nullptr);
        int r = trafo_c(p, (const C *)V.tn, V.tM);
        if (r) return r;
        k_sub_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.uM, V.tM, nullptr, 0, M, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_set_norm<<<1, 1, 0, s>>>(W->st, 1);
        k_normalize<<<gM, 256, 0, s>>>(W->st, V.uM, M, 1);
        // v = A^H u - beta v ; alpha = |v| (in the scalar kernel) ; v /= alpha
        r = adjoint_c(p, (const C *)V.uM, V.tn);
        if (r) return r;
        k_sub_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.v, V.tn, ws, 1, n, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_lsqr_scalars<<<1, 1, 0, s>>>(W->st);
        k_normalize<<<gn, 256, 0, s>>>(W->st, V.v, n, 0);
        k_lsqr_update<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.x, V.w, V.v, n, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_lsqr_test<<<1, 1, 0, s>>>(W->st);
        return cuda_status(cudaGetLastError());
    };
    rc = run_loop(p, W, max_it, step);
    p.skip = nullptr;
    if (rc) return rc;
    // fhat = W^{-1/2} x
    if (ws)
        k_mul<<<gn, 256, 0, s>>>(fhat, V.x, V.ws, n);
    else
        cudaMemcpyAsync(fhat, V.x, sizeof(C) * n, cudaMemcpyDeviceToDevice, s);
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

// largest eigenvalue of the symmetric tridiagonal matrix (diag d, off-diagonal
// e) by bisection on the Sturm count
static double tridiag_max_eig(const std::vector<double> &d, const std::vector<double> &e) {
    const int k = (int)d.size();
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
        hi = std::max(hi, d[i] + r);
    }
    auto count_below = [&](double x) {   // eigenvalues < x
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < k; ++i) {
            q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            c += q < 0;
        }
        return c;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(mid) == k) hi = mid; else lo = mid;
    }
    return hi;
}

// ||F||^2 on the active terms (group-masked if asked) from the Golub--Kahan
// bidiagonalisation F V_k = U_k B_k started at the all-ones vector: the largest
// Ritz value of B_k^T B_k is a lower bound that converges much faster than the
// power iteration (Lanczos on F^H F).  It stops when a step changes it by less
// than 1e-3 relative (after at least 8 steps), or after max_steps steps.  On
// clustered spectra (the d = 30, M = 2e6 workload) the Ritz values creep
// upwards for dozens of steps: at that point they lie within about 1.5 % of
// the 60-step value, so the step bound takes LANCZOS_MARGIN = 1.08 times the
// estimate (1.05 times the 60-step value before).  Scalars in FP64.
constexpr double LANCZOS_MARGIN = 1.08;
template <typename C>
static int lanczos_estimate(Plan &p, SolverWork *W, int max_steps, bool masked, double *out) {
    const Vecs<C> V(W);
    cudaStream_t s = p.stream;
    const long long n = p.n_coeffs, M = p.M;
    const int gn = grid_for(n), gM = grid_for(M);
    C one;
    one.x = 1;
    one.y = 0;
    std::vector<C> ones(n, one);
    cudaMemcpyAsync(V.v, ones.data(), sizeof(C) * n, cudaMemcpyHostToDevice, s);
    if (masked) k_mask_groups<<<p.n_user_terms, 256, 0, s>>>(V.v, W->goff, W->glen, W->gmask);
    SolverState h0;
    std::memset(&h0, 0, sizeof(h0));
    cudaMemcpyAsync(W->st, &h0, sizeof(h0), cudaMemcpyHostToDevice, s);
    // v_1 = ones / |ones|  (the norm goes through beta, which is unused otherwise here)
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.v, V.v, nullptr, n, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 1);
    k_normalize<<<gn, 256, 0, s>>>(W->st, V.v, n, 1);
    // alpha_1 u_1 = F v_1
    int rc = trafo_c(p, (const C *)V.v, V.uM);
    if (rc) return rc;
    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.uM, V.uM, nullptr, M, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
    k_set_norm<<<1, 1, 0, s>>>(W->st, 0);
    k_normalize<<<gM, 256, 0, s>>>(W->st, V.uM, M, 0);
    std::vector<double> alpha, beta;
    double est = 0.0, prev = -1.0;
    for (int it = 0; it < max_steps; ++it) {
        SolverState h;
        cudaMemcpyAsync(&h, W->st, sizeof(h), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        alpha.push_back(h.alpha);
        if (!(h.alpha > 0)) break;
        // beta_i v_{i+1} = F^H u_i - alpha_i v_i
        rc = adjoint_c(p, (const C *)V.uM, V.tn);
        if (rc) return rc;
        if (masked) k_mask_groups<<<p.n_user_terms, 256, 0, s>>>(V.tn, W->goff, W->glen, W->gmask);
        k_sub_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.v, V.tn, nullptr, 0, n, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_set_norm<<<1, 1, 0, s>>>(W->st, 1);
        k_normalize<<<gn, 256, 0, s>>>(W->st, V.v, n, 1);
        // alpha_{i+1} u_{i+1} = F v_{i+1} - beta_i u_i
        rc = trafo_c(p, (const C *)V.v, V.tM);
        if (rc) return rc;
        k_sub_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.uM, V.tM, nullptr, 1, M, W->part);
        finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
        k_set_norm<<<1, 1, 0, s>>>(W->st, 0);
        k_normalize<<<gM, 256, 0, s>>>(W->st, V.uM, M, 0);
        cudaMemcpyAsync(&h, W->st, sizeof(h), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        beta.push_back(h.beta);
        // T = B^T B for the k x k upper bidiagonal B (alpha on the diagonal, beta above)
        const int k = (int)alpha.size();
        std::vector<double> d(k), off(std::max(0, k - 1));
        for (int i = 0; i < k; ++i) d[i] = alpha[i] * alpha[i] + (i > 0 ? beta[i - 1] * beta[i - 1] : 0.0);
        for (int i = 0; i + 1 < k; ++i) off[i] = alpha[i] * beta[i];
        est = tridiag_max_eig(d, off);
        if (k >= 8 && prev > 0 && std::fabs(est - prev) <= 1e-3 * est) break;
        prev = est;
        if (!(h.beta > 0)) break;
    }
    *out = est;
    return cuda_status(cudaGetLastError());
}

template <typename C>
int fista_impl_t(Plan &p, const C *y, const double *w, const double *lambdas, int n_lambda, int max_it,
               double tol, int step_mode, double L0, double eta, const uint8_t *mask, const C *f0,
               C *path, anova_solve_info *info, double *L_out) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    using R = typename CT<C>::R;
    const Vecs<C> V(W);
    const long long M = p.M, n = p.n_coeffs;
    const int gM = grid_for(M), gn = grid_for(n), G = p.n_user_terms;
    cudaStream_t s = p.stream;
    k_weights<<<gn, 256, 0, s>>>(w, V.ws, W->wd, n, 1);
    std::vector<unsigned char> hm(G, 1);
    if (mask)
        for (int u = 0; u < G; ++u) hm[u] = mask[u] ? 1 : 0;
    cudaMemcpyAsync(W->gmask, hm.data(), G, cudaMemcpyHostToDevice, s);
    rc = set_active_terms(p, mask ? hm.data() : nullptr);
    if (rc) return rc;
    double L = L0;
    if (L <= 0) {
        double est = 0.0;
        rc = lanczos_estimate<C>(p, W, 60, mask != nullptr, &est);
        if (rc) return rc;
        L = LANCZOS_MARGIN * est;
        if (!(L > 0)) L = 1.0;
    }
    std::vector<int> ord(n_lambda);
    for (int i = 0; i < n_lambda; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lambdas[a] > lambdas[b]; });
    if (f0) {
        cudaMemcpyAsync(V.f, f0, sizeof(C) * n, cudaMemcpyDeviceToDevice, s);
        if (mask) k_mask_groups<<<G, 256, 0, s>>>(V.f, W->goff, W->glen, W->gmask);
    } else {
        k_zero<<<gn, 256, 0, s>>>(V.f, n);
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
        cudaMemcpyAsync(V.h, V.f, sizeof(C) * n, cudaMemcpyDeviceToDevice, s);
        cudaEventRecord(W->e0, s);
        int n_tr = 0, n_adj = 0;
        if (step_mode == 0) {
            p.skip = &W->st->done;
            auto step = [&]() -> int {
                int r = trafo_c(p, (const C *)V.h, V.rM);
                if (r) return r;
                k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.rM, y, M, nullptr);
                r = adjoint_c(p, (const C *)V.rM, V.g);
                if (r) return r;
                if (mask) k_mask_groups<<<G, 256, 0, s>>>(V.g, W->goff, W->glen, W->gmask);
                k_prox<<<G, 256, 0, s>>>(W->st, V.x, V.h, V.g, W->wd, W->goff, W->glen, W->gmask, w ? 0 : 1);
                k_momentum<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.h, V.f, V.fp, V.x, n, W->part);
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
                rc = trafo_c(p, (const C *)V.h, V.rM);
                ++n_tr;
                if (rc) return rc;
                k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.rM, y, M, nullptr);
                rc = adjoint_c(p, (const C *)V.rM, V.g);
                ++n_adj;
                if (rc) return rc;
                if (mask) k_mask_groups<<<G, 256, 0, s>>>(V.g, W->goff, W->glen, W->gmask);
                for (int trial = 0; trial < 64; ++trial) {
                    // For the quadratic data term the Algorithm's test
                    //   ||y - F f||^2 - ||y - F h||^2 <= 2 Re<f - h, F^H (F h - y)> + L ||f - h||^2
                    // is exactly ||F d||^2 <= L ||d||^2 with d = f - h; that form has no
                    // cancellation of two nearly equal residual norms.
                    k_prox<<<G, 256, 0, s>>>(W->st, V.x, V.h, V.g, W->wd, W->goff, W->glen, W->gmask, w ? 0 : 1);
                    k_diff<<<gn, 256, 0, s>>>(V.tn, V.x, V.h, n);
                    rc = trafo_c(p, (const C *)V.tn, V.tM);
                    ++n_tr;
                    if (rc) return rc;
                    k_scale_copy<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.tM, V.tM, nullptr, M, W->part);
                    k_bt_terms<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.x, V.h, V.g, n, W->part);
                    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 4);
                    cudaMemcpyAsync(&hs, W->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
                    cudaError_t e = cudaStreamSynchronize(s);
                    if (e != cudaSuccess) return cuda_status(e);
                    if (hs.red[0] <= hs.L * hs.red[3]) break;
                    hs.L *= eta;
                    cudaMemcpyAsync(&W->st->L, &hs.L, sizeof(double), cudaMemcpyHostToDevice, s);
                }
                k_momentum<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.h, V.f, V.fp, V.x, n, W->part);
                finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 2);
                k_fista_step<<<1, 1, 0, s>>>(W->st);
                cudaMemcpyAsync(&hs, W->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return cuda_status(e);
                if (hs.done) break;
            }
        }
        // store the solution and the objective 1/2 ||y - F f||^2 + lam sum_u ||f_u||_W
        cudaMemcpyAsync(path + (long long)idx * n, V.f, sizeof(C) * n, cudaMemcpyDeviceToDevice, s);
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
            // leaves the residual F f - y in tM (the screened path's KKT check
            // of a one-lambda call reuses it)
            rc = trafo_c(p, (const C *)V.f, V.tM);
            if (rc) return rc;
            k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.tM, y, M, W->part);
            finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 1);
            k_group_norms<<<G, 256, 0, s>>>(V.f, W->wd, W->goff, W->glen, W->gnorm, 0);
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

// LANCZOS_MARGIN x the Lanczos estimate of ||F||^2 over all terms (FP32 plans):
// a valid FISTA step bound for the full problem and for every group-masked one
int lipschitz_estimate(Plan &p, double *L) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    rc = set_active_terms(p, nullptr);
    if (rc) return rc;
    double est = 0.0;
    {
        StreamScope scope(p, W);
        rc = lanczos_estimate<float2>(p, W, 60, false, &est);
    }
    if (rc) return rc;
    *L = est > 0 ? LANCZOS_MARGIN * est : 1.0;
    return cuda_status(cudaStreamSynchronize(p.stream));
}

int fista_impl(Plan &p, const float2 *y, const double *w, const double *lambdas, int n_lambda, int max_it,
               double tol, int step_mode, double L0, double eta, const uint8_t *mask, const float2 *f0,
               float2 *path, anova_solve_info *info, double *L_out) {
    return fista_impl_t<float2>(p, y, w, lambdas, n_lambda, max_it, tol, step_mode, L0, eta, mask, f0, path, info,
                                L_out);
}

}  // namespace agft

namespace agft {

// KKT residuals of a group-lasso solution (see k_kkt) into viol_out (host).
template <typename C>
static int kkt_impl(Plan &p, const C *y, const double *w_dev, const C *fhat, double lambda, double rtol,
                    double *viol_out, int *n_viol) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    const Vecs<C> V(W);
    cudaStream_t s = p.stream;
    const long long n = p.n_coeffs, M = p.M;
    const int G = p.n_user_terms;
    k_weights<<<grid_for(n), 256, 0, s>>>(w_dev, V.ws, W->wd, n, 1);
    SolverState z;
    std::memset(&z, 0, sizeof(z));
    cudaMemcpyAsync(W->st, &z, sizeof(z), cudaMemcpyHostToDevice, s);
    rc = set_active_terms(p, nullptr);
    if (rc) return rc;
    rc = trafo_c(p, fhat, V.tM);
    if (rc) return rc;
    // F f - y, then q = F^H (F f - y)
    k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(W->st, V.tM, y, M, nullptr);
    rc = adjoint_c(p, (const C *)V.tM, V.g);
    if (rc) return rc;
    k_kkt<<<G, 256, 0, s>>>(V.g, fhat, W->wd, W->goff, W->glen, lambda, W->gnorm);
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

}  // namespace agft

using namespace agft;

extern "C" {

int lsqr_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, double lambda, int max_it, double atol,
               double btol, void *fhat_dev, anova_solve_info *info) {
    if (!plan || !fhat_dev || lambda < 0 || max_it < 1 || atol < 0 || btol < 0) return ANOVA_ERR_INVALID;
    cudaGetLastError();   // do not report an earlier, unrelated error
    Plan &p = plan->p;
    if (p.M > 0 && !y_dev) return ANOVA_ERR_INVALID;
    const bool f64 = p.precision == ANOVA_PREC_F64;
    if (p.M == 0) {
        cudaMemsetAsync(fhat_dev, 0, (f64 ? sizeof(double2) : sizeof(float2)) * p.n_coeffs, p.stream);
        if (info) std::memset(info, 0, sizeof(*info));
        return cuda_status(cudaStreamSynchronize(p.stream));
    }
    if (f64)
        return lsqr_impl<double2>(p, (const double2 *)y_dev, w_dev, lambda, max_it, atol, btol, (double2 *)fhat_dev,
                                  info);
    return lsqr_impl<float2>(p, (const float2 *)y_dev, w_dev, lambda, max_it, atol, btol, (float2 *)fhat_dev, info);
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
    if (p.M == 0) return ANOVA_ERR_INVALID;
    if (p.precision == ANOVA_PREC_F64)
        return fista_impl_t<double2>(p, (const double2 *)y_dev, w_dev, lambdas, n_lambda, max_it, tol, step_mode, L0,
                                     eta, group_mask, warm_start ? (const double2 *)fhat_path_dev : nullptr,
                                     (double2 *)fhat_path_dev, info, nullptr);
    return fista_impl_t<float2>(p, (const float2 *)y_dev, w_dev, lambdas, n_lambda, max_it, tol, step_mode, L0, eta,
                                group_mask, warm_start ? (const float2 *)fhat_path_dev : nullptr,
                                (float2 *)fhat_path_dev, info, nullptr);
}

// KKT check of a group-lasso solution: viol_out[u] for every user term (host
// array), returns the number of groups above rtol in *n_viol.
int anova_kkt_check(anova_plan_t plan, const void *y_dev, const double *w_dev, const void *fhat_dev, double lambda,
                    double rtol, double *viol_out, int *n_viol) {
    if (!plan || !fhat_dev || !(lambda > 0)) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Plan &p = plan->p;
    if (p.M > 0 && !y_dev) return ANOVA_ERR_INVALID;
    if (p.precision == ANOVA_PREC_F64)
        return kkt_impl<double2>(p, (const double2 *)y_dev, w_dev, (const double2 *)fhat_dev, lambda, rtol, viol_out,
                                 n_viol);
    return kkt_impl<float2>(p, (const float2 *)y_dev, w_dev, (const float2 *)fhat_dev, lambda, rtol, viol_out, n_viol);
}

}  // extern "C"
