// Learned group screening along a group-lasso lambda path.
//
// No counterpart in the paper.  For each lambda (largest first, warm started
// as in the experiments of Sec. 4.2) the MLP of mlp.cu proposes the groups
// that will be nonzero, FISTA runs with the transforms restricted to the
// proposed groups, and a full KKT check (one grouped_trafo and one
// grouped_adjoint over all terms: Lemma (iii) for the groups held at zero)
// re-admits every violating group and re-solves, until none violates.  The
// result is therefore the full group-lasso solution; the network only decides
// how much transform work is spent on groups that end at zero.
//
// Features of group u at the step lambda_prev -> lambda (q = F^H (F f - y) at
// the previous solution f, all norms FP64):
//   0 log(1 + ||q_u||_{W^{-1}} / lambda)       KKT score at the new lambda
//   1 log(1 + ||q_u||_{W^{-1}} / lambda_prev)  score at the previous lambda
//   2 ||f_u||_W / max_v ||f_v||_W              relative size at the previous lambda
//   3 [f_u != 0]
//   4 |u| / 3
//   5 log(1 + |I_u|) / 8
//   6 log(lambda_prev / lambda)
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "solver_kernels.cuh"

namespace agft {

constexpr int N_FEAT = 7;

__global__ void k_features(const float2 *__restrict__ q, const float2 *__restrict__ f, const double *__restrict__ wd,
                           const long long *goff, const long long *glen, const int *order, double lam, double lam_prev,
                           double fmax, float *X) {
    __shared__ double sh[2][256];
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double aq = 0.0, af = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 a = q[o + i], b = f[o + i];
        double om = wd[o + i];
        aq += ((double)a.x * a.x + (double)a.y * a.y) / om;
        af += ((double)b.x * b.x + (double)b.y * b.y) * om;
    }
    sh[0][threadIdx.x] = aq;
    sh[1][threadIdx.x] = af;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double qs = sqrt(sh[0][0]), fs = sqrt(sh[1][0]);
        float *x = X + (size_t)u * N_FEAT;
        x[0] = (float)log1p(qs / lam);
        x[1] = (float)log1p(qs / lam_prev);
        x[2] = (float)(fmax > 0 ? fs / fmax : 0.0);
        x[3] = fs > 0 ? 1.f : 0.f;
        x[4] = (float)order[u] / 3.f;
        x[5] = (float)(log1p((double)m) / 8.0);
        x[6] = (float)log(lam_prev / lam);
    }
}

// ||q_u||_{W^{-1}} and ||f_u||_W per group into out[2u], out[2u+1]
__global__ void k_group_pair(const float2 *__restrict__ q, const float2 *__restrict__ f, const double *__restrict__ wd,
                             const long long *goff, const long long *glen, double *out) {
    __shared__ double sh[2][256];
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double aq = 0.0, af = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        float2 a = q[o + i], b = f[o + i];
        double om = wd[o + i];
        aq += ((double)a.x * a.x + (double)a.y * a.y) / om;
        af += ((double)b.x * b.x + (double)b.y * b.y) * om;
    }
    sh[0][threadIdx.x] = aq;
    sh[1][threadIdx.x] = af;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * u] = sqrt(sh[0][0]);
        out[2 * u + 1] = sqrt(sh[1][0]);
    }
}

struct ScreenWork {
    float *X = nullptr, *prob = nullptr;
    float2 *q = nullptr, *fprev = nullptr, *fcur = nullptr;
    double *pair = nullptr;
    int *order = nullptr;
    ~ScreenWork() {
        void *b[] = {X, prob, q, fprev, fcur, pair, order};
        for (void *p : b)
            if (p) cudaFree(p);
    }
};

// q = F^H (F f - y) over all terms
// q = F^H (F f - y) over all groups.  f is zero outside the groups of fmask
// (user terms; NULL: any group), so the forward runs over those only; the
// adjoint, which the KKT scores need for every group, over all of them.
// residual_ready: W->tM already holds F f - y (a one-lambda fista_impl call
// with info leaves its solution's residual there), so only the adjoint runs.
static int full_gradient(Plan &p, SolverWork *W, const float2 *y, const float2 *f, float2 *q,
                         const uint8_t *fmask, bool residual_ready = false) {
    float2 *tM = (float2 *)W->tM;
    if (!residual_ready) {
        int rc = set_active_terms(p, fmask);
        if (rc) return rc;
        rc = launch_trafo_f32(p, f, tM);
        if (rc) return rc;
        k_residual<<<RED_BLOCKS, RED_THREADS, 0, p.stream>>>(W->st, tM, y, p.M, nullptr);
    }
    int rc = set_active_terms(p, nullptr);
    if (rc) return rc;
    return launch_adjoint_f32(p, tM, q);
}

static int features_host(Plan &p, SolverWork *W, ScreenWork &S, const float2 *f, std::vector<double> &pairs) {
    const int G = p.n_user_terms;
    k_group_pair<<<G, 256, 0, p.stream>>>(S.q, f, W->wd, W->goff, W->glen, S.pair);
    pairs.resize(2 * G);
    cudaMemcpyAsync(pairs.data(), S.pair, sizeof(double) * 2 * G, cudaMemcpyDeviceToHost, p.stream);
    return cuda_status(cudaStreamSynchronize(p.stream));
}

}  // namespace agft

using namespace agft;

extern "C" {

int anova_screen_features(anova_plan_t plan, const void *y_dev, const double *w_dev, const void *fhat_dev,
                          double lambda, double lambda_prev, float *X_dev) {
    if (!plan || !y_dev || !fhat_dev || !X_dev || !(lambda > 0) || !(lambda_prev >= lambda)) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (p.precision != ANOVA_PREC_F32 || p.M == 0) return ANOVA_ERR_UNSUPPORTED;
    cudaGetLastError();
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    const int G = p.n_user_terms;
    const long long n = p.n_coeffs;
    k_weights<<<304, 256, 0, p.stream>>>(w_dev, (float *)W->ws, W->wd, n, 1);
    SolverState z;
    std::memset(&z, 0, sizeof(z));
    cudaMemcpyAsync(W->st, &z, sizeof(z), cudaMemcpyHostToDevice, p.stream);
    ScreenWork S;
    cudaError_t e = cudaMalloc(&S.q, sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&S.pair, sizeof(double) * 2 * G);
    if (e == cudaSuccess) e = cudaMalloc(&S.order, sizeof(int) * G);
    if (e != cudaSuccess) return cuda_status(e);
    cudaMemcpyAsync(S.order, p.h_user_order, sizeof(int) * G, cudaMemcpyHostToDevice, p.stream);
    rc = full_gradient(p, W, (const float2 *)y_dev, (const float2 *)fhat_dev, S.q, nullptr);
    if (rc) return rc;
    std::vector<double> pairs;
    rc = features_host(p, W, S, (const float2 *)fhat_dev, pairs);
    if (rc) return rc;
    double fmax = 0.0;
    for (int u = 0; u < G; ++u) fmax = std::max(fmax, pairs[2 * u + 1]);
    k_features<<<G, 256, 0, p.stream>>>(S.q, (const float2 *)fhat_dev, W->wd, W->goff, W->glen, S.order, lambda,
                                        lambda_prev, fmax, X_dev);
    return cuda_status(cudaStreamSynchronize(p.stream));
}

int fista_screened_path(anova_plan_t plan, anova_mlp_t mlp, const void *y_dev, const double *w_dev,
                        const double *lambdas, int n_lambda, int max_it, double tol, double threshold,
                        double kkt_tol, void *fhat_path_dev, anova_solve_info *info, anova_screen_stats *stats) {
    if (!plan || !mlp || !y_dev || !lambdas || n_lambda < 1 || max_it < 1 || !fhat_path_dev) return ANOVA_ERR_INVALID;
    for (int i = 0; i < n_lambda; ++i)
        if (!(lambdas[i] > 0)) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (p.precision != ANOVA_PREC_F32 || p.M == 0) return ANOVA_ERR_UNSUPPORTED;
    cudaGetLastError();
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    const int G = p.n_user_terms;
    const long long n = p.n_coeffs;
    const float2 *y = (const float2 *)y_dev;
    float2 *path = (float2 *)fhat_path_dev;
    ScreenWork S;
    cudaError_t e = cudaMalloc(&S.X, sizeof(float) * N_FEAT * G);
    if (e == cudaSuccess) e = cudaMalloc(&S.prob, sizeof(float) * G);
    if (e == cudaSuccess) e = cudaMalloc(&S.q, sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&S.fprev, sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&S.pair, sizeof(double) * 2 * G);
    if (e == cudaSuccess) e = cudaMalloc(&S.order, sizeof(int) * G);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<int> ord(n_lambda);
    for (int i = 0; i < n_lambda; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lambdas[a] > lambdas[b]; });
    auto t0 = std::chrono::steady_clock::now();
    {
        StreamScope scope(p, W);
        k_weights<<<304, 256, 0, p.stream>>>(w_dev, (float *)W->ws, W->wd, n, 1);
        cudaMemcpyAsync(S.order, p.h_user_order, sizeof(int) * G, cudaMemcpyHostToDevice, p.stream);
        k_zero<<<304, 256, 0, p.stream>>>(S.fprev, n);
        SolverState z;
        std::memset(&z, 0, sizeof(z));
        cudaMemcpyAsync(W->st, &z, sizeof(z), cudaMemcpyHostToDevice, p.stream);
        // f = 0: the forward is the empty set's coefficient alone
        std::vector<uint8_t> none(p.n_user_terms, 0);
        rc = full_gradient(p, W, y, S.fprev, S.q, none.data());
        if (rc) return rc;
        e = cudaStreamSynchronize(p.stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // a step bound for the whole path: ||F_S||^2 <= ||F||^2 for every group set S
    double Lpath = 0.0;
    rc = lipschitz_estimate(p, &Lpath);
    if (rc) return rc;
    double lam_prev = lambdas[ord[0]];
    std::vector<double> pairs;
    std::vector<float> prob(G);
    std::vector<uint8_t> mask(G);
    // the step bound of a small proposal depends only on its group set: kept
    // for the next solve on the same set (consecutive sparse lambdas mostly
    // propose the same groups), which saves its Lanczos estimate
    std::vector<uint8_t> bound_mask;
    double bound_L = 0.0;
    long long proposed_total = 0, readmitted_total = 0, rounds_total = 0, term_iters = 0, full_term_iters = 0;
    for (int li = 0; li < n_lambda; ++li) {
        const int idx = ord[li];
        const double lam = lambdas[idx];
        // features from the previous solution and the MLP proposal
        {
            StreamScope scope(p, W);
            rc = features_host(p, W, S, S.fprev, pairs);
            if (rc) return rc;
            double fmax = 0.0;
            for (int u = 0; u < G; ++u) fmax = std::max(fmax, pairs[2 * u + 1]);
            k_features<<<G, 256, 0, p.stream>>>(S.q, S.fprev, W->wd, W->goff, W->glen, S.order, lam, lam_prev, fmax,
                                                S.X);
        }
        e = cudaStreamSynchronize(p.stream);   // features ready (the scope joined the solver stream)
        if (e != cudaSuccess) return cuda_status(e);
        rc = anova_mlp_forward(mlp, S.X, G, S.prob);
        if (rc) return rc;
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_status(e);
        cudaMemcpy(prob.data(), S.prob, sizeof(float) * G, cudaMemcpyDeviceToHost);
        int proposed = 0;
        for (int u = 0; u < G; ++u) {
            mask[u] = (prob[u] > threshold || pairs[2 * u + 1] > 0 || p.h_user_order[u] == 0) ? 1 : 0;
            proposed += mask[u];
        }
        proposed_total += proposed;
        // solve on the proposed groups; re-admit KKT violators until none is left
        anova_solve_info I;
        int rounds = 0, readmitted = 0;
        for (; rounds < 16; ++rounds) {
            // a small proposal gets its own (smaller, cheap to estimate) step bound;
            // a large one the path's bound, which costs no extra transforms
            int prop_terms = 0;
            for (int u = 0; u < G; ++u) prop_terms += mask[u] && p.h_user_order[u] > 0;
            const bool small = 4 * prop_terms <= p.n_terms;
            double L0 = small ? 0.0 : Lpath;
            if (small && bound_L > 0.0 && bound_mask == mask) L0 = bound_L;
            double L = 0.0;
            rc = fista_impl(p, y, w_dev, &lam, 1, max_it, tol, 0, L0, 2.0, mask.data(), S.fprev,
                            path + (long long)idx * n, &I, &L);
            if (rc) return rc;
            if (small) {
                bound_mask = mask;
                bound_L = L;
            }
            int act_terms = 0;
            for (int u = 0; u < G; ++u) act_terms += mask[u] && p.h_user_order[u] > 0;
            term_iters += (long long)I.iterations * act_terms;
            full_term_iters += (long long)I.iterations * p.n_terms;
            {
                StreamScope scope(p, W);
                rc = full_gradient(p, W, y, path + (long long)idx * n, S.q, mask.data(), true);
                if (rc) return rc;
                rc = features_host(p, W, S, path + (long long)idx * n, pairs);
                if (rc) return rc;
            }
            int added = 0;
            for (int u = 0; u < G; ++u)
                if (!mask[u] && pairs[2 * u] > lam * (1.0 + kkt_tol)) {
                    mask[u] = 1;
                    ++added;
                }
            readmitted += added;
            if (!added) break;
        }
        readmitted_total += readmitted;
        rounds_total += rounds + 1;
        if (info) info[idx] = I;
        // warm start for the next lambda
        cudaMemcpyAsync(S.fprev, path + (long long)idx * n, sizeof(float2) * n, cudaMemcpyDeviceToDevice, p.stream);
        lam_prev = lam;
    }
    e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->proposed_groups = proposed_total;
        stats->readmitted_groups = readmitted_total;
        stats->rounds = rounds_total;
        stats->term_iterations = term_iters;
        stats->full_term_iterations = full_term_iters;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return ANOVA_OK;
}

}  // extern "C"
