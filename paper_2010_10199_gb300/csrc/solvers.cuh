// Solver internals shared by solvers.cu and screen.cu.
#pragma once

#include "internal.cuh"

namespace agft {

// Every kernel that produces partial sums runs exactly RED_BLOCKS blocks
// (grid-stride loops; a block without work writes 0), so finish_sums always
// adds the same slots in the same order: deterministic and free of stale data.
constexpr int RED_BLOCKS = 304;
constexpr int RED_THREADS = 256;

struct SolverState {
    // LSQR
    double alpha, beta, rhobar, phibar, anorm2, bnorm, xnorm2, rnorm, arnorm, damp, res2;
    double phi_rho, theta_rho, atol, btol, tiny_rel;
    double red[8];          // finished reductions
    // FISTA
    double t, L, lam, tol, diff2, fn2, rh2, rf2, cross, dh2, eta;
    int done, iters, stop, status, max_it, accepted;
};

struct SolverWork {
    long long M = 0, n = 0;
    // complex vectors in the plan's precision (float2 or double2 elements)
    void *uM = nullptr, *tM = nullptr, *rM = nullptr;                          // node-sized
    void *v = nullptr, *w = nullptr, *x = nullptr, *tn = nullptr, *h = nullptr;  // coefficient-sized
    void *f = nullptr, *fp = nullptr, *g = nullptr;
    void *ws = nullptr;           // omega^{-1/2} (LSQR) or omega (FISTA) per coefficient, real type of the plan
    double *wd = nullptr;         // omega per coefficient (FP64)
    double *part = nullptr;       // [8][RED_BLOCKS] partial sums
    double *gnorm = nullptr;      // per-group values
    long long *goff = nullptr, *glen = nullptr;
    unsigned char *gmask = nullptr;
    double *grho = nullptr;        // per-group Sobol indices (analysis.cu)
    unsigned char *gact = nullptr; // and the active-set flags
    int *gorder = nullptr;         // |u| per user term
    SolverState *st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, join = nullptr;
    cudaStream_t stream = nullptr;   // own non-blocking stream: graph capture needs one
};

// Runs the solver on its own stream, ordered after the caller's stream and
// joined back into it at the end.
struct StreamScope {
    Plan &p;
    SolverWork *W;
    cudaStream_t user;
    StreamScope(Plan &p_, SolverWork *W_) : p(p_), W(W_), user(p_.stream) {
        cudaEventRecord(W->join, user);
        cudaStreamWaitEvent(W->stream, W->join, 0);
        p.stream = W->stream;
    }
    ~StreamScope() {
        cudaEventRecord(W->join, W->stream);
        cudaStreamWaitEvent(user, W->join, 0);
        p.stream = user;
    }
};


// LSQR initial scalars after beta u = y, alpha v = A^H u
__device__ inline void lsqr_init_dev(SolverState *st) {
    st->bnorm = st->beta;
    st->phibar = st->beta;
    st->rhobar = st->alpha;
    st->anorm2 = 0.0;
    st->iters = 0;
    st->stop = 0;
    st->status = 0;
    if (!isfinite(st->alpha) || !isfinite(st->beta)) {   // non-finite data (NaN or Inf in y)
        st->status = ANOVA_ERR_NOT_FINITE;
        st->done = 1;
    } else if (st->alpha == 0.0 || st->beta == 0.0) {
        st->done = 1;
        st->stop = 1;
    }
}

// rotations of one LSQR step: uses st->beta (new) and st->red[0] = |v_new|^2
__device__ inline void lsqr_scalars_dev(SolverState *st) {
    if (st->done) return;
    const double alpha_old = st->alpha;
    const double beta = st->beta;
    const double alpha = sqrt(st->red[0]);
    st->anorm2 += alpha_old * alpha_old + beta * beta + st->damp * st->damp;
    const double rhohat = hypot(st->rhobar, st->damp);
    const double c1 = st->rhobar / rhohat, s1 = st->damp / rhohat;
    const double psi = s1 * st->phibar;
    const double phibar1 = c1 * st->phibar;
    const double rho = hypot(rhohat, beta);
    if (!isfinite(rho) || !isfinite(alpha)) {
        st->status = ANOVA_ERR_NOT_FINITE;
        st->done = 1;
        return;
    }
    if (!(rho > 0)) {   // alpha = beta = 0: the Krylov space is exhausted
        st->stop = 1;
        st->done = 1;
        return;
    }
    const double c = rhohat / rho, s = beta / rho;
    const double theta = s * alpha;
    st->rhobar = -c * alpha;
    const double phi = c * phibar1;
    st->phibar = s * phibar1;
    st->phi_rho = phi / rho;
    st->theta_rho = theta / rho;
    st->alpha = alpha;
    st->res2 += psi * psi;   // damped residual: sum of the psi_k^2 so far plus phibar^2
    st->rnorm = sqrt(st->res2 + st->phibar * st->phibar);
    st->arnorm = alpha * fabs(s * phi);
    st->iters += 1;
    if (!isfinite(rho) || !isfinite(phi) || !isfinite(theta)) {
        st->status = ANOVA_ERR_NOT_FINITE;
        st->done = 1;
    }
}

// stopping tests after an LSQR step (st->red[0] = |x|^2 of the scaled unknown)
__device__ inline void lsqr_test_dev(SolverState *st) {
    if (st->done) return;
    const double xnorm = sqrt(st->red[0]);
    const double anorm = sqrt(st->anorm2);
    // breakdown: alpha or beta at the accuracy level of the transforms
    const double tiny = st->tiny_rel * anorm;
    if (st->beta <= tiny || st->alpha <= tiny) {
        st->stop = 1;
        st->done = 1;
    } else if (st->btol > 0 && st->rnorm <= st->btol * st->bnorm + st->atol * anorm * xnorm) {
        st->stop = 2;
        st->done = 1;
    } else if (st->atol > 0 && st->arnorm <= st->atol * anorm * st->rnorm) {
        st->stop = 3;
        st->done = 1;
    } else if (st->iters >= st->max_it) {
        st->stop = 0;
        st->done = 1;
    }
}


// block-wide FP64 sum (result valid in thread 0); blockDim a multiple of 32
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

SolverWork *get_work(Plan &p, int &rc);

__global__ void finish_sums(SolverState *st, const double *part, int nslots);

}  // namespace agft
