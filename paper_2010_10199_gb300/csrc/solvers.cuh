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
    float2 *uM = nullptr, *tM = nullptr, *rM = nullptr;                          // node-sized
    float2 *v = nullptr, *w = nullptr, *x = nullptr, *tn = nullptr, *h = nullptr;  // coefficient-sized
    float2 *f = nullptr, *fp = nullptr, *g = nullptr;
    float *ws = nullptr;          // omega^{-1/2} (LSQR) or omega (FISTA) per coefficient
    double *wd = nullptr;         // omega per coefficient (FP64)
    double *part = nullptr;       // [8][RED_BLOCKS] partial sums
    double *gnorm = nullptr;      // per-group values
    long long *goff = nullptr, *glen = nullptr;
    unsigned char *gmask = nullptr;
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


SolverWork *get_work(Plan &p, int &rc);

__global__ void finish_sums(SolverState *st, const double *part, int nslots);
__global__ void k_residual(const SolverState *st, float2 *r, const float2 *y, long long n, double *part);
__global__ void k_mask_groups(float2 *v, const long long *goff, const long long *glen, const unsigned char *gmask);
__global__ void k_weights(const double *w, float *ws, double *wd, long long n, int mode);
__global__ void k_zero(float2 *v, long long n);

}  // namespace agft
