/*
 * anova_gft.h -- C ABI of the GB300 grouped Fourier transform library.
 *
 * Grouped Fourier transform (Bartel, Potts, Schmischke, "Grouped
 * Transformations and Regularization in High-Dimensional Explainable ANOVA
 * Approximation"):
 *
 *   f_j = sum_{u in U} sum_{k in I_{N_u}^{u,d}} fhat_k exp(+2 pi i <k, x_j>)
 *                                  (Definition "grouped Fourier transform", Sec. 3)
 *   (F^H y)_k = sum_j y_j exp(-2 pi i <k, x_j>)    (stacked adjoint, Sec. 3)
 *
 * computed per ANOVA term u through the low-dimensional identity of eq.
 * (somafm): zero-extend the block fhat(u) to ghat(u), deconvolve by the
 * window's Fourier coefficients, oversampled FFT, and window gather/spread
 * with a Kaiser--Bessel window (the NFFT the paper cites after eq. (somafm)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All pointers named *_dev are DEVICE pointers on the device that was
 *   current when the plan was created; all other pointers are host pointers.
 *   The caller owns every pointer it passes; the library never frees them and
 *   keeps no reference to them after the call returns (the plan copies the
 *   nodes it is given).
 * - Complex vectors are interleaved (re, im).  Their element type follows the
 *   plan's precision: float pairs (anova_cfloat) for ANOVA_PREC_F32,
 *   ANOVA_PREC_BF16 and ANOVA_PREC_F16 (the 16-bit modes only change how the
 *   oversampled grids are stored), double pairs for ANOVA_PREC_F64.
 * - Nodes x are SoA [d][M] (coordinate t of node j at x[t*M + j]) in the
 *   plan's real type, on the torus T = R/Z; values outside [-1/2, 1/2) are
 *   wrapped (a node at exactly 1/2 is the node -1/2).
 * - Terms: term_dims is a host array [n_terms][3] of coordinate ids, each
 *   row ascending and padded with -1 (a row of three -1 is the empty set);
 *   bandwidth[i] is N_u (even, >= 2; ignored for the empty set).  The term
 *   order given here is the coefficient block order.  Inside a block the
 *   multi-index over the term's coordinates is row-major (last coordinate
 *   fastest), each coordinate running -N/2, ..., -1, 1, ..., N/2-1
 *   (I_N minus {0}, Remark "cardinality"); the empty set is the single k = 0
 *   coefficient.  The number of coefficients is sum_u (N_u - 1)^{|u|}.
 * - Work is enqueued on the plan's stream; calls return once the work is
 *   enqueued unless stated otherwise.  Calls on one plan must not overlap.
 * - Every call returns an int status: ANOVA_OK (0) or a negative code below;
 *   anova_status_string() names it.  No exception or longjmp crosses the ABI.
 */
#ifndef ANOVA_GFT_H
#define ANOVA_GFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct anova_plan_s *anova_plan_t;
typedef struct { float re, im; } anova_cfloat;
typedef struct { double re, im; } anova_cdouble;

enum anova_precision {
    ANOVA_PREC_F32 = 0,   /* grids, vectors and accumulation in FP32 */
    ANOVA_PREC_BF16 = 1,  /* grids stored in BF16, FP32 accumulation */
    ANOVA_PREC_F16 = 2,   /* grids stored in FP16, FP32 accumulation */
    ANOVA_PREC_F64 = 3    /* everything in FP64 */
};

/* The orthonormal system of the transform (Remark on other systems, Sec. 3):
 * ANOVA_BASIS_EXP  exp(2 pi i <k, x>) on the torus [-1/2, 1/2)^d, groups
 *                  k_j in I_N minus {0} = {-N/2, .., -1, 1, .., N/2 - 1} (N even);
 * ANOVA_BASIS_COS  the half-period cosine system of Sec. 5 on the cube [0, 1]^d,
 *                  phi_k(x) = sqrt(2)^{|supp k|} prod_{j in supp k} cos(pi k_j x_j),
 *                  groups 1 <= k_j <= N - 1 (any N >= 2), row-major, last axis
 *                  fastest; the empty set is phi_0 = 1.  Nodes outside [0, 1]
 *                  act through the even, 2-periodic extension.  The adjoint is
 *                  g_k = sum_j y_j phi_k(x_j) (real phi_k: no conjugation).
 * Cosine terms are computed on the exponential kernels at the halved nodes x/2
 * with the doubled bandwidth 2N (each cosine coefficient stands for 2^{|u|}
 * mirrored exponential ones), so their oversampled grids are those of an
 * exponential term of bandwidth 2N and the grid limits below apply to 2N
 * (FP32: two-dimensional cosine terms up to N = 24, three-dimensional up to
 * N = 5 at sigma = 2). */
enum anova_basis {
    ANOVA_BASIS_EXP = 0,
    ANOVA_BASIS_COS = 1
};

enum anova_status {
    ANOVA_OK = 0,
    ANOVA_ERR_INVALID = -1,      /* bad argument (null pointer, size, term, bandwidth) */
    ANOVA_ERR_UNSUPPORTED = -2,  /* valid but outside what this build handles (|u| > 3, huge grid) */
    ANOVA_ERR_NOMEM = -3,        /* device or host allocation failed */
    ANOVA_ERR_CUDA = -4,         /* a CUDA call failed; the plan may be unusable */
    ANOVA_ERR_BREAKDOWN = -5,    /* solver breakdown (reported in info, x still valid) */
    ANOVA_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
    ANOVA_ERR_NOT_FINITE = -7    /* a solver scalar became NaN or Inf */
};

/* Options of anova_plan_create; zero-initialise and set what you need. */
typedef struct {
    int precision;      /* enum anova_precision */
    double eps;         /* target relative l2 error of F and F^H (0: default for the precision) */
    int window_m_col;   /* window half-width along the fastest grid axis (0: auto) */
    int window_m_row;   /* window half-width along the other axes (0: auto: 4 for eps below
                           5e-5, which holds every term's block within 1e-5 in FP32; else 3) */
    double sigma;       /* minimal oversampling factor n_u / N_u (0: 2.0) */
    int n_ctas;         /* adjoint: most node chunks (partial grids) per term, <= 64 (0: auto) */
    int node_sort;      /* adjoint: 0 = keep a copy of the nodes sorted by grid cell for every
                           term of order <= 2 when it fits in half the free device memory
                           (16 bytes per node and term); -1 = never */
    int cell_kernel;    /* terms of order <= 2 with sorted nodes: 0 = the per-cell products on
                           the tensor cores (operands split into two TF32 parts, three
                           products, FP32 sums): the adjoint spread of FP32, FP16 and BF16
                           plans, and the forward gather of FP32 plans without third-order
                           terms; 1 = on the CUDA cores (FP32) */
    int basis;          /* enum anova_basis (0: the exponential system) */
} anova_plan_options;

/*
 * anova_plan_create -- build the term table, grids and window tables for a
 * fixed node set (Sec. 3: the grouped index set of eq. (groupedset) and the
 * block order of eq. (bananarama)).
 *   out        : receives the plan handle (host pointer, required)
 *   d          : spatial dimension, 1 <= d
 *   M          : number of nodes, 0 <= M < 2^31
 *   x_dev      : nodes [d][M] (device, plan's real type); copied into the plan
 *   n_terms    : number of terms, >= 1
 *   term_dims  : host [n_terms][3], see conventions
 *   bandwidth  : host [n_terms], even N_u >= 2 for non-empty terms
 *   opts       : host, may be NULL for defaults (FP32, eps 1e-5)
 *   stream     : cudaStream_t used by every later call on this plan (NULL = legacy default)
 * Errors: ANOVA_ERR_INVALID for bad sizes/terms, ANOVA_ERR_UNSUPPORTED for
 * |u| > 3 or a grid that does not fit the kernels (two copies of the
 * n_u^{|u|} FFT array in shared memory: 200 KB, i.e. 3-D terms up to n = 23
 * in FP32 and n = 18 in FP64; one stored grid of at most 100 KB, FP64 200 KB),
 * ANOVA_ERR_NOMEM.  FP64 plans also precompute window tables of
 * 68 bytes per node for every (window, coordinate) pair in use.
 * Synchronises the stream before returning.
 */
int anova_plan_create(anova_plan_t *out, int d, int64_t M, const void *x_dev, int n_terms,
                      const int32_t *term_dims, const int32_t *bandwidth,
                      const anova_plan_options *opts, void *stream);

/* Release the plan and all device memory it owns.  NULL is a no-op. */
void anova_plan_destroy(anova_plan_t plan);

/* Number of coefficients |I_N(U)| = sum_u (N_u - 1)^{|u|} (Remark "cardinality"); -1 for NULL. */
int64_t anova_num_coeffs(anova_plan_t plan);

/* Offset and length of block u in the coefficient vector. */
int anova_term_offset(anova_plan_t plan, int u, int64_t *off, int64_t *len);

/* Oversampled grid size n_u and window half-widths (col, row) chosen for term u. */
int anova_term_grid(anova_plan_t plan, int u, int *n, int *m_col, int *m_row);

/*
 * grouped_trafo -- f = F(X, I_N(U)) fhat  (Definition "grouped Fourier
 * transform" and eq. (somafm), Sec. 3).
 *   fhat_dev : [num_coeffs] complex (plan's vector type), read only
 *   f_dev    : [M] complex, overwritten
 * The two buffers must not overlap.  Accuracy: relative l2 error against the
 * exact sum near the plan's eps (FP32 plans: about 3e-6 at the default eps
 * 1e-5).  FP32 plans with sorted nodes sum every node's terms in 64-bit fixed
 * point, so the result is bitwise reproducible for a plan.  FP32 plans need
 * the oversampled grid values (about sum_k |fhat_k| at most) below 2^114
 * (2e34) in magnitude: the tensor-core kernels split each operand x into two
 * TF32 parts through 8193 x, which must stay finite.
 */
int grouped_trafo(anova_plan_t plan, const void *fhat_dev, void *f_dev);

/*
 * grouped_adjoint -- fhat = F(X, I_N(U))^H y  (stacked adjoint after the
 * error remark, Sec. 3).
 *   y_dev    : [M] complex, read only
 *   fhat_dev : [num_coeffs] complex, overwritten
 * Accuracy as for grouped_trafo (FP32 plans: about 5e-6 at the default eps),
 * whichever cell_kernel the plan uses.  The order of the shared-memory float
 * additions inside a CTA is not fixed, so repeated calls may differ at the
 * rounding level.  FP32 plans need |y_j| below 2^114 (2e34), as for
 * grouped_trafo.
 */
int grouped_adjoint(anova_plan_t plan, const void *y_dev, void *fhat_dev);

/* Summary of a solve; fields a solver does not use are zero. */
typedef struct {
    int iterations;        /* iterations run (last lambda for paths) */
    int status;            /* 0 ok, or an anova_status code (breakdown, not finite, ...) */
    int stop_reason;       /* LSQR: 0 max_it, 1 breakdown, 2 residual test, 3 normal-eq test;
                              FISTA: 0 max_it, 1 step tolerance */
    int n_trafo;           /* grouped_trafo applications */
    int n_adjoint;         /* grouped_adjoint applications */
    int active_groups;     /* FISTA: groups with f_u != 0 at the end */
    double rnorm;          /* LSQR: estimate of sqrt(||y - F f||^2 + 2 lam ||f||_W^2); FISTA: ||y - F f|| */
    double arnorm;         /* LSQR: estimate of the normal-equation residual */
    double objective;      /* FISTA: 1/2 ||y - F f||^2 + lam sum_u ||f_u||_W */
    double L;              /* FISTA: final step constant */
    double seconds;        /* device time of the solve (CUDA events) */
} anova_solve_info;

/*
 * lsqr_solve -- minimiser of 1/2 ||y - F f||^2 + lambda f^H W f
 * (eq. (new_min_prob), Sec. 4.1) by LSQR (Paige and Saunders 1982) on
 * A = F W^{-1/2} with damping sqrt(2 lambda), started from f = 0.
 * The regulariser of eq. (new_min_prob) has no factor 1/2, hence sqrt(2 lambda).
 *   y_dev      : [M] complex
 *   w_dev      : [num_coeffs] double weights omega_k >= 1 (W = diag(omega)), or NULL for W = I
 *   lambda     : >= 0
 *   max_it     : iteration cap (>= 1)
 *   atol, btol : Paige--Saunders stopping tolerances (0 disables the tests)
 *   fhat_dev   : [num_coeffs] complex, overwritten with the solution
 *   info       : host, may be NULL
 * Vector updates run in the plan's precision; the bidiagonalisation scalars
 * (alpha, beta, rho, phi, c, s, norms) are FP64 on the device.  The iteration
 * is driven on the device (no host round trip per iteration); the call
 * returns after the solve has finished.
 */
int lsqr_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, double lambda,
               int max_it, double atol, double btol, void *fhat_dev, anova_solve_info *info);

/*
 * fista_solve -- group lasso min 1/2 ||y - F f||^2 + lambda sum_u ||f_u||_{W_u}
 * (eq. (alligatoah), Sec. 4.2) by Algorithm "FISTA for group lasso" along a
 * warm-started lambda path (largest first, f_0 = 0 or fhat_path_dev[0] on entry
 * when warm_start is set).
 *   y_dev        : [M] complex
 *   w_dev        : [num_coeffs] double weights, or NULL for W = I
 *   lambdas      : host [n_lambda], any order (solved largest first)
 *   max_it, tol  : per lambda; stop when ||f_k - f_{k-1}|| <= tol ||f_k||.  FP32 plans
 *                  resolve relative changes down to about 1e-7 (their rounding
 *                  level); below that the iterates may cycle at the rounding level
 *                  and a smaller tol then runs to max_it
 *   step_mode    : 0 constant step L (Remark after the Algorithm), 1 backtracking
 *   L0, eta      : step constant (constant mode: L; backtracking: L_0) and eta > 1;
 *                  L0 <= 0 asks for 1.08 times a Lanczos (Golub-Kahan) estimate of ||F||^2
 *                  over the allowed groups (stopped when a step changes it by less than
 *                  1e-3 relative, after 8 to 60 transform pairs)
 *   group_mask   : host [n_terms] uint8, 1 = group may be nonzero; NULL = all groups
 *   fhat_path_dev: [n_lambda][num_coeffs] complex, solution per lambda in the
 *                  order lambdas are given
 *   info         : host [n_lambda] (may be NULL)
 */
int fista_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, const double *lambdas,
                int n_lambda, int max_it, double tol, int step_mode, double L0, double eta,
                const uint8_t *group_mask, int warm_start, void *fhat_path_dev,
                anova_solve_info *info);

/*
 * anova_kkt_check -- optimality of a group-lasso solution of eq. (alligatoah).
 * With r = y - F f: an inactive group (f_u = 0) must satisfy
 * ||W^{-1/2} (F^H r)_u|| <= lambda (Lemma (iii)); an active group must satisfy
 * (F^H r)_u = lambda W f_u / ||f_u||_W (stationarity in the proof of Lemma (ii)).
 *   fhat_dev : [num_coeffs] complex, the candidate solution
 *   viol_out : host [n_terms] (may be NULL): (||W^{-1/2} q_u|| - lambda)/lambda for
 *              inactive groups, ||(F^H r)_u - lambda W f_u/||f_u||_W|| / lambda for active ones
 *   n_viol   : host, number of groups with viol > rtol
 * One grouped_trafo and one grouped_adjoint over all terms; synchronises.
 */
int anova_kkt_check(anova_plan_t plan, const void *y_dev, const double *w_dev, const void *fhat_dev,
                    double lambda, double rtol, double *viol_out, int *n_viol);

/*
 * anova_sobol_indices -- global sensitivity (Sobol) indices of the partial sum
 * S f = sum_u sum_{k in I_u} fhat_k exp(2 pi i <k, x>) (eq. (gsi), Sec. 2):
 * rho(u) = sigma^2(f_u) / sigma^2(f) with sigma^2(f_u) = ||fhat_u||^2 (the
 * blocks are orthogonal on the torus: Parseval) and sigma^2(f) = ||f||^2 -
 * |c_0|^2, the sum over the non-empty terms; rho(empty set) = 0 (and every
 * rho is 0 when all non-empty blocks vanish).  With thresholds it also returns
 * the active set of eq. (activeset), Sec. 4:
 * U* = {empty set} u {u : rho(u) > eps_|u|} (strict inequality).
 *   fhat_dev     : [num_coeffs] complex (plan's vector type)
 *   rho_out      : host [n_terms] (required), in the user's term order
 *   eps_by_order : host [3] thresholds eps_1, eps_2, eps_3 >= 0, or NULL
 *   active_out   : host [n_terms], 1 for u in U* (required with eps_by_order)
 * Block energies and their total are FP64 sums in a fixed order on the device.
 * Synchronises the plan's stream.
 */
int anova_sobol_indices(anova_plan_t plan, const void *fhat_dev, double *rho_out, const double *eps_by_order,
                        uint8_t *active_out);

/*
 * anova_l2_error -- relative L2 error of eq. (L2error), Sec. 4, of the partial
 * sum with coefficients fhat against a function f whose Fourier coefficients
 * c on I_N(U) and squared norm ||f||^2 are known, through Parseval's identity:
 *   err = sqrt(max(0, ||f||^2 + sum_I |fhat_k - c_k|^2 - sum_I |c_k|^2) / ||f||^2).
 *   fhat_dev, c_dev : [num_coeffs] complex (plan's vector type)
 *   norm2           : ||f||^2 > 0
 *   err_out         : host
 * FP64 sums in a fixed order on the device; synchronises the plan's stream.
 */
int anova_l2_error(anova_plan_t plan, const void *fhat_dev, const void *c_dev, double norm2, double *err_out);

/* ------------------------------------------------------------------------
 * Many independent problems in one launch per kernel.  A batch holds one
 * plan per problem (same options); its vectors are the concatenation of the
 * problems' vectors (problem p's nodes at node_off[p] .. node_off[p+1], its
 * coefficients at coef_off[p] .. coef_off[p+1]).  Every problem needs at
 * least one non-empty term.  The problems are independent as the terms are
 * (Sec. 3, after eq. (somafm)); each kernel runs once for all of them.
 * ------------------------------------------------------------------------ */
typedef struct anova_batch_s *anova_batch_t;

/* x_dev[p]: device nodes [d[p]][M[p]] of problem p; term_dims[p] / bandwidth[p]
 * as for anova_plan_create.  Synchronises `stream`. */
int anova_batch_create(anova_batch_t *out, int n_problems, const int *d, const int64_t *M,
                       const float *const *x_dev, const int *n_terms, const int32_t *const *term_dims,
                       const int32_t *const *bandwidth, const anova_plan_options *opts, void *stream);
void anova_batch_destroy(anova_batch_t batch);
/* node_off / coef_off: host arrays of n_problems + 1 entries (either may be NULL). */
int anova_batch_layout(anova_batch_t batch, int64_t *node_off, int64_t *coef_off);
/* f = F fhat for every problem (concatenated vectors, FP32 complex). */
int grouped_trafo_batch(anova_batch_t batch, const void *fhat_dev, void *f_dev);
/* fhat = F^H y for every problem. */
int grouped_adjoint_batch(anova_batch_t batch, const void *y_dev, void *fhat_dev);
/* One Tikhonov LSQR (eq. (new_min_prob), W = I, damping sqrt(2 lambda)) per
 * problem, all in the same launches, each with its own FP64 scalars and
 * stopping tests; info: host [n_problems] (may be NULL).  Synchronises. */
int lsqr_solve_batch(anova_batch_t batch, const void *y_dev, double lambda, int max_it, void *fhat_dev,
                     anova_solve_info *info);

/* ------------------------------------------------------------------------
 * Learned group screening (no counterpart in the paper).  A two-hidden-layer
 * MLP (ReLU, sigmoid output, FP32) proposes, along a group-lasso lambda path,
 * which groups will be nonzero; fista_screened_path verifies every proposal
 * with the full KKT conditions, so the network changes only the work done.
 * ------------------------------------------------------------------------ */
typedef struct anova_mlp_s *anova_mlp_t;

/* Create a network with n_features inputs and two hidden layers of `hidden`
 * units from initial parameters (host, FP32, packed W1[F][H] | b1[H] |
 * W2[H][H] | b2[H] | W3[H] | b3[1], row-major).  Work runs on `stream`. */
int anova_mlp_create(anova_mlp_t *out, int n_features, int hidden, const float *params_host, void *stream);
void anova_mlp_destroy(anova_mlp_t mlp);
int64_t anova_mlp_num_params(anova_mlp_t mlp);
/* Copy the current parameters and the last computed gradients (either may be NULL); synchronises. */
int anova_mlp_get_params(anova_mlp_t mlp, float *params_host, float *grads_host);
/* prob_dev[g] = sigmoid(z_g) for the G feature rows X_dev [G][n_features] (device). */
int anova_mlp_forward(anova_mlp_t mlp, const float *X_dev, int G, float *prob_dev);
/* Forward + backward of the positive-weighted binary cross-entropy on logits,
 * loss = mean_g [pw y_g softplus(-z_g) + (1 - y_g) softplus(z_g)], labels y_dev [G]
 * in {0, 1}; gradients are kept for anova_mlp_get_params; *loss_out gets the loss. */
int anova_mlp_gradients(anova_mlp_t mlp, const float *X_dev, const float *y_dev, int G, float pos_weight,
                        double *loss_out);
/* Adam (beta1 0.9, beta2 0.999, eps 1e-8) over `epochs` passes of consecutive
 * mini-batches of `batch` rows; loss_history (host, may be NULL) gets the mean
 * loss per epoch. */
int anova_mlp_train(anova_mlp_t mlp, const float *X_dev, const float *y_dev, int n_samples, int batch, int epochs,
                    float lr, float pos_weight, double *loss_history);

/* Screening features of every group (device X_dev [n_terms][7]) for the step
 * lambda_prev -> lambda at the solution fhat_dev of lambda_prev (one
 * grouped_trafo and one grouped_adjoint over all terms); see screen.cu. */
int anova_screen_features(anova_plan_t plan, const void *y_dev, const double *w_dev, const void *fhat_dev,
                          double lambda, double lambda_prev, float *X_dev);

typedef struct {
    int64_t proposed_groups;      /* groups the network (or a nonzero warm start) proposed, summed over lambdas */
    int64_t readmitted_groups;    /* groups added back by the KKT check */
    int64_t rounds;               /* FISTA solves (proposal + re-admission rounds) */
    int64_t term_iterations;      /* sum over FISTA iterations of the terms transformed */
    int64_t full_term_iterations; /* the same iterations times all terms (work without screening) */
    double seconds;               /* wall time of the path */
} anova_screen_stats;

/* Group-lasso path (eq. (alligatoah)) with learned screening: per lambda
 * (largest first, warm started) propose groups with prob > threshold (plus
 * groups nonzero at the previous lambda and the empty set), run constant-step
 * FISTA with the transforms restricted to them, then re-admit every held-out
 * group whose KKT score ||W^{-1/2} (F^H r)_u|| exceeds lambda (1 + kkt_tol) and
 * re-solve until none does.  Output layout and tol as fista_solve. */
int fista_screened_path(anova_plan_t plan, anova_mlp_t mlp, const void *y_dev, const double *w_dev,
                        const double *lambdas, int n_lambda, int max_it, double tol, double threshold,
                        double kkt_tol, void *fhat_path_dev, anova_solve_info *info, anova_screen_stats *stats);

/*
 * Per-kernel timing (no counterpart in the paper; measurement support).
 * anova_profile_enable(plan, 1) makes every later call record CUDA events on
 * the plan's stream around each kernel it launches; anova_profile_read
 * synchronises the stream and returns, for each stage s < *n_stages, the
 * summed device milliseconds ms[s] and launch count launches[s] since the last
 * reset (reset = 1 clears them after reading).  Stages:
 *   0 trafo_pre (deconvolve + FFT), 1 gather, 2 spread, 3 reduce_partials,
 *   4 adjoint_post (fold + FFT + deconvolve), 5 empty-set sum, 6 solver vector ops
 * name_out (may be NULL) receives a static name per stage.
 */
int anova_profile_enable(anova_plan_t plan, int on);
int anova_profile_read(anova_plan_t plan, double *ms, int64_t *launches, const char **names, int max_stages,
                       int *n_stages, int reset);

/*
 * anova_plan_autotune -- choose plan options for one node set and term list
 * by measurement (the NFFT's error falls as the window widens and the
 * oversampling grows, Sec. 3 after eq. (somafm); its cost rises with both).
 * A reference plan (sigma 2.5, 8 x 8 taps) transforms two fixed pseudo-random
 * vectors; every candidate plan transforms the same vectors, its estimated
 * error is the largest relative l2 distance to the reference of F fhat, of
 * F^H y and of each coefficient block of F^H y on its own, and its time is
 * the mean of `reps` timed pairs after one warm-up pair on `stream`.
 * Candidates: sigma in {1.75, 2, 2.5} x row half-width in {3, 4}; then, around
 * the fastest one within eps_target, node chunks per term (n_ctas) in
 * {4, 16, 64}, the original node order (node_sort = -1) and the CUDA-core
 * cell kernels (cell_kernel = 1).
 *   opts       : in: base options (precision must be ANOVA_PREC_F32);
 *                out: the fastest candidate with est_error <= eps_target
 *   d .. bandwidth : as for anova_plan_create
 *   trials     : host array [max_trials] receiving every candidate tried
 *                (ms_pair and est_error are INFINITY for one that could not
 *                be built), in order; *n_trials gets the count (may be NULL)
 * Errors: ANOVA_ERR_INVALID, ANOVA_ERR_UNSUPPORTED (not FP32, or no candidate
 * met eps_target), errors of anova_plan_create.  Creates and destroys plans
 * (device allocations); synchronises the stream.  The paper has no tuner.
 */
typedef struct {
    double sigma;
    int window_m_row;
    int n_ctas;
    int node_sort;
    int cell_kernel;
    double ms_pair;    /* mean time of one forward + adjoint pair */
    double est_error;  /* estimated relative l2 error against the reference plan */
    int chosen;        /* 1 for the candidate written to opts */
} anova_tune_trial;

int anova_plan_autotune(anova_plan_options *opts, int d, int64_t M, const void *x_dev, int n_terms,
                        const int32_t *term_dims, const int32_t *bandwidth, double eps_target, int reps,
                        anova_tune_trial *trials, int max_trials, int *n_trials, void *stream);

/*
 * grouped_trafo_noalloc -- f = F(X, I_N(U)) fhat without a plan and without
 * allocating anything.  The paper has no counterpart: this is a deployment
 * variant of grouped_trafo for callers that cannot allocate device memory when
 * they need the transform -- for example a host program whose device memory is
 * already fully reserved by its own pool allocator, a plug-in that runs inside
 * a callback with a fixed memory budget, or a latency-critical loop in which
 * cudaMalloc/cudaFree (which synchronise the device) are not allowed.
 *
 * It computes what grouped_trafo computes with default options (FP32,
 * eps 1e-5, sigma 2) for the same arguments as anova_plan_create plus the
 * vectors.  All working data -- term table, window polynomials,
 * deconvolution factors, a wrapped copy of the nodes and the oversampled grids
 * -- lives in one file-scope device array of 32 MiB that every GPU loading
 * the library keeps until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   x_dev    : [d][M] FP32 nodes (device), read only
 *   fhat_dev : [num_coeffs] complex FP32 (device), read only
 *   f_dev    : [M] complex FP32 (device), overwritten
 *   stream   : cudaStream_t for all work (NULL = legacy default stream)
 * Limits: the tables plus 4*d*M bytes of nodes plus the grids must fit in
 * the 32 MiB array (at d = 20 and the |u| <= 2, N = 64/32 term set this
 * allows M up to about 300,000); larger problems return ANOVA_ERR_UNSUPPORTED
 * without launching anything.  At most 4096 terms.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Every call reuses the same array and overwrites the
 * previous call's contents, so calls that can overlap on the GPU (different
 * streams or devices sharing a context, or host threads) race: serialise them.
 * A call on a stream that is capturing returns ANOVA_ERR_UNSUPPORTED and
 * enqueues nothing: its table uploads read host staging memory that the next
 * call overwrites.  An error left pending by earlier, unrelated work is
 * cleared at entry, not reported.
 * Returns after enqueueing the work.
 */
int grouped_trafo_noalloc(int d, int64_t M, const float *x_dev, int n_terms, const int32_t *term_dims,
                          const int32_t *bandwidth, const anova_cfloat *fhat_dev, anova_cfloat *f_dev,
                          void *stream);

/*
 * anova_debug_fail_allocation -- fault injection for tests (no counterpart in
 * the paper).  After a call with k > 0, the k-th following device or host
 * allocation made by anova_plan_create (or by the first solver call on a plan,
 * which creates the solver workspace) fails as if the device or host were out
 * of memory; the allocations after it succeed again.  k = 0 cancels a pending
 * failure.  A failing plan creation returns ANOVA_ERR_NOMEM after freeing
 * everything it had allocated, or -- where the failed allocation was an
 * optional one (the cell-sorted node copy, the fixed-point accumulators) --
 * builds the plan without it.  Process-wide; not for concurrent use.
 * Errors: ANOVA_ERR_INVALID for k < 0.
 */
int anova_debug_fail_allocation(int k);

/* Human-readable name of a status code (static string). */
const char *anova_status_string(int status);

/* Library version string. */
const char *anova_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ANOVA_GFT_H */
