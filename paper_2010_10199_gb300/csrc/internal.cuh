// Internal definitions shared by the CUDA translation units of the library.
//
// Method: grouped Fourier transform of Sec. 3 (Definition "grouped Fourier
// transform", identity eq. (somafm), stacked adjoint), evaluated per ANOVA term
// with an NFFT: deconvolution by the window's Fourier coefficients, an
// oversampled FFT, and a Kaiser--Bessel window gather (forward) or spread
// (adjoint).  The window is
//     psi(d) = sinh(b sqrt(m^2 - d^2)) / (pi sqrt(m^2 - d^2)),  |d| <= m,
// in grid units d = n x - q, with b = pi (2 - 1/sigma), sigma = n/N, and
// Fourier transform (1/n) I_0(m sqrt(b^2 - (2 pi k / n)^2)) of psi(n x).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <new>

#include "anova_gft.h"

namespace agft {

constexpr int MAX_ORDER = 3;
constexpr int MAXM = 8;          // largest window half-width
constexpr int NCOEF = 8;         // coefficients of the per-tap polynomial (degree 7)
constexpr int GATHER_TILE = 128;   // nodes per gather tile (gather.cu)
constexpr int SPREAD_THREADS = 256;
constexpr int SPREAD_MAX_CTAS_PER_SM = 4;
constexpr int SPREAD_MAX_K = 64;     // largest number of node chunks (partial grids) per term
constexpr int MAX_SMEM = 227 * 1024;

// One window shape (half-width m, oversampling sigma).  Tap j of a node with
// grid position t = n x sits at grid index floor(t) - m + 1 + j and has weight
// psi(tau + m - 1 - j) / psi(0), tau = t - floor(t); the weight is stored as a
// degree-7 polynomial in v = 2 tau - 1 (Chebyshev interpolation, monomial form).
// The same polynomial in the Chebyshev basis: tap j = sum_i ch[j][i] X_i(v) with
// X_i = s_i T_i, signs s = (+, +, -, -, +, +, -, -), which turn the three-term
// recurrence into X_{i+1} = X_{i-1} + (-1)^i 2 v X_i (one fma per step).
struct Window {
    float c[2 * MAXM][NCOEF];
    float ch[2 * MAXM][NCOEF];
    int m;
    float b;          // shape parameter pi (2 - 1/sigma)
    float inv_psi0;   // 1 / psi(0)
    double bd, inv_psi0d;
};

// A term in kernel schedule order.  Grid layout: erows x stride (complex
// elements), the last coordinate of the term along a row.  Orders 1 and 2
// store halos so that a window never wraps: periodic column q sits at stored
// column q + hc (hc = m_col - 1) and the stored columns q + hc +- n repeat it;
// order-2 rows likewise with hr = m_row - 1.  Order-3 grids have no halo: the
// row index is i_first * n + i_second and all indices wrap modulo n.  The row
// stride is = 8 (mod 16) complex elements, so two consecutive rows of eight
// columns fall in complementary shared-memory bank halves.
struct Term {
    int order;          // 1..3 (the empty set is handled separately)
    int col;            // coordinate along the row
    int row0, row1;     // other coordinates (-1 if absent)
    int N, n, stride;
    int rows;           // n^(order-1)
    int wc, wr;         // window ids: column axis, row axes
    int mc, mr;         // their half-widths
    int new_rowgroup;   // 1 if the row weights cached by the gather must be recomputed
    int hr, hc;         // halo widths (rows, columns): stored index = periodic index + halo
    int erows;          // stored rows (order 2: n + 2 hr + 1; order 1: 1; order 3: n^2, no halo)
    int sort_slot;      // slot of this term's cell-sorted node copy (-1: none)
    long long grid_off;   // element offset in the grid buffer
    long long grid_bytes; // bytes (multiple of 16)
    long long coef_off;   // offset in the coefficient vector
    long long coef_len;
    int dc_off, dr_off;   // offsets of the column / row deconvolution factors
    int user_index;
    int slot_c;           // FP64 plans: window-table slots of the column and row coordinates
    int slot_r0, slot_r1;
    int basis;            // ANOVA_BASIS_EXP, or ANOVA_BASIS_COS (N above is then the doubled bandwidth)
};

// What the forward gather needs of an active term, in one 48-byte record
// (prefetched by every warp one term ahead).
struct ActRec {
    int order, newgroup;   // newgroup: 1 if the row weights must be recomputed
    int wc, wr;            // window ids (column axis, row axes)
    int col, row0, n, stride;
    long long grid_off;
    int grid_bytes, term;  // term: index into the term table
};

inline ActRec make_act_rec(const Term &T, int term, int newgroup) {
    ActRec a;
    a.order = T.order;
    a.newgroup = newgroup;
    a.wc = T.wc;
    a.wr = T.wr;
    a.col = T.col;
    a.row0 = T.row0;
    a.n = T.n;
    a.stride = T.stride;
    a.grid_off = T.grid_off;
    a.grid_bytes = (int)T.grid_bytes;
    a.term = term;
    return a;
}

// A node in the cell order of one term (16 bytes, stored as float4):
//   x: 2 tau_row - 1 (order 2; 0 for order 1), y: 2 tau_col - 1, the window
//   polynomial arguments of the node's fractional grid positions;
//   z (int bits): stored-grid offset of the first tap, i_row * stride + i_col
//   (order 1: i_col), which identifies the cell;
//   w (int bits): the node's original index.
// Built in sort.cu by the same FP32 operations the unsorted kernels apply.

// Device-visible view of a plan (passed by value to kernels).
struct DevPlan {
    int d;
    long long M;
    int n_terms;              // scheduled (non-empty) terms
    int n_empty;              // empty-set terms
    const float *x;           // [d][M] FP32 nodes (or null)
    const double *xd;         // [d][M] FP64 nodes (or null)
    const Term *terms;
    const Window *windows;
    const float *deconv;      // deconvolution factors
    const double *deconvd;
    const long long *empty_off;  // coefficient offsets of the empty terms
    long long grid_elems;     // total grid elements (complex)
    long long max_grid_bytes;
    int *err;                 // device error word (bounded waits)
    const int *act;           // active schedule: indices into terms, n_act entries
    const ActRec *act_rec;    // per active entry: the gather's view of the term
    int n_act;
    const int *skip;          // if non-null and nonzero, kernels return at once
    const float2 *grids;      // stored grids of this problem
    float2 *partials;         // adjoint partial grids [spread_chunks][grid_elems]
    int spread_chunks;        // node chunks of the adjoint (one partial grid each)
    const float4 *srec;       // [slot][M] nodes sorted by grid cell, see SortedNode
    unsigned long long *facc; // sorted forward: fixed-point accumulators [M][2] (or null)
    int *fexp;                // and their exponent
    long long n_coeffs;
    long long vec_node_off;   // offset of this problem's nodes in batched node vectors
    long long vec_coef_off;   // offset of this problem's coefficients in batched coefficient vectors
    int basis;                // ANOVA_BASIS_EXP or ANOVA_BASIS_COS
};

// Work lists of a launch over several problems (a batch).  With plans == null
// the launch covers the single problem given by the DevPlan parameter and
// every table below is unused.
struct BatchArgs {
    const DevPlan *plans;     // device array [P]
    int P;
    const int *tile_prob;     // gather: problem of each tile of 128 nodes
    const int *tile0;         // first tile of each problem
    const int4 *items;        // spread work items (problem, active term, node chunk, chunks)
    const int *blk_prob;      // pre/post: problem of each (problem, active term) block
    const int *blk0;          // first block of each problem
};

constexpr int N_STAGES = 7;
struct Profiler;   // per-stage CUDA-event timing (profile.cu)

struct Plan {
    Profiler *prof;
    int device;
    cudaStream_t stream;
    int precision;
    int basis;              // ANOVA_BASIS_EXP or ANOVA_BASIS_COS
    double eps;             // target relative error of the transforms
    int d;
    long long M;
    int n_user_terms;
    long long n_coeffs;
    // host copies
    Term *h_terms;
    int n_terms;
    int n_empty;
    long long *h_user_off;  // per user term: coefficient offset
    long long *h_user_len;
    int *h_user_n, *h_user_mc, *h_user_mr, *h_user_order;
    // device buffers
    void *x;                // FP32 or FP64 nodes [d][M]
    Term *terms;
    Window *windows;
    int n_windows;
    float *deconv;
    double *deconvd;
    long long *empty_off;
    void *grids;            // complex grid buffer (precision dependent)
    long long grid_elems;
    long long max_grid_bytes;
    int max_fft_elems;      // largest n^order
    int pitch2;             // row pitch shared by all order-2 grids
    // active term list (all scheduled terms unless a group mask restricts it)
    int *act;
    ActRec *act_rec;
    ActRec *act_rec3;       // active third-order terms without sorted records (point-major gather)
    int n_act3;
    int n_act;
    int *h_act;
    const int *skip;        // device flag read by every transform kernel (or null)
    void *partials;         // adjoint partial grids [spread_kmax][grid_elems]
    int spread_kmax;        // partial grids allocated (largest chunk count per term)
    int spread_K;           // node chunks per term for the current active list
    int4 *items;            // spread work items (device, n_terms * spread_kmax slots)
    int4 *h_items;
    int n_items;
    int n_items3;           // the first n_items3 items are those of third-order terms
    int *counter;           // work-queue counter of the spread
    float4 *srec;           // cell-sorted node records (null: none), n_sorted slots of M
    bool cell_tc;           // order-1/2 spread of sorted records on the tensor cores
    int n_sorted;
    unsigned long long *facc;   // sorted forward: fixed-point accumulators [M][2]
    int *fexp;              // and their exponent
    // FP64 plans: window weights per (window, coordinate) slot and node, the
    // precomputed form of psi (taps 0..2m-1, zero padded to 8), and the first
    // tap's grid index floor(n x + n/2) in [0, n)
    double *wt64;           // [n_slots][M][8]
    int *wb64;              // [n_slots][M]
    int4 *slots64;          // per slot: (window id, coordinate, n, m)
    int n_slots64;
    int gather_ctas;
    int *err;
    void *scratch;          // reduction scratch
    size_t scratch_bytes;
    int sm_count;
    void *solver;           // solver workspaces (solvers.cu), created on first use
    void (*solver_free)(void *);
};

DevPlan dev_view(const Plan &p);
int set_active_terms(Plan &p, const unsigned char *user_mask);
inline cudaError_t cuda_err_of(int status) {
    return status == ANOVA_OK ? cudaSuccess : status == ANOVA_ERR_NOMEM ? cudaErrorMemoryAllocation : cudaErrorUnknown;
}

// Allocations of plan construction and of the solver workspaces go through
// these two, so that a test can make the k-th of them fail the way an
// exhausted device or host would (anova_debug_fail_allocation).
bool alloc_fault();
cudaError_t plan_malloc_raw(void **ptr, size_t bytes);
template <typename T>
inline cudaError_t plan_malloc(T **ptr, size_t bytes) {
    return plan_malloc_raw((void **)ptr, bytes);
}
template <typename T>
inline T *plan_new(size_t n) {
    return alloc_fault() ? nullptr : new (std::nothrow) T[n];
}

// host-side table builders shared with plan construction (plan.cu)
double deconv_factor(int k, int n, int m, double b);
void window_polys(Window &w, int m, double b);
int fft_size(int N, double sigma);
int row_stride(int n);
// out = in * scale wrapped into [-1/2, 1/2) (scale 1/2 for cosine plans: x in [0, 1] -> x / 2)
__global__ void wrap_nodes_f32(const float *in, float *out, long long total, float scale);

// stage timing: call stage_begin before and stage_end after a kernel launch
void stage_begin(Plan &p, int stage);
void stage_end(Plan &p, int stage);
void profiler_free(Plan &p);
enum { ST_PRE = 0, ST_GATHER = 1, ST_SPREAD = 2, ST_REDUCE = 3, ST_POST = 4, ST_SUMY = 5, ST_SOLVER = 6 };

// kernels launched by the entry points (trafo.cu / adjoint.cu)
int launch_trafo_f32(Plan &p, const float2 *fhat, float2 *f);
int launch_gather_f32(Plan &p, const float2 *fhat, float2 *f);
// Sorted forward (gather_sorted.cu): order-1/2 terms over the cell-sorted
// records, accumulated into f with atomics; f must hold the other terms' sum.
int launch_gather_sorted_f32(Plan &p, const float2 *fhat, float2 *f);
// The same for one problem (B.plans == null) or a batch of P problems, every one
// with records and accumulators: f = empty-set coefficient + all terms.
// Sorted forward of one problem or a batch: fixed-point passes around the
// gather of items [0, item_end); the first n_items3 are third-order items;
// with tc and none of those, the gather runs on the tensor cores.
int gather_sorted_launch(cudaStream_t st, const DevPlan &v, const BatchArgs &B, int P, const float2 *fhat,
                         float2 *f, const int4 *items, int n_items3, int item_end, int *counter,
                         long long max_grid_bytes, long long max_M, int sm_count, int mr, double *part, bool tc);
int launch_adjoint_f32(Plan &p, const float2 *y, float2 *fhat);
int adjoint_launch(Plan *prof, cudaStream_t st, const DevPlan &v, const BatchArgs &B, int P, const float2 *y,
                   float2 *fhat, int n_items, int n_items3, int *counter, int n_blocks, int mr,
                   long long max_grid_bytes, int max_fft_elems, int sm_count, long long max_grid_elems,
                   bool any_empty, double2 *scratch, int prec, bool tc);
size_t spread_smem_bytes(long long max_grid_bytes, bool o3, int sp);
int spread_block_nodes(long long max_grid_bytes);
// Sorts the nodes by grid cell for every term with sort_slot >= 0 (sort.cu).
int sort_nodes_by_cell(Plan &p);
// FP64 path (f64.cu): window tables, forward and adjoint transforms.
int build_window_tables_f64(Plan &p);
int launch_trafo_f64(Plan &p, const double2 *fhat, double2 *f);
int launch_adjoint_f64(Plan &p, const double2 *y, double2 *fhat);
// CTAs per SM of the order-1/2 spread kernel (tc: the tensor-core one)
int spread_ctas_per_sm(long long max_grid_bytes, bool tc);
// Node chunks per term for a spread over n_act_total active terms (all
// problems of a launch) on sm_count SMs: about three items per resident
// spread CTA (with third-order terms, order3, per CTA of 3 per SM at least),
// at most kmax, at least 2048 nodes per chunk.
int spread_chunks_for(long long M, int n_act_total, int kmax, long long max_grid_bytes, int sm_count, bool tc,
                      bool order3);
// Appends the spread work items of one problem, K chunks per active term:
// those of the third-order terms (sel = 3) or of the others, order 2 before
// order 1 (sel = 0).  Returns the count.
int append_spread_items(const Plan &p, int prob, int K, int4 *out, int sel);
int lipschitz_estimate(Plan &p, double *L);
int fista_impl(Plan &p, const float2 *y, const double *w, const double *lambdas, int n_lambda, int max_it,
               double tol, int step_mode, double L0, double eta, const uint8_t *mask, const float2 *f0,
               float2 *path, anova_solve_info *info, double *L_out);

// Runs `set` (kernel attribute calls) unless it already ran on the current
// device: attributes such as the dynamic shared-memory limit belong to a
// device, so each device needs its own call.  One bit per device id < 64 in
// `seen`; larger ids run `set` every time.  Concurrent first calls may both
// run `set`, which is harmless.
template <typename F>
inline void once_per_device(std::atomic<unsigned long long> &seen, F &&set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ULL << dev : 0ULL;
    if (bit && (seen.load(std::memory_order_acquire) & bit)) return;
    set();
    if (bit) seen.fetch_or(bit, std::memory_order_release);
}

// status from a CUDA error
inline int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return ANOVA_OK;
    if (e == cudaErrorMemoryAllocation) return ANOVA_ERR_NOMEM;
    return ANOVA_ERR_CUDA;
}

}  // namespace agft

struct anova_plan_s {
    agft::Plan p;
};
