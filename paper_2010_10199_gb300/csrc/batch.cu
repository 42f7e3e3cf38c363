// Many independent problems in one launch per kernel.
//
// The paper notes that the low-dimensional transforms are independent of each
// other (after eq. (somafm) and after the stacked adjoint, Sec. 3); independent
// problems are independent in the same way.  A batch holds one ordinary plan
// per problem plus device work lists: (problem, tile of 128 nodes) for the
// gather, (problem, term, node chunk) for the spread and (problem, term) for the
// deconvolution/FFT passes, so each kernel is launched once for all problems
// and the GPU is filled even when every single problem is small.  Vectors of a
// batch are the concatenation of the problems' vectors.
//
// lsqr_solve_batch runs one LSQR (eq. (new_min_prob), Sec. 4.1) per problem
// with its own FP64 scalars; every vector kernel works on the problems'
// segments in one launch (blockIdx.y = problem) and a problem whose stopping
// test fired is skipped by every kernel, the transforms included.
#include <algorithm>
#include <cstring>
#include <vector>

#include "solvers.cuh"

namespace agft {

int gather_launch(cudaStream_t st, const DevPlan &v, const BatchArgs &B, const float2 *fhat, float2 *f, int n_tiles,
                  int mr, int pitch, long long max_grid_bytes, int dmax, int sm_count, int prec);
__global__ void trafo_pre_f32(DevPlan single, BatchArgs B, const float2 *__restrict__ fhat_base);

constexpr int BRB = 32;   // partial sums per problem segment

struct Batch {
    int P = 0;
    cudaStream_t stream = nullptr;
    std::vector<anova_plan_t> plans;
    std::vector<long long> node_off, coef_off;   // [P + 1]
    std::vector<DevPlan> views;
    DevPlan *d_plans = nullptr;
    int *d_tables = nullptr;   // tile_prob | tile0 | blk_prob | blk0
    int4 *d_items = nullptr;   // spread work items
    int *counter = nullptr;
    BatchArgs args;
    int n_tiles = 0, n_items = 0, n_items3 = 0, n_blocks = 0, mr = 3, pitch = 0, dmax = 1, max_fft = 1,
        sm_count = 152;
    long long max_grid_bytes = 16, max_grid_elems = 0;
    bool any_empty = false;
    bool sorted_fwd = true;   // every problem has cell-sorted records for all its terms
    bool cell_tc = true;      // every problem runs its order-1/2 spread on the tensor cores
    long long max_M = 0;
    double2 *scratch = nullptr;
    // batched LSQR workspace
    float2 *u = nullptr, *tM = nullptr, *v = nullptr, *w = nullptr, *x = nullptr, *tn = nullptr;
    SolverState *st = nullptr;
    double *part = nullptr;
    long long *d_node_off = nullptr, *d_coef_off = nullptr;
    cudaStream_t sstream = nullptr;
    cudaEvent_t join = nullptr, e0 = nullptr, e1 = nullptr;
};

static void free_batch(Batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    void *bufs[] = {b->d_plans, b->d_tables, b->d_items, b->counter, b->scratch, b->u, b->tM, b->v, b->w, b->x, b->tn, b->st, b->part,
                    b->d_node_off, b->d_coef_off};
    for (void *q : bufs)
        if (q) cudaFree(q);
    if (b->sstream) cudaStreamDestroy(b->sstream);
    if (b->join) cudaEventDestroy(b->join);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    for (anova_plan_t p : b->plans) anova_plan_destroy(p);
    delete b;
}

static int upload_views(Batch &b) {
    cudaError_t e = cudaMemcpyAsync(b.d_plans, b.views.data(), sizeof(DevPlan) * b.P, cudaMemcpyHostToDevice, b.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b.stream);
    return cuda_status(e);
}

static int batch_trafo(Batch &b, cudaStream_t st, const float2 *fhat, float2 *f) {
    const size_t pre_smem = (size_t)b.max_fft * 2 * sizeof(float2);
    static std::atomic<unsigned long long> attr_seen{0};
    once_per_device(attr_seen, [] {
        cudaFuncSetAttribute(trafo_pre_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    trafo_pre_f32<<<b.n_blocks, 256, pre_smem, st>>>(b.views[0], b.args, fhat);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    if (b.sorted_fwd)
        return gather_sorted_launch(st, b.views[0], b.args, b.P, fhat, f, b.args.items, b.n_items3, b.n_items,
                                    b.counter, b.max_grid_bytes, b.max_M, b.sm_count, b.mr, (double *)b.scratch,
                                    b.cell_tc);
    return gather_launch(st, b.views[0], b.args, fhat, f, b.n_tiles, b.mr, b.pitch, b.max_grid_bytes, b.dmax,
                         b.sm_count, ANOVA_PREC_F32);
}

static int batch_adjoint(Batch &b, cudaStream_t st, const float2 *y, float2 *fhat) {
    return adjoint_launch(nullptr, st, b.views[0], b.args, b.P, y, fhat, b.n_items, b.n_items3, b.counter,
                          b.n_blocks, b.mr, b.max_grid_bytes, b.max_fft, b.sm_count, b.max_grid_elems, b.any_empty,
                          b.scratch, ANOVA_PREC_F32, b.cell_tc);
}

// ----------------------------------------------------- segmented kernels --

// out = (scale_in) in ; partial |out|^2 per segment
__global__ void k_bs_copy(const SolverState *st, float2 *out, const float2 *in, const long long *seg, double *part) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    double acc = 0.0;
    if (!st[p].done) {
        for (long long i = seg[p] + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < seg[p + 1];
             i += (long long)gridDim.x * blockDim.x) {
            float2 v = in[i];
            out[i] = v;
            acc += (double)v.x * v.x + (double)v.y * v.y;
        }
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && part) part[p * BRB + blockIdx.x] = s;
}

// out = a - c out with c = alpha (which 0) or beta (1) of the segment's problem
__global__ void k_bs_sub(const SolverState *st, float2 *out, const float2 *a, int which, const long long *seg,
                         double *part) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    double acc = 0.0;
    if (!st[p].done) {
        const float c = (float)(which == 0 ? st[p].alpha : st[p].beta);
        for (long long i = seg[p] + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < seg[p + 1];
             i += (long long)gridDim.x * blockDim.x) {
            float2 av = a[i], o = out[i];
            o.x = av.x - c * o.x;
            o.y = av.y - c * o.y;
            out[i] = o;
            acc += (double)o.x * o.x + (double)o.y * o.y;
        }
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[p * BRB + blockIdx.x] = s;
}

__global__ void k_bs_finish(SolverState *st, const double *part) {
    __shared__ double sh[32];
    const int p = blockIdx.x;
    double v = threadIdx.x < BRB ? part[p * BRB + threadIdx.x] : 0.0;
    double s = block_sum(v, sh);
    if (threadIdx.x == 0 && !st[p].done) st[p].red[0] = s;
}

__global__ void k_bs_set_norm(SolverState *st, int P, int which) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || st[p].done) return;
    const double nv = sqrt(st[p].red[0]);
    if (which == 0)
        st[p].alpha = nv;
    else
        st[p].beta = nv;
}

__global__ void k_bs_normalize(const SolverState *st, float2 *v, int which, const long long *seg) {
    const int p = blockIdx.y;
    if (st[p].done) return;
    const double nv = which == 0 ? st[p].alpha : st[p].beta;
    const float inv = nv > 0 ? (float)(1.0 / nv) : 0.f;
    for (long long i = seg[p] + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < seg[p + 1];
         i += (long long)gridDim.x * blockDim.x) {
        float2 a = v[i];
        v[i] = make_float2(a.x * inv, a.y * inv);
    }
}

__global__ void k_bs_init(SolverState *st, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) lsqr_init_dev(&st[p]);
}

__global__ void k_bs_scalars(SolverState *st, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) lsqr_scalars_dev(&st[p]);
}

__global__ void k_bs_test(SolverState *st, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) lsqr_test_dev(&st[p]);
}

__global__ void k_bs_update(const SolverState *st, float2 *x, float2 *w, const float2 *v, const long long *seg,
                            double *part) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    double acc = 0.0;
    if (!st[p].done) {
        const float a = (float)st[p].phi_rho, bb = (float)st[p].theta_rho;
        for (long long i = seg[p] + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < seg[p + 1];
             i += (long long)gridDim.x * blockDim.x) {
            float2 wi = w[i], xi = x[i], vi = v[i];
            xi.x += a * wi.x;
            xi.y += a * wi.y;
            wi.x = vi.x - bb * wi.x;
            wi.y = vi.y - bb * wi.y;
            x[i] = xi;
            w[i] = wi;
            acc += (double)xi.x * xi.x + (double)xi.y * xi.y;
        }
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[p * BRB + blockIdx.x] = s;
}

__global__ void k_bs_zero(float2 *v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = make_float2(0.f, 0.f);
}

__global__ void k_bs_all_done(const SolverState *st, int P, int *flag) {
    if (threadIdx.x != 0) return;
    int d = 1;
    for (int p = 0; p < P; ++p) d &= st[p].done != 0;
    *flag = d;
}

}  // namespace agft

using namespace agft;

struct anova_batch_s {
    Batch *b;
};

extern "C" {

int anova_batch_create(anova_batch_t *out, int n_problems, const int *d, const int64_t *M, const float *const *x_dev,
                       const int *n_terms, const int32_t *const *term_dims, const int32_t *const *bandwidth,
                       const anova_plan_options *opts, void *stream) {
    if (!out || n_problems < 1 || !d || !M || !x_dev || !n_terms || !term_dims || !bandwidth) return ANOVA_ERR_INVALID;
    *out = nullptr;
    cudaGetLastError();
    anova_plan_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.precision != ANOVA_PREC_F32) return ANOVA_ERR_UNSUPPORTED;
    Batch *b = new Batch();
    b->P = n_problems;
    b->stream = (cudaStream_t)stream;
    b->node_off.assign(n_problems + 1, 0);
    b->coef_off.assign(n_problems + 1, 0);
    std::vector<int> tile_prob, tile0, blk_prob, blk0;
    int total_act = 0;
    int pitch = -1;
    bool mixed_pitch = false;
    for (int p = 0; p < n_problems; ++p) {
        if (M[p] < 1) {
            free_batch(b);
            return ANOVA_ERR_INVALID;
        }
        anova_plan_t h = nullptr;
        int rc = anova_plan_create(&h, d[p], M[p], x_dev[p], n_terms[p], term_dims[p], bandwidth[p], &o, stream);
        if (rc) {
            free_batch(b);
            return rc;
        }
        b->plans.push_back(h);
        Plan &pl = h->p;
        if (pl.n_terms < 1) {   // every problem needs a non-empty term in a batch
            free_batch(b);
            return ANOVA_ERR_UNSUPPORTED;
        }
        b->node_off[p + 1] = b->node_off[p] + pl.M;
        b->coef_off[p + 1] = b->coef_off[p] + pl.n_coeffs;
        DevPlan v = dev_view(pl);
        v.vec_node_off = b->node_off[p];
        v.vec_coef_off = b->coef_off[p];
        b->views.push_back(v);
        const int tiles = (int)((pl.M + GATHER_TILE - 1) / GATHER_TILE);
        tile0.push_back(b->n_tiles);
        for (int t = 0; t < tiles; ++t) tile_prob.push_back(p);
        b->n_tiles += tiles;
        total_act += pl.n_act;
        blk0.push_back(b->n_blocks);
        for (int t = 0; t < pl.n_act; ++t) blk_prob.push_back(p);
        b->n_blocks += pl.n_act;
        for (int s = 0; s < pl.n_terms; ++s)
            if (pl.h_terms[s].mr > 0) b->mr = pl.h_terms[s].mr;
        if (pl.pitch2 > 8) {
            if (pitch < 0) pitch = pl.pitch2;
            else if (pitch != pl.pitch2) mixed_pitch = true;
        }
        b->dmax = std::max(b->dmax, pl.d);
        b->max_fft = std::max(b->max_fft, pl.max_fft_elems);
        b->max_grid_bytes = std::max(b->max_grid_bytes, pl.max_grid_bytes);
        b->max_grid_elems = std::max(b->max_grid_elems, pl.grid_elems);
        b->any_empty = b->any_empty || pl.n_empty > 0;
        b->sorted_fwd = b->sorted_fwd && pl.srec && pl.facc && pl.n_act3 == 0;
        b->cell_tc = b->cell_tc && pl.srec && pl.cell_tc;
        b->max_M = std::max(b->max_M, pl.M);
        b->sm_count = pl.sm_count;
    }
    b->pitch = mixed_pitch || pitch < 0 ? 0 : pitch;
    // spread items: every problem's active terms split into K_p node chunks,
    // K_p sized for all problems sharing the GPU
    std::vector<int4> items;
    std::vector<int> Ks(n_problems);
    bool order3 = false;
    for (int p = 0; p < n_problems; ++p) {
        const Plan &pl = b->plans[p]->p;
        for (int i = 0; i < pl.n_act; ++i) order3 = order3 || pl.h_terms[pl.h_act[i]].order == 3;
    }
    for (int p = 0; p < n_problems; ++p) {
        Plan &pl = b->plans[p]->p;
        Ks[p] = spread_chunks_for(pl.M, total_act, pl.spread_kmax, b->max_grid_bytes, b->sm_count, b->cell_tc,
                                  order3);
        b->views[p].spread_chunks = Ks[p];
    }
    // third-order items of every problem first, then the others
    for (int sel : {3, 0}) {
        for (int p = 0; p < n_problems; ++p) {
            Plan &pl = b->plans[p]->p;
            const size_t at = items.size();
            items.resize(at + (size_t)pl.n_act * Ks[p]);
            items.resize(at + append_spread_items(pl, p, Ks[p], items.data() + at, sel));
        }
        if (sel == 3) b->n_items3 = (int)items.size();
    }
    b->n_items = (int)items.size();
    cudaError_t e = cudaMalloc(&b->d_plans, sizeof(DevPlan) * n_problems);
    const size_t nt = tile_prob.size() + tile0.size() + blk_prob.size() + blk0.size();
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tables, sizeof(int) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int4) * std::max<size_t>(1, items.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->scratch, sizeof(double2) * 256 * n_problems);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_status(e);
    }
    std::vector<int> tab;
    tab.reserve(nt);
    int *base = b->d_tables;
    auto put = [&](const std::vector<int> &v) {
        const int *ptr = base + tab.size();
        tab.insert(tab.end(), v.begin(), v.end());
        return ptr;
    };
    b->args.plans = b->d_plans;
    b->args.P = n_problems;
    b->args.tile_prob = put(tile_prob);
    b->args.tile0 = put(tile0);
    b->args.items = b->d_items;
    b->args.blk_prob = put(blk_prob);
    b->args.blk0 = put(blk0);
    e = cudaMemcpyAsync(b->d_tables, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_status(e);
    }
    int rc = upload_views(*b);
    if (rc) {
        free_batch(b);
        return rc;
    }
    anova_batch_s *h = new anova_batch_s;
    h->b = b;
    *out = h;
    return ANOVA_OK;
}

void anova_batch_destroy(anova_batch_t batch) {
    if (!batch) return;
    free_batch(batch->b);
    delete batch;
}

int anova_batch_layout(anova_batch_t batch, int64_t *node_off, int64_t *coef_off) {
    if (!batch) return ANOVA_ERR_INVALID;
    Batch &b = *batch->b;
    for (int p = 0; p <= b.P; ++p) {
        if (node_off) node_off[p] = b.node_off[p];
        if (coef_off) coef_off[p] = b.coef_off[p];
    }
    return ANOVA_OK;
}

int grouped_trafo_batch(anova_batch_t batch, const void *fhat_dev, void *f_dev) {
    if (!batch || !fhat_dev || !f_dev) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Batch &b = *batch->b;
    return batch_trafo(b, b.stream, (const float2 *)fhat_dev, (float2 *)f_dev);
}

int grouped_adjoint_batch(anova_batch_t batch, const void *y_dev, void *fhat_dev) {
    if (!batch || !y_dev || !fhat_dev) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Batch &b = *batch->b;
    return batch_adjoint(b, b.stream, (const float2 *)y_dev, (float2 *)fhat_dev);
}

int lsqr_solve_batch(anova_batch_t batch, const void *y_dev, double lambda, int max_it, void *fhat_dev,
                     anova_solve_info *info) {
    if (!batch || !y_dev || !fhat_dev || lambda < 0 || max_it < 1) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Batch &b = *batch->b;
    const int P = b.P;
    const long long Mt = b.node_off[P], nt = b.coef_off[P];
    cudaError_t e = cudaSuccess;
    if (!b.st) {
        auto A = [&](void **ptr, size_t bytes) {
            if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
        };
        A((void **)&b.u, sizeof(float2) * Mt);
        A((void **)&b.tM, sizeof(float2) * Mt);
        A((void **)&b.v, sizeof(float2) * nt);
        A((void **)&b.w, sizeof(float2) * nt);
        A((void **)&b.x, sizeof(float2) * nt);
        A((void **)&b.tn, sizeof(float2) * nt);
        A((void **)&b.st, sizeof(SolverState) * P + 64);
        A((void **)&b.part, sizeof(double) * P * BRB);
        A((void **)&b.d_node_off, sizeof(long long) * (P + 1));
        A((void **)&b.d_coef_off, sizeof(long long) * (P + 1));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b.sstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&b.e0);
        if (e == cudaSuccess) e = cudaEventCreate(&b.e1);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b.d_node_off, b.node_off.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice,
                                b.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b.d_coef_off, b.coef_off.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice,
                                b.stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // per-problem skip flags = done flags of the per-problem solver states
    for (int p = 0; p < P; ++p) b.views[p].skip = &b.st[p].done;
    int rc = upload_views(b);
    if (rc) return rc;
    cudaStream_t s = b.sstream;
    cudaEventRecord(b.join, b.stream);
    cudaStreamWaitEvent(s, b.join, 0);
    std::vector<SolverState> h0(P);
    std::memset(h0.data(), 0, sizeof(SolverState) * P);
    for (int p = 0; p < P; ++p) {
        h0[p].damp = std::sqrt(2.0 * lambda);
        h0[p].max_it = max_it;
        h0[p].tiny_rel = std::max(1e-6, b.plans[p]->p.eps);
    }
    cudaMemcpyAsync(b.st, h0.data(), sizeof(SolverState) * P, cudaMemcpyHostToDevice, s);
    const float2 *y = (const float2 *)y_dev;
    const dim3 gM(BRB, P), gn(BRB, P);
    const int tb = (P + 127) / 128;
    cudaEventRecord(b.e0, s);
    // beta u = y ; alpha v = A^H u
    k_bs_copy<<<gM, 256, 0, s>>>(b.st, b.u, y, b.d_node_off, b.part);
    k_bs_finish<<<P, 64, 0, s>>>(b.st, b.part);
    k_bs_set_norm<<<tb, 128, 0, s>>>(b.st, P, 1);
    k_bs_normalize<<<gM, 256, 0, s>>>(b.st, b.u, 1, b.d_node_off);
    rc = batch_adjoint(b, s, b.u, b.tn);
    if (rc) return rc;
    k_bs_copy<<<gn, 256, 0, s>>>(b.st, b.v, b.tn, b.d_coef_off, b.part);
    k_bs_finish<<<P, 64, 0, s>>>(b.st, b.part);
    k_bs_set_norm<<<tb, 128, 0, s>>>(b.st, P, 0);
    k_bs_normalize<<<gn, 256, 0, s>>>(b.st, b.v, 0, b.d_coef_off);
    cudaMemcpyAsync(b.w, b.v, sizeof(float2) * nt, cudaMemcpyDeviceToDevice, s);
    k_bs_zero<<<304, 256, 0, s>>>(b.x, nt);
    k_bs_init<<<tb, 128, 0, s>>>(b.st, P);
    auto step = [&]() -> int {
        k_bs_copy<<<gn, 256, 0, s>>>(b.st, b.tn, b.v, b.d_coef_off, nullptr);
        int r = batch_trafo(b, s, b.tn, b.tM);
        if (r) return r;
        k_bs_sub<<<gM, 256, 0, s>>>(b.st, b.u, b.tM, 0, b.d_node_off, b.part);
        k_bs_finish<<<P, 64, 0, s>>>(b.st, b.part);
        k_bs_set_norm<<<tb, 128, 0, s>>>(b.st, P, 1);
        k_bs_normalize<<<gM, 256, 0, s>>>(b.st, b.u, 1, b.d_node_off);
        r = batch_adjoint(b, s, b.u, b.tn);
        if (r) return r;
        k_bs_sub<<<gn, 256, 0, s>>>(b.st, b.v, b.tn, 1, b.d_coef_off, b.part);
        k_bs_finish<<<P, 64, 0, s>>>(b.st, b.part);
        k_bs_scalars<<<tb, 128, 0, s>>>(b.st, P);
        k_bs_normalize<<<gn, 256, 0, s>>>(b.st, b.v, 0, b.d_coef_off);
        k_bs_update<<<gn, 256, 0, s>>>(b.st, b.x, b.w, b.v, b.d_coef_off, b.part);
        k_bs_finish<<<P, 64, 0, s>>>(b.st, b.part);
        k_bs_test<<<tb, 128, 0, s>>>(b.st, P);
        return cuda_status(cudaGetLastError());
    };
    // first iteration uncaptured, then one recorded iteration replayed
    rc = step();
    if (rc) return rc;
    int *all_done = (int *)((char *)b.st + sizeof(SolverState) * P);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (max_it > 1) {
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e);
        rc = step();
        e = cudaStreamEndCapture(s, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : cuda_status(e);
        }
        e = cudaGraphInstantiate(&ge, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_status(e);
        }
        for (int it = 1; it < max_it;) {
            const int k = std::min(16, max_it - it);
            for (int j = 0; j < k && e == cudaSuccess; ++j) e = cudaGraphLaunch(ge, s);
            it += k;
            k_bs_all_done<<<1, 32, 0, s>>>(b.st, P, all_done);
            int done = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&done, all_done, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess || done) break;
        }
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaMemcpyAsync(fhat_dev, b.x, sizeof(float2) * nt, cudaMemcpyDeviceToDevice, s);
    cudaEventRecord(b.e1, s);
    std::vector<SolverState> hs(P);
    cudaMemcpyAsync(hs.data(), b.st, sizeof(SolverState) * P, cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    cudaEventRecord(b.join, s);
    cudaStreamWaitEvent(b.stream, b.join, 0);
    for (int p = 0; p < P; ++p) b.views[p].skip = nullptr;
    int rc2 = upload_views(b);
    if (e != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b.e0, b.e1);
    int status = ANOVA_OK;
    for (int p = 0; p < P; ++p) {
        if (info) {
            std::memset(&info[p], 0, sizeof(anova_solve_info));
            info[p].iterations = hs[p].iters;
            info[p].status = hs[p].status;
            info[p].stop_reason = hs[p].stop;
            info[p].n_trafo = hs[p].iters;
            info[p].n_adjoint = hs[p].iters + 1;
            info[p].rnorm = hs[p].rnorm;
            info[p].arnorm = hs[p].arnorm;
            info[p].seconds = ms * 1e-3;
        }
        if (hs[p].status && !status) status = hs[p].status;
    }
    return status ? status : rc2;
}

}  // extern "C"
