// Plan autotuner: picks the oversampling factor, the row window half-width,
// the number of node chunks per term of the adjoint, the node order of the
// spread and the cell kernels (tensor or CUDA cores) for one node set and term
// list, by timing transform pairs of
// candidate plans on the device and estimating each candidate's error against
// a wider-window, more oversampled reference plan (the NFFT error falls with
// both, Sec. 3 after eq. (somafm)).  The fastest candidate whose estimated
// error meets the target wins.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace agft {

// deterministic test vectors: SplitMix64 of the index, two uniforms in [-1, 1)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_tune_vec(float2 *v, long long n, unsigned long long salt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = mix64(salt + 2 * (unsigned long long)i);
        const unsigned long long b = mix64(salt + 2 * (unsigned long long)i + 1);
        v[i] = make_float2((float)((a >> 11) * 0x1.0p-52 - 1.0), (float)((b >> 11) * 0x1.0p-52 - 1.0));
    }
}

// partial sums of |a - b|^2 and |b|^2 (FP64), one pair per block
__global__ void k_tune_diff(const float2 *a, const float2 *b, long long n, double2 *part) {
    __shared__ double2 sh[256];
    double d2 = 0.0, b2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 u = a[i], v = b[i];
        const double dx = (double)u.x - v.x, dy = (double)u.y - v.y;
        d2 += dx * dx + dy * dy;
        b2 += (double)v.x * v.x + (double)v.y * v.y;
    }
    sh[threadIdx.x] = make_double2(d2, b2);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x].x += sh[threadIdx.x + o].x;
            sh[threadIdx.x].y += sh[threadIdx.x + o].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// per coefficient block u: partial sums of |a - b|^2 and |b|^2 (one block per term)
__global__ void k_tune_block_diff(const float2 *a, const float2 *b, const long long *off, const long long *len,
                                  double2 *out) {
    __shared__ double2 sh[256];
    const long long o = off[blockIdx.x], m = len[blockIdx.x];
    double d2 = 0.0, b2 = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 u = a[o + i], v = b[o + i];
        const double dx = (double)u.x - v.x, dy = (double)u.y - v.y;
        d2 += dx * dx + dy * dy;
        b2 += (double)v.x * v.x + (double)v.y * v.y;
    }
    sh[threadIdx.x] = make_double2(d2, b2);
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[threadIdx.x].x += sh[threadIdx.x + s].x;
            sh[threadIdx.x].y += sh[threadIdx.x + s].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

namespace {

struct TuneBuffers {
    float2 *fhat = nullptr, *y = nullptr, *f = nullptr, *g = nullptr, *f_ref = nullptr, *g_ref = nullptr;
    double2 *part = nullptr, *bpart = nullptr;
    long long *boff = nullptr, *blen = nullptr;
    ~TuneBuffers() {
        void *b[] = {fhat, y, f, g, f_ref, g_ref, part, bpart, boff, blen};
        for (void *q : b)
            if (q) cudaFree(q);
    }
};

constexpr int TUNE_BLOCKS = 256;

double rel_diff(const float2 *a, const float2 *b, long long n, double2 *part, cudaStream_t st) {
    if (n == 0) return 0.0;
    k_tune_diff<<<TUNE_BLOCKS, 256, 0, st>>>(a, b, n, part);
    std::vector<double2> h(TUNE_BLOCKS);
    cudaMemcpyAsync(h.data(), part, sizeof(double2) * TUNE_BLOCKS, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return INFINITY;
    double d2 = 0.0, b2 = 0.0;
    for (const double2 &v : h) {
        d2 += v.x;
        b2 += v.y;
    }
    return std::sqrt(d2 / std::max(b2, 1e-300));
}

// the largest relative l2 distance over the coefficient blocks (blocks whose
// reference is zero are skipped)
double worst_block(const float2 *a, const float2 *b, const long long *off, const long long *len, int G,
                   double2 *out, cudaStream_t st) {
    if (G == 0) return 0.0;
    k_tune_block_diff<<<G, 256, 0, st>>>(a, b, off, len, out);
    std::vector<double2> h(G);
    cudaMemcpyAsync(h.data(), out, sizeof(double2) * G, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return INFINITY;
    double w = 0.0;
    for (const double2 &v : h)
        if (v.y > 0) w = std::max(w, std::sqrt(v.x / v.y));
    return w;
}

}  // namespace

}  // namespace agft

using namespace agft;

extern "C" {

int anova_plan_autotune(anova_plan_options *opts, int d, int64_t M, const void *x_dev, int n_terms,
                        const int32_t *term_dims, const int32_t *bandwidth, double eps_target, int reps,
                        anova_tune_trial *trials, int max_trials, int *n_trials, void *stream) {
    if (!opts || !(eps_target > 0) || reps < 1 || M < 1 || (max_trials > 0 && !trials)) return ANOVA_ERR_INVALID;
    if (opts->precision != ANOVA_PREC_F32) return ANOVA_ERR_UNSUPPORTED;
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    int nt = 0;
    if (n_trials) *n_trials = 0;

    // reference: sigma 2.5 and the widest windows
    anova_plan_options ro = *opts;
    ro.sigma = 2.5;
    ro.window_m_row = 4;
    ro.eps = 1e-8;
    anova_plan_t ref = nullptr;
    int rc = anova_plan_create(&ref, d, M, x_dev, n_terms, term_dims, bandwidth, &ro, stream);
    if (rc) return rc;
    const long long n = anova_num_coeffs(ref);
    TuneBuffers T;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t b) {
        if (e == cudaSuccess) e = cudaMalloc(p, b);
    };
    A((void **)&T.fhat, sizeof(float2) * std::max<long long>(1, n));
    A((void **)&T.g, sizeof(float2) * std::max<long long>(1, n));
    A((void **)&T.g_ref, sizeof(float2) * std::max<long long>(1, n));
    A((void **)&T.y, sizeof(float2) * M);
    A((void **)&T.f, sizeof(float2) * M);
    A((void **)&T.f_ref, sizeof(float2) * M);
    A((void **)&T.part, sizeof(double2) * TUNE_BLOCKS);
    A((void **)&T.bpart, sizeof(double2) * n_terms);
    A((void **)&T.boff, sizeof(long long) * n_terms);
    A((void **)&T.blen, sizeof(long long) * n_terms);
    if (e == cudaSuccess) {
        std::vector<long long> ho(n_terms), hl(n_terms);
        for (int u = 0; u < n_terms; ++u) {
            int64_t o = 0, l = 0;
            anova_term_offset(ref, u, &o, &l);
            ho[u] = o;
            hl[u] = l;
        }
        e = cudaMemcpyAsync(T.boff, ho.data(), sizeof(long long) * n_terms, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T.blen, hl.data(), sizeof(long long) * n_terms, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        anova_plan_destroy(ref);
        return cuda_status(e);
    }
    k_tune_vec<<<TUNE_BLOCKS, 256, 0, st>>>(T.fhat, n, 0x5EEDULL);
    k_tune_vec<<<TUNE_BLOCKS, 256, 0, st>>>(T.y, M, 0xF00DULL);
    rc = grouped_trafo(ref, T.fhat, T.f_ref);
    if (!rc) rc = grouped_adjoint(ref, T.y, T.g_ref);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    anova_plan_destroy(ref);
    if (rc) return rc;

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    struct Cand {
        anova_plan_options o;
        double ms, err;
        bool ok;
    };
    std::vector<Cand> done;
    auto trial = [&](const anova_plan_options &o) -> int {
        Cand c{o, INFINITY, INFINITY, false};
        anova_plan_t p = nullptr;
        int r = anova_plan_create(&p, d, M, x_dev, n_terms, term_dims, bandwidth, &o, stream);
        if (r == ANOVA_ERR_UNSUPPORTED || r == ANOVA_ERR_NOMEM) {
            cudaGetLastError();
            done.push_back(c);   // not buildable: recorded, never chosen
            return ANOVA_OK;
        }
        if (r) return r;
        r = grouped_trafo(p, T.fhat, T.f);   // warm-up, also the error sample
        if (!r) r = grouped_adjoint(p, T.y, T.g);
        if (!r) {
            const double ef = rel_diff(T.f, T.f_ref, M, T.part, st);
            const double eg = rel_diff(T.g, T.g_ref, n, T.part, st);
            const double eb = worst_block(T.g, T.g_ref, T.boff, T.blen, n_terms, T.bpart, st);
            c.err = std::max(ef, std::max(eg, eb));
            cudaEventRecord(e0, st);
            for (int i = 0; i < reps && !r; ++i) {
                r = grouped_trafo(p, T.fhat, T.f);
                if (!r) r = grouped_adjoint(p, T.y, T.g);
            }
            cudaEventRecord(e1, st);
            if (!r) r = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            c.ms = ms / reps;
            c.ok = c.err <= eps_target;
        }
        anova_plan_destroy(p);
        done.push_back(c);
        return r;
    };
    auto best = [&]() -> int {
        int b = -1;
        for (int i = 0; i < (int)done.size(); ++i)
            if (done[i].ok && (b < 0 || done[i].ms < done[b].ms)) b = i;
        return b;
    };
    // stage 1: oversampling and row window, default chunks and node order
    for (double sg : {1.75, 2.0, 2.5})
        for (int mr : {3, 4}) {
            anova_plan_options o = *opts;
            o.sigma = sg;
            o.window_m_row = mr;
            o.n_ctas = 0;
            o.node_sort = 0;
            o.cell_kernel = 0;
            rc = trial(o);
            if (rc) break;
        }
    // stage 2: node chunks per term and node order around the best so far
    int b = rc ? -1 : best();
    if (b >= 0) {
        const anova_plan_options base = done[b].o;
        for (int k : {4, 16, 64}) {
            anova_plan_options o = base;
            o.n_ctas = k;
            rc = trial(o);
            if (rc) break;
        }
        if (!rc) {
            anova_plan_options o = base;
            o.node_sort = -1;
            rc = trial(o);
        }
        if (!rc) {
            anova_plan_options o = base;
            o.cell_kernel = 1;
            rc = trial(o);
        }
        b = best();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < (int)done.size(); ++i) {
        if (nt < max_trials) {
            anova_tune_trial &t = trials[nt++];
            t.sigma = done[i].o.sigma;
            t.window_m_row = done[i].o.window_m_row;
            t.n_ctas = done[i].o.n_ctas;
            t.node_sort = done[i].o.node_sort;
            t.cell_kernel = done[i].o.cell_kernel;
            t.ms_pair = done[i].ms;
            t.est_error = done[i].err;
            t.chosen = i == b;
        }
    }
    if (n_trials) *n_trials = nt;
    if (rc) return rc;
    if (b < 0) return ANOVA_ERR_UNSUPPORTED;   // no candidate met the target
    *opts = done[b].o;
    return ANOVA_OK;
}

}  // extern "C"
