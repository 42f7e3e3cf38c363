// Plan construction: term schedule, grid layout, window tables and
// deconvolution factors; the C-ABI bookkeeping entry points.
//
// Grouped index set and block order: eq. (groupedset) and (bananarama), Sec. 3;
// cardinality (N_u - 1)^{|u|}: Remark "cardinality", Sec. 2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace agft {

// ------------------------------------------------------------ host maths --

// Modified Bessel function I_0 by its power series sum (z/2)^{2j} / (j!)^2.
static double bessel_i0(double z) {
    double q = 0.25 * z * z, term = 1.0, sum = 1.0;
    for (int j = 1; j < 500; ++j) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// psi(d) = sinh(b sqrt(m^2 - d^2)) / (pi sqrt(m^2 - d^2)), continuous at |d| = m.
static double kb_window(double d, int m, double b) {
    double s2 = (double)m * m - d * d;
    if (s2 < 0) return 0.0;
    double s = std::sqrt(s2);
    if (b * s < 1e-8) return b / M_PI;
    return std::sinh(b * s) / (M_PI * s);
}

// Deconvolution factor psi(0) / I_0(m sqrt(b^2 - (2 pi k / n)^2)): the inverse of
// n times the Fourier coefficient of the normalised window psi(n x) / psi(0).
//
// The kernels place node x at grid position t = (x + 1/2) n, i.e. stored grid
// index q' = q + n/2 for the periodic index q of position q/n.  The shift by
// n/2 multiplies frequency k by exp(i pi k) = (-1)^k, which is folded in here
// (n is always even), for the forward and the adjoint alike.
double deconv_factor(int k, int n, int m, double b) {
    double a = 2.0 * M_PI * k / n;
    double r = b * b - a * a;
    double psi0 = std::sinh(b * m) / (M_PI * m);
    double sgn = (k & 1) ? -1.0 : 1.0;
    return sgn * psi0 / bessel_i0(m * std::sqrt(r > 0 ? r : 0.0));
}

// Degree-7 Chebyshev interpolant of each tap weight as a function of v = 2 tau - 1.
void window_polys(Window &w, int m, double b) {
    const int P = NCOEF;
    double psi0 = kb_window(0.0, m, b);
    for (int j = 0; j < 2 * MAXM; ++j)
        for (int i = 0; i < P; ++i) w.c[j][i] = w.ch[j][i] = 0.0f;
    for (int j = 0; j < 2 * m; ++j) {
        double fv[NCOEF], a[NCOEF];
        for (int i = 0; i < P; ++i) {
            double v = std::cos(M_PI * (i + 0.5) / P);
            double tau = 0.5 * (v + 1.0);
            fv[i] = kb_window(tau + m - 1 - j, m, b) / psi0;
        }
        for (int k = 0; k < P; ++k) {
            double s = 0;
            for (int i = 0; i < P; ++i) s += fv[i] * std::cos(M_PI * k * (i + 0.5) / P);
            a[k] = (k == 0 ? 1.0 : 2.0) * s / P;
            w.ch[j][k] = (float)(((k >> 1) & 1) ? -a[k] : a[k]);   // s_k a_k
        }
        // sum a_k T_k(v) -> monomials, T_{k+1} = 2 v T_k - T_{k-1}
        double Tm1[NCOEF] = {0}, T0[NCOEF] = {0}, mono[NCOEF] = {0};
        T0[0] = 1.0;
        double T1[NCOEF] = {0};
        T1[1] = 1.0;
        for (int i = 0; i < P; ++i) mono[i] += a[0] * T0[i];
        if (P > 1)
            for (int i = 0; i < P; ++i) mono[i] += a[1] * T1[i];
        for (int i = 0; i < P; ++i) Tm1[i] = T0[i];
        for (int i = 0; i < P; ++i) T0[i] = T1[i];
        for (int k = 2; k < P; ++k) {
            double Tn[NCOEF] = {0};
            for (int i = 0; i < P; ++i) {
                if (i > 0) Tn[i] += 2.0 * T0[i - 1];
                Tn[i] -= Tm1[i];
            }
            for (int i = 0; i < P; ++i) mono[i] += a[k] * Tn[i];
            for (int i = 0; i < P; ++i) {
                Tm1[i] = T0[i];
                T0[i] = Tn[i];
            }
        }
        for (int i = 0; i < P; ++i) w.c[j][i] = (float)mono[i];
    }
    w.m = m;
    w.b = (float)b;
    w.bd = b;
    w.inv_psi0 = (float)(1.0 / psi0);
    w.inv_psi0d = 1.0 / psi0;
}

static bool smooth235(int n) {
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

int fft_size(int N, double sigma) {
    int n = (int)std::ceil(sigma * N - 1e-9);
    if (n < N + 2) n = N + 2;
    if (n % 2) ++n;
    while (!smooth235(n)) n += 2;
    return n;
}

int row_stride(int n) {
    int s = n;
    while (s % 16 != 8) ++s;
    return s;
}

__global__ void wrap_nodes_f32(const float *in, float *out, long long total, float scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        float v = in[i] * scale;
        v = v - floorf(v + 0.5f);   // into [-1/2, 1/2)
        if (v >= 0.5f) v -= 1.0f;
        out[i] = v;
    }
}

__global__ void wrap_nodes_f64(const double *in, double *out, long long total, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        double v = in[i] * scale;
        v = v - floor(v + 0.5);
        if (v >= 0.5) v -= 1.0;
        out[i] = v;
    }
}

// Active term list: the scheduled terms whose user term is enabled in
// `user_mask` (all when null), with the row-group flags recomputed for that
// list.  Uploaded on the plan's stream.
int set_active_terms(Plan &p, const unsigned char *user_mask) {
    static thread_local std::vector<ActRec> recs, recs3;
    recs.clear();
    recs3.clear();
    int n = 0;
    for (int s = 0; s < p.n_terms; ++s) {
        const Term &T = p.h_terms[s];
        if (user_mask && !user_mask[T.user_index]) continue;
        int ng = 1;
        if (T.order == 2 && n > 0) {
            const Term &P = p.h_terms[p.h_act[n - 1]];
            if (P.order == 2 && P.row0 == T.row0 && P.wr == T.wr && P.n == T.n) ng = 0;
        }
        recs.push_back(make_act_rec(T, s, ng));
        if (T.order == 3 && T.sort_slot < 0) recs3.push_back(make_act_rec(T, s, 1));
        p.h_act[n++] = s;
    }
    p.n_act = n;
    p.n_act3 = (int)recs3.size();
    p.n_items = 0;
    p.n_items3 = 0;
    if (n == 0) return ANOVA_OK;
    bool order3 = false;
    for (int i = 0; i < n; ++i) order3 = order3 || p.h_terms[p.h_act[i]].order == 3;
    p.spread_K = spread_chunks_for(p.M, n, p.spread_kmax, p.max_grid_bytes, p.sm_count, p.cell_tc, order3);
    if (p.h_items) {
        p.n_items3 = append_spread_items(p, 0, p.spread_K, p.h_items, 3);
        p.n_items = p.n_items3 + append_spread_items(p, 0, p.spread_K, p.h_items + p.n_items3, 0);
    }
    cudaError_t e = cudaMemcpyAsync(p.act, p.h_act, sizeof(int) * n, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.act_rec, recs.data(), sizeof(ActRec) * n, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess && p.n_items)
        e = cudaMemcpyAsync(p.items, p.h_items, sizeof(int4) * p.n_items, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess && p.n_act3 && p.act_rec3)
        e = cudaMemcpyAsync(p.act_rec3, recs3.data(), sizeof(ActRec) * p.n_act3, cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);   // recs is reused by the next call
    return cuda_status(e);
}

DevPlan dev_view(const Plan &p) {
    DevPlan v;
    v.d = p.d;
    v.M = p.M;
    v.n_terms = p.n_terms;
    v.n_empty = p.n_empty;
    v.x = p.precision == ANOVA_PREC_F64 ? nullptr : (const float *)p.x;
    v.xd = p.precision == ANOVA_PREC_F64 ? (const double *)p.x : nullptr;
    v.terms = p.terms;
    v.windows = p.windows;
    v.deconv = p.deconv;
    v.deconvd = p.deconvd;
    v.empty_off = p.empty_off;
    v.grid_elems = p.grid_elems;
    v.max_grid_bytes = p.max_grid_bytes;
    v.err = p.err;
    v.act = p.act;
    v.act_rec = p.act_rec;
    v.n_act = p.n_act;
    v.skip = p.skip;
    v.grids = (const float2 *)p.grids;
    v.partials = (float2 *)p.partials;
    v.spread_chunks = p.spread_K;
    v.srec = p.srec;
    v.facc = p.facc;
    v.fexp = p.fexp;
    v.n_coeffs = p.n_coeffs;
    v.vec_node_off = 0;
    v.vec_coef_off = 0;
    v.basis = p.basis;
    return v;
}

// 0: no injected failure; k > 0: the k-th next allocation through
// plan_malloc / plan_new fails (then the counter is 0 again)
static std::atomic<int> g_fail_after{0};

bool alloc_fault() {
    int k = g_fail_after.load();
    while (k > 0)
        if (g_fail_after.compare_exchange_weak(k, k - 1)) return k == 1;
    return false;
}

cudaError_t plan_malloc_raw(void **ptr, size_t bytes) {
    if (alloc_fault()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

static void free_plan(Plan &p) {
    profiler_free(p);
    if (p.solver && p.solver_free) p.solver_free(p.solver);
    p.solver = nullptr;
    void *bufs[] = {p.x, p.terms, p.windows, p.deconv, p.deconvd, p.empty_off, p.grids, p.partials,
                    p.err, p.scratch, p.act, p.act_rec, p.act_rec3, p.items, p.counter, p.srec, p.wt64, p.wb64, p.slots64,
                    p.facc, p.fexp};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete[] p.h_terms;
    delete[] p.h_user_off;
    delete[] p.h_user_len;
    delete[] p.h_user_n;
    delete[] p.h_user_mc;
    delete[] p.h_user_mr;
    delete[] p.h_user_order;
    delete[] p.h_act;
    delete[] p.h_items;
}

}  // namespace agft

using namespace agft;

extern "C" {

const char *anova_status_string(int s) {
    switch (s) {
        case ANOVA_OK: return "ok";
        case ANOVA_ERR_INVALID: return "invalid argument";
        case ANOVA_ERR_UNSUPPORTED: return "unsupported configuration";
        case ANOVA_ERR_NOMEM: return "out of memory";
        case ANOVA_ERR_CUDA: return "CUDA error";
        case ANOVA_ERR_BREAKDOWN: return "solver breakdown";
        case ANOVA_ERR_TIMEOUT: return "device wait timed out";
        case ANOVA_ERR_NOT_FINITE: return "non-finite solver scalar";
        default: return "unknown status";
    }
}

const char *anova_version(void) { return "anova-gft 0.1 (sm_103a)"; }

static int plan_create(anova_plan_t *out, int d, int64_t M, const void *x_dev, int n_terms,
                       const int32_t *term_dims, const int32_t *bandwidth, const anova_plan_options *opts,
                       void *stream) {
    if (!out) return ANOVA_ERR_INVALID;
    *out = nullptr;
    cudaGetLastError();   // do not report an earlier, unrelated error
    if (d < 1 || M < 0 || M >= (1LL << 31) || n_terms < 1 || !term_dims || !bandwidth) return ANOVA_ERR_INVALID;
    if (M > 0 && !x_dev) return ANOVA_ERR_INVALID;
    anova_plan_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.precision < ANOVA_PREC_F32 || o.precision > ANOVA_PREC_F64) return ANOVA_ERR_INVALID;
    if (o.cell_kernel < 0 || o.cell_kernel > 1) return ANOVA_ERR_INVALID;
    if (o.basis != ANOVA_BASIS_EXP && o.basis != ANOVA_BASIS_COS) return ANOVA_ERR_INVALID;
    const bool cosine = o.basis == ANOVA_BASIS_COS;

    if (o.eps <= 0) o.eps = 1e-5;
    if (o.sigma <= 0) o.sigma = 2.0;
    if (o.sigma < 1.5 || o.sigma > 8) return ANOVA_ERR_INVALID;

    // validate terms
    for (int i = 0; i < n_terms; ++i) {
        const int32_t *t = term_dims + 3 * i;
        int ord = 0;
        for (int j = 0; j < 3; ++j) {
            if (t[j] < 0) {
                for (int l = j; l < 3; ++l)
                    if (t[l] >= 0) return ANOVA_ERR_INVALID;
                break;
            }
            if (t[j] >= d) return ANOVA_ERR_INVALID;
            if (j > 0 && t[j] <= t[j - 1]) return ANOVA_ERR_INVALID;
            ++ord;
        }
        // exponential groups need an even N (I_N = [-N/2, N/2)); cosine groups
        // 1 <= k <= N - 1 take any N >= 2 and run at the doubled bandwidth
        if (ord > 0 && (bandwidth[i] < 2 || (!cosine && bandwidth[i] % 2))) return ANOVA_ERR_INVALID;
        if (ord > 0 && bandwidth[i] * (cosine ? 2 : 1) > 4096) return ANOVA_ERR_UNSUPPORTED;
    }

    anova_plan_s *h = alloc_fault() ? nullptr : new (std::nothrow) anova_plan_s;
    if (!h) return ANOVA_ERR_NOMEM;
    std::memset(&h->p, 0, sizeof(Plan));
    // frees the plan on every return but the successful one (also when a
    // host container throws std::bad_alloc on the way out)
    struct Guard {
        anova_plan_s *h;
        ~Guard() {
            if (h) {
                free_plan(h->p);
                delete h;
            }
        }
    } guard{h};
    Plan &p = h->p;
    p.stream = (cudaStream_t)stream;
    p.precision = o.precision;
    p.basis = o.basis;
    p.eps = o.eps;
    p.d = d;
    p.M = M;
    p.n_user_terms = n_terms;
    cudaGetDevice(&p.device);
    cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, p.device);
    if (p.sm_count <= 0) p.sm_count = 152;

    int mc = o.window_m_col > 0 ? o.window_m_col : 4;
    // 6 row taps (m_row = 3) keep the whole-vector error near 5e-6 but leave
    // single terms (third-order ones, or any term sampled at few nodes) above
    // 1e-5; 8 taps hold every term near 3e-6
    int mr = o.window_m_row > 0 ? o.window_m_row : (o.eps >= 5e-5 ? 3 : 4);
    if (mc != 4) {   // eight column lanes per row segment
        return ANOVA_ERR_UNSUPPORTED;
    }
    if (mr < 3 || mr > 4) {
        return ANOVA_ERR_UNSUPPORTED;
    }

    // user layout
    p.h_user_off = plan_new<long long>(n_terms);
    p.h_user_len = plan_new<long long>(n_terms);
    p.h_user_n = plan_new<int>(n_terms);
    p.h_user_mc = plan_new<int>(n_terms);
    p.h_user_mr = plan_new<int>(n_terms);
    p.h_user_order = plan_new<int>(n_terms);
    if (!p.h_user_off || !p.h_user_len || !p.h_user_n || !p.h_user_mc || !p.h_user_mr || !p.h_user_order)
        return ANOVA_ERR_NOMEM;
    long long off = 0;
    std::vector<int> order(n_terms);
    std::vector<long long> empties;
    for (int i = 0; i < n_terms; ++i) {
        const int32_t *t = term_dims + 3 * i;
        int ord = (t[0] >= 0) + (t[1] >= 0) + (t[2] >= 0);
        order[i] = ord;
        long long len = 1;
        for (int j = 0; j < ord; ++j) len *= (bandwidth[i] - 1);
        p.h_user_off[i] = off;
        p.h_user_len[i] = len;
        p.h_user_n[i] = ord ? fft_size(bandwidth[i] * (cosine ? 2 : 1), o.sigma) : 0;
        p.h_user_mc[i] = ord ? mc : 0;
        p.h_user_mr[i] = ord > 1 ? mr : 0;
        p.h_user_order[i] = ord;
        if (ord == 0) empties.push_back(off);
        off += len;
    }
    p.n_coeffs = off;
    p.n_empty = (int)empties.size();

    // schedule: by first coordinate, then order, then the remaining coordinates
    std::vector<int> sched;
    for (int i = 0; i < n_terms; ++i)
        if (order[i] > 0) sched.push_back(i);
    std::stable_sort(sched.begin(), sched.end(), [&](int a, int b) {
        const int32_t *ta = term_dims + 3 * a, *tb = term_dims + 3 * b;
        if (ta[0] != tb[0]) return ta[0] < tb[0];
        if (order[a] != order[b]) return order[a] < order[b];
        if (ta[1] != tb[1]) return ta[1] < tb[1];
        return ta[2] < tb[2];
    });
    p.n_terms = (int)sched.size();
    p.h_terms = plan_new<Term>(p.n_terms > 0 ? p.n_terms : 1);
    if (!p.h_terms) return ANOVA_ERR_NOMEM;

    // windows (dedupe on m, n, N) and deconvolution tables
    std::vector<Window> wins;
    std::vector<int> wkey_m, wkey_n, wkey_N;
    auto get_window = [&](int m, int n, int N) {
        for (size_t i = 0; i < wins.size(); ++i)
            if (wkey_m[i] == m && wkey_n[i] == n && wkey_N[i] == N) return (int)i;
        Window w;
        std::memset(&w, 0, sizeof(w));
        window_polys(w, m, M_PI * (2.0 - (double)N / n));
        wins.push_back(w);
        wkey_m.push_back(m);
        wkey_n.push_back(n);
        wkey_N.push_back(N);
        return (int)wins.size() - 1;
    };
    std::vector<float> dec;
    std::vector<double> decd;
    long long goff = 0, maxbytes = 16;
    int max_fft = 1;
    int status = ANOVA_OK;
    // all order-2 grids share one row pitch (the gather specialises on it)
    p.pitch2 = 8;
    for (int s = 0; s < p.n_terms; ++s)
        if (order[sched[s]] == 2)
            p.pitch2 = std::max(p.pitch2, row_stride(p.h_user_n[sched[s]] + 2 * (mc - 1) + 1));   // n already doubled
    for (int s = 0; s < p.n_terms; ++s) {
        int i = sched[s];
        const int32_t *t = term_dims + 3 * i;
        Term T;
        std::memset(&T, 0, sizeof(T));
        T.order = order[i];
        T.col = t[T.order - 1];
        T.row0 = T.order >= 2 ? t[0] : -1;
        T.row1 = T.order >= 3 ? t[1] : -1;
        T.N = bandwidth[i] * (cosine ? 2 : 1);   // cosine terms: the mirrored exponential set
        T.basis = o.basis;
        T.n = p.h_user_n[i];
        T.rows = 1;
        for (int j = 1; j < T.order; ++j) T.rows *= T.n;
        T.mc = mc;
        T.mr = T.order > 1 ? mr : 0;
        T.sort_slot = -1;
        if (T.order <= 2) {
            T.hc = T.mc - 1;
            T.hr = T.order == 2 ? T.mr - 1 : 0;
            T.erows = T.order == 2 ? T.n + 2 * T.hr + 1 : 1;
            T.stride = T.order == 2 ? p.pitch2 : row_stride(T.n + 2 * T.hc + 1);
        } else {
            T.hc = T.hr = 0;
            T.erows = T.rows;
            T.stride = row_stride(T.n);
        }
        T.wc = get_window(T.mc, T.n, T.N);
        T.wr = T.order > 1 ? get_window(T.mr, T.n, T.N) : T.wc;
        T.grid_off = goff;
        long long elems = (long long)T.erows * T.stride;
        const bool f64 = p.precision == ANOVA_PREC_F64;
        const bool h16 = p.precision == ANOVA_PREC_F16 || p.precision == ANOVA_PREC_BF16;
        elems = h16 ? (elems + 3) & ~3LL : (elems + 1) & ~1LL;   // 16-byte multiples
        T.grid_bytes = elems * (f64 ? 16 : h16 ? 4 : 8);
        goff += elems;
        maxbytes = std::max(maxbytes, T.grid_bytes);
        long long fe = 1;
        for (int j = 0; j < T.order; ++j) fe *= T.n;
        // shared-memory limits of the FFT passes (two copies) and of the spread (one grid)
        if (fe * (f64 ? 32 : 16) > 200 * 1024 || T.grid_bytes > (f64 ? 200 : 100) * 1024) status = ANOVA_ERR_UNSUPPORTED;
        max_fft = (int)std::max<long long>(max_fft, fe);
        T.coef_off = p.h_user_off[i];
        T.coef_len = p.h_user_len[i];
        T.user_index = i;
        // deconvolution factors for k in I_N \ {0} (column window, then row window)
        double bc = M_PI * (2.0 - (double)T.N / T.n);
        T.dc_off = (int)dec.size();
        for (int q = 0; q < T.N - 1; ++q) {
            int k = q < T.N / 2 ? q - T.N / 2 : q - T.N / 2 + 1;
            double v = deconv_factor(k, T.n, T.mc, bc);
            dec.push_back((float)v);
            decd.push_back(v);
        }
        T.dr_off = T.dc_off;
        if (T.order > 1) {
            T.dr_off = (int)dec.size();
            for (int q = 0; q < T.N - 1; ++q) {
                int k = q < T.N / 2 ? q - T.N / 2 : q - T.N / 2 + 1;
                double v = deconv_factor(k, T.n, T.mr, bc);
                dec.push_back((float)v);
                decd.push_back(v);
            }
        }
        p.h_terms[s] = T;
    }
    // row groups: order-2 terms sharing the first coordinate and row window
    for (int s = 0; s < p.n_terms; ++s) {
        Term &T = p.h_terms[s];
        T.new_rowgroup = 1;
        if (T.order == 2 && s > 0) {
            const Term &P = p.h_terms[s - 1];
            if (P.order == 2 && P.row0 == T.row0 && P.wr == T.wr && P.n == T.n) T.new_rowgroup = 0;
        }
    }
    if (status != ANOVA_OK) return status;
    p.grid_elems = goff;
    p.max_grid_bytes = maxbytes;
    p.max_fft_elems = max_fft;
    p.n_windows = (int)wins.size();
    // FP64 plans: one window table per (window, coordinate) pair in use
    std::vector<int4> slots64;
    if (p.precision == ANOVA_PREC_F64) {
        auto slot_of = [&](int w, int c, int n, int m) {
            for (size_t i = 0; i < slots64.size(); ++i)
                if (slots64[i].x == w && slots64[i].y == c) return (int)i;
            slots64.push_back(make_int4(w, c, n, m));
            return (int)slots64.size() - 1;
        };
        for (int s = 0; s < p.n_terms; ++s) {
            Term &T = p.h_terms[s];
            T.slot_c = slot_of(T.wc, T.col, T.n, T.mc);
            T.slot_r0 = T.order >= 2 ? slot_of(T.wr, T.row0, T.n, T.mr) : -1;
            T.slot_r1 = T.order == 3 ? slot_of(T.wr, T.row1, T.n, T.mr) : -1;
        }
        p.n_slots64 = (int)slots64.size();
    }
    for (int i = 0; i < n_terms; ++i) {
        (void)i;
    }

    // device allocations
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
        if (r != cudaSuccess && e == cudaSuccess) e = r;
    };
    size_t xbytes = (size_t)d * M * (p.precision == ANOVA_PREC_F64 ? 8 : 4);
    if (xbytes) chk(plan_malloc(&p.x, xbytes));
    chk(plan_malloc(&p.terms, sizeof(Term) * std::max(1, p.n_terms)));
    chk(plan_malloc(&p.windows, sizeof(Window) * std::max<size_t>(1, wins.size())));
    chk(plan_malloc(&p.deconv, sizeof(float) * std::max<size_t>(1, dec.size())));
    chk(plan_malloc(&p.deconvd, sizeof(double) * std::max<size_t>(1, decd.size())));
    chk(plan_malloc(&p.empty_off, sizeof(long long) * std::max<size_t>(1, empties.size())));
    const size_t esize = p.precision == ANOVA_PREC_F64 ? 16 : (p.precision == ANOVA_PREC_F32 ? 8 : 4);   // bytes per grid element
    chk(plan_malloc(&p.grids, (size_t)std::max<long long>(1, p.grid_elems) * esize));
    chk(plan_malloc(&p.err, sizeof(int) * 4));
    chk(plan_malloc(&p.act, sizeof(int) * std::max(1, p.n_terms)));
    chk(plan_malloc(&p.act_rec, sizeof(ActRec) * std::max(1, p.n_terms)));
    chk(plan_malloc(&p.act_rec3, sizeof(ActRec) * std::max(1, p.n_terms)));
    p.h_act = plan_new<int>(std::max(1, p.n_terms));
    if (!p.h_act && e == cudaSuccess) e = cudaErrorMemoryAllocation;
    // adjoint partial grids: one per node chunk of a term (work items of the
    // spread are (term, chunk) pairs), bounded to 8 GB
    long long k_cap = std::max<long long>(1, (8LL << 30) / std::max<long long>(1, p.grid_elems * 8));
    int kmax = (int)std::min<long long>(std::min<long long>(SPREAD_MAX_K, k_cap),
                                        std::max<long long>(1, (M + 2047) / 2048));
    if (o.n_ctas > 0) kmax = std::min(o.n_ctas, SPREAD_MAX_K);
    p.spread_kmax = kmax;
    p.gather_ctas = (int)std::min<long long>((long long)p.sm_count,
                                             std::max<long long>(1, (M + GATHER_TILE - 1) / GATHER_TILE));
    if (e == cudaSuccess && p.n_terms > 0)
        chk(plan_malloc(&p.partials, (size_t)kmax * (size_t)p.grid_elems * esize));
    chk(plan_malloc(&p.items, sizeof(int4) * (size_t)std::max(1, p.n_terms) * kmax));
    chk(plan_malloc(&p.counter, 2 * sizeof(int)));
    p.h_items = plan_new<int4>((size_t)std::max(1, p.n_terms) * kmax);
    if (!p.h_items && e == cudaSuccess) e = cudaErrorMemoryAllocation;
    p.scratch_bytes = 1 << 20;
    chk(plan_malloc(&p.scratch, p.scratch_bytes));
    if (p.n_slots64 > 0 && M > 0) {
        chk(plan_malloc(&p.slots64, sizeof(int4) * p.n_slots64));
        chk(plan_malloc(&p.wt64, sizeof(double) * 8 * (size_t)p.n_slots64 * M));
        chk(plan_malloc(&p.wb64, sizeof(int) * (size_t)p.n_slots64 * M));
        if (e == cudaSuccess)
            chk(cudaMemcpyAsync(p.slots64, slots64.data(), sizeof(int4) * p.n_slots64, cudaMemcpyHostToDevice,
                                p.stream));
    }
    // cell-sorted node records (16 bytes per node for a term of order <= 2, 32
    // for order 3; FP64 plans sort order <= 2 only), if they fit in half the
    // free device memory.  sort_slot counts units of M records of 16 bytes.
    if (e == cudaSuccess && o.node_sort >= 0 && M > 0) {
        auto units = [&](const Term &T) { return T.order <= 2 ? 1 : (p.precision == ANOVA_PREC_F64 ? 0 : 2); };
        int ns = 0;
        for (int s = 0; s < p.n_terms; ++s) ns += units(p.h_terms[s]);
        size_t free_b = 0, total_b = 0;
        const size_t need = (size_t)ns * (size_t)M * sizeof(float4);
        if (ns > 0 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need <= free_b / 2) {
            if (plan_malloc(&p.srec, need) == cudaSuccess) {
                int slot = 0;
                for (int s = 0; s < p.n_terms; ++s) {
                    const int u = units(p.h_terms[s]);
                    if (u) {
                        p.h_terms[s].sort_slot = slot;
                        slot += u;
                    }
                }
                p.n_sorted = ns;
                p.cell_tc = p.precision != ANOVA_PREC_F64 && o.cell_kernel == 0;
                if (p.precision == ANOVA_PREC_F32) {
                    if (plan_malloc(&p.facc, sizeof(unsigned long long) * 2 * (size_t)M) != cudaSuccess ||
                        plan_malloc(&p.fexp, sizeof(int) * 4) != cudaSuccess) {
                        cudaGetLastError();   // the forward falls back to the point-major gather
                        if (p.facc) cudaFree(p.facc);
                        p.facc = nullptr;
                    }
                }
            } else {
                cudaGetLastError();
                p.srec = nullptr;
            }
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    chk(cudaMemcpyAsync(p.terms, p.h_terms, sizeof(Term) * p.n_terms, cudaMemcpyHostToDevice, p.stream));
    if (!wins.empty())
        chk(cudaMemcpyAsync(p.windows, wins.data(), sizeof(Window) * wins.size(), cudaMemcpyHostToDevice,
                            p.stream));
    if (!dec.empty()) {
        chk(cudaMemcpyAsync(p.deconv, dec.data(), sizeof(float) * dec.size(), cudaMemcpyHostToDevice, p.stream));
        chk(cudaMemcpyAsync(p.deconvd, decd.data(), sizeof(double) * decd.size(), cudaMemcpyHostToDevice,
                            p.stream));
    }
    if (!empties.empty())
        chk(cudaMemcpyAsync(p.empty_off, empties.data(), sizeof(long long) * empties.size(),
                            cudaMemcpyHostToDevice, p.stream));
    chk(cudaMemsetAsync(p.err, 0, sizeof(int) * 4, p.stream));
    if (xbytes) {
        long long total = (long long)d * M;
        int blocks = (int)std::min<long long>(4096, (total + 255) / 256);
        if (p.precision == ANOVA_PREC_F64)
            wrap_nodes_f64<<<blocks, 256, 0, p.stream>>>((const double *)x_dev, (double *)p.x, total,
                                                          cosine ? 0.5 : 1.0);
        else
            wrap_nodes_f32<<<blocks, 256, 0, p.stream>>>((const float *)x_dev, (float *)p.x, total,
                                                          cosine ? 0.5f : 1.0f);
        chk(cudaGetLastError());
    }
    if (e == cudaSuccess && p.precision == ANOVA_PREC_F64) chk(cuda_err_of(build_window_tables_f64(p)));
    if (e == cudaSuccess) chk(cuda_err_of(sort_nodes_by_cell(p)));
    if (e == cudaSuccess) chk(cuda_err_of(set_active_terms(p, nullptr)));
    chk(cudaStreamSynchronize(p.stream));
    // wins vector is copied; keep host term table
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    guard.h = nullptr;
    *out = h;
    return ANOVA_OK;
}

int anova_plan_create(anova_plan_t *out, int d, int64_t M, const void *x_dev, int n_terms,
                      const int32_t *term_dims, const int32_t *bandwidth, const anova_plan_options *opts,
                      void *stream) {
    try {
        return plan_create(out, d, M, x_dev, n_terms, term_dims, bandwidth, opts, stream);
    } catch (const std::bad_alloc &) {
        return ANOVA_ERR_NOMEM;
    } catch (...) {
        return ANOVA_ERR_CUDA;
    }
}

int anova_debug_fail_allocation(int k) {
    if (k < 0) return ANOVA_ERR_INVALID;
    g_fail_after.store(k);
    return ANOVA_OK;
}

void anova_plan_destroy(anova_plan_t plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->p.stream);
    free_plan(plan->p);
    delete plan;
}

int64_t anova_num_coeffs(anova_plan_t plan) { return plan ? plan->p.n_coeffs : -1; }

int anova_term_offset(anova_plan_t plan, int u, int64_t *off, int64_t *len) {
    if (!plan || u < 0 || u >= plan->p.n_user_terms) return ANOVA_ERR_INVALID;
    if (off) *off = plan->p.h_user_off[u];
    if (len) *len = plan->p.h_user_len[u];
    return ANOVA_OK;
}

int anova_term_grid(anova_plan_t plan, int u, int *n, int *m_col, int *m_row) {
    if (!plan || u < 0 || u >= plan->p.n_user_terms) return ANOVA_ERR_INVALID;
    if (n) *n = plan->p.h_user_n[u];
    if (m_col) *m_col = plan->p.h_user_mc[u];
    if (m_row) *m_row = plan->p.h_user_mr[u];
    return ANOVA_OK;
}

int grouped_trafo(anova_plan_t plan, const void *fhat_dev, void *f_dev) {
    if (!plan) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (p.M > 0 && !f_dev) return ANOVA_ERR_INVALID;
    if (p.n_coeffs > 0 && !fhat_dev) return ANOVA_ERR_INVALID;
    if (p.M == 0) return ANOVA_OK;
    cudaGetLastError();
    if (p.precision == ANOVA_PREC_F64) return launch_trafo_f64(p, (const double2 *)fhat_dev, (double2 *)f_dev);
    return launch_trafo_f32(p, (const float2 *)fhat_dev, (float2 *)f_dev);
}

int grouped_adjoint(anova_plan_t plan, const void *y_dev, void *fhat_dev) {
    if (!plan) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (!fhat_dev) return ANOVA_ERR_INVALID;
    if (p.M > 0 && !y_dev) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    if (p.precision == ANOVA_PREC_F64) return launch_adjoint_f64(p, (const double2 *)y_dev, (double2 *)fhat_dev);
    return launch_adjoint_f32(p, (const float2 *)y_dev, (float2 *)fhat_dev);
}

}  // extern "C"
