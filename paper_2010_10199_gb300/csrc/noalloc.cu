// Allocation-free forward grouped transform.
//
// Some callers cannot allocate device memory at the point where they need a
// transform: a host application whose device memory is already fully carved
// up by its own pool allocator, a plug-in that may only run inside a callback
// with a fixed memory budget, or a latency-critical loop where cudaMalloc and
// cudaFree (which synchronise the device) are not acceptable.  For them this
// file offers grouped_trafo_noalloc: the same computation as grouped_trafo
// with default options (FP32, Kaiser--Bessel window, sigma = 2), but with no
// plan object and no allocation.  Everything the transform needs besides the
// caller's inputs and outputs -- term table, window polynomials,
// deconvolution factors, a wrapped copy of the nodes and the oversampled
// grids -- lives in one file-scope __device__ array of NOALLOC_SCRATCH_BYTES.
// Every GPU that loads the library holds that array until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace agft {

constexpr size_t NOALLOC_SCRATCH_BYTES = 32u << 20;   // 32 MiB
constexpr int NOALLOC_MAX_TERMS = 4096;
constexpr int NOALLOC_MAX_WINDOWS = 64;
constexpr int NOALLOC_MAX_DECONV = 1 << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// host staging tables (static storage: built per call without heap allocation)
static Window s_windows[NOALLOC_MAX_WINDOWS];
static int s_wkey[NOALLOC_MAX_WINDOWS][3];
static float s_deconv[NOALLOC_MAX_DECONV];
static long long s_empty[NOALLOC_MAX_TERMS];
static int s_order[NOALLOC_MAX_TERMS];
static int s_sched[NOALLOC_MAX_TERMS];
static int s_act[NOALLOC_MAX_TERMS];
static ActRec s_rec[NOALLOC_MAX_TERMS];
static std::mutex s_lock;
static void *s_dev_ptr[NOALLOC_MAX_DEVICES];

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace agft

using namespace agft;

extern "C" int grouped_trafo_noalloc(int d, int64_t M, const float *x_dev, int n_terms, const int32_t *term_dims,
                                     const int32_t *bandwidth, const anova_cfloat *fhat_dev, anova_cfloat *f_dev,
                                     void *stream) {
    if (d < 1 || M < 0 || M >= (1LL << 31) || n_terms < 1 || !term_dims || !bandwidth) return ANOVA_ERR_INVALID;
    if (n_terms > NOALLOC_MAX_TERMS) return ANOVA_ERR_UNSUPPORTED;
    if (M > 0 && (!x_dev || !f_dev || !fhat_dev)) return ANOVA_ERR_INVALID;
    const int mc = 4, mr = 3;
    const double sigma = 2.0;
    for (int i = 0; i < n_terms; ++i) {
        const int32_t *t = term_dims + 3 * i;
        int ord = 0;
        for (int j = 0; j < 3; ++j) {
            if (t[j] < 0) {
                for (int l = j; l < 3; ++l)
                    if (t[l] >= 0) return ANOVA_ERR_INVALID;
                break;
            }
            if (t[j] >= d || (j > 0 && t[j] <= t[j - 1])) return ANOVA_ERR_INVALID;
            ++ord;
        }
        if (ord > 0 && (bandwidth[i] < 2 || bandwidth[i] % 2)) return ANOVA_ERR_INVALID;
        if (ord > 0 && bandwidth[i] > 4096) return ANOVA_ERR_UNSUPPORTED;
    }
    if (M == 0) return ANOVA_OK;
    cudaGetLastError();   // do not report an earlier, unrelated error
    cudaStream_t st = (cudaStream_t)stream;
    // The table uploads below read host staging arrays that the next call
    // overwrites, so a captured call would replay another call's tables:
    // refuse a capturing stream before anything is enqueued.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return ANOVA_ERR_UNSUPPORTED;
    }
    if (cs != cudaStreamCaptureStatusNone) return ANOVA_ERR_UNSUPPORTED;

    std::lock_guard<std::mutex> guard(s_lock);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return ANOVA_ERR_UNSUPPORTED;
    // one-time set-up per device (with that device current): the device
    // address of the scratch array; host code must not use the symbol itself
    if (!s_dev_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        s_dev_ptr[dev] = ptr;
    }
    unsigned char *base = (unsigned char *)s_dev_ptr[dev];

    // term layout and schedule (same rules as anova_plan_create with default options)
    static long long s_uoff[NOALLOC_MAX_TERMS], s_ulen[NOALLOC_MAX_TERMS];
    long long off = 0;
    int n_empty = 0, n_sched = 0;
    for (int i = 0; i < n_terms; ++i) {
        const int32_t *t = term_dims + 3 * i;
        int ord = (t[0] >= 0) + (t[1] >= 0) + (t[2] >= 0);
        s_order[i] = ord;
        long long len = 1;
        for (int j = 0; j < ord; ++j) len *= (bandwidth[i] - 1);
        if (ord == 0)
            s_empty[n_empty++] = off;
        else
            s_sched[n_sched++] = i;
        s_uoff[i] = off;
        s_ulen[i] = len;
        off += len;
    }
    // std::sort (no temporary buffer) with the index as final key equals a stable sort
    std::sort(s_sched, s_sched + n_sched, [&](int a, int b) {
        const int32_t *ta = term_dims + 3 * a, *tb = term_dims + 3 * b;
        if (ta[0] != tb[0]) return ta[0] < tb[0];
        if (s_order[a] != s_order[b]) return s_order[a] < s_order[b];
        if (ta[1] != tb[1]) return ta[1] < tb[1];
        if (ta[2] != tb[2]) return ta[2] < tb[2];
        return a < b;
    });
    int pitch2 = 8;
    for (int s = 0; s < n_sched; ++s)
        if (s_order[s_sched[s]] == 2)
            pitch2 = std::max(pitch2, row_stride(fft_size(bandwidth[s_sched[s]], sigma) + 2 * (mc - 1) + 1));
    int n_win = 0;
    auto get_window = [&](int m, int n, int N) -> int {
        for (int w = 0; w < n_win; ++w)
            if (s_wkey[w][0] == m && s_wkey[w][1] == n && s_wkey[w][2] == N) return w;
        if (n_win >= NOALLOC_MAX_WINDOWS) return -1;
        std::memset(&s_windows[n_win], 0, sizeof(Window));
        window_polys(s_windows[n_win], m, M_PI * (2.0 - (double)N / n));
        s_wkey[n_win][0] = m;
        s_wkey[n_win][1] = n;
        s_wkey[n_win][2] = N;
        return n_win++;
    };
    long long goff = 0, maxbytes = 16;
    int max_fft = 1, n_dec = 0;
    static Term s_sched_terms[NOALLOC_MAX_TERMS];
    for (int s = 0; s < n_sched; ++s) {
        const int i = s_sched[s];
        const int32_t *t = term_dims + 3 * i;
        Term T;
        std::memset(&T, 0, sizeof(T));
        T.sort_slot = -1;
        T.order = s_order[i];
        T.col = t[T.order - 1];
        T.row0 = T.order >= 2 ? t[0] : -1;
        T.row1 = T.order >= 3 ? t[1] : -1;
        T.N = bandwidth[i];
        T.n = fft_size(T.N, sigma);
        T.rows = 1;
        for (int j = 1; j < T.order; ++j) T.rows *= T.n;
        T.mc = mc;
        T.mr = T.order > 1 ? mr : 0;
        if (T.order <= 2) {
            T.hc = mc - 1;
            T.hr = T.order == 2 ? mr - 1 : 0;
            T.erows = T.order == 2 ? T.n + 2 * T.hr + 1 : 1;
            T.stride = T.order == 2 ? pitch2 : row_stride(T.n + 2 * T.hc + 1);
        } else {
            T.erows = T.rows;
            T.stride = row_stride(T.n);
        }
        T.wc = get_window(T.mc, T.n, T.N);
        T.wr = T.order > 1 ? get_window(T.mr, T.n, T.N) : T.wc;
        if (T.wc < 0 || T.wr < 0) return ANOVA_ERR_UNSUPPORTED;
        T.grid_off = goff;
        long long elems = ((long long)T.erows * T.stride + 1) & ~1LL;
        T.grid_bytes = elems * 8;
        goff += elems;
        maxbytes = std::max(maxbytes, T.grid_bytes);
        long long fe = 1;
        for (int j = 0; j < T.order; ++j) fe *= T.n;
        if (fe * 16 > 200 * 1024 || T.grid_bytes > 100 * 1024) return ANOVA_ERR_UNSUPPORTED;
        max_fft = (int)std::max<long long>(max_fft, fe);
        T.coef_off = s_uoff[i];
        T.coef_len = s_ulen[i];
        T.user_index = i;
        const double b = M_PI * (2.0 - (double)T.N / T.n);
        if (n_dec + 2 * (T.N - 1) > NOALLOC_MAX_DECONV) return ANOVA_ERR_UNSUPPORTED;
        T.dc_off = n_dec;
        for (int q = 0; q < T.N - 1; ++q) {
            int k = q < T.N / 2 ? q - T.N / 2 : q - T.N / 2 + 1;
            s_deconv[n_dec++] = (float)deconv_factor(k, T.n, T.mc, b);
        }
        T.dr_off = T.dc_off;
        if (T.order > 1) {
            T.dr_off = n_dec;
            for (int q = 0; q < T.N - 1; ++q) {
                int k = q < T.N / 2 ? q - T.N / 2 : q - T.N / 2 + 1;
                s_deconv[n_dec++] = (float)deconv_factor(k, T.n, T.mr, b);
            }
        }
        s_sched_terms[s] = T;
    }
    for (int s = 0; s < n_sched; ++s) {
        Term &T = s_sched_terms[s];
        T.new_rowgroup = 1;
        if (T.order == 2 && s > 0) {
            const Term &P = s_sched_terms[s - 1];
            if (P.order == 2 && P.row0 == T.row0 && P.wr == T.wr && P.n == T.n) T.new_rowgroup = 0;
        }
        s_act[s] = s;
        s_rec[s] = make_act_rec(T, s, T.new_rowgroup);
    }

    // carve the scratch array; reject what does not fit
    size_t o_terms = 0;
    size_t o_win = align256(o_terms + sizeof(Term) * std::max(1, n_sched));
    size_t o_dec = align256(o_win + sizeof(Window) * std::max(1, n_win));
    size_t o_empty = align256(o_dec + sizeof(float) * std::max(1, n_dec));
    size_t o_act = align256(o_empty + sizeof(long long) * std::max(1, n_empty));
    size_t o_ng = align256(o_act + sizeof(int) * std::max(1, n_sched));
    size_t o_err = align256(o_ng + sizeof(ActRec) * std::max(1, n_sched));
    size_t o_x = align256(o_err + 16);
    size_t o_grid = align256(o_x + sizeof(float) * (size_t)d * (size_t)M);
    size_t total = o_grid + (size_t)goff * 8;
    if (total > NOALLOC_SCRATCH_BYTES) return ANOVA_ERR_UNSUPPORTED;

    // upload the tables; clear the error word (the array keeps the last call's contents)
    if (n_sched) e = cudaMemcpyAsync(base + o_terms, s_sched_terms, sizeof(Term) * n_sched, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_win)
        e = cudaMemcpyAsync(base + o_win, s_windows, sizeof(Window) * n_win, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_dec)
        e = cudaMemcpyAsync(base + o_dec, s_deconv, sizeof(float) * n_dec, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_empty)
        e = cudaMemcpyAsync(base + o_empty, s_empty, sizeof(long long) * n_empty, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_sched)
        e = cudaMemcpyAsync(base + o_act, s_act, sizeof(int) * n_sched, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_sched)
        e = cudaMemcpyAsync(base + o_ng, s_rec, sizeof(ActRec) * n_sched, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_err, 0, 16, st);
    if (e != cudaSuccess) return cuda_status(e);
    const long long total_x = (long long)d * M;
    wrap_nodes_f32<<<(int)std::min<long long>(4096, (total_x + 255) / 256), 256, 0, st>>>(
        x_dev, (float *)(base + o_x), total_x, 1.0f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);

    // a plan view onto the scratch array; the regular launch path does the rest
    Plan p;
    std::memset(&p, 0, sizeof(p));
    p.stream = st;
    p.device = dev;
    p.precision = ANOVA_PREC_F32;
    p.d = d;
    p.M = M;
    p.n_terms = n_sched;
    p.n_empty = n_empty;
    p.h_terms = s_sched_terms;
    p.x = base + o_x;
    p.terms = (Term *)(base + o_terms);
    p.windows = (Window *)(base + o_win);
    p.n_windows = n_win;
    p.deconv = (float *)(base + o_dec);
    p.empty_off = (long long *)(base + o_empty);
    p.grids = base + o_grid;
    p.grid_elems = goff;
    p.max_grid_bytes = maxbytes;
    p.max_fft_elems = max_fft;
    p.pitch2 = pitch2;
    p.err = (int *)(base + o_err);
    p.act = (int *)(base + o_act);
    p.act_rec = (ActRec *)(base + o_ng);
    p.n_act = n_sched;
    p.h_act = s_act;
    cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (p.sm_count <= 0) p.sm_count = 1;
    return launch_trafo_f32(p, (const float2 *)fhat_dev, (float2 *)f_dev);
}
