/*
 * FP64 oracle for the grouped Fourier transform -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  It shares nothing with the CUDA path.
 *
 * What it computes is the plain definition, by direct summation:
 *
 *   forward  (Definition "grouped Fourier transform", Sec. 3, and the Fourier
 *            matrix of eq. (FM)):
 *       f_j = sum_{u in U} sum_{k in I_{N_u}^{u,d}} fhat_k exp(+2 pi i <k, x_j>)
 *
 *   adjoint  (the stacked adjoint right after the error remark in Sec. 3):
 *       (F^H y)_k = sum_j y_j exp(-2 pi i <k, x_j>)
 *
 * Because supp k = u, <k, x_j> = sum_{t in u} k_t x_{j,t}, and the exponential
 * factorises exactly: exp(2 pi i <k,x>) = prod_{t in u} exp(2 pi i k_t x_t).
 * For each node and each coordinate of a term the code tabulates
 * exp(2 pi i k x_t) for the N_u - 1 nonzero k in I_{N_u} = [-N_u/2, N_u/2) (the
 * group of eq. (metallica), Remark "cardinality"), each entry from cos/sin of
 * 2 pi times the fractional part of k*x_t reduced in FP64, and multiplies the
 * table entries.  No window, no FFT, no blocking.
 *
 * Coefficient layout: blocks in term order; inside a block the multi-index over
 * the term's sorted coordinates is row-major, last coordinate fastest, and each
 * coordinate runs -N/2, ..., -1, 1, ..., N/2-1.  The empty term is the single
 * k = 0 coefficient.
 *
 * Complex vectors are interleaved (re, im) doubles.  Nodes are SoA [d][M].
 * Work is split across pthreads by outputs only (points for the forward,
 * terms for the adjoint), so every output's summation order is fixed and the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAX_ORDER 6

typedef struct {
    int d;
    int64_t M;
    const double *x;      /* [d][M] */
    int n_terms;
    const int32_t *order; /* |u| per term */
    const int32_t *dims;  /* [n_terms][MAX_ORDER], coordinate ids */
    const int32_t *N;     /* bandwidth per term */
    const int64_t *off;   /* coefficient offset per term */
    const double *in;     /* fhat (forward) or y (adjoint) */
    double *out;          /* f (forward) or F^H y (adjoint) */
    int64_t n_rows;       /* dense matrix: number of rows */
    int64_t n_cols;
    pthread_mutex_t lock;
    int64_t next;         /* next work item (point chunk or term) */
    int64_t n_items;
    int64_t chunk;
} job_t;

/* frequency value of position i in (I_N \ {0}) : -N/2..-1, 1..N/2-1 */
static inline int freq_of(int i, int N) { return (i < N / 2) ? i - N / 2 : i - N / 2 + 1; }

/* exp(2 pi i k x) with the argument reduced to [-1/2, 1/2] in FP64 */
static inline void cis(double kx, double *c, double *s) {
    double r = kx - nearbyint(kx);
    *c = cos(2.0 * M_PI * r);
    *s = sin(2.0 * M_PI * r);
}

/* per-coordinate tables for one node and one term: tab[t][i] = exp(2 pi i freq(i) x_t) */
static void tables(const job_t *J, int term, int64_t j, double *tab /* [MAX_ORDER][2*(N-1)] */) {
    int s = J->order[term], N = J->N[term];
    for (int t = 0; t < s; ++t) {
        double xt = J->x[(int64_t)J->dims[term * MAX_ORDER + t] * J->M + j];
        double *row = tab + (size_t)t * 2 * (N - 1);
        for (int i = 0; i < N - 1; ++i) cis((double)freq_of(i, N) * xt, &row[2 * i], &row[2 * i + 1]);
    }
}

/* product of table entries for multi-index idx */
static inline void prod_entry(const double *tab, int s, int N, const int *idx, double *pr, double *pi) {
    double re = 1.0, im = 0.0;
    for (int t = 0; t < s; ++t) {
        const double *e = tab + (size_t)t * 2 * (N - 1) + 2 * idx[t];
        double nr = re * e[0] - im * e[1];
        double ni = re * e[1] + im * e[0];
        re = nr;
        im = ni;
    }
    *pr = re;
    *pi = im;
}

/* advance a row-major multi-index (last fastest); returns 0 when done */
static inline int odometer(int *idx, int s, int N) {
    for (int t = s - 1; t >= 0; --t) {
        if (++idx[t] < N - 1) return 1;
        idx[t] = 0;
    }
    return 0;
}

static int64_t grab(job_t *J) {
    pthread_mutex_lock(&J->lock);
    int64_t it = J->next++;
    pthread_mutex_unlock(&J->lock);
    return it < J->n_items ? it : -1;
}

static int max_N(const job_t *J) {
    int m = 2;
    for (int u = 0; u < J->n_terms; ++u)
        if (J->N[u] > m) m = J->N[u];
    return m;
}

/* forward: items are chunks of points */
static void *fwd_worker(void *arg) {
    job_t *J = (job_t *)arg;
    double *tab = (double *)malloc(sizeof(double) * MAX_ORDER * 2 * (size_t)max_N(J));
    int64_t it;
    while ((it = grab(J)) >= 0) {
        int64_t j0 = it * J->chunk, j1 = j0 + J->chunk;
        if (j1 > J->M) j1 = J->M;
        for (int64_t j = j0; j < j1; ++j) {
            double ar = 0.0, ai = 0.0;
            for (int u = 0; u < J->n_terms; ++u) {
                const double *c = J->in + 2 * J->off[u];
                int s = J->order[u], N = J->N[u];
                if (s == 0) {
                    ar += c[0];
                    ai += c[1];
                    continue;
                }
                tables(J, u, j, tab);
                int idx[MAX_ORDER] = {0};
                int64_t q = 0;
                do {
                    double er, ei;
                    prod_entry(tab, s, N, idx, &er, &ei);
                    ar += c[2 * q] * er - c[2 * q + 1] * ei;
                    ai += c[2 * q] * ei + c[2 * q + 1] * er;
                    ++q;
                } while (odometer(idx, s, N));
            }
            J->out[2 * j] = ar;
            J->out[2 * j + 1] = ai;
        }
    }
    free(tab);
    return NULL;
}

/* adjoint: items are terms; every coefficient sums the nodes in order 0..M-1 */
static void *adj_worker(void *arg) {
    job_t *J = (job_t *)arg;
    double *tab = (double *)malloc(sizeof(double) * MAX_ORDER * 2 * (size_t)max_N(J));
    int64_t u;
    while ((u = grab(J)) >= 0) {
        int s = J->order[u], N = J->N[u];
        double *c = J->out + 2 * J->off[u];
        int64_t len = 1;
        for (int t = 0; t < s; ++t) len *= (N - 1);
        memset(c, 0, sizeof(double) * 2 * (size_t)len);
        for (int64_t j = 0; j < J->M; ++j) {
            double yr = J->in[2 * j], yi = J->in[2 * j + 1];
            if (s == 0) {
                c[0] += yr;
                c[1] += yi;
                continue;
            }
            tables(J, (int)u, j, tab);
            int idx[MAX_ORDER] = {0};
            int64_t q = 0;
            do {
                double er, ei;
                prod_entry(tab, s, N, idx, &er, &ei);
                /* y * conj(e) */
                c[2 * q] += yr * er + yi * ei;
                c[2 * q + 1] += yi * er - yr * ei;
                ++q;
            } while (odometer(idx, s, N));
        }
    }
    free(tab);
    return NULL;
}

/* dense Fourier matrix, row-major [M][n_cols]: items are rows */
static void *mat_worker(void *arg) {
    job_t *J = (job_t *)arg;
    double *tab = (double *)malloc(sizeof(double) * MAX_ORDER * 2 * (size_t)max_N(J));
    int64_t j;
    while ((j = grab(J)) >= 0) {
        double *row = J->out + 2 * j * J->n_cols;
        for (int u = 0; u < J->n_terms; ++u) {
            double *c = row + 2 * J->off[u];
            int s = J->order[u], N = J->N[u];
            if (s == 0) {
                c[0] = 1.0;
                c[1] = 0.0;
                continue;
            }
            tables(J, u, j, tab);
            int idx[MAX_ORDER] = {0};
            int64_t q = 0;
            do {
                prod_entry(tab, s, N, idx, &c[2 * q], &c[2 * q + 1]);
                ++q;
            } while (odometer(idx, s, N));
        }
    }
    free(tab);
    return NULL;
}

static int run(job_t *J, void *(*fn)(void *), int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    pthread_mutex_init(&J->lock, NULL);
    J->next = 0;
    int started = 0;
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[i], NULL, fn, J) == 0) ++started;
        else break;
    fn(J);
    for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J->lock);
    return 0;
}

static int check(int d, int n_terms, const int32_t *order, const int32_t *dims, const int32_t *N) {
    for (int u = 0; u < n_terms; ++u) {
        if (order[u] < 0 || order[u] > MAX_ORDER) return -1;
        if (order[u] > 0 && (N[u] < 2 || N[u] % 2)) return -2;
        for (int t = 0; t < order[u]; ++t)
            if (dims[u * MAX_ORDER + t] < 0 || dims[u * MAX_ORDER + t] >= d) return -3;
    }
    return 0;
}

int oracle_max_order(void) { return MAX_ORDER; }

int oracle_grouped_trafo(int d, int64_t M, const double *x, int n_terms, const int32_t *order,
                         const int32_t *dims, const int32_t *N, const int64_t *off,
                         const double *fhat, double *f, int n_threads) {
    int rc = check(d, n_terms, order, dims, N);
    if (rc) return rc;
    job_t J = {0};
    J.d = d; J.M = M; J.x = x; J.n_terms = n_terms; J.order = order; J.dims = dims; J.N = N;
    J.off = off; J.in = fhat; J.out = f;
    J.chunk = 64;
    J.n_items = (M + J.chunk - 1) / J.chunk;
    return run(&J, fwd_worker, n_threads);
}

int oracle_grouped_adjoint(int d, int64_t M, const double *x, int n_terms, const int32_t *order,
                           const int32_t *dims, const int32_t *N, const int64_t *off,
                           const double *y, double *fhat, int n_threads) {
    int rc = check(d, n_terms, order, dims, N);
    if (rc) return rc;
    job_t J = {0};
    J.d = d; J.M = M; J.x = x; J.n_terms = n_terms; J.order = order; J.dims = dims; J.N = N;
    J.off = off; J.in = y; J.out = fhat;
    J.n_items = n_terms;
    return run(&J, adj_worker, n_threads);
}

int oracle_fourier_matrix(int d, int64_t M, const double *x, int n_terms, const int32_t *order,
                          const int32_t *dims, const int32_t *N, const int64_t *off,
                          int64_t n_cols, double *F, int n_threads) {
    int rc = check(d, n_terms, order, dims, N);
    if (rc) return rc;
    job_t J = {0};
    J.d = d; J.M = M; J.x = x; J.n_terms = n_terms; J.order = order; J.dims = dims; J.N = N;
    J.off = off; J.out = F; J.n_cols = n_cols;
    J.n_items = M;
    return run(&J, mat_worker, n_threads);
}
