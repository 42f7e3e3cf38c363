// Group-screening MLP: forward, backward and Adam on the device (FP32).
//
// No counterpart in the paper.  The network proposes which ANOVA groups will
// be nonzero at the next lambda of a group-lasso path (eq. (alligatoah),
// Sec. 4.2); the screened path driver in screen.cu checks every proposal with
// the full KKT conditions, so the network only changes cost, never the result.
//
//   h1 = relu(X W1 + b1), h2 = relu(h1 W2 + b2), z = h2 W3 + b3, p = sigmoid(z)
//   loss = mean_g [pw y softplus(-z) + (1 - y) softplus(z)]
//
// Row-major storage: X [G][F], W1 [F][H], W2 [H][H], W3 [H][1].  The matrix
// products use one tiled shared-memory SIMT kernel (the layers are far too
// small for the tensor-core path to matter).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace agft {

struct Mlp {
    int F = 0, H = 0;
    int cap = 0;                  // samples the activation buffers hold
    float *params = nullptr;      // W1 | b1 | W2 | b2 | W3 | b3
    float *grads = nullptr;
    float *m = nullptr, *v = nullptr;   // Adam moments
    float *a1 = nullptr, *a2 = nullptr, *h1 = nullptr, *h2 = nullptr, *z = nullptr;
    float *d1 = nullptr, *d2 = nullptr, *dz = nullptr;
    double *loss = nullptr;       // [2] loss accumulator
    long long step = 0;
    cudaStream_t stream = nullptr;
    size_t np() const { return (size_t)F * H + H + (size_t)H * H + H + H + 1; }
    float *W1() { return params; }
    float *b1() { return params + (size_t)F * H; }
    float *W2() { return b1() + H; }
    float *b2() { return W2() + (size_t)H * H; }
    float *W3() { return b2() + H; }
    float *b3() { return W3() + H; }
    float *gW1() { return grads; }
    float *gb1() { return grads + (size_t)F * H; }
    float *gW2() { return gb1() + H; }
    float *gb2() { return gW2() + (size_t)H * H; }
    float *gW3() { return gb2() + H; }
    float *gb3() { return gW3() + H; }
};

// C[M][N] = beta * C + op(A) op(B) (+ bias[N]); op(A) is [M][K], op(B) [K][N].
// ta: A stored [K][M]; tb: B stored [N][K].  16 x 16 tiles.
constexpr int TS = 16;
__global__ void k_gemm(int Mr, int Nc, int K, const float *__restrict__ A, int ta, const float *__restrict__ B, int tb,
                       float *C, float beta, const float *__restrict__ bias) {
    __shared__ float As[TS][TS + 1], Bs[TS][TS + 1];
    const int row = blockIdx.y * TS + threadIdx.y, col = blockIdx.x * TS + threadIdx.x;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TS) {
        int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        float av = 0.f, bv = 0.f;
        if (row < Mr && ka < K) av = ta ? A[(size_t)ka * Mr + row] : A[(size_t)row * K + ka];
        if (col < Nc && kb < K) bv = tb ? B[(size_t)col * K + kb] : B[(size_t)kb * Nc + col];
        As[threadIdx.y][threadIdx.x] = av;
        Bs[threadIdx.y][threadIdx.x] = bv;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TS; ++k) acc = fmaf(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
        __syncthreads();
    }
    if (row < Mr && col < Nc) {
        float c = beta != 0.f ? beta * C[(size_t)row * Nc + col] : 0.f;
        C[(size_t)row * Nc + col] = c + acc + (bias ? bias[col] : 0.f);
    }
}

static void gemm(cudaStream_t s, int Mr, int Nc, int K, const float *A, int ta, const float *B, int tb, float *C,
                 float beta, const float *bias) {
    dim3 blk(TS, TS), grd((Nc + TS - 1) / TS, (Mr + TS - 1) / TS);
    k_gemm<<<grd, blk, 0, s>>>(Mr, Nc, K, A, ta, B, tb, C, beta, bias);
}

__global__ void k_relu(const float *a, float *h, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        h[i] = fmaxf(a[i], 0.f);
}

__global__ void k_relu_grad(float *d, const float *a, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) d[i] = 0.f;
}

__device__ __forceinline__ float softplusf(float z) { return z > 20.f ? z : (z < -20.f ? expf(z) : log1pf(expf(z))); }
__device__ __forceinline__ float sigmoidf_(float z) { return 0.5f * (1.f + tanhf(0.5f * z)); }

// dz = ((1 - y) s - pw y (1 - s)) / G and the loss sum (FP64)
__global__ void k_bce(const float *z, const float *y, int G, float pw, float *dz, double *loss) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        float zi = z[i], yi = y[i], s = sigmoidf_(zi);
        dz[i] = ((1.f - yi) * s - pw * yi * (1.f - s)) / (float)G;
        acc += (double)(pw * yi * softplusf(-zi) + (1.f - yi) * softplusf(zi));
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0]);
}

// column sums of d [G][N] into out[N] (bias gradients)
__global__ void k_colsum(const float *d, int G, int N, float *out) {
    const int c = blockIdx.x;
    __shared__ float sh[256];
    float acc = 0.f;
    for (int g = threadIdx.x; g < G; g += blockDim.x) acc += d[(size_t)g * N + c];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

__global__ void k_sigmoid(const float *z, float *p, int G) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) p[i] = sigmoidf_(z[i]);
}

// Adam (Kingma and Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, step with bias correction
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static int grid1(long long n) { return (int)std::max<long long>(1, std::min<long long>(4096, (n + 255) / 256)); }

static int ensure_cap(Mlp &N, int G) {
    if (G <= N.cap) return ANOVA_OK;
    float *bufs[8] = {N.a1, N.a2, N.h1, N.h2, N.z, N.d1, N.d2, N.dz};
    for (float *b : bufs)
        if (b) cudaFree(b);
    int cap = std::max(G, 1024);
    size_t gh = (size_t)cap * N.H * sizeof(float), g1 = (size_t)cap * sizeof(float);
    cudaError_t e = cudaSuccess;
    auto A = [&](float **p, size_t b) {
        *p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(p, b);
    };
    A(&N.a1, gh);
    A(&N.a2, gh);
    A(&N.h1, gh);
    A(&N.h2, gh);
    A(&N.z, g1);
    A(&N.d1, gh);
    A(&N.d2, gh);
    A(&N.dz, g1);
    if (e != cudaSuccess) {
        N.cap = 0;
        return cuda_status(e);
    }
    N.cap = cap;
    return ANOVA_OK;
}

static void forward(Mlp &N, const float *X, int G) {
    cudaStream_t s = N.stream;
    const long long gh = (long long)G * N.H;
    gemm(s, G, N.H, N.F, X, 0, N.W1(), 0, N.a1, 0.f, N.b1());
    k_relu<<<grid1(gh), 256, 0, s>>>(N.a1, N.h1, gh);
    gemm(s, G, N.H, N.H, N.h1, 0, N.W2(), 0, N.a2, 0.f, N.b2());
    k_relu<<<grid1(gh), 256, 0, s>>>(N.a2, N.h2, gh);
    gemm(s, G, 1, N.H, N.h2, 0, N.W3(), 0, N.z, 0.f, N.b3());
}

static void backward(Mlp &N, const float *X, const float *y, int G, float pw) {
    cudaStream_t s = N.stream;
    const long long gh = (long long)G * N.H;
    cudaMemsetAsync(N.loss, 0, sizeof(double), s);
    k_bce<<<std::min(256, (G + 255) / 256), 256, 0, s>>>(N.z, y, G, pw, N.dz, N.loss);
    // layer 3
    gemm(s, N.H, 1, G, N.h2, 1, N.dz, 0, N.gW3(), 0.f, nullptr);     // h2^T dz
    k_colsum<<<1, 256, 0, s>>>(N.dz, G, 1, N.gb3());
    gemm(s, G, N.H, 1, N.dz, 0, N.W3(), 1, N.d2, 0.f, nullptr);       // dz W3^T
    k_relu_grad<<<grid1(gh), 256, 0, s>>>(N.d2, N.a2, gh);
    // layer 2
    gemm(s, N.H, N.H, G, N.h1, 1, N.d2, 0, N.gW2(), 0.f, nullptr);    // h1^T dA2
    k_colsum<<<N.H, 256, 0, s>>>(N.d2, G, N.H, N.gb2());
    gemm(s, G, N.H, N.H, N.d2, 0, N.W2(), 1, N.d1, 0.f, nullptr);     // dA2 W2^T
    k_relu_grad<<<grid1(gh), 256, 0, s>>>(N.d1, N.a1, gh);
    // layer 1
    gemm(s, N.F, N.H, G, X, 1, N.d1, 0, N.gW1(), 0.f, nullptr);       // X^T dA1
    k_colsum<<<N.H, 256, 0, s>>>(N.d1, G, N.H, N.gb1());
}

}  // namespace agft

using namespace agft;

struct anova_mlp_s {
    Mlp n;
};

extern "C" {

int anova_mlp_create(anova_mlp_t *out, int n_features, int hidden, const float *params_host, void *stream) {
    if (!out || n_features < 1 || hidden < 1 || hidden > 4096 || !params_host) return ANOVA_ERR_INVALID;
    *out = nullptr;
    cudaGetLastError();
    anova_mlp_s *h = new anova_mlp_s;
    Mlp &N = h->n;
    N.F = n_features;
    N.H = hidden;
    N.stream = (cudaStream_t)stream;
    const size_t np = N.np();
    cudaError_t e = cudaMalloc(&N.params, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N.grads, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N.m, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N.v, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N.loss, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(N.params, params_host, np * sizeof(float), cudaMemcpyHostToDevice, N.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(N.m, 0, np * sizeof(float), N.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(N.v, 0, np * sizeof(float), N.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(N.stream);
    if (e != cudaSuccess) {
        anova_mlp_destroy(h);
        return cuda_status(e);
    }
    *out = h;
    return ANOVA_OK;
}

void anova_mlp_destroy(anova_mlp_t mlp) {
    if (!mlp) return;
    Mlp &N = mlp->n;
    cudaStreamSynchronize(N.stream);
    float *b[] = {N.params, N.grads, N.m, N.v, N.a1, N.a2, N.h1, N.h2, N.z, N.d1, N.d2, N.dz};
    for (float *q : b)
        if (q) cudaFree(q);
    if (N.loss) cudaFree(N.loss);
    delete mlp;
}

int64_t anova_mlp_num_params(anova_mlp_t mlp) { return mlp ? (int64_t)mlp->n.np() : -1; }

int anova_mlp_get_params(anova_mlp_t mlp, float *params_host, float *grads_host) {
    if (!mlp) return ANOVA_ERR_INVALID;
    Mlp &N = mlp->n;
    cudaError_t e = cudaSuccess;
    if (params_host) e = cudaMemcpyAsync(params_host, N.params, N.np() * sizeof(float), cudaMemcpyDeviceToHost, N.stream);
    if (e == cudaSuccess && grads_host)
        e = cudaMemcpyAsync(grads_host, N.grads, N.np() * sizeof(float), cudaMemcpyDeviceToHost, N.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(N.stream);
    return cuda_status(e);
}

int anova_mlp_forward(anova_mlp_t mlp, const float *X_dev, int G, float *prob_dev) {
    if (!mlp || G < 0 || (G > 0 && (!X_dev || !prob_dev))) return ANOVA_ERR_INVALID;
    if (G == 0) return ANOVA_OK;
    cudaGetLastError();
    Mlp &N = mlp->n;
    int rc = ensure_cap(N, G);
    if (rc) return rc;
    forward(N, X_dev, G);
    k_sigmoid<<<grid1(G), 256, 0, N.stream>>>(N.z, prob_dev, G);
    return cuda_status(cudaGetLastError());
}

int anova_mlp_gradients(anova_mlp_t mlp, const float *X_dev, const float *y_dev, int G, float pos_weight,
                        double *loss_out) {
    if (!mlp || G < 1 || !X_dev || !y_dev) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Mlp &N = mlp->n;
    int rc = ensure_cap(N, G);
    if (rc) return rc;
    forward(N, X_dev, G);
    backward(N, X_dev, y_dev, G, pos_weight);
    double l = 0;
    cudaError_t e = cudaMemcpyAsync(&l, N.loss, sizeof(double), cudaMemcpyDeviceToHost, N.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(N.stream);
    if (loss_out) *loss_out = l / G;
    return cuda_status(e);
}

int anova_mlp_train(anova_mlp_t mlp, const float *X_dev, const float *y_dev, int n_samples, int batch, int epochs,
                    float lr, float pos_weight, double *loss_history) {
    if (!mlp || n_samples < 1 || batch < 1 || epochs < 1 || !X_dev || !y_dev || !(lr > 0)) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Mlp &N = mlp->n;
    const int B = std::min(batch, n_samples);
    int rc = ensure_cap(N, B);
    if (rc) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const long long np = (long long)N.np();
    for (int ep = 0; ep < epochs; ++ep) {
        double ep_loss = 0.0;
        for (int s0 = 0; s0 < n_samples; s0 += B) {
            const int G = std::min(B, n_samples - s0);
            const float *Xb = X_dev + (size_t)s0 * N.F;
            const float *yb = y_dev + s0;
            forward(N, Xb, G);
            backward(N, Xb, yb, G, pos_weight);
            N.step += 1;
            const float c1 = 1.f - powf(b1, (float)N.step), c2 = 1.f - powf(b2, (float)N.step);
            k_adam<<<grid1(np), 256, 0, N.stream>>>(N.params, N.grads, N.m, N.v, np, lr, b1, b2, eps, c1, c2);
            if (loss_history) {
                double l = 0;
                cudaMemcpyAsync(&l, N.loss, sizeof(double), cudaMemcpyDeviceToHost, N.stream);
                cudaError_t e = cudaStreamSynchronize(N.stream);
                if (e != cudaSuccess) return cuda_status(e);
                ep_loss += l;
            }
        }
        if (loss_history) loss_history[ep] = ep_loss / n_samples;
    }
    return cuda_status(cudaStreamSynchronize(N.stream));
}

}  // extern "C"
