// Model selection and error measures on a coefficient vector, on the device.
//
// * Global sensitivity (Sobol) indices, eq. (gsi), Sec. 2: for the Fourier
//   partial sum S f = sum_u sum_{k in I_u} fhat_k exp(2 pi i <k, x>) the ANOVA
//   term of u is the block fhat_u, and by Parseval sigma^2(f_u) = ||fhat_u||^2
//   and sigma^2(f) = ||f||^2 - |c_0|^2 = sum over the non-empty blocks.
//   rho(u) = sigma^2(f_u) / sigma^2(f); rho(empty set) = 0.
// * The active set of eq. (activeset), Sec. 4: U* = {empty} u {u : rho(u) >
//   eps_|u|}, the terms kept for the re-solve with I_N(U*).
// * The relative L2 error of eq. (L2error) through Parseval's identity:
//   ||f - S f||^2 = ||f||^2 + sum_I |fhat_k - c_k|^2 - sum_I |c_k|^2, for a
//   function whose coefficients c_k on I and norm ||f||^2 are known.
// Every sum is FP64 and runs in a fixed order (one block per group; fixed
// RED_BLOCKS partials), so the results are reproducible.
#include <cmath>
#include <cstring>

#include "solver_kernels.cuh"

namespace agft {

// ||fhat_u||^2 per user term (one block per term)
template <typename C>
__global__ void k_group_energy(const C *__restrict__ f, const long long *goff, const long long *glen, double *e) {
    __shared__ double sh[32];
    const int u = blockIdx.x;
    const long long o = goff[u], m = glen[u];
    double a = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        const C v = f[o + i];
        a += (double)v.x * v.x + (double)v.y * v.y;
    }
    const double s = block_sum(a, sh);
    if (threadIdx.x == 0) e[u] = s;
}

// rho(u) = e_u / sum_{v non-empty} e_v and the active-set flags (one block)
__global__ void k_sobol(const double *e, const int *order, int G, double eps1, double eps2, double eps3, double *rho,
                        unsigned char *act) {
    __shared__ double sh[32];
    __shared__ double total;
    double a = 0.0;
    for (int u = threadIdx.x; u < G; u += blockDim.x)
        if (order[u] > 0) a += e[u];
    const double s = block_sum(a, sh);
    if (threadIdx.x == 0) total = s;
    __syncthreads();
    for (int u = threadIdx.x; u < G; u += blockDim.x) {
        const int o = order[u];
        const double r = o > 0 && total > 0.0 ? e[u] / total : 0.0;
        rho[u] = r;
        const double eps = o == 1 ? eps1 : o == 2 ? eps2 : eps3;
        act[u] = (o == 0 || r > eps) ? 1 : 0;
    }
}

// partials of sum |fhat - c|^2 (slot 0) and sum |c|^2 (slot 1), RED_BLOCKS blocks
template <typename C>
__global__ void k_l2_parts(const C *__restrict__ fhat, const C *__restrict__ c, long long n, double *part) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const C f = fhat[i], t = c[i];
        const double dx = (double)f.x - (double)t.x, dy = (double)f.y - (double)t.y;
        a += dx * dx + dy * dy;
        b += (double)t.x * t.x + (double)t.y * t.y;
    }
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sa;
        part[RED_BLOCKS + blockIdx.x] = sb;
    }
}

// relative error sqrt(max(0, ||f||^2 + red[0] - red[1]) / ||f||^2) into red[2]
__global__ void k_l2_finish(SolverState *st, double norm2) {
    const double e2 = norm2 + st->red[0] - st->red[1];
    st->red[2] = sqrt(fmax(e2, 0.0) / norm2);
}

template <typename C>
static int sobol_impl(Plan &p, const C *fhat, double *rho_out, const double *eps, uint8_t *active_out) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    cudaStream_t s = p.stream;
    const int G = p.n_user_terms;
    k_group_energy<C><<<G, 256, 0, s>>>(fhat, W->goff, W->glen, W->gnorm);
    k_sobol<<<1, 256, 0, s>>>(W->gnorm, W->gorder, G, eps ? eps[0] : 0.0, eps ? eps[1] : 0.0, eps ? eps[2] : 0.0,
                              W->grho, W->gact);
    cudaError_t e = cudaMemcpyAsync(rho_out, W->grho, sizeof(double) * G, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && eps && active_out)
        e = cudaMemcpyAsync(active_out, W->gact, G, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e == cudaSuccess ? cudaGetLastError() : e);
}

template <typename C>
static int l2_impl(Plan &p, const C *fhat, const C *c, double norm2, double *err) {
    int rc;
    SolverWork *W = get_work(p, rc);
    if (!W) return rc;
    StreamScope scope(p, W);
    cudaStream_t s = p.stream;
    SolverState z;
    std::memset(&z, 0, sizeof(z));
    cudaMemcpyAsync(W->st, &z, sizeof(z), cudaMemcpyHostToDevice, s);
    k_l2_parts<C><<<RED_BLOCKS, RED_THREADS, 0, s>>>(fhat, c, p.n_coeffs, W->part);
    finish_sums<<<1, 256, 0, s>>>(W->st, W->part, 2);
    k_l2_finish<<<1, 1, 0, s>>>(W->st, norm2);
    SolverState h;
    cudaError_t e = cudaMemcpyAsync(&h, W->st, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    *err = h.red[2];
    return ANOVA_OK;
}

}  // namespace agft

using namespace agft;

extern "C" {

int anova_sobol_indices(anova_plan_t plan, const void *fhat_dev, double *rho_out, const double *eps_by_order,
                        uint8_t *active_out) {
    if (!plan || !fhat_dev || !rho_out) return ANOVA_ERR_INVALID;
    if (eps_by_order && !active_out) return ANOVA_ERR_INVALID;
    if (eps_by_order)
        for (int i = 0; i < 3; ++i)
            if (!(eps_by_order[i] >= 0.0)) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Plan &p = plan->p;
    if (p.precision == ANOVA_PREC_F64)
        return sobol_impl<double2>(p, (const double2 *)fhat_dev, rho_out, eps_by_order, active_out);
    return sobol_impl<float2>(p, (const float2 *)fhat_dev, rho_out, eps_by_order, active_out);
}

int anova_l2_error(anova_plan_t plan, const void *fhat_dev, const void *c_dev, double norm2, double *err_out) {
    if (!plan || !fhat_dev || !c_dev || !err_out || !(norm2 > 0.0)) return ANOVA_ERR_INVALID;
    cudaGetLastError();
    Plan &p = plan->p;
    if (p.precision == ANOVA_PREC_F64)
        return l2_impl<double2>(p, (const double2 *)fhat_dev, (const double2 *)c_dev, norm2, err_out);
    return l2_impl<float2>(p, (const float2 *)fhat_dev, (const float2 *)c_dev, norm2, err_out);
}

}  // extern "C"
