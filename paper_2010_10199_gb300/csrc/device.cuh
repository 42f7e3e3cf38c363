// Device helpers: window evaluation, bulk async copies with bounded mbarrier
// waits, and the shared-memory mixed-radix FFT used for the oversampled grids.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "internal.cuh"

namespace agft {

// ---------------------------------------------------------- grid elements --

// Storage type of an FP32-computing plan's grids: complex FP32 (float2) or a
// pair of 16-bit floats (FP16 or BF16); values are widened to FP32 on load and
// rounded to nearest on store, every sum stays in FP32.
template <typename G>
struct GridEl;
template <>
struct GridEl<float2> {
    static __device__ __forceinline__ float2 load(float2 v) { return v; }
    static __device__ __forceinline__ float2 store(float a, float b) { return make_float2(a, b); }
};
template <>
struct GridEl<__half2> {
    static __device__ __forceinline__ float2 load(__half2 v) { return __half22float2(v); }
    static __device__ __forceinline__ __half2 store(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct GridEl<__nv_bfloat162> {
    static __device__ __forceinline__ float2 load(__nv_bfloat162 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ __nv_bfloat162 store(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

// ------------------------------------------------------------ cosine terms --
//
// A term of the half-period cosine system (Sec. 5) runs on the exponential
// grids: prod_t cos(pi k_t x_t) = 2^{-s} sum over sign patterns eps of
// exp(2 pi i <eps k, x / 2>), so with the nodes halved (plan time) its block
// coefficient fhat_k, k in {1..N/2-1}^s (N the term's doubled bandwidth),
// stands for 2^{-s/2} fhat_k at each of the 2^s exponential frequencies eps k,
// and the adjoint's coefficient is 2^{-s/2} times the sum over those
// frequencies.  cos_decode: block position q -> k (row-major, last axis
// fastest); cos_mirror: grid position of sign pattern sg (bit t negates axis
// t; negative frequencies at k + n) and the product of its deconvolution
// factors (column table on the last axis, row table on the others).
__device__ __forceinline__ void cos_decode(long long q, int s, int N, int (&k)[3]) {
    const int nc = N / 2 - 1;
    for (int t = s - 1; t >= 0; --t) {
        k[t] = (int)(q % nc) + 1;
        q /= nc;
    }
}

template <typename R>
__device__ __forceinline__ int cos_mirror(const int (&k)[3], int s, int sg, int N, int n, const R *deconv, int dc_off,
                                          int dr_off, R &D) {
    int pos = 0, mul = 1;
    for (int t = s - 1; t >= 0; --t) {
        const int kt = (sg >> t) & 1 ? -k[t] : k[t];
        const int it = kt < 0 ? kt + N / 2 : kt + N / 2 - 1;   // index in I_N minus {0}
        pos += (kt < 0 ? kt + n : kt) * mul;
        mul *= n;
        D *= (t == s - 1) ? deconv[dc_off + it] : deconv[dr_off + it];
    }
    return pos;
}

// 2^{-s/2}
__host__ __device__ __forceinline__ double cos_amp(int s) {
    return s == 1 ? 0.70710678118654752440 : s == 2 ? 0.5 : 0.35355339059327376220;
}

// ---- packed FP32 pairs ----
//
// sm_100-class GPUs execute two FP32 fused multiply-adds of one lane in one
// instruction (fma.rn.f32x2 on a 64-bit register pair) at the same FMA rate,
// which halves the issue slots of independent pairs of operations; each half
// rounds exactly as the scalar fmaf does.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------- windows --

// ---- TF32 tensor-core products with FP32-level accuracy ----
//
// The fragment layouts of mma.m16n8k8 with TF32 operands (PTX ISA), lane =
// 4 g + t: A (16 x 8) a0 = A[g][t], a1 = A[g + 8][t], a2 = A[g][t + 4],
// a3 = A[g + 8][t + 4]; B (8 x 8) b0 = B[t][g], b1 = B[t + 4][g]; C, D
// (16 x 8) d0 = D[g][2t], d1 = D[g][2t + 1], d2 = D[g + 8][2t],
// d3 = D[g + 8][2t + 1].  A product a b of FP32 values is taken as
// ah bh + ah bl + al bh with x = xh + xl split below.
// x = hi + lo for finite x: hi keeps the sign, the exponent and the leading
// 10 mantissa bits of x rounded half away from zero (adding half a unit of
// the 10th bit to the bit pattern carries into the exponent where it should),
// lo = x - hi is exact in FP32; the tensor core reads the leading 10 mantissa
// bits of lo (error below 2^-21 |x|)
__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// The same split for two values at once in three packed operations (instead
// of two integer and one FP32 operation per value): c = fl(x + 2^13 x) =
// fl(8193 x), hi = c - 2^13 x (exact: one fma), lo = x - hi (exact: the
// rounding error of c).  ulp(c) >= 2^13 ulp(x), so hi is a multiple of
// 2^13 ulp(x) no larger than 2 |x| in magnitude: at most 11 significant
// bits, exact in TF32.  |lo| <= ulp(c) / 2 <= 2^-10 |x| (2^-11 |x| unless the
// mantissa of x is within 2^-13 of 2), and the tensor core's truncation of lo
// errs by less than 2^-20 |x|.  Finite |x| below 2^114 (c must not overflow).
// Written with fma rather than as Veltkamp's c - (c - x): in a probe of the
// packed subtraction form the compiled code returned hi = x.
__device__ __forceinline__ void split_tf32_x2(f32x2 x, unsigned &h0, unsigned &l0, unsigned &h1, unsigned &l1) {
    const f32x2 c = fma2(x, pk2(8192.0f, 8192.0f), x);
    const f32x2 hi = fma2(x, pk2(-8192.0f, -8192.0f), c);
    const f32x2 lo = sub2(x, hi);
    float a, b;
    upk2(hi, a, b);
    h0 = __float_as_uint(a);
    h1 = __float_as_uint(b);
    upk2(lo, a, b);
    l0 = __float_as_uint(a);
    l1 = __float_as_uint(b);
}

// d += a b on the tensor core (mma.m16n8k8, TF32 operands, FP32 sums)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Horner evaluation of a degree-7 polynomial held in registers.
__device__ __forceinline__ float horner8(const float c[NCOEF], float v) {
    float s = c[NCOEF - 1];
#pragma unroll
    for (int i = NCOEF - 2; i >= 0; --i) s = fmaf(s, v, c[i]);
    return s;
}

// The same polynomial at v and at -v from its even and odd parts,
// p(+-v) = E(v^2) +- v O(v^2): 9 operations instead of two Horner chains of 7.
// Tap 2m - 1 - j of the (even) window at v is tap j at -v.
__device__ __forceinline__ void horner8_pm(const float c[NCOEF], float v, float &p, float &m) {
    static_assert(NCOEF == 8, "even/odd split of a degree-7 polynomial");
    const float v2 = v * v;
    const float e = fmaf(fmaf(fmaf(c[6], v2, c[4]), v2, c[2]), v2, c[0]);
    const float o = fmaf(fmaf(fmaf(c[7], v2, c[5]), v2, c[3]), v2, c[1]);
    p = fmaf(v, o, e);
    m = fmaf(-v, o, e);
}

// Two degree-7 polynomials at once: coefficient pairs cp[i] = (a_i, b_i),
// arguments (va, vb); the same operations as horner8 on each half.
__device__ __forceinline__ void horner8_x2(const f32x2 cp[NCOEF], float va, float vb, float &pa, float &pb) {
    const f32x2 v = pk2(va, vb);
    f32x2 s = cp[NCOEF - 1];
#pragma unroll
    for (int i = NCOEF - 2; i >= 0; --i) s = fma2(s, v, cp[i]);
    upk2(s, pa, pb);
}

// Direct evaluation of the normalised Kaiser--Bessel window at distance d
// (grid units); used where no per-tap polynomial is kept in registers.
__device__ __forceinline__ float kb_direct(float d, int m, float b, float inv_psi0) {
    float s2 = fmaf(-d, d, (float)(m * m));
    if (s2 <= 0.0f) return s2 == 0.0f ? b * (1.0f / 3.14159265358979f) * inv_psi0 : 0.0f;
    float s = sqrtf(s2);
    float bs = b * s;
    float v;
    if (bs < 1e-2f) {
        v = b * (1.0f + bs * bs * (1.0f / 6.0f));
    } else {
        float e = expf(bs);
        v = 0.5f * (e - 1.0f / e) / s;
    }
    return v * (1.0f / 3.14159265358979f) * inv_psi0;
}

__device__ __forceinline__ double kb_direct_d(double d, int m, double b, double inv_psi0) {
    double s2 = fma(-d, d, (double)(m * m));
    if (s2 <= 0.0) return s2 == 0.0 ? b / 3.141592653589793238 * inv_psi0 : 0.0;
    double s = sqrt(s2);
    return sinh(b * s) / (3.141592653589793238 * s) * inv_psi0;
}

// Grid position of a coordinate x in [-1/2, 1/2): t = (x + 1/2) n wrapped to
// [0, n).  Returns floor(t) and writes tau = t - floor(t).
__device__ __forceinline__ int grid_pos(float x, int n, float &tau) {
    float t = (x + 0.5f) * (float)n;
    float fl = floorf(t);
    tau = t - fl;
    int i = (int)fl;
    if (i >= n) i -= n;   // x rounded up to 1/2
    if (i < 0) i += n;
    return i;
}

__device__ __forceinline__ int grid_pos_d(double x, int n, double &tau) {
    double t = (x + 0.5) * (double)n;
    double fl = floor(t);
    tau = t - fl;
    int i = (int)fl;
    if (i >= n) i -= n;
    if (i < 0) i += n;
    return i;
}

__device__ __forceinline__ int wrap(int i, int n) {
    i = i < 0 ? i + n : i;
    return i >= n ? i - n : i;
}

// ------------------------------------------------------- async bulk copies --

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- cp.async (Ampere-style asynchronous copies to shared memory) ----
// 16 bytes through L2 only (no L1 line is allocated)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// wait until at most N of this thread's most recent groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_n() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// L2 prefetch of bytes (a multiple of 16) at a 16-byte aligned global address
__device__ __forceinline__ void prefetch_l2_bulk(const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy (16-byte aligned, size multiple of 16), completion
// counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for the mbarrier phase with parity `parity`.  Gives up after
// `limit` polls, records `code` in *err and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code,
                                          long long limit = (1LL << 22)) {
    uint32_t a = smem_addr(bar);
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    if (err) atomicCAS(err, 0, code);
    return false;
}

// ----------------------------------------------------------- shared FFT ---

// Mixed-radix Stockham FFT over a batch of lines held in shared memory.
// Line l, element i lives at base[l * lstride + i * estride] in both ping-pong
// buffers.  Computes X[q] = sum_i x[i] exp(sign 2 pi i i q / n) (unnormalised).
// Radices 4, 2, 3, 5.  All threads of the block must call it; returns the
// buffer (0 = a, 1 = b) that holds the result.
template <typename C, typename R>
struct CplxOps;

template <>
struct CplxOps<float2, float> {
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
};
template <>
struct CplxOps<double2, double> {
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

__host__ __device__ inline int fft_radices(int n, int *rad) {
    int k = 0;
    while (n % 4 == 0) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0) { rad[k++] = 3; n /= 3; }
    while (n % 5 == 0) { rad[k++] = 5; n /= 5; }
    return n == 1 ? k : -1;
}

template <typename C, typename R>
__device__ int smem_fft(C *a, C *b, int n, int nlines, int lstride, int estride, int sign) {
    using O = CplxOps<C, R>;
    int rad[24];
    int ns = fft_radices(n, rad);
    C *src = a, *dst = b;
    int which = 0;
    int Ns = 1;
    for (int s = 0; s < ns; ++s) {
        const int Rr = rad[s];
        const int nb = n / Rr;
        for (int w = threadIdx.x; w < nlines * nb; w += blockDim.x) {
            const int l = w / nb, j = w - l * nb;
            const C *in = src + (size_t)l * lstride;
            C *out = dst + (size_t)l * lstride;
            C v[5];
            const int jm = j % Ns;
            // twiddles exp(sign 2 pi i r jm / (Ns Rr))
            for (int r = 0; r < Rr; ++r) {
                C x = in[(size_t)(j + r * nb) * estride];
                if (r && jm) {
                    R sn, cs;
                    O::sincospi_((R)(2 * sign * r * jm) / (R)(Ns * Rr), &sn, &cs);
                    x = cmul(x, O::mk(cs, sn));
                }
                v[r] = x;
            }
            C V[5];
            if (Rr == 2) {
                V[0] = O::mk(v[0].x + v[1].x, v[0].y + v[1].y);
                V[1] = O::mk(v[0].x - v[1].x, v[0].y - v[1].y);
            } else if (Rr == 4) {
                C s0 = O::mk(v[0].x + v[2].x, v[0].y + v[2].y);
                C d0 = O::mk(v[0].x - v[2].x, v[0].y - v[2].y);
                C s1 = O::mk(v[1].x + v[3].x, v[1].y + v[3].y);
                C d1 = O::mk(v[1].x - v[3].x, v[1].y - v[3].y);
                // multiply d1 by (sign) i
                C jd1 = sign > 0 ? O::mk(-d1.y, d1.x) : O::mk(d1.y, -d1.x);
                V[0] = O::mk(s0.x + s1.x, s0.y + s1.y);
                V[2] = O::mk(s0.x - s1.x, s0.y - s1.y);
                V[1] = O::mk(d0.x + jd1.x, d0.y + jd1.y);
                V[3] = O::mk(d0.x - jd1.x, d0.y - jd1.y);
            } else {
                for (int q = 0; q < Rr; ++q) {
                    C acc = v[0];
                    for (int r = 1; r < Rr; ++r) {
                        R sn, cs;
                        O::sincospi_((R)(2 * sign * ((r * q) % Rr)) / (R)Rr, &sn, &cs);
                        C t = cmul(v[r], O::mk(cs, sn));
                        acc.x += t.x;
                        acc.y += t.y;
                    }
                    V[q] = acc;
                }
            }
            const int idxD = (j / Ns) * Ns * Rr + jm;
            for (int r = 0; r < Rr; ++r) out[(size_t)(idxD + r * Ns) * estride] = V[r];
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
        which ^= 1;
        Ns *= Rr;
    }
    return which;
}

// Unnormalised FFT with sign `sign` along every axis of an n^s array held in
// shared memory (a; b is scratch of the same size), s = 1..3: all lines of an
// axis at once, line bases (l / inner) * inner * n + l % inner for the axis
// whose element stride is `inner`.  All threads of the block call it; returns
// the buffer that holds the result.
template <typename C, typename R>
__device__ C *grid_fft(C *a, C *b, int n, int s, int sign) {
    using O = CplxOps<C, R>;
    int fe = n;
    for (int j = 1; j < s; ++j) fe *= n;
    C *cur = a, *oth = b;
    int inner = 1;
    int rad[24];
    const int ns = fft_radices(n, rad);
    for (int ax = s - 1; ax >= 0; --ax) {
        const int nlines = fe / n;
        C *src = cur, *dst = oth;
        int which = 0, Ns = 1;
        for (int st = 0; st < ns; ++st) {
            const int Rr = rad[st];
            const int nb = n / Rr;
            for (int w = threadIdx.x; w < nlines * nb; w += blockDim.x) {
                const int l = w / nb, j = w - l * nb;
                const int base = (l / inner) * inner * n + (l % inner);
                const C *in = src + base;
                C *out = dst + base;
                C v[5];
                const int jm = j % Ns;
                for (int r = 0; r < Rr; ++r) {
                    C x = in[(j + r * nb) * inner];
                    if (r && jm) {
                        R sn, cs;
                        O::sincospi_((R)(2 * sign * r * jm) / (R)(Ns * Rr), &sn, &cs);
                        x = cmul(x, O::mk(cs, sn));
                    }
                    v[r] = x;
                }
                C V[5];
                if (Rr == 2) {
                    V[0] = O::mk(v[0].x + v[1].x, v[0].y + v[1].y);
                    V[1] = O::mk(v[0].x - v[1].x, v[0].y - v[1].y);
                } else if (Rr == 4) {
                    const C s0 = O::mk(v[0].x + v[2].x, v[0].y + v[2].y);
                    const C d0 = O::mk(v[0].x - v[2].x, v[0].y - v[2].y);
                    const C s1 = O::mk(v[1].x + v[3].x, v[1].y + v[3].y);
                    const C d1 = O::mk(v[1].x - v[3].x, v[1].y - v[3].y);
                    const C jd1 = sign > 0 ? O::mk(-d1.y, d1.x) : O::mk(d1.y, -d1.x);   // sign i d1
                    V[0] = O::mk(s0.x + s1.x, s0.y + s1.y);
                    V[2] = O::mk(s0.x - s1.x, s0.y - s1.y);
                    V[1] = O::mk(d0.x + jd1.x, d0.y + jd1.y);
                    V[3] = O::mk(d0.x - jd1.x, d0.y - jd1.y);
                } else {
                    for (int q = 0; q < Rr; ++q) {
                        C acc = v[0];
                        for (int r = 1; r < Rr; ++r) {
                            R sn, cs;
                            O::sincospi_((R)(2 * sign * ((r * q) % Rr)) / (R)Rr, &sn, &cs);
                            const C t = cmul(v[r], O::mk(cs, sn));
                            acc.x += t.x;
                            acc.y += t.y;
                        }
                        V[q] = acc;
                    }
                }
                const int idxD = (j / Ns) * Ns * Rr + jm;
                for (int r = 0; r < Rr; ++r) out[(idxD + r * Ns) * inner] = V[r];
            }
            __syncthreads();
            C *t = src;
            src = dst;
            dst = t;
            which ^= 1;
            Ns *= Rr;
        }
        if (which) {
            C *t = cur;
            cur = oth;
            oth = t;
        }
        inner *= n;
    }
    return cur;
}

}  // namespace agft
