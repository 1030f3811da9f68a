// Spectral scaling, FP64 reductions and vector updates of libclaire (sm_103a).
// The spectral kernel applies the per-wavenumber 3x3 symbols of the
// regularisation operator, its inverse (the PCG preconditioner) and the
// paper's K operator in one pass over the three half-spectra (Sec. 2.2:
// "two FFTs and one Hadamard product"); cuFFT does the transforms.
#include "internal.h"

namespace claire {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float s, float2 z) { return make_float2(s * z.x, s * z.y); }

// Per-mode pieces of the symbol S(k) = a I + c u u^T on the half spectrum:
// a = beta_v |k|^2 (H1) or beta_v |k|^4 (H2), c = beta_w (1 + |k|^2), u = k
// with Nyquist components set to zero; wt = multiplicity of the mode in the
// full spectrum (1 on the x3 = 0 and Nyquist planes, else 2).
struct Mode {
    float u1, u2, u3, a, c, kk, wt;
};

__device__ __forceinline__ Mode mode_of(const Grid& g, size_t idx, int n3h, const RegParams& rp)
{
    Mode m;
    const int k3i = static_cast<int>(idx % n3h);
    const size_t r = idx / n3h;
    const int j = static_cast<int>(r % g.n2);
    const int i = static_cast<int>(r / g.n2);
    const float k1 = static_cast<float>(i <= g.n1 / 2 ? i : i - g.n1);
    const float k2 = static_cast<float>(j <= g.n2 / 2 ? j : j - g.n2);
    const float k3 = static_cast<float>(k3i);
    m.kk = k1 * k1 + k2 * k2 + k3 * k3;
    m.u1 = (2 * i == g.n1) ? 0.0f : k1;
    m.u2 = (2 * j == g.n2) ? 0.0f : k2;
    m.u3 = (2 * k3i == g.n3) ? 0.0f : k3;
    m.a = rp.beta_v * (rp.reg == 2 ? m.kk * m.kk : m.kk);
    m.c = rp.beta_w * (1.0f + m.kk);
    m.wt = (k3i == 0 || 2 * k3i == g.n3) ? 1.0f : 2.0f;
    return m;
}

// y = S x for one mode
__device__ __forceinline__ void apply_S(const Mode& m, float2 x0, float2 x1, float2 x2, float2& y0,
                                        float2& y1, float2& y2)
{
    const float2 ud = make_float2(m.u1 * x0.x + m.u2 * x1.x + m.u3 * x2.x,
                                  m.u1 * x0.y + m.u2 * x1.y + m.u3 * x2.y);
    y0 = make_float2(m.a * x0.x + m.c * m.u1 * ud.x, m.a * x0.y + m.c * m.u1 * ud.y);
    y1 = make_float2(m.a * x1.x + m.c * m.u2 * ud.x, m.a * x1.y + m.c * m.u2 * ud.y);
    y2 = make_float2(m.a * x2.x + m.c * m.u3 * ud.x, m.a * x2.y + m.c * m.u3 * ud.y);
}

// y = S^{-1} x (op SPEC_INV) or (a I)^{-1} x (op SPEC_AINV); identity at k = 0
__device__ __forceinline__ void apply_inv(const Mode& m, int op, float2 x0, float2 x1, float2 x2,
                                          float2& y0, float2& y1, float2& y2)
{
    if (m.kk == 0.0f) {
        y0 = x0; y1 = x1; y2 = x2;
        return;
    }
    const float ia = 1.0f / m.a;
    if (op == SPEC_AINV) {
        y0 = cmul(ia, x0); y1 = cmul(ia, x1); y2 = cmul(ia, x2);
        return;
    }
    const float2 ud = make_float2(m.u1 * x0.x + m.u2 * x1.x + m.u3 * x2.x,
                                  m.u1 * x0.y + m.u2 * x1.y + m.u3 * x2.y);
    const float f = m.c / (m.a + m.c * (m.u1 * m.u1 + m.u2 * m.u2 + m.u3 * m.u3));
    y0 = cmul(ia, make_float2(x0.x - f * m.u1 * ud.x, x0.y - f * m.u1 * ud.y));
    y1 = cmul(ia, make_float2(x1.x - f * m.u2 * ud.x, x1.y - f * m.u2 * ud.y));
    y2 = cmul(ia, make_float2(x2.x - f * m.u3 * ud.x, x2.y - f * m.u3 * ud.y));
}

// In place: xh <- scale * M(k) xh for the three half-spectra.
__global__ void __launch_bounds__(kThreads) k_spectral(Grid g, float2* __restrict__ xh, size_t cs,
                                                        int op, RegParams rp, float scale)
{
    const int n3h = g.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * n3h;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        const int k3i = static_cast<int>(idx % n3h);
        const size_t r = idx / n3h;
        const int j = static_cast<int>(r % g.n2);
        const int i = static_cast<int>(r / g.n2);
        const float k1 = static_cast<float>(i <= g.n1 / 2 ? i : i - g.n1);
        const float k2 = static_cast<float>(j <= g.n2 / 2 ? j : j - g.n2);
        const float k3 = static_cast<float>(k3i);
        const float kk = k1 * k1 + k2 * k2 + k3 * k3;
        const float u1 = (2 * i == g.n1) ? 0.0f : k1;
        const float u2 = (2 * j == g.n2) ? 0.0f : k2;
        const float u3 = (2 * k3i == g.n3) ? 0.0f : k3;
        const float a = rp.beta_v * (rp.reg == 2 ? kk * kk : kk);
        const float c = rp.beta_w * (1.0f + kk);
        float2 x0 = xh[idx], x1 = xh[cs + idx], x2 = xh[2 * cs + idx];
        const float2 ud = make_float2(u1 * x0.x + u2 * x1.x + u3 * x2.x,
                                      u1 * x0.y + u2 * x1.y + u3 * x2.y);
        float2 y0, y1, y2;
        if (op == SPEC_REG) {
            y0 = make_float2(a * x0.x + c * u1 * ud.x, a * x0.y + c * u1 * ud.y);
            y1 = make_float2(a * x1.x + c * u2 * ud.x, a * x1.y + c * u2 * ud.y);
            y2 = make_float2(a * x2.x + c * u3 * ud.x, a * x2.y + c * u3 * ud.y);
        } else if (kk == 0.0f) {
            y0 = x0;
            y1 = x1;
            y2 = x2;
        } else if (op == SPEC_AINV) {
            const float ia = 1.0f / a;
            y0 = cmul(ia, x0);
            y1 = cmul(ia, x1);
            y2 = cmul(ia, x2);
        } else {
            // K = I - c u u^T / (a + c |u|^2);  S^{-1} = K / a  (Sherman-Morrison)
            const float f = c / (a + c * (u1 * u1 + u2 * u2 + u3 * u3));
            y0 = make_float2(x0.x - f * u1 * ud.x, x0.y - f * u1 * ud.y);
            y1 = make_float2(x1.x - f * u2 * ud.x, x1.y - f * u2 * ud.y);
            y2 = make_float2(x2.x - f * u3 * ud.x, x2.y - f * u3 * ud.y);
            if (op == SPEC_INV) {
                const float ia = 1.0f / a;
                y0 = cmul(ia, y0);
                y1 = cmul(ia, y1);
                y2 = cmul(ia, y2);
            }
        }
        xh[idx] = cmul(scale, y0);
        xh[cs + idx] = cmul(scale, y1);
        xh[2 * cs + idx] = cmul(scale, y2);
    }
}

// Preconditioner in Fourier space: zh = scale * M(k) rh in place (M = S^{-1}
// or (a I)^{-1}) and block partial sums of sum_k wt Re(conj(rh) zh), which is
// sum_x r(x) z(x) by Parseval (zh already carries the 1/N of the inverse FFT).
__global__ void __launch_bounds__(kThreads) k_spectral_precond(Grid g, float2* __restrict__ xh, size_t cs,
                                                                int op, RegParams rp, float scale,
                                                                double* __restrict__ partials)
{
    const int n3h = g.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * n3h;
    double acc = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        const Mode m = mode_of(g, idx, n3h, rp);
        const float2 x0 = xh[idx], x1 = xh[cs + idx], x2 = xh[2 * cs + idx];
        float2 y0, y1, y2;
        apply_inv(m, op, x0, x1, x2, y0, y1, y2);
        y0 = cmul(scale, y0); y1 = cmul(scale, y1); y2 = cmul(scale, y2);
        xh[idx] = y0;
        xh[cs + idx] = y1;
        xh[2 * cs + idx] = y2;
        const float re = x0.x * y0.x + x0.y * y0.y + x1.x * y1.x + x1.y * y1.y + x2.x * y2.x + x2.y * y2.y;
        acc += static_cast<double>(m.wt * re);
    }
    block_sum(acc, partials);
}

// PCG direction in Fourier space: z~ = M r~ (recomputed from r~, not
// stored), p~ = z~ + beta p~ (p~ = z~ when first), copied to cp for the
// inverse FFT that yields p (it overwrites its input).
__global__ void __launch_bounds__(kThreads) k_spectral_direction(Grid g, const float2* __restrict__ rh,
                                                                  float2* __restrict__ ph,
                                                                  float2* __restrict__ cp, size_t cs,
                                                                  float beta, int first, int op, RegParams rp)
{
    const int n3h = g.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * n3h;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        const Mode m = mode_of(g, idx, n3h, rp);
        float2 z[3];
        apply_inv(m, op, rh[idx], rh[cs + idx], rh[2 * cs + idx], z[0], z[1], z[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 p = z[c];
            if (!first) {
                const float2 o = ph[c * cs + idx];
                p = make_float2(fmaf(beta, o.x, z[c].x), fmaf(beta, o.y, z[c].y));
            }
            ph[c * cs + idx] = p;
            cp[c * cs + idx] = p;
        }
    }
}

// ---- PCG carried entirely in Fourier space ----
// Vectors are scaled half-spectra u~ = F[u] / N, so that the unnormalised
// inverse FFT returns u and sum_x u(x) w(x) = N sum_k wt Re(conj(u~) w~)
// (Parseval on the half spectrum; wt = multiplicity of the mode).

__device__ __forceinline__ void block_sum2(double a, double b, double* pa, double* pb)
{
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double x = lane < nw ? sa[lane] : 0.0;
        double y = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        if (lane == 0) {
            pa[blockIdx.x] = x;
            pb[blockIdx.x] = y;
        }
    }
}

__device__ __forceinline__ float cdot3(float2 a0, float2 a1, float2 a2, float2 b0, float2 b1, float2 b2)
{
    return a0.x * b0.x + a0.y * b0.y + a1.x * b1.x + a1.y * b1.y + a2.x * b2.x + a2.y * b2.y;
}

// Start: r~ = -scale g^ (spec holds F[g]), x~ = 0; partials of |r~|^2 and
// <r~, z~> with z~ = M r~ (recomputed by the direction kernel).
__global__ void __launch_bounds__(kThreads) k_fs_start(Grid g, float2* __restrict__ spec,
                                                        float2* __restrict__ rh, float2* __restrict__ xh,
                                                        size_t cs, int op, RegParams rp, float scale,
                                                        double* __restrict__ prr, double* __restrict__ prz)
{
    const int n3h = g.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * n3h;
    double arr = 0.0, arz = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        const Mode m = mode_of(g, idx, n3h, rp);
        const float2 r0 = cmul(-scale, spec[idx]), r1 = cmul(-scale, spec[cs + idx]),
                     r2 = cmul(-scale, spec[2 * cs + idx]);
        float2 z0, z1, z2;
        apply_inv(m, op, r0, r1, r2, z0, z1, z2);
        rh[idx] = r0; rh[cs + idx] = r1; rh[2 * cs + idx] = r2;
        xh[idx] = make_float2(0.f, 0.f); xh[cs + idx] = make_float2(0.f, 0.f); xh[2 * cs + idx] = make_float2(0.f, 0.f);
        arr += static_cast<double>(m.wt * cdot3(r0, r1, r2, r0, r1, r2));
        arz += static_cast<double>(m.wt * cdot3(r0, r1, r2, z0, z1, z2));
    }
    block_sum2(arr, arz, prr, prz);
}

// H p~ = S p~ + scale F[body] (in spec2), or K of that for the paper's
// gradient form; written into spec; partials of <p~, H p~>.
__global__ void __launch_bounds__(kThreads) k_fs_hp(Grid g, float2* __restrict__ spec,
                                                     const float2* __restrict__ spec2,
                                                     const float2* __restrict__ ph, size_t cs, int kform,
                                                     RegParams rp, float scale, double* __restrict__ ppq)
{
    const int n3h = g.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * n3h;
    double acc = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        const Mode m = mode_of(g, idx, n3h, rp);
        const float2 p0 = ph[idx], p1 = ph[cs + idx], p2 = ph[2 * cs + idx];
        float2 h[3];
        apply_S(m, p0, p1, p2, h[0], h[1], h[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 b = spec2[c * cs + idx];
            h[c] = make_float2(fmaf(scale, b.x, h[c].x), fmaf(scale, b.y, h[c].y));
        }
        if (kform && m.kk != 0.0f) {
            const float2 ud = make_float2(m.u1 * h[0].x + m.u2 * h[1].x + m.u3 * h[2].x,
                                          m.u1 * h[0].y + m.u2 * h[1].y + m.u3 * h[2].y);
            const float f = m.c / (m.a + m.c * (m.u1 * m.u1 + m.u2 * m.u2 + m.u3 * m.u3));
            h[0] = make_float2(h[0].x - f * m.u1 * ud.x, h[0].y - f * m.u1 * ud.y);
            h[1] = make_float2(h[1].x - f * m.u2 * ud.x, h[1].y - f * m.u2 * ud.y);
            h[2] = make_float2(h[2].x - f * m.u3 * ud.x, h[2].y - f * m.u3 * ud.y);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) spec[c * cs + idx] = h[c];
        acc += static_cast<double>(m.wt * cdot3(p0, p1, p2, h[0], h[1], h[2]));
    }
    block_sum(acc, ppq);
}

// x~ += alpha p~, r~ -= alpha H p~ (H p~ in spec); partials of |r~|^2 and
// <r~, z~> with z~ = M r~ (recomputed by the next direction kernel), or, when
// a stored preconditioned residual zc is given, of <H p~, zc> instead.
__global__ void __launch_bounds__(kThreads) k_fs_update(Grid g, const float2* __restrict__ spec,
                                                         const float2* __restrict__ ph,
                                                         float2* __restrict__ xh, float2* __restrict__ rh,
                                                         const float2* __restrict__ zc, size_t cs, float alpha,
                                                         int op, RegParams rp, double* __restrict__ prr,
                                                         double* __restrict__ prz)
{
    const int n3h = g.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * n3h;
    double arr = 0.0, arz = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        float2 r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 p = ph[c * cs + idx], hp = spec[c * cs + idx];
            float2 x = xh[c * cs + idx], rr = rh[c * cs + idx];
            x = make_float2(fmaf(alpha, p.x, x.x), fmaf(alpha, p.y, x.y));
            rr = make_float2(fmaf(-alpha, hp.x, rr.x), fmaf(-alpha, hp.y, rr.y));
            xh[c * cs + idx] = x;
            rh[c * cs + idx] = rr;
            r[c] = rr;
        }
        const Mode m = mode_of(g, idx, n3h, rp);
        arr += static_cast<double>(m.wt * cdot3(r[0], r[1], r[2], r[0], r[1], r[2]));
        if (zc) {
            arz += static_cast<double>(m.wt * cdot3(spec[idx], spec[cs + idx], spec[2 * cs + idx], zc[idx],
                                                     zc[cs + idx], zc[2 * cs + idx]));
        } else {
            float2 z0, z1, z2;
            apply_inv(m, op, r[0], r[1], r[2], z0, z1, z2);
            arz += static_cast<double>(m.wt * cdot3(r[0], r[1], r[2], z0, z1, z2));
        }
    }
    block_sum2(arr, arz, prr, prz);
}

__device__ __forceinline__ bool aligned16(const void* p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

__global__ void __launch_bounds__(kThreads) k_dot_partial(const float* __restrict__ x,
                                                           const float* __restrict__ y, size_t n,
                                                           double* __restrict__ partials)
{
    double acc = 0.0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    const size_t t0 = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    size_t done = 0;
    if (aligned16(x) && aligned16(y)) {
        const size_t n4 = n / 4;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* y4 = reinterpret_cast<const float4*>(y);
        for (size_t i = t0; i < n4; i += stride) {
            const float4 a = __ldg(x4 + i), b = __ldg(y4 + i);
            acc += static_cast<double>(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w);
        }
        done = n4 * 4;
    }
    for (size_t i = done + t0; i < n; i += stride) acc += static_cast<double>(x[i] * y[i]);
    block_sum(acc, partials);
}

template <class S>
__global__ void __launch_bounds__(kThreads) k_sqdiff_partial(const S* __restrict__ a, const S* __restrict__ b,
                                                              size_t n, double* __restrict__ partials)
{
    double acc = 0.0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    const size_t t0 = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    size_t done = 0;
    if constexpr (sizeof(S) == 4) {
        if (aligned16(a) && aligned16(b)) {
            const size_t n4 = n / 4;
            const float4* a4 = reinterpret_cast<const float4*>(a);
            const float4* b4 = reinterpret_cast<const float4*>(b);
            for (size_t i = t0; i < n4; i += stride) {
                const float4 p = __ldg(a4 + i), q = __ldg(b4 + i);
                const float d0 = p.x - q.x, d1 = p.y - q.y, d2 = p.z - q.z, d3 = p.w - q.w;
                acc += static_cast<double>(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3);
            }
            done = n4 * 4;
        }
    }
    for (size_t i = done + t0; i < n; i += stride) {
        const float d = ldf<S>(a + i) - ldf<S>(b + i);
        acc += static_cast<double>(d * d);
    }
    block_sum(acc, partials);
}

// max over points of |v|_2^2; partials holds 2 * gridDim.x doubles (the
// first half receives the block maxima, the second half is scratch).
__global__ void __launch_bounds__(kThreads) k_maxnorm3_partial(const float* __restrict__ v, size_t N,
                                                                double* __restrict__ partials)
{
    double hi = 0.0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < N; i += stride) {
        const double a = v[i], b = v[N + i], c = v[2 * N + i];
        const double s = a * a + b * b + c * c;
        hi = max_nan(hi, s);  // a NaN component makes the result NaN
    }
    block_minmax(hi, hi, partials + gridDim.x, partials);
}

// Dice counts (Sec. 4.1): both = 0 counts a >= t and b >= t into pa, pb;
// both = 1 counts (a >= t) and (b >= t) into pa (pb gets zeros).  Per-block
// FP64 partial sums of integers: exact below 2^53.
__global__ void __launch_bounds__(kThreads) k_count_partial(const float* __restrict__ a, const float* __restrict__ b,
                                                             size_t n, float t, int both, double* __restrict__ pa,
                                                             double* __restrict__ pb)
{
    unsigned long long ca = 0, cb = 0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n; i += stride) {
        const bool ia = a[i] >= t, ib = b[i] >= t;
        if (both) {
            ca += (ia && ib) ? 1u : 0u;
        } else {
            ca += ia ? 1u : 0u;
            cb += ib ? 1u : 0u;
        }
    }
    block_sum2(static_cast<double>(ca), static_cast<double>(cb), pa, pb);
}

__global__ void __launch_bounds__(kThreads) k_final_sum(const double* __restrict__ partials, int nb,
                                                         double scale, double* __restrict__ out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += partials[i];
    block_sum(acc, out);
    if (threadIdx.x == 0) out[0] *= scale;
}

__global__ void __launch_bounds__(kThreads) k_final_minmax(const double* __restrict__ pmin,
                                                            const double* __restrict__ pmax, int nb,
                                                            double* __restrict__ out2)
{
    double lo = 1e300, hi = -1e300;
    for (int i = threadIdx.x; i < nb; i += kThreads) {
        const double a = pmin ? pmin[i] : lo;
        const double b = pmax[i];
        lo = min_nan(lo, a);
        hi = max_nan(hi, b);
    }
    block_minmax(lo, hi, out2, out2 + 1);
}

// The vector updates take a float4 path when every pointer is 16-byte aligned
// (the context's buffers always are) and a scalar loop for the tail.
__global__ void __launch_bounds__(kThreads) k_axpy(float a, const float* __restrict__ x,
                                                    float* __restrict__ y, size_t n)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    const size_t t0 = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    size_t done = 0;
    if (aligned16(x) && aligned16(y)) {
        const size_t n4 = n / 4;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        float4* y4 = reinterpret_cast<float4*>(y);
        for (size_t i = t0; i < n4; i += stride) {
            const float4 u = __ldg(x4 + i);
            float4 w = y4[i];
            w.x = fmaf(a, u.x, w.x); w.y = fmaf(a, u.y, w.y); w.z = fmaf(a, u.z, w.z); w.w = fmaf(a, u.w, w.w);
            y4[i] = w;
        }
        done = n4 * 4;
    }
    for (size_t i = done + t0; i < n; i += stride) y[i] = fmaf(a, x[i], y[i]);
}

__global__ void __launch_bounds__(kThreads) k_xpay(const float* __restrict__ x, float a,
                                                    const float* y, float* z, size_t n)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    const size_t t0 = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    size_t done = 0;
    if (aligned16(x) && aligned16(y) && aligned16(z)) {
        const size_t n4 = n / 4;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* y4 = reinterpret_cast<const float4*>(y);
        float4* z4 = reinterpret_cast<float4*>(z);
        for (size_t i = t0; i < n4; i += stride) {
            const float4 u = __ldg(x4 + i);
            const float4 v = y4[i];
            z4[i] = make_float4(fmaf(a, v.x, u.x), fmaf(a, v.y, u.y), fmaf(a, v.z, u.z), fmaf(a, v.w, u.w));
        }
        done = n4 * 4;
    }
    for (size_t i = done + t0; i < n; i += stride) z[i] = fmaf(a, y[i], x[i]);
}

__global__ void __launch_bounds__(kThreads) k_pcg_update(float alpha, const float* __restrict__ p,
                                                          const float* __restrict__ q,
                                                          float* __restrict__ x,
                                                          float* __restrict__ r, size_t n,
                                                          double* __restrict__ partials)
{
    double acc = 0.0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    const size_t t0 = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    size_t done = 0;
    if (aligned16(p) && aligned16(q) && aligned16(x) && aligned16(r)) {
        const size_t n4 = n / 4;
        const float4* p4 = reinterpret_cast<const float4*>(p);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        float4* x4 = reinterpret_cast<float4*>(x);
        float4* r4 = reinterpret_cast<float4*>(r);
        for (size_t i = t0; i < n4; i += stride) {
            const float4 pp = __ldg(p4 + i), qq = __ldg(q4 + i);
            float4 xx = x4[i], rr = r4[i];
            xx.x = fmaf(alpha, pp.x, xx.x); xx.y = fmaf(alpha, pp.y, xx.y);
            xx.z = fmaf(alpha, pp.z, xx.z); xx.w = fmaf(alpha, pp.w, xx.w);
            rr.x = fmaf(-alpha, qq.x, rr.x); rr.y = fmaf(-alpha, qq.y, rr.y);
            rr.z = fmaf(-alpha, qq.z, rr.z); rr.w = fmaf(-alpha, qq.w, rr.w);
            x4[i] = xx;
            r4[i] = rr;
            acc += static_cast<double>(rr.x * rr.x + rr.y * rr.y + rr.z * rr.z + rr.w * rr.w);
        }
        done = n4 * 4;
    }
    for (size_t i = done + t0; i < n; i += stride) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        acc += static_cast<double>(ri * ri);
    }
    block_sum(acc, partials);
}

__global__ void __launch_bounds__(kThreads) k_fill(float* __restrict__ x, float value, size_t n)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n; i += stride)
        x[i] = value;
}

unsigned stream_blocks(size_t n)
{
    size_t b = (n + kThreads - 1) / kThreads;
    const size_t cap = 152 * 16;  // enough resident blocks to cover the GPU, grid-stride beyond
    return static_cast<unsigned>(b < cap ? (b ? b : 1) : cap);
}


// B-spline prefilter in Fourier space: every mode of ncomp half spectra is
// divided by N prod_axes (2 + cos(k_a h_a)) / 3 (the sampled cubic B-spline),
// so that the inverse transform gives the interpolating spline's coefficients.
__global__ void k_bspline_scale(Grid g, cufftComplex* __restrict__ spec, size_t M, int ncomp, float invN)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (e >= M * ncomp) return;
    const size_t m = e % M;
    const int n3h = g.n3 / 2 + 1;
    const int j3 = static_cast<int>(m % n3h);
    const int j2 = static_cast<int>((m / n3h) % g.n2);
    const int j1 = static_cast<int>(m / (static_cast<size_t>(n3h) * g.n2));
    const float two_pi = 6.283185307179586f;
    const float s1 = (2.0f + cosf(two_pi * j1 / g.n1)) * (1.0f / 3.0f);
    const float s2 = (2.0f + cosf(two_pi * j2 / g.n2)) * (1.0f / 3.0f);
    const float s3 = (2.0f + cosf(two_pi * j3 / g.n3)) * (1.0f / 3.0f);
    const float f = invN / (s1 * s2 * s3);
    spec[e].x *= f;
    spec[e].y *= f;
}
// out = w_end (m^0 + m^nt) + w_mid (m^1 + ... + m^{nt-1}) (trapezoid over the stored levels)
template <class S>
__global__ void __launch_bounds__(kThreads) k_mean_levels(const S* __restrict__ m, int nt, float w_end,
                                                           float w_mid, size_t N, float* __restrict__ out)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < N;
         i += static_cast<size_t>(gridDim.x) * kThreads) {
        float acc = w_end * (ldf<S>(m + i) + ldf<S>(m + static_cast<size_t>(nt) * N + i));
        for (int j = 1; j < nt; ++j) acc = fmaf(w_mid, ldf<S>(m + static_cast<size_t>(j) * N + i), acc);
        out[i] = acc;
    }
}

__global__ void __launch_bounds__(kThreads) k_cscale(float2* __restrict__ x, size_t n, float s)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * kThreads)
        x[i] = cmul(s, x[i]);
}

// ---- two-level zero-velocity preconditioner (Sec. 2.2) ----
// The coarse grid gc keeps the modes |k_i| < gc.n_i / 2 of the fine grid gf
// (its Nyquist planes are dropped); the inner PCG runs on those modes without
// the mean (k = 0), the "kept" modes, in the same scaled half-spectrum
// convention as the outer PCG (coefficients are resolution independent, so
// restriction and prolongation copy them).

// Wavenumbers of half-spectrum mode idx of grid g.
__device__ __forceinline__ void wavenumbers(const Grid& g, size_t idx, int& k1, int& k2, int& k3)
{
    const int n3h = g.n3 / 2 + 1;
    k3 = static_cast<int>(idx % n3h);
    const size_t r = idx / n3h;
    const int j = static_cast<int>(r % g.n2);
    const int i = static_cast<int>(r / g.n2);
    k1 = i <= g.n1 / 2 ? i : i - g.n1;
    k2 = j <= g.n2 / 2 ? j : j - g.n2;
}

// |k_i| < n_i / 2 on every axis of grid g (no Nyquist plane)
__device__ __forceinline__ bool below_nyquist(const Grid& g, int k1, int k2, int k3)
{
    return 2 * abs(k1) < g.n1 && 2 * abs(k2) < g.n2 && 2 * k3 < g.n3;
}

// Half-spectrum index of wavenumber k on grid g (k assumed representable).
__device__ __forceinline__ size_t mode_index(const Grid& g, int k1, int k2, int k3)
{
    const int i = k1 >= 0 ? k1 : k1 + g.n1;
    const int j = k2 >= 0 ? k2 : k2 + g.n2;
    return (static_cast<size_t>(i) * g.n2 + j) * (g.n3 / 2 + 1) + k3;
}

// Coarse spectrum of a fine field given by its unnormalised R2C transform F
// (scaled by 1/N here): every coarse mode below the coarse Nyquist, mean
// included (the restriction R of the mean state gradient).
__global__ void __launch_bounds__(kThreads) k_tl_restrict(Grid gf, const float2* __restrict__ F, size_t csf,
                                                           Grid gc, float2* __restrict__ out, size_t csc,
                                                           float invN)
{
    const size_t Mc = static_cast<size_t>(gc.n1) * gc.n2 * (gc.n3 / 2 + 1);
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < Mc;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        int k1, k2, k3;
        wavenumbers(gc, idx, k1, k2, k3);
        const bool keep = below_nyquist(gc, k1, k2, k3);
        const size_t f = keep ? mode_index(gf, k1, k2, k3) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c * csc + idx] = keep ? cmul(invN, F[c * csf + f]) : make_float2(0.f, 0.f);
    }
}

// Start of the inner PCG: r = Q R rf (kept modes of the fine residual), x = 0,
// z = M r, p = z (and its copy cp for the inverse transform); partials of
// |r|^2 and <r, z>.
__global__ void __launch_bounds__(kThreads) k_tl_start(Grid gf, const float2* __restrict__ rf, size_t csf,
                                                        Grid gc, float2* __restrict__ rh, float2* __restrict__ xh,
                                                        float2* __restrict__ ph, float2* __restrict__ cp, size_t cs,
                                                        int op, RegParams rp, double* __restrict__ prr,
                                                        double* __restrict__ prz)
{
    const int n3h = gc.n3 / 2 + 1;
    const size_t Mc = static_cast<size_t>(gc.n1) * gc.n2 * n3h;
    double arr = 0.0, arz = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < Mc;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        int k1, k2, k3;
        wavenumbers(gc, idx, k1, k2, k3);
        const bool keep = below_nyquist(gc, k1, k2, k3) && (k1 | k2 | k3) != 0;
        const size_t f = keep ? mode_index(gf, k1, k2, k3) : 0;
        const float2 zero = make_float2(0.f, 0.f);
        float2 r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = keep ? rf[c * csf + f] : zero;
        const Mode m = mode_of(gc, idx, n3h, rp);
        float2 z[3];
        apply_inv(m, op, r[0], r[1], r[2], z[0], z[1], z[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rh[c * cs + idx] = r[c];
            xh[c * cs + idx] = zero;
            ph[c * cs + idx] = z[c];
            cp[c * cs + idx] = z[c];
        }
        arr += static_cast<double>(m.wt * cdot3(r[0], r[1], r[2], r[0], r[1], r[2]));
        arz += static_cast<double>(m.wt * cdot3(r[0], r[1], r[2], z[0], z[1], z[2]));
    }
    block_sum2(arr, arz, prr, prz);
}

// In place on the coarse real fields: p <- gbar (gbar . p).
__global__ void __launch_bounds__(kThreads) k_tl_rank1(const float* __restrict__ gbar, float* __restrict__ p,
                                                        size_t Nc)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < Nc;
         i += static_cast<size_t>(gridDim.x) * kThreads) {
        const float g0 = gbar[i], g1 = gbar[Nc + i], g2 = gbar[2 * Nc + i];
        const float s = g0 * p[i] + g1 * p[Nc + i] + g2 * p[2 * Nc + i];
        p[i] = s * g0;
        p[Nc + i] = s * g1;
        p[2 * Nc + i] = s * g2;
    }
}

// q = Q (S p + scale T) (K of the sum for the paper's gradient form), T the
// unnormalised transform of gbar (gbar . p); partials of <p, q>.
__global__ void __launch_bounds__(kThreads) k_tl_hp(Grid gc, const float2* __restrict__ T,
                                                     const float2* __restrict__ ph, float2* __restrict__ q,
                                                     size_t cs, int kform, RegParams rp, float scale,
                                                     double* __restrict__ ppq)
{
    const int n3h = gc.n3 / 2 + 1;
    const size_t Mc = static_cast<size_t>(gc.n1) * gc.n2 * n3h;
    double acc = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < Mc;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        int k1, k2, k3;
        wavenumbers(gc, idx, k1, k2, k3);
        const bool keep = below_nyquist(gc, k1, k2, k3) && (k1 | k2 | k3) != 0;
        const Mode m = mode_of(gc, idx, n3h, rp);
        const float2 p0 = ph[idx], p1 = ph[cs + idx], p2 = ph[2 * cs + idx];
        float2 h[3];
        apply_S(m, p0, p1, p2, h[0], h[1], h[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 b = T[c * cs + idx];
            h[c] = make_float2(fmaf(scale, b.x, h[c].x), fmaf(scale, b.y, h[c].y));
        }
        if (kform && m.kk != 0.0f) {
            const float2 ud = make_float2(m.u1 * h[0].x + m.u2 * h[1].x + m.u3 * h[2].x,
                                          m.u1 * h[0].y + m.u2 * h[1].y + m.u3 * h[2].y);
            const float f = m.c / (m.a + m.c * (m.u1 * m.u1 + m.u2 * m.u2 + m.u3 * m.u3));
            h[0] = make_float2(h[0].x - f * m.u1 * ud.x, h[0].y - f * m.u1 * ud.y);
            h[1] = make_float2(h[1].x - f * m.u2 * ud.x, h[1].y - f * m.u2 * ud.y);
            h[2] = make_float2(h[2].x - f * m.u3 * ud.x, h[2].y - f * m.u3 * ud.y);
        }
        if (!keep) h[0] = h[1] = h[2] = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c * cs + idx] = h[c];
        acc += static_cast<double>(m.wt * cdot3(p0, p1, p2, h[0], h[1], h[2]));
    }
    block_sum(acc, ppq);
}

// x += alpha p, r -= alpha q, z = M r (stored); partials of |r|^2 and <r, z>.
// Scalars of the inner PCG kept on the device (slots of TlScalar): after the
// curvature pq (stage 0) alpha = rz / pq, or 0 with the breakdown flag set
// when pq <= 0 (1) or NaN (2); before the direction update (stage 1) beta = rz_new / rz and
// rz <- rz_new.  FP64 divisions, as the host would do them.
__global__ void k_tl_scalars(double* __restrict__ s, int stage)
{
    if (stage == 0) {
        const double pq = s[kTlPq];
        s[kTlAlpha] = pq > 0.0 ? s[kTlRz] / pq : 0.0;
        s[kTlFlag] = pq > 0.0 ? 0.0 : (pq == pq ? 1.0 : 2.0);  // 2: pq is NaN
    } else {
        s[kTlBeta] = s[kTlRzNew] / s[kTlRz];
        s[kTlRz] = s[kTlRzNew];
    }
}

__global__ void __launch_bounds__(kThreads) k_tl_update(Grid gc, const float2* __restrict__ ph,
                                                         const float2* __restrict__ q, float2* __restrict__ xh,
                                                         float2* __restrict__ rh, float2* __restrict__ zh, size_t cs,
                                                         const double* __restrict__ alpha_dev, int op, RegParams rp,
                                                         double* __restrict__ prr, double* __restrict__ prz)
{
    const float alpha = static_cast<float>(*alpha_dev);
    const int n3h = gc.n3 / 2 + 1;
    const size_t Mc = static_cast<size_t>(gc.n1) * gc.n2 * n3h;
    double arr = 0.0, arz = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < Mc;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        float2 r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 p = ph[c * cs + idx], hq = q[c * cs + idx];
            float2 x = xh[c * cs + idx], rr = rh[c * cs + idx];
            x = make_float2(fmaf(alpha, p.x, x.x), fmaf(alpha, p.y, x.y));
            rr = make_float2(fmaf(-alpha, hq.x, rr.x), fmaf(-alpha, hq.y, rr.y));
            xh[c * cs + idx] = x;
            rh[c * cs + idx] = rr;
            r[c] = rr;
        }
        const Mode m = mode_of(gc, idx, n3h, rp);
        float2 z0, z1, z2;
        apply_inv(m, op, r[0], r[1], r[2], z0, z1, z2);
        zh[idx] = z0; zh[cs + idx] = z1; zh[2 * cs + idx] = z2;
        arr += static_cast<double>(m.wt * cdot3(r[0], r[1], r[2], r[0], r[1], r[2]));
        arz += static_cast<double>(m.wt * cdot3(r[0], r[1], r[2], z0, z1, z2));
    }
    block_sum2(arr, arz, prr, prz);
}

// p = z + beta p (p = z when first) and its copy cp for the inverse transform;
// on any grid (the inner PCG, and the outer PCG when z is stored).
__global__ void __launch_bounds__(kThreads) k_dir_stored(Grid g, const float2* __restrict__ zh,
                                                          float2* __restrict__ ph, float2* __restrict__ cp, size_t cs,
                                                          float beta_host, const double* __restrict__ beta_dev,
                                                          int first)
{
    const float beta = beta_dev ? static_cast<float>(*beta_dev) : beta_host;
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * (g.n3 / 2 + 1);
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 z = zh[c * cs + idx];
            float2 p = z;
            if (!first) {
                const float2 o = ph[c * cs + idx];
                p = make_float2(fmaf(beta, o.x, z.x), fmaf(beta, o.y, z.y));
            }
            ph[c * cs + idx] = p;
            cp[c * cs + idx] = p;
        }
    }
}

// Outer preconditioned residual: z = E x (kept coarse modes), r on the mean,
// M r on every other mode; partials of <r, z> and <r, zold> (zold may be null).
__global__ void __launch_bounds__(kThreads) k_tl_finish(Grid gf, const float2* __restrict__ rf,
                                                         float2* __restrict__ zf, const float2* __restrict__ zold,
                                                         size_t csf, Grid gc, const float2* __restrict__ xc,
                                                         size_t csc, int op, RegParams rp, double* __restrict__ prz,
                                                         double* __restrict__ pro)
{
    const int n3h = gf.n3 / 2 + 1;
    const size_t M = static_cast<size_t>(gf.n1) * gf.n2 * n3h;
    double az = 0.0, ao = 0.0;
    for (size_t idx = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; idx < M;
         idx += static_cast<size_t>(gridDim.x) * kThreads) {
        int k1, k2, k3;
        wavenumbers(gf, idx, k1, k2, k3);
        const bool low = below_nyquist(gc, k1, k2, k3) && (k1 | k2 | k3) != 0;
        const Mode m = mode_of(gf, idx, n3h, rp);
        const float2 r0 = rf[idx], r1 = rf[csf + idx], r2 = rf[2 * csf + idx];
        float2 z[3];
        if (low) {
            const size_t ci = mode_index(gc, k1, k2, k3);
#pragma unroll
            for (int c = 0; c < 3; ++c) z[c] = xc[c * csc + ci];
        } else {
            apply_inv(m, op, r0, r1, r2, z[0], z[1], z[2]);  // identity at k = 0
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) zf[c * csf + idx] = z[c];
        az += static_cast<double>(m.wt * cdot3(r0, r1, r2, z[0], z[1], z[2]));
        if (zold)
            ao += static_cast<double>(m.wt * cdot3(r0, r1, r2, zold[idx], zold[csf + idx], zold[2 * csf + idx]));
    }
    block_sum2(az, ao, prz, pro);
}

}  // namespace

void launch_spectral(const Grid& g, cufftComplex* xh, size_t cstride, SpectralOp op, RegParams rp,
                     float scale, cudaStream_t st)
{
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * (g.n3 / 2 + 1);
    k_spectral<<<stream_blocks(M), kThreads, 0, st>>>(g, reinterpret_cast<float2*>(xh), cstride,
                                                     static_cast<int>(op), rp, scale);
}

void launch_spectral_precond(const Grid& g, cufftComplex* xh, size_t cstride, SpectralOp op,
                             RegParams rp, float scale, double* partials, int nblocks, cudaStream_t st)
{
    k_spectral_precond<<<nblocks, kThreads, 0, st>>>(g, reinterpret_cast<float2*>(xh), cstride,
                                                    static_cast<int>(op), rp, scale, partials);
}

void launch_spectral_direction(const Grid& g, const cufftComplex* rh, cufftComplex* ph, cufftComplex* cp,
                               size_t cstride, float beta, int first, SpectralOp op, RegParams rp,
                               cudaStream_t st)
{
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * (g.n3 / 2 + 1);
    k_spectral_direction<<<stream_blocks(M), kThreads, 0, st>>>(
        g, reinterpret_cast<const float2*>(rh), reinterpret_cast<float2*>(ph), reinterpret_cast<float2*>(cp),
        cstride, beta, first, static_cast<int>(op), rp);
}

void launch_fs_start(const Grid& g, cufftComplex* spec, cufftComplex* rh, cufftComplex* xh, size_t cs,
                     SpectralOp op, RegParams rp, float scale, double* prr, double* prz, int nblocks,
                     cudaStream_t st)
{
    k_fs_start<<<nblocks, kThreads, 0, st>>>(g, reinterpret_cast<float2*>(spec), reinterpret_cast<float2*>(rh),
                                             reinterpret_cast<float2*>(xh), cs, static_cast<int>(op), rp,
                                             scale, prr, prz);
}

void launch_fs_hp(const Grid& g, cufftComplex* spec, const cufftComplex* spec2, const cufftComplex* ph,
                  size_t cs, int kform, RegParams rp, float scale, double* ppq, int nblocks, cudaStream_t st)
{
    k_fs_hp<<<nblocks, kThreads, 0, st>>>(g, reinterpret_cast<float2*>(spec),
                                          reinterpret_cast<const float2*>(spec2),
                                          reinterpret_cast<const float2*>(ph), cs, kform, rp, scale, ppq);
}

void launch_fs_update(const Grid& g, cufftComplex* spec, const cufftComplex* ph, cufftComplex* xh,
                      cufftComplex* rh, const cufftComplex* zc, size_t cs, float alpha, SpectralOp op, RegParams rp,
                      double* prr, double* prz, int nblocks, cudaStream_t st)
{
    k_fs_update<<<nblocks, kThreads, 0, st>>>(g, reinterpret_cast<const float2*>(spec),
                                              reinterpret_cast<const float2*>(ph),
                                              reinterpret_cast<float2*>(xh), reinterpret_cast<float2*>(rh),
                                              reinterpret_cast<const float2*>(zc), cs, alpha, static_cast<int>(op),
                                              rp, prr, prz);
}

void launch_mean_levels(const void* m, int nt, float w_end, float w_mid, size_t N, float* out, Storage sto,
                        cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_mean_levels<SType><<<stream_blocks(N), kThreads, 0, st>>>(static_cast<const SType*>(m), nt, w_end, w_mid,
                                                                    N, out);
    });
}

// Coarse preconditioner correction: gbar_c <- sqrt(max(w, 0)) gbar_c on the
// coarse grid (three components of n values), so that the zero-velocity
// operator of the result is S + gbar_c w gbar_c^T.
__global__ void k_tl_weight(float* __restrict__ g, const float* __restrict__ w, size_t n)
{
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float s = sqrtf(fmaxf(w[e], 0.0f));
        g[e] *= s;
        g[n + e] *= s;
        g[2 * n + e] *= s;
    }
}

void launch_tl_weight(float* gbar_c, const float* w, size_t n, cudaStream_t st)
{
    k_tl_weight<<<stream_blocks(n), kThreads, 0, st>>>(gbar_c, w, n);
}

void launch_cscale(cufftComplex* x, size_t n, float s, cudaStream_t st)
{
    k_cscale<<<stream_blocks(n), kThreads, 0, st>>>(reinterpret_cast<float2*>(x), n, s);
}

void launch_tl_restrict(const Grid& gf, const cufftComplex* F, size_t csf, const Grid& gc, cufftComplex* out,
                        size_t csc, float invN, cudaStream_t st)
{
    const size_t Mc = static_cast<size_t>(gc.n1) * gc.n2 * (gc.n3 / 2 + 1);
    k_tl_restrict<<<stream_blocks(Mc), kThreads, 0, st>>>(gf, reinterpret_cast<const float2*>(F), csf, gc,
                                                          reinterpret_cast<float2*>(out), csc, invN);
}

void launch_tl_start(const Grid& gf, const cufftComplex* rf, size_t csf, const Grid& gc, cufftComplex* rh,
                     cufftComplex* xh, cufftComplex* ph, cufftComplex* cp, size_t cs, SpectralOp op, RegParams rp,
                     double* prr, double* prz, int nblocks, cudaStream_t st)
{
    k_tl_start<<<nblocks, kThreads, 0, st>>>(gf, reinterpret_cast<const float2*>(rf), csf, gc,
                                             reinterpret_cast<float2*>(rh), reinterpret_cast<float2*>(xh),
                                             reinterpret_cast<float2*>(ph), reinterpret_cast<float2*>(cp), cs,
                                             static_cast<int>(op), rp, prr, prz);
}

void launch_tl_rank1(const float* gbar, float* p, size_t Nc, cudaStream_t st)
{
    k_tl_rank1<<<stream_blocks(Nc), kThreads, 0, st>>>(gbar, p, Nc);
}

void launch_tl_hp(const Grid& gc, const cufftComplex* T, const cufftComplex* ph, cufftComplex* q, size_t cs,
                  int kform, RegParams rp, float scale, double* ppq, int nblocks, cudaStream_t st)
{
    k_tl_hp<<<nblocks, kThreads, 0, st>>>(gc, reinterpret_cast<const float2*>(T), reinterpret_cast<const float2*>(ph),
                                          reinterpret_cast<float2*>(q), cs, kform, rp, scale, ppq);
}

void launch_tl_update(const Grid& gc, const cufftComplex* ph, const cufftComplex* q, cufftComplex* xh,
                      cufftComplex* rh, cufftComplex* zh, size_t cs, const double* alpha_dev, SpectralOp op,
                      RegParams rp, double* prr, double* prz, int nblocks, cudaStream_t st)
{
    k_tl_update<<<nblocks, kThreads, 0, st>>>(gc, reinterpret_cast<const float2*>(ph),
                                              reinterpret_cast<const float2*>(q), reinterpret_cast<float2*>(xh),
                                              reinterpret_cast<float2*>(rh), reinterpret_cast<float2*>(zh), cs,
                                              alpha_dev, static_cast<int>(op), rp, prr, prz);
}

void launch_tl_scalars(double* s, int stage, cudaStream_t st)
{
    k_tl_scalars<<<1, 1, 0, st>>>(s, stage);
}

void launch_dir_stored(const Grid& g, const cufftComplex* zh, cufftComplex* ph, cufftComplex* cp, size_t cs,
                       float beta, int first, cudaStream_t st, const double* beta_dev)
{
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * (g.n3 / 2 + 1);
    k_dir_stored<<<stream_blocks(M), kThreads, 0, st>>>(g, reinterpret_cast<const float2*>(zh),
                                                        reinterpret_cast<float2*>(ph), reinterpret_cast<float2*>(cp),
                                                        cs, beta, beta_dev, first);
}

void launch_tl_finish(const Grid& gf, const cufftComplex* rf, cufftComplex* zf, const cufftComplex* zold, size_t csf,
                      const Grid& gc, const cufftComplex* xc, size_t csc, SpectralOp op, RegParams rp, double* prz,
                      double* pro, int nblocks, cudaStream_t st)
{
    k_tl_finish<<<nblocks, kThreads, 0, st>>>(gf, reinterpret_cast<const float2*>(rf), reinterpret_cast<float2*>(zf),
                                              reinterpret_cast<const float2*>(zold), csf, gc,
                                              reinterpret_cast<const float2*>(xc), csc, static_cast<int>(op), rp, prz,
                                              pro);
}

void launch_dot_partial(const float* x, const float* y, size_t n, double* partials, int nblocks,
                        cudaStream_t st)
{
    k_dot_partial<<<nblocks, kThreads, 0, st>>>(x, y, n, partials);
}

void launch_sqdiff_partial(const void* a, const void* b, size_t n, double* partials, int nblocks,
                           Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_sqdiff_partial<SType><<<nblocks, kThreads, 0, st>>>(static_cast<const SType*>(a),
                                                             static_cast<const SType*>(b), n, partials);
    });
}

void launch_maxnorm3_partial(const float* v, size_t N, double* partials, int nblocks,
                             cudaStream_t st)
{
    k_maxnorm3_partial<<<nblocks, kThreads, 0, st>>>(v, N, partials);
}

void launch_count_partial(const float* a, const float* b, size_t n, float t, int both, double* pa, double* pb,
                          int nblocks, cudaStream_t st)
{
    k_count_partial<<<nblocks, kThreads, 0, st>>>(a, b, n, t, both, pa, pb);
}

void launch_final_sum(const double* partials, int nblocks, double scale, double* out,
                      cudaStream_t st)
{
    k_final_sum<<<1, kThreads, 0, st>>>(partials, nblocks, scale, out);
}

void launch_final_max(const double* partials, int nblocks, double* out, cudaStream_t st)
{
    // out[0] receives a throw-away min, out[1] the max
    k_final_minmax<<<1, kThreads, 0, st>>>(nullptr, partials, nblocks, out);
}

void launch_final_minmax(const double* pmin, const double* pmax, int nblocks, double* out2,
                         cudaStream_t st)
{
    k_final_minmax<<<1, kThreads, 0, st>>>(pmin, pmax, nblocks, out2);
}

void launch_axpy(float a, const float* x, float* y, size_t n, cudaStream_t st)
{
    k_axpy<<<stream_blocks(n), kThreads, 0, st>>>(a, x, y, n);
}

void launch_xpay(const float* x, float a, const float* y, float* z, size_t n, cudaStream_t st)
{
    k_xpay<<<stream_blocks(n), kThreads, 0, st>>>(x, a, y, z, n);
}

void launch_pcg_update(float alpha, const float* p, const float* q, float* x, float* r, size_t n,
                       double* partials, int nblocks, cudaStream_t st)
{
    k_pcg_update<<<nblocks, kThreads, 0, st>>>(alpha, p, q, x, r, n, partials);
}

void launch_fill(float* x, float value, size_t n, cudaStream_t st)
{
    k_fill<<<stream_blocks(n), kThreads, 0, st>>>(x, value, n);
}

}  // namespace claire

namespace claire {
void launch_bspline_scale(const Grid& g, cufftComplex* spec, size_t M, int ncomp, cudaStream_t st)
{
    const size_t n = M * ncomp;
    k_bspline_scale<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(g, spec, M, ncomp,
                                                                          1.0f / static_cast<float>(g.N));
}
}  // namespace claire
