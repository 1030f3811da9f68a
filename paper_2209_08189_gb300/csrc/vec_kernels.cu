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

// Symbol S(k) = a I + c u u^T with a = beta_v |k|^2 (H1) or beta_v |k|^4 (H2),
// c = beta_w (1 + |k|^2) and u = k with Nyquist components set to zero.
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

__global__ void __launch_bounds__(kThreads) k_sqdiff_partial(const float* __restrict__ a,
                                                              const float* __restrict__ b, size_t n,
                                                              double* __restrict__ partials)
{
    double acc = 0.0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    const size_t t0 = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    size_t done = 0;
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
    for (size_t i = done + t0; i < n; i += stride) {
        const float d = a[i] - b[i];
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
        hi = (s != s) ? s : fmax(hi, s);
    }
    block_minmax(hi, hi, partials + gridDim.x, partials);
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
        lo = (a != a) ? a : fmin(lo, a);
        hi = (b != b) ? b : fmax(hi, b);
    }
    block_minmax(lo, hi, out2, out2 + 1);
}

__global__ void __launch_bounds__(kThreads) k_axpy(float a, const float* __restrict__ x,
                                                    float* __restrict__ y, size_t n)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n; i += stride)
        y[i] = fmaf(a, x[i], y[i]);
}

__global__ void __launch_bounds__(kThreads) k_xpay(const float* __restrict__ x, float a,
                                                    const float* __restrict__ y,
                                                    float* __restrict__ z, size_t n)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n; i += stride)
        z[i] = fmaf(a, y[i], x[i]);
}

__global__ void __launch_bounds__(kThreads) k_pcg_update(float alpha, const float* __restrict__ p,
                                                          const float* __restrict__ q,
                                                          float* __restrict__ x,
                                                          float* __restrict__ r, size_t n,
                                                          double* __restrict__ partials)
{
    double acc = 0.0;
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n; i += stride) {
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

}  // namespace

void launch_spectral(const Grid& g, cufftComplex* xh, size_t cstride, SpectralOp op, RegParams rp,
                     float scale, cudaStream_t st)
{
    const size_t M = static_cast<size_t>(g.n1) * g.n2 * (g.n3 / 2 + 1);
    k_spectral<<<stream_blocks(M), kThreads, 0, st>>>(g, reinterpret_cast<float2*>(xh), cstride,
                                                     static_cast<int>(op), rp, scale);
}

void launch_dot_partial(const float* x, const float* y, size_t n, double* partials, int nblocks,
                        cudaStream_t st)
{
    k_dot_partial<<<nblocks, kThreads, 0, st>>>(x, y, n, partials);
}

void launch_sqdiff_partial(const float* a, const float* b, size_t n, double* partials, int nblocks,
                           cudaStream_t st)
{
    k_sqdiff_partial<<<nblocks, kThreads, 0, st>>>(a, b, n, partials);
}

void launch_maxnorm3_partial(const float* v, size_t N, double* partials, int nblocks,
                             cudaStream_t st)
{
    k_maxnorm3_partial<<<nblocks, kThreads, 0, st>>>(v, N, partials);
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
