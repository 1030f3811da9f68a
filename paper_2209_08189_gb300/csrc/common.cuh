// Device-side building blocks shared by the sm_103a kernels of libclaire:
// periodic index wrapping, 1-D interpolation weights and the off-grid gather
// of one or three fields.  Internal header (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "storage.cuh"

namespace claire {

// Grid geometry passed by value to every kernel.
struct Grid {
    int n1, n2, n3;       // nodes per axis, x3 fastest
    int n23;              // n2 * n3
    uint32_t N;           // n1 * n2 * n3 (< 2^31)
    float h1, h2, h3;     // 2 pi / n_c
    float ih1, ih2, ih3;  // n_c / (2 pi)
};

__host__ __device__ __forceinline__ int wrap_index(int x, int n)
{
    int r = x % n;
    return r < 0 ? r + n : r;
}

// Largest displacement magnitude (grid cells) the index arithmetic takes as is.
constexpr float kDispLimit = 1048576.0f;  // 2^20

// Split a grid-unit displacement into its integer cell offset and fraction
// t in [0,1).  The offset is clamped to [-2^20, 2^20] so that index
// arithmetic cannot overflow for absurd inputs (the wrapped index then stays
// in range); a NaN becomes -2^20 with a NaN fraction.
__host__ __device__ __forceinline__ int split_disp(float d, float& t)
{
    float fl = floorf(d);
    t = d - fl;
    fl = fminf(fmaxf(fl, -kDispLimit), kDispLimit);
    return static_cast<int>(fl);
}

// True when d is finite and |d| < 2^20, i.e. when split_disp does not clamp
// and a plain floor gives the same cell (false for NaN and +-Inf).
__host__ __device__ __forceinline__ bool disp_ok(float d) { return fabsf(d) < kDispLimit; }

// Cubic Lagrange cardinal functions on the nodes -1, 0, 1, 2 at t in [0,1):
// w0 = -t (t-1)(t-2)/6, w1 = (t+1)(t-1)(t-2)/2, w2 = -(t+1) t (t-2)/2,
// w3 = (t+1) t (t-1)/6, factored through a = t (t-1) and
// b = (t+1)(t-2) = a - 2 (ten operations; exact 0/1 weights at t = 0).
__device__ __forceinline__ void cubic_weights(float t, float w[4])
{
    const float a = fmaf(t, t, -t);
    const float b = a - 2.0f;
    w[0] = a * fmaf(t, -1.0f / 6.0f, 1.0f / 3.0f);
    w[1] = b * fmaf(t, 0.5f, -0.5f);
    w[2] = b * (-0.5f * t);
    w[3] = a * fmaf(t, 1.0f / 6.0f, 1.0f / 6.0f);
}

// Uniform cubic B-spline basis on the nodes -1, 0, 1, 2 at t in [0,1)
// (applied to prefiltered coefficients, not to the samples).
__device__ __forceinline__ void bspline_weights(float t, float w[4])
{
    const float s = 1.0f - t, t2 = t * t, t3 = t2 * t;
    w[0] = (1.0f / 6.0f) * s * s * s;
    w[1] = (1.0f / 6.0f) * (3.0f * t3 - 6.0f * t2 + 4.0f);
    w[2] = (1.0f / 6.0f) * (-3.0f * t3 + 3.0f * t2 + 3.0f * t + 1.0f);
    w[3] = (1.0f / 6.0f) * t3;
}

// Interpolation schemes: ORDER 1 trilinear (nodes 0, 1), 3 cubic Lagrange
// and 4 cubic B-spline (nodes -1..2).
template <int ORDER>
struct Scheme {
    static constexpr int M = (ORDER == 1) ? 2 : 4;    // nodes per axis
    static constexpr int OFF = (ORDER == 1) ? 0 : 1;  // first node below the cell
};

template <int ORDER>
__device__ __forceinline__ void scheme_weights(float t, float w[4])
{
    if constexpr (ORDER == 3) {
        cubic_weights(t, w);
    } else if constexpr (ORDER == 4) {
        bspline_weights(t, w);
    } else {
        w[0] = 1.0f - t;
        w[1] = t;
    }
}

// Stencil of one axis: wrapped node indices and weights.
template <int ORDER>
struct Axis {
    static constexpr int M = Scheme<ORDER>::M;
    int idx[M];
    float w[M];
    __device__ __forceinline__ void build(int node, float disp, int n)
    {
        float t;
        int base = node + split_disp(disp, t) - Scheme<ORDER>::OFF;
        int b = wrap_index(base, n);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            int q = b + a;
            idx[a] = q >= n ? q - n : q;
        }
        scheme_weights<ORDER>(t, w);
    }
};

// Tensor-product stencil at the off-grid point (i + d1, j + d2, k + d3).
template <int ORDER>
struct Stencil {
    Axis<ORDER> a1, a2, a3;
    __device__ __forceinline__ void build(const Grid& g, int i, int j, int k, float d1, float d2,
                                          float d3)
    {
        a1.build(i, d1, g.n1);
        a2.build(j, d2, g.n2);
        a3.build(k, d3, g.n3);
#pragma unroll
        for (int a = 0; a < Axis<ORDER>::M; ++a) {
            a1.idx[a] *= g.n23;
            a2.idx[a] *= g.n3;
        }
    }
    // Separable contraction: x3 first (contiguous loads), then x2, then x1.
    template <class S = float>
    __device__ __forceinline__ float eval(const S* __restrict__ f) const
    {
        constexpr int M = Axis<ORDER>::M;
        float r = 0.0f;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            float sa = 0.0f;
#pragma unroll
            for (int b = 0; b < M; ++b) {
                const S* row = f + a1.idx[a] + a2.idx[b];
                float sb = 0.0f;
#pragma unroll
                for (int c = 0; c < M; ++c) sb = fmaf(a3.w[c], ldf<S>(row + a3.idx[c]), sb);
                sa = fmaf(a2.w[b], sb, sa);
            }
            r = fmaf(a1.w[a], sa, r);
        }
        return r;
    }
    // Three fields sharing the stencil (f, f + stride, f + 2 stride).
    __device__ __forceinline__ void eval3(const float* __restrict__ f, uint32_t stride,
                                          float out[3]) const
    {
        constexpr int M = Axis<ORDER>::M;
        float r0 = 0.0f, r1 = 0.0f, r2 = 0.0f;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
            for (int b = 0; b < M; ++b) {
                const float* row = f + a1.idx[a] + a2.idx[b];
                float q0 = 0.0f, q1 = 0.0f, q2 = 0.0f;
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const int o = a3.idx[c];
                    q0 = fmaf(a3.w[c], __ldg(row + o), q0);
                    q1 = fmaf(a3.w[c], __ldg(row + stride + o), q1);
                    q2 = fmaf(a3.w[c], __ldg(row + 2 * stride + o), q2);
                }
                s0 = fmaf(a2.w[b], q0, s0);
                s1 = fmaf(a2.w[b], q1, s1);
                s2 = fmaf(a2.w[b], q2, s2);
            }
            r0 = fmaf(a1.w[a], s0, r0);
            r1 = fmaf(a1.w[a], s1, r1);
            r2 = fmaf(a1.w[a], s2, r2);
        }
        out[0] = r0;
        out[1] = r1;
        out[2] = r2;
    }
};

// Grid coordinates of linear index p.
__device__ __forceinline__ void coords_of(const Grid& g, uint32_t p, int& i, int& j, int& k)
{
    i = static_cast<int>(p / static_cast<uint32_t>(g.n23));
    uint32_t r = p - static_cast<uint32_t>(i) * static_cast<uint32_t>(g.n23);
    j = static_cast<int>(r / static_cast<uint32_t>(g.n3));
    k = static_cast<int>(r - static_cast<uint32_t>(j) * static_cast<uint32_t>(g.n3));
}

}  // namespace claire
