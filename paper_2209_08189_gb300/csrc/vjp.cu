// Reverse-mode derivative of the discrete semi-Lagrangian transport
// (discretise-then-differentiate) for sm_103a.
//
// Forward map (grid units, u = v / h, per node x): predictor y = x - dt u(x),
// U = I[u](y), displacement d = -dt/2 (u(x) + U), X = x + d,
// m^{j+1}(x) = I[m^j](X(x)), j = 0..nt-1 (Sec. 2.2: SL with RK2).
// Given gbar = dL/dm^{nt} the kernels below produce dL/dm^0 and dL/dv:
//   dbar_c  += mbar^{j+1} d_c I[m^j](X)        (interpolant gradient at X)
//   mbar^j   = W(X)^T mbar^{j+1}               (scatter transpose)
//   Ubar     = -dt/2 dbar,  ubar = -dt/2 dbar - dt sum_c Ubar_c grad I[u_c](y)
//              + W(y)^T Ubar                   (through the predictor)
//   vbar     = ubar / h.
// The scatter transposes accumulate 64-bit fixed-point integers, so their
// sums do not depend on the order of the atomic additions: the result is
// bitwise deterministic.
#include "internal.h"

#include <climits>
#include <cmath>

namespace claire {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(size_t n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }

// 1-D basis and its t-derivative.
template <int ORDER>
__device__ __forceinline__ void basis_and_deriv(float t, float w[4], float dw[4])
{
    if constexpr (ORDER == 4) {
        bspline_weights(t, w);
        const float s = 1.0f - t;
        dw[0] = -0.5f * s * s;
        dw[1] = 1.5f * t * t - 2.0f * t;
        dw[2] = -1.5f * t * t + t + 0.5f;
        dw[3] = 0.5f * t * t;
    } else if constexpr (ORDER == 3) {
        cubic_weights(t, w);
        const float t2 = t * t;
        dw[0] = -(1.0f / 6.0f) * (3.0f * t2 - 6.0f * t + 2.0f);
        dw[1] = 0.5f * (3.0f * t2 - 4.0f * t - 1.0f);
        dw[2] = -0.5f * (3.0f * t2 - 2.0f * t - 2.0f);
        dw[3] = (1.0f / 6.0f) * (3.0f * t2 - 1.0f);
    } else {
        w[0] = 1.0f - t;
        w[1] = t;
        dw[0] = -1.0f;
        dw[1] = 1.0f;
    }
}

// Wrapped node offsets and weights (plus derivatives) of one axis.
template <int ORDER>
struct DAxis {
    static constexpr int M = Scheme<ORDER>::M;
    int idx[M];
    float w[4], dw[4];
    __device__ __forceinline__ void build(int node, float disp, int n, int stride)
    {
        float t;
        const int b = wrap_index(node + split_disp(disp, t) - Scheme<ORDER>::OFF, n);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            const int q = b + a;
            idx[a] = (q >= n ? q - n : q) * stride;
        }
        basis_and_deriv<ORDER>(t, w, dw);
    }
};

// Gradient of the interpolant of f at node (i,j,k) + (d1,d2,d3), grid units.
template <int ORDER>
__device__ __forceinline__ void interp_gradient(const Grid& g, const float* __restrict__ f, int i, int j,
                                                int k, float d1, float d2, float d3, float grad[3])
{
    constexpr int M = DAxis<ORDER>::M;
    DAxis<ORDER> a1, a2, a3;
    a1.build(i, d1, g.n1, g.n23);
    a2.build(j, d2, g.n2, g.n3);
    a3.build(k, d3, g.n3, 1);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;  // d1-weighted, plain for d2 and d3 paths
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const float* row = f + a1.idx[a] + a2.idx[b];
            float r = 0.f, rd = 0.f;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                const float fv = __ldg(row + a3.idx[c]);
                r = fmaf(a3.w[c], fv, r);
                rd = fmaf(a3.dw[c], fv, rd);
            }
            s0 = fmaf(a2.w[b], r, s0);
            s1 = fmaf(a2.dw[b], r, s1);
            s2 = fmaf(a2.w[b], rd, s2);
        }
        g0 = fmaf(a1.dw[a], s0, g0);
        g1 = fmaf(a1.w[a], s1, g1);
        g2 = fmaf(a1.w[a], s2, g2);
    }
    grad[0] = g0;
    grad[1] = g1;
    grad[2] = g2;
}

// dbar_c(p) += mbar(p) * d_c I[m](X(p))
template <int ORDER>
__global__ void __launch_bounds__(kThreads) k_grad_accum(Grid g, const float* __restrict__ m,
                                                          const float* __restrict__ d,
                                                          const float* __restrict__ mbar,
                                                          float* __restrict__ dbar)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    float gr[3];
    interp_gradient<ORDER>(g, m, i, j, k, __ldg(d + p), __ldg(d + N + p), __ldg(d + 2 * N + p), gr);
    const float mb = __ldg(mbar + p);
#pragma unroll
    for (int c = 0; c < 3; ++c) dbar[c * N + p] = fmaf(mb, gr[c], dbar[c * N + p]);
}

// Fixed-point scale 2^(48 - e) with max|y| <= 2^e, so every scaled term
// stays below 2^48 in magnitude and a node can receive 2^14 full-size terms
// before the 64-bit sum could overflow.  0 for y = 0, NaN when max|y| is not
// finite (the maximum kernel maps NaN to infinity).
__device__ __forceinline__ double fixed_scale_of(double mx)
{
    if (mx == 0.0) return 0.0;
    if (!isfinite(mx)) return __longlong_as_double(0x7ff8000000000000ll);
    int e;
    frexp(mx, &e);
    return ldexp(1.0, 48 - e);
}

// Displacement of point p (grid units): d if given, else the RK2 predictor -sdt v / h.
__device__ __forceinline__ void scatter_disp(const Grid& g, const float* __restrict__ d,
                                             const float* __restrict__ v, float sdt, uint32_t p, float& d1,
                                             float& d2, float& d3)
{
    const size_t N = g.N;
    if (d) {
        d1 = __ldg(d + p); d2 = __ldg(d + N + p); d3 = __ldg(d + 2 * N + p);
    } else {
        d1 = -sdt * __ldg(v + p) * g.ih1;
        d2 = -sdt * __ldg(v + N + p) * g.ih2;
        d3 = -sdt * __ldg(v + 2 * N + p) * g.ih3;
    }
}

// Fixed-point contribution of (scale y w_a w_b) w_c: the product is formed in
// FP32 (|value| <= 2^48 fits its exponent range; FP64 throughput is low on
// this part) and rounded to the integer grid, so every term is a
// deterministic integer and the sums do not depend on their order.
__device__ __forceinline__ unsigned long long fixed_term(float wab, float wc)
{
    return static_cast<unsigned long long>(__float2ll_rn(wab * wc));
}

// Scatter-transpose tiles: a CTA owns a 4 x 8 x 32 tile of source points
// (256 threads, 4 points each along x1), like the gather tiles.  The
// destination stencils of the tile span a box that is accumulated in shared
// memory (64-bit integer atomics) and flushed with one global atomic per
// touched node, instead of 64 global atomics per point.  Boxes larger than
// kScatterCap nodes fall back to global atomics.  Integer sums do not depend
// on the order of additions, so either path gives the same bits.
constexpr int kST1 = 4, kST2 = 8, kST3 = 32;
constexpr int kScatterCap = 6112;  // 64-bit accumulators: with the static arrays, within 48 KB

template <int ORDER>
__global__ void __launch_bounds__(kThreads) k_scatter_tiled(Grid g, const float* __restrict__ yv,
                                                             const float* __restrict__ d,
                                                             const float* __restrict__ v, float sdt,
                                                             const double* __restrict__ maxabs,
                                                             unsigned long long* __restrict__ acc)
{
    extern __shared__ unsigned long long sbox[];
    __shared__ int red[6][kST2];
    __shared__ int par[7];
    constexpr int M = DAxis<ORDER>::M;
    constexpr int OFF = Scheme<ORDER>::OFF;
    const double scale = fixed_scale_of(*maxabs);
    if (!(scale > 0.0)) return;  // uniform: zero or non-finite cotangent
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.y * kST2 + warp, k = blockIdx.x * kST3 + lane, i0 = blockIdx.z * kST1;
    const bool col_ok = j < g.n2 && k < g.n3;
    float dd[kST1][3], yy[kST1];
    int lo1 = INT_MAX, lo2 = INT_MAX, lo3 = INT_MAX, hi1 = INT_MIN, hi2 = INT_MIN, hi3 = INT_MIN;
#pragma unroll
    for (int q = 0; q < kST1; ++q) {
        yy[q] = 0.0f;
        const int i = i0 + q;
        if (!(col_ok && i < g.n1)) continue;
        const uint32_t p = (static_cast<uint32_t>(i) * g.n2 + j) * g.n3 + k;
        yy[q] = __ldg(yv + p);
        if (yy[q] == 0.0f) continue;
        scatter_disp(g, d, v, sdt, p, dd[q][0], dd[q][1], dd[q][2]);
        float t;
        const int b1 = i + split_disp(dd[q][0], t) - OFF;
        const int b2 = j + split_disp(dd[q][1], t) - OFF;
        const int b3 = k + split_disp(dd[q][2], t) - OFF;
        lo1 = min(lo1, b1); hi1 = max(hi1, b1);
        lo2 = min(lo2, b2); hi2 = max(hi2, b2);
        lo3 = min(lo3, b3); hi3 = max(hi3, b3);
    }
    lo1 = __reduce_min_sync(0xffffffffu, lo1);
    lo2 = __reduce_min_sync(0xffffffffu, lo2);
    lo3 = __reduce_min_sync(0xffffffffu, lo3);
    hi1 = __reduce_max_sync(0xffffffffu, hi1);
    hi2 = __reduce_max_sync(0xffffffffu, hi2);
    hi3 = __reduce_max_sync(0xffffffffu, hi3);
    if (lane == 0) {
        red[0][warp] = lo1; red[1][warp] = lo2; red[2][warp] = lo3;
        red[3][warp] = hi1; red[4][warp] = hi2; red[5][warp] = hi3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a1 = INT_MAX, a2 = INT_MAX, a3 = INT_MAX, z1 = INT_MIN, z2 = INT_MIN, z3 = INT_MIN;
        for (int w = 0; w < kST2; ++w) {
            a1 = min(a1, red[0][w]); a2 = min(a2, red[1][w]); a3 = min(a3, red[2][w]);
            z1 = max(z1, red[3][w]); z2 = max(z2, red[4][w]); z3 = max(z3, red[5][w]);
        }
        par[0] = a1; par[1] = a2; par[2] = a3;
        if (a1 > z1) {
            par[6] = 0;  // no non-zero point in the tile
        } else {
            const long long e1 = (long long)z1 - a1 + M, e2 = (long long)z2 - a2 + M, e3 = (long long)z3 - a3 + M;
            const bool fits = e1 * e2 * e3 <= kScatterCap;
            par[3] = (int)e1; par[4] = (int)e2; par[5] = (int)e3;
            par[6] = fits ? 1 : 2;
        }
    }
    __syncthreads();
    const int mode = par[6];
    if (mode == 0) return;
    const int o1 = par[0], o2 = par[1], o3 = par[2];
    const int e1 = par[3], e2 = par[4], e3 = par[5];
    const int vol = e1 * e2 * e3;
    if (mode == 1)
        for (int t = threadIdx.x; t < vol; t += kThreads) sbox[t] = 0ull;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kST1; ++q) {
        if (yy[q] == 0.0f) continue;
        const int i = i0 + q;
        DAxis<ORDER> a1x, a2x, a3x;
        const float ys = static_cast<float>(scale * static_cast<double>(yy[q]));
        if (mode == 1) {
            // box-relative stencil: unwrapped first node minus the box origin
            float t1, t2, t3;
            const int r1 = i + split_disp(dd[q][0], t1) - OFF - o1;
            const int r2 = j + split_disp(dd[q][1], t2) - OFF - o2;
            const int r3 = k + split_disp(dd[q][2], t3) - OFF - o3;
            float w1[4], w2[4], w3[4], dw[4];
            basis_and_deriv<ORDER>(t1, w1, dw);
            basis_and_deriv<ORDER>(t2, w2, dw);
            basis_and_deriv<ORDER>(t3, w3, dw);
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = 0; b < M; ++b) {
                    const float wab = ys * (w1[a] * w2[b]);
                    unsigned long long* row = sbox + ((r1 + a) * e2 + (r2 + b)) * e3 + r3;
#pragma unroll
                    for (int c = 0; c < M; ++c) atomicAdd(row + c, fixed_term(wab, w3[c]));
                }
        } else {
            a1x.build(i, dd[q][0], g.n1, g.n23);
            a2x.build(j, dd[q][1], g.n2, g.n3);
            a3x.build(k, dd[q][2], g.n3, 1);
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = 0; b < M; ++b) {
                    const float wab = ys * (a1x.w[a] * a2x.w[b]);
                    const size_t row = static_cast<size_t>(a1x.idx[a]) + a2x.idx[b];
#pragma unroll
                    for (int c = 0; c < M; ++c) atomicAdd(acc + row + a3x.idx[c], fixed_term(wab, a3x.w[c]));
                }
        }
    }
    if (mode != 1) return;
    __syncthreads();
    for (int t = threadIdx.x; t < vol; t += kThreads) {
        const unsigned long long val = sbox[t];
        if (!val) continue;
        const int c3 = t % e3, c2 = (t / e3) % e2, c1 = t / (e3 * e2);
        const size_t node = (static_cast<size_t>(wrap_index(o1 + c1, g.n1)) * g.n2 + wrap_index(o2 + c2, g.n2)) *
                                g.n3 + wrap_index(o3 + c3, g.n3);
        atomicAdd(acc + node, val);
    }
}

// out = mult ((accumulate ? out : 0) + acc / scale); acc is cleared for reuse.
__global__ void __launch_bounds__(kThreads) k_fixed_to_float(unsigned long long* __restrict__ acc,
                                                              const double* __restrict__ maxabs,
                                                              int accumulate, float mult,
                                                              float* __restrict__ out, size_t n)
{
    const size_t p = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    if (p >= n) return;
    const double scale = fixed_scale_of(*maxabs);
    double val = 0.0;
    if (scale > 0.0)
        val = static_cast<double>(static_cast<long long>(acc[p])) / scale;
    else if (scale != scale)
        val = scale;  // non-finite cotangent: propagate NaN
    acc[p] = 0ull;
    out[p] = mult * static_cast<float>(accumulate ? val + static_cast<double>(out[p]) : val);
}

// Predictor terms: Ubar = -dt/2 dbar; ubar(x) = -dt/2 dbar(x) - dt sum_c Ubar_c grad I[u_c](y)
// with y = x - dt u(x); writes ubar (grid units) and Ubar.
// vc: the field the predictor interpolates (v itself, or its cubic B-spline
// coefficients); v gives the predictor displacement at the node.
template <int ORDER>
__global__ void __launch_bounds__(kThreads) k_predictor_terms(Grid g, const float* __restrict__ v,
                                                               const float* __restrict__ vc, float dt,
                                                               const float* __restrict__ dbar,
                                                               float* __restrict__ ubar,
                                                               float* __restrict__ Ubar)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    const float ih[3] = {g.ih1, g.ih2, g.ih3};
    const float e1 = -dt * __ldg(v + p) * g.ih1, e2 = -dt * __ldg(v + N + p) * g.ih2,
                e3 = -dt * __ldg(v + 2 * N + p) * g.ih3;
    float yb[3] = {0.f, 0.f, 0.f};
    float Ub[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ub[c] = -0.5f * dt * __ldg(dbar + c * N + p);
        float gr[3];
        interp_gradient<ORDER>(g, vc + c * N, i, j, k, e1, e2, e3, gr);  // gradient of v_c; u_c = v_c ih_c
#pragma unroll
        for (int e = 0; e < 3; ++e) yb[e] = fmaf(Ub[c] * ih[c], gr[e], yb[e]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ubar[c * N + p] = Ub[c];
        ubar[c * N + p] = -0.5f * dt * __ldg(dbar + c * N + p) - dt * yb[c];
    }
}

// y = a (y + x): the unit factor that k_fixed_to_float applies when it
// accumulates, for a term added after a prefilter.
__global__ void __launch_bounds__(kThreads) k_scale_add(float* __restrict__ y, float a, const float* __restrict__ x,
                                                         size_t n)
{
    const size_t p = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x;
    if (p < n) y[p] = a * (y[p] + x[p]);
}

// max |x| over n values; partials hold 2 * gridDim.x doubles
__global__ void __launch_bounds__(kThreads) k_maxabs_partial(const float* __restrict__ x, size_t n,
                                                              double* __restrict__ partials)
{
    double hi = 0.0;
    for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * kThreads)
    {
        const double a = fabs(static_cast<double>(x[i]));
        hi = fmax(hi, a <= 1.0e308 ? a : HUGE_VAL);  // NaN -> infinity, which the reductions keep
    }
    block_minmax(hi, hi, partials + gridDim.x, partials);
}

}  // namespace

void launch_grad_accum(const Grid& g, int order, const float* m, const float* d, const float* mbar, float* dbar,
                       cudaStream_t st)
{
    if (order == 3)
        k_grad_accum<3><<<blocks_for(g.N), kThreads, 0, st>>>(g, m, d, mbar, dbar);
    else if (order == 4)
        k_grad_accum<4><<<blocks_for(g.N), kThreads, 0, st>>>(g, m, d, mbar, dbar);
    else
        k_grad_accum<1><<<blocks_for(g.N), kThreads, 0, st>>>(g, m, d, mbar, dbar);
}

void launch_scatter_fixed(const Grid& g, int order, const float* yv, const float* d, const float* v, float sdt,
                          const double* maxabs, unsigned long long* acc, cudaStream_t st)
{
    const dim3 grid((g.n3 + kST3 - 1) / kST3, (g.n2 + kST2 - 1) / kST2, (g.n1 + kST1 - 1) / kST1);
    const size_t smem = kScatterCap * sizeof(unsigned long long);
    if (order == 3)
        k_scatter_tiled<3><<<grid, kThreads, smem, st>>>(g, yv, d, v, sdt, maxabs, acc);
    else if (order == 4)
        k_scatter_tiled<4><<<grid, kThreads, smem, st>>>(g, yv, d, v, sdt, maxabs, acc);
    else
        k_scatter_tiled<1><<<grid, kThreads, smem, st>>>(g, yv, d, v, sdt, maxabs, acc);
}

void launch_fixed_to_float(unsigned long long* acc, const double* maxabs, int accumulate, float mult, float* out,
                           size_t n, cudaStream_t st)
{
    k_fixed_to_float<<<blocks_for(n), kThreads, 0, st>>>(acc, maxabs, accumulate, mult, out, n);
}

void launch_predictor_terms(const Grid& g, int order, const float* v, const float* vc, float dt, const float* dbar,
                            float* ubar, float* Ubar, cudaStream_t st)
{
    if (order == 3)
        k_predictor_terms<3><<<blocks_for(g.N), kThreads, 0, st>>>(g, v, vc, dt, dbar, ubar, Ubar);
    else if (order == 4)
        k_predictor_terms<4><<<blocks_for(g.N), kThreads, 0, st>>>(g, v, vc, dt, dbar, ubar, Ubar);
    else
        k_predictor_terms<1><<<blocks_for(g.N), kThreads, 0, st>>>(g, v, vc, dt, dbar, ubar, Ubar);
}

void launch_scale_add(float* y, float a, const float* x, size_t n, cudaStream_t st)
{
    k_scale_add<<<blocks_for(n), kThreads, 0, st>>>(y, a, x, n);
}

void launch_maxabs(const float* x, size_t n, double* partials, int nblocks, double* out2, cudaStream_t st)
{
    k_maxabs_partial<<<nblocks, kThreads, 0, st>>>(x, n, partials);
    launch_final_max(partials, nblocks, out2, st);
}

}  // namespace claire
