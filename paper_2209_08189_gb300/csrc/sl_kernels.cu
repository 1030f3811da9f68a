// Semi-Lagrangian kernels of libclaire (sm_103a): RK2 backtrace, off-grid
// gathers with the fused source terms of the state, adjoint and incremental
// solves, 8th-order finite differences, deformation-map transport and the
// Jacobian determinant.  Method: "CLAIRE at scale" (arXiv 2209.08189),
// Sec. 2.2 (SL with RK2, FD8) and Sec. 3 (IP and FD kernels).
#include "internal.h"
#include "sl_tiled.cuh"

#include <type_traits>

namespace claire {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(uint32_t n) { return (n + kThreads - 1) / kThreads; }

// ---------------------------------------------------------------------------
// gathers
// ---------------------------------------------------------------------------

// Heun characteristic: sign = +1 gives X = x - dt/2 [v(x) + v(x - dt v(x))],
// sign = -1 gives X+ = x + dt/2 [v(x) + v(x + dt v(x))]; d in grid units.
// The three velocity gathers at the predictor point are served from a
// shared-memory box per 4 x 8 x 32 tile (one box, staged once per component;
// the predictor points of a tile share its bounds).  TBW (grids the tiles
// cover exactly): also write the tile-bounds table of d (tile_index order),
// from the same FP32 values that are stored, for the gathers at d.
template <int ORDER, bool FULL, bool TBW>
__global__ void __launch_bounds__(kTileThreads, CLAIRE_TILE_MIN_BLOCKS)
    k_backtrace_tiled(Grid g, const float* __restrict__ v, const float* __restrict__ vc, float dt, float sign,
                      float* __restrict__ d, int4* __restrict__ tb)
{
    extern __shared__ float box[];
    __shared__ int red[6][TILE2];
    __shared__ int par[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * TILE3 + lane;
    const int j = blockIdx.y * TILE2 + warp;
    const int i0 = blockIdx.z * TILE1;
    const size_t N = g.N;
    const bool col_ok = FULL || ((k < g.n3) && (j < g.n2));
    const uint32_t p0 = static_cast<uint32_t>(i0) * g.n23 + j * g.n3 + k;
    const float sdt = sign * dt;
    float u1[TILE1], u2[TILE1], u3[TILE1];
    int lo1 = INT_MAX, lo2 = INT_MAX, lo3 = INT_MAX, hi1 = INT_MIN, hi2 = INT_MIN, hi3 = INT_MIN;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < TILE1; ++q) {
        u1[q] = u2[q] = u3[q] = 0.0f;
        if (FULL || (col_ok && i0 + q < g.n1)) {
            const uint32_t p = p0 + q * g.n23;
            u1[q] = __ldg(v + p) * g.ih1;
            u2[q] = __ldg(v + N + p) * g.ih2;
            u3[q] = __ldg(v + 2 * N + p) * g.ih3;
            bounds_add(i0 + q, -sdt * u1[q], lo1, hi1, bad);
            bounds_add(j, -sdt * u2[q], lo2, hi2, bad);
            bounds_add(k, -sdt * u3[q], lo3, hi3, bad);
        }
    }
    // a non-finite or huge predictor displacement sends the tile to the
    // global-memory gather (clamped split, indices always in range)
    const BoxPar bp = tile_box<ORDER, 4>(g, lo1, lo2, lo3, hi1, hi2, hi3, bad, red, par, lane, warp);
    const bool use_box = bp.E1 != 0;
    if (!use_box && threadIdx.x == 0) atomicAdd(&g_gather_global_tiles, 1ull);
    const float cc = -0.5f * sdt;
    // bounds of the characteristic itself (TBW)
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    bool dbad = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* f = vc + c * N;
        const float ih = c == 0 ? g.ih1 : (c == 1 ? g.ih2 : g.ih3);
        if (use_box) {
            tile_load_box<float>(g, f, box, bp, lane, warp);
            cp_async_wait_all();
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < TILE1; ++q) {
            const int i = i0 + q;
            if (!(FULL || (col_ok && i < g.n1))) continue;
            const float vsq = use_box
                                  ? tile_eval<ORDER>(box, bp, i, j, k, -sdt * u1[q], -sdt * u2[q], -sdt * u3[q])
                                  : gather_global<ORDER, float>(g, f, i, j, k, -sdt * u1[q], -sdt * u2[q],
                                                                -sdt * u3[q]);
            const float uc = c == 0 ? u1[q] : (c == 1 ? u2[q] : u3[q]);
            const float dc = cc * (uc + vsq * ih);
            d[c * N + p0 + q * g.n23] = dc;
            if constexpr (TBW) bounds_add(c == 0 ? i : (c == 1 ? j : k), dc, lo[c], hi[c], dbad);
        }
        if (use_box) __syncthreads();  // every read of this component is done before the next staging
    }
    if constexpr (TBW) {
        static_assert(FULL, "tile-bounds tables cover exactly tiled grids only");
        int b[6];
        const bool any_bad = tile_bounds(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], dbad, red, lane, warp, b);
        if (threadIdx.x == 0) {
            const unsigned t = tile_index();
            tb[2 * t] = make_int4(b[0], b[1], b[2], any_bad ? 1 : 0);
            tb[2 * t + 1] = make_int4(b[3], b[4], b[5], 0);
        }
    }
}

template <int ORDER, bool FULL, bool TBW>
void launch_backtrace_tiled_as(const Grid& g, const float* v, const float* vc, float dt, float sign, float* d,
                               int4* tb, cudaStream_t st)
{
    if (kTiledSmemBytes > 48 * 1024)
        cudaFuncSetAttribute(k_backtrace_tiled<ORDER, FULL, TBW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kTiledSmemBytes));
    k_backtrace_tiled<ORDER, FULL, TBW><<<tiled_grid(g), kTileThreads, kTiledSmemBytes, st>>>(g, v, vc, dt, sign,
                                                                                              d, tb);
}

template <int ORDER>
void launch_backtrace_tiled(const Grid& g, const float* v, const float* vc, float dt, float sign, float* d,
                            int4* tb, cudaStream_t st)
{
    if (tiles_cover_grid(g) && tb)
        launch_backtrace_tiled_as<ORDER, true, true>(g, v, vc, dt, sign, d, tb, st);
    else if (tiles_cover_grid(g))
        launch_backtrace_tiled_as<ORDER, true, false>(g, v, vc, dt, sign, d, nullptr, st);
    else
        launch_backtrace_tiled_as<ORDER, false, false>(g, v, vc, dt, sign, d, nullptr, st);
}

// Sources of the incremental state for every time level at once:
// f^j = -vt . grad m^j; q0 = coef0 f^0 starts the Heun recursion and
// f^1..f^nt go to F (slot j at F + j N).  S: storage of grad m, q0, F.
// ---------------------------------------------------------------------------
// 8th-order central finite differences
// ---------------------------------------------------------------------------

// The 8th-order central difference (grid units) from the values at +s and -s
// nodes, s = 1..4: sum_s c_s (f(+s) - f(-s)) with c_s = 4/5, -1/5, 4/105,
// -1/280 (the standard stencil), accumulated in this order.
__device__ __forceinline__ float fd8_combine(const float fp[4], const float fm[4])
{
    const float cs[4] = {0.8f, -0.2f, 0.0380952380952381f, -0.003571428571428571f};
    float acc = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) acc = fmaf(cs[s], fp[s] - fm[s], acc);
    return acc;
}

template <class S = float>
__device__ __forceinline__ float fd8_axis(const S* __restrict__ f, uint32_t p, int idx, int n,
                                          int stride)
{
    const long base = static_cast<long>(p) - static_cast<long>(idx) * stride;
    float fp[4], fm[4];
#pragma unroll
    for (int s = 1; s <= 4; ++s) {
        int ip = idx + s;
        ip = ip >= n ? ip - n : ip;
        int im = idx - s;
        im = im < 0 ? im + n : im;
        fp[s - 1] = ldf<S>(f + base + static_cast<long>(ip) * stride);
        fm[s - 1] = ldf<S>(f + base + static_cast<long>(im) * stride);
    }
    return fd8_combine(fp, fm);
}

// FD8 gradient of f at node p = (i, j, k), physical units
template <class S>
__device__ __forceinline__ void fd8_grad_at(const Grid& g, const S* __restrict__ f, uint32_t p, int i, int j,
                                            int k, float& g0, float& g1, float& g2)
{
    g0 = fd8_axis<S>(f, p, i, g.n1, g.n23) * g.ih1;
    g1 = fd8_axis<S>(f, p, j, g.n2, g.n3) * g.ih2;
    g2 = fd8_axis<S>(f, p, k, g.n3, 1) * g.ih3;
}

// Incremental-state sources with grad m^j computed here (FD8 of the stored
// states, no stored gradients): f^j = -vt . grad m^j; q0 = coef0 f^0,
// F[j] = f^j for j = 1..nt.
template <class S>
__global__ void __launch_bounds__(kThreads) k_inc_sources_fd(Grid g, const float* __restrict__ vt,
                                                              const S* __restrict__ m, int nt, float coef0,
                                                              S* __restrict__ q0, S* __restrict__ F)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    const float v0 = __ldg(vt + p), v1 = __ldg(vt + N + p), v2 = __ldg(vt + 2 * N + p);
    for (int l = 0; l <= nt; ++l) {
        float g0, g1, g2;
        fd8_grad_at<S>(g, m + l * N, p, i, j, k, g0, g1, g2);
        const float f = -(v0 * g0 + v1 * g1 + v2 * g2);
        if (l == 0)
            stf<S>(q0 + p, coef0 * f);
        else
            stf<S>(F + l * N + p, f);
    }
}

// Gradient body with grad m^j computed here: out_c (+)= sum_j w_j lambda^j grad_c m^j.
template <class S>
__global__ void __launch_bounds__(kThreads) k_body_fd(Grid g, const S* __restrict__ lam, const S* __restrict__ m,
                                                       int nt, float w_end, float w_mid, int accumulate,
                                                       float* __restrict__ out)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
    for (int l = 0; l <= nt; ++l) {
        const float wl = (l == 0 || l == nt ? w_end : w_mid) * ldf<S>(lam + l * N + p);
        float g0, g1, g2;
        fd8_grad_at<S>(g, m + l * N, p, i, j, k, g0, g1, g2);
        b0 = fmaf(wl, g0, b0);
        b1 = fmaf(wl, g1, b1);
        b2 = fmaf(wl, g2, b2);
    }
    if (accumulate) {
        b0 += out[p];
        b1 += out[N + p];
        b2 += out[2 * N + p];
    }
    out[p] = b0;
    out[N + p] = b1;
    out[2 * N + p] = b2;
}

template <class S>
__global__ void __launch_bounds__(kThreads) k_inc_sources(Grid g, const float* __restrict__ vt,
                                                           const S* __restrict__ gm, int nt,
                                                           float coef0, S* __restrict__ q0,
                                                           S* __restrict__ F)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    const size_t N = g.N;
    const float v0 = __ldg(vt + p), v1 = __ldg(vt + N + p), v2 = __ldg(vt + 2 * N + p);
    for (int j = 0; j <= nt; ++j) {
        const S* gj = gm + 3 * j * N;
        const float f = -(v0 * ldf<S>(gj + p) + v1 * ldf<S>(gj + N + p) + v2 * ldf<S>(gj + 2 * N + p));
        if (j == 0)
            stf<S>(q0 + p, coef0 * f);
        else
            stf<S>(F + j * N + p, f);
    }
}

// q0 = coef0 f^0 with f^0 = -vt . grad m^0, the start of the incremental
// state when the later steps form their sources in place (EpiIncGrad).
template <class S>
__global__ void __launch_bounds__(kThreads) k_inc_source0(Grid g, const float* __restrict__ vt,
                                                          const S* __restrict__ gm, float coef0, S* __restrict__ q0)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    stf<S>(q0 + p, coef0 * inc_source_at<S>(vt, gm, g.N, p));
}

// Gradient body by trapezoid in time, added to out (FP32):
// out_c (+)= sum_j w_j lambda^j grad_c m^j, w_0 = w_nt = w_end, else w_mid.
template <class S>
__global__ void __launch_bounds__(kThreads) k_body(Grid g, const S* __restrict__ lam,
                                                    const S* __restrict__ gm, int nt, float w_end,
                                                    float w_mid, int accumulate, float* __restrict__ out)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    const size_t N = g.N;
    float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
    for (int j = 0; j <= nt; ++j) {
        const float wl = (j == 0 || j == nt ? w_end : w_mid) * ldf<S>(lam + j * N + p);
        const S* gj = gm + 3 * j * N;
        b0 = fmaf(wl, ldf<S>(gj + p), b0);
        b1 = fmaf(wl, ldf<S>(gj + N + p), b1);
        b2 = fmaf(wl, ldf<S>(gj + 2 * N + p), b2);
    }
    if (accumulate) {
        b0 += out[p];
        b1 += out[N + p];
        b2 += out[2 * N + p];
    }
    out[p] = b0;
    out[N + p] = b1;
    out[2 * N + p] = b2;
}

// out = a - s in storage S (start of the adjoint: lambda^{nt} = m1 - m^{nt})
template <class S>
__global__ void __launch_bounds__(kThreads) k_sub(const S* __restrict__ a, const S* __restrict__ s,
                                                   S* __restrict__ out, uint32_t n)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p < n) stf<S>(out + p, ldf<S>(a + p) - ldf<S>(s + p));
}

// out = convert(in): FP32 <-> storage S
template <class Si, class So>
__global__ void __launch_bounds__(kThreads) k_convert(const Si* __restrict__ in, So* __restrict__ out,
                                                       uint32_t n)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p < n) stf<So>(out + p, ldf<Si>(in + p));
}

// Deformation map step: u^{j+1} = u^j(X) + (X - x), three components.
template <int ORDER>
__global__ void __launch_bounds__(kThreads) k_map_step(Grid g, const float* __restrict__ u_prev,
                                                        const float* __restrict__ d,
                                                        float* __restrict__ u)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    const float d1 = __ldg(d + p), d2 = __ldg(d + N + p), d3 = __ldg(d + 2 * N + p);
    Stencil<ORDER> s;
    s.build(g, i, j, k, d1, d2, d3);
    float r[3];
    s.eval3(u_prev, g.N, r);
    u[p] = fmaf(d1, g.h1, r[0]);
    u[N + p] = fmaf(d2, g.h2, r[1]);
    u[2 * N + p] = fmaf(d3, g.h3, r[2]);
}

template <class S>
__global__ void __launch_bounds__(kThreads) k_fd8_grad(Grid g, const S* __restrict__ f,
                                                        S* __restrict__ out)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    stf<S>(out + p, fd8_axis<S>(f, p, i, g.n1, g.n23) * g.ih1);
    stf<S>(out + N + p, fd8_axis<S>(f, p, j, g.n2, g.n3) * g.ih2);
    stf<S>(out + 2 * N + p, fd8_axis<S>(f, p, k, g.n3, 1) * g.ih3);
}

// FD8 gradient on grids whose (x2, x3) planes the 8 x 32 tiles cover exactly:
// a CTA owns an 8 x 32 column of kFdZ consecutive x1 planes.  Each plane of the
// tile, with a halo of 4 nodes in x2 and x3 (periodically wrapped), is staged
// in shared memory (two buffers, one barrier per plane) for the x2 and x3
// differences; every thread keeps the nine values of its own column along x1
// in registers for the x1 difference, loading one new plane value per step.
// Each value then crosses HBM about once and L2 about 2.5 times, instead of
// the 24 scattered neighbour loads per point of k_fd8_grad; the arithmetic is
// fd8_combine in the same order, so the results are identical.
constexpr int kFdZ = 16;                           // x1 planes per CTA
constexpr int kFdRows = 8 + 8, kFdCols = 32 + 8;   // staged plane with its halo of 4

template <class S>
__global__ void __launch_bounds__(kThreads) k_fd8_grad_tiled(Grid g, const S* __restrict__ f,
                                                              S* __restrict__ out)
{
    __shared__ float sh[2][kFdRows][kFdCols];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane, j = blockIdx.y * 8 + warp;
    const int i0 = blockIdx.z * kFdZ;
    const int i1 = min(i0 + kFdZ, g.n1);
    const size_t N = g.N;
    // the up to three halo-plane values this thread stages: plane offsets of
    // the wrapped (x2, x3) nodes (n2, n3 >= 8 > 4, so one wrap suffices)
    constexpr int kPlane = kFdRows * kFdCols;
    int soff[3], srow[3], scol[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int e = min(static_cast<int>(threadIdx.x) + u * kThreads, kPlane - 1);
        srow[u] = e / kFdCols;
        scol[u] = e - srow[u] * kFdCols;
        int gj = static_cast<int>(blockIdx.y) * 8 + srow[u] - 4;
        gj = gj < 0 ? gj + g.n2 : (gj >= g.n2 ? gj - g.n2 : gj);
        int gk = static_cast<int>(blockIdx.x) * 32 + scol[u] - 4;
        gk = gk < 0 ? gk + g.n3 : (gk >= g.n3 ? gk - g.n3 : gk);
        soff[u] = gj * g.n3 + gk;
    }
    const bool s2 = threadIdx.x + 2 * kThreads < kPlane;
    const uint32_t col = static_cast<uint32_t>(j) * g.n3 + k;
    auto wrap1 = [&](int i) { return i < 0 ? i + g.n1 : (i >= g.n1 ? i - g.n1 : i); };
    // x1 queue: the column's values at planes i-4 .. i+4
    float q[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) q[s] = ldf<S>(f + static_cast<size_t>(wrap1(i0 - 4 + s)) * g.n23 + col);
    for (int i = i0; i < i1; ++i) {
        const int b = (i - i0) & 1;
        const S* plane = f + static_cast<size_t>(i) * g.n23;
        sh[b][srow[0]][scol[0]] = ldf<S>(plane + soff[0]);
        sh[b][srow[1]][scol[1]] = ldf<S>(plane + soff[1]);
        if (s2) sh[b][srow[2]][scol[2]] = ldf<S>(plane + soff[2]);
        // next plane's column value, requested before the barrier
        const float qn = ldf<S>(f + static_cast<size_t>(wrap1(i + 5)) * g.n23 + col);
        __syncthreads();
        float fp[4], fm[4];
#pragma unroll
        for (int s = 1; s <= 4; ++s) {
            fp[s - 1] = q[4 + s];
            fm[s - 1] = q[4 - s];
        }
        const float d1 = fd8_combine(fp, fm);
#pragma unroll
        for (int s = 1; s <= 4; ++s) {
            fp[s - 1] = sh[b][warp + 4 + s][lane + 4];
            fm[s - 1] = sh[b][warp + 4 - s][lane + 4];
        }
        const float d2 = fd8_combine(fp, fm);
#pragma unroll
        for (int s = 1; s <= 4; ++s) {
            fp[s - 1] = sh[b][warp + 4][lane + 4 + s];
            fm[s - 1] = sh[b][warp + 4][lane + 4 - s];
        }
        const float d3 = fd8_combine(fp, fm);
        const size_t p = static_cast<size_t>(i) * g.n23 + col;
        stf<S>(out + p, d1 * g.ih1);
        stf<S>(out + N + p, d2 * g.ih2);
        stf<S>(out + 2 * N + p, d3 * g.ih3);
#pragma unroll
        for (int s = 0; s < 8; ++s) q[s] = q[s + 1];
        q[8] = qn;
    }
}

// divergence of an FP32 vector field, stored as S
template <class S>
__global__ void __launch_bounds__(kThreads) k_fd8_div(Grid g, const float* __restrict__ v,
                                                       S* __restrict__ out)
{
    const uint32_t p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= g.N) return;
    int i, j, k;
    coords_of(g, p, i, j, k);
    const size_t N = g.N;
    stf<S>(out + p, fd8_axis(v, p, i, g.n1, g.n23) * g.ih1 + fd8_axis(v + N, p, j, g.n2, g.n3) * g.ih2 +
                        fd8_axis(v + 2 * N, p, k, g.n3, 1) * g.ih3);
}

// det(I + grad u) in FP64 with block-wise min / max partials.
__global__ void __launch_bounds__(kThreads) k_detj_minmax(Grid g, const float* __restrict__ u,
                                                           double* __restrict__ pmin,
                                                           double* __restrict__ pmax)
{
    double lo = 1e300, hi = -1e300;
    const size_t N = g.N;
    for (uint32_t p = blockIdx.x * kThreads + threadIdx.x; p < g.N; p += gridDim.x * kThreads) {
        int i, j, k;
        coords_of(g, p, i, j, k);
        double F[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* uc = u + c * N;
            F[c][0] = fd8_axis(uc, p, i, g.n1, g.n23) * g.ih1;
            F[c][1] = fd8_axis(uc, p, j, g.n2, g.n3) * g.ih2;
            F[c][2] = fd8_axis(uc, p, k, g.n3, 1) * g.ih3;
            F[c][c] += 1.0;
        }
        const double det = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                           F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                           F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
        lo = min_nan(lo, det);  // a NaN propagates to both extrema
        hi = max_nan(hi, det);
    }
    block_minmax(lo, hi, pmin, pmax);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

#define CLAIRE_DISPATCH(order, KERNEL, ...)                                       \
    do {                                                                          \
        if ((order) == 3)                                                         \
            KERNEL<3><<<blocks_for(g.N), kThreads, 0, st>>>(__VA_ARGS__);         \
        else if ((order) == 4)                                                    \
            KERNEL<4><<<blocks_for(g.N), kThreads, 0, st>>>(__VA_ARGS__);         \
        else                                                                      \
            KERNEL<1><<<blocks_for(g.N), kThreads, 0, st>>>(__VA_ARGS__);         \
    } while (0)

// tiled gathers: cubic B-spline (order 4) only for FP32 fields
#define CLAIRE_TILED(order, EPI, fs, d, e)                                        \
    do {                                                                          \
        if ((order) == 3)                                                         \
            launch_tiled<3, EPI<SType>, SType>(g, fs, d, e, st, tb);              \
        else if ((order) == 1)                                                    \
            launch_tiled<1, EPI<SType>, SType>(g, fs, d, e, st, tb);              \
        else if constexpr (std::is_same<SType, float>::value)                     \
            launch_tiled<4, EPI<SType>, SType>(g, fs, d, e, st, tb);              \
    } while (0)

void launch_interp(const Grid& g, int order, const void* f, const float* d, void* out, Storage sto,
                   cudaStream_t st, const int4* tb)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        EpiStore<SType> e{static_cast<SType*>(out)};
        const SType* fs = static_cast<const SType*>(f);
        CLAIRE_TILED(order, EpiStore, fs, d, e);
    });
}

template <int ORDER>
void launch_fields_as(const Grid& g, const float* f, int nf, const float* d, float* out, cudaStream_t st)
{
    if (tiles_cover_grid(g)) {
        if (kTiledSmemBytes > 48 * 1024)
            cudaFuncSetAttribute(k_gather_tiled_fields<ORDER, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kTiledSmemBytes));
        k_gather_tiled_fields<ORDER, true><<<tiled_grid(g), kTileThreads, kTiledSmemBytes, st>>>(g, f, nf, d, out);
    } else {
        if (kTiledSmemBytes > 48 * 1024)
            cudaFuncSetAttribute(k_gather_tiled_fields<ORDER, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kTiledSmemBytes));
        k_gather_tiled_fields<ORDER, false><<<tiled_grid(g), kTileThreads, kTiledSmemBytes, st>>>(g, f, nf, d, out);
    }
}

void launch_interp_fields(const Grid& g, int order, const float* f, int nf, const float* d, float* out,
                          cudaStream_t st)
{
    if (order == 3)
        launch_fields_as<3>(g, f, nf, d, out, st);
    else if (order == 4)
        launch_fields_as<4>(g, f, nf, d, out, st);
    else
        launch_fields_as<1>(g, f, nf, d, out, st);
}

cudaError_t gather_fallback_tiles(unsigned long long* count, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(count, g_gather_global_tiles, sizeof(unsigned long long));
    if (e != cudaSuccess || !reset) return e;
    const unsigned long long z = 0;
    return cudaMemcpyToSymbol(g_gather_global_tiles, &z, sizeof(z));
}

void launch_backtrace(const Grid& g, int order, const float* v, const float* vc, float dt, int sign, float* d,
                      cudaStream_t st, int4* tb)
{
    const float* f = vc ? vc : v;
    const float sg = static_cast<float>(sign);
    if (order == 3)
        launch_backtrace_tiled<3>(g, v, f, dt, sg, d, tb, st);
    else if (order == 4)
        launch_backtrace_tiled<4>(g, v, f, dt, sg, d, tb, st);
    else
        launch_backtrace_tiled<1>(g, v, f, dt, sg, d, tb, st);
}

void launch_adj_step(const Grid& g, int order, const void* lam_next, const float* dA, const void* divv,
                     const void* divXp, float dt, void* lam, Storage sto, cudaStream_t st, const int4* tb)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        EpiAdjointOnly<SType> e{static_cast<const SType*>(divv), static_cast<const SType*>(divXp),
                                static_cast<SType*>(lam), dt};
        const SType* fs = static_cast<const SType*>(lam_next);
        CLAIRE_TILED(order, EpiAdjointOnly, fs, dA, e);
    });
}

void launch_inc_sources(const Grid& g, const float* vt, const void* gm, int nt, float coef0, void* q0,
                        void* F, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_inc_sources<SType><<<blocks_for(g.N), kThreads, 0, st>>>(
            g, vt, static_cast<const SType*>(gm), nt, coef0, static_cast<SType*>(q0), static_cast<SType*>(F));
    });
}

void launch_inc_sources_fd(const Grid& g, const float* vt, const void* m, int nt, float coef0, void* q0, void* F,
                           Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_inc_sources_fd<SType><<<blocks_for(g.N), kThreads, 0, st>>>(
            g, vt, static_cast<const SType*>(m), nt, coef0, static_cast<SType*>(q0), static_cast<SType*>(F));
    });
}

void launch_body_fd(const Grid& g, const void* lam, const void* m, int nt, float w_end, float w_mid, int accumulate,
                    float* out, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_body_fd<SType><<<blocks_for(g.N), kThreads, 0, st>>>(g, static_cast<const SType*>(lam),
                                                              static_cast<const SType*>(m), nt, w_end, w_mid,
                                                              accumulate, out);
    });
}

void launch_body(const Grid& g, const void* lam, const void* gm, int nt, float w_end, float w_mid,
                 int accumulate, float* out, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_body<SType><<<blocks_for(g.N), kThreads, 0, st>>>(g, static_cast<const SType*>(lam),
                                                           static_cast<const SType*>(gm), nt, w_end, w_mid,
                                                           accumulate, out);
    });
}

void launch_inc_step_src(const Grid& g, int order, const void* q_prev, const float* d, const void* F,
                         float coef, void* q, Storage sto, cudaStream_t st, const int4* tb)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        EpiIncSource<SType> e{static_cast<const SType*>(F), static_cast<SType*>(q), coef};
        const SType* fs = static_cast<const SType*>(q_prev);
        CLAIRE_TILED(order, EpiIncSource, fs, d, e);
    });
}

void launch_inc_last_src(const Grid& g, int order, const void* q_prev, const float* d, const void* F,
                         float coef, void* lam, Storage sto, cudaStream_t st, const int4* tb)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        EpiIncSourceLast<SType> e{static_cast<const SType*>(F), static_cast<SType*>(lam), coef};
        const SType* fs = static_cast<const SType*>(q_prev);
        CLAIRE_TILED(order, EpiIncSourceLast, fs, d, e);
    });
}

void launch_inc_source0(const Grid& g, const float* vt, const void* gm, float coef0, void* q0, Storage sto,
                        cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_inc_source0<SType><<<blocks_for(g.N), kThreads, 0, st>>>(g, vt, static_cast<const SType*>(gm), coef0,
                                                                   static_cast<SType*>(q0));
    });
}

void launch_inc_step_grad(const Grid& g, int order, const void* q_prev, const float* d, const float* vt,
                          const void* gm, float coef, void* q, Storage sto, cudaStream_t st, const int4* tb)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        EpiIncGrad<SType> e{vt, static_cast<const SType*>(gm), static_cast<SType*>(q), coef, g.N};
        const SType* fs = static_cast<const SType*>(q_prev);
        CLAIRE_TILED(order, EpiIncGrad, fs, d, e);
    });
}

void launch_inc_last_grad(const Grid& g, int order, const void* q_prev, const float* d, const float* vt,
                          const void* gm, float coef, void* lam, Storage sto, cudaStream_t st, const int4* tb)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        EpiIncGradLast<SType> e{vt, static_cast<const SType*>(gm), static_cast<SType*>(lam), coef, g.N};
        const SType* fs = static_cast<const SType*>(q_prev);
        CLAIRE_TILED(order, EpiIncGradLast, fs, d, e);
    });
}

void launch_sub(const void* a, const void* b, void* out, size_t n, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_sub<SType><<<blocks_for(static_cast<uint32_t>(n)), kThreads, 0, st>>>(
            static_cast<const SType*>(a), static_cast<const SType*>(b), static_cast<SType*>(out),
            static_cast<uint32_t>(n));
    });
}

void launch_to_storage(const float* in, void* out, size_t n, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_convert<float, SType><<<blocks_for(static_cast<uint32_t>(n)), kThreads, 0, st>>>(
            in, static_cast<SType*>(out), static_cast<uint32_t>(n));
    });
}

void launch_from_storage(const void* in, float* out, size_t n, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_convert<SType, float><<<blocks_for(static_cast<uint32_t>(n)), kThreads, 0, st>>>(
            static_cast<const SType*>(in), out, static_cast<uint32_t>(n));
    });
}

void launch_map_step(const Grid& g, int order, const float* u_prev, const float* d, float* u,
                     cudaStream_t st)
{
    CLAIRE_DISPATCH(order, k_map_step, g, u_prev, d, u);
}

void launch_fd8_grad(const Grid& g, const void* f, void* out, Storage sto, cudaStream_t st)
{
    if (g.n3 % 32 == 0 && g.n2 % 8 == 0) {
        const dim3 grid(g.n3 / 32, g.n2 / 8, (g.n1 + kFdZ - 1) / kFdZ);
        CLAIRE_STORAGE_DISPATCH(sto, {
            k_fd8_grad_tiled<SType><<<grid, kThreads, 0, st>>>(g, static_cast<const SType*>(f),
                                                               static_cast<SType*>(out));
        });
        return;
    }
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_fd8_grad<SType><<<blocks_for(g.N), kThreads, 0, st>>>(g, static_cast<const SType*>(f),
                                                               static_cast<SType*>(out));
    });
}

void launch_fd8_div(const Grid& g, const float* v, void* out, Storage sto, cudaStream_t st)
{
    CLAIRE_STORAGE_DISPATCH(sto, {
        k_fd8_div<SType><<<blocks_for(g.N), kThreads, 0, st>>>(g, v, static_cast<SType*>(out));
    });
}

void launch_detj_minmax(const Grid& g, const float* u, double* pmin, double* pmax, int nblocks,
                        cudaStream_t st)
{
    k_detj_minmax<<<nblocks, kThreads, 0, st>>>(g, u, pmin, pmax);
}

}  // namespace claire
