// Tiled semi-Lagrangian gather for sm_103a.
//
// A CTA owns a TILE1 x TILE2 x TILE3 block of arrival points (x3 fastest; a
// warp covers 32 consecutive x3 nodes of one x2 row, each thread TILE1
// points along x1).  Because the velocity is smooth, the departure points of
// a tile fall in a small box of the grid.  The CTA reduces the box bounds of
// its stencils, copies the box (periodically wrapped) from global memory into
// shared memory with cp.async, and then evaluates every stencil from shared
// memory, so the 64 (cubic) or 8 (linear) reads per point hit on-chip memory
// instead of issuing scattered L1/L2 requests.  A tile whose box does not fit
// (very large local compression of the characteristic map) falls back to the
// direct global-memory gather for that tile only.  The result of each point
// goes to an epilogue functor that fuses the step's source terms.
#pragma once

#include <climits>

#include "common.cuh"

namespace claire {

#ifndef CLAIRE_TILE1
#define CLAIRE_TILE1 4  // arrival points per thread along x1
#endif
#ifndef CLAIRE_TILE_MIN_BLOCKS
#define CLAIRE_TILE_MIN_BLOCKS 4  // resident CTAs per SM the register budget targets
#endif

#ifndef CLAIRE_FFMA2
#define CLAIRE_FFMA2 1  // packed FP32x2 FMA (sm_100+) for the separable stencil contraction
#endif
#ifndef CLAIRE_LDS_ASM
#define CLAIRE_LDS_ASM 1  // explicit 32-bit ld.shared with immediate offsets for the stencil reads
#endif
#ifndef CLAIRE_BOX_CAP
#define CLAIRE_BOX_CAP 11776  // floats of dynamic shared memory per CTA (46 KB)
#endif

#ifndef CLAIRE_TILE2
#define CLAIRE_TILE2 8  // x2 rows per tile: one warp each
#endif

constexpr int TILE1 = CLAIRE_TILE1, TILE2 = CLAIRE_TILE2, TILE3 = 32;

// CTAs of the tiled gathers (in this translation unit) whose box did not fit
// and which took the global-memory path; one atomic per such CTA, read by
// claire_gather_fallback_tiles.
__device__ unsigned long long g_gather_global_tiles = 0;
constexpr int kTileThreads = TILE2 * 32;
constexpr int kBoxCapFloats = CLAIRE_BOX_CAP;

__device__ __forceinline__ void cp_async_f32(float* smem_dst, const float* gmem_src)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int ORDER>
__device__ __forceinline__ void axis_weights(float t, float w[4])
{
    scheme_weights<ORDER>(t, w);
}

// Direct global-memory gather for tiles whose departure box does not fit
// (kept out of line so that it does not add to the register budget of the
// shared-memory path).
template <int ORDER, class S>
__device__ __noinline__ float gather_global(const Grid g, const S* __restrict__ f, int i, int j,
                                            int k, float d1, float d2, float d3)
{
    Stencil<ORDER> s;
    s.build(g, i, j, k, d1, d2, d3);
    return s.template eval<S>(f);
}

// ---- building blocks of the tiled gathers ----

// Geometry of the CTA's stencil box, shared by all threads of the CTA.
struct BoxPar {
    int O1, O2, O3;  // first node (unwrapped grid coordinates)
    int E1, E2, E3;  // extents; E1 == 0 means "does not fit: gather from global memory"
    int S3;          // row stride, a multiple of 32
};

// Box geometry from the bounds [a, z] (per axis) of the first-node cells
// (before the -OFF shift) of a tile's stencils: par[0..2] the first node
// (unwrapped grid coordinates), par[3..5] the extents and par[6] the row
// stride, with par[3..6] = 0 when the box does not fit the shared-memory cap
// or the grid, when the bounds are not ordered (z < a), or when `bad` says
// that a displacement of the tile failed disp_ok (non-finite or at least 2^20
// cells).  Such a tile is gathered from global memory with the clamped split,
// whose indices always wrap into range.
// ES: bytes per stored value of the field (4, or 2 for FP16 / BF16 storage,
// whose box is staged as raw 16-bit pairs before widening to FP32).
template <int ORDER, int ES = 4>
__host__ __device__ __forceinline__ void box_geometry(const Grid& g, int a1, int a2, int a3, int z1, int z2, int z3,
                                                      bool bad, int par[7])
{
    constexpr int M = Scheme<ORDER>::M;
    constexpr int OFF = Scheme<ORDER>::OFF;
    // box of the stencils: cells [a - OFF, z - OFF + M); the tile always
    // holds at least one valid point
    long long o3 = (long long)a3 - OFF;
    long long e3 = (long long)z3 - a3 + M;
    if (ES == 2 && (g.n3 & 7) == 0) {  // x3 origin and extent multiples of 8: 16-byte chunks of halves
        const long long o3e = o3 & ~7LL;
        e3 = (e3 + (o3 - o3e) + 7) & ~7LL;
        o3 = o3e;
    } else if (ES == 2) {  // even x3 origin and extent: 4-byte aligned 16-bit pairs
        const long long o3e = o3 & ~1LL;
        e3 = (e3 + (o3 - o3e) + 1) & ~1LL;
        o3 = o3e;
    } else if ((g.n3 & 3) == 0) {  // x3 origin and extent multiples of 4: 16-byte row chunks
        const long long o3e = o3 & ~3LL;
        e3 = (e3 + (o3 - o3e) + 3) & ~3LL;
        o3 = o3e;
    }
    const long long e1 = (long long)z1 - a1 + M, e2 = (long long)z2 - a2 + M;
    const long long s3 = (e3 + 31) / 32 * 32;  // bank-aligned row stride
    // FP32 box plus, for 16-bit storage, the staging copy (half its size)
    const long long need = e1 * e2 * s3 * (ES == 2 ? 3 : 2) / 2;
    const bool fits = !bad && e1 >= M && e2 >= M && e3 >= M && e1 <= g.n1 && e2 <= g.n2 && e3 <= g.n3 &&
                      need <= kBoxCapFloats;
    par[0] = fits ? a1 - OFF : 0;
    par[1] = fits ? a2 - OFF : 0;
    par[2] = fits ? static_cast<int>(o3) : 0;
    par[3] = static_cast<int>(fits ? e1 : 0);
    par[4] = static_cast<int>(fits ? e2 : 0);
    par[5] = static_cast<int>(fits ? e3 : 0);
    par[6] = static_cast<int>(fits ? s3 : 0);
}

// Fold one point's displacement (grid units) along an axis into the tile's
// bounds of first-node cells; `bad` records a displacement that fails disp_ok.
__host__ __device__ __forceinline__ void bounds_add(int node, float d, int& lo, int& hi, bool& bad)
{
#ifdef __CUDA_ARCH__
    // one floor conversion: for |d| < 2^20 it equals the clamped split; any
    // other value marks the tile bad, whose bounds are then not used
    const int b = node + __float2int_rd(d);
#else
    float t;
    const int b = node + split_disp(d, t);
#endif
    lo = lo < b ? lo : b;
    hi = hi > b ? hi : b;
    bad = bad || !disp_ok(d);
}

#ifdef __CUDACC__
// Block-wide bounds of the first-node cells [lo, hi] per axis and the vote on
// `bad` (any thread).  Thread 0 gets the tile's bounds in b = (a1, a2, a3, z1,
// z2, z3); every thread gets the vote.
__device__ __forceinline__ bool tile_bounds(int lo1, int lo2, int lo3, int hi1, int hi2, int hi3, bool bad,
                                            int (*red)[TILE2], int lane, int warp, int b[6])
{
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
    const bool any_bad = __syncthreads_or(bad) != 0;
    if (threadIdx.x == 0) {
        b[0] = b[1] = b[2] = INT_MAX;
        b[3] = b[4] = b[5] = INT_MIN;
#pragma unroll
        for (int w = 0; w < TILE2; ++w) {
            b[0] = min(b[0], red[0][w]); b[1] = min(b[1], red[1][w]); b[2] = min(b[2], red[2][w]);
            b[3] = max(b[3], red[3][w]); b[4] = max(b[4], red[4][w]); b[5] = max(b[5], red[5][w]);
        }
    }
    return any_bad;
}

// Block-wide box of the stencils whose first-node cells span [lo, hi] per
// axis, with the vote on `bad`; thread 0 publishes the box in par.
template <int ORDER, int ES = 4>
__device__ __forceinline__ BoxPar tile_box(const Grid& g, int lo1, int lo2, int lo3, int hi1, int hi2,
                                           int hi3, bool bad, int (*red)[TILE2], int* par, int lane, int warp)
{
    int b[6];
    const bool any_bad = tile_bounds(lo1, lo2, lo3, hi1, hi2, hi3, bad, red, lane, warp, b);
    if (threadIdx.x == 0) box_geometry<ORDER, ES>(g, b[0], b[1], b[2], b[3], b[4], b[5], any_bad, par);
    __syncthreads();
    BoxPar bp;
    bp.O1 = par[0]; bp.O2 = par[1]; bp.O3 = par[2];
    bp.E1 = par[3]; bp.E2 = par[4]; bp.E3 = par[5]; bp.S3 = par[6];
    return bp;
}

// Tile-bounds table of a displacement field, written by the backtrace that
// produced the field: entry t (the CTA index of the tiled grid, x fastest) is
// tb[2t] = (a1, a2, a3, bad) and tb[2t + 1] = (z1, z2, z3, 0), the first-node
// cell bounds of the tile's points (before the -OFF shift) and whether a
// displacement failed disp_ok.  Only for grids the tiles cover exactly.
__device__ __forceinline__ unsigned tile_index()
{
    return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
}
#endif

#ifndef CLAIRE_F16_OWN_WIDEN
#define CLAIRE_F16_OWN_WIDEN 1  // 16-bit boxes: each thread widens its own chunks (no barrier between)
#endif

// Two 16-bit values packed in a word (low half first) widened to FP32.
template <class S>
__device__ __forceinline__ float2 widen2(uint32_t w)
{
    S lo, hi;
    const unsigned short ulo = static_cast<unsigned short>(w & 0xffffu);
    const unsigned short uhi = static_cast<unsigned short>(w >> 16);
    memcpy(&lo, &ulo, 2);
    memcpy(&hi, &uhi, 2);
    return make_float2(to_f32<S>(lo), to_f32<S>(hi));
}

// Copy the (periodically wrapped) box of f into shared memory as FP32:
// asynchronously (cp.async) for FP32 storage, converting loads otherwise.
template <class S>
__device__ __forceinline__ void box_copy(float* dst, const S* src)
{
    if constexpr (sizeof(S) == 4)
        cp_async_f32(dst, reinterpret_cast<const float*>(src));
    else
        *dst = ldf<S>(src);
}

// Whether the box of f is staged in 16-byte chunks: the x3 origin, the x3
// extent and n3 are multiples of the values per chunk (so no chunk straddles
// the x3 wrap) and f itself is 16-byte aligned (a field passed by a caller
// may start at any 4-byte boundary); otherwise 4-byte copies.
template <class S>
__device__ __forceinline__ bool box_chunks16(const Grid& g, const S* f, const BoxPar& bp)
{
    constexpr int VPC = 16 / static_cast<int>(sizeof(S));
    return ((bp.O3 | bp.E3 | g.n3) & (VPC - 1)) == 0 && (reinterpret_cast<uintptr_t>(f) & 15u) == 0;
}

#ifndef CLAIRE_STAGE_COLS
#define CLAIRE_STAGE_COLS 1  // 16-byte box staging: each thread one (row, chunk) column through all planes
#endif

// 16-byte box staging by columns: thread t owns row b = t / 16 (+16 per
// pass) and chunk c = t % 16 (+16) of every box plane and copies that chunk
// of each of the E1 planes in turn, so the wrapped x2 / x3 indices and the
// row pointer are formed once per (b, c) and a plane costs one address step.
// VPC: values per 16-byte chunk (4 FP32, 8 halves); dst: the box (FP32) or
// the 16-bit staging area, whose row stride is S3 / (4 / sizeof(S)) words.
// Returns nothing; the caller waits for the copies.
template <class S>
__device__ __forceinline__ void stage_box_columns(const Grid& g, const S* __restrict__ f, uint32_t dst0,
                                                  const BoxPar& bp, int w1, int w2, int w3)
{
    constexpr int VPC = 16 / sizeof(S);
    const int nch = bp.E3 / VPC;
    const uint32_t row_bytes = static_cast<uint32_t>(bp.S3) * sizeof(S);
    const uint32_t plane_bytes = row_bytes * static_cast<uint32_t>(bp.E2);
    for (int b = threadIdx.x >> 4; b < bp.E2; b += kTileThreads / 16) {
        int gj = w2 + b;
        gj = gj >= g.n2 ? gj - g.n2 : gj;
        for (int c = threadIdx.x & 15; c < nch; c += 16) {
            int gk = w3 + VPC * c;
            gk = gk >= g.n3 ? gk - g.n3 : gk;
            const S* src = f + static_cast<size_t>(gj) * g.n3 + gk;
            uint32_t dst = dst0 + static_cast<uint32_t>(b) * row_bytes + 16u * c;
            int gi = w1;
            for (int a = 0; a < bp.E1; ++a) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst),
                             "l"(src + static_cast<size_t>(gi) * g.n23)
                             : "memory");
                dst += plane_bytes;
                gi = gi + 1 == g.n1 ? 0 : gi + 1;
            }
        }
    }
}

template <class S>
__device__ __forceinline__ void tile_load_box(const Grid& g, const S* __restrict__ f, float* box,
                                              const BoxPar& bp, int lane, int warp)
{
    const int w1 = wrap_index(bp.O1, g.n1), w2 = wrap_index(bp.O2, g.n2), w3 = wrap_index(bp.O3, g.n3);
    int gk0 = w3 + lane;
    gk0 = gk0 >= g.n3 ? gk0 - g.n3 : gk0;
    int gk1 = w3 + lane + 32;
    gk1 = gk1 >= g.n3 ? gk1 - g.n3 : gk1;
    if constexpr (sizeof(S) == 4) {
#if CLAIRE_STAGE_COLS
        if (box_chunks16<S>(g, f, bp)) {
            stage_box_columns<S>(g, f, static_cast<uint32_t>(__cvta_generic_to_shared(box)), bp, w1, w2, w3);
            return;
        }
#endif
        if (box_chunks16<S>(g, f, bp)) {
            // 16-byte chunks: a chunk never straddles the x3 wrap (n3 and the
            // origin are multiples of 4); 16 threads per row, 16 rows per pass
            const int nch = bp.E3 >> 2, rows = bp.E1 * bp.E2;
            const int ch0 = threadIdx.x & 15;
            int r = threadIdx.x >> 4;
            int a = r / bp.E2, b = r - a * bp.E2;
            for (; r < rows; r += kTileThreads / 16) {
                int gi = w1 + a;
                gi = gi >= g.n1 ? gi - g.n1 : gi;
                int gj = w2 + b;
                gj = gj >= g.n2 ? gj - g.n2 : gj;
                const float* src = reinterpret_cast<const float*>(f) + static_cast<size_t>(gi) * g.n23 +
                                   static_cast<size_t>(gj) * g.n3;
                const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(box + r * bp.S3));
                for (int c = ch0; c < nch; c += 16) {
                    int gk = w3 + 4 * c;
                    gk = gk >= g.n3 ? gk - g.n3 : gk;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * c), "l"(src + gk)
                                 : "memory");
                }
                b += kTileThreads / 16;
                while (b >= bp.E2) {
                    b -= bp.E2;
                    ++a;
                }
            }
            return;
        }
        for (int a = 0; a < bp.E1; ++a) {
            int gi = w1 + a;
            gi = gi >= g.n1 ? gi - g.n1 : gi;
            const S* plane = f + static_cast<size_t>(gi) * g.n23;
            for (int b = warp; b < bp.E2; b += TILE2) {
                int gj = w2 + b;
                gj = gj >= g.n2 ? gj - g.n2 : gj;
                const S* src = plane + gj * g.n3;
                float* dst = box + (a * bp.E2 + b) * bp.S3;
                if (lane < bp.E3) box_copy<S>(dst + lane, src + gk0);
                if (lane + 32 < bp.E3) box_copy<S>(dst + lane + 32, src + gk1);
                for (int c = lane + 64; c < bp.E3; c += 32) {
                    int gk = w3 + c;
                    gk = gk >= g.n3 ? gk - g.n3 : gk;
                    box_copy<S>(dst + c, src + gk);
                }
            }
        }
    } else {
        // 16-bit storage: raw pairs (4 bytes, aligned: even origin, even n3)
        // go asynchronously to a staging area behind the FP32 box; after they
        // land they are widened to FP32 in the box (tile_widen_box: each
        // thread its own copies; else here, after a barrier, a share each).
        const int rows = bp.E1 * bp.E2;
        const int pairs = bp.E3 / 2;
        uint32_t* stage = reinterpret_cast<uint32_t*>(box + rows * bp.S3);
#if CLAIRE_STAGE_COLS
        if (box_chunks16<S>(g, f, bp)) {
            stage_box_columns<S>(g, f, static_cast<uint32_t>(__cvta_generic_to_shared(stage)), bp, w1, w2, w3);
        } else
#endif
        if (box_chunks16<S>(g, f, bp)) {
            // 16-byte chunks of 8 values (no chunk straddles the x3 wrap), 16 threads per row
            const int nch = bp.E3 >> 3;
            const int ch0 = threadIdx.x & 15;
            int r = threadIdx.x >> 4;
            int a = r / bp.E2, b = r - a * bp.E2;
            for (; r < rows; r += kTileThreads / 16) {
                int gi = w1 + a;
                gi = gi >= g.n1 ? gi - g.n1 : gi;
                int gj = w2 + b;
                gj = gj >= g.n2 ? gj - g.n2 : gj;
                const S* src = f + static_cast<size_t>(gi) * g.n23 + static_cast<size_t>(gj) * g.n3;
                const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(stage + r * (bp.S3 / 2)));
                for (int c = ch0; c < nch; c += 16) {
                    int gk = w3 + 8 * c;
                    gk = gk >= g.n3 ? gk - g.n3 : gk;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * c), "l"(src + gk)
                                 : "memory");
                }
                b += kTileThreads / 16;
                while (b >= bp.E2) {
                    b -= bp.E2;
                    ++a;
                }
            }
        } else {
        for (int a = 0; a < bp.E1; ++a) {
            int gi = w1 + a;
            gi = gi >= g.n1 ? gi - g.n1 : gi;
            const S* plane = f + static_cast<size_t>(gi) * g.n23;
            for (int b = warp; b < bp.E2; b += TILE2) {
                int gj = w2 + b;
                gj = gj >= g.n2 ? gj - g.n2 : gj;
                const S* src = plane + gj * g.n3;
                uint32_t* dst = stage + (a * bp.E2 + b) * (bp.S3 / 2);
                for (int c = lane; c < pairs; c += 32) {
                    int gk = w3 + 2 * c;
                    gk = gk >= g.n3 ? gk - g.n3 : gk;
                    cp_async_f32(reinterpret_cast<float*>(dst + c), reinterpret_cast<const float*>(src + gk));
                }
            }
        }
        }
#if !CLAIRE_F16_OWN_WIDEN
        cp_async_wait_all();
        __syncthreads();
        for (int r = warp; r < rows; r += TILE2) {
            const uint32_t* sp = stage + r * (bp.S3 / 2);
            float* dst = box + r * bp.S3;
            for (int c = lane; c < pairs; c += 32) {
                const float2 w = widen2<S>(sp[c]);
                dst[2 * c] = w.x;
                dst[2 * c + 1] = w.y;
            }
        }
#endif
    }
}

// Completion of tile_load_box for 16-bit storage with CLAIRE_F16_OWN_WIDEN:
// every thread waits for its own copies and widens exactly the chunks (or
// pairs) it issued, in the same order, so no barrier separates the copy from
// the widening; the caller's barrier before the stencils publishes the box.
// FP32 storage: nothing (the caller waits for the copies).
template <class S>
__device__ __forceinline__ void tile_widen_box(const Grid& g, const S* f, float* box, const BoxPar& bp, int lane,
                                               int warp)
{
#if CLAIRE_F16_OWN_WIDEN
    if constexpr (sizeof(S) == 2) {
        const int rows = bp.E1 * bp.E2;
        const uint32_t* stage = reinterpret_cast<const uint32_t*>(box + rows * bp.S3);
        cp_async_wait_all();
#if CLAIRE_STAGE_COLS
        if (box_chunks16<S>(g, f, bp)) {
            // the chunks stage_box_columns issued from this thread, in its order
            const int nch = bp.E3 >> 3;
            for (int b = threadIdx.x >> 4; b < bp.E2; b += kTileThreads / 16)
                for (int c = threadIdx.x & 15; c < nch; c += 16)
                    for (int a = 0; a < bp.E1; ++a) {
                        const int r = a * bp.E2 + b;
                        const uint4 w = reinterpret_cast<const uint4*>(stage + r * (bp.S3 / 2))[c];
                        float4* dp = reinterpret_cast<float4*>(box + r * bp.S3);
                        const float2 p0 = widen2<S>(w.x), p1 = widen2<S>(w.y), p2 = widen2<S>(w.z),
                                     p3 = widen2<S>(w.w);
                        dp[2 * c] = make_float4(p0.x, p0.y, p1.x, p1.y);
                        dp[2 * c + 1] = make_float4(p2.x, p2.y, p3.x, p3.y);
                    }
        } else
#endif
        if (box_chunks16<S>(g, f, bp)) {
            const int nch = bp.E3 >> 3;
            const int ch0 = threadIdx.x & 15;
            for (int r = threadIdx.x >> 4; r < rows; r += kTileThreads / 16) {
                const uint4* sp = reinterpret_cast<const uint4*>(stage + r * (bp.S3 / 2));
                float4* dp = reinterpret_cast<float4*>(box + r * bp.S3);
                for (int c = ch0; c < nch; c += 16) {
                    const uint4 w = sp[c];
                    const float2 p0 = widen2<S>(w.x), p1 = widen2<S>(w.y), p2 = widen2<S>(w.z),
                                 p3 = widen2<S>(w.w);
                    dp[2 * c] = make_float4(p0.x, p0.y, p1.x, p1.y);
                    dp[2 * c + 1] = make_float4(p2.x, p2.y, p3.x, p3.y);
                }
            }
        } else {
            const int pairs = bp.E3 / 2;
            for (int a = 0; a < bp.E1; ++a)
                for (int b = warp; b < bp.E2; b += TILE2) {
                    const int r = a * bp.E2 + b;
                    const uint32_t* sp = stage + r * (bp.S3 / 2);
                    float* dst = box + r * bp.S3;
                    for (int c = lane; c < pairs; c += 32) {
                        const float2 w = widen2<S>(sp[c]);
                        dst[2 * c] = w.x;
                        dst[2 * c + 1] = w.y;
                    }
                }
        }
    }
#else
    (void)g; (void)f; (void)box; (void)bp; (void)lane; (void)warp;
#endif
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 32-bit shared-memory load at a byte address plus an immediate byte offset.
template <int BYTE_OFF>
__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];\n" : "=f"(v) : "r"(addr), "n"(BYTE_OFF));
    return v;
}

template <int ORDER>
__device__ __forceinline__ float row_dot(uint32_t addr, const float w[4])
{
    if constexpr (Scheme<ORDER>::M == 4) {
        float s = w[0] * lds_f32<0>(addr);
        s = fmaf(w[1], lds_f32<4>(addr), s);
        s = fmaf(w[2], lds_f32<8>(addr), s);
        return fmaf(w[3], lds_f32<12>(addr), s);
    } else {
        return fmaf(w[1], lds_f32<4>(addr), w[0] * lds_f32<0>(addr));
    }
}

// Split of a displacement inside a fitting box: floor and fraction.  Every
// displacement of a tile whose box fits passed disp_ok (finite, |d| < 2^20),
// where this floor equals the clamped split of the bounds pass; with a box
// from a tile-bounds table, every point also passed in_box.
__host__ __device__ __forceinline__ int split_in_box(float d, float& t)
{
#ifdef __CUDA_ARCH__
    const int fl = __float2int_rd(d);
#else
    // the device conversion: floor, saturated to the int range, NaN to 0
    const float f = floorf(d);
    const int fl = d != d ? 0 : (f >= 2147483648.0f ? INT_MAX : (f < -2147483648.0f ? INT_MIN : static_cast<int>(f)));
#endif
    t = d - static_cast<float>(fl);
    return fl;
}

// Offset in the box (floats) of the first stencil node of the point
// (i, j, k) + (d1, d2, d3), and the three fractions.
template <int ORDER>
__host__ __device__ __forceinline__ int tile_offset(const BoxPar& bp, int i, int j, int k, float d1, float d2,
                                                    float d3, float& t1, float& t2, float& t3)
{
    constexpr int OFF = Scheme<ORDER>::OFF;
    const int P = bp.E2 * bp.S3;
    return (i + split_in_box(d1, t1) - OFF - bp.O1) * P + (j + split_in_box(d2, t2) - OFF - bp.O2) * bp.S3 +
           (k + split_in_box(d3, t3) - OFF - bp.O3);
}

// Whether the stencil of (i, j, k) + (d1, d2, d3) lies inside the box: its
// first-node offsets along each axis in [0, E - M].  The floor saturates for
// |d| >= 2^31 and is 0 for NaN (as the device conversion does), and the
// offsets are formed in unsigned arithmetic, so no input reaches an index
// outside the box without failing this test.
template <int ORDER>
__host__ __device__ __forceinline__ bool in_box(const BoxPar& bp, int i, int j, int k, float d1, float d2, float d3)
{
    constexpr int M = Scheme<ORDER>::M;
    constexpr int OFF = Scheme<ORDER>::OFF;
    float t;
    const unsigned r1 = static_cast<unsigned>(i) - static_cast<unsigned>(OFF + bp.O1) +
                        static_cast<unsigned>(split_in_box(d1, t));
    const unsigned r2 = static_cast<unsigned>(j) - static_cast<unsigned>(OFF + bp.O2) +
                        static_cast<unsigned>(split_in_box(d2, t));
    const unsigned r3 = static_cast<unsigned>(k) - static_cast<unsigned>(OFF + bp.O3) +
                        static_cast<unsigned>(split_in_box(d3, t));
    return bp.E1 >= M && bp.E2 >= M && bp.E3 >= M && r1 <= static_cast<unsigned>(bp.E1 - M) &&
           r2 <= static_cast<unsigned>(bp.E2 - M) && r3 <= static_cast<unsigned>(bp.E3 - M);
}

template <int ORDER>
__device__ __forceinline__ float tile_eval(const float* box, const BoxPar& bp, int i, int j, int k, float d1,
                                           float d2, float d3)
{
    constexpr int M = Scheme<ORDER>::M;
    const int P = bp.E2 * bp.S3;
    float t1, t2, t3, w1[4], w2[4], w3[4];
    const int o = tile_offset<ORDER>(bp, i, j, k, d1, d2, d3, t1, t2, t3);
    axis_weights<ORDER>(t1, w1);
    axis_weights<ORDER>(t2, w2);
    axis_weights<ORDER>(t3, w3);
    float val = 0.0f;
#if CLAIRE_FFMA2
    // rows b and b+1 of plane a are contracted along x3 together in one
    // packed FMA per node; then the x2 weights pair up the same way
    // rows b and b+1 of plane a are contracted together, one packed FMA per
    // x3 node with the products w2[b] w3[c], w2[b+1] w3[c] formed once per point
    const uint32_t base = smem_u32(box) + 4u * static_cast<uint32_t>(o);
    const uint32_t P4 = 4u * static_cast<uint32_t>(P), S4 = 4u * static_cast<uint32_t>(bp.S3);
    float2 W[M / 2][M];
#pragma unroll
    for (int b = 0; b < M; b += 2)
#pragma unroll
        for (int c = 0; c < M; ++c) W[b / 2][c] = __fmul2_rn(make_float2(w2[b], w2[b + 1]), make_float2(w3[c], w3[c]));
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const uint32_t r0a = base + a * P4;
        float2 acc = __fmul2_rn(W[0][0], make_float2(lds_f32<0>(r0a), lds_f32<0>(r0a + S4)));
#pragma unroll
        for (int b = 0; b < M; b += 2) {
            const uint32_t r0 = r0a + b * S4, r1 = r0 + S4;
            if (b > 0) acc = __ffma2_rn(W[b / 2][0], make_float2(lds_f32<0>(r0), lds_f32<0>(r1)), acc);
            acc = __ffma2_rn(W[b / 2][1], make_float2(lds_f32<4>(r0), lds_f32<4>(r1)), acc);
            if constexpr (Scheme<ORDER>::M == 4) {
                acc = __ffma2_rn(W[b / 2][2], make_float2(lds_f32<8>(r0), lds_f32<8>(r1)), acc);
                acc = __ffma2_rn(W[b / 2][3], make_float2(lds_f32<12>(r0), lds_f32<12>(r1)), acc);
            }
        }
        val = fmaf(w1[a], acc.x + acc.y, val);
    }
#elif CLAIRE_LDS_ASM
    const uint32_t base = smem_u32(box) + 4u * static_cast<uint32_t>(o);
    const uint32_t P4 = 4u * static_cast<uint32_t>(P), S4 = 4u * static_cast<uint32_t>(bp.S3);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        float sa = 0.0f;
#pragma unroll
        for (int b = 0; b < M; ++b) sa = fmaf(w2[b], row_dot<ORDER>(base + a * P4 + b * S4, w3), sa);
        val = fmaf(w1[a], sa, val);
    }
#else
#pragma unroll
    for (int a = 0; a < M; ++a) {
        float sa = 0.0f;
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const int row = o + a * P + b * bp.S3;
            float sb = 0.0f;
#pragma unroll
            for (int c = 0; c < M; ++c) sb = fmaf(w3[c], box[row + c], sb);
            sa = fmaf(w2[b], sb, sa);
        }
        val = fmaf(w1[a], sa, val);
    }
#endif
    return val;
}

// Gather f at x + d for the CTA's tile and hand each value to the epilogue.
//
// Shared-memory layout of the box: element (a, b, c) at (a E2 + b) S3 + c
// with the row stride S3 a multiple of 32 floats, so an element's bank is its
// column mod 32 whatever its row: the 32 lanes of a warp (consecutive x3
// arrivals, hence consecutive departure columns, but rows that vary with the
// x1/x2 displacement) read 32 different banks.  The epilogue's operands are
// requested (prefetch) while the box is in flight and consumed (finish) after
// the stencil is evaluated.
// FULL: the tiles cover the grid exactly (n3 % 32 = n2 % 8 = n1 % TILE1 = 0),
// so no point of a tile is out of range and the bounds tests compile away.
// TB (FULL grids only): the box comes from the tile-bounds table tb that the
// backtrace wrote with d, so the CTA starts staging it at once, reads the
// displacements and the epilogue operands while it is in flight, and needs no
// block reduction.  Every point is checked against the box (in_box); if any
// fails, which a table written with this d never causes, the tile takes the
// global-memory path.
template <int ORDER, class Epi, class S, bool FULL, bool TB = false>
__global__ void __launch_bounds__(kTileThreads, CLAIRE_TILE_MIN_BLOCKS)
    k_gather_tiled(Grid g, const S* __restrict__ f, const float* __restrict__ d, Epi epi,
                   const int4* __restrict__ tb = nullptr)
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
    auto valid = [&](int q) { return FULL || (col_ok && i0 + q < g.n1); };

    if constexpr (TB) {
        static_assert(FULL, "tile-bounds tables cover exactly tiled grids only");
        const unsigned t = tile_index();
        const int4 lo = __ldg(tb + 2 * t), hi = __ldg(tb + 2 * t + 1);
        int gp[7];
        box_geometry<ORDER, sizeof(S)>(g, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, lo.w != 0, gp);
        BoxPar bp;
        bp.O1 = gp[0]; bp.O2 = gp[1]; bp.O3 = gp[2];
        bp.E1 = gp[3]; bp.E2 = gp[4]; bp.E3 = gp[5]; bp.S3 = gp[6];
        if (bp.E1 != 0) tile_load_box<S>(g, f, box, bp, lane, warp);  // E1 is the same in every thread
        float e1[TILE1], e2[TILE1], e3[TILE1];
        typename Epi::Pre pre[TILE1];
        bool out = bp.E1 == 0;
#pragma unroll
        for (int q = 0; q < TILE1; ++q) {
            const uint32_t p = p0 + q * g.n23;
            e1[q] = __ldg(d + p);
            e2[q] = __ldg(d + N + p);
            e3[q] = __ldg(d + 2 * N + p);
            pre[q] = epi.prefetch(p);
        }
#pragma unroll
        for (int q = 0; q < TILE1; ++q) out = out || !in_box<ORDER>(bp, i0 + q, j, k, e1[q], e2[q], e3[q]);
        if (bp.E1 != 0) tile_widen_box<S>(g, f, box, bp, lane, warp);
        cp_async_wait_all();
        if (__syncthreads_or(out)) {
            if (threadIdx.x == 0) atomicAdd(&g_gather_global_tiles, 1ull);
#pragma unroll
            for (int q = 0; q < TILE1; ++q)
                epi.finish(p0 + q * g.n23, gather_global<ORDER, S>(g, f, i0 + q, j, k, e1[q], e2[q], e3[q]), pre[q]);
            return;
        }
#pragma unroll
        for (int q = 0; q < TILE1; ++q)
            epi.finish(p0 + q * g.n23, tile_eval<ORDER>(box, bp, i0 + q, j, k, e1[q], e2[q], e3[q]), pre[q]);
        return;
    }
    float d1[TILE1], d2[TILE1], d3[TILE1];
    int lo1 = INT_MAX, lo2 = INT_MAX, lo3 = INT_MAX, hi1 = INT_MIN, hi2 = INT_MIN, hi3 = INT_MIN;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < TILE1; ++q) {
        if (valid(q)) {
            const uint32_t p = p0 + q * g.n23;
            d1[q] = __ldg(d + p);
            d2[q] = __ldg(d + N + p);
            d3[q] = __ldg(d + 2 * N + p);
            bounds_add(i0 + q, d1[q], lo1, hi1, bad);
            bounds_add(j, d2[q], lo2, hi2, bad);
            bounds_add(k, d3[q], lo3, hi3, bad);
        }
    }
    const BoxPar bp = tile_box<ORDER, sizeof(S)>(g, lo1, lo2, lo3, hi1, hi2, hi3, bad, red, par, lane, warp);
    if (bp.E1 == 0) {
        // the tile's box does not fit: gather it from global memory (kept out
        // of the shared-memory path, which then has no call in its loop)
        if (threadIdx.x == 0) atomicAdd(&g_gather_global_tiles, 1ull);
#pragma unroll
        for (int q = 0; q < TILE1; ++q) {
            if (!valid(q)) continue;
            const uint32_t p = p0 + q * g.n23;
            const typename Epi::Pre pr = epi.prefetch(p);
            epi.finish(p, gather_global<ORDER, S>(g, f, i0 + q, j, k, d1[q], d2[q], d3[q]), pr);
        }
        return;
    }
    tile_load_box<S>(g, f, box, bp, lane, warp);
    // epilogue operands of every point are requested while the box is in flight
    typename Epi::Pre pre[TILE1];
#pragma unroll
    for (int q = 0; q < TILE1; ++q)
        if (valid(q)) pre[q] = epi.prefetch(p0 + q * g.n23);
    tile_widen_box<S>(g, f, box, bp, lane, warp);
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TILE1; ++q) {
        if (!valid(q)) continue;
        const float val = tile_eval<ORDER>(box, bp, i0 + q, j, k, d1[q], d2[q], d3[q]);
        epi.finish(p0 + q * g.n23, val, pre[q]);
    }
}

// nf fields f + q N (q < nf) gathered at one displacement d into out + q N:
// the displacements, bounds and box geometry are taken once per tile, and the
// box of each field is staged into the same shared memory in turn.  Per point
// and field this moves (8 nf + 12) / nf bytes instead of 20.
template <int ORDER, bool FULL>
__global__ void __launch_bounds__(kTileThreads, CLAIRE_TILE_MIN_BLOCKS)
    k_gather_tiled_fields(Grid g, const float* __restrict__ f, int nf, const float* __restrict__ d,
                          float* __restrict__ out)
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
    auto valid = [&](int q) { return FULL || (col_ok && i0 + q < g.n1); };
    float d1[TILE1], d2[TILE1], d3[TILE1];
    int lo1 = INT_MAX, lo2 = INT_MAX, lo3 = INT_MAX, hi1 = INT_MIN, hi2 = INT_MIN, hi3 = INT_MIN;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < TILE1; ++q) {
        if (valid(q)) {
            const uint32_t p = p0 + q * g.n23;
            d1[q] = __ldg(d + p);
            d2[q] = __ldg(d + N + p);
            d3[q] = __ldg(d + 2 * N + p);
            bounds_add(i0 + q, d1[q], lo1, hi1, bad);
            bounds_add(j, d2[q], lo2, hi2, bad);
            bounds_add(k, d3[q], lo3, hi3, bad);
        }
    }
    const BoxPar bp = tile_box<ORDER, 4>(g, lo1, lo2, lo3, hi1, hi2, hi3, bad, red, par, lane, warp);
    if (bp.E1 == 0) {
        if (threadIdx.x == 0) atomicAdd(&g_gather_global_tiles, 1ull);
        for (int fld = 0; fld < nf; ++fld)
#pragma unroll
            for (int q = 0; q < TILE1; ++q) {
                if (!valid(q)) continue;
                const uint32_t p = p0 + q * g.n23;
                out[fld * N + p] = gather_global<ORDER, float>(g, f + fld * N, i0 + q, j, k, d1[q], d2[q], d3[q]);
            }
        return;
    }
    for (int fld = 0; fld < nf; ++fld) {
        tile_load_box<float>(g, f + fld * N, box, bp, lane, warp);
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TILE1; ++q) {
            if (!valid(q)) continue;
            out[fld * N + p0 + q * g.n23] = tile_eval<ORDER>(box, bp, i0 + q, j, k, d1[q], d2[q], d3[q]);
        }
        __syncthreads();  // every read of this field's box is done before the next staging
    }
}

inline bool tiles_cover_grid(const Grid& g)
{
    return g.n3 % TILE3 == 0 && g.n2 % TILE2 == 0 && g.n1 % TILE1 == 0;
}

inline dim3 tiled_grid(const Grid& g)
{
    return dim3((g.n3 + TILE3 - 1) / TILE3, (g.n2 + TILE2 - 1) / TILE2, (g.n1 + TILE1 - 1) / TILE1);
}

constexpr size_t kTiledSmemBytes = kBoxCapFloats * sizeof(float);

template <int ORDER, class Epi, class S>
inline void launch_tiled(const Grid& g, const S* f, const float* d, const Epi& e, cudaStream_t st,
                         const int4* tb = nullptr)
{
    if (tiles_cover_grid(g) && tb) {
        if (kTiledSmemBytes > 48 * 1024)
            cudaFuncSetAttribute(k_gather_tiled<ORDER, Epi, S, true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kTiledSmemBytes));
        k_gather_tiled<ORDER, Epi, S, true, true><<<tiled_grid(g), kTileThreads, kTiledSmemBytes, st>>>(g, f, d, e,
                                                                                                        tb);
    } else if (tiles_cover_grid(g)) {
        if (kTiledSmemBytes > 48 * 1024)
            cudaFuncSetAttribute(k_gather_tiled<ORDER, Epi, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kTiledSmemBytes));
        k_gather_tiled<ORDER, Epi, S, true><<<tiled_grid(g), kTileThreads, kTiledSmemBytes, st>>>(g, f, d, e);
    } else {
        if (kTiledSmemBytes > 48 * 1024)
            cudaFuncSetAttribute(k_gather_tiled<ORDER, Epi, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kTiledSmemBytes));
        k_gather_tiled<ORDER, Epi, S, false><<<tiled_grid(g), kTileThreads, kTiledSmemBytes, st>>>(g, f, d, e);
    }
}

// ---- epilogues: prefetch(p) loads the point's operands early, finish(p, v, pre)
// completes; S is the storage type of the fields they read and write ----

// plain interpolation / state step: out = f(X)
template <class S>
struct EpiStore {
    S* __restrict__ out;
    struct Pre {};
    __device__ __forceinline__ Pre prefetch(uint32_t) const { return Pre{}; }
    __device__ __forceinline__ void finish(uint32_t p, float v, const Pre&) const { stf<S>(out + p, v); }
};

// adjoint step (Eq. (4), Heun along X+): lambda^j from lambda^{j+1}(X+)
template <class S>
struct EpiAdjointOnly {
    const S* __restrict__ divv;
    const S* __restrict__ divXp;
    S* __restrict__ lam;
    float dt;
    struct Pre {
        float dX, dx;
    };
    __device__ __forceinline__ Pre prefetch(uint32_t p) const { return Pre{ldf<S>(divXp + p), ldf<S>(divv + p)}; }
    __device__ __forceinline__ void finish(uint32_t p, float a, const Pre& r) const
    {
        const float adX = a * r.dX;
        const float pred = fmaf(dt, adX, a);
        stf<S>(lam + p, fmaf(0.5f * dt, fmaf(pred, r.dx, adX), a));
    }
};

// incremental state with precomputed source: q = f(X) + coef F
template <class S>
struct EpiIncSource {
    const S* __restrict__ F;
    S* __restrict__ q;
    float coef;
    struct Pre {
        float f;
    };
    __device__ __forceinline__ Pre prefetch(uint32_t p) const { return Pre{ldf<S>(F + p)}; }
    __device__ __forceinline__ void finish(uint32_t p, float a, const Pre& r) const
    {
        stf<S>(q + p, fmaf(coef, r.f, a));
    }
};

// last incremental state step, start of the incremental adjoint: lt = -(f(X) + coef F)
template <class S>
struct EpiIncSourceLast {
    const S* F;  // may alias lam: each point reads its F before writing lam
    S* lam;
    float coef;
    struct Pre {
        float f;
    };
    __device__ __forceinline__ Pre prefetch(uint32_t p) const { return Pre{to_f32<S>(F[p])}; }
    __device__ __forceinline__ void finish(uint32_t p, float a, const Pre& r) const
    {
        stf<S>(lam + p, -fmaf(coef, r.f, a));
    }
};

// Incremental state step with its source formed in place (grad m^{j+1}
// stored): f = -vt . grad m^{j+1} at the arrival point, rounded to the
// storage type as a stored source would be, then q = f(X) + coef f.  It
// reads vt and grad m^{j+1} (24 B) instead of a precomputed source (4 B), so
// the pass that wrote every level's source is not needed.
template <class S>
__device__ __forceinline__ float inc_source_at(const float* __restrict__ vt, const S* __restrict__ gm, uint32_t N,
                                               uint32_t p)
{
    const float f = -(__ldg(vt + p) * ldf<S>(gm + p) + __ldg(vt + N + p) * ldf<S>(gm + N + p) +
                      __ldg(vt + 2 * N + p) * ldf<S>(gm + 2 * N + p));
    return to_f32<S>(from_f32<S>(f));
}

template <class S>
struct EpiIncGrad {
    const float* __restrict__ vt;
    const S* __restrict__ gm;  // grad m^{j+1}, 3N values
    S* __restrict__ q;
    float coef;
    uint32_t N;
    struct Pre {
        float f;
    };
    __device__ __forceinline__ Pre prefetch(uint32_t p) const { return Pre{inc_source_at<S>(vt, gm, N, p)}; }
    __device__ __forceinline__ void finish(uint32_t p, float a, const Pre& r) const
    {
        stf<S>(q + p, fmaf(coef, r.f, a));
    }
};

// last step with its source formed in place: lt = -(f(X) + coef f)
template <class S>
struct EpiIncGradLast {
    const float* __restrict__ vt;
    const S* __restrict__ gm;  // grad m^{nt}
    S* __restrict__ lam;
    float coef;
    uint32_t N;
    struct Pre {
        float f;
    };
    __device__ __forceinline__ Pre prefetch(uint32_t p) const { return Pre{inc_source_at<S>(vt, gm, N, p)}; }
    __device__ __forceinline__ void finish(uint32_t p, float a, const Pre& r) const
    {
        stf<S>(lam + p, -fmaf(coef, r.f, a));
    }
};

}  // namespace claire
