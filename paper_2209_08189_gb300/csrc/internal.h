// Internal declarations of libclaire: kernel launchers (one per kernel) and
// block-level reduction helpers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>

#include "claire.h"
#include "common.cuh"

namespace claire {

// ---- block reductions (256-thread blocks, fixed order: deterministic) ----
#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Sum of x over the block written to out[blockIdx.x] by thread 0.
__device__ __forceinline__ void block_sum(double x, double* out)
{
    __shared__ double sh[32];
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double y = lane < nw ? sh[lane] : 0.0;
        y = warp_sum(y);
        if (lane == 0) out[blockIdx.x] = y;
    }
}

// min / max that keep a NaN operand (fmin / fmax return the other operand),
// so that a NaN anywhere in a reduction reaches its result
__device__ __forceinline__ double min_nan(double a, double b) { return (a != a || b != b) ? a + b : fmin(a, b); }
__device__ __forceinline__ double max_nan(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

// Block minimum of lo and maximum of hi into pmin / pmax[blockIdx.x]; a NaN
// in either propagates to that result.
__device__ __forceinline__ void block_minmax(double lo, double hi, double* pmin, double* pmax)
{
    __shared__ double slo[32], shi[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min_nan(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = max_nan(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        slo[wid] = lo;
        shi[wid] = hi;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double a = lane < nw ? slo[lane] : 1e300;
        double b = lane < nw ? shi[lane] : -1e300;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = min_nan(a, __shfl_down_sync(0xffffffffu, a, o));
            b = max_nan(b, __shfl_down_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
            pmin[blockIdx.x] = a;
            pmax[blockIdx.x] = b;
        }
    }
}
#endif

// ---- semi-Lagrangian and FD kernels (sl_kernels.cu) ----
// Pointers typed void* hold scalar fields in the storage type `sto` (FP32,
// FP16 or BF16); float* ones are always FP32 (displacements, velocities,
// vector work fields).
// tb: the tile-bounds table of d written by launch_backtrace (or null: the
// gathers reduce the bounds themselves); used on grids the tiles cover exactly
void launch_interp(const Grid& g, int order, const void* f, const float* d, void* out, Storage sto,
                   cudaStream_t st, const int4* tb = nullptr);
// nf FP32 fields [nf][N] at one displacement into out [nf][N]
void launch_interp_fields(const Grid& g, int order, const float* f, int nf, const float* d, float* out,
                          cudaStream_t st);
// CTAs of the tiled gathers that took the global-memory path (device-wide counter)
cudaError_t gather_fallback_tiles(unsigned long long* count, bool reset);
// tb (may be null): also write the tile-bounds table of d (2 int4 per tile of
// the tiled grid) on grids the tiles cover exactly
void launch_backtrace(const Grid& g, int order, const float* v, const float* vc, float dt, int sign, float* d,
                      cudaStream_t st, int4* tb = nullptr);
// One SL step of Eq. (4): lam = Heun(lam_next(X+), div v(X+), div v).
void launch_adj_step(const Grid& g, int order, const void* lam_next, const float* dA, const void* divv,
                     const void* divXp, float dt, void* lam, Storage sto, cudaStream_t st,
                     const int4* tb = nullptr);
// f^j = -vt . grad m^j for j = 0..nt: q0 = coef0 f^0, F + j N <- f^j (j >= 1).
void launch_inc_sources(const Grid& g, const float* vt, const void* gm, int nt, float coef0, void* q0,
                        void* F, Storage sto, cudaStream_t st);
// out (+)= sum_j w_j lam^j grad m^j (lam slots j N, trapezoid weights w_end / w_mid).
// as launch_inc_sources / launch_body, with grad m^j computed from the stored states m (FD8)
void launch_inc_sources_fd(const Grid& g, const float* vt, const void* m, int nt, float coef0, void* q0, void* F,
                           Storage sto, cudaStream_t st);
void launch_body_fd(const Grid& g, const void* lam, const void* m, int nt, float w_end, float w_mid, int accumulate,
                    float* out, Storage sto, cudaStream_t st);
void launch_body(const Grid& g, const void* lam, const void* gm, int nt, float w_end, float w_mid,
                 int accumulate, float* out, Storage sto, cudaStream_t st);
// q = q_prev(X) + coef F;   lam = -(q_prev(X) + coef F)  (F may alias lam)
void launch_inc_step_src(const Grid& g, int order, const void* q_prev, const float* d, const void* F,
                         float coef, void* q, Storage sto, cudaStream_t st, const int4* tb = nullptr);
void launch_inc_last_src(const Grid& g, int order, const void* q_prev, const float* d, const void* F,
                         float coef, void* lam, Storage sto, cudaStream_t st, const int4* tb = nullptr);
#ifndef CLAIRE_INC_FUSED
#define CLAIRE_INC_FUSED 1  // incremental state steps form their sources in place when grad m^j is stored
#endif
// With grad m^j stored: q0 = coef0 f^0, and the steps above with the source
// f^{j+1} = -vt . grad m^{j+1} formed at each arrival point (gm: grad m^{j+1},
// 3N values in `sto`), so no pass writes the sources of every level.
void launch_inc_source0(const Grid& g, const float* vt, const void* gm, float coef0, void* q0, Storage sto,
                        cudaStream_t st);
void launch_inc_step_grad(const Grid& g, int order, const void* q_prev, const float* d, const float* vt,
                          const void* gm, float coef, void* q, Storage sto, cudaStream_t st, const int4* tb = nullptr);
void launch_inc_last_grad(const Grid& g, int order, const void* q_prev, const float* d, const float* vt,
                          const void* gm, float coef, void* lam, Storage sto, cudaStream_t st,
                          const int4* tb = nullptr);
// out = a - b; conversions FP32 <-> storage
void launch_sub(const void* a, const void* b, void* out, size_t n, Storage sto, cudaStream_t st);
void launch_to_storage(const float* in, void* out, size_t n, Storage sto, cudaStream_t st);
void launch_from_storage(const void* in, float* out, size_t n, Storage sto, cudaStream_t st);
void launch_map_step(const Grid& g, int order, const float* u_prev, const float* d, float* u,
                     cudaStream_t st);
void launch_fd8_grad(const Grid& g, const void* f, void* out, Storage sto, cudaStream_t st);
void launch_fd8_div(const Grid& g, const float* v, void* out, Storage sto, cudaStream_t st);
void launch_detj_minmax(const Grid& g, const float* u, double* pmin, double* pmax, int nblocks,
                        cudaStream_t st);

// ---- context accessors for host-side drivers in other units (engine.cu) ----
cudaStream_t ctx_stream(const claire_ctx* c);
size_t ctx_points(const claire_ctx* c);
claire_status ctx_fail(claire_ctx* c, claire_status st, const char* msg);

// spectra of ncomp fields divided by N times the sampled cubic B-spline symbol (vec_kernels.cu)
void launch_bspline_scale(const Grid& g, cufftComplex* spec, size_t M, int ncomp, cudaStream_t st);

// ---- reverse-mode transport (vjp.cu) ----
// dbar_c += mbar * d_c I[m](X)   (interpolant gradient at x + d, grid units)
void launch_grad_accum(const Grid& g, int order, const float* m, const float* d, const float* mbar, float* dbar,
                       cudaStream_t st);
// acc += fixed-point(W(x + disp)^T yv), scale from *maxabs = max |yv| (device);
// disp = d, or -sdt v / h when d is null
void launch_scatter_fixed(const Grid& g, int order, const float* yv, const float* d, const float* v, float sdt,
                          const double* maxabs, unsigned long long* acc, cudaStream_t st);
// out = mult ((accumulate ? out : 0) + acc / scale); clears acc
void launch_fixed_to_float(unsigned long long* acc, const double* maxabs, int accumulate, float mult, float* out,
                           size_t n, cudaStream_t st);
// predictor terms of the velocity cotangent (grid units): ubar, Ubar from dbar
// y = a (y + x)
void launch_scale_add(float* y, float a, const float* x, size_t n, cudaStream_t st);
void launch_predictor_terms(const Grid& g, int order, const float* v, const float* vc, float dt, const float* dbar,
                            float* ubar, float* Ubar, cudaStream_t st);
// out2[1] = max |x| (out2[0] scratch)
void launch_maxabs(const float* x, size_t n, double* partials, int nblocks, double* out2, cudaStream_t st);

// ---- spectral scaling, vector ops and reductions (vec_kernels.cu) ----
enum SpectralOp { SPEC_REG = 0, SPEC_INV = 1, SPEC_K = 2, SPEC_AINV = 3 };

struct RegParams {
    float beta_v, beta_w;
    int reg;  // 1 = H1 seminorm, 2 = H2 seminorm
};

// In-place scaling of the three half-spectra xh[c], c = 0..2 (each
// n1 * n2 * (n3/2+1) complex values, stride cstride) by the 3x3 symbol of op,
// times scale (the 1/N of the unnormalised inverse transform).
void launch_spectral(const Grid& g, cufftComplex* xh, size_t cstride, SpectralOp op,
                     RegParams rp, float scale, cudaStream_t st);

// PCG preconditioner in Fourier space: xh <- scale * M(k) xh (SPEC_INV or
// SPEC_AINV) with block partial sums of sum_x r z (Parseval) in partials.
void launch_spectral_precond(const Grid& g, cufftComplex* xh, size_t cstride, SpectralOp op,
                             RegParams rp, float scale, double* partials, int nblocks, cudaStream_t st);
// PCG direction in Fourier space: ph = zh + beta ph (first: ph = zh), cp = ph, zh <- S ph.
void launch_spectral_direction(const Grid& g, const cufftComplex* rh, cufftComplex* ph, cufftComplex* cp,
                               size_t cstride, float beta, int first, SpectralOp op, RegParams rp,
                               cudaStream_t st);

// Fourier-space PCG (vectors are half spectra scaled by 1/N; partial sums are
// of sum_k wt Re(conj(a) b), wt the multiplicity of the mode):
//   start:  r~ = -scale spec, x~ = 0, spec <- M r~;  partials |r~|^2 (prr), <r~, M r~> (prz)
//   hp:     spec <- spec + scale spec2 (K applied if kform);  partials <p~, H p~>
//   update: x~ += alpha p~, r~ -= alpha spec, spec <- M r~;  partials as in start
void launch_fs_start(const Grid& g, cufftComplex* spec, cufftComplex* rh, cufftComplex* xh, size_t cs,
                     SpectralOp op, RegParams rp, float scale, double* prr, double* prz, int nblocks,
                     cudaStream_t st);
void launch_fs_hp(const Grid& g, cufftComplex* spec, const cufftComplex* spec2, const cufftComplex* ph,
                  size_t cs, int kform, RegParams rp, float scale, double* ppq, int nblocks, cudaStream_t st);
void launch_fs_update(const Grid& g, cufftComplex* spec, const cufftComplex* ph, cufftComplex* xh,
                      cufftComplex* rh, const cufftComplex* zc, size_t cs, float alpha, SpectralOp op, RegParams rp,
                      double* prr, double* prz, int nblocks, cudaStream_t st);

// Deterministic FP64 reductions: partial sums per block, then a one-block
// final sum in fixed order.  `partials` holds at least nblocks doubles.
// two-level zero-velocity preconditioner (coarse grid gc of the fine grid gf; cs* = component strides)
void launch_mean_levels(const void* m, int nt, float w_end, float w_mid, size_t N, float* out, Storage sto,
                        cudaStream_t st);
void launch_cscale(cufftComplex* x, size_t n, float s, cudaStream_t st);
void launch_tl_restrict(const Grid& gf, const cufftComplex* F, size_t csf, const Grid& gc, cufftComplex* out,
                        size_t csc, float invN, cudaStream_t st);
// coarse preconditioner correction: gbar_c [3][n] <- sqrt(max(w, 0)) gbar_c
void launch_tl_weight(float* gbar_c, const float* w, size_t n, cudaStream_t st);
void launch_tl_start(const Grid& gf, const cufftComplex* rf, size_t csf, const Grid& gc, cufftComplex* rh,
                     cufftComplex* xh, cufftComplex* ph, cufftComplex* cp, size_t cs, SpectralOp op, RegParams rp,
                     double* prr, double* prz, int nblocks, cudaStream_t st);
void launch_tl_rank1(const float* gbar, float* p, size_t Nc, cudaStream_t st);
void launch_tl_hp(const Grid& gc, const cufftComplex* T, const cufftComplex* ph, cufftComplex* q, size_t cs,
                  int kform, RegParams rp, float scale, double* ppq, int nblocks, cudaStream_t st);
// Device scalars of the inner PCG (slots of a small FP64 array)
constexpr int kTlRz = 0, kTlPq = 1, kTlAlpha = 2, kTlRr = 3, kTlFlag = 4, kTlRzNew = 5, kTlBeta = 6, kTlSlots = 8;
// stage 0: alpha = rz / pq (0 and the breakdown flag when pq <= 0); stage 1: beta = rz_new / rz, rz <- rz_new
void launch_tl_scalars(double* s, int stage, cudaStream_t st);
void launch_tl_update(const Grid& gc, const cufftComplex* ph, const cufftComplex* q, cufftComplex* xh,
                      cufftComplex* rh, cufftComplex* zh, size_t cs, const double* alpha_dev, SpectralOp op,
                      RegParams rp, double* prr, double* prz, int nblocks, cudaStream_t st);
// beta from beta_dev when it is not null, else the host value
void launch_dir_stored(const Grid& g, const cufftComplex* zh, cufftComplex* ph, cufftComplex* cp, size_t cs,
                       float beta, int first, cudaStream_t st, const double* beta_dev = nullptr);
void launch_tl_finish(const Grid& gf, const cufftComplex* rf, cufftComplex* zf, const cufftComplex* zold, size_t csf,
                      const Grid& gc, const cufftComplex* xc, size_t csc, SpectralOp op, RegParams rp, double* prz,
                      double* pro, int nblocks, cudaStream_t st);
void launch_dot_partial(const float* x, const float* y, size_t n, double* partials, int nblocks,
                        cudaStream_t st);
void launch_sqdiff_partial(const void* a, const void* b, size_t n, double* partials, int nblocks,
                           Storage sto, cudaStream_t st);
void launch_maxnorm3_partial(const float* v, size_t N, double* partials, int nblocks,
                             cudaStream_t st);
// Dice counts: |a >= t| and |b >= t| (both = 0) or |(a >= t) and (b >= t)| (both = 1)
void launch_count_partial(const float* a, const float* b, size_t n, float t, int both, double* pa, double* pb,
                          int nblocks, cudaStream_t st);
void launch_final_sum(const double* partials, int nblocks, double scale, double* out,
                      cudaStream_t st);
void launch_final_max(const double* partials, int nblocks, double* out, cudaStream_t st);
void launch_final_minmax(const double* pmin, const double* pmax, int nblocks, double* out2,
                         cudaStream_t st);

// y = a x + y
void launch_axpy(float a, const float* x, float* y, size_t n, cudaStream_t st);
// z = x + a y
void launch_xpay(const float* x, float a, const float* y, float* z, size_t n, cudaStream_t st);
// x += alpha p; r -= alpha q; partial sums of r . r
void launch_pcg_update(float alpha, const float* p, const float* q, float* x, float* r, size_t n,
                       double* partials, int nblocks, cudaStream_t st);
void launch_fill(float* x, float value, size_t n, cudaStream_t st);

}  // namespace claire
