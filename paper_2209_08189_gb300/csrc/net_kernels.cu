// Kernels of the learned warm start: a 3D U-Net over periodic volumes with
// BF16 activations and weights and FP32 accumulation, for sm_103a.
//
// Layout: activations channels-last [B][D][H][W][C] (C contiguous, a
// tensor may be a channel slice of a wider buffer: channel stride Cs >= C);
// 3x3x3 conv weights [Cout][27][Cin] with tap = kd*9 + kh*3 + kw, offsets
// (kd-1, kh-1, kw-1); padding is periodic, like the registration domain.
//
// The 3x3x3 convolution is an implicit GEMM on the tensor cores
// (mma.sync m16n8k16 BF16 -> FP32): rows = output voxels, columns = output
// channels, reduction over (tap, input channel).  A CTA owns a brick of 64
// output voxels; per 16-channel slice of the input it stages the brick's halo
// in shared memory (cp.async, XOR-swizzled 16-byte halves so that ldmatrix
// rows hit distinct banks), then each warp runs 27 taps of m16 x (8 NT) x k16
// products, with the weights read through the read-only cache.
// Backward-data is the same kernel on flipped, transposed weights; the
// weight gradient is a second implicit GEMM (rows = output channels, columns
// = input channels, reduction over voxels) with per-chunk FP32 partials
// reduced in a fixed order, so results are deterministic.
#include "claire_net.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <algorithm>
#include <mutex>

namespace claire {
namespace net {

namespace {

constexpr int kBrick = 64;       // output voxels per CTA
constexpr int kHaloMax = 324;    // (BD+2)(BH+2)(BW+2) for the allowed bricks
constexpr int kConvThreads = 128;

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

// L1-allocating variant, for sources read more than once by the same CTA
__device__ __forceinline__ void cp_async16_ca(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_all;\n" ::);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// byte offset of 16-byte half h of row s in a [rows][16 x bf16] swizzled tile
__device__ __forceinline__ uint32_t swz(int s, int h) { return static_cast<uint32_t>((2 * s + (h ^ ((s >> 2) & 1))) * 16); }

// 8 channels per thread (16 bytes) helpers
struct V8 {
    float f[8];
};

__device__ __forceinline__ V8 load8(const __nv_bfloat16* p)
{
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
    V8 r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h[q]);
        r.f[2 * q] = f.x;
        r.f[2 * q + 1] = f.y;
    }
    return r;
}

__device__ __forceinline__ void store8(__nv_bfloat16* p, const V8& r)
{
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(r.f[2 * q], r.f[2 * q + 1]);
    *reinterpret_cast<uint4*>(p) = u;
}

struct Vol {
    int B, D, H, W;
};

struct Brick {
    int bd, bh, bw;  // brick extent (bd * bh * bw = 64)
    int nd, nh, nw;  // bricks per axis
};

// decode CTA index into the brick origin
__device__ __forceinline__ void brick_origin(const Vol& v, const Brick& k, int cta, int& b, int& d0, int& h0,
                                             int& w0)
{
    int r = cta;
    const int iw = r % k.nw; r /= k.nw;
    const int ih = r % k.nh; r /= k.nh;
    const int id = r % k.nd; r /= k.nd;
    b = r;
    d0 = id * k.bd;
    h0 = ih * k.bh;
    w0 = iw * k.bw;
}

// stage 16 channels (c0..c0+15) of the halo of a brick into swizzled smem
__device__ __forceinline__ void stage_halo(const __nv_bfloat16* __restrict__ X, int Cs, int c0, const Vol& v,
                                           const Brick& k, int b, int d0, int h0, int w0, uint32_t sbase)
{
    const int hw = k.bw + 2, hh = k.bh + 2;
    const int nslots = (k.bd + 2) * hh * hw;
    for (int e = threadIdx.x; e < 2 * nslots; e += blockDim.x) {
        const int s = e >> 1, half = e & 1;
        const int sw = s % hw, sh = (s / hw) % hh, sd = s / (hw * hh);
        const int d = wrapi(d0 + sd - 1, v.D), h = wrapi(h0 + sh - 1, v.H), w = wrapi(w0 + sw - 1, v.W);
        const size_t vox = ((static_cast<size_t>(b) * v.D + d) * v.H + h) * v.W + w;
        cp_async16(sbase + swz(s, half), X + vox * Cs + c0 + 8 * half);
    }
}

// Y[p][co] = act(bias[co] + sum_{tap,ci} X[p + off(tap)][ci] W[co][tap][ci])
template <int NT>
__global__ void __launch_bounds__(kConvThreads) k_conv3d(const __nv_bfloat16* __restrict__ X, int Cxs, int Cin,
                                                         const __nv_bfloat16* __restrict__ Wt,
                                                         const float* __restrict__ bias, float slope, int act,
                                                         __nv_bfloat16* __restrict__ Y, int Cys, Vol v, Brick k)
{
    __shared__ __align__(128) unsigned char halo[kHaloMax * 32];
    int b, d0, h0, w0;
    brick_origin(v, k, blockIdx.x, b, d0, h0, w0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hw = k.bw + 2, hh = k.bh + 2;
    // this lane's ldmatrix row: voxel r of the brick
    const int r = 16 * warp + (lane & 7) + 8 * ((lane >> 3) & 1);
    const int rw = r % k.bw, rh = (r / k.bw) % k.bh, rd = r / (k.bw * k.bh);
    const int slot0 = (rd * hh + rh) * hw + rw;  // halo slot of tap (0,0,0) offset (-1,-1,-1)
    const int khalf = lane >> 4;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t sbase = smem_addr(halo);

    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;

    for (int c0 = 0; c0 < Cin; c0 += 16) {
        __syncthreads();
        stage_halo(X, Cxs, c0, v, k, b, d0, h0, w0, sbase);
        cp_async_wait();
        __syncthreads();
        const __nv_bfloat16* wrow = Wt + static_cast<size_t>(g) * 27 * Cin + c0 + 2 * t;
#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
            const int kd = tap / 9, kh = (tap / 3) % 3, kw = tap % 3;
            const int s = slot0 + (kd * hh + kh) * hw + kw;
            uint32_t a0, a1, a2, a3;
            ldsm_x4(sbase + swz(s, khalf), a0, a1, a2, a3);
            const __nv_bfloat16* wp = wrow + static_cast<size_t>(tap) * Cin;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const __nv_bfloat16* q = wp + static_cast<size_t>(n) * 8 * 27 * Cin;
                const uint32_t b0 = __ldg(reinterpret_cast<const unsigned int*>(q));
                const uint32_t b1 = __ldg(reinterpret_cast<const unsigned int*>(q + 8));
                mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // epilogue: rows g and g + 8 of this warp's 16 voxels
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int rr = 16 * warp + g + 8 * half;
        const int ew = rr % k.bw, eh = (rr / k.bw) % k.bh, ed = rr / (k.bw * k.bh);
        const size_t vox = ((static_cast<size_t>(b) * v.D + d0 + ed) * v.H + h0 + eh) * v.W + w0 + ew;
        __nv_bfloat16* yrow = Y + vox * Cys;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int co = 8 * n + 2 * t;
            float y0 = acc[n][2 * half], y1 = acc[n][2 * half + 1];
            if (bias) {
                y0 += __ldg(bias + co);
                y1 += __ldg(bias + co + 1);
            }
            if (act) {
                y0 = y0 > 0.f ? y0 : slope * y0;
                y1 = y1 > 0.f ? y1 : slope * y1;
            }
            *reinterpret_cast<__nv_bfloat162*>(yrow + co) = __floats2bfloat162_rn(y0, y1);
        }
    }
}

// ---------------------------------------------------------------------------
// tcgen05 (5th-generation tensor core) version of the forward convolution
// ---------------------------------------------------------------------------
// A CTA owns a brick of BDc x 16 x 8 output voxels: BDc planes of M = 128
// voxels (one TMEM lane per voxel of a plane) and all Cout channels (N =
// Cout FP32 columns per plane).  Per 16-channel slice of the input it stages,
// with cp.async, the brick's halo ((BDc+2) x 18 x 10 voxels) and the slice of
// all 27 taps' weights into shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix, two 8-channel half
// planes), then one elected thread issues 27 x BDc tcgen05.mma.kind::f16
// (M128 x N x K16): the A operand of a (plane, tap) pair is the halo at a
// shifted start address, because every core matrix is 8 consecutive voxels
// along W and the next one is the next H row (a constant stride).  The halo
// is shared by the BDc planes; with two stages the next slice is staged while
// the tensor cores work on the current one.  tcgen05.commit signals an
// mbarrier (waits are bounded); the epilogue reads TMEM with tcgen05.ld.
constexpr int kTcBH = 16, kTcBW = 8;
constexpr int kTcHaloH = kTcBH + 2, kTcHaloW = kTcBW + 2;
constexpr int kTcPlaneSlots = kTcHaloH * kTcHaloW;  // 180 halo voxels per D plane
constexpr uint32_t kTcSpinLimit = 1u << 22;  // default polls of a bounded mbarrier wait
constexpr int kTcMaxSmem = 231424;  // dynamic shared memory per CTA: the 227 KB opt-in limit less 1 KB for the static part

// CTAs of the tcgen05 kernels whose bounded mbarrier wait gave up (read by
// claire_net_device_errors)
__device__ int g_tc_wait_errors = 0;
// CTAs that gave up and whose MMAs did not drain either: they return without
// tcgen05.dealloc (their columns may still be written); never seen in practice
__device__ int g_tc_tmem_kept = 0;
// polls of one bounded wait, and the failure-detection hook: when set, every
// CTA first waits on a completion phase that nothing signals, before any MMA
// is issued (set through claire_net_set_wait_test)
__device__ uint32_t g_tc_spin_limit = kTcSpinLimit;
__device__ int g_tc_test_stall = 0;

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // start >> 4 [0,14), leading byte offset >> 4 [16,30), stride byte
    // offset >> 4 [32,46), descriptor version 1 [46,48), no swizzle
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    const uint32_t limit = g_tc_spin_limit;
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// After a give-up: thread `issuer` (the one that issued every MMA of the CTA)
// commits to the fresh mbarrier `drain`, which then completes once all of its
// earlier tcgen05 operations have; the block agrees on whether they did.  Only
// then may the CTA release its TMEM columns.  Called by every thread.
__device__ __forceinline__ bool tc_drain(uint32_t drain, bool issuer)
{
    bool ok = true;
    if (issuer) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain)
                     : "memory");
        ok = mbar_wait(drain, 0);
    }
    return __syncthreads_and(ok) != 0;
}

// TMEM release at the end of a CTA: dealloc when the MMAs are known complete
// (`release`), else count the columns kept.  Called by every thread.
__device__ __forceinline__ void tc_release(uint32_t tmem, uint32_t cols, bool release)
{
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (!release) {
        if (threadIdx.x == 0) atomicAdd(&g_tc_tmem_kept, 1);
        return;
    }
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// 16 consecutive TMEM columns of this warp's 32 lanes (32x32b shape)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&q)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]), "=r"(q[8]),
          "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

struct TcShape {
    int bdc;        // D planes per brick
    int ccols;      // TMEM columns per plane (Cout rounded up to 32)
    int nstage;     // 1 or 2 staging buffers
    int plane;      // bytes of one 8-channel half plane of the halo
    int stage;      // bytes of one stage (halo + weights)
    uint32_t cols;  // TMEM columns allocated (power of two)
};

__global__ void __launch_bounds__(kConvThreads) k_conv3d_tc(const __nv_bfloat16* __restrict__ X, int Cxs, int Cin,
                                                            const __nv_bfloat16* __restrict__ Wt,
                                                            const float* __restrict__ bias, float slope, int act,
                                                            __nv_bfloat16* __restrict__ Y, int Cys, int Cout,
                                                            TcShape sh, Vol v, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar, drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int stall;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bdc = sh.bdc;
    // brick origin
    const int nbw = v.W / kTcBW, nbh = v.H / kTcBH, nbd = v.D / bdc;
    int r = blockIdx.x;
    const int w0 = (r % nbw) * kTcBW; r /= nbw;
    const int h0 = (r % nbh) * kTcBH; r /= nbh;
    const int d0 = (r % nbd) * bdc;
    const int b = r / nbd;
    const int slots = (bdc + 2) * kTcPlaneSlots;
    const uint32_t smem_s = smem_addr(tc_smem), mbar_s = smem_addr(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(sh.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const uint32_t drain_s = smem_addr(&drain);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_s), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(drain_s), "r"(1));
        stall = g_tc_test_stall;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    // failure-detection hook: a wait on phase 0 of mbar, which only the first
    // commit would complete, before any MMA is issued (it runs out)
    bool ok = true;
    if (stall) ok = __syncthreads_and(mbar_wait(mbar_s, 0)) != 0;
    const bool stalled = !ok;  // gave up before any MMA was issued
    // instruction descriptor: D F32, A and B BF16, both K-major, N = Cout, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((static_cast<uint32_t>(Cout) >> 3) << 17) |
                           ((128u >> 4) << 24);
    const int nchunks = Cin / 16;
    // stage a slice: halo slot s = (sd * 18 + sh) * 10 + sw in half plane h; weight piece (tap, half, co)
    auto issue = [&](int c, int stg) {
        const int c0 = 16 * c;
        const uint32_t base = smem_s + stg * sh.stage;
        for (int e = tid; e < 2 * slots; e += kConvThreads) {
            const int hlf = e / slots, sl = e - hlf * slots;
            const int sw = sl % kTcHaloW, shh = (sl / kTcHaloW) % kTcHaloH, sd = sl / kTcPlaneSlots;
            const int d = wrapi(d0 + sd - 1, v.D), h = wrapi(h0 + shh - 1, v.H), w = wrapi(w0 + sw - 1, v.W);
            const size_t vox = ((static_cast<size_t>(b) * v.D + d) * v.H + h) * v.W + w;
            cp_async16(base + hlf * sh.plane + sl * 16, X + vox * Cxs + c0 + 8 * hlf);
        }
        const uint32_t wb = base + 2 * sh.plane;
        const int npieces = 27 * 2 * Cout;
        for (int e = tid; e < npieces; e += kConvThreads) {
            const int co = e % Cout, hlf = (e / Cout) & 1, tap = e / (2 * Cout);
            cp_async16(wb + e * 16, Wt + (static_cast<size_t>(co) * 27 + tap) * Cin + c0 + 8 * hlf);
        }
        cp_async_commit();
    };
    if (ok) issue(0, 0);
    for (int c = 0; c < nchunks && ok; ++c) {
        const int stg = sh.nstage == 2 ? (c & 1) : 0;
        // every completion phase is waited for exactly once and in order, so
        // a parity wait never sees two outstanding phases; the block agrees on
        // the outcome, so every thread takes the same barriers
        if (c >= 1) ok = __syncthreads_and(mbar_wait(mbar_s, (c - 1) & 1)) != 0;
        if (!ok) break;
        if (sh.nstage == 2) {
            if (c + 1 < nchunks) {
                issue(c + 1, (c + 1) & 1);  // the stage slice c-1 used; overlaps the MMAs of slice c
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
        } else {
            if (c >= 1) issue(c, 0);
            cp_async_wait_group<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t base = smem_s + stg * sh.stage;
            const uint32_t wb = base + 2 * sh.plane;
#pragma unroll 1
            for (int z = 0; z < bdc; ++z)
#pragma unroll 1
                for (int tap = 0; tap < 27; ++tap) {
                    const int kd = tap / 9, kh = (tap / 3) % 3, kw = tap % 3;
                    const uint32_t a_addr = base + (((z + kd) * kTcHaloH + kh) * kTcHaloW + kw) * 16;
                    const uint64_t ad = umma_desc(a_addr, sh.plane, kTcHaloW * 16);
                    const uint64_t bd = umma_desc(wb + tap * 2 * Cout * 16, Cout * 16, 128);
                    const uint32_t accum = (c > 0 || tap > 0) ? 1u : 0u;
                    const uint32_t dt = tmem + static_cast<uint32_t>(z * sh.ccols);
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                 "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_s)
                         : "memory");
        }
    }
    if (ok) ok = __syncthreads_and(mbar_wait(mbar_s, (nchunks - 1) & 1)) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    bool release = true;
    if (!ok) {
        cp_async_wait_group<0>();
        if (tid == 0) atomicAdd(err, 1);
        // after the stall hook no MMA was issued: nothing to drain
        release = stalled ? true : tc_drain(drain_s, tid == 0);
    } else {
        // epilogue: warp w owns TMEM lanes 32w..32w+31 = rows m = 32w + lane of every plane
        const int m = 32 * warp + lane;
        const int eh = m / kTcBW, ew = m % kTcBW;
        for (int z = 0; z < bdc; ++z) {
            const size_t vox = ((static_cast<size_t>(b) * v.D + d0 + z) * v.H + h0 + eh) * v.W + w0 + ew;
            __nv_bfloat16* yrow = Y + vox * Cys;
            for (int c0 = 0; c0 < Cout; c0 += 16) {
                uint32_t q[16];
                const uint32_t ta = tmem + (static_cast<uint32_t>(32 * warp) << 16) +
                                    static_cast<uint32_t>(z * sh.ccols + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
                      "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]),
                      "=r"(q[14]), "=r"(q[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                V8 o0, o1;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float y0 = __uint_as_float(q[j]), y1 = __uint_as_float(q[8 + j]);
                    if (bias) {
                        y0 += __ldg(bias + c0 + j);
                        y1 += __ldg(bias + c0 + 8 + j);
                    }
                    if (act) {
                        y0 = y0 > 0.f ? y0 : slope * y0;
                        y1 = y1 > 0.f ? y1 : slope * y1;
                    }
                    o0.f[j] = y0;
                    o1.f[j] = y1;
                }
                store8(yrow + c0, o0);
                store8(yrow + c0 + 8, o1);
            }
        }
    }
    tc_release(tmem, sh.cols, release);
}

// tcgen05 weight gradient.  Per tap, dW[co][tap][ci] = sum_p dY[p][co] X[p + off(tap)][ci]:
// K = voxels (16 per MMA, two rows of a 1 x 16 x 8 brick), M = output
// channels, N = input channels x taps.  Both operands are MN-major (channels
// contiguous, as the activations are stored) in 8 x 16-byte core matrices.
//
// Rows.  With at most 32 output channels (nsa = 3) the A tile stacks the dY
// brick at depths d0-1, d0, d0+1 as row blocks s = 0, 1, 2: summed over all
// bricks, dY[p + (s-1) e_d] X[p + (0, kh-1, kw-1)] is the kd = 2 - s tap, so
// one MMA covers the three kd taps and X is staged for depth d0 only.
// Otherwise (nsa = 1) the rows are a block of up to 128 output channels and X
// is staged at three depths, kd picking the plane.
// Columns.  The X halo is staged so that one MMA covers three kh taps (nkw =
// 1: rows (sd, sh, q) of ten 16-byte voxel slots, the kh taps and the nq
// channel blocks being core matrices 160 bytes apart, kw a 16-byte start
// offset) or all nine (kh, kw) taps (nkw = 3, for 16-channel blocks: each
// (sd, sh) row holds the three kw-shifted copies of its eight brick voxels).
// An MMA "unit" is one (kd, kw) choice left to the start addresses; a CTA
// holds `units` of them in TMEM.
// Warp roles.  Warps 2..7 form nstage loader groups; group g stages bricks
// g, g + nstage, ... into smem stage g with cp.async and announces each on
// the stage's "full" mbarrier; lane 0 of warp 0 issues the MMAs of a full
// stage and frees it through tcgen05.commit on its "empty" mbarrier; warp 1
// sums dY for the bias from the same stage and also arrives on "empty".
// Each stage is used by every nstage-th brick, so every wait is for the
// newest phase of its barrier.  Per-chunk FP32 partials are reduced in a
// fixed order afterwards.
constexpr int kWgThreads = 256;
constexpr int kWgLoaders = 192;  // warps 2..7

struct TcWg {
    int nsa;        // dY row blocks (3: kd from the rows, 1: plain)
    int npl;        // X depth planes staged (1 when nsa == 3, else 3)
    int nkw;        // 3: kw taps in N (nc = 16), 1: kw by start offset
    int mpad;       // TMEM lanes used (64 or 128)
    int nc;         // input channels per CTA
    int nci, nco;   // input / output channel blocks
    int nunits;     // MMA units over all taps
    int units;      // MMA units per CTA
    int ntg;        // tap groups (CTAs sharing a brick's taps)
    int abytes;     // bytes of the dY tile (128 voxels x mpad rows x 2)
    int hbytes;     // bytes of the X halo
    int per_sm;     // CTAs resident per SM (TMEM)
    int nstage;     // smem stages (2 or 3)
    uint32_t cols;  // TMEM columns allocated
};

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__global__ void __launch_bounds__(kWgThreads) k_wgrad_tc(const __nv_bfloat16* __restrict__ X, int Cxs, int Cin,
                                                         const __nv_bfloat16* __restrict__ dY, int Cys, int Cout,
                                                         Vol v, TcWg wg, int nbricks, int per, int chunks,
                                                         float* __restrict__ P, float* __restrict__ Pb,
                                                         int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char wg_smem[];
    __shared__ __align__(8) uint64_t full[3], empty[3], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed, stall;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int bid = blockIdx.x;
    const int pc = bid % chunks; bid /= chunks;
    const int cib = bid % wg.nci; bid /= wg.nci;
    const int cob = bid % wg.nco;
    const int tg = bid / wg.nco;
    const int co0 = cob * 128, ci0 = cib * wg.nc;
    const int cnt = min(wg.nsa == 3 ? Cout : wg.mpad, Cout - co0);  // output channels of this block
    const int u0 = tg * wg.units, nun = min(wg.units, wg.nunits - u0);
    const int nkwu = 3 / wg.nkw;  // kw choices left to start addresses
    const int nq = wg.nc / 8, cbn = cnt / 8;
    const int albo = wg.mpad / 8 * 128;  // bytes per 8-voxel block of the dY tile
    const int N = 3 * wg.nkw * wg.nc;
    const bool bias = Pb != nullptr && tg == 0 && cib == 0;
    const int S = wg.nstage;
    const int stage_bytes = wg.abytes + wg.hbytes;
    const uint32_t s0 = smem_addr(wg_smem);
    const int first = pc * per, nbr = max(0, min(nbricks, first + per) - first);
    // padded rows of every dY tile stay zero
    for (int e = tid; e < S * stage_bytes / 16; e += kWgThreads) {
        const int st = e / (stage_bytes / 16), o = e - st * (stage_bytes / 16);
        if (o < wg.abytes / 16) reinterpret_cast<uint4*>(wg_smem + st * stage_bytes)[o] = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(wg.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[i])), "r"(kWgLoaders / S));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[i])), "r"(bias ? 2 : 1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&drain)), "r"(1));
        failed = 0;
        stall = g_tc_test_stall;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    // failure-detection hook: a wait on phase 0 of drain, which nothing
    // signals yet, before any load or MMA (it runs out; no role loop runs)
    const bool stalled = stall && !__syncthreads_and(mbar_wait(smem_addr(&drain), 0));
    const int smid = wg.nsa == 3 ? 1 : 0;
    // bias warp: lane -> (8-channel block cb, voxel residue r of nres)
    const int nres = 32 / max(cbn, 1);
    const int b_cb = lane % max(cbn, 1), b_r = lane / max(cbn, 1);
    float bacc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) bacc[i] = 0.f;
    bool ok = !stalled;
    if (stalled) {
        // no role runs
    } else if (warp >= 2) {
        // ---- loaders: group g of kWgLoaders / S threads owns stage g and
        // stages bricks g, g + S, g + 2S, ... (S independent load chains) ----
        const int nl = kWgLoaders / S;
        const int grp = (tid - 64) / nl, lt = (tid - 64) - grp * nl;
        // a row's pieces are spread over the group's threads (several rows
        // per pass when a row has fewer pieces than the group has threads)
        const int tja = 8 * cbn;  // dY: pieces per brick row
        const int rppa = tja <= nl ? nl / tja : 1, stepa = tja <= nl ? tja : nl;
        const int ja_r = tja <= nl ? lt / tja : 0, ja0 = tja <= nl ? lt - ja_r * tja : lt;
        const int tjx = kTcHaloW * nq;  // X: pieces per halo row
        const int rppx = tjx <= nl ? nl / tjx : 1, stepx = tjx <= nl ? tjx : nl;
        const int jx_r = tjx <= nl ? lt / tjx : 0, jx0 = tjx <= nl ? lt - jx_r * tjx : lt;
        const size_t row_y = static_cast<size_t>(v.W) * Cys, row_x = static_cast<size_t>(v.W) * Cxs;
        const int nbw = v.W / kTcBW, nbh = v.H / kTcBH;
        const uint32_t a_s = s0 + grp * stage_bytes, h_s = a_s + wg.abytes;
        for (int j = grp; j < nbr; j += S) {
            if (j >= S) {
                // the MMAs (and bias sums) of brick j - S are done with this stage
                bool w = true;
                if (lane == 0) w = mbar_wait(smem_addr(&empty[grp]), ((j / S) - 1) & 1);
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    ok = false;
                    break;
                }
            }
            // depth fastest: consecutive bricks of a chunk are depth neighbours, so
            // the dY (and X) planes d0 - 1 .. d0 + 1 that a brick shares with the
            // next one are still in L2 when it stages them
            int r = first + j;
            const int d0 = r % v.D; r /= v.D;
            const int w0 = (r % nbw) * kTcBW; r /= nbw;
            const int h0 = (r % nbh) * kTcBH;
            const int b = r / nbh;
            // dY rows (s, hr): 8 voxels x cbn pieces -> hr * albo + (s * cbn + cb) * 128 + voxel * 16
            if (ja_r < rppa) {
                for (int rr = ja_r; rr < 16 * wg.nsa; rr += rppa) {
                    const int sb = rr >> 4, hr = rr & 15;
                    const int d = wg.nsa == 3 ? wrapi(d0 + sb - 1, v.D) : d0;
                    const __nv_bfloat16* rowp = dY + ((static_cast<size_t>(b) * v.D + d) * v.H + h0 + hr) * row_y +
                                                static_cast<size_t>(w0) * Cys + co0;
                    for (int jj = ja0; jj < tja; jj += stepa) {
                        const int vox = jj / cbn, cb = jj - vox * cbn;
                        cp_async16(a_s + hr * albo + (sb * cbn + cb) * 128 + vox * 16,
                                   rowp + static_cast<size_t>(vox) * Cys + 8 * cb);
                    }
                }
            }
            // X halo rows (sd, sh): 10 voxel slots x nq pieces
            if (jx_r < rppx) {
                for (int rr = jx_r; rr < kTcHaloH * wg.npl; rr += rppx) {
                    const int sd = rr / kTcHaloH, sh = rr - sd * kTcHaloH;
                    const int d = wg.npl == 3 ? wrapi(d0 + sd - 1, v.D) : d0;
                    const int h = wrapi(h0 + sh - 1, v.H);
                    const __nv_bfloat16* rowp =
                        X + ((static_cast<size_t>(b) * v.D + d) * v.H + h) * row_x + ci0;
                    for (int jj = jx0; jj < tjx; jj += stepx) {
                        const int x_sw = jj / nq, x_q = jj - x_sw * nq;
                        const __nv_bfloat16* src =
                            rowp + static_cast<size_t>(wrapi(w0 + x_sw - 1, v.W)) * Cxs + 8 * x_q;
                        if (wg.nkw == 1) {
                            cp_async16(h_s + (rr * nq + x_q) * 160 + x_sw * 16, src);
                        } else {
#pragma unroll
                            for (int kw = 0; kw < 3; ++kw) {
                                const int ww = x_sw - kw;
                                if (ww >= 0 && ww < 8)
                                    cp_async16_ca(h_s + ((rr * 3 + kw) * nq + x_q) * 128 + ww * 16, src);
                            }
                        }
                    }
                }
            }
            // this thread's part of brick j has landed: make it visible to the
            // tensor cores and announce it
            cp_async_wait();
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(smem_addr(&full[grp]));
        }
        cp_async_wait();
    } else if (warp == 0) {
        // ---- MMA issue ----
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                   ((static_cast<uint32_t>(N) >> 3) << 17) |
                                   ((static_cast<uint32_t>(wg.mpad) >> 4) << 24);
            for (int j = 0; j < nbr; ++j) {
                const int sidx = j % S;
                if (!mbar_wait(smem_addr(&full[sidx]), (j / S) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a_s = s0 + sidx * stage_bytes, h_s = a_s + wg.abytes;
#pragma unroll 1
                for (int ks = 0; ks < 8; ++ks) {
                    const uint64_t ad = umma_desc(a_s + 2 * ks * albo, albo, 128);
                    const uint32_t accum = (j > 0 || ks > 0) ? 1u : 0u;
#pragma unroll 1
                    for (int jj = 0; jj < nun; ++jj) {
                        const int u = u0 + jj, kd = u / nkwu, kw = u - kd * nkwu;
                        const int sd = wg.npl == 3 ? kd : 0;
                        uint64_t bd;
                        if (wg.nkw == 1)
                            bd = umma_desc(h_s + (sd * kTcHaloH + 2 * ks) * nq * 160 + kw * 16, nq * 160, 160);
                        else
                            bd = umma_desc(h_s + (sd * kTcHaloH + 2 * ks) * 3 * nq * 128, 3 * nq * 128, 128);
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                         tmem + static_cast<uint32_t>(N * jj)),
                                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(&empty[sidx]))
                             : "memory");
            }
        }
    } else if (bias) {
        // ---- bias sums (warp 1) ----
        for (int j = 0; j < nbr; ++j) {
            const int sidx = j % S;
            bool w = true;
            if (lane == 0) w = mbar_wait(smem_addr(&full[sidx]), (j / S) & 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) {
                ok = false;
                break;
            }
            if (b_r < nres) {
                const unsigned char* At = wg_smem + sidx * stage_bytes + (smid * cbn + b_cb) * 128;
                for (int p = b_r; p < 128; p += nres) {
                    const uint4 q4 = *reinterpret_cast<const uint4*>(At + (p / 8) * albo + (p % 8) * 16);
                    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&q4);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 f = __bfloat1622float2(h2[i]);
                        bacc[2 * i] += f.x;
                        bacc[2 * i + 1] += f.y;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[sidx]));
        }
    }
    if (!ok) failed = 1;
    __syncthreads();
    // the last brick's stage is released once all MMAs (each commit covers
    // the earlier ones) and the bias sums are done
    bool okw = failed == 0;
    if (okw && nbr > 0 && tid == 0)
        okw = mbar_wait(smem_addr(&empty[(nbr - 1) % S]), ((nbr - 1) / S) & 1);
    ok = __syncthreads_and(okw);
    asm volatile("tcgen05.fence::after_thread_sync;");
    bool release = true;
    if (!ok) {
        if (tid == 0) atomicAdd(err, 1);
        // tid 0 issued every MMA; after the stall hook it issued none
        release = stalled ? true : tc_drain(smem_addr(&drain), tid == 0);
    } else if (nbr > 0) {
        // an M = 128 accumulator holds row m in lane m, an M = 64 one in lane
        // (m / 16) * 32 + m % 16; warps w and w + 4 share lane quadrant w % 4
        const int qd = warp & 3, half = warp >> 2;
        const int row = wg.mpad == 128 ? 32 * qd + lane : (lane < 16 ? 16 * qd + lane : wg.mpad);
        const bool valid = row < wg.nsa * cnt;
        const int sb = valid ? row / cnt : 0;
        const int co = co0 + (valid ? row - sb * cnt : 0);
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * qd) << 16);
        float* Pp = P + static_cast<size_t>(pc) * Cout * 27 * Cin;
        for (int j = 0; j < nun; ++j) {
            const int u = u0 + j, kdu = u / nkwu, kwu = u - kdu * nkwu;
            const int kd = wg.nsa == 3 ? 2 - sb : kdu;
            for (int c16 = half; c16 < N / 16; c16 += 2) {
                uint32_t q[16];
                tmem_ld16(lane_base + static_cast<uint32_t>(N * j + 16 * c16), q);
                const int n = 16 * c16;
                int kh, kw, ci;
                if (wg.nkw == 3) {
                    kh = n / (3 * wg.nc);
                    const int rem = n - kh * 3 * wg.nc;
                    kw = rem / wg.nc;
                    ci = rem - kw * wg.nc;
                } else {
                    kh = n / wg.nc;
                    kw = kwu;
                    ci = n - kh * wg.nc;
                }
                if (valid) {
                    float* dst = Pp + (static_cast<size_t>(co) * 27 + kd * 9 + kh * 3 + kw) * Cin + ci0 + ci;
#pragma unroll
                    for (int i = 0; i < 16; ++i) dst[i] = __uint_as_float(q[i]);
                }
            }
        }
        if (bias) {
            // fixed-order reduction of the bias warp's voxel residues (the stages are free now)
            float* red = reinterpret_cast<float*>(wg_smem);
            if (warp == 1 && b_r < nres)
#pragma unroll
                for (int i = 0; i < 8; ++i) red[b_r * cnt + b_cb * 8 + i] = bacc[i];
            __syncthreads();
            if (tid < cnt) {
                float t = 0.f;
                for (int j = 0; j < nres; ++j) t += red[j * cnt + tid];
                Pb[static_cast<size_t>(pc) * Cout + co0 + tid] = t;
            }
        }
    }
    tc_release(tmem, wg.cols, release);
}

// Wgrad partials: P[pc][co][tap][ci] = sum over the chunk's voxels p of
// dY[p][co] X[p + off(tap)][ci]; Pb[pc][co] = sum dY[p][co] (ci chunk 0 only).
// grid: (Cin/16, Cout/16, chunks); each CTA loops over its bricks.
__global__ void __launch_bounds__(kConvThreads) k_conv3d_wgrad(const __nv_bfloat16* __restrict__ X, int Cxs,
                                                               int Cin, const __nv_bfloat16* __restrict__ dY,
                                                               int Cys, int Cout, Vol v, Brick k, int nbricks,
                                                               int per_chunk, float* __restrict__ P,
                                                               float* __restrict__ Pb)
{
    __shared__ __align__(128) unsigned char halo[kHaloMax * 32];
    __shared__ __align__(128) unsigned char dys[kBrick * 32];
    const int ci0 = 16 * blockIdx.x, co0 = 16 * blockIdx.y, pc = blockIdx.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hw = k.bw + 2, hh = k.bh + 2;
    const uint32_t hbase = smem_addr(halo), dbase = smem_addr(dys);
    const int i = lane >> 3, j = lane & 7;
    const int g = lane >> 2, t = lane & 3;
    // taps of this warp: warp, warp + 4, ... (7 or 6 taps)
    float acc[7][2][4];
#pragma unroll
    for (int a = 0; a < 7; ++a)
#pragma unroll
        for (int n = 0; n < 2; ++n) acc[a][n][0] = acc[a][n][1] = acc[a][n][2] = acc[a][n][3] = 0.f;
    float bsum = 0.f;  // thread tid < 16: column co0 + tid

    const int first = pc * per_chunk;
    const int last = min(nbricks, first + per_chunk);
    for (int br = first; br < last; ++br) {
        int b, d0, h0, w0;
        brick_origin(v, k, br, b, d0, h0, w0);
        __syncthreads();
        stage_halo(X, Cxs, ci0, v, k, b, d0, h0, w0, hbase);
        for (int e = threadIdx.x; e < 2 * kBrick; e += blockDim.x) {
            const int p = e >> 1, half = e & 1;
            const int pw = p % k.bw, ph = (p / k.bw) % k.bh, pd = p / (k.bw * k.bh);
            const size_t vox = ((static_cast<size_t>(b) * v.D + d0 + pd) * v.H + h0 + ph) * v.W + w0 + pw;
            cp_async16(dbase + swz(p, half), dY + vox * Cys + co0 + 8 * half);
        }
        cp_async_wait();
        __syncthreads();
        if (blockIdx.x == 0 && threadIdx.x < 16) {
            const int h = threadIdx.x >> 3, c = threadIdx.x & 7;
            for (int p = 0; p < kBrick; ++p)
                bsum += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(dys + swz(p, h) + 2 * c));
        }
#pragma unroll 1
        for (int ks = 0; ks < 4; ++ks) {
            // A = dY^T (co x p): stored rows p, columns co
            uint32_t a0, a1, a2, a3;
            {
                const int p = 16 * ks + j + 8 * (i >> 1);
                ldsm_x4_t(dbase + swz(p, i & 1), a0, a1, a2, a3);
            }
            // B rows p (shifted by the tap), columns ci
            const int p = 16 * ks + j + 8 * (i & 1);
            const int pw = p % k.bw, ph = (p / k.bw) % k.bh, pd = p / (k.bw * k.bh);
            const int slot0 = (pd * hh + ph) * hw + pw;
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                const int tap = warp + 4 * a;
                if (tap < 27) {
                    const int kd = tap / 9, kh = (tap / 3) % 3, kw = tap % 3;
                    const int s = slot0 + (kd * hh + kh) * hw + kw;
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_t(hbase + swz(s, i >> 1), b0, b1, b2, b3);
                    mma_bf16(acc[a][0], a0, a1, a2, a3, b0, b1);
                    mma_bf16(acc[a][1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
    }
    // write partials
    float* Pp = P + static_cast<size_t>(pc) * Cout * 27 * Cin;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        const int tap = warp + 4 * a;
        if (tap >= 27) continue;
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int co = co0 + g + 8 * half;
                const int ci = ci0 + 8 * n + 2 * t;
                float* q = Pp + (static_cast<size_t>(co) * 27 + tap) * Cin + ci;
                q[0] = acc[a][n][2 * half];
                q[1] = acc[a][n][2 * half + 1];
            }
    }
    if (blockIdx.x == 0 && threadIdx.x < 16) {
        const int h = threadIdx.x >> 3, c = threadIdx.x & 7;
        Pb[static_cast<size_t>(pc) * Cout + co0 + 8 * h + c] = bsum;
    }
}

// out[e] = sum_{pc < n} P[pc * stride + e]  (fixed order)
__global__ void k_reduce_partials(const float* __restrict__ P, int nchunks, size_t stride,
                                  float* __restrict__ out)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (e >= stride) return;
    float s = 0.f;
    for (int pc = 0; pc < nchunks; ++pc) s += P[pc * stride + e];
    out[e] = s;
}

// W'[ci][tap][co] = W[co][26 - tap][ci]   (weights of the adjoint convolution)
__global__ void k_flip_weights(const __nv_bfloat16* __restrict__ W, int Cout, int Cin,
                               __nv_bfloat16* __restrict__ Wf)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    const size_t n = static_cast<size_t>(Cout) * 27 * Cin;
    if (e >= n) return;
    const int co = static_cast<int>(e % Cout);
    const int tap = static_cast<int>((e / Cout) % 27);
    const int ci = static_cast<int>(e / (static_cast<size_t>(Cout) * 27));
    Wf[e] = W[(static_cast<size_t>(co) * 27 + (26 - tap)) * Cin + ci];
}

// coarse voxel index and channel group of element e (groups of 8 channels)
__device__ __forceinline__ bool decode8(size_t e, int C, const Vol& v, size_t& vox, int& c)
{
    const int G = C / 8;
    const size_t nvox = static_cast<size_t>(v.B) * v.D * v.H * v.W;
    if (e >= nvox * G) return false;
    c = 8 * static_cast<int>(e % G);
    vox = e / G;
    return true;
}

__device__ __forceinline__ size_t fine_vox(const Vol& c, size_t vox, int a)
{
    // child a (bits d,h,w) of coarse voxel vox on the 2x finer grid
    const int w = static_cast<int>(vox % c.W);
    size_t r = vox / c.W;
    const int h = static_cast<int>(r % c.H);
    r /= c.H;
    const int d = static_cast<int>(r % c.D);
    const size_t b = r / c.D;
    const int fd = 2 * d + ((a >> 2) & 1), fh = 2 * h + ((a >> 1) & 1), fw = 2 * w + (a & 1);
    return ((b * (2 * c.D) + fd) * (2 * c.H) + fh) * (2 * c.W) + fw;
}

// Y (coarse) = mean of the 2x2x2 children of X (fine)
__global__ void k_pool2(const __nv_bfloat16* __restrict__ X, int Cxs, int C, __nv_bfloat16* __restrict__ Y,
                        int Cys, Vol coarse)
{
    size_t vox;
    int c;
    if (!decode8(blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x, C, coarse, vox, c)) return;
    V8 s = {};
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
        const V8 x = load8(X + fine_vox(coarse, vox, a) * Cxs + c);
#pragma unroll
        for (int q = 0; q < 8; ++q) s.f[q] += x.f[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s.f[q] *= 0.125f;
    store8(Y + vox * Cys + c, s);
}

// dX (fine) = dY (coarse) / 8 [+ add (fine)]
__global__ void k_pool2_bwd(const __nv_bfloat16* __restrict__ dY, int Cys, const __nv_bfloat16* __restrict__ add,
                            int Cas, int C, __nv_bfloat16* __restrict__ dX, int Cxs, Vol coarse)
{
    size_t vox;
    int c;
    if (!decode8(blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x, C, coarse, vox, c)) return;
    V8 d = load8(dY + vox * Cys + c);
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
        const size_t f = fine_vox(coarse, vox, a);
        V8 o;
        if (add) {
            const V8 x = load8(add + f * Cas + c);
#pragma unroll
            for (int q = 0; q < 8; ++q) o.f[q] = fmaf(0.125f, d.f[q], x.f[q]);
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) o.f[q] = 0.125f * d.f[q];
        }
        store8(dX + f * Cxs + c, o);
    }
}

// Y (fine) = X (coarse) repeated over the 2x2x2 children
__global__ void k_up2(const __nv_bfloat16* __restrict__ X, int Cxs, int C, __nv_bfloat16* __restrict__ Y, int Cys,
                      Vol coarse)
{
    size_t vox;
    int c;
    if (!decode8(blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x, C, coarse, vox, c)) return;
    const uint4 u = *reinterpret_cast<const uint4*>(X + vox * Cxs + c);
#pragma unroll 1
    for (int a = 0; a < 8; ++a) *reinterpret_cast<uint4*>(Y + fine_vox(coarse, vox, a) * Cys + c) = u;
}

// dX (coarse) = sum of dY over the 2x2x2 children (fine)
__global__ void k_up2_bwd(const __nv_bfloat16* __restrict__ dY, int Cys, int C, __nv_bfloat16* __restrict__ dX,
                          int Cxs, Vol coarse)
{
    size_t vox;
    int c;
    if (!decode8(blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x, C, coarse, vox, c)) return;
    V8 s = {};
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
        const V8 x = load8(dY + fine_vox(coarse, vox, a) * Cys + c);
#pragma unroll
        for (int q = 0; q < 8; ++q) s.f[q] += x.f[q];
    }
    store8(dX + vox * Cxs + c, s);
}

// dP = dY * (Y > 0 ? 1 : slope)   (leaky ReLU through its output)
__global__ void k_leaky_bwd(const __nv_bfloat16* __restrict__ dY, int Cds, const __nv_bfloat16* __restrict__ Y,
                            int Cys, int C, float slope, __nv_bfloat16* __restrict__ dP, int Cps, Vol v)
{
    size_t vox;
    int c;
    if (!decode8(blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x, C, v, vox, c)) return;
    V8 d = load8(dY + vox * Cds + c);
    const V8 y = load8(Y + vox * Cys + c);
#pragma unroll
    for (int q = 0; q < 8; ++q) d.f[q] = y.f[q] > 0.f ? d.f[q] : slope * d.f[q];
    store8(dP + vox * Cps + c, d);
}

// X[b][p][0..Cs) = (a0 * m0[b][p], a1 * m1[b][p], 0, ...)   (network input)
__global__ void k_pack_inputs(const float* __restrict__ m0, const float* __restrict__ m1, float a0, float a1,
                              size_t nvox, __nv_bfloat16* __restrict__ X, int Cs)
{
    const size_t p = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (p >= nvox) return;
    __nv_bfloat16* x = X + p * Cs;
    *reinterpret_cast<__nv_bfloat162*>(x) = __floats2bfloat162_rn(a0 * m0[p], a1 * m1[p]);
    for (int c = 2; c < Cs; c += 2) *reinterpret_cast<__nv_bfloat162*>(x + c) = __floats2bfloat162_rn(0.f, 0.f);
}

// Output head (1x1x1 conv to NOUT FP32 channels, channels-first per sample):
// V[b][c][p] = scale (bias[c] + sum_ci X[b,p][ci] Wh[c][ci]).  NOUT = 3: the
// velocity; NOUT = 4: the velocity and the logit of the coarse preconditioner
// weight.
template <int CIN, int NOUT>
__global__ void k_head(const __nv_bfloat16* __restrict__ X, int Cxs, const float* __restrict__ Wh,
                       const float* __restrict__ bh, float scale, size_t nvox_per, int B, float* __restrict__ V)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (e >= nvox_per * B) return;
    const size_t b = e / nvox_per, p = e % nvox_per;
    float s[NOUT];
#pragma unroll
    for (int c = 0; c < NOUT; ++c) s[c] = bh[c];
    const __nv_bfloat16* x = X + e * Cxs;
#pragma unroll
    for (int c = 0; c < CIN; c += 8) {
        const V8 xv = load8(x + c);
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int o = 0; o < NOUT; ++o) s[o] = fmaf(xv.f[q], __ldg(Wh + o * CIN + c + q), s[o]);
    }
    float* vb = V + b * NOUT * nvox_per + p;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) vb[o * nvox_per] = scale * s[o];
}

// head backward: dX[b,p][ci] = scale sum_c dV[b][c][p] Wh[c][ci]; per-block
// partials of dWh[c][ci] = scale sum_p dV X and dbh[c] = scale sum_p dV,
// layout [block][NOUT CIN + NOUT].
template <int CIN, int NOUT>
__global__ void __launch_bounds__(256) k_head_bwd(const __nv_bfloat16* __restrict__ X, int Cxs,
                                                  const float* __restrict__ Wh, float scale, size_t nvox_per,
                                                  int B, const float* __restrict__ dV,
                                                  __nv_bfloat16* __restrict__ dX, int Cdxs,
                                                  float* __restrict__ part)
{
    constexpr int NR = NOUT * CIN + NOUT;
    __shared__ float red[8][NR];
    float loc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) loc[q] = 0.f;
    const size_t n = nvox_per * B;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const size_t b = e / nvox_per, p = e % nvox_per;
        const float* db = dV + b * NOUT * nvox_per + p;
        float g[NOUT];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) g[o] = scale * db[o * nvox_per];
#pragma unroll
        for (int c = 0; c < CIN; c += 8) {
            const V8 xv = load8(X + e * Cxs + c);
            V8 ov;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float t = 0.f;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    t += g[o] * __ldg(Wh + o * CIN + c + q);
                    loc[o * CIN + c + q] += g[o] * xv.f[q];
                }
                ov.f[q] = t;
            }
            if (dX) store8(dX + e * Cdxs + c, ov);
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) loc[NOUT * CIN + o] += g[o];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        float v = loc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NR; q += blockDim.x) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += red[w][q];
        part[static_cast<size_t>(blockIdx.x) * NR + q] = v;
    }
}

// Adam (bias-corrected) on FP32 master weights; optional BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ s, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2, float gscale, __nv_bfloat16* __restrict__ wb)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (e >= n) return;
    const float g = gscale * gr[e];
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float ss = b2 * s[e] + (1.f - b2) * g * g;
    m[e] = mm;
    s[e] = ss;
    const float wn = w[e] - lr * (mm * c1) / (sqrtf(ss * c2) + eps);
    w[e] = wn;
    if (wb) wb[e] = __float2bfloat16_rn(wn);
}

// dv = a (v - vs) + b gv (gv may be null); *sum += sum (v - vs)^2
__global__ void __launch_bounds__(256) k_vel_loss(const float* __restrict__ v, const float* __restrict__ vs,
                                                  const float* __restrict__ gv, float a, float b, size_t n,
                                                  float* __restrict__ dv, double* __restrict__ sum)
{
    double loc = 0.0;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float d = v[e] - vs[e];
        loc += static_cast<double>(d) * d;
        dv[e] = gv ? fmaf(a, d, b * gv[e]) : a * d;
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        if (sum) atomicAdd(sum, s);
    }
}

// r = x - y; *sum += sum r^2
// (r may alias x: each element is read and written by one thread)
__global__ void __launch_bounds__(256) k_residual(const float* x, const float* __restrict__ y, size_t n, float* r,
                                                  double* __restrict__ sum)
{
    double loc = 0.0;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float d = x[e] - y[e];
        loc += static_cast<double>(d) * d;
        if (r) r[e] = d;
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        if (sum) atomicAdd(sum, s);
    }
}

// ---- coarse preconditioner correction: fit statistics, training loss, weight ----

// Least-squares statistics of the model D ~ gbar w (gbar . p) for the data
// term D = hp - sp of a Gauss-Newton matvec on the probe p (vector fields
// [3][n]): num += a (gbar . D), den += a^2 |gbar|^2, a = gbar . p.
__global__ void __launch_bounds__(256) k_pcw_stats(const float* __restrict__ gbar, const float* __restrict__ p,
                                                   const float* __restrict__ hp, const float* __restrict__ sp,
                                                   size_t n, float* __restrict__ num, float* __restrict__ den)
{
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        float a = 0.f, dd = 0.f, g2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float gc = gbar[c * n + e];
            a = fmaf(gc, p[c * n + e], a);
            dd = fmaf(gc, hp[c * n + e] - sp[c * n + e], dd);
            g2 = fmaf(gc, gc, g2);
        }
        num[e] = fmaf(a, dd, num[e]);
        den[e] = fmaf(a * a, g2, den[e]);
    }
}

// *tot += sum x (FP64)
__global__ void __launch_bounds__(256) k_sum_f64(const float* __restrict__ x, size_t n, double* __restrict__ tot)
{
    double loc = 0.0;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x)
        loc += x[e];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(tot, s);
    }
}

__device__ __forceinline__ float softplus_f(float o) { return o > 20.f ? o : log1pf(expf(o)); }

// Loss of the weight w = softplus(o) against the statistics pooled over the
// 2 x 2 x 2 cell of each voxel (A = sum den, B = sum num of the cell):
// L = sum_x (A w^2 - 2 B w + B^2 / A) / (8 T), T = *tot (sum of den), whose
// minimiser is w = B / A in every cell with A > 0; dout = scale dL/do.
// *loss += L.  Grid n1 x n2 x n3, all even.
__global__ void __launch_bounds__(256) k_pcw_loss(const float* __restrict__ o, const float* __restrict__ num,
                                                  const float* __restrict__ den, int n1, int n2, int n3,
                                                  const double* __restrict__ tot, float scale,
                                                  float* __restrict__ dout, double* __restrict__ loss)
{
    const size_t n = static_cast<size_t>(n1) * n2 * n3;
    const double T = *tot;
    const float inv = T > 0.0 ? static_cast<float>(1.0 / (8.0 * T)) : 0.f;
    double loc = 0.0;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(e % n3), j = static_cast<int>((e / n3) % n2),
                  i = static_cast<int>(e / (static_cast<size_t>(n2) * n3));
        const size_t c0 = (static_cast<size_t>(i & ~1) * n2 + (j & ~1)) * n3 + (k & ~1);
        float A = 0.f, B = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const size_t q = c0 + (static_cast<size_t>(a) * n2 + b) * n3 + c;
                    A += den[q];
                    B += num[q];
                }
        const float ov = o[e];
        const float w = softplus_f(ov);
        const float sig = 1.f / (1.f + expf(-ov));
        dout[e] = scale * 2.f * inv * (A * w - B) * sig;
        if (A > 0.f) loc += (static_cast<double>(A) * w * w - 2.0 * B * w + static_cast<double>(B) * B / A) * inv;
    }
    __shared__ double red[8];
    for (int s = 16; s > 0; s >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(loss, s);
    }
}

// w = softplus(o)
__global__ void k_pcw_weight(const float* __restrict__ o, float* __restrict__ w, size_t n)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (e < n) w[e] = softplus_f(o[e]);
}

inline unsigned nblk(size_t n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

}  // namespace

bool brick_for(int D, int H, int W, int* bd, int* bh, int* bw)
{
    const int w = W >= 16 ? 16 : W;
    const int h = H >= kBrick / w ? kBrick / w : H;
    const int d = kBrick / (w * h);
    if (w < 4 || w * h * d != kBrick || d > D || D % d || H % h || W % w) return false;
    *bd = d;
    *bh = h;
    *bw = w;
    return (d + 2) * (h + 2) * (w + 2) <= kHaloMax;
}

// tiling forced by claire_net_set_conv_tiling (0 = automatic)
int g_tc_force_bdc = 0, g_tc_force_nstage = 0;

// The tcgen05 kernels need more than 48 KB of dynamic shared memory; the
// attribute that allows it is per device, so it is set once on each device
// (done[] indexed by device, under a lock).
constexpr int kMaxDevices = 64;
std::mutex g_attr_mutex;

cudaError_t smem_attr_once(const void* kernel, bool (&done)[kMaxDevices])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem);
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (!done[dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem);
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

bool tc_eligible(int Cin, int Cout, int D, int H, int W)
{
    (void)D;
    return H % kTcBH == 0 && W % kTcBW == 0 && Cin % 16 == 0 && Cout % 16 == 0 && Cout >= 16 && Cout <= 192;
}

cudaError_t conv3d(const void* X, int Cxs, int Cin, const void* Wt, const float* bias, float slope, int act,
                   void* Y, int Cys, int Cout, int B, int D, int H, int W, cudaStream_t st)
{
    const Vol v{B, D, H, W};
    auto x = static_cast<const __nv_bfloat16*>(X);
    auto w = static_cast<const __nv_bfloat16*>(Wt);
    auto y = static_cast<__nv_bfloat16*>(Y);
    if (tc_eligible(Cin, Cout, D, H, W)) {
        // tcgen05 path: bricks of bdc x 16 x 8 voxels; the deepest brick whose
        // TMEM columns (bdc planes x Cout rounded to 32) and shared memory fit
        TcShape sh{};
        sh.ccols = (Cout + 31) / 32 * 32;
        const int wbytes = 27 * 2 * Cout * 16;
        int nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 152;
        // choose the brick depth and staging: the deepest brick (halo shared
        // by more planes, weights staged once for more voxels) that still
        // leaves two waves of CTAs at the occupancy that its shared memory and
        // TMEM allow; one stage unless a forced setting asks for two
        for (int bdc = 4; bdc >= 1; bdc >>= 1) {
            if (D % bdc || bdc * sh.ccols > 512) continue;
            if (g_tc_force_bdc && bdc != g_tc_force_bdc) continue;
            const int plane = (bdc + 2) * kTcPlaneSlots * 16;
            const int stage = 2 * plane + wbytes;
            const int nstage = g_tc_force_nstage ? g_tc_force_nstage : 1;
            if (nstage * stage > kTcMaxSmem) continue;
            uint32_t cols = 32;
            while (cols < static_cast<uint32_t>(bdc * sh.ccols)) cols <<= 1;
            const int per_sm = std::max(1, std::min(kTcMaxSmem / (nstage * stage), static_cast<int>(512 / cols)));
            const long long grid = static_cast<long long>(B) * (D / bdc) * (H / kTcBH) * (W / kTcBW);
            if (!g_tc_force_bdc && bdc > 1 && grid < 2LL * nsm * per_sm) continue;
            sh.bdc = bdc;
            sh.plane = plane;
            sh.stage = stage;
            sh.nstage = nstage;
            break;
        }
        if (sh.bdc == 0) return cudaErrorInvalidValue;
        sh.cols = 32;
        while (sh.cols < static_cast<uint32_t>(sh.bdc * sh.ccols)) sh.cols <<= 1;
        const size_t smem = static_cast<size_t>(sh.nstage) * sh.stage;
        static bool attr_done[kMaxDevices] = {};
        cudaError_t ea = smem_attr_once(reinterpret_cast<const void*>(k_conv3d_tc), attr_done);
        if (ea != cudaSuccess) return ea;
        int* err = nullptr;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_tc_wait_errors);
        if (e != cudaSuccess) return e;
        const unsigned grid = static_cast<unsigned>(B * (D / sh.bdc) * (H / kTcBH) * (W / kTcBW));
        k_conv3d_tc<<<grid, kConvThreads, smem, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, Cout, sh, v, err);
        return cudaGetLastError();
    }
    int bd, bh, bw;
    if (!brick_for(D, H, W, &bd, &bh, &bw)) return cudaErrorInvalidValue;
    const Brick k{bd, bh, bw, D / bd, H / bh, W / bw};
    const unsigned grid = static_cast<unsigned>(B * k.nd * k.nh * k.nw);
    switch (Cout / 8) {
    case 2: k_conv3d<2><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    case 4: k_conv3d<4><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    case 6: k_conv3d<6><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    case 8: k_conv3d<8><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    case 12: k_conv3d<12><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    case 16: k_conv3d<16><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    case 24: k_conv3d<24><<<grid, kConvThreads, 0, st>>>(x, Cxs, Cin, w, bias, slope, act, y, Cys, v, k); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int read_tc_errors(bool reset)
{
    int n = 0;
    if (cudaMemcpyFromSymbol(&n, g_tc_wait_errors, sizeof(int)) != cudaSuccess) return -1;
    if (reset) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_tc_wait_errors, &z, sizeof(int)) != cudaSuccess) return -1;
    }
    return n;
}

cudaError_t flip_weights(const void* W, int Cout, int Cin, void* Wf, cudaStream_t st)
{
    const size_t n = static_cast<size_t>(Cout) * 27 * Cin;
    k_flip_weights<<<nblk(n, 256), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(W), Cout, Cin,
                                                 static_cast<__nv_bfloat16*>(Wf));
    return cudaGetLastError();
}

// input-channel block of the tcgen05 weight gradient forced by
// claire_net_set_wgrad_tiling (0 = automatic)
int g_wg_force_nc = 0;

bool wg_tc_config(int Cin, int Cout, int nc, TcWg* wg)
{
    if (Cin % nc) return false;
    TcWg g{};
    g.nsa = 3 * Cout <= 128 ? 3 : 1;
    g.npl = g.nsa == 3 ? 1 : 3;
    g.mpad = g.nsa == 3 ? (3 * Cout <= 64 ? 64 : 128) : (Cout <= 64 ? 64 : 128);
    g.nco = g.nsa == 3 ? 1 : (Cout + 127) / 128;
    g.nc = nc;
    g.nci = Cin / nc;
    g.nkw = nc == 16 ? 3 : 1;
    const int N = 3 * g.nkw * nc;
    g.nunits = (g.nsa == 3 ? 1 : 3) * (3 / g.nkw);
    g.units = std::min(g.nunits, 512 / N);
    if (g.units < 1) return false;
    g.ntg = (g.nunits + g.units - 1) / g.units;
    g.abytes = 128 * g.mpad * 2;
    g.hbytes = g.nkw == 3 ? g.npl * kTcHaloH * 3 * (nc / 8) * 128 : g.npl * kTcHaloH * (nc / 8) * 160;
    g.cols = 32;
    while (g.cols < static_cast<uint32_t>(N * g.units)) g.cols <<= 1;
    const int stage = g.abytes + g.hbytes;
    if (g.cols > 512 || 2 * stage > kTcMaxSmem) return false;
    // two CTAs per SM where TMEM and shared memory allow (each with as many
    // stages, up to three, as half the SM holds), else one with up to three
    if (g.cols <= 256 && 2 * (2 * stage + 2048) <= 233472) {
        g.per_sm = 2;
        g.nstage = 2 * (3 * stage + 2048) <= 233472 ? 3 : 2;
    } else {
        g.per_sm = 1;
        g.nstage = 3 * stage <= kTcMaxSmem ? 3 : 2;
    }
    *wg = g;
    return true;
}

bool wg_tc_shape(int Cin, int Cout, int B, int D, int H, int W, int nsm, TcWg* wg, int* nbricks, int* chunks)
{
    if (H % kTcBH || W % kTcBW || Cin % 16 || Cout % 16) return false;
    TcWg g{};
    if (g_wg_force_nc) {
        if (!wg_tc_config(Cin, Cout, g_wg_force_nc, &g)) return false;
    } else {
        // stacked kd rows: the widest channel block that divides Cin (fewest
        // passes over each brick); otherwise 16 channels with all nine
        // (kh, kw) taps in one MMA
        bool found = false;
        if (3 * Cout <= 128)
            for (int nc : {48, 32, 16})
                if (!found && wg_tc_config(Cin, Cout, nc, &g)) found = true;
        if (!found && !wg_tc_config(Cin, Cout, 16, &g)) return false;
    }
    const int nb = B * D * (H / kTcBH) * (W / kTcBW);
    // one wave of resident CTAs
    const int ctas = g.ntg * g.nco * g.nci;
    int c = std::max(1, nsm * g.per_sm / ctas);
    c = std::min(c, nb);
    const int per = (nb + c - 1) / c;
    *wg = g;
    *nbricks = nb;
    *chunks = (nb + per - 1) / per;
    return true;
}

int wgrad_chunks(int Cin, int Cout, int B, int D, int H, int W, int nsm)
{
    TcWg g;
    int nb, ch;
    if (wg_tc_shape(Cin, Cout, B, D, H, W, nsm, &g, &nb, &ch)) return ch;
    int bd, bh, bw;
    if (!brick_for(D, H, W, &bd, &bh, &bw)) return 0;
    const int nbricks = B * (D / bd) * (H / bh) * (W / bw);
    const int pairs = (Cin / 16) * (Cout / 16);
    int chunks = (8 * nsm + pairs - 1) / pairs;
    if (chunks > nbricks) chunks = nbricks;
    if (chunks < 1) chunks = 1;
    const int per = (nbricks + chunks - 1) / chunks;
    return (nbricks + per - 1) / per;
}

cudaError_t conv3d_wgrad(const void* X, int Cxs, int Cin, const void* dY, int Cys, int Cout, int B, int D, int H,
                         int W, int chunks, float* part, float* partb, float* dW, float* db, cudaStream_t st)
{
    {
        int nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 152;
        TcWg g;
        int nb, ch;
        if (wg_tc_shape(Cin, Cout, B, D, H, W, nsm, &g, &nb, &ch)) {
            if (ch != chunks) return cudaErrorInvalidValue;
            static bool attr_done[kMaxDevices] = {};
            cudaError_t ea = smem_attr_once(reinterpret_cast<const void*>(k_wgrad_tc), attr_done);
            if (ea != cudaSuccess) return ea;
            int* err = nullptr;
            cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_tc_wait_errors);
            if (e != cudaSuccess) return e;
            const int per = (nb + chunks - 1) / chunks;
            const Vol v{B, D, H, W};
            // enough shared memory that no more CTAs than TMEM holds share an SM
            // (a surplus one would wait in tcgen05.alloc)
            const size_t need = static_cast<size_t>(g.nstage) * (g.abytes + g.hbytes);
            const size_t floor_smem = static_cast<size_t>(233472 / (g.per_sm + 1) - 1024);
            const size_t smem = std::min(std::max(need, floor_smem), static_cast<size_t>(kTcMaxSmem));
            const unsigned grid = static_cast<unsigned>(g.ntg * g.nco * g.nci * chunks);
            k_wgrad_tc<<<grid, kWgThreads, smem, st>>>(static_cast<const __nv_bfloat16*>(X), Cxs, Cin,
                                                        static_cast<const __nv_bfloat16*>(dY), Cys, Cout, v, g, nb,
                                                        per, chunks, part, db ? partb : nullptr, err);
            const size_t nw = static_cast<size_t>(Cout) * 27 * Cin;
            k_reduce_partials<<<nblk(nw, 256), 256, 0, st>>>(part, chunks, nw, dW);
            if (db) k_reduce_partials<<<nblk(Cout, 256), 256, 0, st>>>(partb, chunks, Cout, db);
            return cudaGetLastError();
        }
    }
    int bd, bh, bw;
    if (!brick_for(D, H, W, &bd, &bh, &bw)) return cudaErrorInvalidValue;
    const Vol v{B, D, H, W};
    const Brick k{bd, bh, bw, D / bd, H / bh, W / bw};
    const int nbricks = B * k.nd * k.nh * k.nw;
    const int per = (nbricks + chunks - 1) / chunks;
    if ((nbricks + per - 1) / per != chunks) return cudaErrorInvalidValue;
    const dim3 grid(Cin / 16, Cout / 16, chunks);
    k_conv3d_wgrad<<<grid, kConvThreads, 0, st>>>(static_cast<const __nv_bfloat16*>(X), Cxs, Cin,
                                                  static_cast<const __nv_bfloat16*>(dY), Cys, Cout, v, k,
                                                  nbricks, per, part, partb);
    const size_t nw = static_cast<size_t>(Cout) * 27 * Cin;
    k_reduce_partials<<<nblk(nw, 256), 256, 0, st>>>(part, chunks, nw, dW);
    if (db) k_reduce_partials<<<nblk(Cout, 256), 256, 0, st>>>(partb, chunks, Cout, db);
    return cudaGetLastError();
}

cudaError_t pool2(const void* X, int Cxs, int C, void* Y, int Cys, int B, int Dc, int Hc, int Wc, cudaStream_t st)
{
    const Vol c{B, Dc, Hc, Wc};
    const size_t n = static_cast<size_t>(B) * Dc * Hc * Wc * (C / 8);
    k_pool2<<<nblk(n, 256), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), Cxs, C,
                                          static_cast<__nv_bfloat16*>(Y), Cys, c);
    return cudaGetLastError();
}

cudaError_t pool2_bwd(const void* dY, int Cys, const void* add, int Cas, int C, void* dX, int Cxs, int B, int Dc,
                      int Hc, int Wc, cudaStream_t st)
{
    const Vol c{B, Dc, Hc, Wc};
    const size_t n = static_cast<size_t>(B) * Dc * Hc * Wc * (C / 8);
    k_pool2_bwd<<<nblk(n, 256), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(dY), Cys,
                                              static_cast<const __nv_bfloat16*>(add), Cas, C,
                                              static_cast<__nv_bfloat16*>(dX), Cxs, c);
    return cudaGetLastError();
}

cudaError_t up2(const void* X, int Cxs, int C, void* Y, int Cys, int B, int Dc, int Hc, int Wc, cudaStream_t st)
{
    const Vol c{B, Dc, Hc, Wc};
    const size_t n = static_cast<size_t>(B) * Dc * Hc * Wc * (C / 8);
    k_up2<<<nblk(n, 256), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), Cxs, C,
                                        static_cast<__nv_bfloat16*>(Y), Cys, c);
    return cudaGetLastError();
}

cudaError_t up2_bwd(const void* dY, int Cys, int C, void* dX, int Cxs, int B, int Dc, int Hc, int Wc,
                    cudaStream_t st)
{
    const Vol c{B, Dc, Hc, Wc};
    const size_t n = static_cast<size_t>(B) * Dc * Hc * Wc * (C / 8);
    k_up2_bwd<<<nblk(n, 256), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(dY), Cys, C,
                                            static_cast<__nv_bfloat16*>(dX), Cxs, c);
    return cudaGetLastError();
}

cudaError_t leaky_bwd(const void* dY, int Cds, const void* Y, int Cys, int C, float slope, void* dP, int Cps, int B,
                      int D, int H, int W, cudaStream_t st)
{
    const Vol v{B, D, H, W};
    const size_t n = static_cast<size_t>(B) * D * H * W * (C / 8);
    k_leaky_bwd<<<nblk(n, 256), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(dY), Cds,
                                              static_cast<const __nv_bfloat16*>(Y), Cys, C, slope,
                                              static_cast<__nv_bfloat16*>(dP), Cps, v);
    return cudaGetLastError();
}

cudaError_t pack_inputs(const float* m0, const float* m1, float a0, float a1, size_t nvox, void* X, int Cs,
                        cudaStream_t st)
{
    k_pack_inputs<<<nblk(nvox, 256), 256, 0, st>>>(m0, m1, a0, a1, nvox, static_cast<__nv_bfloat16*>(X), Cs);
    return cudaGetLastError();
}

cudaError_t head(const void* X, int Cxs, int Cin, int Nout, const float* Wh, const float* bh, float scale,
                 size_t nvox_per, int B, float* V, cudaStream_t st)
{
    auto x = static_cast<const __nv_bfloat16*>(X);
    const unsigned g = nblk(nvox_per * B, 256);
    if (Cin == 16 && Nout == 3)
        k_head<16, 3><<<g, 256, 0, st>>>(x, Cxs, Wh, bh, scale, nvox_per, B, V);
    else if (Cin == 32 && Nout == 3)
        k_head<32, 3><<<g, 256, 0, st>>>(x, Cxs, Wh, bh, scale, nvox_per, B, V);
    else if (Cin == 16 && Nout == 4)
        k_head<16, 4><<<g, 256, 0, st>>>(x, Cxs, Wh, bh, scale, nvox_per, B, V);
    else if (Cin == 32 && Nout == 4)
        k_head<32, 4><<<g, 256, 0, st>>>(x, Cxs, Wh, bh, scale, nvox_per, B, V);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int head_bwd_blocks(size_t nvox, int nsm)
{
    const size_t want = (nvox + 255) / 256;
    const size_t cap = static_cast<size_t>(2 * nsm);
    return static_cast<int>(want < cap ? (want ? want : 1) : cap);
}

cudaError_t head_bwd(const void* X, int Cxs, int Cin, int Nout, const float* Wh, float scale, size_t nvox_per,
                     int B, const float* dV, void* dX, int Cdxs, int nblocks, float* part, float* dWb,
                     cudaStream_t st)
{
    auto x = static_cast<const __nv_bfloat16*>(X);
    auto dx = static_cast<__nv_bfloat16*>(dX);
    if (Cin == 16 && Nout == 3)
        k_head_bwd<16, 3><<<nblocks, 256, 0, st>>>(x, Cxs, Wh, scale, nvox_per, B, dV, dx, Cdxs, part);
    else if (Cin == 32 && Nout == 3)
        k_head_bwd<32, 3><<<nblocks, 256, 0, st>>>(x, Cxs, Wh, scale, nvox_per, B, dV, dx, Cdxs, part);
    else if (Cin == 16 && Nout == 4)
        k_head_bwd<16, 4><<<nblocks, 256, 0, st>>>(x, Cxs, Wh, scale, nvox_per, B, dV, dx, Cdxs, part);
    else if (Cin == 32 && Nout == 4)
        k_head_bwd<32, 4><<<nblocks, 256, 0, st>>>(x, Cxs, Wh, scale, nvox_per, B, dV, dx, Cdxs, part);
    else
        return cudaErrorInvalidValue;
    const size_t nred = static_cast<size_t>(Nout * Cin + Nout);
    k_reduce_partials<<<nblk(nred, 256), 256, 0, st>>>(part, nblocks, nred, dWb);
    return cudaGetLastError();
}

cudaError_t adam(float* w, const float* g, float* m, float* s, size_t n, float lr, float b1, float b2, float eps,
                 int step, float gscale, void* wb, cudaStream_t st)
{
    const float c1 = 1.0f / (1.0f - powf(b1, static_cast<float>(step)));
    const float c2 = 1.0f / (1.0f - powf(b2, static_cast<float>(step)));
    k_adam<<<nblk(n, 256), 256, 0, st>>>(w, g, m, s, n, lr, b1, b2, eps, c1, c2, gscale,
                                         static_cast<__nv_bfloat16*>(wb));
    return cudaGetLastError();
}

cudaError_t vel_loss(const float* v, const float* vs, const float* gv, float a, float b, size_t n, float* dv,
                     double* sum, int nsm, cudaStream_t st)
{
    const unsigned g = static_cast<unsigned>(std::min<size_t>(nblk(n, 256), static_cast<size_t>(4 * nsm)));
    k_vel_loss<<<g ? g : 1, 256, 0, st>>>(v, vs, gv, a, b, n, dv, sum);
    return cudaGetLastError();
}

cudaError_t residual(const float* x, const float* y, size_t n, float* r, double* sum, int nsm, cudaStream_t st)
{
    const unsigned g = static_cast<unsigned>(std::min<size_t>(nblk(n, 256), static_cast<size_t>(4 * nsm)));
    k_residual<<<g ? g : 1, 256, 0, st>>>(x, y, n, r, sum);
    return cudaGetLastError();
}

cudaError_t pcw_stats(const float* gbar, const float* p, const float* hp, const float* sp, size_t n, float* num,
                      float* den, int nsm, cudaStream_t st)
{
    const unsigned g = static_cast<unsigned>(std::min<size_t>(nblk(n, 256), static_cast<size_t>(8 * nsm)));
    k_pcw_stats<<<g ? g : 1, 256, 0, st>>>(gbar, p, hp, sp, n, num, den);
    return cudaGetLastError();
}

cudaError_t pcw_loss(const float* o, const float* num, const float* den, const int grid[3], float scale,
                     float* dout, double* sums, int nsm, cudaStream_t st)
{
    const size_t n = static_cast<size_t>(grid[0]) * grid[1] * grid[2];
    const unsigned g = static_cast<unsigned>(std::min<size_t>(nblk(n, 256), static_cast<size_t>(8 * nsm)));
    k_sum_f64<<<g ? g : 1, 256, 0, st>>>(den, n, sums);
    k_pcw_loss<<<g ? g : 1, 256, 0, st>>>(o, num, den, grid[0], grid[1], grid[2], sums, scale, dout, sums + 1);
    return cudaGetLastError();
}

cudaError_t pcw_weight(const float* o, float* w, size_t n, cudaStream_t st)
{
    k_pcw_weight<<<nblk(n ? n : 1, 256), 256, 0, st>>>(o, w, n);
    return cudaGetLastError();
}

}  // namespace net
}  // namespace claire

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace claire {
namespace net {
namespace {

thread_local char g_net_err[256] = "";

claire_status net_fail(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_net_err, sizeof(g_net_err), fmt, ap);
    va_end(ap);
    return CLAIRE_EINVAL;
}

claire_status net_status(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return CLAIRE_OK;
    std::snprintf(g_net_err, sizeof(g_net_err), "%s: %s", what, cudaGetErrorString(e));
    return CLAIRE_ECUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool pow2_ge4(int n) { return n >= 4 && (n & (n - 1)) == 0; }

claire_status check_vol(const int vol[4])
{
    if (!vol) return net_fail("null vol");
    if (vol[0] < 1 || !pow2_ge4(vol[1]) || !pow2_ge4(vol[2]) || !pow2_ge4(vol[3]))
        return net_fail("vol {%d,%d,%d,%d}: B >= 1 and D, H, W powers of two >= 4 required", vol[0], vol[1],
                        vol[2], vol[3]);
    return CLAIRE_OK;
}

claire_status check_slice(const void* p, int stride, int c, const char* name)
{
    if (!p) return net_fail("%s: null pointer", name);
    if (!aligned16(p)) return net_fail("%s: pointer not 16-byte aligned", name);
    if (c < 8 || c % 8 || stride < c || stride % 8)
        return net_fail("%s: channels %d / stride %d must be multiples of 8 with stride >= channels", name, c,
                        stride);
    return CLAIRE_OK;
}

int device_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 152;
    return n > 0 ? n : 152;
}

#define NET_TRY(expr)                       \
    do {                                    \
        const claire_status s_ = (expr);    \
        if (s_ != CLAIRE_OK) return s_;     \
    } while (0)

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

}  // namespace net
}  // namespace claire

using namespace claire::net;

extern "C" claire_status claire_net_conv3d(const void* x, int x_stride, int cin, const void* w, const float* bias,
                                           float slope, int act, void* y, int y_stride, int cout, const int vol[4],
                                           void* stream)
{
    NET_TRY(check_vol(vol));
    NET_TRY(check_slice(x, x_stride, cin, "conv3d x"));
    NET_TRY(check_slice(y, y_stride, cout, "conv3d y"));
    if (!w || !aligned16(w)) return net_fail("conv3d: weights null or not 16-byte aligned");
    const int nt = cout / 8;
    const bool nt_ok = nt == 2 || nt == 4 || nt == 6 || nt == 8 || nt == 12 || nt == 16 || nt == 24;
    if (cin % 16 || cout % 8 || !nt_ok)
        return net_fail("conv3d: cin %d (multiple of 16), cout %d (16, 32, 48, 64, 96, 128 or 192)", cin, cout);
    int bd, bh, bw;
    if (!tc_eligible(cin, cout, vol[1], vol[2], vol[3]) && !brick_for(vol[1], vol[2], vol[3], &bd, &bh, &bw))
        return net_fail("conv3d: grid %dx%dx%d has fewer than 64 voxels", vol[1], vol[2], vol[3]);
    if (act != 0 && act != 1) return net_fail("conv3d: act %d", act);
    return net_status(conv3d(x, x_stride, cin, w, bias, slope, act, y, y_stride, cout, vol[0], vol[1], vol[2],
                             vol[3], as_stream(stream)),
                      "conv3d");
}

extern "C" claire_status claire_net_conv3d_flip(const void* w, int cout, int cin, void* wf, void* stream)
{
    if (!w || !wf || cin < 1 || cout < 1) return net_fail("conv3d_flip: bad arguments");
    return net_status(flip_weights(w, cout, cin, wf, as_stream(stream)), "conv3d_flip");
}

extern "C" claire_status claire_net_conv3d_wgrad_chunks(int cin, int cout, const int vol[4], int* chunks)
{
    NET_TRY(check_vol(vol));
    if (!chunks || cin % 16 || cout % 16 || cin < 16 || cout < 16)
        return net_fail("conv3d_wgrad_chunks: cin %d, cout %d must be multiples of 16", cin, cout);
    const int c = wgrad_chunks(cin, cout, vol[0], vol[1], vol[2], vol[3], device_sms());
    if (c < 1) return net_fail("conv3d_wgrad_chunks: grid has fewer than 64 voxels");
    *chunks = c;
    return CLAIRE_OK;
}

extern "C" claire_status claire_net_conv3d_wgrad(const void* x, int x_stride, int cin, const void* dy,
                                                 int dy_stride, int cout, const int vol[4], int chunks,
                                                 float* part, float* part_bias, float* dw, float* db, void* stream)
{
    NET_TRY(check_vol(vol));
    NET_TRY(check_slice(x, x_stride, cin, "conv3d_wgrad x"));
    NET_TRY(check_slice(dy, dy_stride, cout, "conv3d_wgrad dy"));
    if (cin % 16 || cout % 16) return net_fail("conv3d_wgrad: cin %d, cout %d must be multiples of 16", cin, cout);
    if (!part || !part_bias || !dw) return net_fail("conv3d_wgrad: null partial or output buffer");
    int expect = 0;
    NET_TRY(claire_net_conv3d_wgrad_chunks(cin, cout, vol, &expect));
    if (chunks != expect) return net_fail("conv3d_wgrad: chunks %d, expected %d", chunks, expect);
    return net_status(conv3d_wgrad(x, x_stride, cin, dy, dy_stride, cout, vol[0], vol[1], vol[2], vol[3], chunks,
                                   part, part_bias, dw, db, as_stream(stream)),
                      "conv3d_wgrad");
}

extern "C" claire_status claire_net_pool2(const void* x, int x_stride, int c, void* y, int y_stride,
                                          const int vol[4], void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("pool2: bad vol");
    NET_TRY(check_slice(x, x_stride, c, "pool2 x"));
    NET_TRY(check_slice(y, y_stride, c, "pool2 y"));
    return net_status(pool2(x, x_stride, c, y, y_stride, vol[0], vol[1], vol[2], vol[3], as_stream(stream)),
                      "pool2");
}

extern "C" claire_status claire_net_pool2_bwd(const void* dy, int dy_stride, const void* add, int add_stride,
                                              int c, void* dx, int dx_stride, const int vol[4], void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("pool2_bwd: bad vol");
    NET_TRY(check_slice(dy, dy_stride, c, "pool2_bwd dy"));
    NET_TRY(check_slice(dx, dx_stride, c, "pool2_bwd dx"));
    if (add) NET_TRY(check_slice(add, add_stride, c, "pool2_bwd add"));
    return net_status(pool2_bwd(dy, dy_stride, add, add_stride, c, dx, dx_stride, vol[0], vol[1], vol[2], vol[3],
                                as_stream(stream)),
                      "pool2_bwd");
}

extern "C" claire_status claire_net_up2(const void* x, int x_stride, int c, void* y, int y_stride, const int vol[4],
                                        void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("up2: bad vol");
    NET_TRY(check_slice(x, x_stride, c, "up2 x"));
    NET_TRY(check_slice(y, y_stride, c, "up2 y"));
    return net_status(up2(x, x_stride, c, y, y_stride, vol[0], vol[1], vol[2], vol[3], as_stream(stream)), "up2");
}

extern "C" claire_status claire_net_up2_bwd(const void* dy, int dy_stride, int c, void* dx, int dx_stride,
                                            const int vol[4], void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("up2_bwd: bad vol");
    NET_TRY(check_slice(dy, dy_stride, c, "up2_bwd dy"));
    NET_TRY(check_slice(dx, dx_stride, c, "up2_bwd dx"));
    return net_status(up2_bwd(dy, dy_stride, c, dx, dx_stride, vol[0], vol[1], vol[2], vol[3], as_stream(stream)),
                      "up2_bwd");
}

extern "C" claire_status claire_net_leaky_bwd(const void* dy, int dy_stride, const void* y, int y_stride, int c,
                                              float slope, void* dp, int dp_stride, const int vol[4], void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("leaky_bwd: bad vol");
    NET_TRY(check_slice(dy, dy_stride, c, "leaky_bwd dy"));
    NET_TRY(check_slice(y, y_stride, c, "leaky_bwd y"));
    NET_TRY(check_slice(dp, dp_stride, c, "leaky_bwd dp"));
    return net_status(leaky_bwd(dy, dy_stride, y, y_stride, c, slope, dp, dp_stride, vol[0], vol[1], vol[2], vol[3],
                                as_stream(stream)),
                      "leaky_bwd");
}

extern "C" claire_status claire_net_pack(const float* m0, const float* m1, float a0, float a1, size_t nvox, void* x,
                                         int stride, void* stream)
{
    if (!m0 || !m1 || !x || stride < 2 || stride % 2 || !aligned16(x)) return net_fail("pack: bad arguments");
    return net_status(pack_inputs(m0, m1, a0, a1, nvox, x, stride, as_stream(stream)), "pack");
}

extern "C" claire_status claire_net_head(const void* x, int x_stride, int cin, int nout, const float* wh,
                                         const float* bh, float scale, void* v, const int vol[4], void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("head: bad vol");
    NET_TRY(check_slice(x, x_stride, cin, "head x"));
    if (cin != 16 && cin != 32) return net_fail("head: cin %d (16 or 32)", cin);
    if (nout != 3 && nout != 4) return net_fail("head: nout %d (3 or 4)", nout);
    if (!wh || !bh || !v) return net_fail("head: null pointer");
    const size_t nvox = static_cast<size_t>(vol[1]) * vol[2] * vol[3];
    return net_status(head(x, x_stride, cin, nout, wh, bh, scale, nvox, vol[0], static_cast<float*>(v),
                           as_stream(stream)),
                      "head");
}

extern "C" claire_status claire_net_head_bwd_blocks(const int vol[4], int* blocks)
{
    if (!vol || !blocks || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1)
        return net_fail("head_bwd_blocks: bad arguments");
    *blocks = head_bwd_blocks(static_cast<size_t>(vol[0]) * vol[1] * vol[2] * vol[3], device_sms());
    return CLAIRE_OK;
}

extern "C" claire_status claire_net_head_bwd(const void* x, int x_stride, int cin, int nout, const float* wh,
                                             float scale, const float* dv, void* dx, int dx_stride,
                                             const int vol[4], int blocks, float* part, float* dwb, void* stream)
{
    if (!vol || vol[0] < 1 || vol[1] < 1 || vol[2] < 1 || vol[3] < 1) return net_fail("head_bwd: bad vol");
    NET_TRY(check_slice(x, x_stride, cin, "head_bwd x"));
    if (dx) NET_TRY(check_slice(dx, dx_stride, cin, "head_bwd dx"));
    if (cin != 16 && cin != 32) return net_fail("head_bwd: cin %d (16 or 32)", cin);
    if (nout != 3 && nout != 4) return net_fail("head_bwd: nout %d (3 or 4)", nout);
    int expect = 0;
    NET_TRY(claire_net_head_bwd_blocks(vol, &expect));
    if (blocks != expect) return net_fail("head_bwd: blocks %d, expected %d", blocks, expect);
    if (!wh || !dv || !part || !dwb) return net_fail("head_bwd: null pointer");
    const size_t nvox = static_cast<size_t>(vol[1]) * vol[2] * vol[3];
    return net_status(head_bwd(x, x_stride, cin, nout, wh, scale, nvox, vol[0], dv, dx, dx_stride, blocks, part,
                               dwb, as_stream(stream)),
                      "head_bwd");
}

extern "C" claire_status claire_net_adam(float* w, const float* g, float* m, float* s, size_t n, float lr,
                                         float beta1, float beta2, float eps, int step, float gscale, void* wb,
                                         void* stream)
{
    if (!w || !g || !m || !s || step < 1) return net_fail("adam: bad arguments");
    return net_status(adam(w, g, m, s, n, lr, beta1, beta2, eps, step, gscale, wb, as_stream(stream)), "adam");
}

extern "C" const char* claire_net_last_error(void) { return g_net_err; }

extern "C" claire_status claire_net_vel_loss(const float* v, const float* vstar, const float* gv, float a, float b,
                                             size_t n, float* dv, double* sum, void* stream)
{
    if (!v || !vstar || !dv) return net_fail("vel_loss: null pointer");
    return net_status(vel_loss(v, vstar, gv, a, b, n, dv, sum, device_sms(), as_stream(stream)), "vel_loss");
}

extern "C" claire_status claire_net_residual(const float* x, const float* y, size_t n, float* r, double* sum,
                                             void* stream)
{
    if (!x || !y) return net_fail("residual: null pointer");
    return net_status(residual(x, y, n, r, sum, device_sms(), as_stream(stream)), "residual");
}

extern "C" claire_status claire_net_pcw_stats(const float* gbar, const float* p, const float* hp, const float* sp,
                                              size_t n, float* num, float* den, void* stream)
{
    if (!gbar || !p || !hp || !sp || !num || !den) return net_fail("pcw_stats: null pointer");
    return net_status(pcw_stats(gbar, p, hp, sp, n, num, den, device_sms(), as_stream(stream)), "pcw_stats");
}

extern "C" claire_status claire_net_pcw_loss(const float* o, const float* num, const float* den, const int grid[3],
                                             float scale, float* dout, double* sums, void* stream)
{
    if (!o || !num || !den || !grid || !dout || !sums) return net_fail("pcw_loss: null pointer");
    if (grid[0] < 2 || grid[1] < 2 || grid[2] < 2 || (grid[0] | grid[1] | grid[2]) & 1)
        return net_fail("pcw_loss: grid %d x %d x %d (even extents >= 2)", grid[0], grid[1], grid[2]);
    return net_status(pcw_loss(o, num, den, grid, scale, dout, sums, device_sms(), as_stream(stream)), "pcw_loss");
}

extern "C" claire_status claire_net_pcw_weight(const float* o, float* w, size_t n, void* stream)
{
    if (!o || !w) return net_fail("pcw_weight: null pointer");
    return net_status(pcw_weight(o, w, n, as_stream(stream)), "pcw_weight");
}

extern "C" claire_status claire_net_device_errors(int* count, int reset)
{
    if (!count) return net_fail("device_errors: null pointer");
    const int n = read_tc_errors(reset != 0);
    if (n < 0) return net_status(cudaErrorUnknown, "device_errors");
    *count = n;
    return CLAIRE_OK;
}

extern "C" claire_status claire_net_set_wait_test(unsigned int spin_limit, int stall, int* tmem_kept)
{
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return net_status(e, "set_wait_test");
    const uint32_t lim = spin_limit ? spin_limit : kTcSpinLimit;
    const int st = stall ? 1 : 0;
    if ((e = cudaMemcpyToSymbol(g_tc_spin_limit, &lim, sizeof(lim))) != cudaSuccess ||
        (e = cudaMemcpyToSymbol(g_tc_test_stall, &st, sizeof(st))) != cudaSuccess)
        return net_status(e, "set_wait_test");
    if (tmem_kept && (e = cudaMemcpyFromSymbol(tmem_kept, g_tc_tmem_kept, sizeof(int))) != cudaSuccess)
        return net_status(e, "set_wait_test");
    return CLAIRE_OK;
}

extern "C" claire_status claire_net_set_wgrad_tiling(int nc)
{
    if (nc != 0 && nc != 16 && nc != 32 && nc != 48 && nc != 64)
        return net_fail("set_wgrad_tiling: nc %d not in {0, 16, 32, 48, 64}", nc);
    g_wg_force_nc = nc;
    return CLAIRE_OK;
}

extern "C" claire_status claire_net_set_conv_tiling(int bdc, int nstage)
{
    if ((bdc != 0 && bdc != 1 && bdc != 2 && bdc != 4) || nstage < 0 || nstage > 2)
        return net_fail("set_conv_tiling: bdc in {0, 1, 2, 4}, nstage in {0, 1, 2}");
    g_tc_force_bdc = bdc;
    g_tc_force_nstage = nstage;
    return CLAIRE_OK;
}
