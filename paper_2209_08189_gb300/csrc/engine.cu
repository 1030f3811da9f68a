// Host engine and C ABI of libclaire: context and workspaces, the
// semi-Lagrangian solves of the reduced-space Gauss-Newton-Krylov method
// ("CLAIRE at scale", arXiv 2209.08189, Sec. 2.2, Eqs. (1), (3)-(6)),
// matrix-free PCG and the Armijo line search.  Every numeric step runs in
// the kernels of sl_kernels.cu / vec_kernels.cu or in cuFFT on the
// context's stream; the host only sequences launches and reads FP64 scalars.
#include "claire.h"
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace claire;

namespace {

// Kernel classes tracked for the per-kernel statistics (CUDA-event timed
// when opts.timing is set; byte counts are algorithmic: each value once).
enum KernelKind {
    KK_INTERP = 0,   // state step / plain gather
    KK_BACKTRACE,
    KK_ADJ_STEP,
    KK_INC_STEP,
    KK_INC_LAST,
    KK_POINTWISE,    // adj_init, inc_init
    KK_FD8,
    KK_SPECTRAL,
    KK_FFT,          // cuFFT executions (library)
    KK_REDUCE,
    KK_VECTOR,
    KK_MAP,
    KK_DETJ,
    KK_VJP_GRAD,     // interpolant-gradient accumulation (reverse mode)
    KK_VJP_SCATTER,  // fixed-point scatter transpose (reverse mode)
    KK_COUNT
};

const char* kKernelNames[KK_COUNT] = {
    "sl_interp",  "sl_backtrace_rk2", "sl_adjoint_step", "sl_incremental_step",
    "sl_incremental_last", "sl_pointwise", "fd8", "spectral_scale", "cufft", "reduce_f64",
    "vector_update", "sl_map_step", "detj_minmax", "vjp_interp_grad", "vjp_scatter"};

struct KernelStat {
    double launches = 0, seconds = 0, bytes = 0, points = 0;
};

struct EventPair {
    cudaEvent_t a, b;
    int kind;
    int phase;
};

}  // namespace

// Coarse-grid state of the two-level zero-velocity preconditioner (allocated
// on first use): cuFFT plans of the coarse grid, the restricted mean state
// gradient gbar, the inner PCG vectors in Fourier space and, for the flexible
// outer PCG, the fine preconditioned residual.
struct TwoLevel {
    Grid g{};
    int factor = 0;
    size_t N = 0, M = 0;
    cufftHandle r2c = 0, c2r = 0;
    bool plans = false;
    void* work = nullptr;
    void* block = nullptr;
    float* gbar = nullptr;  // 3 Nc
    float* real = nullptr;  // 3 Nc scratch
    cufftComplex *xh = nullptr, *rh = nullptr, *zh = nullptr, *ph = nullptr, *cp = nullptr, *q = nullptr,
                 *T = nullptr;  // 3 Mc each
    cufftComplex* zf = nullptr;  // 3 M (fine): the stored preconditioned residual
    double* sc = nullptr;        // kTlSlots FP64 scalars of the inner PCG (device)
    ~TwoLevel()
    {
        if (plans) {
            cufftDestroy(r2c);
            cufftDestroy(c2r);
        }
        if (work) cudaFree(work);
        if (block) cudaFree(block);
    }
};

struct claire_ctx {
    Grid grid{};
    int n[3]{};
    size_t N = 0, M = 0;  // real points, complex modes per component
    int nt = 0;
    double dt = 0, beta_v = 0, hvol = 0;
    claire_opts o{};
    RegParams rp{};
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 0, red_blocks = 0;
    cufftHandle r2c = 0, c2r = 0;
    bool plans = false;
    void* fft_work = nullptr;             // one work area shared by both plans
    // cubic B-spline interpolation (interp = 4): coefficient scratch, its
    // spectra and single-field plans, allocated on first use
    float* bsc = nullptr;                 // 3N floats
    cufftComplex* bspec = nullptr;        // 3M modes
    cufftHandle r2c1 = 0, c2r1 = 0;
    bool bs_plans = false;
    size_t fft_work_bytes = 0;
    std::string err;

    // workspace arena
    void* arena = nullptr;
    size_t arena_bytes = 0;
    // scalar fields stored in the storage type `sto` (es bytes per value)
    Storage sto = Storage::F32;
    size_t es = 4;
    char *m0 = nullptr, *m1 = nullptr;
    float *v = nullptr;                   // linearisation point
    float *dS = nullptr, *dA = nullptr;   // state / adjoint characteristics
    // their tile-bounds tables, written by every backtrace into dS / dA (the
    // only writer of either field), read by the gathers at dS / dA
    int4 *tbS = nullptr, *tbA = nullptr;
    char *divv = nullptr, *divXp = nullptr;
    char *m = nullptr, *gm = nullptr;     // (nt+1) N states m^j, (nt+1) 3N gradients (null when lowmem)
    char *l0 = nullptr, *l1 = nullptr;    // rolling scalar fields (FP32-sized: transport uses them as FP32)
    char* tl = nullptr;                   // (nt+1) N: adjoint levels lambda^j / incremental sources f^j
    float *g = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr;
    cufftComplex* spec = nullptr;
    cufftComplex* phat = nullptr;         // PCG search direction in Fourier space
    cufftComplex* spec2 = nullptr;        // second transform buffer
    cufftComplex* xh = nullptr;           // PCG solution, Fourier space
    cufftComplex* rh = nullptr;           // PCG residual, Fourier space
    double* partials = nullptr;           // 2 * red_blocks
    double* dres = nullptr;               // device scalars
    double* hres = nullptr;               // pinned host scalars

    // reverse-mode transport scratch, allocated by the first claire_transport_vjp
    // spectrum of the Gauss-Newton iterate inside claire_register (spectral_iterate = 1):
    // S v is formed from it instead of from a transform of v, allocated by the first
    // claire_register (3M modes)
    cufftComplex* vh = nullptr;
    bool vh_on = false;
    float* vjp_states = nullptr;            // (nt+1) N, FP32 (2 N when checkpointing)
    size_t vjp_states_n = 0;
    unsigned long long* vjp_acc = nullptr;  // N fixed-point accumulators
    bool have_images = false, have_lin = false;
    double J_lin = 0, mis_lin = 0, reg_lin = 0;
    TwoLevel* tl2 = nullptr;         // two-level preconditioner state (precond = 1)
    // coarse preconditioner correction (claire_set_pc_weight): weight of the
    // zero-velocity data term on the coarse grid pcw_grid, Nc floats
    float* pcw = nullptr;
    size_t pcw_n = 0;
    int pcw_grid[3]{};
    bool pcw_on = false;
    long long pc_inner_total = 0;    // its inner PCG iterations so far

    // statistics and timing
    KernelStat ks[KK_COUNT];
    double phase_s[8]{};
    std::vector<EventPair> pending;
    std::vector<cudaEvent_t> pool;
    int cur_phase = -1;

    ~claire_ctx() { release(); }

    void release()
    {
        for (auto& e : pending) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
        pending.clear();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
        if (plans) {
            cufftDestroy(r2c);
            cufftDestroy(c2r);
            plans = false;
        }
        if (fft_work) cudaFree(fft_work);
        fft_work = nullptr;
        if (bs_plans) {
            cufftDestroy(r2c1);
            cufftDestroy(c2r1);
            bs_plans = false;
        }
        if (bsc) cudaFree(bsc);
        bsc = nullptr;
        if (bspec) cudaFree(bspec);
        bspec = nullptr;
        if (arena) cudaFree(arena);
        arena = nullptr;
        if (vjp_states) cudaFree(vjp_states);
        vjp_states = nullptr;
        if (vh) cudaFree(vh);
        vh = nullptr;
        if (vjp_acc) cudaFree(vjp_acc);
        vjp_acc = nullptr;
        if (pcw) cudaFree(pcw);
        pcw = nullptr;
        pcw_on = false;
        if (hres) cudaFreeHost(hres);
        hres = nullptr;
        delete tl2;
        tl2 = nullptr;
    }
};

namespace {

// Address of value `idx` of a storage-typed field.
inline char* at(const claire_ctx* c, char* base, size_t idx) { return base + idx * c->es; }

claire_status fail(claire_ctx* c, claire_status s, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CL_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? CLAIRE_ENOMEM : CLAIRE_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                    \
    } while (0)

#define CL_FFT(ctx, call)                                                                   \
    do {                                                                                    \
        cufftResult e_ = (call);                                                            \
        if (e_ != CUFFT_SUCCESS)                                                            \
            return fail((ctx), e_ == CUFFT_ALLOC_FAILED ? CLAIRE_ENOMEM : CLAIRE_ECUFFT,    \
                        "%s: cufft error %d (%s:%d)", #call, (int)e_, __FILE__, __LINE__); \
    } while (0)

#define CL_TRY(expr)                         \
    do {                                     \
        claire_status s_ = (expr);           \
        if (s_ < 0) return s_;               \
    } while (0)

#define CL_LAUNCHED(ctx) CL_CUDA(ctx, cudaGetLastError())

bool valid_grid(const int grid[3])
{
    if (!grid) return false;
    long long N = 1;
    for (int c = 0; c < 3; ++c) {
        if (grid[c] < 8 || (grid[c] & 1)) return false;
        N *= grid[c];
    }
    return N < (1LL << 31);
}

void fill_defaults(claire_opts* o)
{
    o->interp = CLAIRE_INTERP_CUBIC;
    o->reg = 1;
    o->beta_w = 1e-4;
    o->grad_form = 0;
    o->gtol = 5e-2;
    o->max_gn = 50;
    o->max_pcg = 50;
    o->pcg_rtol_max = 0.5;
    o->pcg_fixed = 0;
    o->armijo_c1 = 1e-4;
    o->max_ls = 10;
    o->wall_limit_s = 0.0;
    o->timing = 0;
    o->storage = CLAIRE_STORAGE_F32;
    o->g0_ref = 0.0;
    o->lowmem = 0;
    o->precond = CLAIRE_PRECOND_SPECTRAL;
    o->pc_coarse = 2;
    o->pc_tol = 1e-1;
    o->pc_maxit = 50;
    o->spectral_iterate = 1;
    o->kernels_only = 0;
}

bool valid_opts(const claire_opts& o)
{
    return (o.interp == 1 || o.interp == 3 || o.interp == 4) && (o.reg == 1 || o.reg == 2) && o.beta_w >= 0 &&
           (o.interp != 4 || o.storage == CLAIRE_STORAGE_F32) &&
           (o.grad_form == 0 || o.grad_form == 1) && o.gtol >= 0 && o.max_gn >= 0 &&
           o.max_pcg >= 1 && o.pcg_rtol_max > 0 && o.armijo_c1 > 0 && o.armijo_c1 < 1 &&
           o.max_ls >= 1 && o.wall_limit_s >= 0 && o.storage >= 0 && o.storage <= 2 &&
           o.g0_ref >= 0 && (o.lowmem == 0 || o.lowmem == 1) &&
           (o.precond == CLAIRE_PRECOND_SPECTRAL || o.precond == CLAIRE_PRECOND_TWO_LEVEL) && o.pc_coarse >= 1 &&
           o.pc_tol >= 0 && o.pc_maxit >= 1 && (o.spectral_iterate == 0 || o.spectral_iterate == 1) &&
           (o.kernels_only == 0 || o.kernels_only == 1);
}

// The two-level grid N_i / f must be whole, even and at least 4 per axis.
bool valid_coarse(const int n[3], int f)
{
    for (int i = 0; i < 3; ++i) {
        if (f < 1 || n[i] % f) return false;
        const int m = n[i] / f;
        if (m < 4 || (m & 1)) return false;
    }
    return true;
}

// Grid geometry of an n1 x n2 x n3 periodic grid on [0, 2 pi)^3.
Grid grid_of(int n1, int n2, int n3)
{
    const double two_pi = 6.283185307179586476925286766559;
    Grid g;
    g.n1 = n1;
    g.n2 = n2;
    g.n3 = n3;
    g.n23 = n2 * n3;
    g.N = static_cast<uint32_t>(static_cast<size_t>(n1) * n2 * n3);
    g.h1 = static_cast<float>(two_pi / n1);
    g.h2 = static_cast<float>(two_pi / n2);
    g.h3 = static_cast<float>(two_pi / n3);
    g.ih1 = static_cast<float>(n1 / two_pi);
    g.ih2 = static_cast<float>(n2 / two_pi);
    g.ih3 = static_cast<float>(n3 / two_pi);
    return g;
}

// Layout of the workspace arena in floats (each region 256-byte aligned).
struct Layout {
    size_t off[32];
    int count = 0;
    size_t total = 0;  // floats
    size_t add(size_t floats)
    {
        size_t o = total;
        off[count++] = o;
        total += (floats + 63) / 64 * 64;
        return o;
    }
};

size_t layout_floats(size_t N, size_t M, int nt, int red_blocks, size_t es, bool lowmem, Layout* L)
{
    Layout tmp;
    Layout& l = L ? *L : tmp;
    auto S = [&](size_t values) { return (values * es + 3) / 4; };  // storage-typed region, in floats
    l.add(S(N));                 // m0
    l.add(S(N));                 // m1
    l.add(3 * N);                // v
    l.add(3 * N);                // dS
    l.add(3 * N);                // dA
    l.add(S(N));                 // divv
    l.add(S(N));                 // divXp
    l.add(S((nt + 1) * N));      // m
    l.add(lowmem ? 0 : S(3 * (nt + 1) * N));  // gm (not stored in low-memory mode)
    l.add(N);                    // l0 (FP32-sized)
    l.add(N);                    // l1 (FP32-sized)
    l.add(S((nt + 1) * N));      // tl
    for (int i = 0; i < 5; ++i) l.add(3 * N);  // g x r z p
    l.add(6 * M);             // spec (3 complex half-spectra)
    l.add(6 * M);             // phat
    l.add(6 * M);             // spec2
    l.add(6 * M);             // xh
    l.add(6 * M);             // rh
    l.add(4 * red_blocks);    // partials (2 * red_blocks doubles)
    l.add(32);                // dres (16 doubles)
    l.add(8 * ((N + 1023) / 1024));  // tbS (2 int4 per 1024-point tile)
    l.add(8 * ((N + 1023) / 1024));  // tbA
    return l.total;
}

bool is_device_ptr(const void* ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// timing
// ---------------------------------------------------------------------------

cudaEvent_t take_event(claire_ctx* c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct KTimer {
    claire_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    KTimer(claire_ctx* cc, int k, double bytes, double points, double launches = 1)
        : c(cc), kind(k)
    {
        c->ks[k].launches += launches;
        c->ks[k].bytes += bytes;
        c->ks[k].points += points;
        if (c->o.timing) {
            a = take_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~KTimer()
    {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({a, b, kind, c->cur_phase});
        }
    }
};

struct PhaseScope {
    claire_ctx* c;
    int prev;
    cudaEvent_t a = nullptr;
    int ph;
    PhaseScope(claire_ctx* cc, int phase) : c(cc), prev(cc->cur_phase), ph(phase)
    {
        c->cur_phase = phase;
        if (c->o.timing) {
            a = take_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~PhaseScope()
    {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({a, b, -1, ph});
        }
        c->cur_phase = prev;
    }
};

// Fold finished event pairs into the statistics (synchronises the stream).
void collect_timing(claire_ctx* c)
{
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto& e : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            if (e.kind >= 0) {
                c->ks[e.kind].seconds += ms * 1e-3;
                if (e.kind == KK_INTERP || e.kind == KK_ADJ_STEP || e.kind == KK_INC_STEP ||
                    e.kind == KK_INC_LAST || e.kind == KK_BACKTRACE || e.kind == KK_MAP)
                    c->phase_s[CLAIRE_PHASE_GATHER] += ms * 1e-3;
            } else if (e.phase >= 0 && e.phase < 8) {
                c->phase_s[e.phase] += ms * 1e-3;
            }
        }
        c->pool.push_back(e.a);
        c->pool.push_back(e.b);
    }
    cudaGetLastError();
    c->pending.clear();
}

// ---------------------------------------------------------------------------
// building blocks on the context's stream
// ---------------------------------------------------------------------------

claire_status sync_scalars(claire_ctx* c, int count)
{
    (void)count;
    CL_CUDA(c, cudaMemcpyAsync(c->hres, c->dres, 16 * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    return CLAIRE_OK;
}

// dres[slot] = scale * sum x*y  (device only; no sync)
claire_status dot_async(claire_ctx* c, const float* x, const float* y, size_t n, double scale,
                        int slot)
{
    KTimer t(c, KK_REDUCE, 8.0 * n, 0, 2);
    launch_dot_partial(x, y, n, c->partials, c->red_blocks, c->stream);
    launch_final_sum(c->partials, c->red_blocks, scale, c->dres + slot, c->stream);
    CL_LAUNCHED(c);
    return CLAIRE_OK;
}

claire_status dot(claire_ctx* c, const float* x, const float* y, size_t n, double* out)
{
    PhaseScope ps(c, CLAIRE_PHASE_VECTOR);
    CL_TRY(dot_async(c, x, y, n, c->hvol, 0));
    CL_TRY(sync_scalars(c, 1));
    *out = c->hres[0];
    if (!std::isfinite(*out)) return fail(c, CLAIRE_ENONFINITE, "non-finite inner product");
    return CLAIRE_OK;
}

// out = F^{-1}[M(k) F[in]] for a 3N vector field
claire_status spectral(claire_ctx* c, const float* in, float* out, SpectralOp op)
{
    PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
    {
        KTimer t(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecR2C(c->r2c, const_cast<float*>(in), c->spec));
    }
    {
        KTimer t(c, KK_SPECTRAL, 48.0 * c->M, 0);
        launch_spectral(c->grid, c->spec, c->M, op, c->rp, static_cast<float>(1.0 / c->N), c->stream);
        CL_LAUNCHED(c);
    }
    {
        KTimer t(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecC2R(c->c2r, c->spec, out));
    }
    return CLAIRE_OK;
}

// out = F^{-1}[M(k) vh] for the iterate's spectrum vh (scaled by 1/N like the
// PCG spectra); vh is copied to the transform buffer first (C2R overwrites its
// input).  No forward transform: its FP32 roundoff, which the symbol M(k)
// would amplify at high |k|, never enters.
claire_status spectral_hat(claire_ctx* c, const cufftComplex* vh, float* out, SpectralOp op)
{
    PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
    CL_CUDA(c, cudaMemcpyAsync(c->spec, vh, 3 * c->M * sizeof(cufftComplex), cudaMemcpyDeviceToDevice, c->stream));
    {
        KTimer t(c, KK_SPECTRAL, 48.0 * c->M, 0);
        launch_spectral(c->grid, c->spec, c->M, op, c->rp, 1.0f, c->stream);
        CL_LAUNCHED(c);
    }
    {
        KTimer t(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecC2R(c->c2r, c->spec, out));
    }
    return CLAIRE_OK;
}

claire_status fd8_grad(claire_ctx* c, const void* f, void* out, Storage sto)
{
    KTimer t(c, KK_FD8, 4.0 * storage_bytes(sto) * c->N, 0);
    launch_fd8_grad(c->grid, f, out, sto, c->stream);
    CL_LAUNCHED(c);
    return CLAIRE_OK;
}

// Cubic B-spline coefficients of ncomp (1 or 3) FP32 fields f (Sec. 3:
// B-spline interpolation acts on prefiltered coefficients): forward
// transform, division by the sampled spline's symbol, inverse transform into
// c->bsc.  Scratch and plans are allocated on first use.
claire_status bspline_coef(claire_ctx* c, const float* f, int ncomp, const float** out)
{
    if (!c->bsc) {
        CL_CUDA(c, cudaMalloc(&c->bsc, 3 * c->N * sizeof(float)));
        CL_CUDA(c, cudaMalloc(&c->bspec, 3 * c->M * sizeof(cufftComplex)));
    }
    if (!c->bs_plans) {
        CL_FFT(c, cufftPlan3d(&c->r2c1, c->n[0], c->n[1], c->n[2], CUFFT_R2C));
        if (cufftPlan3d(&c->c2r1, c->n[0], c->n[1], c->n[2], CUFFT_C2R) != CUFFT_SUCCESS) {
            cufftDestroy(c->r2c1);
            return fail(c, CLAIRE_ECUFFT, "B-spline plans");
        }
        c->bs_plans = true;
    }
    if (ncomp == 3 && !c->plans)
        return fail(c, CLAIRE_ESTATE, "B-spline velocity coefficients need the solver's plans (kernels_only context)");
    cufftHandle fwd = ncomp == 3 ? c->r2c : c->r2c1, inv = ncomp == 3 ? c->c2r : c->c2r1;
    CL_FFT(c, cufftSetStream(c->r2c1, c->stream));
    CL_FFT(c, cufftSetStream(c->c2r1, c->stream));
    {
        KTimer t(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecR2C(fwd, const_cast<float*>(f), c->bspec));
    }
    {
        KTimer t(c, KK_SPECTRAL, 16.0 * ncomp * c->M, 0);
        launch_bspline_scale(c->grid, c->bspec, c->M, ncomp, c->stream);
        CL_LAUNCHED(c);
    }
    {
        KTimer t(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecC2R(inv, c->bspec, c->bsc));
    }
    *out = c->bsc;
    return CLAIRE_OK;
}

// the field a gather reads: f itself, or its B-spline coefficients
claire_status gather_src(claire_ctx* c, const void* f, int ncomp, const void** src)
{
    *src = f;
    if (c->o.interp != 4) return CLAIRE_OK;
    const float* coef;
    CL_TRY(bspline_coef(c, static_cast<const float*>(f), ncomp, &coef));
    *src = coef;
    return CLAIRE_OK;
}

// tile-bounds table of a displacement field of the context (null for others)
int4* tile_table(claire_ctx* c, const float* d)
{
    return d == c->dS ? c->tbS : (d == c->dA ? c->tbA : nullptr);
}

claire_status backtrace(claire_ctx* c, const float* v, float* d, int sign)
{
    const void* vc;
    CL_TRY(gather_src(c, v, 3, &vc));
    KTimer t(c, KK_BACKTRACE, 24.0 * c->N, 3.0 * c->N);
    launch_backtrace(c->grid, c->o.interp, v, static_cast<const float*>(vc), static_cast<float>(c->dt), sign, d,
                     c->stream, tile_table(c, d));
    CL_LAUNCHED(c);
    return CLAIRE_OK;
}

claire_status interp(claire_ctx* c, const void* f, const float* d, void* out, Storage sto)
{
    const void* src;
    CL_TRY(gather_src(c, f, 1, &src));
    KTimer t(c, KK_INTERP, (12.0 + 2.0 * storage_bytes(sto)) * c->N, 1.0 * c->N);
    launch_interp(c->grid, c->o.interp, src, d, out, sto, c->stream, tile_table(c, d));
    CL_LAUNCHED(c);
    return CLAIRE_OK;
}

// Per-velocity data: X, X+, div v, div v (X+).
// div v and div v(X+) are stored in `sto`.
claire_status characteristics(claire_ctx* c, const float* v, float* dS, float* dA, void* divv,
                              void* divXp, Storage sto)
{
    PhaseScope ps(c, CLAIRE_PHASE_BACKTRACE);
    if (dS) CL_TRY(backtrace(c, v, dS, +1));
    if (dA) {
        CL_TRY(backtrace(c, v, dA, -1));
        {
            KTimer t(c, KK_FD8, (12.0 + storage_bytes(sto)) * c->N, 0);
            launch_fd8_div(c->grid, v, divv, sto, c->stream);
            CL_LAUNCHED(c);
        }
        CL_TRY(interp(c, divv, dA, divXp, sto));
    }
    return CLAIRE_OK;
}


// Set the linearisation point: characteristics, states m^j and grad m^j, S v,
// objective pieces.  v (device) is copied into c->v unless it already is c->v.
// With have_state the state characteristic X (c->dS) and the states
// m^1..m^nt of this v are already in place (an accepted line-search trial).
claire_status linearise(claire_ctx* c, const float* v, bool have_state = false)
{
    if (!c->have_images) return fail(c, CLAIRE_ESTATE, "images not set (claire_set_images)");
    c->have_lin = false;
    if (v != c->v)
        CL_CUDA(c, cudaMemcpyAsync(c->v, v, 3 * c->N * sizeof(float), cudaMemcpyDeviceToDevice,
                                   c->stream));
    CL_TRY(characteristics(c, c->v, have_state ? nullptr : c->dS, c->dA, c->divv, c->divXp, c->sto));
    {
        PhaseScope ps(c, CLAIRE_PHASE_STATE);
        const size_t N = c->N;
        CL_CUDA(c, cudaMemcpyAsync(c->m, c->m0, N * c->es, cudaMemcpyDeviceToDevice, c->stream));
        if (!have_state)
            for (int j = 0; j < c->nt; ++j)
                CL_TRY(interp(c, at(c, c->m, j * N), c->dS, at(c, c->m, (j + 1) * N), c->sto));
        if (c->gm)
            for (int j = 0; j <= c->nt; ++j)
                CL_TRY(fd8_grad(c, at(c, c->m, j * N), at(c, c->gm, 3 * j * N), c->sto));
    }
    return CLAIRE_OK;
}

// Backward SL solve of Eq. (4) from lambda^{nt} = a - s (s may be null) into
// the levels tl[j], then out += sum_j w_j lambda^j grad m^j (trapezoid).
// The levels tl[1..nt] may hold the incremental sources on entry (consumed).
claire_status adjoint_and_body(claire_ctx* c, const void* a, const void* s, float* out,
                               bool accumulate = true)
{
    const size_t N = c->N;
    const int nt = c->nt;
    PhaseScope ps(c, CLAIRE_PHASE_ADJOINT);
    const double es = static_cast<double>(c->es);
    if (a) {
        KTimer t(c, KK_POINTWISE, 3.0 * es * N, 0);
        launch_sub(a, s, at(c, c->tl, nt * N), N, c->sto, c->stream);
        CL_LAUNCHED(c);
    }
    for (int j = nt - 1; j >= 0; --j) {
        const void* src;
        CL_TRY(gather_src(c, at(c, c->tl, (j + 1) * N), 1, &src));
        KTimer t(c, KK_ADJ_STEP, (12.0 + 4.0 * es) * N, 1.0 * N);
        launch_adj_step(c->grid, c->o.interp, src, c->dA, c->divv, c->divXp,
                        static_cast<float>(c->dt), at(c, c->tl, j * N), c->sto, c->stream, c->tbA);
        CL_LAUNCHED(c);
    }
    {
        if (c->gm) {
            KTimer t(c, KK_POINTWISE, (4.0 * es * (nt + 1) + (accumulate ? 24.0 : 12.0)) * N, 0);
            launch_body(c->grid, c->tl, c->gm, nt, static_cast<float>(0.5 * c->dt), static_cast<float>(c->dt),
                        accumulate ? 1 : 0, out, c->sto, c->stream);
        } else {
            KTimer t(c, KK_FD8, (2.0 * es * (nt + 1) + (accumulate ? 24.0 : 12.0)) * N, 0);
            launch_body_fd(c->grid, c->tl, c->m, nt, static_cast<float>(0.5 * c->dt), static_cast<float>(c->dt),
                           accumulate ? 1 : 0, out, c->sto, c->stream);
        }
        CL_LAUNCHED(c);
    }
    return CLAIRE_OK;
}

// g = S v + b (grad_form 0) or K(S v + b) at the current linearisation point;
// also returns J, mismatch, reg energy.
claire_status gradient_at_lin(claire_ctx* c, float* g)
{
    const size_t N = c->N;
    if (c->vh_on)
        CL_TRY(spectral_hat(c, c->vh, g, SPEC_REG));
    else
        CL_TRY(spectral(c, c->v, g, SPEC_REG));
    {
        PhaseScope ps(c, CLAIRE_PHASE_VECTOR);
        CL_TRY(dot_async(c, c->v, g, 3 * N, 0.5 * c->hvol, 0));
        KTimer t(c, KK_REDUCE, 8.0 * N, 0, 2);
        launch_sqdiff_partial(at(c, c->m, c->nt * N), c->m1, N, c->partials, c->red_blocks, c->sto, c->stream);
        launch_final_sum(c->partials, c->red_blocks, 0.5 * c->hvol, c->dres + 1, c->stream);
        CL_LAUNCHED(c);
    }
    CL_TRY(adjoint_and_body(c, c->m1, at(c, c->m, c->nt * N), g));
    if (c->o.grad_form == 1) CL_TRY(spectral(c, g, g, SPEC_K));
    CL_TRY(sync_scalars(c, 2));
    c->reg_lin = c->hres[0];
    c->mis_lin = c->hres[1];
    c->J_lin = c->reg_lin + c->mis_lin;
    if (!std::isfinite(c->J_lin)) return fail(c, CLAIRE_ENONFINITE, "non-finite objective");
    c->have_lin = true;
    return CLAIRE_OK;
}

// H vt at the linearisation point into out (out != vt).  body_only: out gets
// only the transport part int lt grad m dt (no S vt, no K), for callers that
// add the regulariser in Fourier space.
claire_status matvec(claire_ctx* c, const float* vt, float* out, bool body_only = false)
{
    if (!c->have_lin) return fail(c, CLAIRE_ESTATE, "no linearisation point (claire_gradient)");
    const size_t N = c->N;
    const int nt = c->nt;
    const float dt = static_cast<float>(c->dt);
    if (!body_only) CL_TRY(spectral(c, vt, out, SPEC_REG));
    {
        PhaseScope ps(c, CLAIRE_PHASE_INCREMENTAL);
        // sources f^j = -vt . grad m^j; Heun: q^0 = dt/2 f^0, q^{j+1} = q^j(X) + dt f^{j+1},
        // mt^{nt} = q^{nt-1}(X) + dt/2 f^{nt}, lt^{nt} = -mt^{nt}
        const double es = static_cast<double>(c->es);
        char* a = c->l0;
        char* b = c->l1;
        if (c->gm && CLAIRE_INC_FUSED) {
            // stored grad m^j: each step forms its source f^{j+1} at the arrival
            // point, so only q^0 = dt/2 f^0 is written beforehand
            {
                KTimer t(c, KK_POINTWISE, (12.0 + 4.0 * es) * N, 0);
                launch_inc_source0(c->grid, vt, c->gm, 0.5f * dt, a, c->sto, c->stream);
                CL_LAUNCHED(c);
            }
            for (int j = 0; j + 1 < nt; ++j) {
                const void* src;
                CL_TRY(gather_src(c, a, 1, &src));
                KTimer t(c, KK_INC_STEP, (24.0 + 5.0 * es) * N, 1.0 * N);
                launch_inc_step_grad(c->grid, c->o.interp, src, c->dS, vt, at(c, c->gm, 3 * (j + 1) * N), dt, b,
                                     c->sto, c->stream, c->tbS);
                CL_LAUNCHED(c);
                std::swap(a, b);
            }
            const void* src;
            CL_TRY(gather_src(c, a, 1, &src));
            KTimer t(c, KK_INC_LAST, (24.0 + 5.0 * es) * N, 1.0 * N);
            launch_inc_last_grad(c->grid, c->o.interp, src, c->dS, vt, at(c, c->gm, 3 * nt * N), 0.5f * dt,
                                 at(c, c->tl, nt * N), c->sto, c->stream, c->tbS);
            CL_LAUNCHED(c);
        } else {
            {
                if (c->gm) {
                    KTimer t(c, KK_POINTWISE, (12.0 + 4.0 * es * (nt + 1)) * N, 0);
                    launch_inc_sources(c->grid, vt, c->gm, nt, 0.5f * dt, a, c->tl, c->sto, c->stream);
                } else {
                    KTimer t(c, KK_FD8, (12.0 + 2.0 * es * (nt + 1)) * N, 0);
                    launch_inc_sources_fd(c->grid, vt, c->m, nt, 0.5f * dt, a, c->tl, c->sto, c->stream);
                }
                CL_LAUNCHED(c);
            }
            for (int j = 0; j + 1 < nt; ++j) {
                const void* src;
                CL_TRY(gather_src(c, a, 1, &src));
                KTimer t(c, KK_INC_STEP, (12.0 + 3.0 * es) * N, 1.0 * N);
                launch_inc_step_src(c->grid, c->o.interp, src, c->dS, at(c, c->tl, (j + 1) * N), dt, b, c->sto,
                                    c->stream, c->tbS);
                CL_LAUNCHED(c);
                std::swap(a, b);
            }
            const void* src;
            CL_TRY(gather_src(c, a, 1, &src));
            KTimer t(c, KK_INC_LAST, (12.0 + 3.0 * es) * N, 1.0 * N);
            launch_inc_last_src(c->grid, c->o.interp, src, c->dS, at(c, c->tl, nt * N), 0.5f * dt,
                                at(c, c->tl, nt * N), c->sto, c->stream, c->tbS);
            CL_LAUNCHED(c);
        }
    }
    // incremental adjoint from lt^{nt} and body, accumulated onto S vt in out
    CL_TRY(adjoint_and_body(c, nullptr, nullptr, out, !body_only));
    if (body_only) return CLAIRE_OK;
    if (c->o.grad_form == 1) CL_TRY(spectral(c, out, out, SPEC_K));
    return CLAIRE_OK;
}

claire_status precond(claire_ctx* c, const float* r, float* z)
{
    return spectral(c, r, z, c->o.grad_form == 1 ? SPEC_AINV : SPEC_INV);
}

// J(v) for a trial v (device, 3N); uses z (displacement), l0/l1, r (S v).
// With into_state the characteristic and the states m^1..m^nt are written to
// c->dS and c->m (the line search, once the linearisation point is spent),
// so that an accepted trial seeds the next linearisation.
claire_status objective_at(claire_ctx* c, const float* v, double* J, double* mis,
                           bool into_state = false)
{
    if (!c->have_images) return fail(c, CLAIRE_ESTATE, "images not set (claire_set_images)");
    const size_t N = c->N;
    PhaseScope ps(c, CLAIRE_PHASE_OBJECTIVE);
    float* d = into_state ? c->dS : c->z;
    if (into_state) c->have_lin = false;
    CL_TRY(backtrace(c, v, d, +1));
    const char* src = c->m0;
    char* a = c->l0;
    char* b = c->l1;
    for (int j = 0; j < c->nt; ++j) {
        char* dst = into_state ? at(c, c->m, (j + 1) * N) : a;
        CL_TRY(interp(c, src, d, dst, c->sto));
        src = dst;
        std::swap(a, b);
    }
    CL_TRY(spectral(c, v, c->r, SPEC_REG));
    CL_TRY(dot_async(c, v, c->r, 3 * N, 0.5 * c->hvol, 0));
    {
        KTimer t(c, KK_REDUCE, 8.0 * N, 0, 2);
        launch_sqdiff_partial(src, c->m1, N, c->partials, c->red_blocks, c->sto, c->stream);
        launch_final_sum(c->partials, c->red_blocks, 0.5 * c->hvol, c->dres + 1, c->stream);
        CL_LAUNCHED(c);
    }
    CL_TRY(sync_scalars(c, 2));
    if (mis) *mis = c->hres[1];
    if (J) *J = c->hres[0] + c->hres[1];
    if (!std::isfinite(c->hres[0] + c->hres[1]))
        return fail(c, CLAIRE_ENONFINITE, "non-finite objective");
    return CLAIRE_OK;
}

// Extrema of det(I + grad u) of the deformation map of v (device, 3N).
// Uses z (displacement), r and p (map), partials.
claire_status detj_of(claire_ctx* c, const float* v, double* lo, double* hi)
{
    const size_t N = c->N;
    CL_TRY(backtrace(c, v, c->z, +1));
    float* a = c->r;
    float* b = c->p;
    CL_CUDA(c, cudaMemsetAsync(a, 0, 3 * N * sizeof(float), c->stream));
    for (int j = 0; j < c->nt; ++j) {
        const void* src;
        CL_TRY(gather_src(c, a, 3, &src));
        KTimer t(c, KK_MAP, 36.0 * N, 3.0 * N);
        launch_map_step(c->grid, c->o.interp, static_cast<const float*>(src), c->z, b, c->stream);
        CL_LAUNCHED(c);
        std::swap(a, b);
    }
    {
        KTimer t(c, KK_DETJ, 12.0 * N, 0, 2);
        launch_detj_minmax(c->grid, a, c->partials + c->red_blocks, c->partials, c->red_blocks,
                           c->stream);
        launch_final_minmax(c->partials + c->red_blocks, c->partials, c->red_blocks, c->dres + 4,
                            c->stream);
        CL_LAUNCHED(c);
    }
    CL_CUDA(c, cudaMemcpyAsync(c->hres + 4, c->dres + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    *lo = c->hres[4];
    *hi = c->hres[5];
    return CLAIRE_OK;
}

claire_status cfl_of(claire_ctx* c, const float* v, double* cfl)
{
    {
        KTimer t(c, KK_REDUCE, 12.0 * c->N, 0, 2);
        launch_maxnorm3_partial(v, c->N, c->partials, c->red_blocks, c->stream);
        launch_final_max(c->partials, c->red_blocks, c->dres + 6, c->stream);
        CL_LAUNCHED(c);
    }
    CL_CUDA(c, cudaMemcpyAsync(c->hres + 6, c->dres + 6, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    const double hmin = std::min(c->grid.h1, std::min(c->grid.h2, c->grid.h3));
    *cfl = std::sqrt(c->hres[7]) * c->dt / hmin;
    return CLAIRE_OK;
}

// Reject a velocity (device, 3N) with a non-finite component before any
// gather runs on it: the FP64 maximum of |v(x)|^2 keeps a NaN or an Inf.
claire_status screen_velocity(claire_ctx* c, const float* v)
{
    double cfl;
    CL_TRY(cfl_of(c, v, &cfl));
    if (!std::isfinite(cfl)) return fail(c, CLAIRE_ENONFINITE, "non-finite velocity");
    return CLAIRE_OK;
}

// Final sums of the two partial-sum arrays of a Fourier-space PCG kernel
// into dres[0], dres[1] (scaled to discrete inner products), then synchronise.
claire_status fs_sums(claire_ctx* c, int count)
{
    const double scale = c->hvol * static_cast<double>(c->N);  // Parseval on scaled spectra
    launch_final_sum(c->partials, c->red_blocks, scale, c->dres, c->stream);
    if (count > 1) launch_final_sum(c->partials + c->red_blocks, c->red_blocks, scale, c->dres + 1, c->stream);
    CL_LAUNCHED(c);
    CL_TRY(sync_scalars(c, count));
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(c->hres[i])) return fail(c, CLAIRE_ENONFINITE, "non-finite PCG inner product");
    return CLAIRE_OK;
}

// ---- two-level zero-velocity preconditioner (Sec. 2.2) ----

// Allocate the coarse-grid state for the current pc_coarse (once).
claire_status tl_ensure(claire_ctx* c)
{
    const int f = c->o.pc_coarse;
    if (c->tl2 && c->tl2->factor == f) return CLAIRE_OK;
    if (!valid_coarse(c->n, f))
        return fail(c, CLAIRE_EINVAL, "pc_coarse %d: every grid size / pc_coarse must be even and >= 4", f);
    delete c->tl2;
    c->tl2 = nullptr;
    TwoLevel* t = new (std::nothrow) TwoLevel();
    if (!t) return fail(c, CLAIRE_ENOMEM, "two-level preconditioner state");
    const int nc[3] = {c->n[0] / f, c->n[1] / f, c->n[2] / f};
    t->factor = f;
    t->g = grid_of(nc[0], nc[1], nc[2]);
    t->N = static_cast<size_t>(nc[0]) * nc[1] * nc[2];
    t->M = static_cast<size_t>(nc[0]) * nc[1] * (nc[2] / 2 + 1);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t realb = up(3 * t->N * sizeof(float)), specb = up(3 * t->M * sizeof(cufftComplex)),
                 fineb = up(3 * c->M * sizeof(cufftComplex));
    const size_t total = 2 * realb + 7 * specb + fineb + up(kTlSlots * sizeof(double));
    if (cudaMalloc(&t->block, total) != cudaSuccess) {
        cudaGetLastError();
        t->block = nullptr;
        delete t;
        return fail(c, CLAIRE_ENOMEM, "two-level preconditioner buffers (%zu bytes)", total);
    }
    char* b = static_cast<char*>(t->block);
    t->gbar = reinterpret_cast<float*>(b); b += realb;
    t->real = reinterpret_cast<float*>(b); b += realb;
    cufftComplex** sp[7] = {&t->xh, &t->rh, &t->zh, &t->ph, &t->cp, &t->q, &t->T};
    for (auto q : sp) {
        *q = reinterpret_cast<cufftComplex*>(b);
        b += specb;
    }
    t->zf = reinterpret_cast<cufftComplex*>(b);
    b += fineb;
    t->sc = reinterpret_cast<double*>(b);
    size_t ws1 = 0, ws2 = 0;
    cufftResult fr = cufftCreate(&t->r2c);
    if (fr == CUFFT_SUCCESS) {
        fr = cufftCreate(&t->c2r);
        if (fr != CUFFT_SUCCESS) cufftDestroy(t->r2c);
    }
    if (fr != CUFFT_SUCCESS) {
        delete t;
        return fail(c, CLAIRE_ECUFFT, "coarse-grid FFT plans");
    }
    t->plans = true;
    int nn[3] = {nc[0], nc[1], nc[2]};
    fr = cufftSetAutoAllocation(t->r2c, 0);
    if (fr == CUFFT_SUCCESS) fr = cufftSetAutoAllocation(t->c2r, 0);
    if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany(t->r2c, 3, nn, nullptr, 1, (int)t->N, nullptr, 1, (int)t->M, CUFFT_R2C, 3, &ws1);
    if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany(t->c2r, 3, nn, nullptr, 1, (int)t->M, nullptr, 1, (int)t->N, CUFFT_C2R, 3, &ws2);
    const size_t ws = std::max<size_t>(std::max(ws1, ws2), 256);
    if (fr == CUFFT_SUCCESS && cudaMalloc(&t->work, ws) != cudaSuccess) {
        cudaGetLastError();
        t->work = nullptr;
        fr = CUFFT_ALLOC_FAILED;
    }
    if (fr == CUFFT_SUCCESS) fr = cufftSetWorkArea(t->r2c, t->work);
    if (fr == CUFFT_SUCCESS) fr = cufftSetWorkArea(t->c2r, t->work);
    if (fr == CUFFT_SUCCESS) fr = cufftSetStream(t->r2c, c->stream);
    if (fr == CUFFT_SUCCESS) fr = cufftSetStream(t->c2r, c->stream);
    if (fr != CUFFT_SUCCESS) {
        delete t;
        return fail(c, fr == CUFFT_ALLOC_FAILED ? CLAIRE_ENOMEM : CLAIRE_ECUFFT, "coarse-grid FFT plans");
    }
    c->tl2 = t;
    return CLAIRE_OK;
}

// gbar = sum_j w_j grad m^j at the linearisation point into out (device,
// 3N): the FD8 gradient of the trapezoid mean of the states (FD8 is linear).
// Uses l0.
claire_status mean_state_gradient(claire_ctx* c, float* out)
{
    if (!c->have_lin) return fail(c, CLAIRE_ESTATE, "no linearisation point (claire_gradient)");
    const size_t N = c->N;
    float* mean = reinterpret_cast<float*>(c->l0);
    {
        KTimer kt(c, KK_POINTWISE, (storage_bytes(c->sto) * (c->nt + 1) + 4.0) * N, 0);
        launch_mean_levels(c->m, c->nt, static_cast<float>(0.5 * c->dt), static_cast<float>(c->dt), N, mean,
                           c->sto, c->stream);
        CL_LAUNCHED(c);
    }
    return fd8_grad(c, mean, out, Storage::F32);
}

// gbar_c = R (sum_j w_j grad m^j) at the linearisation point, restricted
// spectrally; with a coarse preconditioner weight w installed, gbar_c is then
// scaled by sqrt(w), so the coarse operator becomes S + gbar_c w gbar_c^T.
claire_status tl_prepare(claire_ctx* c)
{
    if (!c->have_lin) return fail(c, CLAIRE_ESTATE, "no linearisation point (claire_gradient)");
    CL_TRY(tl_ensure(c));
    TwoLevel* t = c->tl2;
    if (c->pcw_on && (c->pcw_grid[0] != t->g.n1 || c->pcw_grid[1] != t->g.n2 || c->pcw_grid[2] != t->g.n3))
        return fail(c, CLAIRE_EINVAL, "preconditioner weight on %d x %d x %d, coarse grid %d x %d x %d",
                    c->pcw_grid[0], c->pcw_grid[1], c->pcw_grid[2], t->g.n1, t->g.n2, t->g.n3);
    PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
    const size_t N = c->N;
    CL_TRY(mean_state_gradient(c, c->z));
    {
        KTimer kt(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecR2C(c->r2c, c->z, c->spec2));
    }
    launch_tl_restrict(c->grid, c->spec2, c->M, t->g, t->xh, t->M, static_cast<float>(1.0 / N), c->stream);
    CL_LAUNCHED(c);
    {
        KTimer kt(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecC2R(t->c2r, t->xh, t->gbar));
    }
    if (c->pcw_on) {
        KTimer kt(c, KK_POINTWISE, 28.0 * t->N, 0);
        launch_tl_weight(t->gbar, c->pcw, t->N, c->stream);
        CL_LAUNCHED(c);
    }
    return CLAIRE_OK;
}

// zf = P^{-1} rf on scaled fine half spectra; *rz = <rf, zf>, *ro = <rf, zold>
// (0 when zold is null); *its = inner PCG iterations.
claire_status tl_apply(claire_ctx* c, const cufftComplex* rf, cufftComplex* zf, const cufftComplex* zold,
                       double* rz, double* ro, int* its)
{
    TwoLevel* t = c->tl2;
    const SpectralOp op = c->o.grad_form == 1 ? SPEC_AINV : SPEC_INV;
    const int rb = c->red_blocks;
    PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
    *its = 0;
    {
        KTimer kt(c, KK_SPECTRAL, 120.0 * t->M, 0, 2);
        launch_tl_start(c->grid, rf, c->M, t->g, t->rh, t->xh, t->ph, t->cp, t->M, op, c->rp, c->partials,
                        c->partials + rb, rb, c->stream);
    }
    CL_TRY(fs_sums(c, 2));
    const double r0 = std::sqrt(c->hres[0]);
    // rz stays on the device: alpha and beta are formed there (FP64, as the host
    // would), so an iteration reads back only |r|^2 and the breakdown flag
    CL_CUDA(c, cudaMemcpyAsync(t->sc + kTlRz, c->dres + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    const double scale = c->hvol * static_cast<double>(c->N);  // Parseval on scaled spectra, as fs_sums
    for (int it = 1; r0 > 0.0 && it <= c->o.pc_maxit; ++it) {
        {
            KTimer kt(c, KK_FFT, 0, 0);
            CL_FFT(c, cufftExecC2R(t->c2r, t->cp, t->real));
        }
        {
            KTimer kt(c, KK_POINTWISE, 36.0 * t->N, 0);
            launch_tl_rank1(t->gbar, t->real, t->N, c->stream);
            CL_LAUNCHED(c);
        }
        {
            KTimer kt(c, KK_FFT, 0, 0);
            CL_FFT(c, cufftExecR2C(t->r2c, t->real, t->T));
        }
        {
            KTimer kt(c, KK_SPECTRAL, 72.0 * t->M, 0, 3);
            launch_tl_hp(t->g, t->T, t->ph, t->q, t->M, c->o.grad_form, c->rp, static_cast<float>(1.0 / t->N),
                         c->partials, rb, c->stream);
            launch_final_sum(c->partials, rb, scale, t->sc + kTlPq, c->stream);
            launch_tl_scalars(t->sc, 0, c->stream);
            CL_LAUNCHED(c);
        }
        {
            KTimer kt(c, KK_SPECTRAL, 144.0 * t->M, 0, 4);
            launch_tl_update(t->g, t->ph, t->q, t->xh, t->rh, t->zh, t->M, t->sc + kTlAlpha, op, c->rp,
                             c->partials, c->partials + rb, rb, c->stream);
            launch_final_sum(c->partials, rb, scale, t->sc + kTlRr, c->stream);
            launch_final_sum(c->partials + rb, rb, scale, t->sc + kTlRzNew, c->stream);
            CL_LAUNCHED(c);
        }
        CL_CUDA(c, cudaMemcpyAsync(c->hres + 8, t->sc + kTlRr, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
        CL_CUDA(c, cudaStreamSynchronize(c->stream));
        const double rr = c->hres[8], flag = c->hres[9];
        *its = it;
        if (flag == 2.0) return fail(c, CLAIRE_ENONFINITE, "non-finite inner PCG curvature");
        if (flag != 0.0) break;  // pq <= 0: the update above ran with alpha = 0
        if (!std::isfinite(rr)) return fail(c, CLAIRE_ENONFINITE, "non-finite inner PCG residual");
        if (c->o.pc_tol > 0 && std::sqrt(rr) <= c->o.pc_tol * r0) break;
        if (it == c->o.pc_maxit) break;
        {
            KTimer kt(c, KK_SPECTRAL, 72.0 * t->M, 0, 2);
            launch_tl_scalars(t->sc, 1, c->stream);
            launch_dir_stored(t->g, t->zh, t->ph, t->cp, t->M, 0.0f, 0, c->stream, t->sc + kTlBeta);
            CL_LAUNCHED(c);
        }
    }
    {
        KTimer kt(c, KK_SPECTRAL, (zold ? 72.0 : 48.0) * c->M, 0, 2);
        launch_tl_finish(c->grid, rf, zf, zold, c->M, t->g, t->xh, t->M, op, c->rp, c->partials, c->partials + rb,
                         rb, c->stream);
    }
    CL_TRY(fs_sums(c, 2));
    *rz = c->hres[0];
    *ro = zold ? c->hres[1] : 0.0;
    c->pc_inner_total += *its;
    return CLAIRE_OK;
}

// Matrix-free PCG for H x = -g (x0 = 0), preconditioned by the spectral
// inverse of the regulariser or the two-level zero-velocity preconditioner
// (precond = 1, flexible direction update).  x, r and the direction p live in Fourier
// space (scaled half spectra); the preconditioner, the regulariser part of
// H p and every inner product (Parseval) are spectral.  Each iteration takes
// one inverse transform (p, for the transport solves) and one forward
// transform (the transport part of H p).  Returns the iteration count in *its.
claire_status pcg(claire_ctx* c, double eta, int* its)
{
    const SpectralOp op = c->o.grad_form == 1 ? SPEC_AINV : SPEC_INV;
    const float scale = static_cast<float>(1.0 / c->N);
    const double M = static_cast<double>(c->M);
    const bool two_level = c->o.precond == CLAIRE_PRECOND_TWO_LEVEL;
    *its = 0;
    if (two_level) CL_TRY(tl_prepare(c));
    {
        PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
        {
            KTimer t(c, KK_FFT, 0, 0);
            CL_FFT(c, cufftExecR2C(c->r2c, c->g, c->spec));
        }
        KTimer t(c, KK_SPECTRAL, 72.0 * M, 0, 3);
        launch_fs_start(c->grid, c->spec, c->rh, c->xh, c->M, op, c->rp, scale, c->partials,
                        c->partials + c->red_blocks, c->red_blocks, c->stream);
    }
    CL_TRY(fs_sums(c, 2));
    const double r0 = std::sqrt(c->hres[0]);
    double rz = c->hres[1];
    if (r0 == 0.0) {
        CL_CUDA(c, cudaMemsetAsync(c->x, 0, 3 * c->N * sizeof(float), c->stream));
        return CLAIRE_OK;
    }
    // two-level: z~ = P^{-1} r~ is stored (zf) and the direction update is
    // the flexible one, beta = <r_new, z_new - z_old> / <r_old, z_old>
    int inner_its = 0;
    if (two_level) {
        double ro;
        CL_TRY(tl_apply(c, c->rh, c->tl2->zf, nullptr, &rz, &ro, &inner_its));
    }
    double beta = 0.0;
    for (int it = 1; it <= c->o.max_pcg; ++it) {
        *its = it;
        {
            PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
            {
                KTimer t(c, KK_SPECTRAL, (it == 1 ? 72.0 : 96.0) * M, 0);
                if (two_level)
                    launch_dir_stored(c->grid, c->tl2->zf, c->phat, c->spec2, c->M, static_cast<float>(beta),
                                      it == 1 ? 1 : 0, c->stream);
                else
                    launch_spectral_direction(c->grid, c->rh, c->phat, c->spec2, c->M, static_cast<float>(beta),
                                              it == 1 ? 1 : 0, op, c->rp, c->stream);
                CL_LAUNCHED(c);
            }
            KTimer t(c, KK_FFT, 0, 0);
            CL_FFT(c, cufftExecC2R(c->c2r, c->spec2, c->p));
        }
        CL_TRY(matvec(c, c->p, c->z, true));  // transport part of H p
        {
            PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
            {
                KTimer t(c, KK_FFT, 0, 0);
                CL_FFT(c, cufftExecR2C(c->r2c, c->z, c->spec2));
            }
            KTimer t(c, KK_SPECTRAL, 72.0 * M, 0, 2);
            launch_fs_hp(c->grid, c->spec, c->spec2, c->phat, c->M, c->o.grad_form, c->rp, scale,
                         c->partials, c->red_blocks, c->stream);
        }
        CL_TRY(fs_sums(c, 1));
        const double pq = c->hres[0];
        if (pq <= 0.0) {
            if (it == 1)
                CL_CUDA(c, cudaMemcpyAsync(c->xh, c->phat, 3 * c->M * sizeof(cufftComplex),
                                           cudaMemcpyDeviceToDevice, c->stream));
            break;
        }
        const double alpha = rz / pq;
        {
            PhaseScope ps(c, CLAIRE_PHASE_VECTOR);
            KTimer t(c, KK_SPECTRAL, 144.0 * M, 0, 3);
            launch_fs_update(c->grid, c->spec, c->phat, c->xh, c->rh, two_level ? c->tl2->zf : nullptr, c->M,
                             static_cast<float>(alpha), op, c->rp, c->partials, c->partials + c->red_blocks,
                             c->red_blocks, c->stream);
        }
        CL_TRY(fs_sums(c, 2));
        const double rr = c->hres[0];
        if (!c->o.pcg_fixed && std::sqrt(rr) <= eta * r0) break;
        if (it == c->o.max_pcg) break;
        if (two_level) {
            // <r_new, z_old> = <r_old, z_old> - alpha <H p, z_old>; z_new overwrites z_old
            const double ro = rz - alpha * c->hres[1];
            double rz_new, unused;
            CL_TRY(tl_apply(c, c->rh, c->tl2->zf, nullptr, &rz_new, &unused, &inner_its));
            beta = (rz_new - ro) / rz;
            rz = rz_new;
        } else {
            beta = c->hres[1] / rz;
            rz = c->hres[1];
        }
    }
    {
        // the multi-dimensional C2R may overwrite its input: transform a copy, so
        // that xh still holds the solution's spectrum for the iterate's update
        PhaseScope ps(c, CLAIRE_PHASE_SPECTRAL);
        CL_CUDA(c, cudaMemcpyAsync(c->phat, c->xh, 3 * c->M * sizeof(cufftComplex), cudaMemcpyDeviceToDevice,
                                   c->stream));
        KTimer t(c, KK_FFT, 0, 0);
        CL_FFT(c, cufftExecC2R(c->c2r, c->phat, c->x));
    }
    return CLAIRE_OK;
}

// Copy an input array (host or device) to a device pointer usable by kernels.
claire_status device_input(claire_ctx* c, const float* src, size_t n, float* scratch,
                           const float** out)
{
    if (!src) return fail(c, CLAIRE_EINVAL, "null array argument");
    if (is_device_ptr(src)) {
        *out = src;
        return CLAIRE_OK;
    }
    CL_CUDA(c, cudaMemcpyAsync(scratch, src, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    *out = scratch;
    return CLAIRE_OK;
}

claire_status copy_out(claire_ctx* c, float* dst, const float* src, size_t n)
{
    if (!dst) return fail(c, CLAIRE_EINVAL, "null output argument");
    if (dst == src) return CLAIRE_OK;
    CL_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDefault, c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    return CLAIRE_OK;
}

claire_status check_kernel_ptr(claire_ctx* c, const void* p)
{
    if (!p) return fail(c, CLAIRE_EINVAL, "null pointer");
    if (!is_device_ptr(p)) return fail(c, CLAIRE_EINVAL, "kernel-level entry points take device pointers");
    return CLAIRE_OK;
}

// Solver-level calls need the full workspace and the transform plans.
claire_status need_workspace(claire_ctx* c)
{
    if (c->o.kernels_only)
        return fail(c, CLAIRE_ESTATE, "context created with kernels_only = 1 (kernel-level entry points only)");
    return CLAIRE_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

claire_status claire_default_opts(claire_opts* opts)
{
    if (!opts) return CLAIRE_EINVAL;
    fill_defaults(opts);
    return CLAIRE_OK;
}

claire_status claire_query_workspace(const int grid[3], int nt, const claire_opts* opts,
                                     size_t* bytes)
{
    if (!valid_grid(grid) || nt < 1 || !bytes) return CLAIRE_EINVAL;
    const size_t N = (size_t)grid[0] * grid[1] * grid[2];
    const size_t M = (size_t)grid[0] * grid[1] * (grid[2] / 2 + 1);
    const int sto = opts ? opts->storage : 0;
    if (sto < 0 || sto > 2) return CLAIRE_EINVAL;
    const bool lowmem = opts ? opts->lowmem != 0 : false;
    if (opts && opts->kernels_only) {
        *bytes = (2 * 152 * 8 + 16) * sizeof(double);  // reduction partials and device scalars
        return CLAIRE_OK;
    }
    *bytes = layout_floats(N, M, nt, 152 * 8, storage_bytes(static_cast<Storage>(sto)), lowmem, nullptr) *
             sizeof(float);
    return CLAIRE_OK;
}

claire_status claire_create(claire_ctx** out, const int grid[3], double beta_v, int nt,
                            const claire_opts* opts)
{
    if (!out) return CLAIRE_EINVAL;
    *out = nullptr;
    if (!valid_grid(grid) || !(beta_v > 0) || nt < 1) return CLAIRE_EINVAL;
    claire_opts o;
    if (opts)
        o = *opts;
    else
        fill_defaults(&o);
    if (!valid_opts(o)) return CLAIRE_EINVAL;
    if (o.precond == CLAIRE_PRECOND_TWO_LEVEL && !valid_coarse(grid, o.pc_coarse)) return CLAIRE_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return CLAIRE_ECUDA;
    }
    claire_ctx* c = new (std::nothrow) claire_ctx();
    if (!c) return CLAIRE_ENOMEM;
    c->o = o;
    for (int i = 0; i < 3; ++i) c->n[i] = grid[i];
    c->N = (size_t)grid[0] * grid[1] * grid[2];
    c->M = (size_t)grid[0] * grid[1] * (grid[2] / 2 + 1);
    c->nt = nt;
    c->dt = 1.0 / nt;
    c->beta_v = beta_v;
    const double two_pi = 6.283185307179586476925286766559;
    Grid& g = c->grid;
    g.n1 = grid[0];
    g.n2 = grid[1];
    g.n3 = grid[2];
    g.n23 = grid[1] * grid[2];
    g.N = static_cast<uint32_t>(c->N);
    g.h1 = static_cast<float>(two_pi / grid[0]);
    g.h2 = static_cast<float>(two_pi / grid[1]);
    g.h3 = static_cast<float>(two_pi / grid[2]);
    g.ih1 = static_cast<float>(grid[0] / two_pi);
    g.ih2 = static_cast<float>(grid[1] / two_pi);
    g.ih3 = static_cast<float>(grid[2] / two_pi);
    c->hvol = (two_pi / grid[0]) * (two_pi / grid[1]) * (two_pi / grid[2]);
    c->rp.beta_v = static_cast<float>(beta_v);
    c->rp.beta_w = static_cast<float>(o.beta_w);
    c->rp.reg = o.reg;

    claire_status st = CLAIRE_OK;
    auto bail = [&](claire_status s) {
        delete c;
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(CLAIRE_ECUDA);
    }
    c->red_blocks = std::max(1, c->nsm) * 4;
    if (o.kernels_only) {
        // reduction partials and the device scalars only: no fields, no plans
        const size_t bytes = (2 * static_cast<size_t>(c->red_blocks) + 16) * sizeof(double);
        if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->arena = nullptr;
            return bail(CLAIRE_ENOMEM);
        }
        c->arena_bytes = bytes;
        c->partials = static_cast<double*>(c->arena);
        c->dres = c->partials + 2 * c->red_blocks;
        if (cudaMemset(c->dres, 0, 16 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return bail(CLAIRE_ECUDA);
        }
        if (cudaMallocHost(&c->hres, 16 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->hres = nullptr;
            return bail(CLAIRE_ENOMEM);
        }
        st = claire_set_stream(c, nullptr);
        if (st != CLAIRE_OK) return bail(st);
        *out = c;
        return CLAIRE_OK;
    }
    Layout L;
    c->sto = static_cast<Storage>(o.storage);
    c->es = storage_bytes(c->sto);
    size_t floats = layout_floats(c->N, c->M, nt, c->red_blocks, c->es, o.lowmem != 0, &L);
    cudaError_t e = cudaMalloc(&c->arena, floats * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->arena = nullptr;
        return bail(e == cudaErrorMemoryAllocation ? CLAIRE_ENOMEM : CLAIRE_ECUDA);
    }
    c->arena_bytes = floats * sizeof(float);
    float* base = static_cast<float*>(c->arena);
    int k = 0;
    c->m0 = reinterpret_cast<char*>(base + L.off[k++]);
    c->m1 = reinterpret_cast<char*>(base + L.off[k++]);
    c->v = base + L.off[k++];
    c->dS = base + L.off[k++];
    c->dA = base + L.off[k++];
    c->divv = reinterpret_cast<char*>(base + L.off[k++]);
    c->divXp = reinterpret_cast<char*>(base + L.off[k++]);
    c->m = reinterpret_cast<char*>(base + L.off[k++]);
    c->gm = o.lowmem ? nullptr : reinterpret_cast<char*>(base + L.off[k]);
    ++k;
    c->l0 = reinterpret_cast<char*>(base + L.off[k++]);
    c->l1 = reinterpret_cast<char*>(base + L.off[k++]);
    c->tl = reinterpret_cast<char*>(base + L.off[k++]);
    c->g = base + L.off[k++];
    c->x = base + L.off[k++];
    c->r = base + L.off[k++];
    c->z = base + L.off[k++];
    c->p = base + L.off[k++];
    c->spec = reinterpret_cast<cufftComplex*>(base + L.off[k++]);
    c->phat = reinterpret_cast<cufftComplex*>(base + L.off[k++]);
    c->spec2 = reinterpret_cast<cufftComplex*>(base + L.off[k++]);
    c->xh = reinterpret_cast<cufftComplex*>(base + L.off[k++]);
    c->rh = reinterpret_cast<cufftComplex*>(base + L.off[k++]);
    c->partials = reinterpret_cast<double*>(base + L.off[k++]);
    c->dres = reinterpret_cast<double*>(base + L.off[k++]);
    c->tbS = reinterpret_cast<int4*>(base + L.off[k++]);
    c->tbA = reinterpret_cast<int4*>(base + L.off[k++]);
    if (cudaMemset(c->dres, 0, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(CLAIRE_ECUDA);
    }
    if (cudaMallocHost(&c->hres, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->hres = nullptr;
        return bail(CLAIRE_ENOMEM);
    }
    // both plans share one work area (they never run concurrently: one stream)
    int nn[3] = {grid[0], grid[1], grid[2]};
    size_t ws_r2c = 0, ws_c2r = 0;
    cufftResult fr = cufftCreate(&c->r2c);
    if (fr == CUFFT_SUCCESS) {
        fr = cufftCreate(&c->c2r);
        if (fr != CUFFT_SUCCESS) cufftDestroy(c->r2c);
    }
    if (fr != CUFFT_SUCCESS) return bail(CLAIRE_ECUFFT);
    c->plans = true;
    fr = cufftSetAutoAllocation(c->r2c, 0);
    if (fr == CUFFT_SUCCESS) fr = cufftSetAutoAllocation(c->c2r, 0);
    if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany(c->r2c, 3, nn, nullptr, 1, (int)c->N, nullptr, 1, (int)c->M, CUFFT_R2C, 3,
                               &ws_r2c);
    if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany(c->c2r, 3, nn, nullptr, 1, (int)c->M, nullptr, 1, (int)c->N, CUFFT_C2R, 3,
                               &ws_c2r);
    if (fr != CUFFT_SUCCESS) return bail(fr == CUFFT_ALLOC_FAILED ? CLAIRE_ENOMEM : CLAIRE_ECUFFT);
    const size_t ws = std::max<size_t>(std::max(ws_r2c, ws_c2r), 256);
    if (cudaMalloc(&c->fft_work, ws) != cudaSuccess) {
        cudaGetLastError();
        c->fft_work = nullptr;
        return bail(CLAIRE_ENOMEM);
    }
    c->fft_work_bytes = ws;
    fr = cufftSetWorkArea(c->r2c, c->fft_work);
    if (fr == CUFFT_SUCCESS) fr = cufftSetWorkArea(c->c2r, c->fft_work);
    if (fr != CUFFT_SUCCESS) return bail(CLAIRE_ECUFFT);
    st = claire_set_stream(c, nullptr);
    if (st != CLAIRE_OK) return bail(st);
    *out = c;
    return CLAIRE_OK;
}

claire_status claire_destroy(claire_ctx* ctx)
{
    if (!ctx) return CLAIRE_OK;
    cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();
    delete ctx;
    return CLAIRE_OK;
}

claire_status claire_set_stream(claire_ctx* c, void* stream)
{
    if (!c) return CLAIRE_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    if (c->plans) {
        CL_FFT(c, cufftSetStream(c->r2c, c->stream));
        CL_FFT(c, cufftSetStream(c->c2r, c->stream));
    }
    if (c->bs_plans) {
        CL_FFT(c, cufftSetStream(c->r2c1, c->stream));
        CL_FFT(c, cufftSetStream(c->c2r1, c->stream));
    }
    if (c->tl2) {
        CL_FFT(c, cufftSetStream(c->tl2->r2c, c->stream));
        CL_FFT(c, cufftSetStream(c->tl2->c2r, c->stream));
    }
    return CLAIRE_OK;
}

claire_status claire_set_images(claire_ctx* c, const float* m0, const float* m1)
{
    if (!c || !m0 || !m1) return c ? fail(c, CLAIRE_EINVAL, "null image") : CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    const size_t N = c->N;
    if (c->sto == Storage::F32) {
        CL_CUDA(c, cudaMemcpyAsync(c->m0, m0, N * sizeof(float), cudaMemcpyDefault, c->stream));
        CL_CUDA(c, cudaMemcpyAsync(c->m1, m1, N * sizeof(float), cudaMemcpyDefault, c->stream));
    } else {
        // FP32 input (host or device) converted to the storage type on the device
        const float* d0 = nullptr;
        CL_TRY(device_input(c, m0, N, c->p, &d0));
        launch_to_storage(d0, c->m0, N, c->sto, c->stream);
        const float* d1 = nullptr;
        CL_TRY(device_input(c, m1, N, c->z, &d1));
        launch_to_storage(d1, c->m1, N, c->sto, c->stream);
        CL_LAUNCHED(c);
    }
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_images = true;
    c->have_lin = false;
    return CLAIRE_OK;
}

claire_status claire_objective(claire_ctx* c, const float* v, double* J, double* mismatch)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    const float* dv = nullptr;
    CL_TRY(device_input(c, v, 3 * c->N, c->p, &dv));
    CL_TRY(screen_velocity(c, dv));
    claire_status s = objective_at(c, dv, J, mismatch);
    collect_timing(c);
    return s;
}

claire_status claire_gradient(claire_ctx* c, const float* v, float* g, double* J)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!v || !g) return fail(c, CLAIRE_EINVAL, "null argument");
    if (!c->have_images) return fail(c, CLAIRE_ESTATE, "images not set (claire_set_images)");
    const float* dv = nullptr;
    CL_TRY(device_input(c, v, 3 * c->N, c->v, &dv));
    CL_TRY(screen_velocity(c, dv));
    CL_TRY(linearise(c, dv));
    CL_TRY(gradient_at_lin(c, c->g));
    if (J) *J = c->J_lin;
    CL_TRY(copy_out(c, g, c->g, 3 * c->N));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_hessian_matvec(claire_ctx* c, const float* vt, float* Hvt)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!vt || !Hvt) return fail(c, CLAIRE_EINVAL, "null argument");
    const float* dvt = nullptr;
    CL_TRY(device_input(c, vt, 3 * c->N, c->p, &dvt));
    CL_TRY(matvec(c, dvt, c->r));
    CL_TRY(copy_out(c, Hvt, c->r, 3 * c->N));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_precond(claire_ctx* c, const float* r, float* z)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!r || !z) return fail(c, CLAIRE_EINVAL, "null argument");
    const float* dr = nullptr;
    CL_TRY(device_input(c, r, 3 * c->N, c->p, &dr));
    if (c->o.precond == CLAIRE_PRECOND_TWO_LEVEL) {
        CL_TRY(tl_prepare(c));
        CL_FFT(c, cufftExecR2C(c->r2c, const_cast<float*>(dr), c->rh));
        launch_cscale(c->rh, 3 * c->M, static_cast<float>(1.0 / c->N), c->stream);
        CL_LAUNCHED(c);
        double rz, ro;
        int its;
        CL_TRY(tl_apply(c, c->rh, c->tl2->zf, nullptr, &rz, &ro, &its));
        CL_FFT(c, cufftExecC2R(c->c2r, c->tl2->zf, c->r));
    } else {
        CL_TRY(precond(c, dr, c->r));
    }
    CL_TRY(copy_out(c, z, c->r, 3 * c->N));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_register(claire_ctx* c, float* v_inout, claire_report* rep)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!v_inout) return fail(c, CLAIRE_EINVAL, "null v_inout");
    if (!c->have_images) return fail(c, CLAIRE_ESTATE, "images not set (claire_set_images)");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t N = c->N, n3 = 3 * N;
    claire_report R;
    std::memset(&R, 0, sizeof(R));
    collect_timing(c);
    KernelStat ks0[KK_COUNT];
    for (int k = 0; k < KK_COUNT; ++k) ks0[k] = c->ks[k];
    double ph0[8];
    for (int i = 0; i < 8; ++i) ph0[i] = c->phase_s[i];
    const long long pc_inner0 = c->pc_inner_total;

    CL_CUDA(c, cudaMemcpyAsync(c->v, v_inout, n3 * sizeof(float), cudaMemcpyDefault, c->stream));
    CL_TRY(screen_velocity(c, c->v));
    // the iterate's spectrum: one transform of the initial guess, then updated
    // with the PCG solution's spectrum at every accepted step
    c->vh_on = false;
    if (c->o.spectral_iterate) {
        if (!c->vh) {
            if (cudaMalloc(&c->vh, 3 * c->M * sizeof(cufftComplex)) != cudaSuccess) {
                cudaGetLastError();
                c->vh = nullptr;
                return fail(c, CLAIRE_ENOMEM,
                            "spectrum of the iterate (%zu bytes; spectral_iterate = 0 does without it)",
                            3 * c->M * sizeof(cufftComplex));
            }
        }
        {
            KTimer t(c, KK_FFT, 0, 0);
            CL_FFT(c, cufftExecR2C(c->r2c, c->v, c->vh));
        }
        launch_cscale(c->vh, 3 * c->M, static_cast<float>(1.0 / c->N), c->stream);
        CL_LAUNCHED(c);
        c->vh_on = true;
    }
    struct VhOff {
        claire_ctx* c;
        ~VhOff() { c->vh_on = false; }
    } vh_off{c};
    claire_status st = CLAIRE_ENOTCONVERGED;
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    CL_TRY(linearise(c, c->v));
    CL_TRY(gradient_at_lin(c, c->g));
    double gn;
    CL_TRY(dot(c, c->g, c->g, n3, &gn));
    // the tolerance and the PCG forcing are relative to g0_ref when given
    // (a warm start stops at the same absolute gradient as a solve from zero)
    const double g0 = c->o.g0_ref > 0 ? c->o.g0_ref : std::sqrt(gn);
    double rel = 1.0;
    if (g0 == 0.0) st = CLAIRE_OK;
    for (int k = 0; st == CLAIRE_ENOTCONVERGED && k < c->o.max_gn; ++k) {
        CL_TRY(dot(c, c->g, c->g, n3, &gn));
        rel = std::sqrt(gn) / g0;
        if (rel <= c->o.gtol) {
            st = CLAIRE_OK;
            break;
        }
        if (c->o.wall_limit_s > 0 && elapsed() > c->o.wall_limit_s) {
            st = CLAIRE_ETIMEOUT;
            break;
        }
        const double eta = std::min(c->o.pcg_rtol_max, std::sqrt(rel));
        double alpha = 1.0;
        bool ok = false;
        // a step whose two-level solve fails the line search is solved again with
        // the spectral preconditioner (once per step)
        for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
            const bool spectral_retry = attempt == 1;
            if (spectral_retry) {
                if (c->o.precond != CLAIRE_PRECOND_TWO_LEVEL) break;
                ++R.pc_fallbacks;
                // the trials overwrote the state characteristic and states: linearise again at v
                CL_TRY(linearise(c, c->v));
                CL_TRY(gradient_at_lin(c, c->g));
                c->o.precond = CLAIRE_PRECOND_SPECTRAL;
            }
            int its = 0;
            const claire_status ps = pcg(c, eta, &its);
            if (spectral_retry) c->o.precond = CLAIRE_PRECOND_TWO_LEVEL;
            CL_TRY(ps);
            if (k < CLAIRE_MAX_LOGGED_STEPS) R.pcg_iters[k] += its;
            R.pcg_iters_total += its;
            double gtx;
            CL_TRY(dot(c, c->g, c->x, n3, &gtx));
            alpha = 1.0;
            for (int ls = 0; ls < c->o.max_ls; ++ls) {
                {
                    PhaseScope pv(c, CLAIRE_PHASE_VECTOR);
                    KTimer t(c, KK_VECTOR, 12.0 * n3, 0);
                    launch_xpay(c->v, static_cast<float>(alpha), c->x, c->p, n3, c->stream);
                    CL_LAUNCHED(c);
                }
                double Jt;
                CL_TRY(objective_at(c, c->p, &Jt, nullptr, true));
                if (Jt <= c->J_lin + c->o.armijo_c1 * alpha * gtx) {
                    ok = true;
                    break;
                }
                alpha *= 0.5;
            }
        }
        if (!ok) {
            st = CLAIRE_ELINESEARCH;
            break;
        }
        if (k < CLAIRE_MAX_LOGGED_STEPS) R.alpha[k] = alpha;
        {
            PhaseScope ps(c, CLAIRE_PHASE_VECTOR);
            KTimer t(c, KK_VECTOR, 12.0 * n3, 0);
            launch_axpy(static_cast<float>(alpha), c->x, c->v, n3, c->stream);
            CL_LAUNCHED(c);
        }
        if (c->vh_on) {
            // vh += alpha xh (xh: the spectrum of the PCG solution x, same scaling)
            PhaseScope ps(c, CLAIRE_PHASE_VECTOR);
            KTimer t(c, KK_VECTOR, 24.0 * c->M * 3, 0);
            launch_axpy(static_cast<float>(alpha), reinterpret_cast<const float*>(c->xh),
                        reinterpret_cast<float*>(c->vh), 6 * c->M, c->stream);
            CL_LAUNCHED(c);
        }
        R.gn_iters = k + 1;
        CL_TRY(linearise(c, c->v, true));  // c->v equals the accepted trial c->p bit for bit
        CL_TRY(gradient_at_lin(c, c->g));
        CL_TRY(dot(c, c->g, c->g, n3, &gn));
        rel = std::sqrt(gn) / g0;
        if (rel <= c->o.gtol) st = CLAIRE_OK;
    }
    R.gnorm_rel = rel;
    R.pc_inner_iters_total = static_cast<int>(c->pc_inner_total - pc_inner0);
    R.J = c->J_lin;
    R.mismatch = c->mis_lin;
    {
        double den;
        {
            KTimer t(c, KK_REDUCE, 8.0 * N, 0, 2);
            launch_sqdiff_partial(c->m0, c->m1, N, c->partials, c->red_blocks, c->sto, c->stream);
            launch_final_sum(c->partials, c->red_blocks, 0.5 * c->hvol, c->dres + 2, c->stream);
            CL_LAUNCHED(c);
        }
        CL_CUDA(c, cudaMemcpyAsync(c->hres + 2, c->dres + 2, sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
        CL_CUDA(c, cudaStreamSynchronize(c->stream));
        den = c->hres[2];
        R.r = den > 0 ? c->mis_lin / den : 0.0;
    }
    CL_TRY(detj_of(c, c->v, &R.detj_min, &R.detj_max));
    CL_TRY(cfl_of(c, c->v, &R.cfl));
    CL_CUDA(c, cudaMemcpyAsync(v_inout, c->v, n3 * sizeof(float), cudaMemcpyDefault, c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->o.timing >= 2 || c->pending.size() > 200000) collect_timing(c);
    R.status = st;
    R.t_total_s = elapsed();
    for (int i = 0; i < 8; ++i) R.t_phase_s[i] = c->phase_s[i] - ph0[i];
    const int gk[] = {KK_INTERP, KK_BACKTRACE, KK_ADJ_STEP, KK_INC_STEP, KK_INC_LAST, KK_MAP};
    for (int k : gk) {
        R.gather_launches += c->ks[k].launches - ks0[k].launches;
        R.interp_points += c->ks[k].points - ks0[k].points;
        R.interp_bytes += c->ks[k].bytes - ks0[k].bytes;
    }
    if (rep) *rep = R;
    if (st == CLAIRE_ELINESEARCH) return fail(c, st, "Armijo line search failed");
    if (st == CLAIRE_ETIMEOUT) return fail(c, st, "wall-clock limit reached");
    return st;
}

claire_status claire_transport(claire_ctx* c, const float* v, const float* m_in, float* m_out,
                               int flags)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!v || !m_in || !m_out) return fail(c, CLAIRE_EINVAL, "null argument");
    if (flags != CLAIRE_TRANSPORT_FWD && flags != CLAIRE_TRANSPORT_ADJ)
        return fail(c, CLAIRE_EINVAL, "unknown transport flags %d", flags);
    const size_t N = c->N;
    const float* dv = nullptr;
    CL_TRY(device_input(c, v, 3 * N, c->p, &dv));
    CL_TRY(screen_velocity(c, dv));
    // the user-facing transport runs in FP32 whatever the context's storage
    const float* src;
    CL_TRY(device_input(c, m_in, N, reinterpret_cast<float*>(c->l0), &src));
    float* a = reinterpret_cast<float*>(c->l1);
    float* b = reinterpret_cast<float*>(c->l0);
    if (flags == CLAIRE_TRANSPORT_FWD) {
        CL_TRY(backtrace(c, dv, c->z, +1));
        for (int j = 0; j < c->nt; ++j) {
            CL_TRY(interp(c, src, c->z, a, Storage::F32));
            src = a;
            std::swap(a, b);
        }
    } else {
        float* divv = c->r;
        float* divXp = c->r + N;
        CL_TRY(characteristics(c, dv, nullptr, c->z, divv, divXp, Storage::F32));
        for (int j = 0; j < c->nt; ++j) {
            const void* gs;
            CL_TRY(gather_src(c, src, 1, &gs));
            KTimer t(c, KK_ADJ_STEP, 28.0 * N, 1.0 * N);
            launch_adj_step(c->grid, c->o.interp, gs, c->z, divv, divXp, static_cast<float>(c->dt), a,
                            Storage::F32, c->stream);
            CL_LAUNCHED(c);
            src = a;
            std::swap(a, b);
        }
    }
    CL_TRY(sync_scalars(c, 0));
    CL_TRY(copy_out(c, m_out, src, N));
    collect_timing(c);
    return CLAIRE_OK;
}

namespace {

// out = W(x + disp)^T yv (replacing, or added to out), times mult; disp = d or predictor of v.
claire_status scatter_transpose(claire_ctx* c, const float* yv, const float* d, const float* v, float* out,
                                bool accumulate, float mult)
{
    // the fixed-point scale follows max |yv|, computed on the device (no host round trip)
    double* mx = c->dres + 8;
    launch_maxabs(yv, c->N, c->partials, c->red_blocks, mx, c->stream);
    CL_LAUNCHED(c);
    {
        KTimer t(c, KK_VJP_SCATTER, (4.0 + 12.0) * c->N, 1.0 * c->N);
        launch_scatter_fixed(c->grid, c->o.interp, yv, d, v, static_cast<float>(c->dt), mx + 1, c->vjp_acc,
                             c->stream);
        CL_LAUNCHED(c);
    }
    launch_fixed_to_float(c->vjp_acc, mx + 1, accumulate ? 1 : 0, mult, out, c->N, c->stream);
    CL_LAUNCHED(c);
    return CLAIRE_OK;
}

}  // namespace

extern "C" claire_status claire_transport_vjp(claire_ctx* c, const float* v, const float* m0,
                                              const float* gbar, float* gm0, float* gv, int flags)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!v || !m0 || !gbar) return fail(c, CLAIRE_EINVAL, "null argument");
    if (flags & ~CLAIRE_VJP_RECOMPUTE) return fail(c, CLAIRE_EINVAL, "unknown flags %d", flags);
    const size_t N = c->N;
    const int nt = c->nt;
    const bool recompute = (flags & CLAIRE_VJP_RECOMPUTE) != 0;
    if (!c->vjp_acc) {
        CL_CUDA(c, cudaMalloc(&c->vjp_acc, N * sizeof(unsigned long long)));
        CL_CUDA(c, cudaMemsetAsync(c->vjp_acc, 0, N * sizeof(unsigned long long), c->stream));
    }
    const size_t nstates = (recompute ? 2 : nt + 1) * N;
    if (c->vjp_states_n < nstates) {
        if (c->vjp_states) CL_CUDA(c, cudaFree(c->vjp_states));
        c->vjp_states = nullptr;
        c->vjp_states_n = 0;
        CL_CUDA(c, cudaMalloc(&c->vjp_states, nstates * sizeof(float)));
        c->vjp_states_n = nstates;
    }
    c->have_lin = false;  // the work vectors below are shared with the solver
    // FP32 inputs on the device: v -> g, m0 -> states[0], gbar -> r (first N)
    const float* dv = nullptr;
    CL_TRY(device_input(c, v, 3 * N, c->g, &dv));
    CL_TRY(screen_velocity(c, dv));
    CL_CUDA(c, cudaMemcpyAsync(c->vjp_states, m0, N * sizeof(float), cudaMemcpyDefault, c->stream));
    float* d = c->z;                 // characteristic X (grid units)
    float* dbar = c->x;              // cotangent of the displacement
    float* mb = c->r;                // cotangent of the state, two rolling halves
    float* mb2 = c->r + N;
    CL_CUDA(c, cudaMemcpyAsync(mb, gbar, N * sizeof(float), cudaMemcpyDefault, c->stream));
    CL_CUDA(c, cudaMemsetAsync(dbar, 0, 3 * N * sizeof(float), c->stream));
    CL_TRY(backtrace(c, dv, d, +1));
    float* S = c->vjp_states;
    // states m^1..m^{nt} (all stored), or rolling recomputation from m^0
    if (!recompute)
        for (int j = 0; j < nt; ++j) CL_TRY(interp(c, S + j * N, d, S + (j + 1) * N, Storage::F32));
    for (int j = nt - 1; j >= 0; --j) {
        const float* mj = S + j * N;
        if (recompute && j > 0) {
            // checkpointing: rebuild m^j from m^0 in the second slot
            float* a = S + N;
            CL_TRY(interp(c, S, d, a, Storage::F32));
            for (int q = 1; q < j; ++q) {
                CL_TRY(interp(c, a, d, c->p, Storage::F32));
                CL_CUDA(c, cudaMemcpyAsync(a, c->p, N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
            }
            mj = a;
        }
        // cubic B-splines: the interpolant is that of the state's coefficients
        const float* mjc = mj;
        if (c->o.interp == 4) CL_TRY(bspline_coef(c, mj, 1, &mjc));
        {
            KTimer t(c, KK_VJP_GRAD, 32.0 * N, 1.0 * N);
            launch_grad_accum(c->grid, c->o.interp, mjc, d, mb, dbar, c->stream);
            CL_LAUNCHED(c);
        }
        CL_TRY(scatter_transpose(c, mb, d, nullptr, mb2, false, 1.0f));
        if (c->o.interp == 4) {
            // the transpose of "prefilter, then interpolate": scatter, then the
            // prefilter again (its symbol is real and even, so it is symmetric)
            const float* coef;
            CL_TRY(bspline_coef(c, mb2, 1, &coef));
            CL_CUDA(c, cudaMemcpyAsync(mb2, coef, N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        }
        std::swap(mb, mb2);
    }
    if (gm0) CL_TRY(copy_out(c, gm0, mb, N));
    if (gv) {
        float* ub = c->p;
        float* Ub = reinterpret_cast<float*>(c->spec);  // 6 M >= 3 N floats, unused here
        const void* vsrc;
        CL_TRY(gather_src(c, dv, 3, &vsrc));  // v, or its B-spline coefficients
        {
            KTimer t(c, KK_VJP_GRAD, 48.0 * N, 3.0 * N);
            launch_predictor_terms(c->grid, c->o.interp, dv, static_cast<const float*>(vsrc),
                                   static_cast<float>(c->dt), dbar, ub, Ub, c->stream);
            CL_LAUNCHED(c);
        }
        const float ih[3] = {c->grid.ih1, c->grid.ih2, c->grid.ih3};
        for (int comp = 0; comp < 3; ++comp) {
            if (c->o.interp != 4) {
                CL_TRY(scatter_transpose(c, Ub + comp * N, nullptr, dv, ub + comp * N, true, ih[comp]));
                continue;
            }
            // B-splines: scatter into the free half of the state cotangent, prefilter,
            // then ub = ih (ub + that), the conversion the accumulating scatter does
            float* tmp = (mb == c->r) ? c->r + N : c->r;
            CL_TRY(scatter_transpose(c, Ub + comp * N, nullptr, dv, tmp, false, 1.0f));
            const float* coef;
            CL_TRY(bspline_coef(c, tmp, 1, &coef));
            {
                KTimer t(c, KK_VECTOR, 12.0 * N, 0);
                launch_scale_add(ub + comp * N, ih[comp], coef, N, c->stream);
                CL_LAUNCHED(c);
            }
        }
        CL_TRY(copy_out(c, gv, ub, 3 * N));
    }
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_detj(claire_ctx* c, const float* v, double* lo, double* hi)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!v || !lo || !hi) return fail(c, CLAIRE_EINVAL, "null argument");
    const float* dv = nullptr;
    CL_TRY(device_input(c, v, 3 * c->N, c->x, &dv));
    CL_TRY(screen_velocity(c, dv));
    CL_TRY(detj_of(c, dv, lo, hi));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_interp(claire_ctx* c, const float* f, const float* d, float* out, int order)
{
    if (!c) return CLAIRE_EINVAL;
    if (order != 1 && order != 3 && order != 4) return fail(c, CLAIRE_EINVAL, "order must be 1, 3 or 4");
    CL_TRY(check_kernel_ptr(c, f));
    CL_TRY(check_kernel_ptr(c, d));
    CL_TRY(check_kernel_ptr(c, out));
    if (order == 4) CL_TRY(bspline_coef(c, f, 1, &f));
    {
        KTimer t(c, KK_INTERP, 20.0 * c->N, 1.0 * c->N);
        launch_interp(c->grid, order, f, d, out, Storage::F32, c->stream);
        CL_LAUNCHED(c);
    }
    CL_TRY(sync_scalars(c, 0));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_interp_fields(claire_ctx* c, const float* f, int nf, const float* d, float* out, int order)
{
    if (!c) return CLAIRE_EINVAL;
    if (order != 1 && order != 3) return fail(c, CLAIRE_EINVAL, "order must be 1 or 3");
    if (nf < 1) return fail(c, CLAIRE_EINVAL, "nf must be >= 1");
    CL_TRY(check_kernel_ptr(c, f));
    CL_TRY(check_kernel_ptr(c, d));
    CL_TRY(check_kernel_ptr(c, out));
    {
        KTimer t(c, KK_INTERP, (8.0 * nf + 12.0) * c->N, 1.0 * nf * c->N);
        launch_interp_fields(c->grid, order, f, nf, d, out, c->stream);
        CL_LAUNCHED(c);
    }
    CL_TRY(sync_scalars(c, 0));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_dice(claire_ctx* c, const float* a, const float* b, size_t n, double* dice)
{
    if (!c) return CLAIRE_EINVAL;
    if (!dice) return fail(c, CLAIRE_EINVAL, "null output");
    CL_TRY(check_kernel_ptr(c, a));
    CL_TRY(check_kernel_ptr(c, b));
    {
        KTimer t(c, KK_REDUCE, 8.0 * n, 0, 4);
        launch_count_partial(a, b, n, 0.5f, 0, c->partials, c->partials + c->red_blocks, c->red_blocks, c->stream);
        launch_final_sum(c->partials, c->red_blocks, 1.0, c->dres + 10, c->stream);
        launch_final_sum(c->partials + c->red_blocks, c->red_blocks, 1.0, c->dres + 11, c->stream);
        launch_count_partial(a, b, n, 0.5f, 1, c->partials, c->partials + c->red_blocks, c->red_blocks, c->stream);
        launch_final_sum(c->partials, c->red_blocks, 1.0, c->dres + 12, c->stream);
        CL_LAUNCHED(c);
    }
    CL_CUDA(c, cudaMemcpyAsync(c->hres + 10, c->dres + 10, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    const double na = c->hres[10], nb = c->hres[11], nab = c->hres[12];
    *dice = (na + nb) > 0 ? 2.0 * nab / (na + nb) : 1.0;
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_gather_fallback_tiles(unsigned long long* count, int reset)
{
    if (!count) return CLAIRE_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess || gather_fallback_tiles(count, reset != 0) != cudaSuccess) {
        cudaGetLastError();
        return CLAIRE_ECUDA;
    }
    return CLAIRE_OK;
}

claire_status claire_backtrace(claire_ctx* c, const float* v, float* d, int direction)
{
    if (!c) return CLAIRE_EINVAL;
    if (direction != 1 && direction != -1) return fail(c, CLAIRE_EINVAL, "direction must be +1 or -1");
    CL_TRY(check_kernel_ptr(c, v));
    CL_TRY(check_kernel_ptr(c, d));
    CL_TRY(screen_velocity(c, v));
    CL_TRY(backtrace(c, v, d, direction));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_fd8_grad(claire_ctx* c, const float* f, float* g)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(check_kernel_ptr(c, f));
    CL_TRY(check_kernel_ptr(c, g));
    CL_TRY(fd8_grad(c, f, g, Storage::F32));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    return CLAIRE_OK;
}

claire_status claire_fd8_div(claire_ctx* c, const float* v, float* dv)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(check_kernel_ptr(c, v));
    CL_TRY(check_kernel_ptr(c, dv));
    {
        KTimer t(c, KK_FD8, 16.0 * c->N, 0);
        launch_fd8_div(c->grid, v, dv, Storage::F32, c->stream);
        CL_LAUNCHED(c);
    }
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    return CLAIRE_OK;
}

claire_status claire_spectral(claire_ctx* c, const float* in, float* out, int op)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (op < CLAIRE_SPECTRAL_REG || op > CLAIRE_SPECTRAL_K) return fail(c, CLAIRE_EINVAL, "bad op");
    CL_TRY(check_kernel_ptr(c, in));
    CL_TRY(check_kernel_ptr(c, out));
    CL_TRY(spectral(c, in, out, static_cast<SpectralOp>(op)));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_mean_state_gradient(claire_ctx* c, float* gbar)
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    CL_TRY(check_kernel_ptr(c, gbar));
    CL_TRY(mean_state_gradient(c, gbar));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_set_pc_weight(claire_ctx* c, const float* w, const int wgrid[3])
{
    if (!c) return CLAIRE_EINVAL;
    CL_TRY(need_workspace(c));
    if (!w) {
        c->pcw_on = false;
        return CLAIRE_OK;
    }
    if (!wgrid) return fail(c, CLAIRE_EINVAL, "null weight grid");
    const int f = c->o.pc_coarse;
    for (int a = 0; a < 3; ++a)
        if (wgrid[a] < 1 || static_cast<long long>(wgrid[a]) * f != c->n[a])
            return fail(c, CLAIRE_EINVAL, "weight grid %d x %d x %d is not the coarse grid (grid / %d)", wgrid[0],
                        wgrid[1], wgrid[2], f);
    const size_t nc = static_cast<size_t>(wgrid[0]) * wgrid[1] * wgrid[2];
    c->pcw_on = false;
    if (c->pcw && c->pcw_n != nc) {
        cudaFree(c->pcw);
        c->pcw = nullptr;
    }
    if (!c->pcw) {
        if (cudaMalloc(&c->pcw, nc * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            c->pcw = nullptr;
            return fail(c, CLAIRE_ENOMEM, "preconditioner weight (%zu floats)", nc);
        }
        c->pcw_n = nc;
    }
    CL_CUDA(c, cudaMemcpyAsync(c->pcw, w, nc * sizeof(float), cudaMemcpyDefault, c->stream));
    double ss = 0.0;
    CL_TRY(dot(c, c->pcw, c->pcw, nc, &ss));
    if (!std::isfinite(ss)) return fail(c, CLAIRE_ENONFINITE, "non-finite preconditioner weight");
    for (int a = 0; a < 3; ++a) c->pcw_grid[a] = wgrid[a];
    c->pcw_on = true;
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_dot(claire_ctx* c, const float* x, const float* y, size_t n, double* out)
{
    if (!c) return CLAIRE_EINVAL;
    if (!out) return fail(c, CLAIRE_EINVAL, "null output");
    if (n == 0) {
        *out = 0.0;
        return CLAIRE_OK;
    }
    CL_TRY(check_kernel_ptr(c, x));
    CL_TRY(check_kernel_ptr(c, y));
    CL_TRY(dot(c, x, y, n, out));
    collect_timing(c);
    return CLAIRE_OK;
}

claire_status claire_kernel_stats(claire_ctx* c, claire_kernel_stat* out, int capacity, int* count,
                                  int reset)
{
    if (!c || capacity < 0 || (capacity > 0 && !out)) return CLAIRE_EINVAL;
    collect_timing(c);
    int n = 0;
    for (int k = 0; k < KK_COUNT && n < capacity; ++k, ++n) {
        std::memset(out[n].name, 0, sizeof(out[n].name));
        std::strncpy(out[n].name, kKernelNames[k], sizeof(out[n].name) - 1);
        out[n].launches = c->ks[k].launches;
        out[n].seconds = c->ks[k].seconds;
        out[n].bytes = c->ks[k].bytes;
        out[n].points = c->ks[k].points;
    }
    if (count) *count = KK_COUNT;
    if (reset) {
        for (int k = 0; k < KK_COUNT; ++k) c->ks[k] = KernelStat();
        std::fill(c->phase_s, c->phase_s + 8, 0.0);
    }
    return CLAIRE_OK;
}

claire_status claire_set_timing(claire_ctx* c, int on)
{
    if (!c) return CLAIRE_EINVAL;
    collect_timing(c);
    c->o.timing = on ? 1 : 0;
    return CLAIRE_OK;
}

claire_status claire_set_opts(claire_ctx* c, const claire_opts* opts)
{
    if (!c || !opts) return CLAIRE_EINVAL;
    if (!valid_opts(*opts)) return fail(c, CLAIRE_EINVAL, "invalid options");
    if (opts->storage != c->o.storage || opts->lowmem != c->o.lowmem)
        return fail(c, CLAIRE_EINVAL, "storage and lowmem are fixed at claire_create");
    if (opts->precond == CLAIRE_PRECOND_TWO_LEVEL && !valid_coarse(c->n, opts->pc_coarse))
        return fail(c, CLAIRE_EINVAL, "pc_coarse %d: every grid size / pc_coarse must be even and >= 4",
                    opts->pc_coarse);
    collect_timing(c);
    c->o = *opts;
    c->rp.beta_w = static_cast<float>(opts->beta_w);
    c->rp.reg = opts->reg;
    c->have_lin = false;  // the linearisation point depends on interp / reg / beta_w / grad_form
    return CLAIRE_OK;
}

claire_status claire_set_beta(claire_ctx* c, double beta_v, double beta_w)
{
    if (!c) return CLAIRE_EINVAL;
    if (!(beta_v > 0) || !(beta_w >= 0)) return fail(c, CLAIRE_EINVAL, "beta_v must be > 0 and beta_w >= 0");
    c->beta_v = beta_v;
    c->rp.beta_v = static_cast<float>(beta_v);
    c->o.beta_w = beta_w;
    c->rp.beta_w = static_cast<float>(beta_w);
    c->have_lin = false;
    return CLAIRE_OK;
}

claire_status claire_get_beta(const claire_ctx* c, double* beta_v, double* beta_w)
{
    if (!c || !beta_v || !beta_w) return CLAIRE_EINVAL;
    *beta_v = c->beta_v;
    *beta_w = c->o.beta_w;
    return CLAIRE_OK;
}

claire_status claire_get_opts(const claire_ctx* c, claire_opts* opts)
{
    if (!c || !opts) return CLAIRE_EINVAL;
    *opts = c->o;
    return CLAIRE_OK;
}

const char* claire_last_error(const claire_ctx* c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

}  // extern "C"

namespace claire {
cudaStream_t ctx_stream(const claire_ctx* c) { return c->stream; }
size_t ctx_points(const claire_ctx* c) { return c->N; }
claire_status ctx_fail(claire_ctx* c, claire_status st, const char* msg) { return fail(c, st, "%s", msg); }
}  // namespace claire
