// Grid transfer of periodic fields (Sec. 4, the downsampled-registration
// experiments): spectral restriction / prolongation (Fourier coefficients are
// copied between the two spectra, modes the target grid cannot hold are
// dropped, new modes are zero; cuFFT does the transforms, the coefficient
// copy and scaling is a hand-written kernel) and nearest-neighbour sampling.
#include "claire.h"
#include "internal.h"

#include <cufft.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

namespace claire {

namespace {

// Y[j1][j2][j3] (target half-spectrum m1 x m2 x (m3/2+1)) from X (source
// half-spectrum n1 x n2 x (n3/2+1)) scaled by s; a mode is kept when its
// signed wavenumber lies strictly inside both grids' Nyquist limits.
__global__ void k_copy_modes(const cufftComplex* __restrict__ X, int n1, int n2, int n3h, int n3,
                             cufftComplex* __restrict__ Y, int m1, int m2, int m3h, int m3, float s)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    const size_t total = static_cast<size_t>(m1) * m2 * m3h;
    if (e >= total) return;
    const int j3 = static_cast<int>(e % m3h);
    const int j2 = static_cast<int>((e / m3h) % m2);
    const int j1 = static_cast<int>(e / (static_cast<size_t>(m3h) * m2));
    const int k1 = j1 <= m1 / 2 ? j1 : j1 - m1;
    const int k2 = j2 <= m2 / 2 ? j2 : j2 - m2;
    const int k3 = j3;
    auto inside = [](int k, int n) { return 2 * (k < 0 ? -k : k) < n; };
    cufftComplex out = make_cuFloatComplex(0.f, 0.f);
    if (inside(k1, n1) && inside(k1, m1) && inside(k2, n2) && inside(k2, m2) && inside(k3, n3) &&
        inside(k3, m3)) {
        const int i1 = k1 < 0 ? k1 + n1 : k1, i2 = k2 < 0 ? k2 + n2 : k2;
        const cufftComplex x = X[(static_cast<size_t>(i1) * n2 + i2) * n3h + k3];
        out = make_cuFloatComplex(s * x.x, s * x.y);
    }
    Y[e] = out;
}

// out[j] = in[floor(j * n / m)] per axis (nearest-neighbour sampling)
__global__ void k_nearest(const float* __restrict__ in, int n1, int n2, int n3, float* __restrict__ out, int m1,
                          int m2, int m3)
{
    const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    const size_t total = static_cast<size_t>(m1) * m2 * m3;
    if (e >= total) return;
    const int j3 = static_cast<int>(e % m3);
    const int j2 = static_cast<int>((e / m3) % m2);
    const int j1 = static_cast<int>(e / (static_cast<size_t>(m3) * m2));
    const int i1 = static_cast<int>(static_cast<long long>(j1) * n1 / m1);
    const int i2 = static_cast<int>(static_cast<long long>(j2) * n2 / m2);
    const int i3 = static_cast<int>(static_cast<long long>(j3) * n3 / m3);
    out[e] = in[(static_cast<size_t>(i1) * n2 + i2) * n3 + i3];
}

// cuFFT plans and spectra of recently used grid pairs (per device), reused
// across calls; released by claire_resample_release.
struct PlanEntry {
    int device = 0;
    int from[3] = {0, 0, 0}, to[3] = {0, 0, 0};
    cufftHandle fwd = 0, inv = 0;
    cufftComplex* X = nullptr;
    cufftComplex* Y = nullptr;
};
constexpr size_t kMaxPlans = 4;
std::mutex g_plan_mu;
std::vector<PlanEntry> g_plans;

void destroy_entry(PlanEntry& e)
{
    if (e.fwd) cufftDestroy(e.fwd);
    if (e.inv) cufftDestroy(e.inv);
    if (e.X) cudaFree(e.X);
    if (e.Y) cudaFree(e.Y);
    e = PlanEntry{};
}

// Entry for (device, from, to); created on a miss (oldest evicted).  Caller holds g_plan_mu.
claire_status plan_for(const int from[3], const int to[3], PlanEntry** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CLAIRE_ECUDA;
    for (auto& e : g_plans)
        if (e.device == dev && e.from[0] == from[0] && e.from[1] == from[1] && e.from[2] == from[2] &&
            e.to[0] == to[0] && e.to[1] == to[1] && e.to[2] == to[2]) {
            *out = &e;
            return CLAIRE_OK;
        }
    if (g_plans.size() >= kMaxPlans) {
        destroy_entry(g_plans.front());
        g_plans.erase(g_plans.begin());
    }
    PlanEntry e;
    e.device = dev;
    for (int a = 0; a < 3; ++a) {
        e.from[a] = from[a];
        e.to[a] = to[a];
    }
    const size_t Min = static_cast<size_t>(from[0]) * from[1] * (from[2] / 2 + 1);
    const size_t Mout = static_cast<size_t>(to[0]) * to[1] * (to[2] / 2 + 1);
    if (cudaMalloc(&e.X, Min * sizeof(cufftComplex)) != cudaSuccess ||
        cudaMalloc(&e.Y, Mout * sizeof(cufftComplex)) != cudaSuccess) {
        cudaGetLastError();
        destroy_entry(e);
        return CLAIRE_ENOMEM;
    }
    if (cufftPlan3d(&e.fwd, from[0], from[1], from[2], CUFFT_R2C) != CUFFT_SUCCESS ||
        cufftPlan3d(&e.inv, to[0], to[1], to[2], CUFFT_C2R) != CUFFT_SUCCESS) {
        destroy_entry(e);
        return CLAIRE_ECUFFT;
    }
    g_plans.push_back(e);
    *out = &g_plans.back();
    return CLAIRE_OK;
}

}  // namespace

}  // namespace claire

extern "C" claire_status claire_resample_release(void)
{
    std::lock_guard<std::mutex> lock(claire::g_plan_mu);
    for (auto& e : claire::g_plans) claire::destroy_entry(e);
    claire::g_plans.clear();
    return CLAIRE_OK;
}

namespace {

// Device (or managed) memory at a 16-byte aligned address: the kernels and the
// transforms of this file read and write the arrays in place.
bool device_array(const void* p)
{
    if ((reinterpret_cast<uintptr_t>(p) & 15u) != 0) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" claire_status claire_resample(const float* in, const int from[3], float* out, const int to[3], int ncomp,
                                         int mode, void* stream)
{
    using namespace claire;
    if (!in || !out || !from || !to || ncomp < 1) return CLAIRE_EINVAL;
    if (!device_array(in) || !device_array(out)) return CLAIRE_EINVAL;
    if (mode != CLAIRE_RESAMPLE_SPECTRAL && mode != CLAIRE_RESAMPLE_NEAREST) return CLAIRE_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (from[a] < 2 || to[a] < 2 || from[a] % 2 || to[a] % 2) return CLAIRE_EINVAL;
    const size_t Nin = static_cast<size_t>(from[0]) * from[1] * from[2];
    const size_t Nout = static_cast<size_t>(to[0]) * to[1] * to[2];
    const int n3h = from[2] / 2 + 1, m3h = to[2] / 2 + 1;
    const size_t Mout = static_cast<size_t>(to[0]) * to[1] * m3h;
    if (Nin >= (1ull << 31) || Nout >= (1ull << 31)) return CLAIRE_ETOOLARGE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == CLAIRE_RESAMPLE_NEAREST) {
        for (int c = 0; c < ncomp; ++c)
            k_nearest<<<static_cast<unsigned>((Nout + 255) / 256), 256, 0, st>>>(
                in + c * Nin, from[0], from[1], from[2], out + c * Nout, to[0], to[1], to[2]);
        return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_plan_mu);
    PlanEntry* e = nullptr;
    const claire_status status = plan_for(from, to, &e);
    if (status != CLAIRE_OK) return status;
    if (cufftSetStream(e->fwd, st) != CUFFT_SUCCESS || cufftSetStream(e->inv, st) != CUFFT_SUCCESS)
        return CLAIRE_ECUFFT;
    const float s = static_cast<float>(1.0 / static_cast<double>(Nin));
    for (int c = 0; c < ncomp; ++c) {
        if (cufftExecR2C(e->fwd, const_cast<float*>(in) + c * Nin, e->X) != CUFFT_SUCCESS) return CLAIRE_ECUFFT;
        k_copy_modes<<<static_cast<unsigned>((Mout + 255) / 256), 256, 0, st>>>(
            e->X, from[0], from[1], n3h, from[2], e->Y, to[0], to[1], m3h, to[2], s);
        if (cudaGetLastError() != cudaSuccess) return CLAIRE_ECUDA;
        if (cufftExecC2R(e->inv, e->Y, out + c * Nout) != CUFFT_SUCCESS) return CLAIRE_ECUFFT;
    }
    // the cached spectra are reused by the next call (possibly on another stream)
    if (cudaStreamSynchronize(st) != cudaSuccess) return CLAIRE_ECUDA;
    return CLAIRE_OK;
}
