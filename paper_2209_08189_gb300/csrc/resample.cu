// Grid transfer of periodic fields (Sec. 4, the downsampled-registration
// experiments): spectral restriction / prolongation (Fourier coefficients are
// copied between the two spectra, modes the target grid cannot hold are
// dropped, new modes are zero; cuFFT does the transforms, the coefficient
// copy and scaling is a hand-written kernel) and nearest-neighbour sampling.
#include "claire.h"
#include "internal.h"

#include <cufft.h>

#include <cstdio>

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

}  // namespace

}  // namespace claire

extern "C" claire_status claire_resample(const float* in, const int from[3], float* out, const int to[3], int ncomp,
                                         int mode, void* stream)
{
    using namespace claire;
    if (!in || !out || !from || !to || ncomp < 1) return CLAIRE_EINVAL;
    if (mode != CLAIRE_RESAMPLE_SPECTRAL && mode != CLAIRE_RESAMPLE_NEAREST) return CLAIRE_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (from[a] < 2 || to[a] < 2 || from[a] % 2 || to[a] % 2) return CLAIRE_EINVAL;
    const size_t Nin = static_cast<size_t>(from[0]) * from[1] * from[2];
    const size_t Nout = static_cast<size_t>(to[0]) * to[1] * to[2];
    const int n3h = from[2] / 2 + 1, m3h = to[2] / 2 + 1;
    const size_t Min = static_cast<size_t>(from[0]) * from[1] * n3h;
    const size_t Mout = static_cast<size_t>(to[0]) * to[1] * m3h;
    if (Nin >= (1ull << 31) || Nout >= (1ull << 31)) return CLAIRE_ETOOLARGE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == CLAIRE_RESAMPLE_NEAREST) {
        for (int c = 0; c < ncomp; ++c)
            k_nearest<<<static_cast<unsigned>((Nout + 255) / 256), 256, 0, st>>>(
                in + c * Nin, from[0], from[1], from[2], out + c * Nout, to[0], to[1], to[2]);
        return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
    }
    cufftComplex* X = nullptr;
    cufftComplex* Y = nullptr;
    cufftHandle fwd = 0, inv = 0;
    claire_status status = CLAIRE_OK;
    if (cudaMalloc(&X, Min * sizeof(cufftComplex)) != cudaSuccess ||
        cudaMalloc(&Y, Mout * sizeof(cufftComplex)) != cudaSuccess) {
        status = CLAIRE_ENOMEM;
    } else if (cufftPlan3d(&fwd, from[0], from[1], from[2], CUFFT_R2C) != CUFFT_SUCCESS ||
               cufftPlan3d(&inv, to[0], to[1], to[2], CUFFT_C2R) != CUFFT_SUCCESS ||
               cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftSetStream(inv, st) != CUFFT_SUCCESS) {
        status = CLAIRE_ECUFFT;
    } else {
        const float s = static_cast<float>(1.0 / static_cast<double>(Nin));
        for (int c = 0; c < ncomp && status == CLAIRE_OK; ++c) {
            if (cufftExecR2C(fwd, const_cast<float*>(in) + c * Nin, X) != CUFFT_SUCCESS) {
                status = CLAIRE_ECUFFT;
                break;
            }
            k_copy_modes<<<static_cast<unsigned>((Mout + 255) / 256), 256, 0, st>>>(
                X, from[0], from[1], n3h, from[2], Y, to[0], to[1], m3h, to[2], s);
            if (cudaGetLastError() != cudaSuccess) {
                status = CLAIRE_ECUDA;
                break;
            }
            if (cufftExecC2R(inv, Y, out + c * Nout) != CUFFT_SUCCESS) status = CLAIRE_ECUFFT;
        }
        if (status == CLAIRE_OK && cudaStreamSynchronize(st) != cudaSuccess) status = CLAIRE_ECUDA;
    }
    if (fwd) cufftDestroy(fwd);
    if (inv) cufftDestroy(inv);
    if (X) cudaFree(X);
    if (Y) cudaFree(Y);
    return status;
}
