// claire_dot_noalloc: the FP64 inner product of claire_dot for callers that
// cannot allocate device memory.
//
// Who needs it: a caller whose device memory is entirely reserved by another
// allocator (for example a framework's caching allocator that leaves nothing
// for cudaMalloc), a latency-critical loop that cannot accept the implicit
// device-wide synchronisation of cudaMalloc / cudaFree, or code that holds
// no claire context (creating one allocates every workspace up front).  This
// entry point allocates nothing: its partial sums live in a fixed,
// file-scope device array that every GPU loading the library holds until
// the process exits (1 MiB + 256 B per device).
//
// The caller passes the inputs (device pointers) and the output.  Each
// call overwrites the partial-sum slots and the result slot it uses, so no
// state has to start at zero; but all calls on a device share the one array,
// so calls whose kernels overlap on the GPU (different streams, different
// host threads) race and must be serialised by the caller.
#include "claire.h"

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 32;                                  // elements per thread
constexpr size_t kChunk = static_cast<size_t>(kThreads) * kPerThread;  // elements per block
constexpr int kMaxPartials = 131072;                            // 1 MiB of doubles
constexpr size_t kMaxN = kChunk * kMaxPartials;                 // 2^30 elements
static_assert(kMaxN == (size_t(1) << 30), "documented maximum");

// partial sums [0, kMaxPartials) followed by the result slot
static __device__ __align__(256) double g_dot_scratch[kMaxPartials + 32];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Block b sums elements [b * kChunk, (b + 1) * kChunk) in a fixed order:
// FP32 products summed in groups of four, accumulated in FP64.
__global__ void __launch_bounds__(kThreads) k_dot_chunks(const float* __restrict__ x,
                                                          const float* __restrict__ y, size_t n,
                                                          double* __restrict__ partials)
{
    const size_t base = static_cast<size_t>(blockIdx.x) * kChunk;
    double acc = 0.0;
    for (int r = 0; r < kPerThread; r += 4) {
        float s = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t i = base + static_cast<size_t>(r + u) * kThreads + threadIdx.x;
            if (i < n) s += x[i] * y[i];
        }
        acc += static_cast<double>(s);
    }
    __shared__ double sh[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

// One block: result = scale * sum of partials[0, count), fixed order.
__global__ void __launch_bounds__(kThreads) k_dot_final(double* __restrict__ scratch, int count,
                                                         double scale)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += kThreads) acc += scratch[i];
    __shared__ double sh[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) scratch[kMaxPartials] = scale * v;
    }
}

// Device address of g_dot_scratch on the current device, looked up once per
// device (the host-side name of the array is only a stand-in).
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// True for device memory of GPU `dev` (the current device) and for managed
// memory; false for host memory and for device memory of another GPU, which
// the kernels, launched on the current device, might not be able to reach.
bool on_device(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" claire_status claire_dot_noalloc(const float* x, const float* y, size_t n, double scale,
                                            void* stream, double* out)
{
    if (!out) return CLAIRE_EINVAL;
    if (n > kMaxN) return CLAIRE_ETOOLARGE;
    if (n == 0) {
        *out = 0.0;
        return CLAIRE_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CLAIRE_ECUDA;
    }
    if (!x || !y || !on_device(x, dev) || !on_device(y, dev)) return CLAIRE_EINVAL;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return CLAIRE_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = static_cast<int>((n + kChunk - 1) / kChunk);
    k_dot_chunks<<<blocks, kThreads, 0, st>>>(x, y, n, scratch);
    k_dot_final<<<1, kThreads, 0, st>>>(scratch, blocks, scale);
    if (cudaGetLastError() != cudaSuccess) return CLAIRE_ECUDA;
    if (cudaMemcpyAsync(out, scratch + kMaxPartials, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CLAIRE_ECUDA;
    }
    return CLAIRE_OK;
}
