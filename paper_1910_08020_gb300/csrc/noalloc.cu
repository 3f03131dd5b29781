// Allocation-free variant of the sigma^z-type reduction (z2_zsums_static).
//
// Some callers cannot allocate device memory at all: code running inside a
// memory-capped or pre-partitioned process, plug-ins handed a fixed device
// arena, or drivers that must not call cudaMalloc after start-up.  For them
// this file provides one entry point that needs no context and allocates
// nothing: its scratch (per-block partial sums and the final sums) lives in a
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// The device address of that array is looked up once per device, the first
// time the entry point runs on it (cudaGetSymbolAddress with that device
// current); that first call should therefore come before any stream capture.
// The address is remembered together with the CUDA context it belongs to, and
// looked up again when the device's current context changes (after a
// cudaDeviceReset the library's module is loaded anew, at a new address).
// All calls share the one array: calls that overlap on the GPU (for example
// on two streams at once) race and give wrong sums.  Each call overwrites
// every slot it reads, so nothing has to be cleared between calls.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr int SA_THREADS = 256;
constexpr int SA_BLOCKS = 1024;  // partial sums per mask
constexpr int SA_MASKS = 32;     // masks per call
constexpr int SA_RUN = 16;       // amplitudes summed in the state's precision before the FP64 add
constexpr int SA_DEVICES = 64;

// partials [SA_BLOCKS][SA_MASKS] followed by the final sums [SA_MASKS]
static __device__ __align__(256) double g_scratch[SA_BLOCKS * SA_MASKS + SA_MASKS];

struct SMasks {
    uint64_t m[SA_MASKS];
};

template <typename C, typename real>
__global__ void __launch_bounds__(SA_THREADS) zsums_static_kernel(const C *__restrict__ psi, uint64_t per_block,
                                                                  const __grid_constant__ SMasks zm, int n_masks,
                                                                  double *__restrict__ partials) {
    double acc[SA_MASKS];
#pragma unroll
    for (int k = 0; k < SA_MASKS; ++k) acc[k] = 0;
    const uint64_t start = (uint64_t)blockIdx.x * per_block;
    const uint64_t steps = per_block / SA_THREADS;
    for (uint64_t r = 0; r < steps; r += SA_RUN) {
        real run[SA_MASKS];
#pragma unroll
        for (int k = 0; k < SA_MASKS; ++k) run[k] = 0;
        const uint64_t rend = r + SA_RUN < steps ? r + SA_RUN : steps;
        for (uint64_t e = r; e < rend; ++e) {
            const uint64_t i = start + e * SA_THREADS + threadIdx.x;
            const C v = psi[i];
            const real p = v.x * v.x + v.y * v.y;
#pragma unroll
            for (int k = 0; k < SA_MASKS; ++k)
                if (k < n_masks) run[k] += (__popcll(i & zm.m[k]) & 1) ? -p : p;
        }
#pragma unroll
        for (int k = 0; k < SA_MASKS; ++k) acc[k] += (double)run[k];
    }
    __shared__ double wsum[SA_THREADS / 32][SA_MASKS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < SA_MASKS; ++k) {
        if (k < n_masks) {
            double v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wsum[warp][k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)n_masks) {
        double s = 0;
        for (int w = 0; w < SA_THREADS / 32; ++w) s += wsum[w][threadIdx.x];
        partials[(size_t)blockIdx.x * SA_MASKS + threadIdx.x] = s;
    }
}

// out[k] = sum of the block partials of mask k, in a fixed order
__global__ void __launch_bounds__(SA_THREADS) zsums_static_finish(const double *__restrict__ partials, int n_blocks,
                                                                  double *__restrict__ out) {
    const int k = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < n_blocks; b += SA_THREADS) s += partials[(size_t)b * SA_MASKS + k];
    __shared__ double sh[SA_THREADS];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = SA_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

std::mutex g_setup_mu;
double *g_scratch_ptr[SA_DEVICES] = {};
CUcontext g_scratch_ctx[SA_DEVICES] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

// the driver's cuCtxGetCurrent, found through the runtime (no link to libcuda)
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

// device address of g_scratch on the current device: looked up once per device
// and context (a reset device gets a new context and a new address).  Without
// a current context, or without the driver's cuCtxGetCurrent, it is looked up
// on every call; the lookup makes the device's primary context current.
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= SA_DEVICES) return cudaErrorInvalidDevice;
    const CtxGetCurrentFn get = ctx_get_current();
    CUcontext cur = nullptr;
    if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev] || !cur || g_scratch_ctx[dev] != cur) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
        g_scratch_ptr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = cur;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int z2_zsums_static(int32_t n_qubits, int32_t precision, const void *state, const uint64_t *masks,
                               int32_t n_masks, double *out, void *stream) {
    using z2::set_thread_error;
    if (!state || !masks || !out) return set_thread_error(Z2_ERR_ARG, "z2_zsums_static: NULL argument");
    if (n_qubits < 8 || n_qubits > Z2_MAX_LINKS)
        return set_thread_error(Z2_ERR_ARG, "z2_zsums_static: n_qubits must be in 8..34");
    if (precision != Z2_C64 && precision != Z2_C128)
        return set_thread_error(Z2_ERR_ARG, "z2_zsums_static: bad precision");
    if (n_masks < 1 || n_masks > SA_MASKS)
        return set_thread_error(Z2_ERR_ARG, "z2_zsums_static: n_masks " + std::to_string(n_masks) +
                                                " is outside 1..32 (the size of its fixed scratch)");
    if (reinterpret_cast<uintptr_t>(state) % 256)
        return set_thread_error(Z2_ERR_ARG, "z2_zsums_static: state must be 256-byte aligned");
    double *scratch = nullptr;
    if (cudaError_t e = scratch_address(&scratch); e != cudaSuccess)
        return set_thread_error(Z2_ERR_CUDA, std::string("z2_zsums_static: cudaGetSymbolAddress: ") +
                                                 cudaGetErrorString(e));
    SMasks zm{};
    for (int k = 0; k < n_masks; ++k) zm.m[k] = masks[k];
    const uint64_t dim = 1ull << n_qubits;
    // at most SA_BLOCKS blocks, at least one amplitude per thread
    const int bits = n_qubits - 8 > 10 ? 10 : n_qubits - 8;
    const int blocks = 1 << bits;
    const uint64_t per_block = dim / blocks;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *partials = scratch, *sums = scratch + SA_BLOCKS * SA_MASKS;
    if (precision == Z2_C128)
        zsums_static_kernel<double2, double><<<blocks, SA_THREADS, 0, st>>>(static_cast<const double2 *>(state),
                                                                              per_block, zm, n_masks, partials);
    else
        zsums_static_kernel<float2, float><<<blocks, SA_THREADS, 0, st>>>(static_cast<const float2 *>(state),
                                                                            per_block, zm, n_masks, partials);
    if (cudaGetLastError() != cudaSuccess) return z2::set_thread_error(Z2_ERR_CUDA, "z2_zsums_static: launch failed");
    zsums_static_finish<<<n_masks, SA_THREADS, 0, st>>>(partials, blocks, sums);
    if (cudaGetLastError() != cudaSuccess) return z2::set_thread_error(Z2_ERR_CUDA, "z2_zsums_static: launch failed");
    if (cudaMemcpyAsync(out, sums, n_masks * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return z2::set_thread_error(Z2_ERR_CUDA, "z2_zsums_static: copy of the sums failed");
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return z2::set_thread_error(Z2_ERR_CUDA, "z2_zsums_static: stream synchronisation failed");
    return Z2_OK;
}
