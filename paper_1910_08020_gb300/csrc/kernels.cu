// Kernels and their launchers: the fused pass (pass_kernel.cuh), |+>
// initialisation, the all-qubit sigma^x flip, and the FP64 reductions of
// Sec. 2.4 (sigma^z-type expectation values and state overlaps).
#include <algorithm>
#include <cstdio>

#include "pass_kernel.cuh"

static_assert(sizeof(z2::PassStep) == sizeof(z2::PassStepHost), "pass step layout");

namespace z2 {

cudaError_t launch_pass_c64(int tb, int op, void *psi, const PassArgs &a, const void *steps, int n_steps,
                            const void *tables, int fmt, int grid, cudaStream_t st);
cudaError_t launch_pass_c128(int tb, int op, void *psi, const PassArgs &a, const void *steps, int n_steps,
                             const void *tables, int fmt, int grid, cudaStream_t st);

cudaError_t launch_pass_steps(bool c128, int tb, int op, void *psi, const PassArgs &a, const void *steps,
                              int n_steps, const void *tables, int fmt, int grid, cudaStream_t st) {
    return c128 ? launch_pass_c128(tb, op, psi, a, steps, n_steps, tables, fmt, grid, st)
                : launch_pass_c64(tb, op, psi, a, steps, n_steps, tables, fmt, grid, st);
}

cudaError_t launch_pass_tma_c64(int tb, int op, const PassArgs &a, const void *tmap, const void *steps, int n_steps,
                                const void *tables, int *err, int grid, cudaStream_t st);
cudaError_t launch_pass_tma_c128(int tb, int op, const PassArgs &a, const void *tmap, const void *steps, int n_steps,
                                 const void *tables, int *err, int grid, cudaStream_t st);
int tma_smem_bytes_c64(int tb);
int tma_smem_bytes_c128(int tb);

cudaError_t launch_pass_tma(bool c128, int tb, int op, const PassArgs &a, const void *tmap, const void *steps,
                            int n_steps, const void *tables, int *err, int grid, cudaStream_t st) {
    return c128 ? launch_pass_tma_c128(tb, op, a, tmap, steps, n_steps, tables, err, grid, st)
                : launch_pass_tma_c64(tb, op, a, tmap, steps, n_steps, tables, err, grid, st);
}

int tma_tile_limit(bool c128) { return c128 ? 12 : 13; }
int tma_smem_bytes(bool c128, int tb) { return c128 ? tma_smem_bytes_c128(tb) : tma_smem_bytes_c64(tb); }

int pass_threads(bool c128, int tb) { return 1 << (tb - (c128 ? Cfg<double2>::R : Cfg<float2>::R)); }
size_t pass_smem(bool c128, int tb) {
    const int R = c128 ? Cfg<double2>::R : Cfg<float2>::R;
    return (c128 ? 16u : 8u) * ((size_t(1) << tb) + (size_t(1) << (tb - R)));
}

// ---------------------------------------------------------------------------
// |+>^N: every amplitude 2^{-N/2} (Sec. 2.3).
template <typename C>
__global__ void init_plus_kernel(C *__restrict__ psi, uint64_t dim, typename Cfg<C>::real a) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim; i += (uint64_t)gridDim.x * blockDim.x) {
        C v;
        v.x = a;
        v.y = 0;
        psi[i] = v;
    }
}

cudaError_t launch_init_plus(bool c128, void *state, int n, int grid, cudaStream_t st) {
    const uint64_t dim = 1ull << n;
    const int blocks = (int)std::min<uint64_t>((dim + 255) / 256, (uint64_t)grid);
    if (c128)
        init_plus_kernel<double2><<<blocks, 256, 0, st>>>((double2 *)state, dim, exp2(-0.5 * n));
    else
        init_plus_kernel<float2><<<blocks, 256, 0, st>>>((float2 *)state, dim, (float)exp2(-0.5 * n));
    return cudaGetLastError();
}

// psi[i] <-> psi[~i]: prod_l sigma^x_l.  It commutes with both layers (every
// plaquette has four links), so the whole-qubit quarter turns of the gate are
// collected here once per segment.
template <typename C>
__global__ void flip_all_kernel(C *__restrict__ psi, uint64_t dim) {
    const uint64_t half = dim >> 1, mask = dim - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < half; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = i ^ mask;
        C a = psi[i], b = psi[k];
        psi[i] = b;
        psi[k] = a;
    }
}

cudaError_t launch_flip_all(bool c128, void *state, int n, int grid, cudaStream_t st) {
    const uint64_t dim = 1ull << n;
    const int blocks = (int)std::min<uint64_t>((dim / 2 + 255) / 256, (uint64_t)grid);
    if (c128)
        flip_all_kernel<double2><<<blocks, 256, 0, st>>>((double2 *)state, dim);
    else
        flip_all_kernel<float2><<<blocks, 256, 0, st>>>((float2 *)state, dim);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reductions.  Each thread sums its amplitudes in the state's precision in
// short runs (RUN at a time, then into a running sum), a warp combines its 32
// lanes with shuffles, the block combines its warps in FP64 and writes one
// FP64 partial per block; a second kernel adds the partials in FP64 in a
// fixed order, so every result is bit-reproducible for a given launch shape.
constexpr int RED_THREADS = 256;
constexpr int ZMASKS = 32;  // masks per zsums launch
constexpr int RUN = 16;

struct ZMasks {
    uint64_t m[ZMASKS];
};

template <typename C>
__global__ void __launch_bounds__(RED_THREADS) zsums_kernel(const C *__restrict__ psi, uint64_t per_block,
                                                            const __grid_constant__ ZMasks zm, int n_masks,
                                                            double *__restrict__ partials) {
    using real = typename Cfg<C>::real;
    real acc[ZMASKS];
#pragma unroll
    for (int k = 0; k < ZMASKS; ++k) acc[k] = 0;
    const uint64_t start = (uint64_t)blockIdx.x * per_block;
    const uint64_t steps = per_block / RED_THREADS;
    for (uint64_t r = 0; r < steps; r += RUN) {
        real run[ZMASKS];
#pragma unroll
        for (int k = 0; k < ZMASKS; ++k) run[k] = 0;
        const uint64_t rend = r + RUN < steps ? r + RUN : steps;
        for (uint64_t e = r; e < rend; ++e) {
            const uint64_t i = start + e * RED_THREADS + threadIdx.x;
            const C v = psi[i];
            const real p = v.x * v.x + v.y * v.y;
#pragma unroll
            for (int k = 0; k < ZMASKS; ++k) {
                if (k < n_masks) {
                    const int par = __popcll(i & zm.m[k]) & 1;
                    run[k] += par ? -p : p;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < ZMASKS; ++k) acc[k] += run[k];
    }
    __shared__ double wsum[RED_THREADS / 32][ZMASKS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < ZMASKS; ++k) {
        if (k < n_masks) {
            real v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wsum[warp][k] = (double)v;
        }
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)n_masks) {
        double s = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += wsum[w][threadIdx.x];
        partials[(size_t)blockIdx.x * n_masks + threadIdx.x] = s;
    }
}

// out[k] = sum over blocks of partials[b][k], fixed order (one block per k)
__global__ void __launch_bounds__(RED_THREADS) finish_kernel(const double *__restrict__ partials, int n_blocks,
                                                             int n_out, double *__restrict__ out) {
    const int k = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < n_blocks; b += RED_THREADS) s += partials[(size_t)b * n_out + k];
    __shared__ double sh[RED_THREADS];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

int max_zsum_masks() { return ZMASKS; }

// Blocks of a reduction over 2^n amplitudes (n >= 8): about 64 amplitudes per
// thread for n <= 30 (short FP32 runs keep the rounding error of each
// per-thread sum near 2^-24 relative), at most 2^16 blocks (the size of the
// partials buffer).
int reduce_blocks(int n) {
    int bpb = n < 14 ? n : 14;
    if (n - 16 > bpb) bpb = n - 16;
    return 1 << (n - bpb);
}

cudaError_t launch_zsums(bool c128, const void *state, int n, const uint64_t *masks, int n_masks, double *partials,
                         double *d_out, cudaStream_t st) {
    if (n_masks < 1 || n_masks > ZMASKS) return cudaErrorInvalidValue;
    ZMasks zm{};
    for (int k = 0; k < n_masks; ++k) zm.m[k] = masks[k];
    const uint64_t dim = 1ull << n;
    if (n < 8) return cudaErrorInvalidValue;
    const int blocks = reduce_blocks(n);
    const uint64_t per_block = dim / blocks;
    if (c128)
        zsums_kernel<double2><<<blocks, RED_THREADS, 0, st>>>((const double2 *)state, per_block, zm, n_masks, partials);
    else
        zsums_kernel<float2><<<blocks, RED_THREADS, 0, st>>>((const float2 *)state, per_block, zm, n_masks, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_kernel<<<n_masks, RED_THREADS, 0, st>>>(partials, blocks, n_masks, d_out);
    return cudaGetLastError();
}

// Density of states (Sec. 3.3): out[k] = sum of |psi_i|^2 over the amplitudes
// in bin k, where the bin of index i is the number of masks m with
// popcount(i & m) odd (n_masks >= 1: plaquettes with U_p = -1, the Z density
// of states), or popcount(i) (n_masks == 0: links with sigma^x = -1 once the
// state is in the sigma^x basis, the X density of states).  Each thread adds
// FP64 weights into its own column of shared-memory bins (no atomics); the
// block then adds each bin's column in a fixed order, and finish_kernel adds
// the blocks' partials, so results are bit-reproducible for a given size.
constexpr int DOS_THREADS = 128;
constexpr int DOS_BINS = 36;        // >= 35 = 34 qubits + 1, >= 33 = 32 masks + 1
constexpr int DOS_MAX_BLOCKS = 1 << 15;  // DOS_BINS * blocks fits the partials buffer

template <typename C>
__global__ void __launch_bounds__(DOS_THREADS) dos_kernel(const C *__restrict__ psi, uint64_t per_block,
                                                          const __grid_constant__ ZMasks zm, int n_masks, int n_bins,
                                                          double *__restrict__ partials) {
    __shared__ double bins[DOS_BINS * DOS_THREADS];
    for (int k = 0; k < DOS_BINS; ++k) bins[k * DOS_THREADS + threadIdx.x] = 0.0;
    const uint64_t start = (uint64_t)blockIdx.x * per_block;
    for (uint64_t e = threadIdx.x; e < per_block; e += DOS_THREADS) {
        const uint64_t i = start + e;
        const C v = psi[i];
        const double re = (double)v.x, im = (double)v.y;
        int k = 0;
        if (n_masks == 0) {
            k = __popcll(i);
        } else {
#pragma unroll
            for (int q = 0; q < ZMASKS; ++q)
                if (q < n_masks) k += __popcll(i & zm.m[q]) & 1;
        }
        bins[k * DOS_THREADS + threadIdx.x] += re * re + im * im;
    }
    __syncthreads();
    if ((int)threadIdx.x < n_bins) {
        double s = 0;
        for (int t = 0; t < DOS_THREADS; ++t) s += bins[threadIdx.x * DOS_THREADS + t];
        partials[(size_t)blockIdx.x * n_bins + threadIdx.x] = s;
    }
}

cudaError_t launch_dos(bool c128, const void *state, int n, const uint64_t *masks, int n_masks, double *partials,
                       double *d_out, int *n_bins_out, cudaStream_t st) {
    if (n < 8 || n > 34 || n_masks < 0 || n_masks > ZMASKS) return cudaErrorInvalidValue;
    const int n_bins = (n_masks ? n_masks : n) + 1;
    if (n_bins > DOS_BINS) return cudaErrorInvalidValue;
    ZMasks zm{};
    for (int k = 0; k < n_masks; ++k) zm.m[k] = masks[k];
    const int blocks = reduce_blocks(n) < DOS_MAX_BLOCKS ? reduce_blocks(n) : DOS_MAX_BLOCKS;
    const uint64_t per_block = (1ull << n) / (uint64_t)blocks;
    if (c128)
        dos_kernel<double2><<<blocks, DOS_THREADS, 0, st>>>((const double2 *)state, per_block, zm, n_masks, n_bins,
                                                            partials);
    else
        dos_kernel<float2><<<blocks, DOS_THREADS, 0, st>>>((const float2 *)state, per_block, zm, n_masks, n_bins,
                                                           partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_kernel<<<n_bins, RED_THREADS, 0, st>>>(partials, blocks, n_bins, d_out);
    *n_bins_out = n_bins;
    return cudaGetLastError();
}

template <typename C>
__global__ void __launch_bounds__(RED_THREADS) overlap_kernel(const C *__restrict__ a, const C *__restrict__ b,
                                                              uint64_t per_block, double *__restrict__ partials) {
    using real = typename Cfg<C>::real;
    real sre = 0, sim = 0;
    const uint64_t start = (uint64_t)blockIdx.x * per_block;
    const uint64_t steps = per_block / RED_THREADS;
    for (uint64_t r = 0; r < steps; r += RUN) {
        real rre = 0, rim = 0;
        const uint64_t rend = r + RUN < steps ? r + RUN : steps;
        for (uint64_t e = r; e < rend; ++e) {
            const uint64_t i = start + e * RED_THREADS + threadIdx.x;
            const C x = a[i], y = b[i];
            // conj(x) * y
            rre += x.x * y.x + x.y * y.y;
            rim += x.x * y.y - x.y * y.x;
        }
        sre += rre;
        sim += rim;
    }
    __shared__ double wsum[RED_THREADS / 32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    if (lane == 0) {
        wsum[warp][0] = (double)sre;
        wsum[warp][1] = (double)sim;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += wsum[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 2 + threadIdx.x] = s;
    }
}

cudaError_t launch_overlap(bool c128, const void *a, const void *b, int n, double *partials, double *d_out,
                           cudaStream_t st) {
    const uint64_t dim = 1ull << n;
    if (n < 8) return cudaErrorInvalidValue;
    const int blocks = reduce_blocks(n);
    const uint64_t per_block = dim / blocks;
    if (c128)
        overlap_kernel<double2><<<blocks, RED_THREADS, 0, st>>>((const double2 *)a, (const double2 *)b, per_block,
                                                                partials);
    else
        overlap_kernel<float2><<<blocks, RED_THREADS, 0, st>>>((const float2 *)a, (const float2 *)b, per_block,
                                                               partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_kernel<<<2, RED_THREADS, 0, st>>>(partials, blocks, 2, d_out);
    return cudaGetLastError();
}

}  // namespace z2
