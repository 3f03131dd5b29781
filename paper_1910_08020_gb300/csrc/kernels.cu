// Kernels and their launchers: the fused pass (pass_kernel.cuh), |+>
// initialisation, the all-qubit sigma^x flip, and the FP64 reductions of
// Sec. 2.4 (sigma^z-type expectation values and state overlaps).
#include <algorithm>
#include <atomic>
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

// Every amplitude zero (the canvas of the projected start state).
template <typename C>
__global__ void zero_kernel(C *__restrict__ psi, uint64_t dim) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim; i += (uint64_t)gridDim.x * blockDim.x) {
        C v;
        v.x = 0;
        v.y = 0;
        psi[i] = v;
    }
}

// The uniform superposition over the coset c + span(b_0 .. b_{r-1}) of
// GF(2)^N: psi[c ^ (xor of b_i over the set bits i of k)] = amp for every
// k < 2^r.  With linearly independent b_i every k lands on its own index.
// A Hadamard layer turns the span of the plaquette masks into the projected
// state prod_p (1 + U_p)/2 |+>^N of Sec. 2.4, and the offset c = w_mu into
// its topological sector W_mu prod_p (1 + U_p)/2 |+>^N.
struct SpanBasis {
    uint64_t b[64];
};

template <typename C>
__global__ void span_scatter_kernel(C *__restrict__ psi, const __grid_constant__ SpanBasis B, int r, uint64_t c,
                                    typename Cfg<C>::real amp) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < (1ull << r);
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = c;
        for (int i = 0; i < r; ++i)
            if ((k >> i) & 1ull) v ^= B.b[i];
        C x;
        x.x = amp;
        x.y = 0;
        psi[v] = x;
    }
}

cudaError_t launch_span_state(bool c128, void *state, int n, const uint64_t *basis, int r, uint64_t offset, int grid,
                              cudaStream_t st) {
    if (r < 0 || r > 63 || r > n) return cudaErrorInvalidValue;
    SpanBasis B{};
    for (int i = 0; i < r; ++i) B.b[i] = basis[i];
    const uint64_t dim = 1ull << n, cnt = 1ull << r;
    const int zb = (int)std::min<uint64_t>((dim + 255) / 256, (uint64_t)grid);
    const int sb = (int)std::min<uint64_t>((cnt + 255) / 256, (uint64_t)grid);
    if (c128) {
        zero_kernel<double2><<<zb, 256, 0, st>>>((double2 *)state, dim);
        span_scatter_kernel<double2><<<sb, 256, 0, st>>>((double2 *)state, B, r, offset, exp2(-0.5 * r));
    } else {
        zero_kernel<float2><<<zb, 256, 0, st>>>((float2 *)state, dim);
        span_scatter_kernel<float2><<<sb, 256, 0, st>>>((float2 *)state, B, r, offset, (float)exp2(-0.5 * r));
    }
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
// Reductions.  The sigma^z-type expectation values of Sec. 2.4 are
// S_k = sum_i |psi_i|^2 (-1)^popcount(i & m_k): for every mask m_k, one
// coefficient of the Walsh-Hadamard transform of the probabilities.
//
// Large states (zsums_wht_kernel): a warp takes chunks of 2^10 amplitudes.
// Each lane holds 32 probabilities of the chunk (5 index bits in registers, 5
// bits across the lanes), Walsh-Hadamard transforms them in registers, and
// leaves the 32 coefficients in shared memory; lane k then forms mask k's
// coefficient of the chunk as a signed pairwise sum over the 32 lanes' entries
// (1 + 1 per mask, masks k and k + 32), applies the sign of the chunk's upper
// index bits, and adds it to an FP64 accumulator.  So each coefficient of a
// chunk is an FP32 pairwise sum of depth 10 (relative error at most
// 10 * 2^-24 of the chunk's probability), and everything above one chunk -
// across chunks, warps, blocks and the final sum - is FP64.  Per amplitude that
// is about 15 instructions instead of one 64-bit popcount per mask.
//
// Small states (zsums_kernel, fewer than 2^13 amplitudes) and overlaps: each
// thread sums runs of RUN amplitudes in the state's precision and adds each
// run into an FP64 accumulator; warps combine with FP64 shuffles, blocks in
// FP64, and a second kernel adds the block partials in FP64 in a fixed order.
// Every result is bit-reproducible for a given size and device.
constexpr int RED_THREADS = 256;
constexpr int ZMASKS = 32;   // masks per zsums_kernel launch
constexpr int ZW_MASKS = 64; // masks per zsums_wht_kernel launch (two per lane)
constexpr int RUN = 16;
constexpr int ZW_WARPS = RED_THREADS / 32;
constexpr int ZW_CB = 10;    // chunk: 2^10 amplitudes per warp
constexpr int ZW_LD = 33;    // shared-memory row of one lane's 32 coefficients (padded)
constexpr int ZW_MAX_BLOCKS = 2048;

struct ZMasks {
    uint64_t m[ZMASKS];
};
struct ZMasks64 {
    uint64_t m[ZW_MASKS];
};

template <typename C>
__global__ void __launch_bounds__(RED_THREADS) zsums_kernel(const C *__restrict__ psi, uint64_t per_block,
                                                            const __grid_constant__ ZMasks zm, int n_masks,
                                                            double *__restrict__ partials) {
    using real = typename Cfg<C>::real;
    double acc[ZMASKS];
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
        for (int k = 0; k < ZMASKS; ++k) acc[k] += (double)run[k];
    }
    __shared__ double wsum[RED_THREADS / 32][ZMASKS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < ZMASKS; ++k) {
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
        for (int w = 0; w < RED_THREADS / 32; ++w) s += wsum[w][threadIdx.x];
        partials[(size_t)blockIdx.x * n_masks + threadIdx.x] = s;
    }
}

// Index bits of a chunk: complex64 lanes load 16-byte (two-amplitude) vectors,
// so chunk offset o = (j & 1) | lane << 1 | (j >> 1) << 6 for register j;
// complex128: o = lane | j << 5.  u = the mask's register bits (coefficient
// index in registers), v = its lane bits.
template <bool C128>
__device__ __forceinline__ uint32_t zw_u(uint64_t m) {
    return C128 ? (uint32_t)(m >> 5) & 31u : ((uint32_t)m & 1u) | ((uint32_t)(m >> 6) & 15u) << 1;
}
template <bool C128>
__device__ __forceinline__ uint32_t zw_v(uint64_t m) {
    return C128 ? (uint32_t)m & 31u : (uint32_t)(m >> 1) & 31u;
}

// mask coefficient of one chunk: sum over lanes l of (-1)^popc(l & v) row_l[u],
// pairwise, then the sign of the chunk's upper bits
template <typename real>
__device__ __forceinline__ double zw_coeff(const real *sw, uint32_t u, uint32_t v, uint64_t hi_par) {
    real y[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) {
        const real w = sw[l * ZW_LD + u];
        y[l] = (__popc((uint32_t)l & v) & 1) ? -w : w;
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1)
#pragma unroll
        for (int i = 0; i < s; ++i) y[i] += y[i + s];
    const double r = (double)y[0];
    return (__popcll(hi_par) & 1) ? -r : r;
}

template <typename C>
__global__ void __launch_bounds__(RED_THREADS) zsums_wht_kernel(const C *__restrict__ psi, uint64_t n_chunks,
                                                                const __grid_constant__ ZMasks64 zm, int n_masks,
                                                                double *__restrict__ partials) {
    using real = typename Cfg<C>::real;
    constexpr bool C128 = sizeof(C) == 16;
    extern __shared__ __align__(16) unsigned char zw_smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    real *sw = reinterpret_cast<real *>(zw_smem) + warp * (32 * ZW_LD);
    const bool has0 = (int)lane < n_masks, has1 = (int)lane + 32 < n_masks;
    const uint64_t m0 = has0 ? zm.m[lane] : 0, m1 = has1 ? zm.m[lane + 32] : 0;
    const uint32_t u0 = zw_u<C128>(m0), v0 = zw_v<C128>(m0), u1 = zw_u<C128>(m1), v1 = zw_v<C128>(m1);
    double acc0 = 0, acc1 = 0;
    const uint64_t nw = (uint64_t)gridDim.x * ZW_WARPS;
    for (uint64_t ch = (uint64_t)blockIdx.x * ZW_WARPS + warp; ch < n_chunks; ch += nw) {
        const uint64_t base = ch << ZW_CB;
        real x[32];
        if constexpr (C128) {
            const C *p = psi + base + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const C v = p[32 * j];
                x[j] = v.x * v.x + v.y * v.y;
            }
        } else {
            const float4 *p = reinterpret_cast<const float4 *>(psi + base) + lane;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float4 v = p[32 * r];
                x[2 * r] = v.x * v.x + v.y * v.y;
                x[2 * r + 1] = v.z * v.z + v.w * v.w;
            }
        }
        // Walsh-Hadamard transform of the lane's 32 probabilities
#pragma unroll
        for (int b = 1; b < 32; b <<= 1)
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (!(j & b)) {
                    const real a = x[j], d = x[j | b];
                    x[j] = a + d;
                    x[j | b] = a - d;
                }
        __syncwarp();  // the previous chunk's rows have been read
#pragma unroll
        for (int u = 0; u < 32; ++u) sw[lane * ZW_LD + u] = x[u];
        __syncwarp();
        if (has0) acc0 += zw_coeff(sw, u0, v0, base & m0);
        if (has1) acc1 += zw_coeff(sw, u1, v1, base & m1);
    }
    __shared__ double wsum[ZW_WARPS][ZW_MASKS];
    wsum[warp][lane] = acc0;
    wsum[warp][lane + 32] = acc1;
    __syncthreads();
    if ((int)threadIdx.x < n_masks) {
        double s = 0;
        for (int w = 0; w < ZW_WARPS; ++w) s += wsum[w][threadIdx.x];
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

int max_zsum_masks() { return ZW_MASKS; }
int zsums_launches(int n, int n_masks) { return n >= ZW_CB + 3 ? 2 : 2 * ((n_masks + ZMASKS - 1) / ZMASKS); }

// Blocks of a run-based reduction over 2^n amplitudes (n >= 8): about 64
// amplitudes per thread for n <= 30, at most 2^16 blocks (the size of the
// partials buffer).
int reduce_blocks(int n) {
    int bpb = n < 14 ? n : 14;
    if (n - 16 > bpb) bpb = n - 16;
    return 1 << (n - bpb);
}

// Doubles of partial sums any reduction over 2^n amplitudes may write.
size_t reduce_partials_doubles(int n) {
    size_t d = (size_t)reduce_blocks(n) * ZMASKS;
    if (n >= ZW_CB + 3) {
        const size_t b = std::min<size_t>(size_t(1) << (n - ZW_CB - 3), ZW_MAX_BLOCKS);
        d = std::max(d, b * ZW_MASKS);
    }
    return d;
}

// Blocks of zsums_wht_kernel: every SM filled once (a grid-stride loop over
// the chunks), never more than one block per 8 chunks nor ZW_MAX_BLOCKS.
template <typename C>
static int zsums_wht_grid(uint64_t n_chunks, size_t smem) {
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    static int per_sm_cache[64] = {};
    static int sms_cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        if (cudaFuncSetAttribute(zsums_wht_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 0;
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zsums_wht_kernel<C>, RED_THREADS, smem) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        per_sm_cache[dev & 63] = per_sm < 1 ? 1 : per_sm;
        sms_cache[dev & 63] = sms;
        configured |= bit;
    }
    const uint64_t full = (uint64_t)per_sm_cache[dev & 63] * sms_cache[dev & 63];
    uint64_t most = n_chunks / ZW_WARPS < 1 ? 1 : n_chunks / ZW_WARPS;
    if (most > (uint64_t)ZW_MAX_BLOCKS) most = ZW_MAX_BLOCKS;
    return (int)(full < most ? full : most);
}

template <typename C>
static cudaError_t launch_zsums_t(const void *state, int n, const uint64_t *masks, int n_masks, double *partials,
                                  double *d_out, cudaStream_t st) {
    const uint64_t dim = 1ull << n;
    if (n >= ZW_CB + 3) {
        ZMasks64 zm{};
        for (int k = 0; k < n_masks; ++k) zm.m[k] = masks[k];
        const uint64_t n_chunks = dim >> ZW_CB;
        const size_t smem = sizeof(typename Cfg<C>::real) * ZW_WARPS * 32 * ZW_LD;
        const int blocks = zsums_wht_grid<C>(n_chunks, smem);
        if (blocks < 1) return cudaErrorInvalidConfiguration;
        zsums_wht_kernel<C><<<blocks, RED_THREADS, smem, st>>>((const C *)state, n_chunks, zm, n_masks, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        finish_kernel<<<n_masks, RED_THREADS, 0, st>>>(partials, blocks, n_masks, d_out);
        return cudaGetLastError();
    }
    const int blocks = reduce_blocks(n);
    const uint64_t per_block = dim / blocks;
    for (int k0 = 0; k0 < n_masks; k0 += ZMASKS) {
        const int m = n_masks - k0 < ZMASKS ? n_masks - k0 : ZMASKS;
        ZMasks zm{};
        for (int k = 0; k < m; ++k) zm.m[k] = masks[k0 + k];
        zsums_kernel<C><<<blocks, RED_THREADS, 0, st>>>((const C *)state, per_block, zm, m, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        finish_kernel<<<m, RED_THREADS, 0, st>>>(partials, blocks, m, d_out + k0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_zsums(bool c128, const void *state, int n, const uint64_t *masks, int n_masks, double *partials,
                         double *d_out, cudaStream_t st) {
    if (n_masks < 1 || n_masks > ZW_MASKS || n < 8) return cudaErrorInvalidValue;
    return c128 ? launch_zsums_t<double2>(state, n, masks, n_masks, partials, d_out, st)
                : launch_zsums_t<float2>(state, n, masks, n_masks, partials, d_out, st);
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
    double sre = 0, sim = 0;
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
        sre += (double)rre;
        sim += (double)rim;
    }
    __shared__ double wsum[RED_THREADS / 32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    if (lane == 0) {
        wsum[warp][0] = sre;
        wsum[warp][1] = sim;
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
