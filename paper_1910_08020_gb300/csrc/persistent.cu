// One persistent launch that evolves many independent adiabatic runs (the
// batched lambda sweep).
//
// The grid holds one 2^14-amplitude tile CTA per SM, all resident at once,
// grouped into gangs of GANG CTAs.  A gang takes the next run from a queue,
// walks through that run's passes (the same fused passes as z2_evolve, with
// |+> written in place of the first load), splitting each pass's tiles among
// its CTAs, and meets at a gang barrier between passes.  Gangs never wait on
// each other, and a gang's CTAs are co-resident, so the barrier always
// completes; it is still bounded: after a poll limit (2^26 polls by default,
// lower on request, see Z2_OPT_GANG_WAIT_POLLS) it sets the error flag and the
// CTA returns; the gang's other CTAs give up at their next barrier.
#include <cuda_runtime.h>

#include "pass_kernel.cuh"
#include "pass_packed.cuh"

namespace z2 {

constexpr int PERSIST_TB = 14;
constexpr int PERSIST_W = 4;
constexpr int GANG = 8;
constexpr uint32_t GANG_SPIN_LIMIT = 1u << 26;

// run descriptor (device memory, built by the host)
struct PersistRun {
    float2 *state;
    const PassStep *steps;
    const float2 *tables;
    const PassArgs *args;   // per group
    const int32_t *group;   // group of each pass
    int32_t n_passes;
    int32_t n;              // qubits
    float init_amp;         // 2^{-n/2}
    int32_t pad;
};

struct PersistCtl {
    unsigned long long next_run;  // queue head
    unsigned long long bar[64];   // per-gang barrier counters
    unsigned long long run_of[64];
};

__device__ __forceinline__ bool gang_barrier(PersistCtl *ctl, int g, unsigned long long target, int *err,
                                             uint32_t spin_limit) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->bar[g], 1ull);
        int ok = 0;
        for (uint32_t k = 0; k < spin_limit; ++k) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&ctl->bar[g]) : "memory");
            if (v >= target) {
                ok = 1;
                break;
            }
            __nanosleep(64);
        }
        if (!ok) atomicExch(err, 1);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int OP>
__global__ void __launch_bounds__(PTile<PERSIST_TB, PERSIST_W>::NT, 1)
    persistent_kernel(const PersistRun *__restrict__ runs, int n_runs, PersistCtl *ctl, int *err, uint32_t spin_limit) {
    constexpr int TB = PERSIST_TB, W = PERSIST_W;
    using T = PTile<TB, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2 *sm = reinterpret_cast<ulonglong2 *>(smem_raw);
    __shared__ ulonglong2 ptab[PAIR_TAB_ENTRIES];
    __shared__ PassArgs a_s;
    __shared__ unsigned long long run_s;

    const int g = blockIdx.x / GANG, rank = blockIdx.x % GANG;
    const uint32_t t = threadIdx.x;
    unsigned long long epoch = 0;
    for (;;) {
        // the gang leader takes the next run and publishes it to the gang
        if (!gang_barrier(ctl, g, (++epoch) * GANG, err, spin_limit)) return;
        if (rank == 0 && t == 0) {
            ctl->run_of[g] = atomicAdd(&ctl->next_run, 1ull);
            __threadfence();
        }
        if (!gang_barrier(ctl, g, (++epoch) * GANG, err, spin_limit)) return;
        if (t == 0) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&ctl->run_of[g]) : "memory");
            run_s = v;
        }
        __syncthreads();
        const unsigned long long r = run_s;
        if (r >= (unsigned long long)n_runs) return;
        const PersistRun R = runs[r];
        const uint64_t ntiles = 1ull << (R.n - TB > 0 ? R.n - TB : 0);
        const bool single = R.n <= TB;
        const int n_pass_launches = single ? 1 : R.n_passes;
        for (int ps = 0; ps < n_pass_launches; ++ps) {
            const int gi = single ? 0 : R.group[ps];
            // this pass's geometry, cooperatively copied to shared memory
            {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(&R.args[gi]);
                uint32_t *dst = reinterpret_cast<uint32_t *>(&a_s);
                for (uint32_t k = t; k < sizeof(PassArgs) / 4; k += T::NT) dst[k] = src[k];
            }
            __syncthreads();
            const PassArgs &a = a_s;
            const int c = a.c, b = a.b, hib = b + TB - c;
            const uint32_t x0 = 2u * t;
            const uint64_t gthr = (uint64_t)(x0 & ((1u << c) - 1u)) | ((uint64_t)(c < TB ? (x0 >> c) : 0u) << b);
            const int rbit = 1 + T::w0(0);
            const int sj = (c == TB) ? rbit : (b + rbit - c);
            const uint64_t stride = 1ull << sj;
            const bool first = ps == 0, last = ps == n_pass_launches - 1;
            const bool out_split = !single && !last, in_split = !single && !first;
            const int n_steps = single ? R.n_passes : 1;
            const PassStep *steps = single ? R.steps : R.steps + ps;
            for (uint64_t tile = rank; tile < ntiles; tile += GANG) {
                const uint64_t tlo = tile & ((1ull << (b - c)) - 1ull);
                const uint64_t g0 = (tlo << c) | ((tile >> (b - c)) << hib);
                if (!first && tile + GANG < ntiles) {  // the next tile into L2 (see prefetch_tile_l2)
                    const uint64_t nx = tile + GANG, nlo = nx & ((1ull << (b - c)) - 1ull);
                    prefetch_tile_l2<TB>(R.state, (nlo << c) | ((nx >> (b - c)) << hib), c, b, t, T::NT);
                }
                uint32_t ptile = 0;
                for (uint64_t m = g0; m; m &= m - 1) ptile ^= a.colmask[__ffsll((long long)m) - 1];
                u64 re[T::NP], im[T::NP];
                const float2 *p = R.state + g0 + gthr;
                if (first) {
                    const u64 amp = pk2(R.init_amp, R.init_amp);
#pragma unroll
                    for (int j = 0; j < T::NP; ++j) {
                        re[j] = amp;
                        im[j] = 0ull;
                    }
                } else if (in_split) {
#pragma unroll
                    for (int j = 0; j < T::NP; ++j, p += stride) {
                        // L2 only: another CTA of the gang wrote this tile in the previous pass
                        const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
                        re[j] = v.x;
                        im[j] = v.y;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < T::NP; ++j, p += stride) {
                        const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
                        re[j] = pk2(v.x, v.z);
                        im[j] = pk2(v.y, v.w);
                    }
                }
                for (int s = 0; s < n_steps; ++s) {
                    const PassStep st = steps[s];
                    if (st.mid == MID_TABLE) {
                        __syncthreads();
                        load_pair_table(ptab, R.tables + (size_t)st.table * (Z2_MAX_PLAQ + 1), a.np1, a.tcol[0], t,
                                        T::NT);
                        __syncthreads();
                    }
                    pstep<TB, W, OP>(re, im, st, a, (float)st.g1, (float)st.g2, ptile, t, sm, ptab, -1);
                }
                float2 *q = R.state + g0 + gthr;
                if (out_split) {
#pragma unroll
                    for (int j = 0; j < T::NP; ++j, q += stride)
                        __stcg(reinterpret_cast<ulonglong2 *>(q), make_ulonglong2(re[j], im[j]));
                } else {
#pragma unroll
                    for (int j = 0; j < T::NP; ++j, q += stride) {
                        float r0, r1, i0, i1;
                        upk2(re[j], r0, r1);
                        upk2(im[j], i0, i1);
                        __stcg(reinterpret_cast<float4 *>(q), make_float4(r0, i0, r1, i1));
                    }
                }
                __syncthreads();  // the shared scratch is reused by the next tile
            }
            // all tiles of this pass are written before any CTA of the gang reads the next
            if (!gang_barrier(ctl, g, (++epoch) * GANG, err, spin_limit)) return;
        }
    }
}

static_assert(sizeof(PersistRun) == sizeof(PersistRunHost), "run descriptor layout");

int persist_tile_bits() { return PERSIST_TB; }
int persist_gang() { return GANG; }
size_t persist_run_bytes() { return sizeof(PersistRun); }
size_t persist_ctl_bytes() { return sizeof(PersistCtl); }

cudaError_t launch_persistent(const void *runs, int n_runs, void *ctl, int *err, int grid, cudaStream_t st,
                              uint32_t spin_limit) {
    if (spin_limit == 0) spin_limit = GANG_SPIN_LIMIT;
    using T = PTile<PERSIST_TB, PERSIST_W>;
    const size_t smem = sizeof(ulonglong2) * T::SLOTS;
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    const uint64_t dev_bit = current_device_bit();
    if (!(configured.load() & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(persistent_kernel<OP_RX_TAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    // cooperative launch: every CTA is resident at once (or the launch fails),
    // which the gang barriers rely on
    const PersistRun *r = static_cast<const PersistRun *>(runs);
    PersistCtl *c = static_cast<PersistCtl *>(ctl);
    void *params[] = {(void *)&r, (void *)&n_runs, (void *)&c, (void *)&err, (void *)&spin_limit};
    return cudaLaunchCooperativeKernel((const void *)persistent_kernel<OP_RX_TAN>, dim3(grid), dim3(T::NT), params, smem,
                                       st);
}

int persist_max_ctas(int sm_count) {
    using T = PTile<PERSIST_TB, PERSIST_W>;
    int per_sm = 0;
    const size_t smem = sizeof(ulonglong2) * T::SLOTS;
    cudaFuncSetAttribute(persistent_kernel<OP_RX_TAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<OP_RX_TAN>, T::NT, smem) !=
        cudaSuccess)
        return 0;
    return per_sm * sm_count;
}

}  // namespace z2
