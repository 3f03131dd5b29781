// Fused state-vector pass for the digital adiabatic Z2 gauge simulation.
//
// One pass streams the state once.  Each CTA owns tiles of 2^TB amplitudes
// (tile bit i < c <-> global bit i, tile bit i >= c <-> global bit b + i - c),
// keeps them in registers (2^R amplitudes per thread) and applies
//
//   rot1 -> (plaquette phase table | real scale | nothing) -> rot2
//
// where rot1 / rot2 are masks of tile bits that receive the single-qubit
// gate of the pass:
//   OP_RX:       exp(i delta sigma^x) / cos(delta) = 1 + i tan(delta) sigma^x
//                (the transverse-field factor of Sec. 2.2; the cos^k factor is
//                folded into the phase table, which is built in FP64 on the host)
//   OP_HADAMARD: (a, b) -> (a + b, a - b), scale folded into the mid step
//                (the "H sigma^z H" measurement basis change of Sec. 2.4)
// and the plaquette layer D(theta) = exp(i theta sum_p U_p) (Eq. (ara) for
// every plaquette at once) as one table lookup per amplitude: the number k of
// plaquettes with odd parity is popcount of a 32-bit parity vector that is
// linear in the index bits, and the phase is table[k] = scale * exp(i theta
// (N_p - 2k)).
//
// Register layouts: layout q has register bits [r0(q), r0(q) + R) of the tile,
// r0(q) = max(TB - (q+1) R, 0); the remaining tile bits, in increasing order,
// are the thread index.  Layout 0 is the global-memory layout (lanes run along
// the contiguous low tile bits, so loads and stores are coalesced).  Changing
// layout goes through shared memory, one padding slot every 2^R amplitudes
// (slot(x) = x + (x >> R)); that keeps every layout's accesses free of bank
// conflicts and, being additive over disjoint bit sets, lets each register's
// address be a base register plus an immediate offset.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace z2 {

template <typename C>
struct Cfg;
template <>
struct Cfg<float2> {
    using real = float;
    static constexpr int R = 5;  // 32 amplitudes per thread (64 registers)
};
template <>
struct Cfg<double2> {
    using real = double;
    static constexpr int R = 4;  // 16 amplitudes per thread (64 registers)
};

// One entry of the per-launch pass list (device memory).  g1 / g2: the gate
// value (tan(delta) for OP_RX_TAN) of the rot1 / rot2 layer, so every
// rotation layer of a run may have its own angle (the g ramp of Sec. 2.2).
struct PassStep {
    uint32_t rot1, rot2;
    int32_t mid, table;
    double scale;
    double g1, g2;
};

__host__ __device__ constexpr int ctz_c(int x) { return (x & 1) ? 0 : 1 + ctz_c(x >> 1); }

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <int OP, typename C, typename real>
__device__ __forceinline__ void butterfly(C &a, C &b, real t) {
    if (OP == OP_RX_TAN) {
        // a' = a + i t b, b' = b + i t a
        C na, nb;
        na.x = fma(-t, b.y, a.x);
        na.y = fma(t, b.x, a.y);
        nb.x = fma(-t, a.y, b.x);
        nb.y = fma(t, a.x, b.y);
        a = na;
        b = nb;
    } else {
        C na, nb;
        na.x = a.x + b.x;
        na.y = a.y + b.y;
        nb.x = a.x - b.x;
        nb.y = a.y - b.y;
        a = na;
        b = nb;
    }
}

template <typename C, int TB>
struct Tile {
    static constexpr int R = Cfg<C>::R;
    static constexpr int NE = 1 << R;          // amplitudes per thread
    static constexpr int NT = 1 << (TB - R);   // threads per CTA
    static constexpr int K = (TB + R - 1) / R; // number of register layouts
    static constexpr int SMEM_SLOTS = (1 << TB) + (1 << (TB - R));
    // registers are capped at 128 per thread (two 256-thread CTAs per SM)
    static constexpr int NTW = NT < 32 ? 32 : NT;  // registers are allocated per whole warp
    static constexpr int MINB = (512 / NTW) < 1 ? 1 : (512 / NTW);

    __host__ __device__ static constexpr int r0(int q) { return TB - (q + 1) * R > 0 ? TB - (q + 1) * R : 0; }
    // tile bits whose gate is applied while in layout q
    __host__ __device__ static constexpr uint32_t owned(int q) {
        return (q == K - 1 ? ((1u << (TB - q * R)) - 1u)
                           : (((1u << R) - 1u) << r0(q))) & ((1u << TB) - 1u);
    }
    // tile index of register j of thread t in layout q
    __device__ static __forceinline__ uint32_t base(int q, uint32_t t) {
        const int r = r0(q);
        return (t & ((1u << r) - 1u)) | ((t >> r) << (r + R));
    }
    // shared-memory slot of tile index x; slot(base | j<<r0) = slot(base) + slot(j<<r0)
    __host__ __device__ static constexpr uint32_t slot(uint32_t x) { return x + (x >> R); }
};

template <typename C, int TB, int QA, int QB>
__device__ __forceinline__ void relayout(C (&v)[Tile<C, TB>::NE], C *sm, uint32_t t) {
    using T = Tile<C, TB>;
    C *sa = sm + T::slot(T::base(QA, t));
#pragma unroll
    for (int j = 0; j < T::NE; ++j) sa[T::slot((uint32_t)j << T::r0(QA))] = v[j];
    __syncthreads();
    const C *sb = sm + T::slot(T::base(QB, t));
#pragma unroll
    for (int j = 0; j < T::NE; ++j) v[j] = sb[T::slot((uint32_t)j << T::r0(QB))];
}

// rotations of the register bits of layout Q that are in `mask` (tile bits)
template <typename C, int TB, int Q, int OP>
__device__ __forceinline__ void rotate(C (&v)[Tile<C, TB>::NE], uint32_t mask, typename Cfg<C>::real t) {
    using T = Tile<C, TB>;
    const uint32_t m = (mask & T::owned(Q)) >> T::r0(Q);
#pragma unroll
    for (int q = 0; q < T::R; ++q) {
        if (m & (1u << q)) {
#pragma unroll
            for (int j = 0; j < T::NE; ++j)
                if (!(j & (1 << q))) butterfly<OP>(v[j], v[j | (1 << q)], t);
        }
    }
}

// plaquette phase table (or real scale) on the registers of layout Q
template <typename C, int TB, int Q>
__device__ __forceinline__ void apply_mid(C (&v)[Tile<C, TB>::NE], const PassArgs &a, int mid, double scale,
                                          uint32_t ptile, uint32_t t, const C *tab) {
    using T = Tile<C, TB>;
    using real = typename Cfg<C>::real;
    if (mid == MID_SCALE) {
        const real s = (real)scale;
#pragma unroll
        for (int j = 0; j < T::NE; ++j) {
            v[j].x *= s;
            v[j].y *= s;
        }
    } else if (mid == MID_TABLE) {
        // parity vector of the thread's tile bits (all but the register bits)
        uint32_t p = ptile;
        const int r = T::r0(Q);
#pragma unroll
        for (int i = 0; i < TB - T::R; ++i) {
            const int tbit = i < r ? i : i + T::R;
            if ((t >> i) & 1u) p ^= a.tcol[tbit];
        }
        // walk the registers in Gray-code order: one XOR per amplitude
#pragma unroll
        for (int gi = 0; gi < T::NE; ++gi) {
            if (gi) p ^= a.tcol[r + ctz_c(gi)];
            const int j = gi ^ (gi >> 1);
            v[j] = cmul(v[j], tab[__popc(p)]);
        }
    }
}

template <typename C, int TB, int OP>
__device__ __forceinline__ void rotate_in(int q, C (&v)[Tile<C, TB>::NE], uint32_t mask, typename Cfg<C>::real t) {
    switch (q) {
        case 0: rotate<C, TB, 0, OP>(v, mask, t); break;
        case 1: if (Tile<C, TB>::K > 1) rotate<C, TB, 1, OP>(v, mask, t); break;
        case 2: if (Tile<C, TB>::K > 2) rotate<C, TB, 2 < Tile<C, TB>::K ? 2 : 0, OP>(v, mask, t); break;
        default: if (Tile<C, TB>::K > 3) rotate<C, TB, 3 < Tile<C, TB>::K ? 3 : 0, OP>(v, mask, t); break;
    }
}

template <typename C, int TB>
__device__ __forceinline__ void mid_in(int q, C (&v)[Tile<C, TB>::NE], const PassArgs &a, int mid, double scale,
                                       uint32_t ptile, uint32_t t, const C *tab) {
    constexpr int K = Tile<C, TB>::K;
    switch (q) {
        case 0: apply_mid<C, TB, 0>(v, a, mid, scale, ptile, t, tab); break;
        case 1: apply_mid<C, TB, 1 < K ? 1 : 0>(v, a, mid, scale, ptile, t, tab); break;
        case 2: apply_mid<C, TB, 2 < K ? 2 : 0>(v, a, mid, scale, ptile, t, tab); break;
        default: apply_mid<C, TB, 3 < K ? 3 : 0>(v, a, mid, scale, ptile, t, tab); break;
    }
}

template <typename C, int TB, int QA>
__device__ __forceinline__ void relayout_from(int qb, C (&v)[Tile<C, TB>::NE], C *sm, uint32_t t) {
    constexpr int K = Tile<C, TB>::K;
    switch (qb) {
        case 0: relayout<C, TB, QA, 0>(v, sm, t); break;
        case 1: relayout<C, TB, QA, 1 < K ? 1 : 0>(v, sm, t); break;
        case 2: relayout<C, TB, QA, 2 < K ? 2 : 0>(v, sm, t); break;
        default: relayout<C, TB, QA, 3 < K ? 3 : 0>(v, sm, t); break;
    }
}

template <typename C, int TB>
__device__ __forceinline__ void relayout_rt(int qa, int qb, C (&v)[Tile<C, TB>::NE], C *sm, uint32_t t) {
    constexpr int K = Tile<C, TB>::K;
    switch (qa) {
        case 0: relayout_from<C, TB, 0>(qb, v, sm, t); break;
        case 1: relayout_from<C, TB, 1 < K ? 1 : 0>(qb, v, sm, t); break;
        case 2: relayout_from<C, TB, 2 < K ? 2 : 0>(qb, v, sm, t); break;
        default: relayout_from<C, TB, 3 < K ? 3 : 0>(qb, v, sm, t); break;
    }
}

// The pass kernel.  steps[0 .. n_steps) are applied in order; with a single
// tile (n == TB) the whole list runs with the state held in registers, with
// several tiles the host launches one step per kernel.
template <typename C, int TB, int OP>
__global__ void __launch_bounds__(Tile<C, TB>::NT, Tile<C, TB>::MINB) pass_kernel(C *__restrict__ psi, const __grid_constant__ PassArgs a,
                                                                const PassStep *__restrict__ steps, int n_steps,
                                                                const C *__restrict__ tables) {
    using T = Tile<C, TB>;
    using real = typename Cfg<C>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    __shared__ C tab[Z2_MAX_PLAQ + 1];

    const uint32_t t = threadIdx.x;
    const int c = a.c, b = a.b;
    const int hib = b + TB - c;  // first global bit above the tile's strided part
    const uint64_t ntiles = 1ull << (a.n - TB);
    // global index of the layout-0 thread part and register stride
    const uint64_t gthr = (uint64_t)(t & ((1u << c) - 1u)) | ((uint64_t)(c < TB ? (t >> c) : 0u) << b);
    const int r00 = T::r0(0);
    const int sj = (c == TB) ? r00 : (b + r00 - c);

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t tlo = tile & ((1ull << (b - c)) - 1ull);
        const uint64_t thi = tile >> (b - c);
        const uint64_t g0 = (tlo << c) | (thi << hib);
        // plaquette parity of the tile-id bits
        uint32_t ptile = 0;
        for (uint64_t m = g0; m; m &= m - 1) ptile ^= a.colmask[__ffsll((long long)m) - 1];

        C v[T::NE];
        const uint64_t stride = 1ull << sj;
        {
            const C *p = psi + g0 + gthr;
#pragma unroll
            for (int j = 0; j < T::NE; ++j, p += stride) v[j] = *p;
        }

        for (int s = 0; s < n_steps; ++s) {
            const PassStep st = steps[s];
            if (st.mid == MID_TABLE) {
                __syncthreads();  // previous readers of tab are done
                for (uint32_t i = t; i < (uint32_t)a.np1; i += T::NT)
                    tab[i] = tables[(size_t)st.table * (Z2_MAX_PLAQ + 1) + i];
                __syncthreads();
            }
            // phase 1: layouts 0, 1, ... as needed
            int cur = 0;
            rotate_in<C, TB, OP>(0, v, st.rot1, (real)st.g1);
#pragma unroll
            for (int q = 1; q < T::K; ++q) {
                if (st.rot1 & T::owned(q)) {
                    relayout_rt<C, TB>(cur, q, v, sm, t);
                    cur = q;
                    rotate_in<C, TB, OP>(q, v, st.rot1, (real)st.g1);
                }
            }
            mid_in<C, TB>(cur, v, a, st.mid, st.scale, ptile, t, tab);
            // phase 2: the current layout, then the others downwards, end in layout 0
            rotate_in<C, TB, OP>(cur, v, st.rot2, (real)st.g2);
            const int first = cur;
#pragma unroll
            for (int q = T::K - 1; q >= 1; --q) {
                if (q != first && (st.rot2 & T::owned(q))) {
                    relayout_rt<C, TB>(cur, q, v, sm, t);
                    cur = q;
                    rotate_in<C, TB, OP>(q, v, st.rot2, (real)st.g2);
                }
            }
            if (cur != 0) {
                relayout_rt<C, TB>(cur, 0, v, sm, t);
                if (first != 0) rotate_in<C, TB, OP>(0, v, st.rot2, (real)st.g2);
            }
        }
        // recompute the addresses instead of keeping 2^R pointers live
        uint64_t off = g0 + gthr;
        asm volatile("" : "+l"(off));
        C *p = psi + off;
#pragma unroll
        for (int j = 0; j < T::NE; ++j, p += stride) *p = v[j];
    }
}

}  // namespace z2

// ---------------------------------------------------------------------------
// TMA-pipelined variant (persistent CTAs).  Each CTA walks its tiles with a
// two-stage ring of shared-memory buffers: while the registers of tile i are
// being transformed, the tensor-memory-access unit already streams tile i+1
// into the other buffer (cp.async.bulk.tensor, completion on an mbarrier), and
// finished tiles leave through a TMA store.  The buffer of the tile being
// transformed doubles as the scratch of its register-layout changes.
#include <cuda.h>

namespace z2 {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c1, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %2, %2, "
        "%4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}
// the same with the tile coordinates in dimensions 1, 3 and 4 (the row and
// strided coordinates, 0 and 2, are always 0 for a whole-tile box)
__device__ __forceinline__ void tma_load_5c(void *dst, const CUtensorMap *map, uint64_t *bar, int c1, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %2, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_5c(const CUtensorMap *map, const void *src, int c1, int c3, int c4) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %1, %3, %4}], [%5];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(0), "r"(c1), "r"(c3), "r"(c4), "r"(smem_u32(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap *map, const void *src, int c1, int c4) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %1, %1, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(0), "r"(c1), "r"(c4), "r"(smem_u32(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Upper bound on mbarrier polls before a wait is declared failed (each poll
// may suspend the thread for a while; far beyond any legitimate copy).
constexpr uint32_t MBAR_POLL_LIMIT = 1u << 22;

template <typename C, int TB>
struct TmaTile {
    using T = Tile<C, TB>;
    static constexpr uint32_t TILE_BYTES = sizeof(C) << TB;
    static constexpr uint32_t BUF_BYTES = ((sizeof(C) * T::SMEM_SLOTS + 1023) / 1024) * 1024;
    static constexpr uint32_t SMEM_BYTES = 2 * BUF_BYTES + 1024;  // + alignment slack
};

// TMA tile coordinates: the tensor map views the state as
// (x_lo, tile_lo, x_hi1, x_hi2, tile_hi); a tile is (0, t_lo, 0, 0, t_hi).
template <typename C, int TB, int OP>
__global__ void __launch_bounds__(Tile<C, TB>::NT, 1)
    pass_kernel_tma(const __grid_constant__ PassArgs a, const __grid_constant__ CUtensorMap tmap,
                    const PassStep *__restrict__ steps, int n_steps, const C *__restrict__ tables, int *err) {
    using T = Tile<C, TB>;
    using TT = TmaTile<C, TB>;
    using real = typename Cfg<C>::real;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ C tab[Z2_MAX_PLAQ + 1];
    // 1024-byte aligned start, as an offset into the shared array (keeps the
    // accesses in the shared address space)
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    auto buf = [&](int k) { return reinterpret_cast<C *>(base + k * TT::BUF_BYTES); };

    const uint32_t t = threadIdx.x;
    const uint64_t ntiles = 1ull << (a.n - TB);
    const int lo_bits = a.tma_lo_bits;      // tile-id bits below the strided part
    const int c = a.c, b = a.b, hib = b + TB - c;

    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint64_t tile = blockIdx.x;
    if (t == 0 && tile < ntiles) {
        mbar_expect_tx(&mbar[0], TT::TILE_BYTES);
        tma_load_5d(buf(0), &tmap, &mbar[0], (int)(tile & ((1ull << lo_bits) - 1)), (int)(tile >> lo_bits));
    }
    for (uint32_t i = 0; tile < ntiles; ++i, tile += gridDim.x) {
        const int cur = i & 1;
        const uint64_t next = tile + gridDim.x;
        const bool has_next = next < ntiles;
        if (t == 0 && has_next) {
            bulk_wait_read_all();  // the store that last read buf(cur ^ 1) is done with it
            fence_proxy_async();
            mbar_expect_tx(&mbar[cur ^ 1], TT::TILE_BYTES);
            tma_load_5d(buf(cur ^ 1), &tmap, &mbar[cur ^ 1], (int)(next & ((1ull << lo_bits) - 1)),
                        (int)(next >> lo_bits));
        }
        // bounded wait for this tile's data
        bool ok = false;
        for (uint32_t k = 0; k < MBAR_POLL_LIMIT; ++k)
            if ((ok = mbar_try_wait(&mbar[cur], (i >> 1) & 1))) break;
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicExch(err, 1);
                // let the copies in flight finish (bounded) before leaving
                if (has_next)
                    for (uint32_t k = 0; k < MBAR_POLL_LIMIT && !mbar_try_wait(&mbar[cur ^ 1], ((i + 1) >> 1) & 1);
                         ++k) {
                    }
                bulk_wait_all();
            }
            return;
        }
        // plaquette parity of the tile-id bits
        const uint64_t tlo = tile & ((1ull << (b - c)) - 1ull);
        const uint64_t g0 = (tlo << c) | ((tile >> (b - c)) << hib);
        uint32_t ptile = 0;
        for (uint64_t m = g0; m; m &= m - 1) ptile ^= a.colmask[__ffsll((long long)m) - 1];

        C *sm = buf(cur);
        C v[T::NE];
#pragma unroll
        for (int j = 0; j < T::NE; ++j) v[j] = sm[t | ((uint32_t)j << T::r0(0))];
        __syncthreads();  // dense reads done before the padded layout reuses the buffer

        for (int s = 0; s < n_steps; ++s) {
            const PassStep st = steps[s];
            if (st.mid == MID_TABLE) {
                __syncthreads();
                for (uint32_t q = t; q < (uint32_t)a.np1; q += T::NT)
                    tab[q] = tables[(size_t)st.table * (Z2_MAX_PLAQ + 1) + q];
                __syncthreads();
            }
            int cur_l = 0;
            rotate_in<C, TB, OP>(0, v, st.rot1, (real)st.g1);
#pragma unroll
            for (int q = 1; q < T::K; ++q) {
                if (st.rot1 & T::owned(q)) {
                    relayout_rt<C, TB>(cur_l, q, v, sm, t);
                    cur_l = q;
                    rotate_in<C, TB, OP>(q, v, st.rot1, (real)st.g1);
                }
            }
            mid_in<C, TB>(cur_l, v, a, st.mid, st.scale, ptile, t, tab);
            rotate_in<C, TB, OP>(cur_l, v, st.rot2, (real)st.g2);
            const int first = cur_l;
#pragma unroll
            for (int q = T::K - 1; q >= 1; --q) {
                if (q != first && (st.rot2 & T::owned(q))) {
                    relayout_rt<C, TB>(cur_l, q, v, sm, t);
                    cur_l = q;
                    rotate_in<C, TB, OP>(q, v, st.rot2, (real)st.g2);
                }
            }
            if (cur_l != 0) {
                relayout_rt<C, TB>(cur_l, 0, v, sm, t);
                if (first != 0) rotate_in<C, TB, OP>(0, v, st.rot2, (real)st.g2);
            }
        }
        __syncthreads();  // padded reads done before the dense store image is written
#pragma unroll
        for (int j = 0; j < T::NE; ++j) sm[t | ((uint32_t)j << T::r0(0))] = v[j];
        fence_proxy_async();
        __syncthreads();
        if (t == 0) tma_store_5d(&tmap, sm, (int)(tile & ((1ull << lo_bits) - 1)), (int)(tile >> lo_bits));
    }
    if (t == 0) bulk_wait_all();
}

}  // namespace z2
