// Packed-pair fused pass for complex64 states (Blackwell f32x2 arithmetic).
//
// Same operation as pass_kernel (rot1 -> plaquette table | scale -> rot2 on a
// tile of 2^TB amplitudes, see there), organised for half the instructions:
//
//   * amplitudes x and x^1 (tile bit 0 = global bit 0) always travel together
//     as a "pair" held in two 64-bit registers, re = (re_x, re_x^1) and
//     im = (im_x, im_x^1); every butterfly on any other bit then updates two
//     amplitudes per packed instruction (fma.rn.f32x2 / add / sub / mul), the
//     transverse-field butterfly (a, b) -> (a + i t b, b + i t a) costing one
//     f32x2 FMA per amplitude;
//   * a thread holds 2^W pairs; register layout q keeps the pair-index bits
//     [w0(q), w0(q) + W) in registers, the remaining pair-index bits name the
//     thread; changing layout moves the pairs' 8-byte (re, re) and (im, im)
//     halves through two shared-memory arrays, one padding slot every 2^W
//     pairs (conflict-free for every layout and size);
//   * between the passes of one evolution the state is stored "split": each
//     16-byte pair as (re_x, re_x^1, im_x, im_x^1), so loads and stores need
//     no register shuffles; the first and last pass convert from and to the
//     interleaved (re, im) format of the public interface.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace z2 {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(u64 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <int TB, int W>
struct PTile {
    static constexpr int Y = TB - 1;              // pair-index bits
    static constexpr int NP = 1 << W;             // pairs per thread
    static constexpr int NT = 1 << (Y - W);       // threads per CTA
    static constexpr int K = (Y + W - 1) / W;     // register layouts
    static constexpr int SLOTS = (1 << Y) + (1 << (Y - W));
    static constexpr int NTW = NT < 32 ? 32 : NT;
    static constexpr int MINB = (512 / NTW) < 1 ? 1 : (512 / NTW);
    __host__ __device__ static constexpr int w0(int q) { return Y - W * (q + 1) > 0 ? Y - W * (q + 1) : 0; }
    // pair-index bits rotated while in layout q
    __host__ __device__ static constexpr uint32_t ownY(int q) {
        return q == K - 1 ? ((1u << (Y - q * W)) - 1u) : (((1u << W) - 1u) << w0(q));
    }
    __device__ static __forceinline__ uint32_t base(int q, uint32_t t) {
        const int r = w0(q);
        return (t & ((1u << r) - 1u)) | ((t >> r) << (r + W));
    }
    __host__ __device__ static constexpr uint32_t slot(uint32_t y) { return y + (y >> W); }
};

template <int OP>
__device__ __forceinline__ void bfly2(u64 &ra, u64 &ia, u64 &rb, u64 &ib, u64 tt, u64 mt) {
    if (OP == OP_RX_TAN) {
        const u64 nra = fma2(mt, ib, ra), nia = fma2(tt, rb, ia);
        const u64 nrb = fma2(mt, ia, rb), nib = fma2(tt, ra, ib);
        ra = nra;
        ia = nia;
        rb = nrb;
        ib = nib;
    } else {
        const u64 nra = add2(ra, rb), nrb = sub2(ra, rb);
        const u64 nia = add2(ia, ib), nib = sub2(ia, ib);
        ra = nra;
        rb = nrb;
        ia = nia;
        ib = nib;
    }
}

// the gate on tile bit 0: between the two halves of every pair
template <int OP>
__device__ __forceinline__ void bfly_in_pair(u64 &re, u64 &im, float t) {
    float ra, rb, ia, ib;
    upk2(re, ra, rb);
    upk2(im, ia, ib);
    if (OP == OP_RX_TAN) {
        re = pk2(fmaf(-t, ib, ra), fmaf(-t, ia, rb));
        im = pk2(fmaf(t, rb, ia), fmaf(t, ra, ib));
    } else {
        re = pk2(ra + rb, ra - rb);
        im = pk2(ia + ib, ia - ib);
    }
}

template <int TB, int W, int Q, int OP>
__device__ __forceinline__ void prot(u64 (&re)[1 << W], u64 (&im)[1 << W], uint32_t mask, float t) {
    using T = PTile<TB, W>;
    const u64 tt = pk2(t, t), mt = pk2(-t, -t);
    if (Q == 0 && (mask & 1u)) {
#pragma unroll
        for (int j = 0; j < T::NP; ++j) bfly_in_pair<OP>(re[j], im[j], t);
    }
    const uint32_t m = ((mask >> 1) & T::ownY(Q)) >> T::w0(Q);
    if constexpr (OP == OP_RX_TAN) {
        // Every level of the layout runs, with gate 0 (an exact identity of
        // the tan-form butterfly) where the bit is not rotated.  A branch per
        // level would make the registers of the rotated and unrotated paths
        // meet at its join, which costs a register move per amplitude and
        // level; the spare FMAs are cheaper.
        (void)tt;
        (void)mt;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            // register bits that are not this layout's own bits (the last
            // layout owns fewer than W) never rotate here: no code for them
            if (!(((T::ownY(Q) >> T::w0(Q)) >> q) & 1u)) continue;
            const float g = (m & (1u << q)) ? t : 0.0f;
            const u64 tq = pk2(g, g), mq = pk2(-g, -g);
#pragma unroll
            for (int j = 0; j < T::NP; ++j)
                if (!(j & (1 << q))) bfly2<OP>(re[j], im[j], re[j | (1 << q)], im[j | (1 << q)], tq, mq);
        }
    } else {
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (m & (1u << q)) {
#pragma unroll
                for (int j = 0; j < T::NP; ++j)
                    if (!(j & (1 << q))) bfly2<OP>(re[j], im[j], re[j | (1 << q)], im[j | (1 << q)], tt, mt);
            }
        }
    }
}

// barrier over the threads that share one tile: the whole CTA (bar < 0) or
// named barrier `bar` of NT threads (two tiles per CTA)
template <int NT>
__device__ __forceinline__ void tile_sync(int bar) {
    if (bar < 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NT) : "memory");
}

// Relayout through shared memory.  S8 = false: one array of 16-byte
// (re, re, im, im) pair slots.  S8 = true: the real and imaginary halves in
// two arrays of T::SLOTS 8-byte slots (the same SLOTS * 16 bytes): 8-byte
// accesses take each 64-bit register pair as it is, where a 16-byte access
// needs re and im in four adjacent registers, which costs register moves
// after the f32x2 butterflies; it also costs twice the load/store
// instructions.  Both are conflict-free for every layout and tile size
// (checked by enumeration; for S8 the 16 lanes of a half-warp always hit
// distinct slots modulo 16).
template <int TB, int W, int QA, int QB, bool S8>
__device__ __forceinline__ void prelayout(u64 (&re)[1 << W], u64 (&im)[1 << W], ulonglong2 *sm, uint32_t t,
                                          int bar = -1) {
    using T = PTile<TB, W>;
    if constexpr (S8) {
        u64 *sr = reinterpret_cast<u64 *>(sm), *si = sr + T::SLOTS;
        const uint32_t a = T::slot(T::base(QA, t));
#pragma unroll
        for (int j = 0; j < T::NP; ++j) {
            const uint32_t o = a + T::slot((uint32_t)j << T::w0(QA));
            sr[o] = re[j];
            si[o] = im[j];
        }
        tile_sync<T::NT>(bar);
        const uint32_t b = T::slot(T::base(QB, t));
#pragma unroll
        for (int j = 0; j < T::NP; ++j) {
            const uint32_t o = b + T::slot((uint32_t)j << T::w0(QB));
            re[j] = sr[o];
            im[j] = si[o];
        }
    } else {
        ulonglong2 *sa = sm + T::slot(T::base(QA, t));
#pragma unroll
        for (int j = 0; j < T::NP; ++j) sa[T::slot((uint32_t)j << T::w0(QA))] = make_ulonglong2(re[j], im[j]);
        tile_sync<T::NT>(bar);
        const ulonglong2 *sb = sm + T::slot(T::base(QB, t));
#pragma unroll
        for (int j = 0; j < T::NP; ++j) {
            const ulonglong2 v = sb[T::slot((uint32_t)j << T::w0(QB))];
            re[j] = v.x;
            im[j] = v.y;
        }
    }
}

// Pair phase table of a plaquette layer.  The two amplitudes x and x^1 of a
// pair have the parity vectors p and p ^ c0, c0 the plaquette column of
// global bit 0, so their phase indices are k0 = popcount(p) and
// k1 = popcount(p ^ c0) = k0 + popcount(c0) - 2 d with d = popcount(p & c0).
// Entry k0 + PAIR_TAB_STRIDE d holds both phases as the two packed halves the
// butterflies use, (re(tab[k0]), re(tab[k1])) and (im(tab[k0]), im(tab[k1])):
// one 16-byte load per pair in place of four scalar loads.  The stride is 1
// modulo 8, so entry (k0, d) sits in bank group (k0 + d) mod 8 and the lanes
// of a quarter warp, whose k0 differ, mostly hit distinct banks (with the
// index 8 k0 + d every lane of equal d shared four banks).  A link lies in at
// most 2 (dim - 1) = 4 plaquettes, so d < 8; combinations that cannot occur
// (k1 outside the table) hold a clamped entry that is never read.
constexpr int PAIR_TAB_STRIDE = Z2_MAX_PLAQ + 1;
static_assert(PAIR_TAB_STRIDE % 8 == 1, "pair-table stride must be 1 modulo 8");
constexpr int PAIR_TAB_ENTRIES = PAIR_TAB_STRIDE * 8;

__device__ __forceinline__ void load_pair_table(ulonglong2 *ptab, const float2 *tab, int np1, uint32_t c0,
                                                uint32_t tid, uint32_t nth) {
    const int w = __popc(c0);
    for (uint32_t e = tid; e < (uint32_t)PAIR_TAB_ENTRIES; e += nth) {
        const int k0 = (int)(e % PAIR_TAB_STRIDE), d = (int)(e / PAIR_TAB_STRIDE);
        if (k0 >= np1) continue;
        int k1 = k0 + w - 2 * d;
        k1 = k1 < 0 ? 0 : (k1 >= np1 ? np1 - 1 : k1);
        const float2 x = tab[k0], y = tab[k1];
        ptab[e] = make_ulonglong2(pk2(x.x, y.x), pk2(x.y, y.y));
    }
}

// plaquette phase table or real scale, in layout Q
template <int TB, int W, int Q>
__device__ __forceinline__ void pmid(u64 (&re)[1 << W], u64 (&im)[1 << W], const PassArgs &a, int mid, double scale,
                                     uint32_t ptile, uint32_t t, const ulonglong2 *ptab) {
    using T = PTile<TB, W>;
    if (mid == MID_SCALE) {
        const float s = (float)scale;
        const u64 s2 = pk2(s, s);
#pragma unroll
        for (int j = 0; j < T::NP; ++j) {
            re[j] = mul2(re[j], s2);
            im[j] = mul2(im[j], s2);
        }
    } else if (mid == MID_TABLE) {
        const int r = T::w0(Q);
        uint32_t p = ptile;
#pragma unroll
        for (int i = 0; i < T::Y - W; ++i) {
            const int ybit = i < r ? i : i + W;
            if ((t >> i) & 1u) p ^= a.tcol[ybit + 1];
        }
        const uint32_t c0 = a.tcol[0];
#pragma unroll
        for (int gi = 0; gi < T::NP; ++gi) {
            if (gi) p ^= a.tcol[r + ctz_c(gi) + 1];
            const int j = gi ^ (gi >> 1);
            const ulonglong2 e = ptab[(uint32_t)__popc(p) + PAIR_TAB_STRIDE * (uint32_t)__popc(p & c0)];
            const u64 tr = e.x, ti = e.y;
            const u64 nre = sub2(mul2(re[j], tr), mul2(im[j], ti));
            const u64 nim = fma2(re[j], ti, mul2(im[j], tr));
            re[j] = nre;
            im[j] = nim;
        }
    }
}

template <int TB, int W, int OP>
__device__ __forceinline__ void prot_in(int q, u64 (&re)[1 << W], u64 (&im)[1 << W], uint32_t mask, float t) {
    constexpr int K = PTile<TB, W>::K;
    switch (q) {
        case 0: prot<TB, W, 0, OP>(re, im, mask, t); break;
        // tile bit 0 (inside the pairs) belongs to layout 0
        case 1: prot<TB, W, (1 < K ? 1 : 0), OP>(re, im, mask & ~1u, t); break;
        case 2: prot<TB, W, (2 < K ? 2 : 0), OP>(re, im, mask & ~1u, t); break;
        default: prot<TB, W, (3 < K ? 3 : 0), OP>(re, im, mask & ~1u, t); break;
    }
}

template <int TB, int W>
__device__ __forceinline__ void pmid_in(int q, u64 (&re)[1 << W], u64 (&im)[1 << W], const PassArgs &a, int mid,
                                        double scale, uint32_t ptile, uint32_t t, const ulonglong2 *ptab) {
    constexpr int K = PTile<TB, W>::K;
    switch (q) {
        case 0: pmid<TB, W, 0>(re, im, a, mid, scale, ptile, t, ptab); break;
        case 1: pmid<TB, W, (1 < K ? 1 : 0)>(re, im, a, mid, scale, ptile, t, ptab); break;
        case 2: pmid<TB, W, (2 < K ? 2 : 0)>(re, im, a, mid, scale, ptile, t, ptab); break;
        default: pmid<TB, W, (3 < K ? 3 : 0)>(re, im, a, mid, scale, ptile, t, ptab); break;
    }
}

template <int TB, int W, int QA, bool S8>
__device__ __forceinline__ void prelayout_from(int qb, u64 (&re)[1 << W], u64 (&im)[1 << W], ulonglong2 *sm,
                                               uint32_t t, int bar) {
    constexpr int K = PTile<TB, W>::K;
    switch (qb) {
        case 0: prelayout<TB, W, QA, 0, S8>(re, im, sm, t, bar); break;
        case 1: prelayout<TB, W, QA, (1 < K ? 1 : 0), S8>(re, im, sm, t, bar); break;
        case 2: prelayout<TB, W, QA, (2 < K ? 2 : 0), S8>(re, im, sm, t, bar); break;
        default: prelayout<TB, W, QA, (3 < K ? 3 : 0), S8>(re, im, sm, t, bar); break;
    }
}

template <int TB, int W, bool S8>
__device__ __forceinline__ void prelayout_rt(int qa, int qb, u64 (&re)[1 << W], u64 (&im)[1 << W], ulonglong2 *sm,
                                             uint32_t t, int bar = -1) {
    constexpr int K = PTile<TB, W>::K;
    switch (qa) {
        case 0: prelayout_from<TB, W, 0, S8>(qb, re, im, sm, t, bar); break;
        case 1: prelayout_from<TB, W, (1 < K ? 1 : 0), S8>(qb, re, im, sm, t, bar); break;
        case 2: prelayout_from<TB, W, (2 < K ? 2 : 0), S8>(qb, re, im, sm, t, bar); break;
        default: prelayout_from<TB, W, (3 < K ? 3 : 0), S8>(qb, re, im, sm, t, bar); break;
    }
}

// one pass step on the registers of a tile (layout 0 in and out)
template <int TB, int W, int OP, bool S8 = false>
__device__ __forceinline__ void pstep(u64 (&re)[1 << W], u64 (&im)[1 << W], const PassStep &st, const PassArgs &a,
                                      float g1, float g2, uint32_t ptile, uint32_t t, ulonglong2 *sm,
                                      const ulonglong2 *ptab, int bar) {
    using T = PTile<TB, W>;
    int cur = 0;
    prot_in<TB, W, OP>(0, re, im, st.rot1, g1);
#pragma unroll
    for (int q = 1; q < T::K; ++q) {
        if ((st.rot1 >> 1) & T::ownY(q)) {
            prelayout_rt<TB, W, S8>(cur, q, re, im, sm, t, bar);
            cur = q;
            prot_in<TB, W, OP>(q, re, im, st.rot1, g1);
        }
    }
    pmid_in<TB, W>(cur, re, im, a, st.mid, st.scale, ptile, t, ptab);
    if (st.rot2 == 0) {  // no second rotation (uniform over the launch): back to layout 0
        if (cur != 0) prelayout_rt<TB, W, S8>(cur, 0, re, im, sm, t, bar);
        return;
    }
    prot_in<TB, W, OP>(cur, re, im, cur == 0 ? st.rot2 : (st.rot2 & ~1u), g2);
    const int first = cur;
#pragma unroll
    for (int q = T::K - 1; q >= 1; --q) {
        if (q != first && ((st.rot2 >> 1) & T::ownY(q))) {
            prelayout_rt<TB, W, S8>(cur, q, re, im, sm, t, bar);
            cur = q;
            prot_in<TB, W, OP>(q, re, im, st.rot2 & ~1u, g2);
        }
    }
    if (cur != 0) {
        prelayout_rt<TB, W, S8>(cur, 0, re, im, sm, t, bar);
        if (first != 0) prot_in<TB, W, OP>(0, re, im, st.rot2, g2);
    }
}

// Rotation levels on pair-index bits that are lane bits of register layout
// Q.  In layout Q the pair-index bits below w0(Q) are the low bits of the
// thread index, so bit i < 5 there pairs lane l with lane l ^ (1 << i) of the
// same warp, for every register pair alike.  The butterfly is symmetric,
// (a, b) -> (a + i t b, b + i t a): each lane adds i t times its partner's
// amplitude, with the partner's (re, re) and (im, im) halves fetched by warp
// shuffles.  The arithmetic is that of bfly2, so results are bit-identical to
// a visit of the layout that holds the bit in registers, without its two
// relayouts.  LB is the mask of such pair-index bits; a bit that the pass does
// not rotate gets gate 0 (an exact identity).
template <int TB, int W, int Q, int OP, int LB>
__device__ __forceinline__ void prot_lanes(u64 (&re)[1 << W], u64 (&im)[1 << W], uint32_t mask, float t) {
    using T = PTile<TB, W>;
    static_assert(OP == OP_RX_TAN, "lane levels are transverse-field rotations");
    static_assert((LB >> (T::w0(Q) < 5 ? T::w0(Q) : 5)) == 0, "lane levels need lane bits of the layout");
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (!((LB >> i) & 1)) continue;
        const float g = ((mask >> (i + 1)) & 1u) ? t : 0.0f;
        const u64 tq = pk2(g, g), mq = pk2(-g, -g);
#pragma unroll
        for (int j = 0; j < T::NP; ++j) {
            const u64 rp = __shfl_xor_sync(0xffffffffu, re[j], 1 << i);
            const u64 ip = __shfl_xor_sync(0xffffffffu, im[j], 1 << i);
            re[j] = fma2(mq, ip, re[j]);
            im[j] = fma2(tq, rp, im[j]);
        }
    }
}

// Static layout sequences.  pstep chooses at run time which register
// layouts a pass visits; the join points of those choices cost register
// moves.  When the host knows that rot1 and rot2 lie in the register bits of
// layouts 0 .. L-1, pstep_static visits exactly those in a fixed order: rot1
// up through layouts 0 .. L-1, the mid step in layout L-1, then rot2 back down
// to layout 0 (R2), or, for a pass without a second rotation, one relayout
// back to layout 0.  Every rotated bit is rotated once in its own layout, as
// in pstep, so the result is the same.
template <int TB, int W, int OP, bool S8, int Q, int L>
__device__ __forceinline__ void seq_up(u64 (&re)[1 << W], u64 (&im)[1 << W], const PassStep &st, float g1,
                                       ulonglong2 *sm, uint32_t t, int bar) {
    if constexpr (Q < L) {
        prelayout<TB, W, Q - 1, Q, S8>(re, im, sm, t, bar);
        prot<TB, W, Q, OP>(re, im, st.rot1 & ~1u, g1);
        seq_up<TB, W, OP, S8, Q + 1, L>(re, im, st, g1, sm, t, bar);
    }
}

// in layout Q + 1: move to layout Q and apply its rot2 bits, down to layout 0
template <int TB, int W, int OP, bool S8, int Q>
__device__ __forceinline__ void seq_down(u64 (&re)[1 << W], u64 (&im)[1 << W], const PassStep &st, float g2,
                                         ulonglong2 *sm, uint32_t t, int bar) {
    if constexpr (Q >= 0) {
        prelayout<TB, W, Q + 1, Q, S8>(re, im, sm, t, bar);
        prot<TB, W, Q, OP>(re, im, Q == 0 ? st.rot2 : (st.rot2 & ~1u), g2);
        seq_down<TB, W, OP, S8, Q - 1>(re, im, st, g2, sm, t, bar);
    }
}

template <int TB, int W, int OP, bool S8, int L, bool R2, int LB = 0>
__device__ __forceinline__ void pstep_static(u64 (&re)[1 << W], u64 (&im)[1 << W], const PassStep &st,
                                             const PassArgs &a, float g1, float g2, uint32_t ptile, uint32_t t,
                                             ulonglong2 *sm, const ulonglong2 *ptab, int bar) {
    static_assert(L >= 1 && L <= PTile<TB, W>::K, "static sequence beyond the tile's layouts");
    prot<TB, W, 0, OP>(re, im, st.rot1, g1);
    seq_up<TB, W, OP, S8, 1, L>(re, im, st, g1, sm, t, bar);
    if constexpr (LB != 0) prot_lanes<TB, W, L - 1, OP, LB>(re, im, st.rot1, g1);
    pmid<TB, W, L - 1>(re, im, a, st.mid, st.scale, ptile, t, ptab);
    if constexpr (R2) {
        if constexpr (LB != 0) prot_lanes<TB, W, L - 1, OP, LB>(re, im, st.rot2, g2);
        prot<TB, W, L - 1, OP>(re, im, L - 1 == 0 ? st.rot2 : (st.rot2 & ~1u), g2);
        seq_down<TB, W, OP, S8, L - 2>(re, im, st, g2, sm, t, bar);
    } else if constexpr (L > 1) {
        prelayout<TB, W, L - 1, 0, S8>(re, im, sm, t, bar);
    }
}

// SEQ template argument of the ring kernel: 0 = pstep, else 2 L + R2, plus
// 16 LB for lane levels (prot_lanes) in layout L - 1
constexpr int seq_code(int L, bool R2, int lb = 0) { return 2 * L + (R2 ? 1 : 0) + 16 * lb; }

// Ask the TMA unit to pull a tile into L2 ahead of its use (no completion is
// tracked: a prefetch never blocks and never faults on in-range addresses).
// The tile is 2^(TB-c) rows of 2^c contiguous complex64 amplitudes, row r at
// global index g0 + (r << b); threads of the CTA share the rows in units of at
// most 16 KB.
template <int TB>
__device__ __forceinline__ void prefetch_tile_l2(const float2 *psi, uint64_t g0, int c, int b, uint32_t t, uint32_t nt) {
    const int ub = c + 3 < 14 ? c + 3 : 14;  // log2 bytes of one unit
    const uint32_t units_per_row = 1u << (c + 3 - ub), rows = 1u << (TB - c);
    for (uint32_t u = t; u < rows * units_per_row; u += nt) {
        const uint64_t r = u / units_per_row, k = u % units_per_row;
        const char *addr = reinterpret_cast<const char *>(psi + g0 + (r << b)) + (k << ub);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(addr), "r"(1u << ub) : "memory");
    }
}

// fmt bit 0: the input is split-pair, bit 1: write the output split-pair
template <int TB, int W, int OP>
__global__ void __launch_bounds__(PTile<TB, W>::NT, PTile<TB, W>::MINB)
    pass_kernel_packed(float2 *__restrict__ psi, const __grid_constant__ PassArgs a,
                       const PassStep *__restrict__ steps, int n_steps, const float2 *__restrict__ tables, int fmt) {
    using T = PTile<TB, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2 *sm = reinterpret_cast<ulonglong2 *>(smem_raw);
    __shared__ ulonglong2 ptab[PAIR_TAB_ENTRIES];

    const uint32_t t = threadIdx.x;
    const int c = a.c, b = a.b;
    const int hib = b + TB - c;
    const uint64_t ntiles = 1ull << (a.n - TB);
    // global index of the thread's first pair (tile index 2t) and the register stride
    const uint32_t x0 = 2u * t;
    const uint64_t gthr = (uint64_t)(x0 & ((1u << c) - 1u)) | ((uint64_t)(c < TB ? (x0 >> c) : 0u) << b);
    const int rbit = 1 + T::w0(0);  // tile bit of register bit 0 in layout 0
    const int sj = (c == TB) ? rbit : (b + rbit - c);
    const uint64_t stride = 1ull << sj;
    const bool in_split = fmt & 1, out_split = fmt & 2;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t tlo = tile & ((1ull << (b - c)) - 1ull);
        const uint64_t g0 = (tlo << c) | ((tile >> (b - c)) << hib);
        uint32_t ptile = 0;
        for (uint64_t m = g0; m; m &= m - 1) ptile ^= a.colmask[__ffsll((long long)m) - 1];
        // this CTA's next tile streams into L2 while this one is loaded and transformed
        if (tile + gridDim.x < ntiles) {
            const uint64_t nx = tile + gridDim.x, nlo = nx & ((1ull << (b - c)) - 1ull);
            prefetch_tile_l2<TB>(psi, (nlo << c) | ((nx >> (b - c)) << hib), c, b, t, T::NT);
        }

        u64 re[T::NP], im[T::NP];
        {
            const float2 *p = psi + g0 + gthr;
            if (in_split) {
#pragma unroll
                for (int j = 0; j < T::NP; ++j, p += stride) {
                    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
                    re[j] = v.x;
                    im[j] = v.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < T::NP; ++j, p += stride) {
                    const float4 v = *reinterpret_cast<const float4 *>(p);
                    re[j] = pk2(v.x, v.z);
                    im[j] = pk2(v.y, v.w);
                }
            }
        }
        for (int s = 0; s < n_steps; ++s) {
            const PassStep st = steps[s];
            if (st.mid == MID_TABLE) {
                __syncthreads();
                load_pair_table(ptab, tables + (size_t)st.table * (Z2_MAX_PLAQ + 1), a.np1, a.tcol[0], t, T::NT);
                __syncthreads();
            }
            pstep<TB, W, OP>(re, im, st, a, (float)st.g1, (float)st.g2, ptile, t, sm, ptab, -1);
        }
        uint64_t off = g0 + gthr;
        asm volatile("" : "+l"(off));
        float2 *p = psi + off;
        if (out_split) {
#pragma unroll
            for (int j = 0; j < T::NP; ++j, p += stride)
                *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(re[j], im[j]);
        } else {
#pragma unroll
            for (int j = 0; j < T::NP; ++j, p += stride) {
                float r0, r1, i0, i1;
                upk2(re[j], r0, r1);
                upk2(im[j], i0, i1);
                *reinterpret_cast<float4 *>(p) = make_float4(r0, i0, r1, i1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Streaming variant: one CTA per SM made of NW independent workers of NT
// threads, each transforming its own tile with its own named barrier, fed by a
// ring of NB > NW shared-memory tile buffers that the TMA unit fills ahead of
// use (cp.async.bulk.tensor + mbarrier) and drains with TMA stores.  Local
// tile n (global tile blockIdx.x + n * gridDim.x) lives in buffer n % NB and
// is worked on by worker n % NW; when a worker has stored tile n it refills
// that buffer with tile n + NB, so NW tiles are being transformed while
// NB - NW stream in.  Multi-tile, single-step passes only (the host launches
// one per pass).  Requires pass_kernel.cuh (TMA and mbarrier helpers) to be
// included first.
template <int TB, int W>
struct RingTile {
    using T = PTile<TB, W>;
    static constexpr uint32_t BUF = ((T::SLOTS * 16u + 1023u) / 1024u) * 1024u;
    static constexpr uint32_t TILE_BYTES = 8u << TB;
    // workers: up to 512 threads (256 with 32 pairs per thread, for the
    // register file) and 8 named barriers; buffers: up to 2 per worker within
    // 210 KB of shared memory
    static constexpr int MAXT = W >= 5 ? 256 : 512;
    static constexpr int NW = (MAXT / T::NT) < 8 ? (MAXT / T::NT) : 8;
    static constexpr int NB_FIT = (int)((210u * 1024u) / BUF);
    static constexpr int NB = NB_FIT < 2 * NW ? NB_FIT : 2 * NW;
    static constexpr uint32_t SMEM_BYTES = NB * BUF + 1024;
    static_assert(NW >= 1 && NB > NW, "ring needs more buffers than workers");
};

__device__ __forceinline__ bool bar_and(int bar, int n, bool v) {
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(bar), "r"(n)
                 : "memory");
    return r != 0;
}

// Plaquette parity vector of the amplitude at global index g0: the XOR of the
// columns of g0's set bits.  The 64 bits are shared out over the lanes of a
// warp (lane l takes bits l and l + 32) and the warp XOR-reduces, so every
// lane gets the result in a dozen instructions instead of a serial loop over
// the set bits in every thread.  All 32 lanes must take part.
__device__ __forceinline__ uint32_t warp_tile_parity(uint64_t g0, const uint32_t *colm, uint32_t lane) {
    uint32_t v = (((g0 >> lane) & 1ull) ? colm[lane] : 0u) ^ (((g0 >> (lane + 32)) & 1ull) ? colm[lane + 32] : 0u);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int TB, int W, int OP, bool S8 = false, int SEQ = 0>
__global__ void __launch_bounds__(RingTile<TB, W>::NW * PTile<TB, W>::NT, 1)
    pass_kernel_ring(const __grid_constant__ PassArgs a, const __grid_constant__ CUtensorMap tmap,
                     const PassStep *__restrict__ steps, const float2 *__restrict__ tables, int fmt, int *err) {
    using T = PTile<TB, W>;
    using RT = RingTile<TB, W>;
    constexpr int NW = RT::NW, NB = RT::NB;
    static_assert(T::NT % 32 == 0, "ring workers are whole warps (the tile parity is a warp reduction)");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[NB];
    __shared__ uint32_t loads_issued[NB];  // TMA loads issued into each buffer
    __shared__ uint32_t uses_seen[NB];     // loads of each buffer whose completion a worker has observed
    __shared__ int abort_s;                // a worker gave up waiting
    __shared__ ulonglong2 ptab[PAIR_TAB_ENTRIES];
    __shared__ uint32_t colm_s[64];        // plaquette column of each global bit
    // 1024-byte aligned start, as an offset into the shared array (keeps the
    // accesses in the shared address space)
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    auto buf = [&](int k) { return reinterpret_cast<ulonglong2 *>(base + k * RT::BUF); };

    const uint32_t worker = threadIdx.x / T::NT, t = threadIdx.x % T::NT;
    const int bar = 1 + (int)worker;
    // a group may be split in two bit ranges (see the host planner): the
    // tile-id bits above the lower range start at a.hib, and the TMA view
    // takes them in dimension 3 instead of 4
    const int c = a.c, b = a.b, hib = a.hib, lo_bits = a.tma_lo_bits;
    const bool hi3 = a.tma_hi_dim == 3;
    const bool in_split = fmt & 1, out_split = fmt & 2;
    const PassStep st = steps[0];
    const uint64_t ntiles = 1ull << (a.n - TB);
    const uint64_t nloc = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto gtile = [&](uint64_t n) { return (uint64_t)blockIdx.x + n * gridDim.x; };
    auto load_tile = [&](void *dst, uint64_t *mb, uint64_t g) {
        const int lo = (int)(g & ((1ull << lo_bits) - 1)), hi = (int)(g >> lo_bits);
        tma_load_5c(dst, &tmap, mb, lo, hi3 ? hi : 0, hi3 ? 0 : hi);
    };

    if (st.mid == MID_TABLE)
        load_pair_table(ptab, tables + (size_t)st.table * (Z2_MAX_PLAQ + 1), a.np1, a.tcol[0], threadIdx.x,
                        NW * T::NT);
    for (uint32_t q = threadIdx.x; q < 64u; q += NW * T::NT) colm_s[q] = a.colmask[q];
    if (threadIdx.x == 0) {
        for (int k = 0; k < NB; ++k) {
            mbar_init(&mbar[k], 1);
            loads_issued[k] = 0;
            uses_seen[k] = 0;
        }
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (uint64_t n = 0; n < (uint64_t)NB && n < nloc; ++n) {
            const uint64_t g = gtile(n);
            atomicAdd(&loads_issued[n], 1u);
            mbar_expect_tx(&mbar[n], RT::TILE_BYTES);
            load_tile(buf((int)n), &mbar[n], g);
        }

    for (uint64_t n = worker; n < nloc; n += NW) {
        const int bi = (int)(n % NB);
        const uint32_t use = (uint32_t)(n / NB);  // this tile is load number `use` of buffer bi
        // Consecutive uses of a buffer belong to different workers, and this
        // worker may arrive here while load `use - 1` is still in flight.  The
        // barrier is then in phase use - 1, whose parity differs from ours, so
        // the parity test would report the older phase use - 2 as done.  Wait
        // first until the previous use has been observed: from then on the
        // barrier's current phase is `use` and the test is exact.
        bool ok = false;
        for (uint32_t k = 0; k < MBAR_POLL_LIMIT; ++k) {
            if (*reinterpret_cast<volatile int *>(&abort_s)) break;
            if (*reinterpret_cast<volatile uint32_t *>(&uses_seen[bi]) != use) continue;
            if ((ok = mbar_try_wait(&mbar[bi], use & 1))) break;
        }
        if (!bar_and(bar, T::NT, ok)) {
            // this worker stops; the others stop at their next wait, and the
            // CTA drains every copy still in flight before it exits
            if (t == 0) {
                atomicExch(err, 1);
                atomicExch(&abort_s, 1);
            }
            break;
        }
        // every thread of this worker has seen the phase: publish it
        if (t == 0) *reinterpret_cast<volatile uint32_t *>(&uses_seen[bi]) = use + 1;
        const uint64_t tile = gtile(n);
        const uint64_t tlo = tile & ((1ull << (b - c)) - 1ull);
        const uint64_t g0 = (tlo << c) | ((tile >> (b - c)) << hib);
        const uint32_t ptile = warp_tile_parity(g0, colm_s, threadIdx.x & 31u);

        ulonglong2 *sm = buf(bi);
        u64 re[T::NP], im[T::NP];
        // layout 0 from the dense tile image (pair y at slot y)
        if (in_split) {
#pragma unroll
            for (int j = 0; j < T::NP; ++j) {
                const ulonglong2 v = sm[t | ((uint32_t)j << T::w0(0))];
                re[j] = v.x;
                im[j] = v.y;
            }
        } else {
            const float4 *sf = reinterpret_cast<const float4 *>(sm);
#pragma unroll
            for (int j = 0; j < T::NP; ++j) {
                const float4 v = sf[t | ((uint32_t)j << T::w0(0))];
                re[j] = pk2(v.x, v.z);
                im[j] = pk2(v.y, v.w);
            }
        }
        tile_sync<T::NT>(bar);  // dense reads done before the padded layouts reuse the buffer
        if constexpr (SEQ == 0)
            pstep<TB, W, OP, S8>(re, im, st, a, (float)st.g1, (float)st.g2, ptile, t, sm, ptab, bar);
        else
            pstep_static<TB, W, OP, S8, (SEQ & 15) / 2, (SEQ & 1) != 0, (SEQ >> 4)>(
                re, im, st, a, (float)st.g1, (float)st.g2, ptile, t, sm, ptab, bar);
        tile_sync<T::NT>(bar);  // padded reads done before the dense store image is written
        if (out_split) {
#pragma unroll
            for (int j = 0; j < T::NP; ++j) sm[t | ((uint32_t)j << T::w0(0))] = make_ulonglong2(re[j], im[j]);
        } else {
            float4 *sf = reinterpret_cast<float4 *>(sm);
#pragma unroll
            for (int j = 0; j < T::NP; ++j) {
                float r0, r1, i0, i1;
                upk2(re[j], r0, r1);
                upk2(im[j], i0, i1);
                sf[t | ((uint32_t)j << T::w0(0))] = make_float4(r0, i0, r1, i1);
            }
        }
        fence_proxy_async();
        tile_sync<T::NT>(bar);
        if (t == 0) {
            {
                const int lo = (int)(tile & ((1ull << lo_bits) - 1)), hi = (int)(tile >> lo_bits);
                tma_store_5c(&tmap, sm, lo, hi3 ? hi : 0, hi3 ? 0 : hi);
            }
            if (n + NB < nloc) {
                bulk_wait_read_all();  // the store has read the buffer
                const uint64_t g = gtile(n + NB);
                atomicAdd(&loads_issued[bi], 1u);
                mbar_expect_tx(&mbar[bi], RT::TILE_BYTES);
                load_tile(sm, &mbar[bi], g);
            }
        }
    }
    if (t == 0) bulk_wait_all();  // this worker's stores
    __syncthreads();
    // Loads into a buffer are issued one at a time (a refill follows the use
    // of the previous load), so waiting for the last one drains the buffer.
    // After a normal run every load has been consumed and these return at once.
    if (threadIdx.x == 0)
        for (int k = 0; k < NB; ++k) {
            const uint32_t u = loads_issued[k];
            if (!u) continue;
            bool done = false;
            for (uint32_t q = 0; q < MBAR_POLL_LIMIT && !done; ++q) done = mbar_try_wait(&mbar[k], (u - 1) & 1);
            if (!done) atomicExch(err, 1);
        }
}

}  // namespace z2
