// Runtime and C ABI: contexts, execution plans, evolution, measurement.
//
// A run of the digital adiabatic algorithm (Sec. 2.2) is, in application
// order, the operator sequence
//
//     D(theta_0)  R  D(theta_1)  R  ...  R  D(theta_M)
//
// with R = prod_l exp(i dt sigma^x_l) and D(theta) = exp(i theta sum_p U_p):
//   first order (Eq. (a), varying factor first, right-end sampling):
//       theta_k = lambda s_{k+1} dt (k < M), theta_M = 0
//   symmetric (Eq. (s) with its halves merged as in the rewritten product of
//   Sec. 2.2; trapezoid sampling, second order):
//       theta_0 = 0, theta_k = lambda s_k dt, theta_M = lambda s_M dt / 2
//   symmetric, the paper's literal sampling (both halves at s_j):
//       theta_0 = lambda s_1 dt/2, theta_k = lambda (s_k + s_{k+1}) dt/2, theta_M = lambda dt/2
// where s_k = k/M.  The plan splits the N qubits into groups that each fit
// one tile, reverses the group order every step so that the last group of
// step j and the first group of step j+1 share one pass with D(theta_j)
// between them, and therefore streams the state g-1 times per step for g
// groups (g >= 2).
#include <cmath>
#include <complex>
#include <functional>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"

using z2::Lattice;

struct z2_lattice {
    Lattice lat;
};

namespace z2 {
namespace {

thread_local std::string g_last_error;

// A group rotates k global bits: [b, b + k1) and, when k1 < k, also
// [b2, b2 + k - k1) with b2 + k - k1 = n (a group split in two ranges, the
// upper one ending at the top bit).  Its tiles hold the c lowest global bits
// as passengers followed by the group's bits in increasing order.
struct Group {
    int lo = 0, hi = 0;  // for contiguous groups: global bits [lo, hi)
    int tb = 0;          // tile bits of this group's passes
    int c = 0, b = 0;    // tile geometry
    int k = 0, k1 = 0;   // rotated bits, and how many of them start at b
    int b2 = 0;          // start of the upper range (split groups)
    uint32_t rot = 0;    // tile-bit mask of the group's bits
};

struct Geometry {
    int n = 0, tb = 0;
    bool c128 = false;
    std::vector<Group> groups;
    std::vector<int> order;  // application order within an even step
};

struct HostPass {
    int group;
    PassStepHost step;
};

// A compiled segment of a run (or a single layer): passes, tables, flip.
struct Plan {
    Geometry geo;
    int op = OP_RX_TAN;
    std::vector<HostPass> passes;
    std::vector<std::complex<double>> tables;  // n_tables x (Z2_MAX_PLAQ + 1)
    bool flip = false;
    void *d_steps = nullptr;
    void *d_tables = nullptr;
    std::vector<PassArgs> args;  // per group
    bool tma = false;                  // TMA-pipelined persistent kernel
    bool ring = false;                 // complex64 TMA ring kernel (multi-tile passes)
    bool ring_wide = false;            // ... with 32 pairs per thread
    bool strided_wide = false;         // ... for the strided groups only (variant 5)
    int variant = 0;                   // the kernel variant the plan was built for
    ~Plan() {
        if (d_steps) cudaFree(d_steps);
        if (d_tables) cudaFree(d_tables);
    }
};

}  // namespace
}  // namespace z2

struct z2_ctx {
    int device = 0;
    int sm_count = 0;
    std::string last_error;
    double *d_partials = nullptr;  // reduction partials (reduce_partials_doubles(Z2_MAX_LINKS))
    double *d_out = nullptr;       // reduction outputs (256 doubles)
    double *h_out = nullptr;       // pinned copy of d_out
    std::map<std::string, std::unique_ptr<z2::Plan>> plans;
    int tb_override = 0;
    int split_low = 0;  // Z2_OPT_SPLIT_LOW_BITS
    int variant = 0;  // 0 = automatic (ring where it applies, else direct), 1 = direct, 2 = TMA per CTA, 3 = ring,
                      // 4 = ring with 32 pairs per thread
    std::map<std::pair<int, int>, std::pair<int, int>> tuned;  // (qubits, precision) -> (tile bits, variant)
    uint64_t launches = 0;
    int *d_err = nullptr;  // device flag: a bounded wait gave up
    uint32_t gang_wait_polls = 0;  // Z2_OPT_GANG_WAIT_POLLS (0 = the kernel's default)
};

namespace z2 {
namespace {

constexpr int TABLE_STRIDE = Z2_MAX_PLAQ + 1;
constexpr int OUT_DOUBLES = 256;

}  // namespace

int set_thread_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

namespace {

int fail(z2_ctx *ctx, int code, const std::string &msg) {
    if (ctx)
        ctx->last_error = msg;
    else
        g_last_error = msg;
    return code;
}

int cuda_fail(z2_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, Z2_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define Z2_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int tile_limit(bool c128) { return c128 ? 13 : 14; }
int regbits(bool c128) { return c128 ? 4 : 5; }

// the TMA-pipelined variant is used on request only (it holds one CTA per SM)
bool tma_possible(bool c128, int tb, int variant) { return variant == 2 && tb <= tma_tile_limit(c128); }

// Choose the tile size and split the qubits into groups (see file comment).
// A strided group of k qubits has a tile of 2^c contiguous x 2^k strided
// amplitudes, c = tb - k, with 3 <= c (>= 64-byte runs), c <= tb - R (the
// register bits of the global layout lie in the strided part) and c <= 8 (7
// for complex128; one TMA box row is at most 256 elements).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

// whether passes of this geometry run on the complex64 TMA ring kernel
// (tma: the driver's tensor-map encoder is available)
bool ring_plan(bool c128, int variant, int tb, int n_groups, bool tma) {
    return !c128 && (variant == 3 || variant == 0 || (variant == 5 && tb >= 12)) && n_groups > 1 && tb >= 10 &&
           tb <= 13 && tma;
}

bool plan_geometry(int n, bool c128, int tb_override, int variant, Geometry &g, std::string &err,
                   bool tma = encode_fn() != nullptr, int split_low = 0) {
    g = Geometry{};
    g.n = n;
    g.c128 = c128;
    const int R = regbits(c128);
    constexpr int CMIN = 3;
    const int CMAX = c128 ? 7 : 8;
    if (n < 8) {
        err = "states of fewer than 8 qubits are not supported";
        return false;
    }
    if (n <= tile_limit(c128) && (!tb_override || tb_override >= n)) {
        g.tb = n;
        Group gr;
        gr.lo = 0;
        gr.hi = n;
        gr.tb = n;
        gr.k = gr.k1 = n;
        gr.c = n;
        gr.b = n;
        gr.rot = (1u << n) - 1u;
        g.groups.push_back(gr);
        g.order = {0};
        return true;
    }
    auto kmin = [&](int tb) { return std::max(R, tb - CMAX); };
    auto kmax = [&](int tb) { return tb - CMIN; };
    int best_tb = 0, best_h = 1 << 30;
    bool best_tma = false;
    std::vector<int> cands;
    if (tb_override)
        cands.push_back(tb_override);
    else
        for (int tb = tile_limit(c128) - 2; tb <= tile_limit(c128); ++tb) cands.push_back(tb);
    for (int tb : cands) {
        if (tb < 8 || tb > tile_limit(c128) || tb >= n) continue;
        const int rem = n - tb;
        const int h = (rem + kmax(tb) - 1) / kmax(tb);
        const bool tma = tma_possible(c128, tb, variant);
        if (variant == 2 && !tma && !tb_override) continue;
        if (h < best_h || (h == best_h && tma && !best_tma)) {
            best_h = h;
            best_tb = tb;
            best_tma = tma;
        }
    }
    if (!best_tb) {
        err = "no tile size fits this state";
        return false;
    }
    const int tb = best_tb, h = best_h;
    int n_low = tb, rem = n - tb;
    if (rem < kmin(tb) * h) {  // keep every strided group >= kmin bits
        n_low = n - kmin(tb) * h;
        rem = kmin(tb) * h;
    }
    // The complex64 ring kernel runs twice as many workers on tiles one bit
    // smaller.  The low group (contiguous rows, no plaquette layer) gains from
    // that more than it loses, so it takes the smaller tile whenever the
    // strided groups can absorb the extra bit without an extra pass.
    int tb_low = tb;
    if (tb >= 11 && ring_plan(c128, variant, tb, h + 1, tma) && n_low == tb) {
        const int rem1 = n - (tb - 1);
        if ((rem1 + kmax(tb) - 1) / kmax(tb) == h && rem1 >= kmin(tb) * h) {
            tb_low = tb - 1;
            n_low = tb_low;
            rem = rem1;
        }
    }
    // Automatic plans on the 14-bit direct kernel with a single strided group
    // of at most 11 bits (24 qubits): both groups move to 13-bit tiles on the
    // TMA ring, the low group with 13 bits and the strided group with only 2
    // passenger bits (32-byte rows).  Both passes stay merged, one per Trotter
    // step.  The direct kernel holds one 14-bit tile per SM and waits for each
    // load; the ring streams.  At 24 qubits the state is about the size of L2
    // (57% of the sectors hit), where short rows cost little: measured 10.98k
    // Trotter steps/s against 10.23k with the strided group on 14-bit direct
    // tiles (3 passenger bits) and 8.35k for 14 + 10 on the direct kernel.
    if (!c128 && variant == 0 && !tb_override && tma && tb == 14 && h == 1 && n_low == tb && n - 13 <= 11 &&
        n - 13 >= kmin(13)) {
        g.tb = 13;
        Group lo;
        lo.lo = 0;
        lo.hi = lo.k = lo.k1 = lo.tb = lo.c = lo.b = 13;
        lo.rot = (1u << 13) - 1u;
        Group st;
        st.lo = st.b = 13;
        st.hi = n;
        st.k = st.k1 = n - 13;
        st.tb = 13;
        st.c = 13 - st.k;
        st.rot = ((1u << st.k) - 1u) << st.c;
        g.groups = {lo, st};
        g.order = {0, 1};
        return true;
    }
    g.tb = tb;
    Group low;
    low.lo = 0;
    low.hi = n_low;
    low.k = low.k1 = n_low;
    low.tb = tb_low;
    low.c = tb_low;
    low.b = tb_low;
    low.rot = (n_low >= 32) ? 0xffffffffu : ((1u << n_low) - 1u);
    g.groups.push_back(low);
    int lo = n_low;
    for (int i = 0; i < h; ++i) {
        const int k = rem / h + (i < rem % h ? 1 : 0);
        Group gr;
        gr.lo = lo;
        gr.hi = lo + k;
        gr.k = gr.k1 = k;
        gr.tb = tb;
        gr.c = tb - k;
        gr.b = lo;
        gr.rot = ((1u << k) - 1u) << gr.c;
        if (gr.c < CMIN || gr.c > tb - R || gr.c > CMAX || gr.b < gr.c || gr.hi > n) {
            err = "internal tile planning error";
            return false;
        }
        g.groups.push_back(gr);
        lo += k;
    }
    // Two strided groups on the ring: one group takes a few bits at the bottom
    // of the strided range and the top ones, the other the middle ones.  A
    // strided pass streams fastest when many of its rotated bits lie below
    // SPREAD_BITS (rows less than 16 MB apart): measured on a GB300 at 32
    // qubits (13-bit tiles, two 10-bit groups over bits 12..31), Trotter
    // steps/s against the split group's bottom bits a = 2..8 were 29.0, 32.2,
    // 34.2, 34.2, 32.2, 29.0, 29.0, which follows the slower group's share of
    // the bits 12..20, min(a, 9 - a); a contiguous split (bits 12..21 and
    // 22..31) ran the upper group at a third more time per pass.  So the bits
    // below SPREAD_BITS are shared as evenly as the groups allow.
    if (h == 2 && ring_plan(c128, variant, tb, (int)g.groups.size(), tma)) {
        constexpr int SPREAD_BITS = 21;  // 16 MB / 8 bytes per complex64 amplitude
        auto spread = [&](int lo_, int hi_) { return std::max(0, std::min(hi_, SPREAD_BITS) - lo_); };
        const Group A = g.groups[1], B = g.groups[2];
        const int base = A.lo;
        int best = std::min(spread(A.lo, A.hi), spread(B.lo, B.hi)), best_a = -1, best_ks = 0;
        if (split_low > 0) {  // requested width of the split group's lower range
            const int ks = A.k;
            if (split_low >= ks || split_low > 8 || ks - split_low > 8) {
                err = "split width " + std::to_string(split_low) + " does not fit a group of " + std::to_string(ks) +
                      " bits (each range 1..8 bits)";
                return false;
            }
            best_a = split_low;
            best_ks = ks;
        }
        for (int ks : {A.k, B.k}) {  // size of the split group
            if (split_low != 0) break;
            const int km = A.k + B.k - ks;
            for (int a = 1; a < ks && a <= 8; ++a) {
                if (ks - a > 8) continue;  // each range is one TMA box dimension (<= 256)
                const int top_lo = n - (ks - a);
                const int p = std::min(spread(base, base + a) + spread(top_lo, n), spread(base + a, base + a + km));
                if (p > best) {
                    best = p;
                    best_a = a;
                    best_ks = ks;
                }
            }
        }
        if (best_a > 0) {
            const int ks = best_ks, km = A.k + B.k - ks, a = best_a;
            Group S, Mi;
            S.tb = Mi.tb = tb;
            S.k = ks;
            S.k1 = a;
            S.b = base;
            S.b2 = n - (ks - a);
            S.c = tb - ks;
            S.rot = ((1u << ks) - 1u) << S.c;
            Mi.k = Mi.k1 = km;
            Mi.lo = Mi.b = base + a;
            Mi.hi = base + a + km;
            Mi.c = tb - km;
            Mi.rot = ((1u << km) - 1u) << Mi.c;
            if (S.c < CMIN || Mi.c < CMIN || S.b < S.c || Mi.b < Mi.c || Mi.hi != S.b2) {
                err = "internal tile planning error (split groups)";
                return false;
            }
            g.groups[1] = S;
            g.groups[2] = Mi;
        }
    }
    // low group in the middle so that the merged boundary passes are the
    // cheaper strided ones (measured at 32 qubits with the static layout
    // sequences: 36.6 Trotter steps/s against 29.7 with the low group merged)
    if (g.groups.size() >= 3) {
        g.order.push_back(1);
        g.order.push_back(0);
        for (int i = 2; i < (int)g.groups.size(); ++i) g.order.push_back(i);
    } else {
        g.order = {0, 1};
    }
    return true;
}

// 5-D TMA view of the state for one group: (x_lo, tile_lo, x_hi1, x_hi2,
// tile_hi), with box (2^c', 1, 2^k1, 2^k2, 1) = exactly one tile.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_tensor_map(CUtensorMap *m, void *state, int n, int tb, const Group &gr, bool c128, int &lo_bits,
                     int &hi_dim) {
    auto enc = encode_fn();
    if (!enc) return false;
    const uint64_t E = c128 ? 16 : 8;
    if (gr.k1 < gr.k) {
        // split group: (x_lo, tile_a, hi1, tile_b, hi2), box (2^c, 1, 2^k1, 1, 2^(k-k1))
        const int c = gr.c, b = gr.b, k1 = gr.k1, k2 = gr.k - gr.k1, b2 = gr.b2;
        if (c128 || b2 + k2 != n || b2 < b + k1) return false;
        cuuint64_t dims[5] = {cuuint64_t(1) << c, cuuint64_t(1) << (b - c), cuuint64_t(1) << k1,
                              cuuint64_t(1) << (b2 - b - k1), cuuint64_t(1) << k2};
        cuuint64_t strides[4] = {(cuuint64_t(1) << c) * E, (cuuint64_t(1) << b) * E, (cuuint64_t(1) << (b + k1)) * E,
                                 (cuuint64_t(1) << b2) * E};
        cuuint32_t box[5] = {cuuint32_t(1) << c, 1, cuuint32_t(1) << k1, 1, cuuint32_t(1) << k2};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        lo_bits = b - c;
        hi_dim = 3;
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, state, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    hi_dim = 4;
    int cp = gr.c, bp = gr.b;
    const int cmax = c128 ? 7 : 8;  // a box row holds at most 256 FLOAT64 elements
    if (cp > cmax) {                // contiguous tile: view it as 2^cmax x 2^(tb-cmax)
        cp = cmax;
        bp = cmax;
    }
    const int k = tb - cp, k1 = std::min(k, 8), k2 = k - k1;
    const int gap = bp - cp, top = n - bp - k;
    const uint32_t inner = c128 ? 2u : 1u;  // FLOAT64 elements per amplitude
    cuuint64_t dims[5] = {(cuuint64_t(1) << cp) * inner, cuuint64_t(1) << gap, cuuint64_t(1) << k1,
                          cuuint64_t(1) << k2, cuuint64_t(1) << top};
    cuuint64_t strides[4] = {(cuuint64_t(1) << cp) * E, (cuuint64_t(1) << bp) * E, (cuuint64_t(1) << (bp + k1)) * E,
                             (cuuint64_t(1) << (bp + k)) * E};
    cuuint32_t box[5] = {(cuuint32_t(1) << cp) * inner, 1, cuuint32_t(1) << k1, cuuint32_t(1) << k2, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    lo_bits = gap;
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, state, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

PassArgs make_args(const Lattice &lat, const Geometry &g, const Group &gr) {
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = g.n;
    a.c = gr.c;
    a.b = gr.b;
    // first global bit above the tile's lower range: b + (tb - c) for a
    // contiguous group (b itself for the low group, whose tile has no strided
    // part), b + k1 for a split one
    a.hib = gr.b + (gr.k1 < gr.k ? gr.k1 : gr.tb - gr.c);
    a.tma_hi_dim = 4;
    a.np1 = lat.n_plaq + 1;
    for (int i = 0; i < gr.tb; ++i) {
        const int gpos = i < gr.c ? i : (i - gr.c < gr.k1 ? gr.b + i - gr.c : gr.b2 + i - gr.c - gr.k1);
        a.tcol[i] = gpos < 64 ? lat.colmask[gpos] : 0;
    }
    std::memcpy(a.colmask, lat.colmask, sizeof(a.colmask));
    return a;
}

// Event list of a layer sequence: group applications and D events.
struct Event {
    int kind;  // 0 = group, 1 = D
    int group;
    int table;
    double gate = 0;  // group events: the gate value (tan(delta)) of this application
};

void pack_passes(const std::vector<Event> &ev, const Geometry &g, std::vector<HostPass> &out) {
    size_t i = 0;
    while (i < ev.size()) {
        HostPass p{};
        p.group = 0;
        p.step.mid = MID_NONE;
        p.step.table = -1;
        p.step.scale = 1.0;
        if (ev[i].kind == 0) {
            const int gi = ev[i].group;
            p.group = gi;
            p.step.rot1 = g.groups[gi].rot;
            p.step.g1 = ev[i].gate;
            ++i;
            if (i < ev.size() && ev[i].kind == 1) {
                p.step.mid = MID_TABLE;
                p.step.table = ev[i].table;
                ++i;
                if (i < ev.size() && ev[i].kind == 0 && ev[i].group == gi) {
                    p.step.rot2 = g.groups[gi].rot;
                    p.step.g2 = ev[i].gate;
                    ++i;
                }
            }
        } else {
            p.step.mid = MID_TABLE;
            p.step.table = ev[i].table;
            ++i;
            if (i < ev.size() && ev[i].kind == 0) {
                p.group = ev[i].group;
                p.step.rot2 = g.groups[p.group].rot;
                p.step.g2 = ev[i].gate;
                ++i;
            }
        }
        out.push_back(p);
    }
}

// exp(i dt sigma^x) = (i^q cos(delta))^... per qubit: dt = q pi/2 + delta,
// |delta| <= pi/4, exp(i dt sigma^x) = (i sigma^x)^q cos(delta) (1 + i tan(delta) sigma^x)
struct GateSplit {
    int q;
    double delta, t, c;
};
GateSplit split_gate(double dt) {
    GateSplit s;
    const double q = std::nearbyint(dt / (M_PI / 2));
    s.q = (int)std::fmod(q, 4.0);
    if (s.q < 0) s.q += 4;
    s.delta = dt - q * (M_PI / 2);
    s.t = std::tan(s.delta);
    s.c = std::cos(s.delta);
    return s;
}

std::complex<double> ipow(int q) {
    switch (((q % 4) + 4) % 4) {
        case 0: return {1, 0};
        case 1: return {0, 1};
        case 2: return {-1, 0};
        default: return {0, -1};
    }
}

void push_table(Plan &P, const Lattice &lat, double theta, std::complex<double> scale) {
    const int np = lat.n_plaq;
    for (int k = 0; k < TABLE_STRIDE; ++k) {
        std::complex<double> v(0, 0);
        if (k <= np) v = scale * std::exp(std::complex<double>(0, theta * (np - 2 * k)));
        P.tables.push_back(v);
    }
}

int upload_plan(z2_ctx *ctx, const Lattice &lat, Plan &P) {
    const bool c128 = P.geo.c128;
    std::vector<PassStepHost> steps;
    for (auto &hp : P.passes) steps.push_back(hp.step);
    if (!steps.empty()) {
        Z2_CUDA(ctx, cudaMalloc(&P.d_steps, steps.size() * sizeof(PassStepHost)));
        Z2_CUDA(ctx, cudaMemcpy(P.d_steps, steps.data(), steps.size() * sizeof(PassStepHost), cudaMemcpyHostToDevice));
    }
    if (!P.tables.empty()) {
        const size_t cnt = P.tables.size();
        if (c128) {
            std::vector<double2> t(cnt);
            for (size_t i = 0; i < cnt; ++i) t[i] = make_double2(P.tables[i].real(), P.tables[i].imag());
            Z2_CUDA(ctx, cudaMalloc(&P.d_tables, cnt * sizeof(double2)));
            Z2_CUDA(ctx, cudaMemcpy(P.d_tables, t.data(), cnt * sizeof(double2), cudaMemcpyHostToDevice));
        } else {
            std::vector<float2> t(cnt);
            for (size_t i = 0; i < cnt; ++i)
                t[i] = make_float2((float)P.tables[i].real(), (float)P.tables[i].imag());
            Z2_CUDA(ctx, cudaMalloc(&P.d_tables, cnt * sizeof(float2)));
            Z2_CUDA(ctx, cudaMemcpy(P.d_tables, t.data(), cnt * sizeof(float2), cudaMemcpyHostToDevice));
        }
    }
    for (auto &gr : P.geo.groups) P.args.push_back(make_args(lat, P.geo, gr));
    P.tma = tma_possible(c128, P.geo.tb, P.variant) && encode_fn() != nullptr;
    // the ring variant is the automatic choice for multi-tile complex64 passes
    P.ring = ring_plan(c128, P.variant, P.geo.tb, (int)P.geo.groups.size(), encode_fn() != nullptr);
    P.ring_wide = !c128 && P.variant == 4 && P.geo.groups.size() > 1 && P.geo.tb >= 12 && P.geo.tb <= 13 &&
                  encode_fn() != nullptr;
    if (P.ring_wide) P.ring = true;
    // automatic: the strided groups on 32 pairs per thread where that kernel
    // exists (measured fastest at 32 qubits: variant 5 over 3 and 4)
    P.strided_wide = P.ring && (P.variant == 5 || (P.variant == 0 && P.geo.tb >= 12));
    return Z2_OK;
}

// Pair-index bits owned by register layout q of a complex64 tile of tb bits
// with 2^W pairs per thread (the host copy of PTile::ownY in pass_packed.cuh).
uint32_t layout_own_bits(int tb, int W, int q) {
    const int Y = tb - 1, K = (Y + W - 1) / W;
    if (q == K - 1) return (1u << (Y - q * W)) - 1u;
    const int w0 = std::max(Y - W * (q + 1), 0);
    return ((1u << W) - 1u) << w0;
}

// Static layout sequence of a ring pass (pstep_static): the fewest layouts
// 0 .. L-1 that hold every rotated bit of rot1 and rot2, coded 2 L + (rot2 != 0).
// The wide kernel's 13-bit strided pass whose only rotated bit beyond layout 1
// is pair-index bit 1 (a group with two passenger bits) rotates that bit by
// warp shuffles in layout 1, where it is lane bit 1 (code + 16 * lane mask):
// two relayouts instead of four.
int ring_seq(int tb, int W, const PassStepHost &s) {
    const int Y = tb - 1, K = (Y + W - 1) / W;
    const uint32_t bits = (s.rot1 | s.rot2) >> 1;
    const int r2 = s.rot2 ? 1 : 0;
    uint32_t cover = 0;
    for (int L = 1; L <= K; ++L) {
        cover |= layout_own_bits(tb, W, L - 1);
        if (!(bits & ~cover)) {
            if (W == 5 && tb == 13 && L == 3) {
                const uint32_t rest = bits & ~(layout_own_bits(tb, W, 0) | layout_own_bits(tb, W, 1));
                if (rest == 2u) return 2 * 2 + r2 + 16 * 2;
            }
            return 2 * L + r2;
        }
    }
    return 0;
}

// effective tile size and kernel variant for a state of n qubits: explicit
// options first, then the autotuner's choice, else automatic
std::pair<int, int> exec_choice(const z2_ctx *ctx, int n, int precision) {
    int tb = ctx->tb_override, var = ctx->variant;
    auto it = ctx->tuned.find({n, precision});
    if (it != ctx->tuned.end()) {
        if (!tb) tb = it->second.first;
        if (!var) var = it->second.second;
    }
    return {tb, var};
}

// theta_k of the merged sequence for steps j0+1 .. j1 (k = j0 .. j1)
double theta_at(const z2_run_params &p, int k, int j0, int j1) {
    const double M = p.M, dt = p.T / p.M, lam = p.lambda;
    auto s = [&](int j) { return j / M; };
    if (p.decomp == Z2_FIRST_ORDER) return k < j1 ? lam * s(k + 1) * dt : 0.0;
    if (p.sampling == Z2_SAMPLE_PAPER) {
        if (k == j0) return lam * s(j0 + 1) * dt / 2;
        if (k == j1) return lam * s(j1) * dt / 2;
        return lam * (s(k) + s(k + 1)) * dt / 2;
    }
    if (k == j0) return lam * s(j0) * dt / 2;
    if (k == j1) return lam * s(j1) * dt / 2;
    return lam * s(k) * dt;
}

// Build the plan of steps j0+1 .. j1 (an empty plan when j0 == j1).
int build_evolve_plan(z2_ctx *ctx, const Lattice &lat, const z2_run_params &p, int j0, int j1, Plan &P) {
    std::string err;
    const auto ch = exec_choice(ctx, lat.n_links, p.precision);
    P.variant = ch.second;
    if (!plan_geometry(lat.n_links, p.precision == Z2_C128, ch.first, ch.second, P.geo, err,
                       encode_fn() != nullptr, ctx->split_low))
        return fail(ctx, Z2_ERR_LATTICE, err);
    P.op = OP_RX_TAN;
    if (j1 == j0) return upload_plan(ctx, lat, P);
    const GateSplit gs = split_gate(p.T / p.M);
    const auto &g = P.geo;
    std::vector<Event> ev;
    std::complex<double> pending(1, 0);  // gate scale since the last D
    int n_tab = 0;
    const double th0 = theta_at(p, j0, j0, j1);
    if (th0 != 0.0) {
        push_table(P, lat, th0, pending);
        ev.push_back({1, 0, n_tab++});
    }
    for (int j = j0 + 1; j <= j1; ++j) {
        const bool fwd = ((j - 1) & 1) == 0;
        const int G = (int)g.order.size();
        for (int k = 0; k < G; ++k) {
            const int gi = g.order[fwd ? k : G - 1 - k];
            ev.push_back({0, gi, -1, gs.t});
            const int bits = g.groups[gi].k;
            pending *= std::pow(gs.c, bits) * ipow(gs.q * bits);
        }
        push_table(P, lat, theta_at(p, j, j0, j1), pending);
        pending = {1, 0};
        ev.push_back({1, 0, n_tab++});
    }
    pack_passes(ev, g, P.passes);
    P.flip = (gs.q & 1) && ((j1 - j0) & 1);
    return upload_plan(ctx, lat, P);
}

// Plan of substeps J0+1 .. J1 of a fixed-Hamiltonian-form layer sequence:
// substep j is D(tau) R(a_j) (first order, the R layer acting first) or
// D(tau/2) R(a_j) D(tau/2) (symmetric), with a_j = angle(j); adjacent half
// layers D(tau/2) D(tau/2) merge into D(tau).  This is the paper's own ramp
// (Sec. 2.2, Eqs. a and s) and the fixed-g evolution of phase estimation
// (Sec. 2.4, Eq. leap): with Z = -sum U_p and X = -sum sigma^x,
// exp(-i Z tau) = D(tau) and exp(-i g X tau) = R(g tau), so the plaquette
// angle is constant and every R layer may have its own gate value.
int build_substep_plan(z2_ctx *ctx, const Lattice &lat, int precision, bool sym, double tau, int64_t J0, int64_t J1,
                       const std::function<double(int64_t)> &angle, Plan &P) {
    std::string err;
    const auto ch = exec_choice(ctx, lat.n_links, precision);
    P.variant = ch.second;
    if (!plan_geometry(lat.n_links, precision == Z2_C128, ch.first, ch.second, P.geo, err,
                       encode_fn() != nullptr, ctx->split_low))
        return fail(ctx, Z2_ERR_LATTICE, err);
    P.op = OP_RX_TAN;
    if (J1 == J0) return upload_plan(ctx, lat, P);
    const auto &g = P.geo;
    std::vector<Event> ev;
    std::complex<double> pending(1, 0);
    int n_tab = 0, quarter_turns = 0;
    if (sym) {
        push_table(P, lat, tau / 2, pending);
        ev.push_back({1, 0, n_tab++});
    }
    const int G = (int)g.order.size();
    for (int64_t j = J0 + 1; j <= J1; ++j) {
        const GateSplit gs = split_gate(angle(j));
        quarter_turns += gs.q;
        const bool fwd = ((j - 1) & 1) == 0;
        for (int k = 0; k < G; ++k) {
            const int gi = g.order[fwd ? k : G - 1 - k];
            ev.push_back({0, gi, -1, gs.t});
            const int bits = g.groups[gi].k;
            pending *= std::pow(gs.c, bits) * ipow(gs.q * bits);
        }
        push_table(P, lat, sym && j == J1 ? tau / 2 : tau, pending);
        pending = {1, 0};
        ev.push_back({1, 0, n_tab++});
    }
    pack_passes(ev, g, P.passes);
    P.flip = quarter_turns & 1;
    return upload_plan(ctx, lat, P);
}

// Steps k0+1 .. k1 of the paper's own ramp H(g) = Z + g X (Sec. 2.2):
// substep j = (k-1) n + m holds g_j = j g_s / n for tau = t_s / n.
int build_gramp_plan(z2_ctx *ctx, const Lattice &lat, const z2_gramp_params &gp, int k0, int k1, Plan &P) {
    const double tau = gp.t_s / gp.n;
    return build_substep_plan(ctx, lat, gp.precision, gp.decomp == Z2_SYMMETRIC, tau, (int64_t)k0 * gp.n,
                              (int64_t)k1 * gp.n, [&](int64_t j) { return (double)j * gp.g_s / gp.n * tau; }, P);
}

// Linearly independent vectors spanning the same GF(2) space as `vs`.
std::vector<uint64_t> gf2_basis(const std::vector<uint64_t> &vs) {
    uint64_t piv[64] = {};
    for (uint64_t v : vs) {
        for (int b = 63; b >= 0 && v; --b) {
            if (!((v >> b) & 1ull)) continue;
            if (!piv[b]) {
                piv[b] = v;
                v = 0;
            } else {
                v ^= piv[b];
            }
        }
    }
    std::vector<uint64_t> out;
    for (int b = 0; b < 64; ++b)
        if (piv[b]) out.push_back(piv[b]);
    return out;
}

int exec_plan(z2_ctx *ctx, Plan &P, void *state, cudaStream_t st) {
    const auto &g = P.geo;
    const bool c128 = g.c128;
    const uint64_t ntiles = 1ull << (g.n - g.tb);  // of the main tile size
    const size_t step_bytes = sizeof(PassStepHost);
    const bool single = g.groups.size() == 1;
    if ((P.tma || P.ring) && !P.passes.empty()) {
        // tensor maps name the state buffer, so they are encoded per call
        // (a few microseconds) and passed by value to each launch
        std::vector<CUtensorMap> tmaps(g.groups.size());
        for (size_t i = 0; i < g.groups.size(); ++i) {
            int lo_bits = 0, hi_dim = 4;
            if (!make_tensor_map(&tmaps[i], state, g.n, g.groups[i].tb, g.groups[i], c128, lo_bits, hi_dim))
                return fail(ctx, Z2_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            P.args[i].tma_lo_bits = lo_bits;
            P.args[i].tma_hi_dim = hi_dim;
        }
        if (P.ring) {
            const size_t last = P.passes.size() - 1;
            for (size_t i = 0; i < P.passes.size(); ++i) {
                const int gi = P.passes[i].group;
                const int tb = g.groups[gi].tb;
                const uint64_t nt = 1ull << (g.n - tb);
                const int grid = (int)std::min<uint64_t>((nt + 1) / 2, (uint64_t)ctx->sm_count);
                const void *sp = static_cast<const char *>(P.d_steps) + i * step_bytes;
                const int fmt = (i > 0 ? 1 : 0) | (i < last ? 2 : 0);
                const bool wide = P.ring_wide || (P.strided_wide && gi != 0);
                const int seq = ring_seq(tb, wide ? 5 : 4, P.passes[i].step);
                if (wide)
                    Z2_CUDA(ctx, launch_pass_ring5_c64(tb, P.op, P.args[gi], &tmaps[gi], sp, P.d_tables, fmt,
                                                       ctx->d_err, grid, st, P.strided_wide, seq));
                else
                    Z2_CUDA(ctx, launch_pass_ring_c64(tb, P.op, P.args[gi], &tmaps[gi], sp, P.d_tables, fmt,
                                                      ctx->d_err, grid, st, gi != 0, seq));
            }
            ctx->launches += P.passes.size();
            if (P.flip) {
                Z2_CUDA(ctx, launch_flip_all(c128, state, g.n, ctx->sm_count * 8, st));
                ctx->launches += 1;
            }
            return Z2_OK;
        }
        const int smem = tma_smem_bytes(c128, g.tb);
        const int per_sm = std::max(1, std::min(8, (227 * 1024) / (smem + 1024)));
        const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->sm_count * per_sm);
        if (single) {
            Z2_CUDA(ctx, launch_pass_tma(c128, g.tb, P.op, P.args[0], &tmaps[0], P.d_steps, (int)P.passes.size(),
                                         P.d_tables, ctx->d_err, grid, st));
            ctx->launches += 1;
        } else {
            for (size_t i = 0; i < P.passes.size(); ++i) {
                const int gi = P.passes[i].group;
                const void *sp = static_cast<const char *>(P.d_steps) + i * step_bytes;
                Z2_CUDA(ctx, launch_pass_tma(c128, g.tb, P.op, P.args[gi], &tmaps[gi], sp, 1, P.d_tables,
                                             ctx->d_err, grid, st));
            }
            ctx->launches += P.passes.size();
        }
    } else if (!P.passes.empty()) {
        const int grid = (int)std::min<uint64_t>(ntiles, 1u << 20);
        if (single) {
            // single tile: the whole pass list in one launch, state held in registers
            Z2_CUDA(ctx, launch_pass_steps(c128, g.tb, P.op, state, P.args[0], P.d_steps, (int)P.passes.size(),
                                           P.d_tables, 0, grid, st));
            ctx->launches += 1;
        } else {
            // complex64: the passes in between keep the state in the split-pair
            // format; the first converts from, the last back to, (re, im) pairs
            const size_t last = P.passes.size() - 1;
            for (size_t i = 0; i < P.passes.size(); ++i) {
                const void *sp = static_cast<const char *>(P.d_steps) + i * step_bytes;
                const int fmt = c128 ? 0 : ((i > 0 ? 1 : 0) | (i < last ? 2 : 0));
                const int gi = P.passes[i].group;
                const int tb = g.groups[gi].tb;
                const int gr_grid = (int)std::min<uint64_t>(1ull << (g.n - tb), 1u << 20);
                Z2_CUDA(ctx, launch_pass_steps(c128, tb, P.op, state, P.args[gi], sp, 1, P.d_tables, fmt, gr_grid,
                                               st));
            }
            ctx->launches += P.passes.size();
        }
    }
    if (P.flip) {
        Z2_CUDA(ctx, launch_flip_all(c128, state, g.n, ctx->sm_count * 8, st));
        ctx->launches += 1;
    }
    return Z2_OK;
}

int check_device_error(z2_ctx *ctx) {
    int flag = 0;
    Z2_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return fail(ctx, Z2_ERR_DEVICE_TIMEOUT, "a bounded device-side wait gave up; results are invalid");
    }
    return Z2_OK;
}

std::string plan_key(const z2_ctx *ctx, const char *kind, const Lattice &lat, const z2_run_params *p, int a, int b,
                     double x) {
    // the effective tile size and kernel variant are part of the key
    const auto ch = exec_choice(ctx, lat.n_links, p ? p->precision : 0);
    char buf[320];
    std::snprintf(buf, sizeof(buf), "%s|%d|%d,%d,%d|%a|%a|%d|%d|%d|%d|%d|%d|%a|tb%d|v%d|s%d", kind, lat.d, lat.L[0],
                  lat.L[1], lat.L[2], p ? p->lambda : 0.0, p ? p->T : 0.0, p ? p->M : 0, p ? p->decomp : 0,
                  p ? p->precision : 0, p ? p->sampling : 0, a, b, x, ch.first, ch.second, ctx->split_low);
    return buf;
}

int check_params(z2_ctx *ctx, const z2_run_params *p) {
    if (!p) return fail(ctx, Z2_ERR_ARG, "run parameters are NULL");
    if (p->M < 1) return fail(ctx, Z2_ERR_ARG, "M must be >= 1");
    if (p->decomp != Z2_FIRST_ORDER && p->decomp != Z2_SYMMETRIC) return fail(ctx, Z2_ERR_ARG, "bad decomposition");
    if (p->precision != Z2_C64 && p->precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (p->sampling != Z2_SAMPLE_STD && p->sampling != Z2_SAMPLE_PAPER) return fail(ctx, Z2_ERR_ARG, "bad sampling");
    if (!std::isfinite(p->lambda) || !std::isfinite(p->T)) return fail(ctx, Z2_ERR_ARG, "lambda and T must be finite");
    return Z2_OK;
}

int check_state(z2_ctx *ctx, const void *state) {
    if (!state) return fail(ctx, Z2_ERR_ARG, "state pointer is NULL");
    if (reinterpret_cast<uintptr_t>(state) % 256) return fail(ctx, Z2_ERR_ARG, "state must be 256-byte aligned");
    return Z2_OK;
}

Plan *get_plan(z2_ctx *ctx, const std::string &key) {
    auto it = ctx->plans.find(key);
    return it == ctx->plans.end() ? nullptr : it->second.get();
}

// Hadamard layer plan: every group once, scale 2^{-k/2} per group pass.
int build_hadamard_plan(z2_ctx *ctx, const Lattice &lat, bool c128, Plan &P) {
    std::string err;
    const auto ch = exec_choice(ctx, lat.n_links, c128 ? Z2_C128 : Z2_C64);
    P.variant = ch.second;
    if (!plan_geometry(lat.n_links, c128, ch.first, ch.second, P.geo, err, encode_fn() != nullptr, ctx->split_low))
        return fail(ctx, Z2_ERR_LATTICE, err);
    P.op = OP_HADAMARD;
    for (int gi = 0; gi < (int)P.geo.groups.size(); ++gi) {
        HostPass hp{};
        hp.group = gi;
        hp.step.rot1 = P.geo.groups[gi].rot;
        hp.step.rot2 = 0;
        hp.step.mid = MID_SCALE;
        hp.step.table = -1;
        hp.step.scale = std::pow(2.0, -0.5 * P.geo.groups[gi].k);
        P.passes.push_back(hp);
    }
    return upload_plan(ctx, lat, P);
}

int ensure_plan(z2_ctx *ctx, const std::string &key, Plan *&out, const std::function<int(Plan &)> &build) {
    out = get_plan(ctx, key);
    if (out) return Z2_OK;
    auto P = std::make_unique<Plan>();
    int rc = build(*P);
    if (rc != Z2_OK) return rc;
    out = P.get();
    ctx->plans[key] = std::move(P);
    return Z2_OK;
}

}  // namespace
}  // namespace z2

using namespace z2;

static std::string gpu_name(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    std::string n(prop.name);
    for (auto &ch : n)
        if (ch == ' ') ch = '_';
    return n;
}

extern "C" {

const char *z2_version(void) { return "z2lgt 0.1 (sm_103a)"; }

const char *z2_last_error(const z2_ctx *ctx) { return ctx ? ctx->last_error.c_str() : g_last_error.c_str(); }

int z2_ctx_create(int device, z2_ctx **out) {
    if (!out) return fail(nullptr, Z2_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, Z2_ERR_CUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, Z2_ERR_ARG, "no such CUDA device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, Z2_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    auto ctx = std::make_unique<z2_ctx>();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_partials, reduce_partials_doubles(Z2_MAX_LINKS) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->d_out, OUT_DOUBLES * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_out, OUT_DOUBLES * sizeof(double)) != cudaSuccess) {
        if (ctx->d_partials) cudaFree(ctx->d_partials);
        if (ctx->d_out) cudaFree(ctx->d_out);
        return fail(nullptr, Z2_ERR_OOM, "context scratch allocation failed");
    }
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(ctx->d_partials);
        cudaFree(ctx->d_out);
        cudaFreeHost(ctx->h_out);
        return fail(nullptr, Z2_ERR_OOM, "context scratch allocation failed");
    }
    if (const char *path = std::getenv("Z2_TUNE_CACHE")) {
        // lines "<gpu> <qubits> <precision> <tile bits> <variant> <us per step>"; later lines win
        if (FILE *f = std::fopen(path, "r")) {
            const std::string me = gpu_name(device);
            char name[256];
            int n, prec, tb, var;
            double us;
            while (std::fscanf(f, "%255s %d %d %d %d %lf", name, &n, &prec, &tb, &var, &us) == 6)
                if (me == name && tb >= 0 && tb <= 14 && var >= 0 && var <= 5) ctx->tuned[{n, prec}] = {tb, var};
            std::fclose(f);
        }
    }
    if (const char *s = std::getenv("Z2_TILE_BITS")) ctx->tb_override = std::atoi(s);
    if (const char *s = std::getenv("Z2_PASS_VARIANT")) ctx->variant = std::string(s) == "direct" ? 1 : (std::string(s) == "tma" ? 2 : 0);
    *out = ctx.release();
    return Z2_OK;
}

int z2_ctx_destroy(z2_ctx *ctx) {
    if (!ctx) return Z2_OK;
    cudaSetDevice(ctx->device);
    ctx->plans.clear();
    if (ctx->d_partials) cudaFree(ctx->d_partials);
    if (ctx->d_out) cudaFree(ctx->d_out);
    if (ctx->h_out) cudaFreeHost(ctx->h_out);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return Z2_OK;
}

int z2_ctx_launch_count(const z2_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return fail(nullptr, Z2_ERR_ARG, "NULL argument");
    *out = ctx->launches;
    return Z2_OK;
}

int z2_ctx_flush_plans(z2_ctx *ctx) {
    if (!ctx) return fail(nullptr, Z2_ERR_ARG, "NULL argument");
    Z2_CUDA(ctx, cudaDeviceSynchronize());
    ctx->plans.clear();
    return Z2_OK;
}

int z2_ctx_set_option(z2_ctx *ctx, int32_t option, int32_t value) {
    if (!ctx) return fail(nullptr, Z2_ERR_ARG, "NULL argument");
    if (option == Z2_OPT_TILE_BITS) {
        if (value != 0 && (value < 8 || value > 14)) return fail(ctx, Z2_ERR_ARG, "tile bits must be 0 or 8..14");
        ctx->tb_override = value;
    } else if (option == Z2_OPT_SPLIT_LOW_BITS) {
        if (value < 0 || value > 8) return fail(ctx, Z2_ERR_ARG, "split width must be 0 (automatic) or 1..8");
        ctx->split_low = value;
    } else if (option == Z2_OPT_PASS_VARIANT) {
        if (value < 0 || value > 5) return fail(ctx, Z2_ERR_ARG, "pass variant must be 0..5");
        ctx->variant = value;
    } else if (option == Z2_OPT_GANG_WAIT_POLLS) {
        if (value < 0) return fail(ctx, Z2_ERR_ARG, "gang wait polls must be >= 0 (0 = default)");
        ctx->gang_wait_polls = (uint32_t)value;
        return Z2_OK;  // no plan depends on it
    } else {
        return fail(ctx, Z2_ERR_ARG, "unknown option");
    }
    Z2_CUDA(ctx, cudaDeviceSynchronize());
    ctx->plans.clear();
    return Z2_OK;
}

int z2_autotune(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, void *stream,
                z2_tune_result *out) {
    if (!ctx || !lat || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (int rc = check_state(ctx, state)) return rc;
    const int n = lat->lat.n_links;
    const bool c128 = precision == Z2_C128;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::pair<int, int>> cands;
    if (n <= tile_limit(c128)) {
        cands.push_back({0, 1});  // the whole state is one tile: nothing to choose
    } else {
        for (int tb = tile_limit(c128) - 2; tb <= tile_limit(c128); ++tb) {
            if (tb >= n) continue;
            cands.push_back({tb, 1});
            if (!c128 && tb >= 10 && tb <= 13) cands.push_back({tb, 3});
            if (!c128 && tb >= 12 && tb <= 13) cands.push_back({tb, 4});
            if (!c128 && tb >= 12 && tb <= 13) cands.push_back({tb, 5});
        }
    }
    const int saved_tb = ctx->tb_override, saved_var = ctx->variant;
    z2_run_params p{};
    const int S = 16;  // Trotter steps per timing (shorter samples misranked close candidates)
    p.lambda = 1.0;
    p.T = 0.04 * S;
    p.M = S;
    p.decomp = Z2_SYMMETRIC;
    p.precision = precision;
    double best = 1e300;
    std::pair<int, int> best_c = cands.front();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Z2_CUDA(ctx, cudaEventCreate(&e0));
    Z2_CUDA(ctx, cudaEventCreate(&e1));
    int rc = Z2_OK;
    for (auto c : cands) {
        ctx->tb_override = c.first;
        ctx->variant = c.second;
        if ((rc = z2_init_plus(ctx, lat, precision, state, st))) break;
        if ((rc = z2_evolve(ctx, lat, &p, state, 0, S, st))) break;  // builds the plan, warms up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && rc == Z2_OK; ++r) rc = z2_evolve(ctx, lat, &p, state, 0, S, st);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(ctx, Z2_ERR_CUDA, "autotune: event synchronisation failed");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double us = 1000.0 * ms / (3 * S);
        if (us < best) {
            best = us;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tb_override = saved_tb;
    ctx->variant = saved_var;
    if (rc) return rc;
    if (int e = check_device_error(ctx)) return e;
    ctx->tuned[{n, precision}] = best_c;
    out->tile_bits = best_c.first;
    out->variant = best_c.second;
    out->us_per_step = best;
    out->n_candidates = (int)cands.size();
    if (const char *path = std::getenv("Z2_TUNE_CACHE")) {
        if (FILE *f = std::fopen(path, "a")) {
            std::fprintf(f, "%s %d %d %d %d %.3f\n", gpu_name(ctx->device).c_str(), n, precision, best_c.first,
                         best_c.second, best);
            std::fclose(f);
        }
    }
    return Z2_OK;
}

int z2_evolve_plan_info(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, int32_t j0, int32_t j1,
                        z2_plan_info *out) {
    if (!ctx || !lat || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (int rc = check_params(ctx, p)) return rc;
    if (j0 < 0 || j1 > p->M || j0 > j1) return fail(ctx, Z2_ERR_ARG, "need 0 <= j0 <= j1 <= M");
    Plan *P = nullptr;
    const std::string key = plan_key(ctx, "evolve", lat->lat, p, j0, j1, 0);
    if (int rc = ensure_plan(ctx, key, P,
                             [&](Plan &Q) { return build_evolve_plan(ctx, lat->lat, *p, j0, j1, Q); }))
        return rc;
    out->tile_bits = P->geo.tb;
    out->n_groups = (int)P->geo.groups.size();
    out->n_passes = (int)P->passes.size();
    out->n_launches = (P->geo.groups.size() == 1 ? (P->passes.empty() ? 0 : 1) : (int)P->passes.size()) + (P->flip ? 1 : 0);
    out->n_tables = (int)(P->tables.size() / TABLE_STRIDE);
    out->flip = P->flip ? 1 : 0;
    out->low_tile_bits = P->geo.groups.empty() ? 0 : P->geo.groups[0].tb;
    return Z2_OK;
}

int z2_plan_geometry(int32_t n_qubits, int32_t precision, int32_t tile_bits, int32_t variant, int32_t assume_tma,
                     z2_group_info *groups, int32_t max_groups, int32_t *n_groups) {
    if (!groups || !n_groups) return fail(nullptr, Z2_ERR_ARG, "z2_plan_geometry: NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(nullptr, Z2_ERR_ARG, "bad precision");
    if (n_qubits < 8 || n_qubits > Z2_MAX_LINKS) return fail(nullptr, Z2_ERR_ARG, "n_qubits must be in 8..34");
    if (tile_bits != 0 && (tile_bits < 8 || tile_bits > 14)) return fail(nullptr, Z2_ERR_ARG, "tile bits must be 0 or 8..14");
    if (variant < 0 || variant > 5) return fail(nullptr, Z2_ERR_ARG, "pass variant must be 0..5");
    z2::Geometry g;
    std::string err;
    if (!z2::plan_geometry(n_qubits, precision == Z2_C128, tile_bits, variant, g, err, assume_tma != 0))
        return fail(nullptr, Z2_ERR_LATTICE, err);
    if ((int)g.groups.size() > max_groups) return fail(nullptr, Z2_ERR_ARG, "z2_plan_geometry: max_groups too small");
    for (size_t i = 0; i < g.groups.size(); ++i) {
        const auto &gr = g.groups[i];
        groups[i] = z2_group_info{gr.tb, gr.c, gr.b, gr.k, gr.k1, gr.k1 < gr.k ? gr.b2 : 0};
    }
    *n_groups = (int32_t)g.groups.size();
    return Z2_OK;
}

int z2_lattice_create(int32_t d, const int32_t *L, z2_lattice **out) {
    if (!out) return fail(nullptr, Z2_ERR_ARG, "out is NULL");
    *out = nullptr;
    auto lat = std::make_unique<z2_lattice>();
    std::string err;
    if (!build_lattice(d, L, lat->lat, err)) return fail(nullptr, Z2_ERR_LATTICE, err);
    *out = lat.release();
    return Z2_OK;
}

int z2_lattice_destroy(z2_lattice *lat) {
    delete lat;
    return Z2_OK;
}

int z2_lattice_info_get(const z2_lattice *lat, z2_lattice_info *out) {
    if (!lat || !out) return fail(nullptr, Z2_ERR_ARG, "NULL argument");
    out->d = lat->lat.d;
    for (int i = 0; i < 3; ++i) out->L[i] = i < lat->lat.d ? lat->lat.L[i] : 1;
    out->n_links = lat->lat.n_links;
    out->n_plaq = lat->lat.n_plaq;
    out->n_sites = lat->lat.n_sites;
    return Z2_OK;
}

int z2_lattice_masks(const z2_lattice *lat, int32_t kind, uint64_t *out, size_t cap, size_t *n) {
    if (!lat || !n) return fail(nullptr, Z2_ERR_ARG, "NULL argument");
    const Lattice &L = lat->lat;
    std::vector<uint64_t> v;
    switch (kind) {
        case Z2_MASK_PLAQ: v = L.plaq; break;
        case Z2_MASK_STAR: v = L.star; break;
        case Z2_MASK_WILSON_2X2: v = {L.wilson2x2}; break;
        case Z2_MASK_CONTOUR: v = {L.contour[0], L.contour[1], L.contour[2]}; break;
        case Z2_MASK_W_MU: v = L.wmu; break;
        case Z2_MASK_V_MU: v = L.vmu; break;
        default: return fail(nullptr, Z2_ERR_ARG, "unknown mask kind");
    }
    *n = v.size();
    if (cap < v.size() || (!out && !v.empty())) return fail(nullptr, Z2_ERR_ARG, "output capacity too small");
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
    return Z2_OK;
}

int z2_state_bytes(const z2_lattice *lat, int32_t precision, size_t *bytes) {
    if (!lat || !bytes) return fail(nullptr, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(nullptr, Z2_ERR_ARG, "bad precision");
    *bytes = (precision == Z2_C128 ? 16ull : 8ull) << lat->lat.n_links;
    return Z2_OK;
}

int z2_init_plus(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (int rc = check_state(ctx, state)) return rc;
    Z2_CUDA(ctx, launch_init_plus(precision == Z2_C128, state, lat->lat.n_links, ctx->sm_count * 16,
                                  (cudaStream_t)stream));
    ctx->launches += 1;
    return Z2_OK;
}

int z2_evolve(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, void *state, int32_t j0, int32_t j1,
              void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (int rc = check_params(ctx, p)) return rc;
    if (int rc = check_state(ctx, state)) return rc;
    if (j0 < 0 || j1 > p->M || j0 > j1) return fail(ctx, Z2_ERR_ARG, "need 0 <= j0 <= j1 <= M");
    if (j0 == j1) return Z2_OK;
    Plan *P = nullptr;
    const std::string key = plan_key(ctx, "evolve", lat->lat, p, j0, j1, 0);
    if (int rc = ensure_plan(ctx, key, P,
                             [&](Plan &Q) { return build_evolve_plan(ctx, lat->lat, *p, j0, j1, Q); }))
        return rc;
    return exec_plan(ctx, *P, state, (cudaStream_t)stream);
}

int z2_apply_plaquettes(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, double theta,
                        void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (int rc = check_state(ctx, state)) return rc;
    Plan *P = nullptr;
    z2_run_params pp{};
    pp.precision = precision;
    const std::string key = plan_key(ctx, "plaq", lat->lat, &pp, 0, 0, theta);
    if (int rc = ensure_plan(ctx, key, P, [&](Plan &Q) {
            std::string err;
            const auto ch = exec_choice(ctx, lat->lat.n_links, precision);
            Q.variant = ch.second;
            if (!plan_geometry(lat->lat.n_links, precision == Z2_C128, ch.first, ch.second, Q.geo, err,
                               encode_fn() != nullptr, ctx->split_low))
                return fail(ctx, Z2_ERR_LATTICE, err);
            Q.op = OP_RX_TAN;
            push_table(Q, lat->lat, theta, {1, 0});
            HostPass hp{};
            hp.group = 0;
            hp.step.mid = MID_TABLE;
            hp.step.table = 0;
            hp.step.scale = 1;
            Q.passes.push_back(hp);
            return upload_plan(ctx, lat->lat, Q);
        }))
        return rc;
    return exec_plan(ctx, *P, state, (cudaStream_t)stream);
}

int z2_apply_rx_layer(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, double dt, void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (!std::isfinite(dt)) return fail(ctx, Z2_ERR_ARG, "dt must be finite");
    if (int rc = check_state(ctx, state)) return rc;
    Plan *P = nullptr;
    z2_run_params pp{};
    pp.precision = precision;
    const std::string key = plan_key(ctx, "rx", lat->lat, &pp, 0, 0, dt);
    if (int rc = ensure_plan(ctx, key, P, [&](Plan &Q) {
            std::string err;
            const auto ch = exec_choice(ctx, lat->lat.n_links, precision);
            Q.variant = ch.second;
            if (!plan_geometry(lat->lat.n_links, precision == Z2_C128, ch.first, ch.second, Q.geo, err,
                               encode_fn() != nullptr, ctx->split_low))
                return fail(ctx, Z2_ERR_LATTICE, err);
            Q.op = OP_RX_TAN;
            const GateSplit gs = split_gate(dt);
            std::vector<Event> ev;
            std::complex<double> sc(1, 0);
            for (int gi : Q.geo.order) {
                ev.push_back({0, gi, -1, gs.t});
                const int bits = Q.geo.groups[gi].k;
                sc *= std::pow(gs.c, bits) * ipow(gs.q * bits);
            }
            push_table(Q, lat->lat, 0.0, sc);
            ev.push_back({1, 0, 0});
            pack_passes(ev, Q.geo, Q.passes);
            Q.flip = gs.q & 1;
            return upload_plan(ctx, lat->lat, Q);
        }))
        return rc;
    return exec_plan(ctx, *P, state, (cudaStream_t)stream);
}

int z2_apply_hadamard(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (int rc = check_state(ctx, state)) return rc;
    Plan *P = nullptr;
    z2_run_params pp{};
    pp.precision = precision;
    const std::string key = plan_key(ctx, "had", lat->lat, &pp, 0, 0, 0);
    if (int rc = ensure_plan(ctx, key, P,
                             [&](Plan &Q) { return build_hadamard_plan(ctx, lat->lat, precision == Z2_C128, Q); }))
        return rc;
    return exec_plan(ctx, *P, state, (cudaStream_t)stream);
}

struct Scratch {
    double *d_partials;  // reduction partials (reduce_partials_doubles(n) or more)
    double *d_out;       // reduction outputs (OUT_DOUBLES)
    double *h_out;       // pinned copy of d_out
};

static Scratch ctx_scratch(z2_ctx *ctx) { return Scratch{ctx->d_partials, ctx->d_out, ctx->h_out}; }

static int zsums_device(z2_ctx *ctx, const Scratch &sc, int n, bool c128, const void *state, const uint64_t *masks,
                        int n_masks, int out_off, cudaStream_t st) {
    const int chunk = max_zsum_masks();
    for (int k = 0; k < n_masks; k += chunk) {
        const int m = std::min(chunk, n_masks - k);
        Z2_CUDA(ctx, launch_zsums(c128, state, n, masks + k, m, sc.d_partials, sc.d_out + out_off + k, st));
        ctx->launches += zsums_launches(n, m);
    }
    return Z2_OK;
}

int z2_zsums(z2_ctx *ctx, int32_t n_qubits, int32_t precision, const void *state, const uint64_t *masks,
             int32_t n_masks, double *out, void *stream) {
    if (!ctx || !masks || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (n_qubits < 8 || n_qubits > Z2_MAX_LINKS) return fail(ctx, Z2_ERR_ARG, "need 8 <= n_qubits <= 34");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (n_masks < 0 || n_masks > OUT_DOUBLES) return fail(ctx, Z2_ERR_ARG, "need 0 <= n_masks <= 256");
    if (int rc = check_state(ctx, state)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = zsums_device(ctx, ctx_scratch(ctx), n_qubits, precision == Z2_C128, state, masks, n_masks, 0, st))
        return rc;
    Z2_CUDA(ctx, cudaMemcpyAsync(ctx->h_out, ctx->d_out, n_masks * sizeof(double), cudaMemcpyDeviceToHost, st));
    Z2_CUDA(ctx, cudaStreamSynchronize(st));
    std::memcpy(out, ctx->h_out, n_masks * sizeof(double));
    return Z2_OK;
}

int z2_dos(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, int32_t kind, double *out,
           int32_t cap, int32_t *n_bins, void *stream) {
    if (!ctx || !lat || !out || !n_bins) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (kind != Z2_DOS_Z && kind != Z2_DOS_X) return fail(ctx, Z2_ERR_ARG, "kind must be Z2_DOS_Z or Z2_DOS_X");
    if (int rc = check_state(ctx, state)) return rc;
    const Lattice &L = lat->lat;
    const int n = L.n_links;
    const int want = (kind == Z2_DOS_Z ? L.n_plaq : n) + 1;
    if (cap < want) return fail(ctx, Z2_ERR_ARG, "z2_dos: out holds " + std::to_string(cap) + " bins, needs " +
                                                     std::to_string(want));
    cudaStream_t st = (cudaStream_t)stream;
    const bool c128 = precision == Z2_C128;
    int nb = 0;
    if (kind == Z2_DOS_Z) {
        Z2_CUDA(ctx, launch_dos(c128, state, n, L.plaq.data(), (int)L.plaq.size(), ctx->d_partials, ctx->d_out, &nb,
                                st));
        ctx->launches += 2;
    } else {
        // to the sigma^x basis and back (Sec. 2.4, H sigma^z H = sigma^x)
        if (int rc = z2_apply_hadamard(ctx, lat, precision, state, st)) return rc;
        Z2_CUDA(ctx, launch_dos(c128, state, n, nullptr, 0, ctx->d_partials, ctx->d_out, &nb, st));
        ctx->launches += 2;
        if (int rc = z2_apply_hadamard(ctx, lat, precision, state, st)) return rc;
    }
    Z2_CUDA(ctx, cudaMemcpyAsync(ctx->h_out, ctx->d_out, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    Z2_CUDA(ctx, cudaStreamSynchronize(st));
    std::memcpy(out, ctx->h_out, nb * sizeof(double));
    *n_bins = nb;
    return check_device_error(ctx);
}

int z2_overlap(z2_ctx *ctx, int32_t n_qubits, int32_t precision, const void *a, const void *b, double *out,
               void *stream) {
    if (!ctx || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (n_qubits < 8 || n_qubits > Z2_MAX_LINKS) return fail(ctx, Z2_ERR_ARG, "need 8 <= n_qubits <= 34");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (int rc = check_state(ctx, a)) return rc;
    if (int rc = check_state(ctx, b)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Z2_CUDA(ctx, launch_overlap(precision == Z2_C128, a, b, n_qubits, ctx->d_partials, ctx->d_out, st));
    ctx->launches += 2;
    Z2_CUDA(ctx, cudaMemcpyAsync(ctx->h_out, ctx->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    Z2_CUDA(ctx, cudaStreamSynchronize(st));
    out[0] = ctx->h_out[0];
    out[1] = ctx->h_out[1];
    return Z2_OK;
}

// Observable masks of a lattice: sigma^z-type (norm, plaquettes, 2x2 loop,
// contours, W_mu, sigma^z_l) and sigma^x-type (sigma^x_l, stars, V_mu).
static void observable_masks(const Lattice &L, std::vector<uint64_t> &zm, std::vector<uint64_t> &xm) {
    const int n = L.n_links;
    zm.clear();
    xm.clear();
    zm.push_back(0);
    for (auto m : L.plaq) zm.push_back(m);
    zm.push_back(L.wilson2x2);
    for (int k = 0; k < 3; ++k) zm.push_back(L.contour[k]);
    for (auto m : L.wmu) zm.push_back(m);
    for (int l = 0; l < n; ++l) zm.push_back(uint64_t(1) << l);
    for (int l = 0; l < n; ++l) xm.push_back(uint64_t(1) << l);
    for (auto m : L.star) xm.push_back(m);
    for (auto m : L.vmu) xm.push_back(m);
}

// Enqueue every reduction of z2_measure on `st` into sc.d_out and its copy
// to sc.h_out (no synchronisation).  Returns the number of doubles copied.
static int measure_enqueue(z2_ctx *ctx, const z2_lattice *lat, int precision, void *state, const void *ref,
                           cudaStream_t st, const Scratch &sc, int *n_out) {
    const Lattice &L = lat->lat;
    const int n = L.n_links;
    const bool c128 = precision == Z2_C128;
    std::vector<uint64_t> zm, xm;
    observable_masks(L, zm, xm);
    const int nz = (int)zm.size(), nx = (int)xm.size();
    const int off_fid = nz + nx;  // <ref|psi> (2 doubles), then <ref|ref> (2 doubles)
    if (off_fid + 4 > OUT_DOUBLES) return fail(ctx, Z2_ERR_LATTICE, "too many observables");
    if (int rc = zsums_device(ctx, sc, n, c128, state, zm.data(), nz, 0, st)) return rc;
    if (ref) {
        Z2_CUDA(ctx, launch_overlap(c128, ref, state, n, sc.d_partials, sc.d_out + off_fid, st));
        Z2_CUDA(ctx, launch_overlap(c128, ref, ref, n, sc.d_partials, sc.d_out + off_fid + 2, st));
        ctx->launches += 4;
    }
    if (int rc = z2_apply_hadamard(ctx, lat, precision, state, st)) return rc;
    if (int rc = zsums_device(ctx, sc, n, c128, state, xm.data(), nx, nz, st)) return rc;
    if (int rc = z2_apply_hadamard(ctx, lat, precision, state, st)) return rc;
    Z2_CUDA(ctx, cudaMemcpyAsync(sc.h_out, sc.d_out, (off_fid + 4) * sizeof(double), cudaMemcpyDeviceToHost, st));
    *n_out = off_fid + 4;
    return Z2_OK;
}

// Turn the raw sums of measure_enqueue into the results struct.
// gform: the energy is the paper's <H(g)> = -sum<U_p> - g sum<sigma^x_l> with
// g = s (Sec. 2.2), else <H(s)> = -sum<sigma^x_l> - s lambda sum<U_p>.
static void measure_finish(const Lattice &L, double lambda, double s, const double *h, bool has_ref, z2_results *out,
                           bool gform = false) {
    const int n = L.n_links, np = L.n_plaq;
    std::vector<uint64_t> zm, xm;
    observable_masks(L, zm, xm);
    const int nz = (int)zm.size(), nx = (int)xm.size();
    const int off_fid = nz + nx;
    std::memset(out, 0, sizeof(*out));
    const double nan = std::nan("");
    // expectation values <psi|O|psi> / <psi|psi>: the norm differs from 1 only
    // by rounding, and is reported as measured
    const double nrm = h[0];
    const double inv = nrm > 0 ? 1.0 / nrm : nan;
    out->s = s;
    out->norm = nrm;
    double sp = 0;
    for (int k = 0; k < np; ++k) {
        out->plaq[k] = h[1 + k] * inv;
        sp += out->plaq[k];
    }
    out->mean_plaq = sp / np;
    out->wilson_2x2 = L.wilson_degenerate ? nan : h[1 + np] * inv;
    if (L.wilson_degenerate) out->flags |= Z2_FLAG_WILSON_DEGENERATE;
    for (int k = 0; k < 3; ++k) {
        out->contours[k] = L.contour_degenerate[k] ? nan : h[2 + np + k] * inv;
        if (L.contour_degenerate[k]) out->flags |= Z2_FLAG_CONTOUR_DEGENERATE;
    }
    for (int mu = 0; mu < L.d; ++mu) out->wmu[mu] = h[5 + np + mu] * inv;
    for (int l = 0; l < n; ++l) out->sigmaz[l] = h[5 + np + L.d + l] * inv;
    double sx = 0;
    for (int l = 0; l < n; ++l) {
        out->sigmax[l] = h[nz + l] * inv;
        sx += out->sigmax[l];
    }
    double ss = 0;
    for (int k = 0; k < L.n_sites; ++k) {
        out->star[k] = h[nz + n + k] * inv;
        ss += out->star[k];
    }
    out->mean_star = ss / L.n_sites;
    for (int mu = 0; mu < L.d; ++mu) out->vmu[mu] = h[nz + n + L.n_sites + mu] * inv;
    out->energy = gform ? -sp - s * sx : -sx - s * lambda * sp;
    if (has_ref) {
        // |<ref|psi>|^2 / (<ref|ref> <psi|psi>)
        const double rn = h[off_fid + 2];
        out->fidelity = (h[off_fid] * h[off_fid] + h[off_fid + 1] * h[off_fid + 1]) / (rn * nrm);
    } else {
        out->fidelity = nan;
        out->flags |= Z2_FLAG_NO_FIDELITY;
    }
    out->status = Z2_OK;
}

int z2_measure(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, void *state, double s, const void *ref,
               void *stream, z2_results *out) {
    if (!ctx || !lat || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (int rc = check_params(ctx, p)) return rc;
    if (int rc = check_state(ctx, state)) return rc;
    if (ref)
        if (int rc = check_state(ctx, ref)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int n_out = 0;
    if (int rc = measure_enqueue(ctx, lat, p->precision, state, ref, st, ctx_scratch(ctx), &n_out)) return rc;
    Z2_CUDA(ctx, cudaStreamSynchronize(st));
    if (int rc = check_device_error(ctx)) return rc;
    measure_finish(lat->lat, p->lambda, s, ctx->h_out, ref != nullptr, out);
    return Z2_OK;
}

int z2_run(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, void *state, const void *ref, void *stream,
           z2_results *out) {
    if (int rc = check_params(ctx, p)) return rc;
    if (int rc = z2_init_plus(ctx, lat, p->precision, state, stream)) return rc;
    if (int rc = z2_evolve(ctx, lat, p, state, 0, p->M, stream)) return rc;
    return z2_measure(ctx, lat, p, state, 1.0, ref, stream, out);
}

// ---------------------------------------------------------------------------
// The paper's own schedule (Sec. 2.2-2.4): projected start, g ramp.

static int check_gramp(z2_ctx *ctx, const z2_gramp_params *gp) {
    if (!gp) return fail(ctx, Z2_ERR_ARG, "ramp parameters are NULL");
    if (gp->N_s < 1 || gp->n < 1) return fail(ctx, Z2_ERR_ARG, "need N_s >= 1 and n >= 1");
    if ((int64_t)gp->N_s * gp->n > (1 << 24)) return fail(ctx, Z2_ERR_ARG, "N_s * n exceeds 2^24 substeps");
    if (gp->decomp != Z2_FIRST_ORDER && gp->decomp != Z2_SYMMETRIC) return fail(ctx, Z2_ERR_ARG, "bad decomposition");
    if (gp->precision != Z2_C64 && gp->precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (!std::isfinite(gp->g_s) || !std::isfinite(gp->t_s)) return fail(ctx, Z2_ERR_ARG, "g_s and t_s must be finite");
    return Z2_OK;
}

int z2_init_projected(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, uint32_t sectors, void *state,
                      void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (int rc = check_state(ctx, state)) return rc;
    const Lattice &L = lat->lat;
    if (sectors >> L.d) return fail(ctx, Z2_ERR_ARG, "sector bits beyond the lattice dimension");
    // H^N prod_p (1 + U_p)/2 |+>^N = prod_p (1 + X_p)/2 |0>: uniform over the
    // span of the plaquette masks; W_mu = prod sigma^z along its loop becomes
    // the index shift by w_mu
    const std::vector<uint64_t> basis = gf2_basis(L.plaq);
    uint64_t offset = 0;
    for (int mu = 0; mu < L.d; ++mu)
        if ((sectors >> mu) & 1u) offset ^= L.wmu[mu];
    cudaStream_t st = (cudaStream_t)stream;
    Z2_CUDA(ctx, launch_span_state(precision == Z2_C128, state, L.n_links, basis.data(), (int)basis.size(), offset,
                                   ctx->sm_count * 16, st));
    ctx->launches += 2;
    return z2_apply_hadamard(ctx, lat, precision, state, stream);
}

int z2_evolve_gramp(z2_ctx *ctx, const z2_lattice *lat, const z2_gramp_params *gp, void *state, int32_t k0, int32_t k1,
                    void *stream) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (int rc = check_gramp(ctx, gp)) return rc;
    if (int rc = check_state(ctx, state)) return rc;
    if (k0 < 0 || k1 > gp->N_s || k0 > k1) return fail(ctx, Z2_ERR_ARG, "need 0 <= k0 <= k1 <= N_s");
    if (k0 == k1) return Z2_OK;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "|gramp|%a|%a|%d|%d|%d|%d", gp->g_s, gp->t_s, gp->N_s, gp->n, gp->decomp,
                  gp->precision);
    z2_run_params pp{};
    pp.precision = gp->precision;
    const std::string key = plan_key(ctx, "gramp", lat->lat, &pp, k0, k1, 0) + buf;
    Plan *P = nullptr;
    if (int rc = ensure_plan(ctx, key, P, [&](Plan &Q) { return build_gramp_plan(ctx, lat->lat, *gp, k0, k1, Q); }))
        return rc;
    return exec_plan(ctx, *P, state, (cudaStream_t)stream);
}

int z2_measure_gramp(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, double g, void *state, const void *ref,
                     void *stream, z2_results *out) {
    if (!ctx || !lat || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (!std::isfinite(g)) return fail(ctx, Z2_ERR_ARG, "g must be finite");
    if (int rc = check_state(ctx, state)) return rc;
    if (ref)
        if (int rc = check_state(ctx, ref)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int n_out = 0;
    if (int rc = measure_enqueue(ctx, lat, precision, state, ref, st, ctx_scratch(ctx), &n_out)) return rc;
    Z2_CUDA(ctx, cudaStreamSynchronize(st));
    if (int rc = check_device_error(ctx)) return rc;
    measure_finish(lat->lat, 0.0, g, ctx->h_out, ref != nullptr, out, true);
    return Z2_OK;
}

int z2_run_gramp(z2_ctx *ctx, const z2_lattice *lat, const z2_gramp_params *gp, uint32_t sectors, void *state,
                 const void *ref, void *stream, z2_results *out) {
    if (int rc = check_gramp(ctx, gp)) return rc;
    if (int rc = z2_init_projected(ctx, lat, gp->precision, sectors, state, stream)) return rc;
    if (int rc = z2_evolve_gramp(ctx, lat, gp, state, 0, gp->N_s, stream)) return rc;
    return z2_measure_gramp(ctx, lat, gp->precision, gp->N_s * gp->g_s, state, ref, stream, out);
}

// ---------------------------------------------------------------------------
// Phase estimation (Sec. 2.4, Eq. leap): U(t) = |0><0| (x) exp(-iHt) +
// |1><1| (x) exp(iHt) for H = Z + g X at fixed g.  The control qubit is index
// bit N, so the two halves of the state are the two branches: the first
// evolves for +t, the second for -t, by the same n-step Trotter formula.

int z2_controlled_evolution(z2_ctx *ctx, const z2_lattice *lat, const z2_qpe_params *qp, void *state, void *stream) {
    if (!ctx || !lat || !qp) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (qp->n < 1 || qp->n > (1 << 24)) return fail(ctx, Z2_ERR_ARG, "need 1 <= n <= 2^24");
    if (qp->decomp != Z2_FIRST_ORDER && qp->decomp != Z2_SYMMETRIC) return fail(ctx, Z2_ERR_ARG, "bad decomposition");
    if (qp->precision != Z2_C64 && qp->precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (!std::isfinite(qp->g) || !std::isfinite(qp->t)) return fail(ctx, Z2_ERR_ARG, "g and t must be finite");
    if (lat->lat.n_links + 1 > Z2_MAX_LINKS) return fail(ctx, Z2_ERR_LATTICE, "no room for the control qubit");
    if (int rc = check_state(ctx, state)) return rc;
    const size_t half_bytes = (size_t)(qp->precision == Z2_C128 ? 16 : 8) << lat->lat.n_links;
    for (int dir = 0; dir < 2; ++dir) {
        const double t = dir ? -qp->t : qp->t, tau = t / qp->n, g = qp->g;
        char buf[200];
        std::snprintf(buf, sizeof(buf), "|qpe|%a|%a|%d|%d|%d", g, t, qp->n, qp->decomp, qp->precision);
        z2_run_params pp{};
        pp.precision = qp->precision;
        const std::string key = plan_key(ctx, "qpe", lat->lat, &pp, 0, 0, 0) + buf;
        Plan *P = nullptr;
        if (int rc = ensure_plan(ctx, key, P, [&](Plan &Q) {
                return build_substep_plan(ctx, lat->lat, qp->precision, qp->decomp == Z2_SYMMETRIC, tau, 0, qp->n,
                                          [&](int64_t) { return g * tau; }, Q);
            }))
            return rc;
        void *half = static_cast<char *>(state) + (dir ? half_bytes : 0);
        if (int rc = exec_plan(ctx, *P, half, (cudaStream_t)stream)) return rc;
    }
    return Z2_OK;
}

// ---------------------------------------------------------------------------
// Gate-level execution (Sec. 2.3, Eq. ara, Figs. 3 and 4).

static int gate_matrix(int kind, double angle, double m[8]) {
    const double c = std::cos(angle / 2), s = std::sin(angle / 2), r = std::sqrt(0.5);
    switch (kind) {
        case Z2_GATE_RZ:  // exp(-i angle sigma^z / 2)
            m[0] = c, m[1] = -s, m[2] = 0, m[3] = 0, m[4] = 0, m[5] = 0, m[6] = c, m[7] = s;
            return Z2_OK;
        case Z2_GATE_RX:  // exp(-i angle sigma^x / 2)
            m[0] = c, m[1] = 0, m[2] = 0, m[3] = -s, m[4] = 0, m[5] = -s, m[6] = c, m[7] = 0;
            return Z2_OK;
        case Z2_GATE_H:
            m[0] = r, m[1] = 0, m[2] = r, m[3] = 0, m[4] = r, m[5] = 0, m[6] = -r, m[7] = 0;
            return Z2_OK;
        default:
            return Z2_ERR_ARG;
    }
}

static int enqueue_gate(z2_ctx *ctx, int n, bool c128, void *state, int kind, int q0, int q1, double angle,
                        cudaStream_t st) {
    double m[8] = {};
    if (kind != Z2_GATE_CNOT && gate_matrix(kind, angle, m) != Z2_OK) return fail(ctx, Z2_ERR_ARG, "unknown gate");
    Z2_CUDA(ctx, launch_gate(c128, state, n, kind == Z2_GATE_CNOT ? 0 : 1, q0, q1, m, ctx->sm_count * 8, st));
    ctx->launches += 1;
    return Z2_OK;
}

int z2_apply_gate(z2_ctx *ctx, int32_t n_qubits, int32_t precision, void *state, int32_t kind, int32_t q0, int32_t q1,
                  double angle, void *stream) {
    if (!ctx) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (n_qubits < 2 || n_qubits > Z2_MAX_LINKS + 1) return fail(ctx, Z2_ERR_ARG, "need 2 <= n_qubits <= 35");
    if (precision != Z2_C64 && precision != Z2_C128) return fail(ctx, Z2_ERR_ARG, "bad precision");
    if (q0 < 0 || q0 >= n_qubits) return fail(ctx, Z2_ERR_ARG, "qubit out of range");
    if (kind == Z2_GATE_CNOT && (q1 < 0 || q1 >= n_qubits || q1 == q0))
        return fail(ctx, Z2_ERR_ARG, "CNOT needs a target qubit other than the control");
    if (!std::isfinite(angle)) return fail(ctx, Z2_ERR_ARG, "angle must be finite");
    if (int rc = check_state(ctx, state)) return rc;
    return enqueue_gate(ctx, n_qubits, precision == Z2_C128, state, kind, q0, q1, angle, (cudaStream_t)stream);
}

// exp(-i Z tau) = prod_p exp(-i Z_p tau), each plaquette through the ancilla
// (bit N, in |0>): CNOT from each of its links onto the ancilla, R_z(-2 tau)
// on the ancilla, the CNOTs again in reverse order (Eq. ara, Fig. 3)
static int enqueue_plaquettes_circuit(z2_ctx *ctx, const Lattice &L, bool c128, void *state, double tau,
                                      cudaStream_t st, uint64_t &gates) {
    const int n = L.n_links + 1, a = L.n_links;
    for (uint64_t m : L.plaq) {
        int links[64], k = 0;
        for (int l = 0; l < L.n_links; ++l)
            if ((m >> l) & 1ull) links[k++] = l;
        for (int i = 0; i < k; ++i)
            if (int rc = enqueue_gate(ctx, n, c128, state, Z2_GATE_CNOT, links[i], a, 0, st)) return rc;
        if (int rc = enqueue_gate(ctx, n, c128, state, Z2_GATE_RZ, a, -1, -2.0 * tau, st)) return rc;
        for (int i = k - 1; i >= 0; --i)
            if (int rc = enqueue_gate(ctx, n, c128, state, Z2_GATE_CNOT, links[i], a, 0, st)) return rc;
        gates += 2 * k + 1;
    }
    return Z2_OK;
}

int z2_evolve_gramp_circuit(z2_ctx *ctx, const z2_lattice *lat, const z2_gramp_params *gp, void *state, int32_t k0,
                            int32_t k1, void *stream, uint64_t *n_gates) {
    if (!ctx || !lat) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (int rc = check_gramp(ctx, gp)) return rc;
    if (int rc = check_state(ctx, state)) return rc;
    if (k0 < 0 || k1 > gp->N_s || k0 > k1) return fail(ctx, Z2_ERR_ARG, "need 0 <= k0 <= k1 <= N_s");
    const Lattice &L = lat->lat;
    if (L.n_links + 1 > Z2_MAX_LINKS) return fail(ctx, Z2_ERR_LATTICE, "no room for the ancilla");
    const bool c128 = gp->precision == Z2_C128, sym = gp->decomp == Z2_SYMMETRIC;
    cudaStream_t st = (cudaStream_t)stream;
    const double tau = gp->t_s / gp->n;
    uint64_t gates = 0;
    for (int64_t j = (int64_t)k0 * gp->n + 1; j <= (int64_t)k1 * gp->n; ++j) {
        const double g = (double)j * gp->g_s / gp->n;
        if (sym)
            if (int rc = enqueue_plaquettes_circuit(ctx, L, c128, state, tau / 2, st, gates)) return rc;
        // exp(-i g X tau) = prod_l exp(i g tau sigma^x_l) = prod_l R_x(-2 g tau)
        for (int l = 0; l < L.n_links; ++l)
            if (int rc = enqueue_gate(ctx, L.n_links + 1, c128, state, Z2_GATE_RX, l, -1, -2.0 * g * tau, st)) return rc;
        gates += L.n_links;
        if (int rc = enqueue_plaquettes_circuit(ctx, L, c128, state, sym ? tau / 2 : tau, st, gates)) return rc;
    }
    if (n_gates) *n_gates = gates;
    return Z2_OK;
}

// ---------------------------------------------------------------------------
// Batched runs.  A slot is a stream with its own state buffer and reduction
// scratch; runs on one slot execute in stream order, slots run concurrently.
struct RunSlot {
    cudaStream_t st = nullptr;
    void *state = nullptr;
    double *d_partials = nullptr, *d_out = nullptr;
};

static void free_slots(std::vector<RunSlot> &slots) {
    for (auto &sl : slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.state) cudaFree(sl.state);
        if (sl.d_partials) cudaFree(sl.d_partials);
        if (sl.d_out) cudaFree(sl.d_out);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    slots.clear();
}

// |+>, the M steps and the observable reductions of one run, enqueued on st;
// `after_init` (optional) is recorded once the |+> kernel has run
static int enqueue_run(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params &p, void *state, cudaStream_t st,
                       const Scratch &sc, cudaEvent_t after_init = nullptr) {
    if (int rc = z2_init_plus(ctx, lat, p.precision, state, st)) return rc;
    if (after_init) Z2_CUDA(ctx, cudaEventRecord(after_init, st));
    if (int rc = z2_evolve(ctx, lat, &p, state, 0, p.M, st)) return rc;
    int n_out = 0;
    return measure_enqueue(ctx, lat, p.precision, state, nullptr, st, sc, &n_out);
}

// runs of this many qubits or more fill every SM with one pass kernel of their
// own plan (ring tiles), faster than the persistent kernel's fixed tiles
constexpr int PERSIST_MAX_QUBITS = 22;

static int sweep_persistent(z2_ctx *ctx, const z2_run_spec *specs, int32_t n, int32_t n_streams, z2_results *out) {
    const int PT = persist_tile_bits();
    // lattices and, for the runs the persistent kernel takes, plans with its tile size
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<z2_lattice>> lats;
    std::vector<const z2_lattice *> lat_of(n);
    std::vector<Plan *> plan_of(n, nullptr);
    std::vector<char> persist(n, 0);
    size_t total = 0;
    int max_n = 8;
    const int saved_tb = ctx->tb_override, saved_var = ctx->variant;
    auto restore = [&]() {
        ctx->tb_override = saved_tb;
        ctx->variant = saved_var;
    };
    for (int i = 0; i < n; ++i) {
        const auto &sp = specs[i];
        out[i] = z2_results{};
        if (int rc = check_params(ctx, &sp.params)) return rc;
        int32_t L[3] = {sp.L[0], sp.L[1], sp.d == 3 ? sp.L[2] : 1};
        auto key = std::make_tuple(sp.d, L[0], L[1], L[2]);
        auto it = lats.find(key);
        if (it == lats.end()) {
            auto lat = std::make_unique<z2_lattice>();
            std::string err;
            if (!build_lattice(sp.d, L, lat->lat, err)) return fail(ctx, Z2_ERR_LATTICE, err);
            it = lats.emplace(key, std::move(lat)).first;
        }
        lat_of[i] = it->second.get();
        const int nl = lat_of[i]->lat.n_links;
        max_n = std::max(max_n, nl);
        // the persistent kernel takes the runs whose passes do not fill the GPU
        // (fewer than PERSIST_MAX_QUBITS qubits), where a launch per pass is
        // the cost it removes; larger runs go through their own plans on the
        // streams after it
        persist[i] = sp.params.precision == Z2_C64 && nl >= PT && nl < PERSIST_MAX_QUBITS;
        if (persist[i]) {
            ctx->tb_override = PT;
            ctx->variant = 1;
            Plan *P = nullptr;
            const std::string k1 = plan_key(ctx, "evolve", lat_of[i]->lat, &sp.params, 0, sp.params.M, 0);
            int rc = ensure_plan(ctx, k1, P, [&](Plan &Q) {
                return build_evolve_plan(ctx, lat_of[i]->lat, sp.params, 0, sp.params.M, Q);
            });
            restore();
            if (rc) return rc;
            if (P->geo.tb != PT) return fail(ctx, Z2_ERR_LATTICE, "persistent sweep: unexpected tile size");
            plan_of[i] = P;
            total += size_t(8) << nl;
        }
        // the observables use the context's normal plans
        z2_run_params pp{};
        pp.precision = sp.params.precision;
        Plan *H = nullptr;
        const std::string k2 = plan_key(ctx, "had", lat_of[i]->lat, &pp, 0, 0, 0);
        if (int rc = ensure_plan(ctx, k2, H, [&](Plan &Q) {
                return build_hadamard_plan(ctx, lat_of[i]->lat, sp.params.precision == Z2_C128, Q);
            }))
            return rc;
    }
    const int grid = (std::min(persist_max_ctas(ctx->sm_count), 64 * persist_gang()) / persist_gang()) * persist_gang();
    if (grid <= 0) return fail(ctx, Z2_ERR_CUDA, "persistent sweep: kernel cannot be resident");
    // device memory: every persistent run's state, the descriptors and the control block
    std::vector<void *> states(n, nullptr);
    void *d_runs = nullptr, *d_ctl = nullptr, *d_args = nullptr, *d_group = nullptr;
    double *h_all = nullptr;
    std::vector<RunSlot> slots(std::max(1, std::min<int>(n_streams, 64)));
    auto cleanup = [&]() {
        free_slots(slots);
        for (void *p : states)
            if (p) cudaFree(p);
        if (d_runs) cudaFree(d_runs);
        if (d_ctl) cudaFree(d_ctl);
        if (d_args) cudaFree(d_args);
        if (d_group) cudaFree(d_group);
        if (h_all) cudaFreeHost(h_all);
    };
    std::vector<PersistRunHost> runs;
    std::vector<int> run_index;
    std::vector<PassArgs> all_args;
    std::vector<int32_t> all_groups;
    std::vector<size_t> args_off, group_off;
    for (int i = 0; i < n; ++i) {
        if (!persist[i]) continue;
        args_off.push_back(all_args.size());
        group_off.push_back(all_groups.size());
        for (auto &a : plan_of[i]->args) all_args.push_back(a);
        for (auto &hp : plan_of[i]->passes) all_groups.push_back(hp.group);
    }
    bool oom = false;
    for (int i = 0; i < n && !oom; ++i) {
        const size_t bytes = size_t(specs[i].params.precision == Z2_C128 ? 16 : 8) << lat_of[i]->lat.n_links;
        if (persist[i] && cudaMalloc(&states[i], bytes) != cudaSuccess) oom = true;
    }
    if (oom || (!all_args.empty() && (cudaMalloc(&d_args, all_args.size() * sizeof(PassArgs)) != cudaSuccess ||
                                      cudaMalloc(&d_group, all_groups.size() * sizeof(int32_t)) != cudaSuccess))) {
        cleanup();
        return fail(ctx, Z2_ERR_OOM, "persistent sweep: the run states do not fit the device");
    }
    {
        int k = 0;
        for (int i = 0; i < n; ++i) {
            if (!persist[i]) continue;
            const Plan &P = *plan_of[i];
            PersistRunHost r{};
            r.state = states[i];
            r.steps = P.d_steps;
            r.tables = P.d_tables;
            r.args = static_cast<PassArgs *>(d_args) + args_off[k];
            r.group = static_cast<int32_t *>(d_group) + group_off[k];
            r.n_passes = (int32_t)P.passes.size();
            r.n = lat_of[i]->lat.n_links;
            r.init_amp = (float)std::exp2(-0.5 * r.n);
            runs.push_back(r);
            run_index.push_back(i);
            ++k;
        }
    }
    const size_t partial_doubles = reduce_partials_doubles(max_n);
    size_t max_bytes = 0;
    for (int i = 0; i < n; ++i)
        if (!persist[i])
            max_bytes = std::max(max_bytes, size_t(specs[i].params.precision == Z2_C128 ? 16 : 8)
                                                << lat_of[i]->lat.n_links);
    for (auto &sl : slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            (max_bytes && cudaMalloc(&sl.state, max_bytes) != cudaSuccess) ||
            cudaMalloc(&sl.d_partials, partial_doubles * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&sl.d_out, OUT_DOUBLES * sizeof(double)) != cudaSuccess) {
            cleanup();
            return fail(ctx, Z2_ERR_OOM, "persistent sweep: slot allocation failed");
        }
    }
    if (cudaMallocHost(&h_all, (size_t)n * OUT_DOUBLES * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_ctl, persist_ctl_bytes()) != cudaSuccess ||
        (!runs.empty() && cudaMalloc(&d_runs, runs.size() * sizeof(PersistRunHost)) != cudaSuccess)) {
        cleanup();
        return fail(ctx, Z2_ERR_OOM, "persistent sweep: allocation failed");
    }
    cudaStream_t st0 = slots[0].st;
    int rc_all = Z2_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && rc_all == Z2_OK) rc_all = cuda_fail(ctx, e, what);
    };
    if (!all_args.empty()) {
        ck(cudaMemcpyAsync(d_args, all_args.data(), all_args.size() * sizeof(PassArgs), cudaMemcpyHostToDevice, st0),
           "copy run arguments");
        ck(cudaMemcpyAsync(d_group, all_groups.data(), all_groups.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                           st0),
           "copy pass groups");
        ck(cudaMemcpyAsync(d_runs, runs.data(), runs.size() * sizeof(PersistRunHost), cudaMemcpyHostToDevice, st0),
           "copy run descriptors");
    }
    ck(cudaMemsetAsync(d_ctl, 0, persist_ctl_bytes(), st0), "clear control block");
    // 1) every persistent run evolved in one launch
    if (!runs.empty() && rc_all == Z2_OK) {
        ck(launch_persistent(d_runs, (int)runs.size(), d_ctl, ctx->d_err, grid, st0, ctx->gang_wait_polls),
           "persistent launch");
        ctx->launches += 1;
        // odd numbers of quarter turns: the final all-qubit flip of those runs
        for (size_t k = 0; k < runs.size() && rc_all == Z2_OK; ++k)
            if (plan_of[run_index[k]]->flip) {
                ck(launch_flip_all(false, runs[k].state, runs[k].n, ctx->sm_count * 8, st0), "flip");
                ctx->launches += 1;
            }
    }
    cudaEvent_t evolved = nullptr;
    ck(cudaEventCreateWithFlags(&evolved, cudaEventDisableTiming), "event");
    ck(cudaEventRecord(evolved, st0), "event record");
    // 2) observables of those runs, then the remaining runs whole, on the slot streams
    const int S = (int)slots.size();
    for (auto &sl : slots) ck(cudaStreamWaitEvent(sl.st, evolved, 0), "stream wait");
    int j = 0;
    for (int i = 0; i < n && rc_all == Z2_OK; ++i) {
        RunSlot &sl = slots[j++ % S];
        const Scratch sc{sl.d_partials, sl.d_out, h_all + (size_t)i * OUT_DOUBLES};
        int rc;
        if (persist[i]) {
            int n_out = 0;
            rc = measure_enqueue(ctx, lat_of[i], Z2_C64, states[i], nullptr, sl.st, sc, &n_out);
        } else {
            rc = enqueue_run(ctx, lat_of[i], specs[i].params, sl.state, sl.st, sc);
        }
        out[i].status = rc;
        if (rc) rc_all = rc;
    }
    for (auto &sl : slots) ck(cudaStreamSynchronize(sl.st), "cudaStreamSynchronize");
    if (evolved) cudaEventDestroy(evolved);
    if (rc_all == Z2_OK) rc_all = check_device_error(ctx);
    for (int i = 0; i < n; ++i) {
        if (out[i].status == Z2_OK && rc_all == Z2_OK)
            measure_finish(lat_of[i]->lat, specs[i].params.lambda, 1.0, h_all + (size_t)i * OUT_DOUBLES, false,
                           &out[i]);
        else if (out[i].status == Z2_OK)
            out[i].status = rc_all;
    }
    cleanup();
    return rc_all;
}

int z2_sweep(z2_ctx *ctx, const z2_run_spec *specs, int32_t n, int32_t mode, int32_t n_streams, z2_results *out) {
    if (!ctx || (!specs && n > 0) || (!out && n > 0)) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (n < 0) return fail(ctx, Z2_ERR_ARG, "negative run count");
    if (mode < Z2_SWEEP_PLAIN || mode > Z2_SWEEP_PERSISTENT) return fail(ctx, Z2_ERR_ARG, "unknown sweep mode");
    if (n == 0) return Z2_OK;
    if (mode == Z2_SWEEP_PERSISTENT) return sweep_persistent(ctx, specs, n, n_streams, out);
    // lattices (shared between runs of the same shape) and plans, all built
    // before any launch so that nothing allocates while runs are in flight
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<z2_lattice>> lats;
    std::vector<const z2_lattice *> lat_of(n);
    size_t max_bytes = 0;
    int max_n = 8;
    for (int i = 0; i < n; ++i) {
        const auto &sp = specs[i];
        out[i] = z2_results{};
        if (int rc = check_params(ctx, &sp.params)) return rc;
        int32_t L[3] = {sp.L[0], sp.L[1], sp.d == 3 ? sp.L[2] : 1};
        auto key = std::make_tuple(sp.d, L[0], L[1], L[2]);
        auto it = lats.find(key);
        if (it == lats.end()) {
            auto lat = std::make_unique<z2_lattice>();
            std::string err;
            if (!build_lattice(sp.d, L, lat->lat, err)) return fail(ctx, Z2_ERR_LATTICE, err);
            it = lats.emplace(key, std::move(lat)).first;
        }
        lat_of[i] = it->second.get();
        const int nl = lat_of[i]->lat.n_links;
        max_n = std::max(max_n, nl);
        max_bytes = std::max<size_t>(max_bytes, size_t(sp.params.precision == Z2_C128 ? 16 : 8) << nl);
        Plan *P = nullptr;
        const std::string k1 = plan_key(ctx, "evolve", lat_of[i]->lat, &sp.params, 0, sp.params.M, 0);
        if (int rc = ensure_plan(ctx, k1, P, [&](Plan &Q) {
                return build_evolve_plan(ctx, lat_of[i]->lat, sp.params, 0, sp.params.M, Q);
            }))
            return rc;
        z2_run_params pp{};
        pp.precision = sp.params.precision;
        const std::string k2 = plan_key(ctx, "had", lat_of[i]->lat, &pp, 0, 0, 0);
        if (int rc = ensure_plan(ctx, k2, P, [&](Plan &Q) {
                return build_hadamard_plan(ctx, lat_of[i]->lat, sp.params.precision == Z2_C128, Q);
            }))
            return rc;
    }
    const int S = mode == Z2_SWEEP_PLAIN ? 1 : std::max(1, std::min<int>(n_streams, std::min(n, 64)));
    std::vector<RunSlot> slots(S);
    double *h_all = nullptr;
    auto cleanup = [&]() {
        free_slots(slots);
        if (h_all) cudaFreeHost(h_all);
    };
    const size_t partial_doubles = reduce_partials_doubles(max_n);
    for (auto &sl : slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&sl.state, max_bytes) != cudaSuccess ||
            cudaMalloc(&sl.d_partials, partial_doubles * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&sl.d_out, OUT_DOUBLES * sizeof(double)) != cudaSuccess) {
            cleanup();
            return fail(ctx, Z2_ERR_OOM, "sweep: device allocation of the run slots failed");
        }
    }
    if (cudaMallocHost(&h_all, (size_t)n * OUT_DOUBLES * sizeof(double)) != cudaSuccess) {
        cleanup();
        return fail(ctx, Z2_ERR_OOM, "sweep: pinned host allocation failed");
    }
    std::vector<cudaGraphExec_t> execs;
    int rc_all = Z2_OK;
    for (int i = 0; i < n && rc_all == Z2_OK; ++i) {
        RunSlot &sl = slots[i % S];
        const Scratch sc{sl.d_partials, sl.d_out, h_all + (size_t)i * OUT_DOUBLES};
        int rc = Z2_OK;
        if (mode == Z2_SWEEP_GRAPHS) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            if (cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                rc = fail(ctx, Z2_ERR_CUDA, "sweep: stream capture failed to start");
            } else {
                rc = enqueue_run(ctx, lat_of[i], specs[i].params, sl.state, sl.st, sc);
                cudaError_t e = cudaStreamEndCapture(sl.st, &g);
                if (rc == Z2_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaStreamEndCapture");
                if (rc == Z2_OK) {
                    e = cudaGraphInstantiate(&ge, g, 0);
                    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaGraphInstantiate");
                }
                if (rc == Z2_OK) {
                    e = cudaGraphLaunch(ge, sl.st);
                    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaGraphLaunch");
                    execs.push_back(ge);
                }
                if (g) cudaGraphDestroy(g);
            }
        } else {
            rc = enqueue_run(ctx, lat_of[i], specs[i].params, sl.state, sl.st, sc);
            if (rc == Z2_OK && mode == Z2_SWEEP_PLAIN) {
                cudaError_t e = cudaStreamSynchronize(sl.st);
                if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaStreamSynchronize");
            }
        }
        out[i].status = rc;
        if (rc != Z2_OK) rc_all = rc;
    }
    for (auto &sl : slots) {
        cudaError_t e = cudaStreamSynchronize(sl.st);
        if (e != cudaSuccess && rc_all == Z2_OK) rc_all = cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    for (auto ge : execs) cudaGraphExecDestroy(ge);
    if (rc_all == Z2_OK) rc_all = check_device_error(ctx);
    for (int i = 0; i < n; ++i) {
        if (out[i].status == Z2_OK && rc_all == Z2_OK) {
            measure_finish(lat_of[i]->lat, specs[i].params.lambda, 1.0, h_all + (size_t)i * OUT_DOUBLES, false,
                           &out[i]);
        } else if (out[i].status == Z2_OK) {
            out[i].status = rc_all;
        }
    }
    cleanup();
    return rc_all;
}

// ---------------------------------------------------------------------------
// Serving loop (continuous batching).
}  // extern "C"

namespace {

using Clock = std::chrono::steady_clock;

struct ServeReq {
    uint64_t id = 0;
    z2_run_spec spec{};
    int phase = 0;  // 0 queued, 1 running, 2 finished, 3 cancelled
    size_t bytes = 0;
    int qubits = 0;
    z2_results res{};
    Clock::time_point t_submit, t_start, t_end;
    double dev_first = -1, dev_end = -1;  // device clock, seconds since the server's epoch event
};

struct ServeSlot {
    cudaStream_t st = nullptr;
    double *d_partials = nullptr, *d_out = nullptr, *h_out = nullptr;
    cudaEvent_t ev = nullptr;        // end of the run's work (timing event)
    cudaEvent_t ev_first = nullptr;  // after the run's first kernel (timing event)
    bool busy = false;
    uint64_t id = 0;
    void *state = nullptr;
    const z2_lattice *lat = nullptr;
};

}  // namespace

struct z2_server {
    z2_ctx *ctx = nullptr;
    size_t budget = 0;
    int max_slots = 1;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    std::map<uint64_t, ServeReq> reqs;
    std::deque<uint64_t> queue;
    uint64_t next_id = 1;
    z2_serve_stats stats{};
    std::vector<ServeSlot> slots;
    // size classes: runs of at least large_qubits qubits fill every SM with one
    // pass kernel, so running several at once only interleaves them; at most
    // max_large of them are admitted at a time, while smaller runs take any
    // free slot beside them (Z2_SERVE_OPT_*)
    int large_qubits = 22;
    int max_large = 2;
    int active_large = 0;
    cudaEvent_t epoch = nullptr;  // device-clock origin of the request timestamps
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<z2_lattice>> lats;  // worker-owned
    std::string last_error;
};

namespace {

const z2_lattice *serve_lattice(z2_server *srv, const z2_run_spec &sp, std::string &err) {
    int32_t L[3] = {sp.L[0], sp.L[1], sp.d == 3 ? sp.L[2] : 1};
    auto key = std::make_tuple(sp.d, L[0], L[1], L[2]);
    auto it = srv->lats.find(key);
    if (it != srv->lats.end()) return it->second.get();
    auto lat = std::make_unique<z2_lattice>();
    if (!build_lattice(sp.d, L, lat->lat, err)) return nullptr;
    return srv->lats.emplace(key, std::move(lat)).first->second.get();
}

void serve_worker(z2_server *srv) {
    z2_ctx *ctx = srv->ctx;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool progressed = false;
        // retire finished runs
        for (auto &sl : srv->slots) {
            if (!sl.busy || cudaEventQuery(sl.ev) == cudaErrorNotReady) continue;
            ServeReq &rq = srv->reqs[sl.id];
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaSuccess) {
                measure_finish(sl.lat->lat, rq.spec.params.lambda, 1.0, sl.h_out, false, &rq.res);
                float ms0 = 0, ms1 = 0;
                if (cudaEventElapsedTime(&ms0, srv->epoch, sl.ev_first) == cudaSuccess &&
                    cudaEventElapsedTime(&ms1, srv->epoch, sl.ev) == cudaSuccess) {
                    rq.dev_first = 1e-3 * ms0;
                    rq.dev_end = 1e-3 * ms1;
                }
            } else {
                rq.res.status = Z2_ERR_CUDA;
            }
            cudaFreeAsync(sl.state, sl.st);
            srv->stats.hbm_in_use -= rq.bytes;
            srv->stats.completed++;
            srv->stats.active--;
            if (rq.qubits >= srv->large_qubits) srv->active_large--;
            rq.phase = 2;
            rq.t_end = Clock::now();
            sl.busy = false;
            sl.state = nullptr;
            progressed = true;
        }
        if (progressed) srv->cv_done.notify_all();
        // admit in arrival order while a slot and the memory are free; a
        // large run waiting only for a large-run place is passed over by the
        // smaller runs behind it (it keeps its place in the queue)
        for (auto qit = srv->queue.begin(); qit != srv->queue.end();) {
            ServeReq &rq = srv->reqs[*qit];
            if (rq.phase == 3) {  // cancelled while queued
                qit = srv->queue.erase(qit);
                srv->stats.queued--;
                continue;
            }
            ServeSlot *free_slot = nullptr;
            for (auto &sl : srv->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot || srv->stats.hbm_in_use + rq.bytes > srv->budget) break;
            const bool large = rq.qubits >= srv->large_qubits;
            if (large && srv->active_large >= srv->max_large) {
                ++qit;
                continue;
            }
            qit = srv->queue.erase(qit);
            srv->stats.queued--;
            if (large) srv->active_large++;
            rq.phase = 1;
            rq.t_start = Clock::now();
            srv->stats.active++;
            srv->stats.hbm_in_use += rq.bytes;
            srv->stats.hbm_peak = std::max(srv->stats.hbm_peak, srv->stats.hbm_in_use);
            ServeSlot &sl = *free_slot;
            sl.busy = true;
            sl.id = rq.id;
            const z2_run_spec spec = rq.spec;
            lk.unlock();  // host-side planning and launches without the lock
            std::string err;
            int rc = Z2_OK;
            const z2_lattice *lat = serve_lattice(srv, spec, err);
            void *state = nullptr;
            if (!lat) {
                rc = Z2_ERR_LATTICE;
            } else if (cudaMallocAsync(&state, rq.bytes, sl.st) != cudaSuccess) {
                rc = Z2_ERR_OOM;
            } else {
                const Scratch sc{sl.d_partials, sl.d_out, sl.h_out};
                rc = enqueue_run(ctx, lat, spec.params, state, sl.st, sc, sl.ev_first);
                if (rc == Z2_OK && cudaEventRecord(sl.ev, sl.st) != cudaSuccess) rc = Z2_ERR_CUDA;
            }
            lk.lock();
            sl.state = state;
            sl.lat = lat;
            if (rc != Z2_OK) {  // report at once, give the memory back
                if (state) cudaFreeAsync(state, sl.st);
                ServeReq &r2 = srv->reqs[sl.id];
                r2.res.status = rc;
                r2.phase = 2;
                r2.t_end = Clock::now();
                srv->stats.hbm_in_use -= r2.bytes;
                srv->stats.active--;
                if (r2.qubits >= srv->large_qubits) srv->active_large--;
                srv->stats.completed++;
                sl.busy = false;
                sl.state = nullptr;
                srv->cv_done.notify_all();
            }
            progressed = true;
            // the lock was released: the queue may have grown (its iterators
            // are invalid), so the scan starts again from the front
            qit = srv->queue.begin();
        }
        const bool any_busy = std::any_of(srv->slots.begin(), srv->slots.end(), [](const ServeSlot &x) { return x.busy; });
        if (srv->stopping && !any_busy && srv->queue.empty()) break;
        if (!progressed) {
            if (any_busy)
                srv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

extern "C" {

int z2_server_create(z2_ctx *ctx, size_t hbm_budget, int32_t max_slots, z2_server **out) {
    if (!ctx || !out) return fail(ctx, Z2_ERR_ARG, "NULL argument");
    if (max_slots < 1 || max_slots > 64) return fail(ctx, Z2_ERR_ARG, "max_slots must be 1..64");
    *out = nullptr;
    if (hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        Z2_CUDA(ctx, cudaMemGetInfo(&fr, &tot));
        hbm_budget = (size_t)(0.8 * (double)fr);
    }
    // keep freed run memory in the stream-ordered pool instead of returning it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    auto srv = std::make_unique<z2_server>();
    srv->ctx = ctx;
    srv->budget = hbm_budget;
    srv->max_slots = max_slots;
    srv->slots.resize(max_slots);
    const size_t partial_doubles = reduce_partials_doubles(Z2_MAX_LINKS);
    for (auto &sl : srv->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&sl.ev) != cudaSuccess || cudaEventCreate(&sl.ev_first) != cudaSuccess ||
            cudaMalloc(&sl.d_partials, partial_doubles * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&sl.d_out, OUT_DOUBLES * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&sl.h_out, OUT_DOUBLES * sizeof(double)) != cudaSuccess) {
            for (auto &x : srv->slots) {
                if (x.st) cudaStreamDestroy(x.st);
                if (x.ev) cudaEventDestroy(x.ev);
                if (x.ev_first) cudaEventDestroy(x.ev_first);
                if (x.d_partials) cudaFree(x.d_partials);
                if (x.d_out) cudaFree(x.d_out);
                if (x.h_out) cudaFreeHost(x.h_out);
            }
            return fail(ctx, Z2_ERR_OOM, "server: slot allocation failed");
        }
    }
    if (cudaEventCreate(&srv->epoch) != cudaSuccess || cudaEventRecord(srv->epoch, srv->slots[0].st) != cudaSuccess ||
        cudaEventSynchronize(srv->epoch) != cudaSuccess) {
        for (auto &x : srv->slots) {
            cudaStreamDestroy(x.st);
            cudaEventDestroy(x.ev);
            cudaEventDestroy(x.ev_first);
            cudaFree(x.d_partials);
            cudaFree(x.d_out);
            cudaFreeHost(x.h_out);
        }
        if (srv->epoch) cudaEventDestroy(srv->epoch);
        return fail(ctx, Z2_ERR_CUDA, "server: epoch event failed");
    }
    z2_server *p = srv.release();
    p->worker = std::thread(serve_worker, p);
    *out = p;
    return Z2_OK;
}

int z2_server_submit(z2_server *srv, const z2_run_spec *spec, uint64_t *ticket) {
    if (!srv || !spec || !ticket) return Z2_ERR_ARG;
    if (check_params(nullptr, &spec->params) != Z2_OK) return Z2_ERR_ARG;
    Lattice probe;
    std::string err;
    int32_t L[3] = {spec->L[0], spec->L[1], spec->d == 3 ? spec->L[2] : 1};
    if (!build_lattice(spec->d, L, probe, err)) return Z2_ERR_LATTICE;
    const size_t bytes = (size_t)(spec->params.precision == Z2_C128 ? 16 : 8) << probe.n_links;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return Z2_ERR_CANCELLED;
    if (bytes > srv->budget) {
        srv->stats.rejected++;
        return Z2_ERR_BUDGET;
    }
    ServeReq rq;
    rq.id = srv->next_id++;
    rq.spec = *spec;
    rq.bytes = bytes;
    rq.qubits = probe.n_links;
    rq.t_submit = Clock::now();
    srv->reqs[rq.id] = rq;
    srv->queue.push_back(rq.id);
    srv->stats.submitted++;
    srv->stats.queued++;
    *ticket = rq.id;
    srv->cv_work.notify_one();
    return Z2_OK;
}

int z2_server_poll(z2_server *srv, uint64_t ticket, int32_t *done, z2_results *out) {
    if (!srv || !done) return Z2_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return Z2_ERR_NOT_FOUND;
    *done = it->second.phase >= 2;
    if (*done && out) *out = it->second.res;
    return it->second.phase == 3 ? Z2_ERR_CANCELLED : Z2_OK;
}

int z2_server_wait(z2_server *srv, uint64_t ticket, double timeout_s, z2_results *out) {
    if (!srv) return Z2_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return Z2_ERR_NOT_FOUND;
    auto ready = [&] { return srv->reqs[ticket].phase >= 2; };
    if (timeout_s < 0)
        srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
        return Z2_ERR_DEVICE_TIMEOUT;
    const ServeReq &rq = srv->reqs[ticket];
    if (out) *out = rq.res;
    return rq.phase == 3 ? Z2_ERR_CANCELLED : rq.res.status;
}

int z2_server_cancel(z2_server *srv, uint64_t ticket) {
    if (!srv) return Z2_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return Z2_ERR_NOT_FOUND;
    if (it->second.phase != 0) return Z2_ERR_ARG;  // running or finished: not cancellable
    it->second.phase = 3;
    it->second.res.status = Z2_ERR_CANCELLED;
    it->second.t_end = Clock::now();
    srv->stats.cancelled++;
    srv->cv_done.notify_all();
    return Z2_OK;
}

int z2_server_request_times(z2_server *srv, uint64_t ticket, double *queued_s, double *run_s) {
    if (!srv || !queued_s || !run_s) return Z2_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return Z2_ERR_NOT_FOUND;
    const ServeReq &rq = it->second;
    if (rq.phase != 2) return Z2_ERR_ARG;
    *queued_s = std::chrono::duration<double>(rq.t_start - rq.t_submit).count();
    *run_s = std::chrono::duration<double>(rq.t_end - rq.t_start).count();
    return Z2_OK;
}

int z2_server_set_option(z2_server *srv, int32_t option, int32_t value) {
    if (!srv) return Z2_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (option == Z2_SERVE_OPT_LARGE_QUBITS) {
        if (value < 1 || value > Z2_MAX_LINKS + 1) return Z2_ERR_ARG;
        if (srv->stats.active > 0) return Z2_ERR_ARG;  // classes change only while nothing runs
        srv->large_qubits = value;
    } else if (option == Z2_SERVE_OPT_MAX_LARGE) {
        if (value < 1 || value > 64) return Z2_ERR_ARG;
        srv->max_large = value;
    } else {
        return Z2_ERR_ARG;
    }
    srv->cv_work.notify_one();
    return Z2_OK;
}

int z2_server_request_device_times(z2_server *srv, uint64_t ticket, double *first_s, double *end_s) {
    if (!srv || !first_s || !end_s) return Z2_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return Z2_ERR_NOT_FOUND;
    const ServeReq &rq = it->second;
    if (rq.phase != 2 || rq.dev_first < 0) return Z2_ERR_ARG;
    *first_s = rq.dev_first;
    *end_s = rq.dev_end;
    return Z2_OK;
}

int z2_server_stats(z2_server *srv, z2_serve_stats *out) {
    if (!srv || !out) return Z2_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    return Z2_OK;
}

int z2_server_destroy(z2_server *srv) {
    if (!srv) return Z2_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        for (auto id : srv->queue) {
            ServeReq &rq = srv->reqs[id];
            if (rq.phase == 0) {
                rq.phase = 3;
                rq.res.status = Z2_ERR_CANCELLED;
                srv->stats.cancelled++;
            }
        }
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    for (auto &x : srv->slots) {
        if (x.st) cudaStreamSynchronize(x.st);
        if (x.st) cudaStreamDestroy(x.st);
        if (x.ev) cudaEventDestroy(x.ev);
        if (x.ev_first) cudaEventDestroy(x.ev_first);
        if (x.d_partials) cudaFree(x.d_partials);
        if (x.d_out) cudaFree(x.d_out);
        if (x.h_out) cudaFreeHost(x.h_out);
    }
    if (srv->epoch) cudaEventDestroy(srv->epoch);
    delete srv;
    return Z2_OK;
}

}  // extern "C"
