// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <atomic>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "z2lgt.h"

namespace z2 {

// ---------------------------------------------------------------------------
// Lattice (Sec. 2.1): links, plaquettes, stars and loop masks, host side.
struct Lattice {
    int d = 0;
    int L[3] = {1, 1, 1};
    int n_sites = 0, n_links = 0, n_plaq = 0;
    std::vector<uint64_t> plaq, star, wmu, vmu;
    uint64_t wilson2x2 = 0;
    bool wilson_degenerate = false;
    uint64_t contour[3] = {0, 0, 0};
    bool contour_degenerate[3] = {false, false, false};
    // colmask[l]: bit p set when link l belongs to plaquette p
    uint32_t colmask[64] = {};
};
bool build_lattice(int d, const int32_t *L, Lattice &out, std::string &err);
// Record `msg` as this thread's last error (z2_last_error(NULL)); returns code.
int set_thread_error(int code, const std::string &msg);
// Bit of the current device in a per-launcher "attributes set" mask:
// cudaFuncSetAttribute applies to the current device only, so launchers set
// their shared-memory limit once per device, not once per process.
inline uint64_t current_device_bit() {
    int dev = 0;
    cudaGetDevice(&dev);
    return 1ull << (dev & 63);
}

// ---------------------------------------------------------------------------
// One fused pass over the state (Sec. 2.2, both layers of a step).
//
// A pass streams the state once, tile by tile.  A tile holds 2^TB amplitudes:
// tile bit i < c is global bit i (contiguous run of 2^c amplitudes), tile bit
// i >= c is global bit b + i - c.  Inside the tile the pass applies, in order,
//   rot1: the single-qubit gate on the tile bits of mask rot1,
//   mid:  the plaquette phase table (D with the folded gate scale) or a
//         real scale,
//   rot2: the gate on the tile bits of mask rot2.
enum PassOp : int { OP_RX_TAN = 0, OP_RX_GEN = 1, OP_HADAMARD = 2 };
enum MidOp : int { MID_NONE = 0, MID_TABLE = 1, MID_SCALE = 2 };

struct PassDesc {
    int tb = 0;        // tile bits (template instantiation)
    int c = 0, b = 0;  // tile geometry, b >= c, c == tb for a contiguous tile
    uint32_t rot1 = 0, rot2 = 0;
    int mid = MID_NONE;
    int table = -1;    // index of the phase table (MID_TABLE)
    double scale = 1;  // MID_SCALE
};

// Everything a pass kernel needs besides the state pointer.
struct PassArgs {
    int n;                 // qubits
    int c, b;              // tile geometry
    uint32_t rot1, rot2;   // rotation masks over tile bits
    int mid;               // MidOp
    int np1;               // n_plaq + 1 (table length)
    double p0, p1;         // unused (gate values are per pass step)
    double scale;          // MID_SCALE factor
    const void *table;     // device phase table (np1 complex of the state's type)
    int tma_lo_bits;       // tile-id bits below the strided part (b - c of the TMA view)
    int tma_hi_dim;        // TMA dimension of the upper tile-id bits: 4, or 3 for a split group
    int hib;               // first global bit above the tile's lower range (ring kernel)
    uint32_t tcol[16];     // per tile bit: plaquette-membership mask of its global bit
    uint32_t colmask[64];  // per global bit (for the tile-id part)
};

// Launchers (kernels.cu).  All return the cudaError_t of the launch.
// `steps` is a device array of PassStep (pass_kernel.cuh), `tables` a device
// array of phase tables, (Z2_MAX_PLAQ + 1) amplitudes of the state's type each.
// fmt (complex64 only): bit 0 = the input is in the split-pair format,
// bit 1 = write the split-pair format (see pass_packed.cuh).
cudaError_t launch_pass_steps(bool c128, int tb, int op, void *psi, const PassArgs &a, const void *steps,
                              int n_steps, const void *tables, int fmt, int grid, cudaStream_t st);
int pass_threads(bool c128, int tb);
// TMA-pipelined persistent variant: `tmap` is a CUtensorMap (5-D view of the
// state, see make_tensor_map in runtime.cpp); `err` a device flag set to 1 if
// a bounded wait gave up.
cudaError_t launch_pass_tma(bool c128, int tb, int op, const PassArgs &a, const void *tmap, const void *steps,
                            int n_steps, const void *tables, int *err, int grid, cudaStream_t st);
int tma_tile_limit(bool c128);
// complex64 streaming ring variant (pass_packed.cuh): multi-tile passes, one
// step per launch, tile bits 10..13, grid = number of SMs
// s8: relayouts through 8-byte (re | im) slot arrays instead of 16-byte pair
// slots (used for strided passes, see pass_packed.cuh)
// seq: static layout sequence code of the pass (ring_seq in runtime.cpp; 0 =
// the general step); launchers fall back to the general step where no static
// instantiation exists
cudaError_t launch_pass_ring_c64(int tb, int op, const PassArgs &a, const void *tmap, const void *steps,
                                 const void *tables, int fmt, int *err, int grid, cudaStream_t st, bool s8,
                                 int seq = 0);
// the same ring with 32 pairs per thread (pass_c64_ring5.cu), tile bits 12..13
cudaError_t launch_pass_ring5_c64(int tb, int op, const PassArgs &a, const void *tmap, const void *steps,
                                  const void *tables, int fmt, int *err, int grid, cudaStream_t st, bool s8,
                                  int seq = 0);
int tma_smem_bytes(bool c128, int tb);
size_t pass_smem(bool c128, int tb);
cudaError_t launch_init_plus(bool c128, void *state, int n, int grid, cudaStream_t st);
cudaError_t launch_flip_all(bool c128, void *state, int n, int grid, cudaStream_t st);
// one gate (circuit.cu): kind 0 = CNOT(q0 -> q1), 1 = the 2x2 matrix m
// (row-major, (re, im) pairs) on qubit q0; n = qubits of the state
cudaError_t launch_gate(bool c128, void *state, int n, int kind, int q0, int q1, const double *m, int grid,
                        cudaStream_t st);
// zero the state, then 2^(-r/2) at every index offset ^ (span of basis[0..r)),
// basis linearly independent over GF(2) (two launches)
cudaError_t launch_span_state(bool c128, void *state, int n, const uint64_t *basis, int r, uint64_t offset, int grid,
                              cudaStream_t st);
// FP64 reductions over 2^n amplitudes (n >= 8): per-block partials in
// `partials` (reduce_blocks(n) x outputs doubles), then a fixed-order final
// sum into d_out (device).  zsums: 1 <= n_masks <= max_zsum_masks().
cudaError_t launch_zsums(bool c128, const void *state, int n, const uint64_t *masks, int n_masks, double *partials,
                         double *d_out, cudaStream_t st);
cudaError_t launch_overlap(bool c128, const void *a, const void *b, int n, double *partials, double *d_out,
                           cudaStream_t st);
int max_zsum_masks();
int zsums_launches(int n, int n_masks);  // kernel launches of one launch_zsums call
// density of states over 2^n amplitudes: n_masks >= 1 bins by the number of
// masks of odd parity (n_masks + 1 bins), n_masks == 0 by popcount (n + 1
// bins); the bins land in d_out[0 .. *n_bins)
cudaError_t launch_dos(bool c128, const void *state, int n, const uint64_t *masks, int n_masks, double *partials,
                       double *d_out, int *n_bins, cudaStream_t st);
// persistent multi-run evolution (persistent.cu): runs = device array of
// PersistRun, ctl = zeroed control block, grid = a multiple of persist_gang()
// no larger than persist_max_ctas(); runs need >= persist_tile_bits() qubits.
// spin_limit: polls of a gang barrier before it gives up (0 = the default)
cudaError_t launch_persistent(const void *runs, int n_runs, void *ctl, int *err, int grid, cudaStream_t st,
                              uint32_t spin_limit);
int persist_tile_bits();
int persist_gang();
size_t persist_run_bytes();
size_t persist_ctl_bytes();
int persist_max_ctas(int sm_count);
struct PersistRunHost {
    void *state;
    const void *steps;
    const void *tables;
    const void *args;
    const int32_t *group;
    int32_t n_passes;
    int32_t n;
    float init_amp;
    int32_t pad;
};
int reduce_blocks(int n);
// size of the partials buffer that every reduction over 2^n amplitudes fits
size_t reduce_partials_doubles(int n);

struct PassStepHost {
    uint32_t rot1, rot2;
    int32_t mid, table;
    double scale;
    double g1, g2;  // gate values of the rot1 / rot2 layers
};

}  // namespace z2
