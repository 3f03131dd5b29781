// Ring-kernel instantiations for complex64 with 32 pairs (64 amplitudes) per
// thread.  A layout then holds five pair-index bits in registers instead of
// four, so a fused pass over a strided group of up to ten qubits visits two
// register layouts (one relayout there and one back) instead of three (four
// relayouts): about 35% less shared-memory traffic per tile, for twice the
// registers per thread and half the threads per tile.
#include "pass_kernel.cuh"
#include "pass_packed.cuh"

namespace z2 {

namespace {
constexpr int RING5_W = 5;

template <int TB, int OP, bool S8 = false, int SEQ = 0>
cudaError_t launch_ring5_tb(const PassArgs &a, const CUtensorMap &m, const PassStep *steps, const float2 *tables,
                            int fmt, int *err, int grid, cudaStream_t st) {
    using T = PTile<TB, RING5_W>;
    using RT = RingTile<TB, RING5_W>;
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    const uint64_t dev_bit = current_device_bit();
    if (!(configured.load() & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel_ring<TB, RING5_W, OP, S8, SEQ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    pass_kernel_ring<TB, RING5_W, OP, S8, SEQ><<<grid, RT::NW * T::NT, RT::SMEM_BYTES, st>>>(a, m, steps, tables,
                                                                                             fmt, err);
    return cudaGetLastError();
}

template <int OP>
cudaError_t launch_ring5_op(int tb, const PassArgs &a, const CUtensorMap &m, const PassStep *steps,
                            const float2 *tables, int fmt, int *err, int grid, cudaStream_t st) {
    switch (tb) {
        case 12: return launch_ring5_tb<12, OP>(a, m, steps, tables, fmt, err, grid, st);
        case 13: return launch_ring5_tb<13, OP>(a, m, steps, tables, fmt, err, grid, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_pass_ring5_c64(int tb, int op, const PassArgs &a, const void *tmap, const void *steps,
                                  const void *tables, int fmt, int *err, int grid, cudaStream_t st, bool s8, int seq) {
    auto ps = static_cast<const PassStep *>(steps);
    auto tab = static_cast<const float2 *>(tables);
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(tmap);
    // the merged strided passes of the large-state plans: both rotations in
    // register layouts 0 and 1 (static sequence); any other pass: general step
    if (s8 && op == OP_RX_TAN && tb == 13 && seq == seq_code(2, true))
        return launch_ring5_tb<13, OP_RX_TAN, true, seq_code(2, true)>(a, m, ps, tab, fmt, err, grid, st);
    if (s8 && op == OP_RX_TAN && tb == 12 && seq == seq_code(2, true))
        return launch_ring5_tb<12, OP_RX_TAN, true, seq_code(2, true)>(a, m, ps, tab, fmt, err, grid, st);
    // the 24-qubit strided group (two passenger bits): its one rotated bit
    // beyond layout 1 is a lane bit there, rotated by warp shuffles
    if (s8 && op == OP_RX_TAN && tb == 13 && seq == seq_code(2, true, 2))
        return launch_ring5_tb<13, OP_RX_TAN, true, seq_code(2, true, 2)>(a, m, ps, tab, fmt, err, grid, st);
    // a strided group whose bits reach layout 2 otherwise
    if (s8 && op == OP_RX_TAN && tb == 13 && seq == seq_code(3, true))
        return launch_ring5_tb<13, OP_RX_TAN, true, seq_code(3, true)>(a, m, ps, tab, fmt, err, grid, st);
    if (s8 && op == OP_RX_TAN && tb == 12)
        return launch_ring5_tb<12, OP_RX_TAN, true>(a, m, ps, tab, fmt, err, grid, st);
    if (s8 && op == OP_RX_TAN && tb == 13)
        return launch_ring5_tb<13, OP_RX_TAN, true>(a, m, ps, tab, fmt, err, grid, st);
    return op == OP_HADAMARD ? launch_ring5_op<OP_HADAMARD>(tb, a, m, ps, tab, fmt, err, grid, st)
                             : launch_ring5_op<OP_RX_TAN>(tb, a, m, ps, tab, fmt, err, grid, st);
}

}  // namespace z2
