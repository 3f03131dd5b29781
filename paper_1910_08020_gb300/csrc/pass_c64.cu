// Pass-kernel instantiations for c64 states (tile bits 8..14).
#include "pass_kernel.cuh"
#include "pass_packed.cuh"

namespace z2 {
constexpr int PACK_W = 4;  // 16 pairs = 32 amplitudes per thread
}

namespace z2 {

template <int TB, int OP>
static cudaError_t launch_packed_tb(float2 *psi, const PassArgs &a, const PassStep *steps, int n_steps,
                                    const float2 *tables, int fmt, int grid, cudaStream_t st) {
    using T = PTile<TB, PACK_W>;
    const size_t smem = sizeof(ulonglong2) * T::SLOTS;
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    const uint64_t dev_bit = current_device_bit();
    if (!(configured.load() & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel_packed<TB, PACK_W, OP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    pass_kernel_packed<TB, PACK_W, OP><<<grid, T::NT, smem, st>>>(psi, a, steps, n_steps, tables, fmt);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_op(int tb, float2 *psi, const PassArgs &a, const PassStep *steps, int n_steps,
                             const float2 *tables, int fmt, int grid, cudaStream_t st) {
    switch (tb) {
        case 8: return launch_packed_tb<8, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        case 9: return launch_packed_tb<9, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        case 10: return launch_packed_tb<10, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        case 11: return launch_packed_tb<11, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        case 12: return launch_packed_tb<12, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        case 13: return launch_packed_tb<13, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        case 14: return launch_packed_tb<14, OP>(psi, a, steps, n_steps, tables, fmt, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_c64(int tb, int op, void *psi, const PassArgs &a, const void *steps, int n_steps,
                            const void *tables, int fmt, int grid, cudaStream_t st) {
    auto ps = static_cast<const PassStep *>(steps);
    auto p = static_cast<float2 *>(psi);
    auto tab = static_cast<const float2 *>(tables);
    return op == OP_HADAMARD ? launch_op<OP_HADAMARD>(tb, p, a, ps, n_steps, tab, fmt, grid, st)
                             : launch_op<OP_RX_TAN>(tb, p, a, ps, n_steps, tab, fmt, grid, st);
}

int packed_threads(int tb) { return 1 << (tb - 1 - PACK_W); }

template <int TB, int OP, bool S8 = false, int SEQ = 0>
static cudaError_t launch_ring_tb(const PassArgs &a, const CUtensorMap &m, const PassStep *steps,
                                  const float2 *tables, int fmt, int *err, int grid, cudaStream_t st) {
    using T = PTile<TB, PACK_W>;
    using RT = RingTile<TB, PACK_W>;
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    const uint64_t dev_bit = current_device_bit();
    if (!(configured.load() & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel_ring<TB, PACK_W, OP, S8, SEQ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    pass_kernel_ring<TB, PACK_W, OP, S8, SEQ><<<grid, RT::NW * T::NT, RT::SMEM_BYTES, st>>>(a, m, steps, tables,
                                                                                           fmt, err);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_ring_op(int tb, const PassArgs &a, const CUtensorMap &m, const PassStep *steps,
                                  const float2 *tables, int fmt, int *err, int grid, cudaStream_t st) {
    switch (tb) {
        case 10: return launch_ring_tb<10, OP>(a, m, steps, tables, fmt, err, grid, st);
        case 11: return launch_ring_tb<11, OP>(a, m, steps, tables, fmt, err, grid, st);
        case 12: return launch_ring_tb<12, OP>(a, m, steps, tables, fmt, err, grid, st);
        case 13: return launch_ring_tb<13, OP>(a, m, steps, tables, fmt, err, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_ring_c64(int tb, int op, const PassArgs &a, const void *tmap, const void *steps,
                                 const void *tables, int fmt, int *err, int grid, cudaStream_t st, bool s8, int seq) {
    auto ps = static_cast<const PassStep *>(steps);
    auto tab = static_cast<const float2 *>(tables);
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(tmap);
    // static layout sequences of the large-state plans: the unmerged low-group
    // pass on 12-bit tiles (32 qubits) and the merged low-group pass on 13-bit
    // tiles (24 qubits); any other pass runs the general step
    if (!s8 && op == OP_RX_TAN && tb == 12 && seq == seq_code(3, false))
        return launch_ring_tb<12, OP_RX_TAN, false, seq_code(3, false)>(a, m, ps, tab, fmt, err, grid, st);
    if (!s8 && op == OP_RX_TAN && tb == 13 && seq == seq_code(3, true))
        return launch_ring_tb<13, OP_RX_TAN, false, seq_code(3, true)>(a, m, ps, tab, fmt, err, grid, st);
    // 8-byte relayout scratch for the evolution's strided passes on 12- and
    // 13-bit tiles (instruction-bound); the rest keep 16-byte pair slots
    if (s8 && op == OP_RX_TAN && tb == 12)
        return launch_ring_tb<12, OP_RX_TAN, true>(a, m, ps, tab, fmt, err, grid, st);
    if (s8 && op == OP_RX_TAN && tb == 13)
        return launch_ring_tb<13, OP_RX_TAN, true>(a, m, ps, tab, fmt, err, grid, st);
    return op == OP_HADAMARD ? launch_ring_op<OP_HADAMARD>(tb, a, m, ps, tab, fmt, err, grid, st)
                             : launch_ring_op<OP_RX_TAN>(tb, a, m, ps, tab, fmt, err, grid, st);
}

int ring_tile_limits(int *lo, int *hi) {
    *lo = 10;
    *hi = 13;
    return 0;
}

template <typename C, int TB, int OP>
static cudaError_t launch_tma_tb(const PassArgs &a, const CUtensorMap &m, const PassStep *steps, int n_steps,
                                 const C *tables, int *err, int grid, cudaStream_t st) {
    using T = Tile<C, TB>;
    using TT = TmaTile<C, TB>;
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    const uint64_t dev_bit = current_device_bit();
    if (!(configured.load() & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel_tma<C, TB, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TT::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    pass_kernel_tma<C, TB, OP><<<grid, T::NT, TT::SMEM_BYTES, st>>>(a, m, steps, n_steps, tables, err);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_tma_op(int tb, const PassArgs &a, const CUtensorMap &m, const PassStep *steps, int n_steps,
                                 const float2 *tables, int *err, int grid, cudaStream_t st) {
    switch (tb) {
        case 8: return launch_tma_tb<float2, 8, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 9: return launch_tma_tb<float2, 9, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 10: return launch_tma_tb<float2, 10, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 11: return launch_tma_tb<float2, 11, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 12: return launch_tma_tb<float2, 12, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 13: return launch_tma_tb<float2, 13, OP>(a, m, steps, n_steps, tables, err, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_tma_c64(int tb, int op, const PassArgs &a, const void *tmap, const void *steps, int n_steps,
                                   const void *tables, int *err, int grid, cudaStream_t st) {
    auto ps = static_cast<const PassStep *>(steps);
    auto tab = static_cast<const float2 *>(tables);
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(tmap);
    return op == OP_HADAMARD ? launch_tma_op<OP_HADAMARD>(tb, a, m, ps, n_steps, tab, err, grid, st)
                             : launch_tma_op<OP_RX_TAN>(tb, a, m, ps, n_steps, tab, err, grid, st);
}

int tma_smem_bytes_c64(int tb) {
    switch (tb) {
        case 8: return (int)TmaTile<float2, 8>::SMEM_BYTES;
        case 9: return (int)TmaTile<float2, 9>::SMEM_BYTES;
        case 10: return (int)TmaTile<float2, 10>::SMEM_BYTES;
        case 11: return (int)TmaTile<float2, 11>::SMEM_BYTES;
        case 12: return (int)TmaTile<float2, 12>::SMEM_BYTES;
        case 13: return (int)TmaTile<float2, 13>::SMEM_BYTES;
        default: return 0;
    }
}

}  // namespace z2
