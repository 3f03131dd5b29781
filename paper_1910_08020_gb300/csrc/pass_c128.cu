// Pass-kernel instantiations for c128 states (tile bits 8..13).
#include "pass_kernel.cuh"

namespace z2 {

template <typename C, int TB, int OP>
static cudaError_t launch_tb(C *psi, const PassArgs &a, const PassStep *steps, int n_steps, const C *tables,
                             int grid, cudaStream_t st) {
    using T = Tile<C, TB>;
    const size_t smem = sizeof(C) * T::SMEM_SLOTS;
    static std::atomic<uint64_t> configured{0};  // devices whose attributes are set
    const uint64_t dev_bit = current_device_bit();
    if (!(configured.load() & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel<C, TB, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    pass_kernel<C, TB, OP><<<grid, T::NT, smem, st>>>(psi, a, steps, n_steps, tables);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_op(int tb, double2 *psi, const PassArgs &a, const PassStep *steps, int n_steps,
                             const double2 *tables, int grid, cudaStream_t st) {
    switch (tb) {
        case 8: return launch_tb<double2, 8, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 9: return launch_tb<double2, 9, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 10: return launch_tb<double2, 10, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 11: return launch_tb<double2, 11, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 12: return launch_tb<double2, 12, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 13: return launch_tb<double2, 13, OP>(psi, a, steps, n_steps, tables, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_c128(int tb, int op, void *psi, const PassArgs &a, const void *steps, int n_steps,
                               const void *tables, int fmt, int grid, cudaStream_t st) {
    (void)fmt;  // complex128 passes always use the interleaved format
    auto ps = static_cast<const PassStep *>(steps);
    auto p = static_cast<double2 *>(psi);
    auto tab = static_cast<const double2 *>(tables);
    return op == OP_HADAMARD ? launch_op<OP_HADAMARD>(tb, p, a, ps, n_steps, tab, grid, st)
                             : launch_op<OP_RX_TAN>(tb, p, a, ps, n_steps, tab, grid, st);
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
                                 const double2 *tables, int *err, int grid, cudaStream_t st) {
    switch (tb) {
        case 8: return launch_tma_tb<double2, 8, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 9: return launch_tma_tb<double2, 9, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 10: return launch_tma_tb<double2, 10, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 11: return launch_tma_tb<double2, 11, OP>(a, m, steps, n_steps, tables, err, grid, st);
        case 12: return launch_tma_tb<double2, 12, OP>(a, m, steps, n_steps, tables, err, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_tma_c128(int tb, int op, const PassArgs &a, const void *tmap, const void *steps, int n_steps,
                                   const void *tables, int *err, int grid, cudaStream_t st) {
    auto ps = static_cast<const PassStep *>(steps);
    auto tab = static_cast<const double2 *>(tables);
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(tmap);
    return op == OP_HADAMARD ? launch_tma_op<OP_HADAMARD>(tb, a, m, ps, n_steps, tab, err, grid, st)
                             : launch_tma_op<OP_RX_TAN>(tb, a, m, ps, n_steps, tab, err, grid, st);
}

int tma_smem_bytes_c128(int tb) {
    switch (tb) {
        case 8: return (int)TmaTile<double2, 8>::SMEM_BYTES;
        case 9: return (int)TmaTile<double2, 9>::SMEM_BYTES;
        case 10: return (int)TmaTile<double2, 10>::SMEM_BYTES;
        case 11: return (int)TmaTile<double2, 11>::SMEM_BYTES;
        case 12: return (int)TmaTile<double2, 12>::SMEM_BYTES;
        default: return 0;
    }
}

}  // namespace z2
