// Pass-kernel instantiations for c64 states (tile bits 8..14).
#include "pass_kernel.cuh"

namespace z2 {

template <typename C, int TB, int OP>
static cudaError_t launch_tb(C *psi, const PassArgs &a, const PassStep *steps, int n_steps, const C *tables,
                             int grid, cudaStream_t st) {
    using T = Tile<C, TB>;
    const size_t smem = sizeof(C) * T::SMEM_SLOTS;
    static bool configured = false;  // once per instantiation and process
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel<C, TB, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    pass_kernel<C, TB, OP><<<grid, T::NT, smem, st>>>(psi, a, steps, n_steps, tables);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_op(int tb, float2 *psi, const PassArgs &a, const PassStep *steps, int n_steps,
                             const float2 *tables, int grid, cudaStream_t st) {
    switch (tb) {
        case 8: return launch_tb<float2, 8, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 9: return launch_tb<float2, 9, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 10: return launch_tb<float2, 10, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 11: return launch_tb<float2, 11, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 12: return launch_tb<float2, 12, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 13: return launch_tb<float2, 13, OP>(psi, a, steps, n_steps, tables, grid, st);
        case 14: return launch_tb<float2, 14, OP>(psi, a, steps, n_steps, tables, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_c64(int tb, int op, void *psi, const PassArgs &a, const void *steps, int n_steps,
                               const void *tables, int grid, cudaStream_t st) {
    auto ps = static_cast<const PassStep *>(steps);
    auto p = static_cast<float2 *>(psi);
    auto tab = static_cast<const float2 *>(tables);
    return op == OP_HADAMARD ? launch_op<OP_HADAMARD>(tb, p, a, ps, n_steps, tab, grid, st)
                             : launch_op<OP_RX_TAN>(tb, p, a, ps, n_steps, tab, grid, st);
}

}  // namespace z2
