// Gate-level execution (Sec. 2.3, Eq. (ara), Figs. 3 and 4): one launch per
// quantum gate, the way the paper's simulator ran the circuit, for a literal
// comparison with the fused passes and the paper's gate counts.
//
//   gate1_kernel: any 2x2 unitary on one qubit (R_z, R_x, Hadamard), the
//                 matrix built in FP64 on the host and rounded once;
//   cnot_kernel:  controlled NOT, a swap of the amplitude pairs whose control
//                 bit is 1.
//
// Both stream the state once per gate (read + write of the affected half).
#include <cuda_runtime.h>

#include <algorithm>

#include "pass_kernel.cuh"

namespace z2 {

namespace {

// i with a zero bit inserted at position q
__device__ __forceinline__ uint64_t insert_zero(uint64_t i, int q) {
    const uint64_t lo = i & ((1ull << q) - 1ull);
    return ((i >> q) << (q + 1)) | lo;
}

template <typename C>
__device__ __forceinline__ C cfma(C m, C a, C acc) {
    acc.x = fma(m.x, a.x, fma(-m.y, a.y, acc.x));
    acc.y = fma(m.x, a.y, fma(m.y, a.x, acc.y));
    return acc;
}

template <typename C>
__global__ void gate1_kernel(C *__restrict__ psi, uint64_t half, int q, C m00, C m01, C m10, C m11) {
    const uint64_t bit = 1ull << q;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < half; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i0 = insert_zero(i, q), i1 = i0 | bit;
        const C a = psi[i0], b = psi[i1];
        C z;
        z.x = 0;
        z.y = 0;
        psi[i0] = cfma(m01, b, cfma(m00, a, z));
        psi[i1] = cfma(m11, b, cfma(m10, a, z));
    }
}

template <typename C>
__global__ void cnot_kernel(C *__restrict__ psi, uint64_t quarter, int c, int t) {
    const int lo = c < t ? c : t, hi = c < t ? t : c;
    const uint64_t cb = 1ull << c, tb = 1ull << t;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < quarter;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i0 = insert_zero(insert_zero(i, lo), hi) | cb, i1 = i0 | tb;
        const C a = psi[i0];
        psi[i0] = psi[i1];
        psi[i1] = a;
    }
}

template <typename C>
C make_c(double re, double im) {
    C v;
    v.x = (typename Cfg<C>::real)re;
    v.y = (typename Cfg<C>::real)im;
    return v;
}

template <typename C>
cudaError_t launch_gate_t(void *state, int n, int kind, int q0, int q1, const double *m, int grid, cudaStream_t st) {
    const uint64_t dim = 1ull << n;
    if (kind == 0) {
        const uint64_t quarter = dim >> 2;
        const int blocks = (int)std::min<uint64_t>((quarter + 255) / 256, (uint64_t)grid);
        cnot_kernel<C><<<blocks, 256, 0, st>>>(static_cast<C *>(state), quarter, q0, q1);
    } else {
        const uint64_t half = dim >> 1;
        const int blocks = (int)std::min<uint64_t>((half + 255) / 256, (uint64_t)grid);
        gate1_kernel<C><<<blocks, 256, 0, st>>>(static_cast<C *>(state), half, q0, make_c<C>(m[0], m[1]),
                                                make_c<C>(m[2], m[3]), make_c<C>(m[4], m[5]), make_c<C>(m[6], m[7]));
    }
    return cudaGetLastError();
}

}  // namespace

// kind 0: CNOT(control q0, target q1); kind 1: the 2x2 matrix m (row-major,
// complex as (re, im) pairs) on qubit q0
cudaError_t launch_gate(bool c128, void *state, int n, int kind, int q0, int q1, const double *m, int grid,
                        cudaStream_t st) {
    if (n < 2 || q0 < 0 || q0 >= n || (kind == 0 && (q1 < 0 || q1 >= n || q1 == q0))) return cudaErrorInvalidValue;
    return c128 ? launch_gate_t<double2>(state, n, kind, q0, q1, m, grid, st)
                : launch_gate_t<float2>(state, n, kind, q0, q1, m, grid, st);
}

}  // namespace z2
