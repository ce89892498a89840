// FP64 64 x 64 tile helpers of the dense factorisation kernels (band and
// nested-dissection Cholesky): tiles staged in shared memory with a row
// stride of 65, 256 threads, 4 x 4 register micro-tiles per thread.
#pragma once

#include "ddg_internal.cuh"

namespace tile64 {

constexpr int CT = DDG_CT;
constexpr int CLD = CT + 1;

__device__ __forceinline__ void ct_load(double* s, const double* g) {
    for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) s[(i >> 6) * CLD + (i & 63)] = g[i];
}
__device__ __forceinline__ void ct_store(double* g, const double* s) {
    for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) g[i] = s[(i >> 6) * CLD + (i & 63)];
}

// acc += A * B^T (NT) or A * B (NN), 64x64x64
template <bool TRANS_B>
__device__ __forceinline__ void ct_mac(double (&acc)[4][4], const double* A, const double* B) {
    const int r0 = (threadIdx.x >> 4) * 4, c0 = (threadIdx.x & 15) * 4;
#pragma unroll 2
    for (int m = 0; m < CT; ++m) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[(r0 + i) * CLD + m];
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = TRANS_B ? B[(c0 + i) * CLD + m] : B[m * CLD + c0 + i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], b[jj], acc[i][jj]);
    }
}

__device__ __forceinline__ void acc_zero4(double (&acc)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
}

}  // namespace tile64
