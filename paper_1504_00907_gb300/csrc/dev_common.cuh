// Small device helpers shared by the kernels of this library.
#pragma once

#include <cuda_runtime.h>

namespace ddgdev {

// After the call, the lane with index q = (lane / S) % N holds the sum over
// the N lanes of v[q]: a reduce-scatter by recursive halving, N - 1 shuffles.
template <int N, int S, typename V>
__device__ __forceinline__ V reduce_scatter(V (&v)[N], int q) {
#pragma unroll
    for (int half = N / 2; half >= 1; half >>= 1) {
        const bool up = (q & half) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            V send = up ? v[i] : v[i + half];
            V keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half * S);
        }
    }
    return v[0];
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of one value per thread over the block, in a fixed order; the result
// is returned to every thread.  `sh` must hold blockDim.x / 32 values.
template <typename V>
__device__ __forceinline__ V block_sum(V v, V* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    V s = 0;
    for (int i = 0; i < nw; ++i) s += sh[i];
    return s;
}

// Sum of 32 values per thread over the block; out[i] = total of v[i].
// `sh` holds 32 * (blockDim.x / 32) values.
template <typename V>
__device__ __forceinline__ void block_sum32(V (&v)[32], V* sh, V* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const V t = reduce_scatter<32, 1>(v, lane);
    __syncthreads();
    sh[w * 32 + lane] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        V s = 0;
        for (int i = 0; i < nw; ++i) s += sh[i * 32 + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// block_sum32 on K (a multiple of 32) values per thread, 32 at a time.
template <int K, typename V>
__device__ __forceinline__ void block_sum_k(V (&v)[K], V* sh, V* out) {
    if constexpr (K == 32) {
        block_sum32(v, sh, out);
    } else {
#pragma unroll
        for (int c = 0; c < K / 32; ++c) block_sum32(*reinterpret_cast<V(*)[32]>(v + 32 * c), sh, out + 32 * c);
    }
}

// Pseudo stencil kinds of the CSR path: rows of at most 8 / 16 entries are
// applied fully unrolled so that all column and value loads of a row, then
// all x loads, are in flight together (same summation order as the loop).
constexpr int SK_CSR8 = 100;
constexpr int SK_CSR16 = 101;

template <int NMAX, typename V, typename AV>
__device__ __forceinline__ V csr_row_dot_unrolled(int g, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col,
                                                  const AV* __restrict__ val, const V* __restrict__ x,
                                                  int stride, int c) {
    const int64_t e0 = rowptr[g];
    const int cnt = (int)(rowptr[g + 1] - e0);
    int cl[NMAX];
    V vl[NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        cl[i] = i < cnt ? col[e0 + i] : 0;
        vl[i] = i < cnt ? (V)val[e0 + i] : (V)0;
    }
    V s = 0;
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
        if (i < cnt) s = fma(vl[i], x[(int64_t)cl[i] * stride + c], s);
    return s;
}

// Packed upper tile triangle of one local inverse with T tile rows of 32.
// Band row I < T-1 holds, in this order: the diagonal tile (I, I) as an
// upper trapezoid in 8-column blocks (row r keeps columns 8 floor(r/8) .. 31,
// PACKED_DIAG = 640 values, the 8x8 diagonal blocks in full), the full 32x32
// tiles J = I+1 .. T-2, and the last tile column J = T-1 stored 32 x wp with
// wp = n - 32 (T - 1) rounded up to 8.  Band row T-1 holds only its narrow
// diagonal tile, 32 x wp.  Every 8-column block of a row starts on a 16-byte
// boundary for 2-, 4- and 8-byte elements.
constexpr int PACKED_DIAG = 640;

__host__ __device__ __forceinline__ int packed_narrow_width(int n, int T) {
    return ((n - 32 * (T - 1)) + 7) & ~7;
}
__host__ __device__ __forceinline__ size_t packed_row_start(int I, int T, int wp) {
    return (size_t)I * (PACKED_DIAG + 32 * wp) + (size_t)1024 * ((size_t)I * (T - 2) - (size_t)I * (I - 1) / 2);
}
// first element of tile (I, J), J >= I
__host__ __device__ __forceinline__ size_t packed_tile_start(int I, int J, int T, int wp) {
    const size_t rs = packed_row_start(I, T, wp);
    return J == I ? rs : rs + PACKED_DIAG + (size_t)(J - I - 1) * 1024;
}
__host__ __device__ __forceinline__ size_t packed_elems(int T, int wp) {
    return packed_row_start(T - 1, T, wp) + (size_t)32 * wp;
}
// element (r, c), c >= 8 floor(r / 8), of a trapezoid diagonal tile
__host__ __device__ __forceinline__ int packed_diag_offset(int r, int c) {
    const int a = r >> 3, b = r & 7;
    return 256 * a - 32 * a * (a - 1) + b * (32 - 8 * a) + (c - 8 * a);
}

// Long CSR rows (Q1 elasticity: 81 entries) go to groups of CSRW_G lanes
// (4 measured best for 81-entry rows against 8, 16 and 32):
// lane l of a group takes entries l, l + G, ... of its row (coalesced column
// and value loads) and the group sums by a fixed butterfly, after which every
// lane of the group holds the row's dot product.  All lanes of the warp must
// call it; `live` masks the loads of groups past the last row.
constexpr int SK_CSRW = 102;
constexpr int CSRW_G = 4;

template <int G, typename V, typename AV>
__device__ __forceinline__ V csr_row_dot_group(int g, bool live, const int64_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col,
                                               const AV* __restrict__ val, const V* __restrict__ x) {
    V s = 0;
    if (live) {
        const int sub = threadIdx.x & (G - 1);
        const int64_t e1 = rowptr[g + 1];
        for (int64_t e = rowptr[g] + sub; e < e1; e += G) s = fma((V)val[e], x[col[e]], s);
    }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

}  // namespace ddgdev
