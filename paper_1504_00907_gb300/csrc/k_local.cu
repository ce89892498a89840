// Local subdomain operators of the multiplicative Schwarz smoother (Sec. 6).
//
// Setup: A_i = R~_i A R~_i^T is gathered densely (FP64), factored A_i = L L^T
// and inverted (A_i^{-1} = L^{-T} L^{-1}) in 32x32 tiles by one CTA per
// subdomain, and the upper-triangular tiles of the symmetric inverse are
// packed in FP64 / FP32 / BF16 (the last tile column at its valid width).
//
// Apply (per colour c of the sweep; subdomains of one colour do not interact):
//   res_i = (r - A z)[Omega~_i]            local_residual_kernel
//   z[Omega~_i] += A_i^{-1} res_i          local_solve_kernel
// The second kernel streams the packed inverse; every tile (I, J), I < J,
// is read once and used twice (y_I += B x_J and y_J += B^T x_I), which halves
// the bytes of a dense GEMV.  Work items are bands of whole tile rows of one
// subdomain; the CTA that finishes a subdomain's last band sums the band
// partials in a fixed order and scatters into z, so the result is
// deterministic.  Large subdomains (many bands) leave that sum to a
// row-parallel gather kernel with the same order, which keeps one CTA's
// serial sum off the end of the launch.
#include "ddg_internal.cuh"
#include "dev_common.cuh"

namespace {

constexpr int LDT = DDG_LT + 1;  // padded smem row of a 32x32 FP64 tile

__device__ __forceinline__ void tload(double* s, const double* g, int ld) {
    for (int i = threadIdx.x; i < DDG_LT * DDG_LT; i += blockDim.x) {
        int r = i >> 5, c = i & 31;
        s[r * LDT + c] = g[(size_t)r * ld + c];
    }
}

__device__ __forceinline__ void tstore(double* g, const double* s, int ld) {
    for (int i = threadIdx.x; i < DDG_LT * DDG_LT; i += blockDim.x) {
        int r = i >> 5, c = i & 31;
        g[(size_t)r * ld + c] = s[r * LDT + c];
    }
}

enum { NN = 0, NT = 1, TN = 2 };

// acc (2x2 per thread, 256 threads cover 32x32) += op(A) op(B)
template <int MODE>
__device__ __forceinline__ void tile_mac(double (&acc)[2][2], const double* A, const double* B) {
    const int r0 = (threadIdx.x >> 4) * 2, c0 = (threadIdx.x & 15) * 2;
#pragma unroll 4
    for (int m = 0; m < DDG_LT; ++m) {
        double a0, a1, b0, b1;
        if (MODE == TN) {
            a0 = A[m * LDT + r0];
            a1 = A[m * LDT + r0 + 1];
        } else {
            a0 = A[r0 * LDT + m];
            a1 = A[(r0 + 1) * LDT + m];
        }
        if (MODE == NT) {
            b0 = B[c0 * LDT + m];
            b1 = B[(c0 + 1) * LDT + m];
        } else {
            b0 = B[m * LDT + c0];
            b1 = B[m * LDT + c0 + 1];
        }
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
    }
}

__device__ __forceinline__ void acc_zero(double (&acc)[2][2]) {
    acc[0][0] = acc[0][1] = acc[1][0] = acc[1][1] = 0.0;
}

// global tile (row-major, leading dimension ld) <-> accumulator registers
__device__ __forceinline__ void acc_load(double (&acc)[2][2], const double* g, int ld) {
    const int r0 = (threadIdx.x >> 4) * 2, c0 = (threadIdx.x & 15) * 2;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc[a][b] = g[(size_t)(r0 + a) * ld + c0 + b];
}
__device__ __forceinline__ void acc_store(double* g, int ld, const double (&acc)[2][2], double s) {
    const int r0 = (threadIdx.x >> 4) * 2, c0 = (threadIdx.x & 15) * 2;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) g[(size_t)(r0 + a) * ld + c0 + b] = s * acc[a][b];
}
__device__ __forceinline__ void acc_to_smem(double* s, const double (&acc)[2][2]) {
    const int r0 = (threadIdx.x >> 4) * 2, c0 = (threadIdx.x & 15) * 2;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s[(r0 + a) * LDT + c0 + b] = acc[a][b];
}

// unblocked Cholesky of the 32x32 tile in smem (lower; upper zeroed);
// a non-positive pivot sets *bad and continues with pivot 1
__device__ void potrf32(double* S, int* bad) {
    for (int j = 0; j < DDG_LT; ++j) {
        if (threadIdx.x == 0) {
            double d = S[j * LDT + j];
            if (!(d > 0.0)) {
                *bad = 1;
                d = 1.0;
            }
            S[j * LDT + j] = sqrt(d);
        }
        __syncthreads();
        if (threadIdx.x > j && threadIdx.x < DDG_LT) S[threadIdx.x * LDT + j] /= S[j * LDT + j];
        __syncthreads();
        for (int i = threadIdx.x; i < DDG_LT * DDG_LT; i += blockDim.x) {
            int r = i >> 5, c = i & 31;
            if (c > j && r >= c) S[r * LDT + c] -= S[r * LDT + j] * S[c * LDT + j];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < DDG_LT * DDG_LT; i += blockDim.x) {
        int r = i >> 5, c = i & 31;
        if (c > r) S[r * LDT + c] = 0.0;
    }
    __syncthreads();
}

// X = L^{-1} for the lower-triangular 32x32 tile L (column-wise forward
// substitution, one thread per column)
__device__ void trtri32(const double* L, double* X) {
    for (int i = threadIdx.x; i < DDG_LT * DDG_LT; i += blockDim.x) X[(i >> 5) * LDT + (i & 31)] = 0.0;
    __syncthreads();
    if (threadIdx.x < DDG_LT) {
        const int c = threadIdx.x;
        X[c * LDT + c] = 1.0 / L[c * LDT + c];
        for (int r = c + 1; r < DDG_LT; ++r) {
            double s = 0.0;
            for (int m = c; m < r; ++m) s = fma(L[r * LDT + m], X[m * LDT + c], s);
            X[r * LDT + c] = -s / L[r * LDT + r];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- setup
__global__ void local_extract_kernel(int q0, const int32_t* __restrict__ qlist,
                                     const int64_t* __restrict__ ov_off,
                                     const int32_t* __restrict__ ov_nodes,
                                     const int64_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ col,
                                     const double* __restrict__ val, double* ws, int Np) {
    const int b = blockIdx.x, q = qlist ? qlist[q0 + b] : q0 + b;
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    double* A = ws + (size_t)b * Np * Np;
    const int32_t* nodes = ov_nodes + o;
    for (int a = threadIdx.x; a < Np; a += blockDim.x) {
        if (a >= n) {
            A[(size_t)a * Np + a] = 1.0;  // identity padding keeps the block SPD
            continue;
        }
        const int g = nodes[a];
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
            const int c = col[e];
            int lo = 0, hi = n;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (nodes[mid] < c) lo = mid + 1;
                else hi = mid;
            }
            if (lo < n && nodes[lo] == c) A[(size_t)a * Np + lo] = val[e];
        }
    }
}

// In-place: A (Np x Np, row-major) -> its inverse in the upper tiles (I <= J).
__global__ void __launch_bounds__(256) local_factor_invert_kernel(
    int q0, const int32_t* __restrict__ qlist, const int32_t* __restrict__ Tq, double* ws,
    double* invdiag, int Np, int Tmax, int* err) {
    extern __shared__ double sm[];
    double* sA = sm;
    double* sB = sm + DDG_LT * LDT;
    double* sC = sm + 2 * DDG_LT * LDT;
    __shared__ int bad;
    const int b = blockIdx.x;
    const int T = Tq[qlist ? qlist[q0 + b] : q0 + b];
    double* A = ws + (size_t)b * Np * Np;
    double* D = invdiag + (size_t)b * Tmax * DDG_LT * DDG_LT;
    auto tile = [&](int I, int J) { return A + (size_t)I * DDG_LT * Np + J * DDG_LT; };
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double acc[2][2];

    // 1) right-looking blocked Cholesky A = L L^T
    for (int k = 0; k < T; ++k) {
        tload(sA, tile(k, k), Np);
        __syncthreads();
        potrf32(sA, &bad);
        tstore(tile(k, k), sA, Np);
        trtri32(sA, sB);                         // sB = L_kk^{-1}
        tstore(D + (size_t)k * DDG_LT * DDG_LT, sB, DDG_LT);
        __syncthreads();
        for (int i = k + 1; i < T; ++i) {        // L_ik = A_ik L_kk^{-T}
            tload(sA, tile(i, k), Np);
            __syncthreads();
            acc_zero(acc);
            tile_mac<NT>(acc, sA, sB);
            __syncthreads();
            acc_store(tile(i, k), Np, acc, 1.0);
        }
        __syncthreads();
        for (int j = k + 1; j < T; ++j) {        // A_ij -= L_ik L_jk^T
            tload(sB, tile(j, k), Np);
            for (int i = j; i < T; ++i) {
                tload(sA, tile(i, k), Np);
                __syncthreads();
                acc_load(acc, tile(i, j), Np);
                double neg[2][2];
                acc_zero(neg);
                tile_mac<NT>(neg, sA, sB);
                for (int a = 0; a < 2; ++a)
                    for (int c = 0; c < 2; ++c) acc[a][c] -= neg[a][c];
                acc_store(tile(i, j), Np, acc, 1.0);
                __syncthreads();
            }
        }
        __syncthreads();
    }

    // 2) W = L^{-1} in place (lower tiles), column by column
    for (int j = 0; j < T; ++j) {
        tload(sA, D + (size_t)j * DDG_LT * DDG_LT, DDG_LT);
        __syncthreads();
        tstore(tile(j, j), sA, Np);
        __syncthreads();
        for (int i = j + 1; i < T; ++i) {
            acc_zero(acc);
            for (int m = j; m < i; ++m) {        // S = sum_m L_im W_mj
                tload(sA, tile(i, m), Np);
                tload(sB, tile(m, j), Np);
                __syncthreads();
                tile_mac<NN>(acc, sA, sB);
                __syncthreads();
            }
            acc_to_smem(sC, acc);
            tload(sA, D + (size_t)i * DDG_LT * DDG_LT, DDG_LT);
            __syncthreads();
            acc_zero(acc);
            tile_mac<NN>(acc, sA, sC);           // W_ij = -L_ii^{-1} S
            __syncthreads();
            acc_store(tile(i, j), Np, acc, -1.0);
            __syncthreads();
        }
    }

    // 3) A^{-1} = W^T W, upper tiles (I <= J); the diagonal tile of a column last
    for (int j = 0; j < T; ++j) {
        for (int i = 0; i <= j; ++i) {
            acc_zero(acc);
            for (int m = j; m < T; ++m) {
                tload(sA, tile(m, i), Np);
                tload(sB, tile(m, j), Np);
                __syncthreads();
                tile_mac<TN>(acc, sA, sB);
                __syncthreads();
            }
            acc_store(tile(i, j), Np, acc, 1.0);
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && bad) atomicExch(err, 1);
}

__global__ void local_pack_kernel(int q0, const int32_t* __restrict__ qlist, const double* __restrict__ ws,
                                  int Np,
                                  const int64_t* __restrict__ ov_off,
                                  const int32_t* __restrict__ Tq,
                                  const int64_t* __restrict__ tile_off, double* inv64,
                                  float* inv32, __nv_bfloat16* inv16) {
    const int b = blockIdx.x, q = qlist ? qlist[q0 + b] : q0 + b;
    const int n = (int)(ov_off[q + 1] - ov_off[q]);
    const int T = Tq[q];
    const double* A = ws + (size_t)b * Np * Np;
    const int64_t base = tile_off[q];
    const int wp = ddgdev::packed_narrow_width(n, T);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // warp w packs tiles w, w + nw, ... in row-major upper-triangle order
    int t = 0;
    for (int I = 0; I < T; ++I) {
        for (int J = I; J < T; ++J, ++t) {
            if (t % nw != warp) continue;
            const int ld = J == T - 1 ? wp : DDG_LT;   // stored columns of the tile
            if (lane >= ld) continue;
            const bool trap = J == I && I < T - 1;      // upper trapezoid diagonal tile
            const int gc = J * DDG_LT + lane;
            const size_t t0 = (size_t)base + ddgdev::packed_tile_start(I, J, T, wp);
            for (int r = 0; r < DDG_LT; ++r) {
                if (trap && lane < 8 * (r >> 3)) continue;
                const int gr = I * DDG_LT + r;
                const double v = (gr < n && gc < n) ? A[(size_t)gr * Np + gc] : 0.0;
                const size_t dst = t0 + (trap ? (size_t)ddgdev::packed_diag_offset(r, lane) : (size_t)r * ld + lane);
                if (inv64) inv64[dst] = v;
                if (inv32) inv32[dst] = (float)v;
                if (inv16) inv16[dst] = __float2bfloat16_rn((float)v);
            }
        }
    }
}

// ---------------------------------------------------------------- apply
// (r - A z)[g] for grid dof g: CSR rows in general, matrix-free for the
// constant-coefficient Laplacians ([6,-1] 3D, [4,-1] 2D, Dirichlet)
template <int SK, typename V, typename AV>
__device__ __forceinline__ V residual_at(int g, const int64_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ col, const AV* __restrict__ val,
                                         V rg, const V* __restrict__ z, int nx, int ny, int nz) {
    V s = rg;
    if (SK == DDG_STENCIL_7PT_3D || SK == DDG_STENCIL_5PT_2D) {
        const int i = g % nx, j = (g / nx) % ny;
        V az = (SK == DDG_STENCIL_7PT_3D ? (V)6 : (V)4) * z[g];
        if (i > 0) az -= z[g - 1];
        if (i < nx - 1) az -= z[g + 1];
        if (j > 0) az -= z[g - nx];
        if (j < ny - 1) az -= z[g + nx];
        if (SK == DDG_STENCIL_7PT_3D) {
            const int k = g / (nx * ny);
            if (k > 0) az -= z[g - nx * ny];
            if (k < nz - 1) az -= z[g + nx * ny];
        }
        s -= az;
    } else if (SK == ddgdev::SK_CSR8) {
        s -= ddgdev::csr_row_dot_unrolled<8>(g, rowptr, col, val, z, 1, 0);
    } else if (SK == ddgdev::SK_CSR16) {
        s -= ddgdev::csr_row_dot_unrolled<16>(g, rowptr, col, val, z, 1, 0);
    } else {
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) s -= (V)val[e] * z[col[e]];
    }
    return s;
}

template <int SK, typename V, typename AV>
__global__ void local_residual_kernel(int64_t a0, int64_t a1, const int32_t* __restrict__ ov_nodes,
                                      const int64_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ col,
                                      const AV* __restrict__ val, const V* __restrict__ r,
                                      const V* __restrict__ z, V* __restrict__ res, int z_zero,
                                      int nx, int ny, int nz) {
    // launched as a programmatic dependent: the row's node and r (fixed during
    // the sweep) are read before griddepcontrol.wait, z after it
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if constexpr (SK == ddgdev::SK_CSRW) {
        // a group of CSRW_G lanes per local row; the whole warp reaches the shuffles
        constexpr int G = ddgdev::CSRW_G;
        const int64_t a = a0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
        const bool live = a < a1;
        const int g = live ? ov_nodes[a] : 0;
        const V rg = live ? r[g] : (V)0;
        asm volatile("griddepcontrol.wait;" ::: "memory");
        V s = 0;
        if (!z_zero) s = ddgdev::csr_row_dot_group<G>(g, live, rowptr, col, val, z);
        if (live && (threadIdx.x & (G - 1)) == 0) res[a] = rg - s;
    } else {
        const int64_t a = a0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool live = a < a1;
        const int g = live ? ov_nodes[a] : 0;
        const V rg = live ? r[g] : (V)0;
        asm volatile("griddepcontrol.wait;" ::: "memory");
        if (!live) return;
        res[a] = z_zero ? rg : residual_at<SK>(g, rowptr, col, val, rg, z, nx, ny, nz);
    }
}

// lane layout of a 32x32 tile for 16-byte loads of element type E:
// VEC elements per load, LPR lanes per tile row, RPI rows per warp load
// (RPI == VEC), NIT loads per lane (NIT == LPR)
template <typename E> struct Lay {
    static constexpr int VEC = 16 / (int)sizeof(E);
    static constexpr int LPR = 32 / VEC;
    static constexpr int RPI = VEC;
    static constexpr int NIT = LPR;
};

template <typename E, typename V> struct Cvt;
template <> struct Cvt<double, double> {
    static __device__ __forceinline__ void load(const double* p, double (&o)[2]) {
        double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        o[0] = t.x;
        o[1] = t.y;
    }
};
template <> struct Cvt<float, float> {
    static __device__ __forceinline__ void load(const float* p, float (&o)[4]) {
        float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    }
};
template <> struct Cvt<__nv_bfloat16, float> {
    static __device__ __forceinline__ void load(const __nv_bfloat16* p, float (&o)[8]) {
        uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = __bfloat1622float2(h[i]);
            o[2 * i] = f.x;
            o[2 * i + 1] = f.y;
        }
    }
};

// x and yT (Tmax * 32 each) and the per-warp row slices yR of W warps
template <typename V, int W>
constexpr size_t local_solve_smem(int Tmax) {
    return (2 * (size_t)Tmax * DDG_LT + (size_t)W * DDG_BAND_ROWS * DDG_LT) * sizeof(V);
}

// One work item = a band of whole tile rows [I0, I1) of one subdomain's
// packed upper triangle, processed by LS_WARPS warps (a tuning parameter:
// 4 or 8).  Tile (I, J) belongs to warp J mod LS_WARPS, so the
// transposed products B^T x_I land in y[J] entries that only one warp
// writes (one shared accumulator yT, no atomics); each warp keeps the row
// products B x_J of the current row in a register and stores them once per
// row in its slice of yR (at most DDG_BAND_ROWS rows per band).  The chunk
// result yT + sum_w yR[w] is formed in a fixed order, so it is deterministic.
template <typename E, typename V, bool SPLIT, int LS_WARPS>
__global__ void __launch_bounds__(LS_WARPS * 32, (sizeof(V) == 4 ? 4 : 2) * (8 / LS_WARPS)) local_solve_kernel(
    const int4* __restrict__ items, int item_base, const int64_t* __restrict__ ov_off,
    const int32_t* __restrict__ ov_nodes, const int64_t* __restrict__ tile_off,
    const int32_t* __restrict__ Tq, const int32_t* __restrict__ nchunks,
    const int32_t* __restrict__ first_item, const int32_t* __restrict__ row_nchunks,
    const E* __restrict__ inv, const V* __restrict__ res, V* __restrict__ partial,
    unsigned* __restrict__ counter, V* __restrict__ z, int Tmax) {
    using L = Lay<E>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* x = reinterpret_cast<V*>(smraw);
    V* yT = x + Tmax * DDG_LT;
    V* yR = yT + Tmax * DDG_LT;   // [LS_WARPS][DDG_BAND_ROWS][32]
    __shared__ int am_last;

    const int gi = item_base + blockIdx.x;
    const int4 it = items[gi];
    const int q = it.x, I0 = it.y, I1 = it.z;
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    const int T = Tq[q];
    const int NP = T * DDG_LT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // launched as a programmatic dependent: the item and its metadata are
    // fixed; res, z and the tickets are read after griddepcontrol.wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        x[i] = i < n ? res[o + i] : (V)0;
        yT[i] = (V)0;
    }
    __syncthreads();

    const int g = lane / L::LPR, j = lane % L::LPR;
    const int idx = j * L::VEC + g;   // row/col owned by this lane after the reductions
    const E* sub = inv + tile_off[q];
    const int wp = ddgdev::packed_narrow_width(n, T);
    const int lane_32 = g * DDG_LT + j * L::VEC, lane_w = g * wp + j * L::VEC;
    const int kstride_w = L::RPI * wp;
    const bool lane_in_w = j * L::VEC < wp;
    V* myR = yR + warp * (DDG_BAND_ROWS * DDG_LT);

    for (int I = I0; I < I1; ++I) {
        // element offset of tile (I, I) in the packed triangle
        const size_t rowstart = ddgdev::packed_tile_start(I, I, T, wp);
        V racc = (V)0;
        // one tile's products: row part into racc, transposed part into yT[J]
        auto tile = [&](int J, const V (&e)[L::NIT][L::VEC]) {
            V xj[L::VEC];
#pragma unroll
            for (int v = 0; v < L::VEC; ++v) xj[v] = x[J * DDG_LT + j * L::VEC + v];
            V rp[L::NIT];
#pragma unroll
            for (int k = 0; k < L::NIT; ++k) {
                V s = (V)0;
#pragma unroll
                for (int v = 0; v < L::VEC; ++v) s = fma(e[k][v], xj[v], s);
                rp[k] = s;
            }
            racc += ddgdev::reduce_scatter<L::NIT, 1>(rp, j);
            if (I != J) {
                V cp[L::VEC];
#pragma unroll
                for (int v = 0; v < L::VEC; ++v) cp[v] = (V)0;
#pragma unroll
                for (int k = 0; k < L::NIT; ++k) {
                    const V xi = x[I * DDG_LT + k * L::RPI + g];
#pragma unroll
                    for (int v = 0; v < L::VEC; ++v) cp[v] = fma(e[k][v], xi, cp[v]);
                }
                yT[J * DDG_LT + idx] += ddgdev::reduce_scatter<L::VEC, L::LPR>(cp, g);
            }
        };
        // tiles J < T-1 are 32 wide, the last tile column wp wide (lanes past
        // wp read zeros).  4- and 8-byte tiles: one loop selecting precomputed
        // offsets and strides; 2-byte tiles (instruction-bound): the full
        // tiles in a loop of their own and the narrow one after it.
        auto load_tile = [&](int J, bool last, V (&e)[L::NIT][L::VEC]) {
            // tiles right of the diagonal follow the trapezoid diagonal tile;
            // J == I here only for the narrow diagonal tile of band row T-1
            const size_t toff = J == I ? 0 : (size_t)ddgdev::PACKED_DIAG + (size_t)(J - I - 1) * 1024;
            const E* tp = sub + rowstart + toff + (last ? lane_w : lane_32);
            const int ks = last ? kstride_w : L::RPI * DDG_LT;
            if (!last || lane_in_w) {
#pragma unroll
                for (int k = 0; k < L::NIT; ++k) Cvt<E, V>::load(tp + k * ks, e[k]);
            } else {
#pragma unroll
                for (int k = 0; k < L::NIT; ++k)
#pragma unroll
                    for (int v = 0; v < L::VEC; ++v) e[k][v] = (V)0;
            }
        };
        int J = I + ((warp - I) % LS_WARPS + LS_WARPS) % LS_WARPS;
        if (J == I && I < T - 1) {
            // trapezoid diagonal tile: chunks left of the row's 8-column block
            // are not stored (zero here); the row products use every stored
            // chunk, the transposed products skip the 8x8 diagonal blocks,
            // which are stored in full
            const E* dp = sub + rowstart;
            const int cb = (j * L::VEC) >> 3;
            V e[L::NIT][L::VEC];
            bool tr[L::NIT];
#pragma unroll
            for (int k = 0; k < L::NIT; ++k) {
                const int rk = g + k * L::RPI, rb = rk >> 3;
                tr[k] = cb > rb;
                if (cb >= rb) {
                    Cvt<E, V>::load(dp + ddgdev::packed_diag_offset(rk, j * L::VEC), e[k]);
                } else {
#pragma unroll
                    for (int v = 0; v < L::VEC; ++v) e[k][v] = (V)0;
                }
            }
            V xj[L::VEC];
#pragma unroll
            for (int v = 0; v < L::VEC; ++v) xj[v] = x[I * DDG_LT + j * L::VEC + v];
            V rp[L::NIT];
#pragma unroll
            for (int k = 0; k < L::NIT; ++k) {
                V s = (V)0;
#pragma unroll
                for (int v = 0; v < L::VEC; ++v) s = fma(e[k][v], xj[v], s);
                rp[k] = s;
            }
            racc += ddgdev::reduce_scatter<L::NIT, 1>(rp, j);
            V cp[L::VEC];
#pragma unroll
            for (int v = 0; v < L::VEC; ++v) cp[v] = (V)0;
#pragma unroll
            for (int k = 0; k < L::NIT; ++k) {
                if (!tr[k]) continue;
                const V xi = x[I * DDG_LT + k * L::RPI + g];
#pragma unroll
                for (int v = 0; v < L::VEC; ++v) cp[v] = fma(e[k][v], xi, cp[v]);
            }
            yT[I * DDG_LT + idx] += ddgdev::reduce_scatter<L::VEC, L::LPR>(cp, g);
            J += LS_WARPS;
        }
        if constexpr (sizeof(E) == 2) {
            for (; J < T - 1; J += LS_WARPS) {
                V e[L::NIT][L::VEC];
                load_tile(J, false, e);
                tile(J, e);
            }
            if (J == T - 1) {
                V e[L::NIT][L::VEC];
                load_tile(J, true, e);
                tile(J, e);
            }
        } else {
            for (; J < T; J += LS_WARPS) {
                V e[L::NIT][L::VEC];
                load_tile(J, J == T - 1, e);
                tile(J, e);
            }
        }
        myR[(I - I0) * DDG_LT + idx] = racc;
    }
    __syncthreads();
    // rows above the band get nothing from it: only rows >= 32 I0 are stored,
    // and the chunk sums stop at the last band that starts at or above a row
    V* pout = partial + (size_t)gi * Tmax * DDG_LT;
    for (int i = I0 * DDG_LT + threadIdx.x; i < NP; i += blockDim.x) {
        V s = yT[i];
        const int I = i >> 5;
        if (I >= I0 && I < I1) {
#pragma unroll
            for (int w = 0; w < LS_WARPS; ++w) s += yR[(w * DDG_BAND_ROWS + I - I0) * DDG_LT + (i & 31)];
        }
        pout[i] = s;
    }
    if (SPLIT) return;  // local_gather_kernel sums the chunks
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned tk = atomicAdd(&counter[q], 1u);
        am_last = (tk == (unsigned)nchunks[q] - 1u);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int fi = first_item[q];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        V s = (V)0;
        const int nci = row_nchunks[o + i];
        for (int c = 0; c < nci; ++c) s += __ldcg(partial + (size_t)(fi + c) * Tmax * DDG_LT + i);
        const int gnode = ov_nodes[o + i];
        z[gnode] += s;
    }
    if (threadIdx.x == 0) counter[q] = 0u;
}

// z[Omega~_i] += sum over the chunks of subdomain i of their partials, one
// thread per local row of the colour; the chunks are summed in the same
// fixed order as in the last-CTA path, so both give the same bits.
template <typename V>
__global__ void local_gather_kernel(int64_t a0, int64_t a1, const int32_t* __restrict__ ov_sub,
                                    const int64_t* __restrict__ ov_off,
                                    const int32_t* __restrict__ ov_nodes,
                                    const int32_t* __restrict__ nchunks,
                                    const int32_t* __restrict__ first_item,
                                    const int32_t* __restrict__ row_nchunks,
                                    const V* __restrict__ partial, int Tmax, V* __restrict__ z) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t a = a0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= a1) return;
    const int q = ov_sub[a];
    const int i = (int)(a - ov_off[q]);
    const int fi = first_item[q];
    const int nc = row_nchunks[a];
    const size_t stride = (size_t)Tmax * DDG_LT;
    const V* p = partial + (size_t)fi * stride + i;
    V s = (V)0;
    int c = 0;
    for (; c + 8 <= nc; c += 8) {
        V v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + (size_t)(c + k) * stride);
#pragma unroll
        for (int k = 0; k < 8; ++k) s += v[k];
    }
    for (; c < nc; ++c) s += __ldcg(p + (size_t)c * stride);
    z[ov_nodes[a]] += s;
}

}  // namespace

namespace ddg {

void local_extract_factor_invert(ddg_handle h, int q0, int q1, const int32_t* qlist, double* ws,
                                 double* invdiag) {
    const int nb = q1 - q0;
    if (nb <= 0) return;
    const int Np = h->Tmax * DDG_LT;
    DDG_CUDA(cudaMemsetAsync(ws, 0, (size_t)nb * Np * Np * sizeof(double), h->stream));
    local_extract_kernel<<<nb, 256, 0, h->stream>>>(q0, qlist, h->ov_off, h->ov_nodes, h->rowptr, h->col,
                                                    h->val64, ws, Np);
    DDG_CHECK_LAUNCH();
    const size_t smem = 3 * DDG_LT * LDT * sizeof(double);
    local_factor_invert_kernel<<<nb, 256, smem, h->stream>>>(q0, qlist, h->Tq, ws, invdiag, Np, h->Tmax,
                                                            h->errflags + E_LOCAL_SPD);
    DDG_CHECK_LAUNCH();
}

void local_pack(ddg_handle h, int q0, int q1, const int32_t* qlist, const double* ws) {
    const int nb = q1 - q0;
    if (nb <= 0) return;
    local_pack_kernel<<<nb, 256, 0, h->stream>>>(q0, qlist, ws, h->Tmax * DDG_LT, h->ov_off, h->Tq,
                                                 h->tile_off, h->inv64, h->inv32, h->inv16);
    DDG_CHECK_LAUNCH();
}

template <int SK>
static void launch_residual(ddg_handle h, int64_t a0, int64_t a1, bool z_zero, int prec) {
    const int threads = 256;
    const int64_t lanes = (a1 - a0) * (SK == ddgdev::SK_CSRW ? ddgdev::CSRW_G : 1);
    const unsigned blocks = (unsigned)((lanes + threads - 1) / threads);
    const int zz = z_zero ? 1 : 0;
    if (prec == DDG_PREC_FP64)
        launch_pdl(h, local_residual_kernel<SK, double, double>, dim3(blocks), dim3(threads), 0, a0, a1,
                   (const int32_t*)h->ov_nodes, (const int64_t*)h->rowptr, (const int32_t*)h->col,
                   (const double*)h->val64, (const double*)h->rin64, (const double*)h->z64, h->res64, zz,
                   h->nx, h->ny, h->nz);
    else
        launch_pdl(h, local_residual_kernel<SK, float, float>, dim3(blocks), dim3(threads), 0, a0, a1,
                   (const int32_t*)h->ov_nodes, (const int64_t*)h->rowptr, (const int32_t*)h->col,
                   (const float*)h->val32, (const float*)h->r32, (const float*)h->z32, h->res32, zz, h->nx,
                   h->ny, h->nz);
}

void local_residual(ddg_handle h, int c, bool z_zero, int prec) {
    const int64_t a0 = h->h_crow_off[c], a1 = h->h_crow_off[c + 1];
    if (a1 <= a0) return;
#define LR_CALL(SK) launch_residual<SK>(h, a0, a1, z_zero, prec)
    DDG_DISPATCH_SK(h, LR_CALL);
#undef LR_CALL
}

template <typename E, typename V, int W>
static void launch_local_solve_w(ddg_handle h, int c, const E* inv, const V* res, V* partial, V* z) {
    const int i0 = h->h_citem_off[c], i1 = h->h_citem_off[c + 1];
    if (i1 <= i0) return;
    const size_t smem = local_solve_smem<V, W>(h->Tmax);
    auto kern = h->split_gather ? local_solve_kernel<E, V, true, W> : local_solve_kernel<E, V, false, W>;
    launch_pdl(h, kern, dim3(i1 - i0), dim3(W * 32), smem, (const int4*)h->items, i0,
               (const int64_t*)h->ov_off, (const int32_t*)h->ov_nodes, (const int64_t*)h->tile_off,
               (const int32_t*)h->Tq, (const int32_t*)h->nchunks, (const int32_t*)h->first_item,
               (const int32_t*)h->row_nchunks, inv, res, partial, h->counters, z, h->Tmax);
    if (h->split_gather) {
        const int64_t a0 = h->h_crow_off[c], a1 = h->h_crow_off[c + 1];
        const unsigned blocks = (unsigned)((a1 - a0 + 255) / 256);
        launch_pdl(h, local_gather_kernel<V>, dim3(blocks), dim3(256), 0, a0, a1, (const int32_t*)h->ov_sub,
                   (const int64_t*)h->ov_off, (const int32_t*)h->ov_nodes, (const int32_t*)h->nchunks,
                   (const int32_t*)h->first_item, (const int32_t*)h->row_nchunks, (const V*)partial,
                   h->Tmax, z);
    }
}

template <typename E, typename V>
static void launch_local_solve(ddg_handle h, int c, const E* inv, const V* res, V* partial, V* z) {
    if (h->ls_warps == 4) launch_local_solve_w<E, V, 4>(h, c, inv, res, partial, z);
    else launch_local_solve_w<E, V, 8>(h, c, inv, res, partial, z);
}

// The dynamic shared-memory limit is a property of the kernel on each device,
// shared by all handles there: raise it to the largest size any handle on
// that device needs, never lower it.
template <typename E, typename V, int W>
static void configure_local_solve(int Tmax) {
    static PerDeviceMax configured;
    const int smem = (int)local_solve_smem<V, W>(Tmax);
    int dev = -1;
    if (!configured.needs(smem, dev)) return;
    DDG_CUDA(cudaFuncSetAttribute(local_solve_kernel<E, V, false, W>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    DDG_CUDA(cudaFuncSetAttribute(local_solve_kernel<E, V, true, W>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    configured.commit(dev, smem);
}

void local_configure(ddg_handle h) {
    configure_local_solve<double, double, 8>(h->Tmax);
    configure_local_solve<float, float, 8>(h->Tmax);
    configure_local_solve<__nv_bfloat16, float, 8>(h->Tmax);
    configure_local_solve<double, double, 4>(h->Tmax);
    configure_local_solve<float, float, 4>(h->Tmax);
    configure_local_solve<__nv_bfloat16, float, 4>(h->Tmax);
}

void local_solve_colour(ddg_handle h, int c, int prec) {
    if (h->bl.on) {
        band_local_solve_colour(h, c, prec);
        return;
    }
    if (prec == DDG_PREC_FP64)
        launch_local_solve<double, double>(h, c, h->inv64, h->res64, h->partial64, h->z64);
    else if (prec == DDG_PREC_FP32)
        launch_local_solve<float, float>(h, c, h->inv32, h->res32, h->partial32, h->z32);
    else
        launch_local_solve<__nv_bfloat16, float>(h, c, h->inv16, h->res32, h->partial32, h->z32);
}

}  // namespace ddg
