// Many right-hand sides at once (m <= DDG_MCHUNK per group): the same PCG and
// the same preconditioner (Sec. 6, Sec. 7) on an n x m block stored dof-major
// (entry (g, j) at g * m + j), with per-column CG scalars, convergence masks
// and restarts.  Every stage is a multi-column version of the single-RHS
// kernel: the preconditioner reads each local inverse once per colour phase
// for all m columns, which is what makes batching pay.
#include "ddg_internal.cuh"
#include <algorithm>

#include "dev_common.cuh"

namespace {

constexpr int MT = 256;

// threads of the column-mapped kernels: a multiple of m, at most 256
inline int col_block(int m) { return (MT / m) * m; }

// A z at dof g, column c of an n x m block (matrix-free for the Laplacians)
template <int SK, typename V, typename AV>
__device__ __forceinline__ V apply_row(int g, int c, int m, const int64_t* __restrict__ rowptr,
                                       const int32_t* __restrict__ col, const AV* __restrict__ val,
                                       const V* __restrict__ z, int nx, int ny, int nz) {
    if (SK == DDG_STENCIL_7PT_3D || SK == DDG_STENCIL_5PT_2D) {
        const int i = g % nx, j = (g / nx) % ny;
        V az = (SK == DDG_STENCIL_7PT_3D ? (V)6 : (V)4) * z[(int64_t)g * m + c];
        if (i > 0) az -= z[(int64_t)(g - 1) * m + c];
        if (i < nx - 1) az -= z[(int64_t)(g + 1) * m + c];
        if (j > 0) az -= z[(int64_t)(g - nx) * m + c];
        if (j < ny - 1) az -= z[(int64_t)(g + nx) * m + c];
        if (SK == DDG_STENCIL_7PT_3D) {
            const int k = g / (nx * ny);
            if (k > 0) az -= z[(int64_t)(g - nx * ny) * m + c];
            if (k < nz - 1) az -= z[(int64_t)(g + nx * ny) * m + c];
        }
        return az;
    }
    if (SK == ddgdev::SK_CSR8) return ddgdev::csr_row_dot_unrolled<8>(g, rowptr, col, val, z, m, c);
    if (SK == ddgdev::SK_CSR16) return ddgdev::csr_row_dot_unrolled<16>(g, rowptr, col, val, z, m, c);
    V s = 0;
    for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) s = fma((V)val[e], z[(int64_t)col[e] * m + c], s);
    return s;
}

// per-column deterministic reduction: thread t owns column t % m; block
// partials summed in block order by the last block.  Returns true in the
// last block, with tot[c] valid for threads t < m (column t).
template <int NV>
__device__ bool reduce_cols(double (&v)[NV], int m, double* partials, unsigned* counter,
                            double (&tot)[NV]) {
    __shared__ double sh[MT];
    __shared__ bool last;
    const int rpb = blockDim.x / m;
    double bs[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        __syncthreads();
        sh[threadIdx.x] = v[q];
        __syncthreads();
        bs[q] = 0.0;
        if ((int)threadIdx.x < m)
            for (int r = 0; r < rpb; ++r) bs[q] += sh[r * m + threadIdx.x];
    }
    if ((int)threadIdx.x < m)
        for (int q = 0; q < NV; ++q) partials[((size_t)blockIdx.x * NV + q) * m + threadIdx.x] = bs[q];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // the rpb thread groups of a column sum interleaved blocks with four
    // independent accumulators, then the groups combine in group order
    const int gq = threadIdx.x / m, cc = threadIdx.x % m;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        unsigned b = gq;
        const unsigned step = (unsigned)rpb;
        for (; b + 3 * step < gridDim.x; b += 4 * step) {
            s0 += __ldcg(partials + ((size_t)b * NV + q) * m + cc);
            s1 += __ldcg(partials + ((size_t)(b + step) * NV + q) * m + cc);
            s2 += __ldcg(partials + ((size_t)(b + 2 * step) * NV + q) * m + cc);
            s3 += __ldcg(partials + ((size_t)(b + 3 * step) * NV + q) * m + cc);
        }
        for (; b < gridDim.x; b += step) s0 += __ldcg(partials + ((size_t)b * NV + q) * m + cc);
        __syncthreads();
        sh[threadIdx.x] = (s0 + s1) + (s2 + s3);
        __syncthreads();
        if ((int)threadIdx.x < m) {
            double s = 0.0;
            for (int r = 0; r < rpb; ++r) s += sh[r * m + threadIdx.x];
            tot[q] = s;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// scalars: sc[slot * DDG_MCHUNK + column]
__device__ __forceinline__ double& S(double* sc, int slot, int c) { return sc[slot * DDG_MCHUNK + c]; }

template <int SK>
__global__ void __launch_bounds__(MT) spmv_multi_kernel(int64_t n, int m, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ P, double* __restrict__ Q,
                                                        int nx, int ny, int nz, double* partials,
                                                        unsigned* counter, double* sc,
                                                        const int* __restrict__ active) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m, rl = threadIdx.x / m;
    double acc[1] = {0.0};
    if ((int)threadIdx.x < rpb * m)
        for (int64_t g = (int64_t)blockIdx.x * rpb + rl; g < n; g += (int64_t)gridDim.x * rpb) {
            const double q = apply_row<SK, double, double>((int)g, c, m, rowptr, col, val, P, nx, ny, nz);
            Q[g * m + c] = q;
            acc[0] = fma(P[g * m + c], q, acc[0]);
        }
    double tot[1];
    if (reduce_cols<1>(acc, m, partials, counter, tot) && (int)threadIdx.x < m) {
        const double pq = tot[0];
        S(sc, S_PQ, c) = pq;
        if (active[c]) {
            S(sc, S_ALPHA, c) = S(sc, S_RZ, c) / pq;
            if (!(pq > 0.0) || pq != pq) S(sc, S_FLAG, c) = 1.0;
        } else {
            S(sc, S_ALPHA, c) = 0.0;
        }
    }
}

__global__ void __launch_bounds__(MT) update_ur_multi_kernel(int64_t n, int m, double* __restrict__ U,
                                                             double* __restrict__ R,
                                                             const double* __restrict__ P,
                                                             const double* __restrict__ Q,
                                                             double* partials, unsigned* counter,
                                                             double* sc) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m, rl = threadIdx.x / m;
    const double alpha = S(sc, S_ALPHA, c);
    double acc[1] = {0.0};
    if ((int)threadIdx.x < rpb * m)
        for (int64_t g = (int64_t)blockIdx.x * rpb + rl; g < n; g += (int64_t)gridDim.x * rpb) {
            const int64_t e = g * m + c;
            U[e] = fma(alpha, P[e], U[e]);
            const double r = fma(-alpha, Q[e], R[e]);
            R[e] = r;
            acc[0] = fma(r, r, acc[0]);
        }
    double tot[1];
    if (reduce_cols<1>(acc, m, partials, counter, tot) && (int)threadIdx.x < m) {
        S(sc, S_RR, c) = tot[0];
        if (tot[0] != tot[0]) S(sc, S_FLAG, c) = 1.0;
    }
}

// rho' = r^T z, qz = q^T z per column; beta = FR / PR, or 0 for a column
// that restarts; rho <- rho' for active columns
template <typename ZV>
__global__ void __launch_bounds__(MT) dots_multi_kernel(int64_t n, int m, const double* __restrict__ R,
                                                        const double* __restrict__ Q,
                                                        const ZV* __restrict__ Z, int pr,
                                                        double* partials, unsigned* counter, double* sc,
                                                        const int* __restrict__ active,
                                                        const int* __restrict__ restart) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m, rl = threadIdx.x / m;
    double acc[2] = {0.0, 0.0};
    if ((int)threadIdx.x < rpb * m)
        for (int64_t g = (int64_t)blockIdx.x * rpb + rl; g < n; g += (int64_t)gridDim.x * rpb) {
            const int64_t e = g * m + c;
            const double z = (double)Z[e];
            acc[0] = fma(R[e], z, acc[0]);
            acc[1] = fma(Q[e], z, acc[1]);
        }
    double tot[2];
    if (reduce_cols<2>(acc, m, partials, counter, tot) && (int)threadIdx.x < m) {
        if (!active[c]) {
            S(sc, S_BETA, c) = 0.0;
        } else {
            const double rz = tot[0];
            double beta = 0.0;
            if (!restart[c]) beta = pr ? (-S(sc, S_ALPHA, c) * tot[1] / S(sc, S_RZ, c)) : (rz / S(sc, S_RZ, c));
            S(sc, S_BETA, c) = beta;
            S(sc, S_RZ, c) = rz;
            if (rz != rz) S(sc, S_FLAG, c) = 1.0;
        }
    }
}

// element kernels over n x m blocks: block = rpb rows x m columns, so the
// column is threadIdx.x % m and no per-element 64-bit division is needed
template <typename ZV>
__global__ void update_p_multi_kernel(int64_t n, int m, double* __restrict__ P, const ZV* __restrict__ Z,
                                      const double* __restrict__ sc, const int* __restrict__ active) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m;
    const int64_t g = (int64_t)blockIdx.x * rpb + threadIdx.x / m;
    if (g >= n || !active[c]) return;
    const int64_t e = g * m + c;
    P[e] = fma(sc[S_BETA * DDG_MCHUNK + c], P[e], (double)Z[e]);
}

// per-column ||a - A b||^2 (true residual) or ||a||^2 (b = null), into slot
template <int SK>
__global__ void __launch_bounds__(MT) resnorm_multi_kernel(int64_t n, int m, const int64_t* __restrict__ rowptr,
                                                           const int32_t* __restrict__ col,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ A_, const double* __restrict__ B_,
                                                           double* __restrict__ out, int nx, int ny, int nz,
                                                           double* partials, unsigned* counter, double* sc,
                                                           int slot) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m, rl = threadIdx.x / m;
    double acc[1] = {0.0};
    if ((int)threadIdx.x < rpb * m)
        for (int64_t g = (int64_t)blockIdx.x * rpb + rl; g < n; g += (int64_t)gridDim.x * rpb) {
            double r = A_[g * m + c];
            if (B_) r -= apply_row<SK, double, double>((int)g, c, m, rowptr, col, val, B_, nx, ny, nz);
            if (out) out[g * m + c] = r;
            acc[0] = fma(r, r, acc[0]);
        }
    double tot[1];
    if (reduce_cols<1>(acc, m, partials, counter, tot) && (int)threadIdx.x < m) S(sc, slot, c) = tot[0];
}

// copy the columns with replace[c] != 0 from src into dst (restart with the true residual)
__global__ void replace_cols_kernel(int64_t n, int m, const double* __restrict__ src, double* __restrict__ dst,
                                    const int* __restrict__ replace) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m;
    const int64_t g = (int64_t)blockIdx.x * rpb + threadIdx.x / m;
    if (g >= n || !replace[c]) return;
    dst[g * m + c] = src[g * m + c];
}

// dst[g, k0 + t] = src[g, j0 + t] for t < cnt (column blocks of dof-major arrays)
__global__ void copy_cols_kernel(int64_t n, const double* __restrict__ src, int ms, int j0,
                                 double* __restrict__ dst, int md, int k0, int cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * cnt) return;
    const int64_t g = e / cnt;
    const int t = (int)(e % cnt);
    dst[g * md + k0 + t] = src[g * ms + j0 + t];
}

__global__ void to_float_n_kernel(int64_t cnt, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < cnt) b[g] = (float)a[g];
}

// ---------------------------------------------------------------- preconditioner
template <int SK>
__global__ void local_residual_multi_kernel(int64_t a0, int64_t a1, int m, const int32_t* __restrict__ ov_nodes,
                                            const int64_t* __restrict__ rowptr,
                                            const int32_t* __restrict__ col, const float* __restrict__ val,
                                            const float* __restrict__ r, const float* __restrict__ z,
                                            float* __restrict__ res, int z_zero, int nx, int ny, int nz) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m;
    const int64_t a = a0 + (int64_t)blockIdx.x * rpb + threadIdx.x / m;
    if (a >= a1) return;
    const int g = ov_nodes[a];
    float s = r[(int64_t)g * m + c];
    if (!z_zero) s -= apply_row<SK, float, float>(g, c, m, rowptr, col, val, z, nx, ny, nz);
    res[a * m + c] = s;
}

// Y_I = sum_J A_IJ X_J for one 32-row tile row I of one subdomain, all m
// columns; A_IJ is the stored tile (I, J) for J >= I and the transpose of
// (J, I) below the diagonal.  z[rows of I] += Y_I.
template <typename E>
__global__ void __launch_bounds__(MT) local_solve_multi_kernel(
    const int2* __restrict__ items, int item_base, const int64_t* __restrict__ ov_off,
    const int32_t* __restrict__ ov_nodes, const int64_t* __restrict__ tile_off,
    const int32_t* __restrict__ Tq, const E* __restrict__ inv, const float* __restrict__ res,
    float* __restrict__ z, int m) {
    __shared__ float sB[DDG_LT][DDG_LT + 1];
    __shared__ float sX[DDG_LT][DDG_MCHUNK];
    const int2 it = items[item_base + blockIdx.x];
    const int q = it.x, I = it.y;
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    const int T = Tq[q];
    const int r = threadIdx.x >> 3, cg = threadIdx.x & 7;
    float acc[DDG_MCHUNK / 8];
#pragma unroll
    for (int u = 0; u < DDG_MCHUNK / 8; ++u) acc[u] = 0.f;
    const E* base = inv + (size_t)tile_off[q] * 1024;
    for (int J = 0; J < T; ++J) {
        const bool upper = J >= I;
        const int a = upper ? I : J, b = upper ? J : I;
        const E* tp = base + ((size_t)a * T - (size_t)a * (a - 1) / 2 + (b - a)) * 1024;
        for (int e = threadIdx.x; e < 1024; e += MT) {
            const int rr = e >> 5, kk = e & 31;
            const float v = (float)tp[e];
            if (upper) sB[rr][kk] = v;
            else sB[kk][rr] = v;
        }
        for (int e = threadIdx.x; e < DDG_LT * m; e += MT) {
            const int k = e / m, c = e % m;
            const int row = J * DDG_LT + k;
            sX[k][c] = row < n ? res[(o + row) * m + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < DDG_LT; ++k) {
            const float bv = sB[r][k];
#pragma unroll
            for (int u = 0; u < DDG_MCHUNK / 8; ++u)
                if (cg + 8 * u < m) acc[u] = fma(bv, sX[k][cg + 8 * u], acc[u]);
        }
        __syncthreads();
    }
    const int row = I * DDG_LT + r;
    if (row < n) {
        const int g = ov_nodes[o + row];
#pragma unroll
        for (int u = 0; u < DDG_MCHUNK / 8; ++u)
            if (cg + 8 * u < m) z[(int64_t)g * m + cg + 8 * u] += acc[u];
    }
}

// c[(coff_s + jj) m + col] = sum_{g in Omega_s} Q[g, jj] (r - A z)[g, col];
// each thread keeps four nodes in flight (independent load chains)
template <int SK, int KM>
__global__ void __launch_bounds__(MT) coarse_restrict_multi_kernel(
    const int64_t* __restrict__ sub_off, const int32_t* __restrict__ sub_nodes,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
    const float* __restrict__ r, const float* __restrict__ z, const float* __restrict__ Q, int kmax,
    const int32_t* __restrict__ coff, float* __restrict__ cvec, int m, int nx, int ny, int nz) {
    extern __shared__ float shm[];   // [groups][kmax][m]
    const int s = blockIdx.x;
    const int groups = blockDim.x / m;
    const int c = threadIdx.x % m, gq = threadIdx.x / m;
    float acc[KM];
#pragma unroll
    for (int jj = 0; jj < KM; ++jj) acc[jj] = 0.f;
    const int64_t b0 = sub_off[s], b1 = sub_off[s + 1];
    int64_t a = b0 + gq;
    for (; a + 3 * groups < b1; a += 4 * groups) {
        float w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int g = sub_nodes[a + u * groups];
            w[u] = r[(int64_t)g * m + c] - apply_row<SK, float, float>(g, c, m, rowptr, col, val, z, nx, ny, nz);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float* qa = Q + (a + u * groups) * kmax;
#pragma unroll
            for (int jj = 0; jj < KM; ++jj)
                if (jj < kmax) acc[jj] = fma(qa[jj], w[u], acc[jj]);
        }
    }
    for (; a < b1; a += groups) {
        const int g = sub_nodes[a];
        const float w = r[(int64_t)g * m + c] - apply_row<SK, float, float>(g, c, m, rowptr, col, val, z, nx, ny, nz);
        const float* qa = Q + a * kmax;
#pragma unroll
        for (int jj = 0; jj < KM; ++jj)
            if (jj < kmax) acc[jj] = fma(qa[jj], w, acc[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < KM; ++jj)
        if (jj < kmax) shm[(gq * kmax + jj) * m + c] = acc[jj];
    __syncthreads();
    const int ks = coff[s + 1] - coff[s];
    for (int e = threadIdx.x; e < ks * m; e += blockDim.x) {
        const int jj = e / m, cc = e % m;
        float t = 0.f;
        for (int g2 = 0; g2 < groups; ++g2) t += shm[(g2 * kmax + jj) * m + cc];
        cvec[(int64_t)(coff[s] + jj) * m + cc] = t;
    }
}

// Coarse GEMMs of the batched path: (32-row tile, CG_KS-column split) items
constexpr int CG_ROWS = 32, CG_KS = 128;

// ---------------------------------------------------------------- persistent coarse solve
// The whole block-bidiagonal coarse solve for m columns in one cooperative
// launch: every GEMM of the recurrence is split into (32-row tile, 128-column
// split) items spread over the co-resident CTAs, a grid barrier separates the
// partial products from their reduction (done by all threads), and another
// separates the reduction from the next GEMM.  Barrier waits are bounded: a
// wait that runs out sets the error flag and the kernel returns.
struct CoarseStep {            // one GEMM of the recurrence
    const int64_t* rowptr;
    const int32_t* lo;
    const int32_t* hi;
    const float* vals;
    int r0, cbase;
    const float* x;
    const float* a;
    float sign;
    float* out;
};

// partial products of one (row tile, split) item of a step
__device__ void coarse_item(const CoarseStep& S, int B, int rt, int sp, int m, float* __restrict__ part,
                            float (*sM)[33], float (*sX)[DDG_MCHUNK], int* rlo, int* rhi, int64_t* rptr) {
    const int row0 = S.r0 + rt * CG_ROWS;
    const int t = threadIdx.x, r = t >> 3, cg = t & 7;
    __syncthreads();
    if (t < CG_ROWS) {
        rlo[t] = S.lo[row0 + t];
        rhi[t] = S.hi[row0 + t];
        rptr[t] = S.rowptr[row0 + t];
    }
    __syncthreads();
    const int c_lo = S.cbase + sp * CG_KS, c_hi = c_lo + CG_KS;
    int ulo = c_hi, uhi = c_lo;
    for (int q = 0; q < CG_ROWS; ++q)
        if (rhi[q] > rlo[q]) {
            ulo = min(ulo, max(rlo[q], c_lo));
            uhi = max(uhi, min(rhi[q], c_hi));
        }
    float acc[DDG_MCHUNK / 8];
#pragma unroll
    for (int u = 0; u < DDG_MCHUNK / 8; ++u) acc[u] = 0.f;
    for (int jc = c_lo + ((ulo - c_lo) & ~31); jc < uhi; jc += 32) {
        for (int e = t; e < CG_ROWS * 32; e += MT) {
            const int rr = e >> 5, jj = e & 31, j = jc + jj;
            sM[rr][jj] = (j >= rlo[rr] && j < rhi[rr]) ? S.vals[rptr[rr] + (j - rlo[rr])] : 0.f;
        }
        for (int e = t; e < 32 * m; e += MT) {
            const int jj = e / m, c = e % m;
            sX[jj][c] = S.x[(int64_t)(jc + jj) * m + c];
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < 32; ++jj) {
            const float mv = sM[r][jj];
#pragma unroll
            for (int u = 0; u < DDG_MCHUNK / 8; ++u)
                if (cg + 8 * u < m) acc[u] = fma(mv, sX[jj][cg + 8 * u], acc[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < DDG_MCHUNK / 8; ++u)
        if (cg + 8 * u < m) part[((size_t)sp * B + rt * CG_ROWS + r) * m + cg + 8 * u] = acc[u];
}

__global__ void __launch_bounds__(MT) coarse_solve_persistent_kernel(
    ProfileMat Dm, ProfileMat Em, ProfileMat Dt, ProfileMat Et, int B, int nK, int m,
    const float* __restrict__ c, float* y, float* t, float* x, float* part, ddgdev::GridBar* gb, int* err) {
    __shared__ float sM[CG_ROWS][33];
    __shared__ float sX[32][DDG_MCHUNK];
    __shared__ int rlo[CG_ROWS], rhi[CG_ROWS];
    __shared__ int64_t rptr[CG_ROWS];
    const int nsplit = (B + CG_KS - 1) / CG_KS;
    const int ntiles = B / CG_ROWS;
    const int nitems = ntiles * nsplit;
    const unsigned G = gridDim.x;
    auto run = [&](const CoarseStep& S) -> bool {
        for (int it = blockIdx.x; it < nitems; it += G)
            coarse_item(S, B, it / nsplit, it % nsplit, m, part, sM, sX, rlo, rhi, rptr);
        if (!ddgdev::grid_barrier(gb, G, err)) return false;
        // out[rows of the step] = a + sign * sum of the split partials
        const int64_t tot = (int64_t)B * m;
        for (int64_t e = (int64_t)blockIdx.x * MT + threadIdx.x; e < tot; e += (int64_t)G * MT) {
            const float* pp = part + e;
            const size_t st = (size_t)B * m;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int q = 0;
            for (; q + 3 < nsplit; q += 4) {
                s0 += __ldcg(pp + (size_t)q * st);
                s1 += __ldcg(pp + (size_t)(q + 1) * st);
                s2 += __ldcg(pp + (size_t)(q + 2) * st);
                s3 += __ldcg(pp + (size_t)(q + 3) * st);
            }
            for (; q < nsplit; ++q) s0 += __ldcg(pp + (size_t)q * st);
            const int64_t o = (int64_t)S.r0 * m + e;
            S.out[o] = (S.a ? S.a[o] : 0.f) + S.sign * ((s0 + s1) + (s2 + s3));
        }
        return ddgdev::grid_barrier(gb, G, err);
    };
    // forward: y_K = D_K (c_K - E_K y_{K-1})
    for (int K = 0; K < nK; ++K) {
        const float* in = c;
        if (K > 0) {
            if (!run(CoarseStep{Em.rowptr, Em.lo, Em.hi, Em.v32, K * B, (K - 1) * B, y, c, -1.f, t})) return;
            in = t;
        }
        if (!run(CoarseStep{Dm.rowptr, Dm.lo, Dm.hi, Dm.v32, K * B, K * B, in, nullptr, 1.f, y})) return;
    }
    // backward: x_K = D_K^T (y_K - E_{K+1}^T x_{K+1})
    for (int K = nK - 1; K >= 0; --K) {
        const float* in = y;
        if (K < nK - 1) {
            if (!run(CoarseStep{Et.rowptr, Et.lo, Et.hi, Et.v32, K * B, (K + 1) * B, x, y, -1.f, t})) return;
            in = t;
        }
        if (!run(CoarseStep{Dt.rowptr, Dt.lo, Dt.hi, Dt.v32, K * B, K * B, in, nullptr, 1.f, x})) return;
    }
}

__global__ void coarse_prolong_multi_kernel(int64_t n, int m, const int32_t* __restrict__ part,
                                            const int32_t* __restrict__ pos, const float* __restrict__ Q,
                                            int kmax, const int32_t* __restrict__ coff,
                                            const float* __restrict__ y, float* __restrict__ z) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m;
    const int64_t g = (int64_t)blockIdx.x * rpb + threadIdx.x / m;
    if (g >= n) return;
    const int s = part[g];
    const int c0 = coff[s], ks = coff[s + 1] - c0;
    const float* qa = Q + (int64_t)pos[g] * kmax;
    float acc = 0.f;
    for (int jj = 0; jj < ks; ++jj) acc = fma(qa[jj], y[(int64_t)(c0 + jj) * m + c], acc);
    z[g * m + c] += acc;
}

inline unsigned grid_for(int64_t n, int m) {
    const int rpb = MT / m;
    int64_t b = (n + rpb - 1) / rpb;
    if (b > 4 * 152) b = 4 * 152;     // few partials: the final sum stays short
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

namespace ddg {

void multi_ensure(ddg_handle h, int m) {
    MultiWork& w = h->mw;
    if (w.m_alloc >= m) return;
    for (void* p : {(void*)w.R, (void*)w.P, (void*)w.Q, (void*)w.T, (void*)w.Fb, (void*)w.Ub,
                    (void*)w.r32, (void*)w.z32,
                    (void*)w.res32, (void*)w.c32, (void*)w.y32, (void*)w.t32, (void*)w.x32,
                    (void*)w.scal, (void*)w.partials, (void*)w.active, (void*)w.restart,
                    (void*)w.items, (void*)w.gpart, (void*)w.gtick})
        if (p) h->arena.release(p);
    const int64_t n = h->n;
    w.R = h->arena.alloc<double>(n * m);
    w.P = h->arena.alloc<double>(n * m);
    w.Q = h->arena.alloc<double>(n * m);
    w.T = h->arena.alloc<double>(n * m);
    w.Fb = h->arena.alloc<double>(n * m);
    w.Ub = h->arena.alloc<double>(n * m);
    w.r32 = h->arena.alloc<float>(n * m);
    w.z32 = h->arena.alloc<float>(n * m);
    w.res32 = h->arena.alloc<float>(h->sum_local * m);
    const int64_t n0p = h->use_coarse ? h->n0p : 1;
    w.c32 = h->arena.alloc<float>(n0p * m);
    w.y32 = h->arena.alloc<float>(n0p * m);
    w.t32 = h->arena.alloc<float>(n0p * m);
    w.x32 = h->arena.alloc<float>(n0p * m);
    for (float* p : {w.c32, w.y32, w.t32, w.x32})
        DDG_CUDA(cudaMemsetAsync(p, 0, n0p * m * sizeof(float), h->stream));
    if (h->use_coarse) {
        const int nsplit = (h->B + CG_KS - 1) / CG_KS;
        w.gpart = h->arena.alloc<float>((size_t)nsplit * h->B * m);
        w.gtick = h->arena.alloc<unsigned>(std::max(2, h->B / CG_ROWS));
        DDG_CUDA(cudaMemsetAsync(w.gtick, 0, std::max(2, h->B / CG_ROWS) * sizeof(unsigned), h->stream));
    }
    w.scal = h->arena.alloc<double>(S_COUNT * DDG_MCHUNK);
    w.partials = h->arena.alloc<double>((size_t)DDG_RED_BLOCKS * 2 * DDG_MCHUNK);
    w.active = h->arena.alloc<int>(DDG_MCHUNK);
    w.restart = h->arena.alloc<int>(DDG_MCHUNK);
    // work items of the multi-RHS local solve: one per (subdomain, tile row)
    std::vector<int2> it;
    w.h_citem_off.assign(h->ncol + 1, 0);
    std::vector<int> Tq(h->nsub);
    for (int q = 0; q < h->nsub; ++q) {
        const int nq = (int)(h->h_ov_off[q + 1] - h->h_ov_off[q]);
        Tq[q] = (nq + DDG_LT - 1) / DDG_LT;
    }
    for (int c = 0; c < h->ncol; ++c) {
        for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q)
            for (int I = 0; I < Tq[q]; ++I) it.push_back(make_int2(q, I));
        w.h_citem_off[c + 1] = (int)it.size();
    }
    w.items = h->arena.alloc<int2>(it.size());
    h2d(w.items, it.data(), it.size(), h->stream);
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    w.m_alloc = m;
}

// algorithmic bytes of one tensor-core local-solve launch: the BF16 inverse
// (n_i^2 * 2) plus the BF16 residual read and the FP32 z read + write
static double tc_bytes(ddg_handle h, int c, int m) {
    double b = 0.0;
    for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q) {
        const double nq = (double)(h->h_ov_off[q + 1] - h->h_ov_off[q]);
        b += nq * nq * 2.0 + nq * m * (2.0 + 8.0);
    }
    return b;
}

template <int SK>
static void multi_apply_t(ddg_handle h, int m) {
    MultiWork& w = h->mw;
    const int64_t n = h->n;
    const int prec = h->precision;
    to_float_n_kernel<<<(unsigned)((n * m + 255) / 256), 256, 0, h->stream>>>(n * m, w.R, w.r32);
    DDG_CUDA(cudaMemsetAsync(w.z32, 0, n * m * sizeof(float), h->stream));
    const bool tc = prec == DDG_PREC_BF16 && h->tc.A != nullptr;
    if (tc && h->tc.last_m != m) {
        // padding rows/columns of the BF16 residual slabs must read as zero
        DDG_CUDA(cudaMemsetAsync(h->tc.X, 0, h->tc.x_elems * sizeof(__nv_bfloat16), h->stream));
        h->tc.last_m = m;
    }
    auto local = [&](int c, bool zz) {
        if (tc) {
            {
                ProfScope ps(h, DDG_K_LOCAL_RESIDUAL, 1, 0.0);
                tc_residual(h, c, zz, m);
            }
            ProfScope ps(h, DDG_K_LOCAL_SOLVE, 1, tc_bytes(h, c, m));
            tc_local_solve(h, c, m);
            return;
        }
        const int64_t a0 = h->h_crow_off[c], a1 = h->h_crow_off[c + 1];
        ProfScope ps(h, DDG_K_LOCAL_SOLVE, 2, 0.0);
        if (a1 > a0) {
            const int bd = col_block(m), rpb = bd / m;
            local_residual_multi_kernel<SK><<<(unsigned)((a1 - a0 + rpb - 1) / rpb), bd, 0, h->stream>>>(
                a0, a1, m, h->ov_nodes, h->rowptr, h->col, h->val32, w.r32, w.z32, w.res32, zz, h->nx,
                h->ny, h->nz);
        }
        const int i0 = w.h_citem_off[c], i1 = w.h_citem_off[c + 1];
        if (i1 > i0) {
            if (prec == DDG_PREC_BF16 && h->inv16)
                local_solve_multi_kernel<__nv_bfloat16><<<i1 - i0, MT, 0, h->stream>>>(
                    w.items, i0, h->ov_off, h->ov_nodes, h->tile_off, h->Tq, h->inv16, w.res32, w.z32, m);
            else
                local_solve_multi_kernel<float><<<i1 - i0, MT, 0, h->stream>>>(
                    w.items, i0, h->ov_off, h->ov_nodes, h->tile_off, h->Tq, h->inv32, w.res32, w.z32, m);
        }
        DDG_CHECK_LAUNCH();
    };
    for (int c = 0; c < h->ncol; ++c) local(c, c == 0);
    if (h->use_coarse) {
        ProfScope ps(h, DDG_K_COARSE, 2 + 4 * h->nK - 2, 0.0);
        const int bd = col_block(m);
        const size_t smem = (size_t)(bd / m) * h->kmax * m * sizeof(float);
#define RESTRICT_MULTI(KM)                                                                              \
    coarse_restrict_multi_kernel<SK, KM><<<h->nsub, bd, smem, h->stream>>>(                             \
        h->sub_off, h->sub_nodes, h->rowptr, h->col, h->val32, w.r32, w.z32, h->Q32, h->kmax, h->coff, \
        w.c32, m, h->nx, h->ny, h->nz)
        if (h->kmax <= 8) RESTRICT_MULTI(8);
        else if (h->kmax <= 16) RESTRICT_MULTI(16);
        else RESTRICT_MULTI(32);
#undef RESTRICT_MULTI
        const int B = h->B, nK = h->nK;
        {
            // one cooperative launch for the whole recurrence
            static int max_blocks = 0;
            if (!max_blocks) {
                int per_sm = 0, dev = 0, sms = 0;
                DDG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_solve_persistent_kernel, MT, 0));
                DDG_CUDA(cudaGetDevice(&dev));
                DDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                max_blocks = std::max(1, std::min(per_sm, 4)) * sms;
            }
            ProfileMat Dm = h->Dm, Em = h->Em, Dt = h->Dt, Et = h->Et;
            int Bv = B, nKv = nK, mv = m;
            const float* cv = w.c32;
            float *yv = w.y32, *tv = w.t32, *xv = w.x32, *pv = w.gpart;
            ddgdev::GridBar* gbv = reinterpret_cast<ddgdev::GridBar*>(w.gtick);
            int* ev = h->errflags + E_TIMEOUT;
            void* args[] = {&Dm, &Em, &Dt, &Et, &Bv, &nKv, &mv, &cv, &yv, &tv, &xv, &pv, &gbv, &ev};
            DDG_CUDA(cudaLaunchCooperativeKernel((const void*)coarse_solve_persistent_kernel, dim3(max_blocks),
                                                 dim3(MT), args, 0, h->stream));
        }
        coarse_prolong_multi_kernel<<<(unsigned)((n + bd / m - 1) / (bd / m)), bd, 0, h->stream>>>(
            n, m, h->part, h->pos, h->Q32, h->kmax, h->coff, w.x32, w.z32);
        DDG_CHECK_LAUNCH();
    }
    for (int c = h->ncol - 1; c >= 0; --c) local(c, false);
}

void multi_apply(ddg_handle h, int m) {
#define MA_CALL(SK) multi_apply_t<SK>(h, m)
    DDG_DISPATCH_SK(h, MA_CALL);
#undef MA_CALL
}

void multi_spmv_pq(ddg_handle h, int m) {
    MultiWork& w = h->mw;
    const unsigned G = grid_for(h->n, m);
    const int bd = col_block(m);
#define MS_CALL(SK)                                                                                       \
    spmv_multi_kernel<SK><<<G, bd, 0, h->stream>>>(h->n, m, h->rowptr, h->col, h->val64, w.P, w.Q, h->nx, \
                                                   h->ny, h->nz, w.partials, h->red_counter, w.scal, w.active)
    DDG_DISPATCH_SK(h, MS_CALL);
#undef MS_CALL
    DDG_CHECK_LAUNCH();
}

void multi_update_ur(ddg_handle h, int m, double* U) {
    MultiWork& w = h->mw;
    update_ur_multi_kernel<<<grid_for(h->n, m), col_block(m), 0, h->stream>>>(h->n, m, U, w.R, w.P, w.Q, w.partials, h->red_counter, w.scal);
    DDG_CHECK_LAUNCH();
}

void multi_dots(ddg_handle h, int m, int pr) {
    MultiWork& w = h->mw;
    dots_multi_kernel<float><<<grid_for(h->n, m), col_block(m), 0, h->stream>>>(h->n, m, w.R, w.Q, w.z32, pr, w.partials, h->red_counter, w.scal, w.active, w.restart);
    DDG_CHECK_LAUNCH();
}

void multi_update_p(ddg_handle h, int m) {
    MultiWork& w = h->mw;
    const int bd = col_block(m), rpb = bd / m;
    update_p_multi_kernel<float><<<(unsigned)((h->n + rpb - 1) / rpb), bd, 0, h->stream>>>(h->n, m, w.P, w.z32, w.scal, w.active);
    DDG_CHECK_LAUNCH();
}

// slot <- per-column ||a - A b||^2 (b may be null); out (may be null) <- a - A b
void multi_resnorm(ddg_handle h, int m, const double* a, const double* b, double* out, int slot) {
    MultiWork& w = h->mw;
    const unsigned G = grid_for(h->n, m);
    const int bd = col_block(m);
#define MR_CALL(SK)                                                                                        \
    resnorm_multi_kernel<SK><<<G, bd, 0, h->stream>>>(h->n, m, h->rowptr, h->col, h->val64, a, b, out, h->nx, \
                                                      h->ny, h->nz, w.partials, h->red_counter, w.scal, slot)
    DDG_DISPATCH_SK(h, MR_CALL);
#undef MR_CALL
    DDG_CHECK_LAUNCH();
}

void copy_cols(ddg_handle h, const double* src, int ms, int j0, double* dst, int md, int k0, int cnt) {
    copy_cols_kernel<<<(unsigned)((h->n * cnt + 255) / 256), 256, 0, h->stream>>>(h->n, src, ms, j0, dst, md, k0, cnt);
    DDG_CHECK_LAUNCH();
}

void multi_replace_cols(ddg_handle h, int m, const double* src, double* dst, const int* replace) {
    const int bd = col_block(m), rpb = bd / m;
    replace_cols_kernel<<<(unsigned)((h->n + rpb - 1) / rpb), bd, 0, h->stream>>>(h->n, m, src, dst, replace);
    DDG_CHECK_LAUNCH();
}

}  // namespace ddg
