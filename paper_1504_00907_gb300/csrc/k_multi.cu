// Many right-hand sides at once (m <= DDG_MCHUNK per group): the same PCG and
// the same preconditioner (Sec. 6, Sec. 7) on an n x m block stored dof-major
// (entry (g, j) at g * m + j), with per-column CG scalars, convergence masks
// and restarts.  Every stage is a multi-column version of the single-RHS
// kernel: the preconditioner reads each local inverse once per colour phase
// for all m columns, which is what makes batching pay.
#include <cstring>

#include "ddg_internal.cuh"
#include <algorithm>

#include "dev_common.cuh"

namespace {

constexpr int MT = 256;

// threads of the column-mapped kernels: a multiple of m, at most 256
inline int col_block(int m) { return (MT / m) * m; }

// rows per round of the grid-stride reduction kernels (loads issued together)
constexpr int UNR = 4;

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

// A z at dof g for the 4 columns c4..c4+3 (m % 4 == 0: one 16-byte word of
// each z row); the row's CSR entries are shared by the 4 columns
template <int SK>
__device__ __forceinline__ float4 apply_row4(int g, int c4, int m, const int64_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ col, const float* __restrict__ val,
                                             const float* __restrict__ z, int nx, int ny, int nz) {
    auto ld = [&](int gg) { return *reinterpret_cast<const float4*>(z + (int64_t)gg * m + c4); };
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    auto fma4 = [&](float a, const float4& b) {
        s.x = fma(a, b.x, s.x);
        s.y = fma(a, b.y, s.y);
        s.z = fma(a, b.z, s.z);
        s.w = fma(a, b.w, s.w);
    };
    if (SK == DDG_STENCIL_7PT_3D || SK == DDG_STENCIL_5PT_2D) {
        const int i = g % nx, j = (g / nx) % ny;
        fma4(SK == DDG_STENCIL_7PT_3D ? 6.f : 4.f, ld(g));
        if (i > 0) fma4(-1.f, ld(g - 1));
        if (i < nx - 1) fma4(-1.f, ld(g + 1));
        if (j > 0) fma4(-1.f, ld(g - nx));
        if (j < ny - 1) fma4(-1.f, ld(g + nx));
        if (SK == DDG_STENCIL_7PT_3D) {
            const int k = g / (nx * ny);
            if (k > 0) fma4(-1.f, ld(g - nx * ny));
            if (k < nz - 1) fma4(-1.f, ld(g + nx * ny));
        }
        return s;
    }
    if (SK == ddgdev::SK_CSR8 || SK == ddgdev::SK_CSR16) {
        constexpr int NMAX = SK == ddgdev::SK_CSR8 ? 8 : 16;
        const int64_t e0 = rowptr[g];
        const int cnt = (int)(rowptr[g + 1] - e0);
        int cl[NMAX];
        float vl[NMAX];
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            cl[i] = i < cnt ? col[e0 + i] : 0;
            vl[i] = i < cnt ? val[e0 + i] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
            if (i < cnt) fma4(vl[i], ld(cl[i]));
        return s;
    }
    for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) fma4(val[e], ld(col[e]));
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

// also writes R32 = (float)R, the preconditioner's input
__global__ void __launch_bounds__(MT) update_ur_multi_kernel(int64_t n, int m, double* __restrict__ U,
                                                             double* __restrict__ R,
                                                             const double* __restrict__ P,
                                                             const double* __restrict__ Q,
                                                             float* __restrict__ R32,
                                                             double* partials, unsigned* counter,
                                                             double* sc) {
    const int rpb = blockDim.x / m;
    const int c = threadIdx.x % m, rl = threadIdx.x / m;
    const double alpha = S(sc, S_ALPHA, c);
    double acc[1] = {0.0};
    if ((int)threadIdx.x < rpb * m) {
        // UNR rows per round: all loads of the round before its arithmetic,
        // the norm still accumulated row after row
        const int64_t stride = (int64_t)gridDim.x * rpb;
        for (int64_t g0 = (int64_t)blockIdx.x * rpb + rl; g0 < n; g0 += UNR * stride) {
            double pv[UNR], qv[UNR], rv[UNR], uv[UNR];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int64_t g = g0 + k * stride;
                if (g < n) {
                    const int64_t e = g * m + c;
                    pv[k] = P[e];
                    qv[k] = Q[e];
                    rv[k] = R[e];
                    uv[k] = U[e];
                }
            }
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int64_t g = g0 + k * stride;
                if (g < n) {
                    const int64_t e = g * m + c;
                    U[e] = fma(alpha, pv[k], uv[k]);
                    const double r = fma(-alpha, qv[k], rv[k]);
                    R[e] = r;
                    R32[e] = (float)r;
                    acc[0] = fma(r, r, acc[0]);
                }
            }
        }
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
    if ((int)threadIdx.x < rpb * m) {
        const int64_t stride = (int64_t)gridDim.x * rpb;
        for (int64_t g0 = (int64_t)blockIdx.x * rpb + rl; g0 < n; g0 += UNR * stride) {
            double rv[UNR], qv[UNR], zv[UNR];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int64_t g = g0 + k * stride;
                if (g < n) {
                    const int64_t e = g * m + c;
                    zv[k] = (double)Z[e];
                    rv[k] = R[e];
                    qv[k] = Q[e];
                }
            }
#pragma unroll
            for (int k = 0; k < UNR; ++k)
                if (g0 + k * stride < n) {
                    acc[0] = fma(rv[k], zv[k], acc[0]);
                    acc[1] = fma(qv[k], zv[k], acc[1]);
                }
        }
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
                                                           int slot, const int* gate) {
    if (gate && !*gate) return;
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
                                    const int* __restrict__ replace, const int* gate) {
    if (gate && !*gate) return;
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

__global__ void to_float_n_kernel(int64_t cnt, const double* __restrict__ a, float* __restrict__ b,
                                  const int* gate = nullptr) {
    if (gate && !*gate) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < cnt) b[g] = (float)a[g];
}

// ---- control of the graph-driven batched PCG: one block of DDG_MCHUNK
// threads, thread c for column c (the host loop's per-column decisions)
__global__ void mloop_init_kernel(int m, MultiCtl* ctl, const double* sc, int* active, int* restart,
                                  cudaGraphConditionalHandle cond) {
    const int c = threadIdx.x;
    bool act = false;
    if (c < m) {
        const double fn = sqrt(S(const_cast<double*>(sc), S_TMP, c));
        act = fn > 0.0;
        ctl->fn[c] = fn;
        ctl->done_it[c] = act ? -1 : 0;
        ctl->done_rel[c] = act ? -1.0 : 0.0;
        ctl->cstat[c] = DDG_OK;
        ctl->nrest[c] = 0;
        ctl->cand[c] = 0;
    }
    active[c] = act ? 1 : 0;
    restart[c] = 1;
    const int any = __syncthreads_or(act);
    if (c == 0) {
        ctl->it = 0;
        ctl->any_cand = 0;
        ctl->any_restart = 0;
        ctl->any_unfinished = 0;
        ctl->timed_out = 0;
        cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
}

// after the u/r update: breakdown, or the recurrence residual at or below tol
// makes the column a candidate for the true-residual check
__global__ void mloop_decide_recurrence_kernel(int m, MultiCtl* ctl, double* sc, int* active, int* restart) {
    const int c = threadIdx.x;
    const int it = ctl->it + 1;
    restart[c] = 0;   // the dots of this iteration have used it
    bool cand = false;
    if (c < m && active[c]) {
        if (S(sc, S_FLAG, c) != 0.0) {
            ctl->cstat[c] = DDG_EBREAKDOWN;
            active[c] = 0;
            ctl->done_it[c] = it;
        } else if (sqrt(S(sc, S_RR, c)) / ctl->fn[c] <= ctl->tol) {
            cand = true;
        }
    }
    if (c < m) ctl->cand[c] = cand ? 1 : 0;
    const int any = __syncthreads_or(cand);
    if (c == 0) {
        ctl->it = it;
        ctl->any_cand = any;
        ctl->any_restart = 0;
    }
}

// after the true residuals of the candidates: accept, give up after the last
// restart, or restart the column from its true residual; loop condition
__global__ void mloop_decide_true_kernel(int m, MultiCtl* ctl, const double* sc, int* active, int* restart,
                                         const int* errflag, cudaGraphConditionalHandle cond) {
    const int c = threadIdx.x;
    const int it = ctl->it;
    bool rs = false;
    if (c < m && ctl->cand[c]) {
        const double trel = sqrt(S(const_cast<double*>(sc), S_TMP, c)) / ctl->fn[c];
        if (trel <= ctl->tol || ctl->nrest[c] >= DDG_MAX_RESTARTS) {
            active[c] = 0;
            ctl->done_it[c] = it;
            ctl->done_rel[c] = trel;
            ctl->cstat[c] = trel <= ctl->tol ? DDG_OK : DDG_ENOCONV;
        } else {
            restart[c] = 1;
            ctl->nrest[c] += 1;
            rs = true;
        }
        ctl->cand[c] = 0;
    }
    const int anyr = __syncthreads_or(rs);
    const int anya = __syncthreads_or(c < m && active[c]);
    if (c == 0) {
        const int to = *errflag != 0;
        ctl->any_restart = anyr;
        ctl->timed_out = to;
        cudaGraphSetConditional(cond, (anya && it < ctl->maxit && !to) ? 1u : 0u);
    }
}

__global__ void mloop_final_prep_kernel(int m, MultiCtl* ctl) {
    const int c = threadIdx.x;
    const int any = __syncthreads_or(c < m && ctl->done_rel[c] < 0.0);
    if (c == 0) ctl->any_unfinished = any;
}

// columns still running at the end (maxit, or a timeout) or broken down:
// their true residual, and ENOCONV for the ones that never finished
__global__ void mloop_final_kernel(int m, MultiCtl* ctl, const double* sc) {
    const int c = threadIdx.x;
    if (c >= m || !(ctl->done_rel[c] < 0.0)) return;
    ctl->done_rel[c] = sqrt(S(const_cast<double*>(sc), S_TMP, c)) / ctl->fn[c];
    if (ctl->done_it[c] < 0) {
        ctl->done_it[c] = ctl->it;
        ctl->cstat[c] = DDG_ENOCONV;
    }
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
    const E* sub = inv + tile_off[q];
    const int wp = ddgdev::packed_narrow_width(n, T);
    for (int J = 0; J < T; ++J) {
        const bool upper = J >= I;
        const int a = upper ? I : J, b = upper ? J : I;
        const E* tp = sub + ddgdev::packed_tile_start(a, b, T, wp);
        const int ld = b == T - 1 ? wp : DDG_LT;   // stored columns of tile (a, b)
        const bool trap = a == b && a < T - 1;     // upper trapezoid diagonal tile
        for (int e = threadIdx.x; e < 1024; e += MT) {
            const int rr = e >> 5, kk = e & 31;
            float v;
            if (trap) {
                // (rr, kk) left of its row's 8-column block is the mirror (kk, rr)
                v = kk >= 8 * (rr >> 3) ? (float)tp[ddgdev::packed_diag_offset(rr, kk)]
                                        : (float)tp[ddgdev::packed_diag_offset(kk, rr)];
            } else {
                v = kk < ld ? (float)tp[rr * ld + kk] : 0.f;
            }
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

// c = R0 (r - A z) for m % 4 == 0 and kmax <= 32: a CTA of RS_T threads per
// subdomain walks its rows in chunks of RS_ROWS.  The chunk's rows of
// w = r - A z (m/4 threads per row, four columns each, up to four rows in
// flight per thread) and its rows of Q go to shared memory; then every
// thread adds, over the chunk's rows in order, the products for its
// (generator, 4-column) outputs (at most 2 per thread).
constexpr int RS_T = 256, RS_ROWS = 64;
template <int SK>
__global__ void __launch_bounds__(RS_T) coarse_restrict_stage4_kernel(
    const int64_t* __restrict__ sub_off, const int32_t* __restrict__ sub_nodes,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
    const float* __restrict__ r, const float* __restrict__ z, const float* __restrict__ Q, int kmax,
    const int32_t* __restrict__ coff, float* __restrict__ cvec, int m, int nx, int ny, int nz) {
    __shared__ __align__(16) float sw[RS_ROWS * DDG_MCHUNK];
    __shared__ float sq[RS_ROWS * 32];
    const int s = blockIdx.x, tid = threadIdx.x;
    const int q4 = m >> 2, slots = RS_T / q4;
    const int cq = tid % q4, rs = tid / q4;
    const int nout = kmax * q4;
    float4 acc[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    const int64_t b0 = sub_off[s], b1 = sub_off[s + 1];
    for (int64_t a0 = b0; a0 < b1; a0 += RS_ROWS) {
        const int rows = (int)min((int64_t)RS_ROWS, b1 - a0);
        if (rs < slots)
            for (int i0 = rs; i0 < RS_ROWS; i0 += 4 * slots) {
                float4 wv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * slots;
                    if (i < rows) {
                        const int g = sub_nodes[a0 + i];
                        const float4 rv = *reinterpret_cast<const float4*>(r + (int64_t)g * m + 4 * cq);
                        const float4 az = apply_row4<SK>(g, 4 * cq, m, rowptr, col, val, z, nx, ny, nz);
                        wv[u] = make_float4(rv.x - az.x, rv.y - az.y, rv.z - az.z, rv.w - az.w);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * slots;
                    if (i < rows) *reinterpret_cast<float4*>(sw + i * m + 4 * cq) = wv[u];
                }
            }
        for (int e = tid; e < rows * kmax; e += RS_T) sq[e] = Q[a0 * kmax + e];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int o = tid + u * RS_T;
            if (o < nout) {
                const int j = o / q4, c4 = o - j * q4;
                float4 t = acc[u];
                for (int i = 0; i < rows; ++i) {
                    const float qv = sq[i * kmax + j];
                    const float4 wv = *reinterpret_cast<const float4*>(sw + i * m + 4 * c4);
                    t.x = fma(qv, wv.x, t.x);
                    t.y = fma(qv, wv.y, t.y);
                    t.z = fma(qv, wv.z, t.z);
                    t.w = fma(qv, wv.w, t.w);
                }
                acc[u] = t;
            }
        }
        __syncthreads();
    }
    const int ks = coff[s + 1] - coff[s];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int o = tid + u * RS_T;
        if (o < nout) {
            const int j = o / q4, c4 = o - j * q4;
            if (j < ks) *reinterpret_cast<float4*>(cvec + (int64_t)(coff[s] + j) * m + 4 * c4) = acc[u];
        }
    }
}

// z[g, c4..c4+3] += sum_j Q[pos g, j] y[coff_{part g} + j, c4..c4+3]  (m % 4 == 0)
__global__ void coarse_prolong_multi4_kernel(int64_t n, int m, const int32_t* __restrict__ part,
                                             const int32_t* __restrict__ pos, const float* __restrict__ Q,
                                             int kmax, const int32_t* __restrict__ coff,
                                             const float* __restrict__ y, float* __restrict__ z) {
    const int q4 = m >> 2;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * q4) return;
    const int64_t g = e / q4;
    const int c4 = 4 * (int)(e - g * q4);
    const int sb = part[g];
    const int c0 = coff[sb], ks = coff[sb + 1] - c0;
    const float* qa = Q + (int64_t)pos[g] * kmax;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int jj = 0; jj < ks; ++jj) {
        const float qv = qa[jj];
        const float4 yv = *reinterpret_cast<const float4*>(y + (int64_t)(c0 + jj) * m + c4);
        acc.x = fma(qv, yv.x, acc.x);
        acc.y = fma(qv, yv.y, acc.y);
        acc.z = fma(qv, yv.z, acc.z);
        acc.w = fma(qv, yv.w, acc.w);
    }
    float4* zp = reinterpret_cast<float4*>(z + g * m + c4);
    float4 zv = *zp;
    zv.x += acc.x;
    zv.y += acc.y;
    zv.z += acc.z;
    zv.w += acc.w;
    *zp = zv;
}

// ---------------------------------------------------------------- batched coarse solve
// Each GEMM of the block-bidiagonal recurrence, out[r0 + i] = a + sign * M x
// for m columns, is one launch of (32-row tile, 128-column split) CTAs; the
// CTA that finishes a row tile last sums its splits' partial products in a
// fixed order.  Steps are chained by programmatic dependent launch: a CTA
// stages its block of M (which no earlier step writes) in shared memory, and
// only then waits for the previous step before it reads x and a.
struct CoarseStep {            // one GEMM of the recurrence (cbase < 0: block-diagonal)
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

constexpr int CG_LOADS = 16;   // split partials loaded together by the reducing CTA
constexpr int CG_T = 128;      // threads of a step CTA: a 4-row x 4-column block each
constexpr int CG_B = 8;        // loads in flight per thread while staging
constexpr int CG_MT = CG_ROWS + 4;   // row stride of the transposed M block (16-byte rows)

// x rows of the split are staged with a row stride mp = m rounded up to 4
// (zero columns past m) so that every thread reads its 4 columns as one
// 16-byte word; M is staged transposed so that its 4 rows are one word too.
__global__ void __launch_bounds__(CG_T) coarse_step_multi_kernel(CoarseStep S, int B, int m, int nsplit,
                                                                 float* __restrict__ part,
                                                                 unsigned* __restrict__ tickets) {
    extern __shared__ __align__(16) float smx[];      // [CG_KS][mp]
    __shared__ __align__(16) float sMt[CG_KS][CG_MT];
    __shared__ int rlo[CG_ROWS], rhi[CG_ROWS];
    __shared__ int64_t rptr[CG_ROWS];
    __shared__ int span[2];
    __shared__ int am_last;
    const int rt = blockIdx.x / nsplit, sp = blockIdx.x % nsplit;
    const int R = (gridDim.x / nsplit) * CG_ROWS;   // rows of the launch: split stride of part
    const int row0 = S.r0 + rt * CG_ROWS;
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;   // rows 4ty..4ty+3, columns 4tx..4tx+3
    const int mp = (m + 3) & ~3;
    if (t < CG_ROWS) {
        rlo[t] = S.lo[row0 + t];
        rhi[t] = S.hi[row0 + t];
        rptr[t] = S.rowptr[row0 + t];
    }
    __syncthreads();
    if (t == 0) {
        int ulo = INT32_MAX, uhi = INT32_MIN;
        for (int q = 0; q < CG_ROWS; ++q)
            if (rhi[q] > rlo[q]) {
                ulo = min(ulo, rlo[q]);
                uhi = max(uhi, rhi[q]);
            }
        span[0] = ulo;
        span[1] = uhi;
    }
    __syncthreads();
    // the columns of this split that some row of the tile reaches
    const int cb = S.cbase >= 0 ? S.cbase : (row0 / B) * B;   // block-diagonal: own super-block
    const int c_lo = cb + sp * CG_KS;
    const int ulo = max(span[0], c_lo), uhi = min(span[1], c_lo + CG_KS);
    const bool work = uhi > ulo;
    const int jb = ulo - c_lo, je = uhi - c_lo;   // local column range [jb, je)
    // staging loops issue CG_B loads before their first shared-memory store,
    // so a thread waits about one memory latency per CG_B elements
    if (work) {
        for (int e0 = t; e0 < CG_ROWS * CG_KS; e0 += CG_B * CG_T) {
            float v[CG_B];
#pragma unroll
            for (int i = 0; i < CG_B; ++i) {
                const int e = e0 + i * CG_T, rr = e / CG_KS, jj = e % CG_KS, j = c_lo + jj;
                v[i] = (e < CG_ROWS * CG_KS && jj >= jb && jj < je && j >= rlo[rr] && j < rhi[rr])
                           ? S.vals[rptr[rr] + (j - rlo[rr])] : 0.f;
            }
#pragma unroll
            for (int i = 0; i < CG_B; ++i) {
                const int e = e0 + i * CG_T, rr = e / CG_KS, jj = e % CG_KS;
                if (e < CG_ROWS * CG_KS && jj >= jb && jj < je) sMt[jj][rr] = v[i];
            }
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (work) {
        if (mp == m) {
            // whole rows: (je - jb) * m contiguous floats, 16-byte words
            const float4* src = reinterpret_cast<const float4*>(S.x + (int64_t)(c_lo + jb) * m);
            float4* dst = reinterpret_cast<float4*>(smx + jb * m);
            const int n4 = (je - jb) * (m >> 2);
            for (int e0 = t; e0 < n4; e0 += CG_B * CG_T) {
                float4 v[CG_B];
#pragma unroll
                for (int i = 0; i < CG_B; ++i)
                    if (e0 + i * CG_T < n4) v[i] = src[e0 + i * CG_T];
#pragma unroll
                for (int i = 0; i < CG_B; ++i)
                    if (e0 + i * CG_T < n4) dst[e0 + i * CG_T] = v[i];
            }
        } else {
            const int ne = (je - jb) * mp;
            for (int e0 = t; e0 < ne; e0 += CG_B * CG_T) {
                float v[CG_B];
#pragma unroll
                for (int i = 0; i < CG_B; ++i) {
                    const int e = e0 + i * CG_T, jj = jb + e / mp, c = e % mp;
                    v[i] = (e < ne && c < m) ? S.x[(int64_t)(c_lo + jj) * m + c] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < CG_B; ++i) {
                    const int e = e0 + i * CG_T;
                    if (e < ne) smx[jb * mp + e] = v[i];
                }
            }
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
        if (4 * tx < mp) {
#pragma unroll 4
            for (int jj = jb; jj < je; ++jj) {
                const float4 mv = *reinterpret_cast<const float4*>(&sMt[jj][4 * ty]);
                const float4 xv = *reinterpret_cast<const float4*>(&smx[jj * mp + 4 * tx]);
                const float mr[4] = {mv.x, mv.y, mv.z, mv.w};
                const float xc[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[i][k] = fma(mr[i], xc[k], acc[i][k]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = 4 * tx + k;
                if (c < m) part[((size_t)sp * R + rt * CG_ROWS + 4 * ty + i) * m + c] = acc[i][k];
            }
    }
    __threadfence();
    __syncthreads();
    if (t == 0) am_last = atomicAdd(&tickets[rt], 1u) == (unsigned)nsplit - 1u;
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // splits that reach no column of the tile wrote nothing and add nothing;
    // the others are loaded together and summed in split order
    const int sp0 = span[1] > span[0] ? max((span[0] - cb) / CG_KS, 0) : 0;
    const int sp1 = span[1] > span[0] ? min((span[1] - 1 - cb) / CG_KS, nsplit - 1) : -1;
    if (mp == m) {
        // 16-byte words: 4 outputs per load
        const int n4 = CG_ROWS * (m >> 2);
        const float4* p4 = reinterpret_cast<const float4*>(part + (size_t)rt * CG_ROWS * m);
        const size_t st4 = (size_t)R * m / 4;
        for (int e = t; e < n4; e += CG_T) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int q0 = sp0; q0 <= sp1; q0 += CG_LOADS) {
                float4 v[CG_LOADS];
#pragma unroll
                for (int i = 0; i < CG_LOADS; ++i)
                    if (q0 + i <= sp1) v[i] = __ldcg(p4 + (size_t)(q0 + i) * st4 + e);
#pragma unroll
                for (int i = 0; i < CG_LOADS; ++i)
                    if (q0 + i <= sp1) {
                        s.x += v[i].x;
                        s.y += v[i].y;
                        s.z += v[i].z;
                        s.w += v[i].w;
                    }
            }
            const int64_t o = (int64_t)row0 * m + 4 * e;
            float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (S.a) a4 = *reinterpret_cast<const float4*>(S.a + o);
            *reinterpret_cast<float4*>(S.out + o) =
                make_float4(a4.x + S.sign * s.x, a4.y + S.sign * s.y, a4.z + S.sign * s.z, a4.w + S.sign * s.w);
        }
        if (t == 0) tickets[rt] = 0u;
        return;
    }
    for (int e = t; e < CG_ROWS * m; e += CG_T) {
        float s = 0.f;
        for (int q0 = sp0; q0 <= sp1; q0 += CG_LOADS) {
            float v[CG_LOADS];
#pragma unroll
            for (int i = 0; i < CG_LOADS; ++i)
                v[i] = q0 + i <= sp1 ? __ldcg(part + ((size_t)(q0 + i) * R + rt * CG_ROWS) * m + e) : 0.f;
#pragma unroll
            for (int i = 0; i < CG_LOADS; ++i)
                if (q0 + i <= sp1) s += v[i];
        }
        const int64_t o = (int64_t)row0 * m + e;
        S.out[o] = (S.a ? S.a[o] : 0.f) + S.sign * s;
    }
    if (t == 0) tickets[rt] = 0u;
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
                    (void*)w.res32, (void*)w.c32, (void*)w.y32, (void*)w.x32,
                    (void*)w.scal, (void*)w.partials, (void*)w.active, (void*)w.restart,
                    (void*)w.items, (void*)w.gpart, (void*)w.gtick, (void*)w.ndw, (void*)w.ndx, (void*)w.ndp})
        if (p) h->arena.release(p);
    w.ndw = w.ndx = w.ndp = nullptr;
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
    w.x32 = h->arena.alloc<float>(n0p * m);
    for (float* p : {w.c32, w.y32, w.x32})
        DDG_CUDA(cudaMemsetAsync(p, 0, n0p * m * sizeof(float), h->stream));
    if (h->use_coarse && h->nd.on) {
        w.ndw = h->arena.alloc<float>((size_t)h->n0 * m);
        w.ndx = h->arena.alloc<float>((size_t)h->n0 * m);
        w.ndp = h->arena.alloc<float>((size_t)std::max<int64_t>(1, h->nd.urows) * m);
    } else if (h->use_coarse) {
        const int nsplit = (h->B + CG_KS - 1) / CG_KS;
        // a step covers at most all n0p rows (the block-diagonal D launches)
        w.gpart = h->arena.alloc<float>((size_t)nsplit * h->n0p * m);
        // one ticket per 32-row tile of a step; reset by the CTA that uses it last
        w.gtick = h->arena.alloc<unsigned>(h->n0p / CG_ROWS);
        DDG_CUDA(cudaMemsetAsync(w.gtick, 0, (h->n0p / CG_ROWS) * sizeof(unsigned), h->stream));
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
    if (!w.ctl) {
        w.ctl = h->arena.alloc<MultiCtl>(1);
        DDG_CUDA(cudaMallocHost((void**)&w.h_ctl, sizeof(MultiCtl)));
        std::memset(w.h_ctl, 0, sizeof(MultiCtl));
    }
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    w.m_alloc = m;
    ++w.gen;
}

// algorithmic bytes of one tensor-core local-solve launch: the BF16 inverse
// (n_i^2 * 2) plus the BF16 residual read and the FP32 z read + write
static double tc_bytes(ddg_handle h, int c, int m) {
    double b = 0.0;
    for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q) {
        const double nq = (double)(h->h_ov_off[q + 1] - h->h_ov_off[q]);
        // inverse elements and residual slab entries at the operand width, z read and written in FP32
        const double ew = h->tc.kind == DDG_TC_TF32 ? 4.0 : 2.0;
        b += nq * nq * ew + nq * m * (ew + 8.0);
    }
    return b;
}

template <int SK>
static void multi_apply_t(ddg_handle h, int m) {
    MultiWork& w = h->mw;
    const int64_t n = h->n;
    const int prec = h->precision;
    if (!w.r32_current)
        to_float_n_kernel<<<(unsigned)((n * m + 255) / 256), 256, 0, h->stream>>>(n * m, w.R, w.r32);
    DDG_CUDA(cudaMemsetAsync(w.z32, 0, n * m * sizeof(float), h->stream));
    const bool tc = prec == h->tc.prec();
    if (tc && h->tc.last_m != m) {
        // padding rows/columns of the residual slabs must read as zero
        DDG_CUDA(cudaMemsetAsync(h->tc.x_ptr(), 0, h->tc.x_bytes(), h->stream));
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
        ProfScope ps(h, DDG_K_COARSE, 2 + (h->nd.on ? nd_solve_multi_launches(h) : 2 * h->nK), 0.0);
        const int bd = col_block(m);
        const size_t smem = (size_t)(bd / m) * h->kmax * m * sizeof(float);
#define RESTRICT_MULTI(KM)                                                                              \
    coarse_restrict_multi_kernel<SK, KM><<<h->nsub, bd, smem, h->stream>>>(                             \
        h->sub_off, h->sub_nodes, h->rowptr, h->col, h->val32, w.r32, w.z32, h->Q32, h->kmax, h->coff, \
        w.c32, m, h->nx, h->ny, h->nz)
        const bool vec4 = m % 4 == 0;
        if (vec4)
            coarse_restrict_stage4_kernel<SK><<<h->nsub, RS_T, 0, h->stream>>>(
                h->sub_off, h->sub_nodes, h->rowptr, h->col, h->val32, w.r32, w.z32, h->Q32, h->kmax, h->coff,
                w.c32, m, h->nx, h->ny, h->nz);
        else if (h->kmax <= 8) RESTRICT_MULTI(8);
        else if (h->kmax <= 16) RESTRICT_MULTI(16);
        else RESTRICT_MULTI(32);
#undef RESTRICT_MULTI
        const int B = h->B, nK = h->nK;
        const int nsplit = (B + CG_KS - 1) / CG_KS;
        if (h->nd.on) {
            nd_coarse_solve_multi(h, m, w.c32, w.y32, w.x32, w.ndw, w.ndx, w.ndp);
        } else {
        // rows [r0, r0 + rows); cbase < 0: each row's own super-block
        auto step = [&](const ProfileMat& M, int r0, int rows, int cbase, const float* x, const float* a,
                        float sign, float* out) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)((rows / CG_ROWS) * nsplit));
            cfg.blockDim = dim3(CG_T);
            cfg.dynamicSmemBytes = (size_t)CG_KS * ((m + 3) & ~3) * sizeof(float);
            cfg.stream = h->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = h->use_pdl ? 1 : 0;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            static PerDeviceMax configured;   // the attribute is per device
            const int smax = (int)(CG_KS * DDG_MCHUNK * sizeof(float));
            int dev = -1;
            if (configured.needs(smax, dev)) {
                DDG_CUDA(cudaFuncSetAttribute(coarse_step_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smax));
                configured.commit(dev, smax);
            }
            const CoarseStep S{M.rowptr, M.lo, M.hi, M.v32, r0, cbase, x, a, sign, out};
            DDG_CUDA(cudaLaunchKernelEx(&cfg, coarse_step_multi_kernel, S, B, m, nsplit, w.gpart, w.gtick));
        };
        // y = D c (all super-blocks), y_K -= F_K y_{K-1}; x = D^T y, x_K -= G_K x_{K+1}
        const int n0p = h->n0p;
        step(h->Dm, 0, n0p, -1, w.c32, nullptr, 1.f, w.y32);
        for (int K = 1; K < nK; ++K) step(h->Fm, K * B, B, (K - 1) * B, w.y32, w.y32, -1.f, w.y32);
        step(h->Dt, 0, n0p, -1, w.y32, nullptr, 1.f, w.x32);
        for (int K = nK - 2; K >= 0; --K) step(h->Gm, K * B, B, (K + 1) * B, w.x32, w.x32, -1.f, w.x32);
        }
        if (vec4)
            coarse_prolong_multi4_kernel<<<(unsigned)((n * (m / 4) + 255) / 256), 256, 0, h->stream>>>(
                n, m, h->part, h->pos, h->Q32, h->kmax, h->coff, w.x32, w.z32);
        else
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
    update_ur_multi_kernel<<<grid_for(h->n, m), col_block(m), 0, h->stream>>>(h->n, m, U, w.R, w.P, w.Q, w.r32, w.partials, h->red_counter, w.scal);
    DDG_CHECK_LAUNCH();
    w.r32_current = true;
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
void multi_resnorm_gated(ddg_handle h, int m, const double* a, const double* b, double* out, int slot,
                         const int* gate) {
    MultiWork& w = h->mw;
    const unsigned G = grid_for(h->n, m);
    const int bd = col_block(m);
#define MR_CALL(SK)                                                                                        \
    resnorm_multi_kernel<SK><<<G, bd, 0, h->stream>>>(h->n, m, h->rowptr, h->col, h->val64, a, b, out, h->nx, \
                                                      h->ny, h->nz, w.partials, h->red_counter, w.scal, slot, \
                                                      gate)
    DDG_DISPATCH_SK(h, MR_CALL);
#undef MR_CALL
    DDG_CHECK_LAUNCH();
}

void multi_resnorm(ddg_handle h, int m, const double* a, const double* b, double* out, int slot) {
    multi_resnorm_gated(h, m, a, b, out, slot, nullptr);
}

void multi_to_float(ddg_handle h, int m, const int* gate) {
    MultiWork& w = h->mw;
    to_float_n_kernel<<<(unsigned)((h->n * m + 255) / 256), 256, 0, h->stream>>>(h->n * m, w.R, w.r32, gate);
    DDG_CHECK_LAUNCH();
}

void mloop_init(ddg_handle h, int m, cudaGraphConditionalHandle cond) {
    mloop_init_kernel<<<1, DDG_MCHUNK, 0, h->stream>>>(m, h->mw.ctl, h->mw.scal, h->mw.active, h->mw.restart, cond);
    DDG_CHECK_LAUNCH();
}

void mloop_decide_recurrence(ddg_handle h, int m) {
    mloop_decide_recurrence_kernel<<<1, DDG_MCHUNK, 0, h->stream>>>(m, h->mw.ctl, h->mw.scal, h->mw.active,
                                                                    h->mw.restart);
    DDG_CHECK_LAUNCH();
}

void mloop_decide_true(ddg_handle h, int m, cudaGraphConditionalHandle cond) {
    mloop_decide_true_kernel<<<1, DDG_MCHUNK, 0, h->stream>>>(m, h->mw.ctl, h->mw.scal, h->mw.active,
                                                              h->mw.restart, h->errflags + E_TIMEOUT, cond);
    DDG_CHECK_LAUNCH();
}

void mloop_final_prep(ddg_handle h, int m) {
    mloop_final_prep_kernel<<<1, DDG_MCHUNK, 0, h->stream>>>(m, h->mw.ctl);
    DDG_CHECK_LAUNCH();
}

void mloop_final(ddg_handle h, int m) {
    mloop_final_kernel<<<1, DDG_MCHUNK, 0, h->stream>>>(m, h->mw.ctl, h->mw.scal);
    DDG_CHECK_LAUNCH();
}

void copy_cols(ddg_handle h, const double* src, int ms, int j0, double* dst, int md, int k0, int cnt) {
    copy_cols_kernel<<<(unsigned)((h->n * cnt + 255) / 256), 256, 0, h->stream>>>(h->n, src, ms, j0, dst, md, k0, cnt);
    DDG_CHECK_LAUNCH();
}

void multi_replace_cols_gated(ddg_handle h, int m, const double* src, double* dst, const int* replace,
                              const int* gate) {
    const int bd = col_block(m), rpb = bd / m;
    replace_cols_kernel<<<(unsigned)((h->n + rpb - 1) / rpb), bd, 0, h->stream>>>(h->n, m, src, dst, replace,
                                                                                  gate);
    DDG_CHECK_LAUNCH();
}

void multi_replace_cols(ddg_handle h, int m, const double* src, double* dst, const int* replace) {
    h->mw.r32_current = false;
    multi_replace_cols_gated(h, m, src, dst, replace, nullptr);
}

}  // namespace ddg
