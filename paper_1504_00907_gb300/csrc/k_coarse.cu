// The DDG coarse space (Sec. 4) and its exact solve.
//
// Setup
//   coarse_qr           R0: per subdomain, column-pivoted Gram-Schmidt (with one
//                       re-orthogonalisation pass) of F restricted to Omega_i,
//                       keeping column j while |R_jj| > rank_tol |R_00| (Sec. 4:
//                       orthogonalise per subdomain, discard rank-deficient
//                       columns).  Q is stored per node, kmax values.
//   coarse_assemble     A0 = R0 A R0^T block by block (blocks (I, J), I >= J, of
//                       adjacent subdomains) straight into a 64x64-tiled band.
//   band Cholesky       A0 = L L^T (FP64) in the tiled band, right-looking.
//   super-blocks        regroup L into super-blocks of Wt tiles so that L is
//                       block bidiagonal; D_K = L_KK^{-1} (tile forward
//                       substitution) and the coupling blocks
//                       F_K = D_K L_{K,K-1}, G_K = D_K^T L_{K+1,K}^T.
// Apply (FP64 or FP32)
//   c = R0 (r - A z)    coarse_restrict (residual fused)
//   y = A0^{-1} c       y = D c, y_K -= F_K y_{K-1}; x = D^T y, x_K -= G_K x_{K+1}:
//                       profile-row GEMVs, 2 (nK - 1) of them chained
//   z += R0^T y         coarse_prolong
#include <algorithm>

#include "ddg_internal.cuh"
#include "dev_common.cuh"
#include "tile64.cuh"

namespace {

using namespace tile64;

// ---------------------------------------------------------------- R0 (QR)
// KC >= k: per-thread partial sums of KC columns (32, or 96 for k > 32)
template <int KC>
__global__ void __launch_bounds__(256) coarse_qr_kernel(
    const int64_t* __restrict__ sub_off, const int32_t* __restrict__ sub_nodes,
    const double* __restrict__ F, int64_t n, int k, int kmax, double rank_tol, double* Q,
    int32_t* rank_out) {
    __shared__ double red[32 * 8];
    __shared__ double vals[KC];
    __shared__ int piv;
    __shared__ double r00;
    const int s = blockIdx.x;
    const int64_t a0 = sub_off[s], a1 = sub_off[s + 1];
    const int m = (int)(a1 - a0);
    for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
        const int g = sub_nodes[a];
        for (int j = 0; j < kmax; ++j) Q[a * kmax + j] = j < k ? F[g + (int64_t)j * n] : 0.0;
    }
    __syncthreads();
    auto colref = [&](int64_t a, int j) -> double& { return Q[a * kmax + j]; };
    int rank = 0;
    const int kk = min(k, m);
    for (int j = 0; j < kk; ++j) {
        // squared norms of the remaining columns j..k-1
        double v[KC];
#pragma unroll
        for (int c = 0; c < KC; ++c) v[c] = 0.0;
        for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x)
#pragma unroll
            for (int c = 0; c < KC; ++c)
                if (c >= j && c < k) {
                    const double t = colref(a, c);
                    v[c] = fma(t, t, v[c]);
                }
        ddgdev::block_sum_k<KC>(v, red, vals);
        if (threadIdx.x == 0) {
            int p = j;
            for (int c = j + 1; c < k; ++c)
                if (vals[c] > vals[p]) p = c;
            piv = p;
        }
        __syncthreads();
        const int p = piv;
        if (p != j)
            for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                const double t = colref(a, j);
                colref(a, j) = colref(a, p);
                colref(a, p) = t;
            }
        __syncthreads();
        // re-orthogonalise the pivot column against q_0..q_{j-1}
        if (j > 0) {
#pragma unroll
            for (int c = 0; c < KC; ++c) v[c] = 0.0;
            for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                const double t = colref(a, j);
#pragma unroll
                for (int c = 0; c < KC; ++c)
                    if (c < j) v[c] = fma(colref(a, c), t, v[c]);
            }
            ddgdev::block_sum_k<KC>(v, red, vals);
            for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                double t = colref(a, j);
                for (int c = 0; c < j; ++c) t -= vals[c] * colref(a, c);
                colref(a, j) = t;
            }
            __syncthreads();
        }
        double nn = 0.0;
        for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
            const double t = colref(a, j);
            nn = fma(t, t, nn);
        }
        const double rjj = sqrt(ddgdev::block_sum(nn, red));
        if (j == 0) {
            if (threadIdx.x == 0) r00 = rjj;
            __syncthreads();
        }
        if (!(rjj > rank_tol * r00) || !(r00 > 0.0)) break;
        const double inv = 1.0 / rjj;
        for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) colref(a, j) *= inv;
        __syncthreads();
        rank = j + 1;
        // remove q_j from the remaining columns (modified Gram-Schmidt step)
        if (j + 1 < k) {
#pragma unroll
            for (int c = 0; c < KC; ++c) v[c] = 0.0;
            for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                const double qj = colref(a, j);
#pragma unroll
                for (int c = 0; c < KC; ++c)
                    if (c > j && c < k) v[c] = fma(qj, colref(a, c), v[c]);
            }
            ddgdev::block_sum_k<KC>(v, red, vals);
            for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                const double qj = colref(a, j);
                for (int c = j + 1; c < k; ++c) colref(a, c) -= vals[c] * qj;
            }
            __syncthreads();
        }
    }
    for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x)
        for (int j = rank; j < kmax; ++j) colref(a, j) = 0.0;
    if (threadIdx.x == 0) rank_out[s] = rank;
}

// ---------------------------------------------------------------- A0 assembly
__device__ __forceinline__ size_t band_index(int row, int col, int Wt) {
    const int R = row / CT, C = col / CT;
    return ((size_t)R * (Wt + 1) + (R - C)) * CT * CT + (row % CT) * CT + (col % CT);
}

// One CTA per block (I, J), I >= J: A0[(I,s),(J,t)] = sum_{g in Omega_I}
// Q[g,s] sum_{c in row g, part(c) = J} A[g,c] Q[c,t].  With blk set, the
// whole kI x kJ block goes to blk[blockIdx.x][s][t] (row stride kmax)
// instead of the band's lower triangle.
__global__ void coarse_assemble_kernel(const int32_t* __restrict__ bI, const int32_t* __restrict__ bJ,
                                       const int64_t* __restrict__ sub_off,
                                       const int32_t* __restrict__ sub_nodes,
                                       const int32_t* __restrict__ pos,
                                       const int32_t* __restrict__ part,
                                       const int64_t* __restrict__ rowptr,
                                       const int32_t* __restrict__ col,
                                       const double* __restrict__ val,
                                       const double* __restrict__ Q, int kmax,
                                       const int32_t* __restrict__ coff, double* band, int Wt,
                                       double* blk) {
    const int I = bI[blockIdx.x], J = bJ[blockIdx.x];
    const int kI = coff[I + 1] - coff[I], kJ = coff[J + 1] - coff[J];
    for (int pr = threadIdx.x; pr < kI * kJ; pr += blockDim.x) {
        const int s = pr / kJ, t = pr % kJ;
        const int row = coff[I] + s, cl = coff[J] + t;
        if (!blk && row < cl) continue;
        double acc = 0.0;
        for (int64_t a = sub_off[I]; a < sub_off[I + 1]; ++a) {
            const int g = sub_nodes[a];
            double inner = 0.0;
            for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
                const int c = col[e];
                if (part[c] == J) inner = fma(val[e], Q[(int64_t)pos[c] * kmax + t], inner);
            }
            acc = fma(Q[a * kmax + s], inner, acc);
        }
        if (blk) blk[((size_t)blockIdx.x * kmax + s) * kmax + t] = acc;
        else band[band_index(row, cl, Wt)] = acc;
    }
}

__global__ void band_identity_pad_kernel(double* band, int Wt, int n0, int n0p) {
    const int i = n0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n0p) band[band_index(i, i, Wt)] = 1.0;
}

// ---------------------------------------------------------------- band Cholesky
// 64x64 tiles, 256 threads, 4x4 register micro-tiles (tile64.cuh)

// Tile (R, C), R >= C, of a factor stored as a band (tile row R holds the
// tiles R - Wt .. R, offset R - C) or, DENSE, as a full lower triangle of
// tiles in row order (the frontal matrices of the nested-dissection factor).
template <bool DENSE>
__device__ __forceinline__ size_t tile_at(int R, int C, int Wt) {
    return (DENSE ? (size_t)R * (R + 1) / 2 + C : (size_t)R * (Wt + 1) + (R - C)) * CT * CT;
}

// Batched use (local band factors of many subdomains, the fronts of one
// level of the nested-dissection tree): blockIdx.y selects matrix b of a
// batch, stored at band + boff[b] with its tile inverses at dinv + doff[b]
// and nts[b] tile rows, of which the first nss[b] are eliminated (a partial
// factorisation leaves the Schur complement in the trailing tiles; nss ==
// nullptr eliminates all); boff == nullptr is the single band.
template <bool DENSE>
__global__ void __launch_bounds__(256) band_potrf_kernel(double* band, int Wt, int k, double* dinv,
                                                         int* err, const int64_t* boff, const int64_t* doff,
                                                         const int32_t* nts, const int32_t* nss) {
    extern __shared__ double sm[];
    double* S = sm;
    double* X = sm + CT * CLD;
    __shared__ int bad;
    if (boff) {
        if (k >= (nss ? nss[blockIdx.y] : nts[blockIdx.y])) return;
        band += boff[blockIdx.y];
        dinv += doff[blockIdx.y];
    }
    double* tile = band + tile_at<DENSE>(k, k, Wt);
    if (threadIdx.x == 0) bad = 0;
    ct_load(S, tile);
    __syncthreads();
    for (int j = 0; j < CT; ++j) {
        if (threadIdx.x == 0) {
            double d = S[j * CLD + j];
            if (!(d > 0.0)) {
                bad = 1;
                d = 1.0;
            }
            S[j * CLD + j] = sqrt(d);
        }
        __syncthreads();
        if (threadIdx.x > j && threadIdx.x < CT) S[threadIdx.x * CLD + j] /= S[j * CLD + j];
        __syncthreads();
        for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) {
            const int r = i >> 6, c = i & 63;
            if (c > j && r >= c) S[r * CLD + c] -= S[r * CLD + j] * S[c * CLD + j];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) {
        const int r = i >> 6, c = i & 63;
        if (c > r) S[r * CLD + c] = 0.0;
        X[r * CLD + c] = 0.0;
    }
    __syncthreads();
    ct_store(tile, S);
    if (threadIdx.x < CT) {   // X = L_kk^{-1}, one thread per column
        const int c = threadIdx.x;
        X[c * CLD + c] = 1.0 / S[c * CLD + c];
        for (int r = c + 1; r < CT; ++r) {
            double s = 0.0;
            for (int m = c; m < r; ++m) s = fma(S[r * CLD + m], X[m * CLD + c], s);
            X[r * CLD + c] = -s / S[r * CLD + r];
        }
    }
    __syncthreads();
    ct_store(dinv + (size_t)k * CT * CT, X);
    if (threadIdx.x == 0 && bad) atomicExch(err, 1);
}

// L_ik = A_ik L_kk^{-T} for i = k+1 .. k+m
template <bool DENSE>
__global__ void __launch_bounds__(256) band_trsm_kernel(double* band, int Wt, int k,
                                                        const double* dinv, const int64_t* boff,
                                                        const int64_t* doff, const int32_t* nts,
                                                        const int32_t* nss) {
    extern __shared__ double sm[];
    double* A = sm;
    double* X = sm + CT * CLD;
    const int i = k + 1 + blockIdx.x;
    if (boff) {
        if (i >= nts[blockIdx.y] || (nss && k >= nss[blockIdx.y])) return;
        band += boff[blockIdx.y];
        dinv += doff[blockIdx.y];
    }
    double* tile = band + tile_at<DENSE>(i, k, Wt);
    ct_load(A, tile);
    ct_load(X, dinv + (size_t)k * CT * CT);
    __syncthreads();
    double acc[4][4];
    acc_zero4(acc);
    ct_mac<true>(acc, A, X);
    const int r0 = (threadIdx.x >> 4) * 4, c0 = (threadIdx.x & 15) * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) tile[(r0 + a) * CT + c0 + b] = acc[a][b];
}

// A_ij -= L_ik L_jk^T for k < j <= i <= k+m
template <bool DENSE>
__global__ void __launch_bounds__(256) band_update_kernel(double* band, int Wt, int k, const int64_t* boff,
                                                          const int32_t* nts, const int32_t* nss) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Bt = sm + CT * CLD;
    int p = blockIdx.x, i = k + 1, w = 1;
    while (p >= w) {   // pairs (i, j) enumerated row by row: row i has i - k tiles
        p -= w;
        ++i;
        ++w;
    }
    const int j = k + 1 + p;
    if (boff) {
        if (i >= nts[blockIdx.y] || (nss && k >= nss[blockIdx.y])) return;
        band += boff[blockIdx.y];
    }
    ct_load(A, band + tile_at<DENSE>(i, k, Wt));
    ct_load(Bt, band + tile_at<DENSE>(j, k, Wt));
    __syncthreads();
    double acc[4][4];
    acc_zero4(acc);
    ct_mac<true>(acc, A, Bt);
    double* C = band + tile_at<DENSE>(i, j, Wt);
    const int r0 = (threadIdx.x >> 4) * 4, c0 = (threadIdx.x & 15) * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) C[(r0 + a) * CT + c0 + b] -= acc[a][b];
}

// W = L_KK^{-1} of super-block K, tile column jj: W_jj = dinv, and for
// ii > jj: W_ij = -dinv_i sum_{m=jj}^{ii-1} L_im W_mj (tile forward substitution).
// DENSE: one super-block per batch entry, its nss[b] eliminated tiles.
template <bool DENSE>
__global__ void __launch_bounds__(256) superblock_inverse_kernel(const double* band, int Wt,
                                                                 const double* dinv, double* W,
                                                                 int NT, const int64_t* boff,
                                                                 const int64_t* doff, const int64_t* woff,
                                                                 const int32_t* nts, const int32_t* nss) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Bm = sm + CT * CLD;
    const int K = blockIdx.y, jj = blockIdx.x;
    const int Wl = Wt;   // tiles per super-block; the band layout's Wt
    if (boff) {
        NT = nts[blockIdx.z];
        if (DENSE) {
            Wt = nss[blockIdx.z];
            NT = Wt;
            if (jj >= Wt) return;
        }
        if (K * Wt >= NT) return;
        band += boff[blockIdx.z];
        dinv += doff[blockIdx.z];
        W += woff[blockIdx.z];
    }
    const int base = K * Wt;
    const size_t Ptiles = (size_t)Wt * (Wt + 1) / 2;
    auto wtile = [&](int ii, int j2) { return W + ((size_t)K * Ptiles + (size_t)ii * (ii + 1) / 2 + j2) * CT * CT; };
    const double* dj = dinv + (size_t)(base + jj) * CT * CT;
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) wtile(jj, jj)[e] = dj[e];
    __syncthreads();
    const int r0 = (threadIdx.x >> 4) * 4, c0 = (threadIdx.x & 15) * 4;
    for (int ii = jj + 1; ii < Wt; ++ii) {
        const int Ri = base + ii;
        if (Ri >= NT) break;
        double acc[4][4];
        acc_zero4(acc);
        for (int mm = jj; mm < ii; ++mm) {
            const int Rm = base + mm;
            ct_load(A, band + tile_at<DENSE>(Ri, Rm, Wl));
            ct_load(Bm, wtile(mm, jj));
            __syncthreads();
            ct_mac<false>(acc, A, Bm);
            __syncthreads();
        }
        // S -> Bm, dinv_i -> A, W_ij = -dinv_i S
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Bm[(r0 + a) * CLD + c0 + b] = acc[a][b];
        ct_load(A, dinv + (size_t)Ri * CT * CT);
        __syncthreads();
        acc_zero4(acc);
        ct_mac<false>(acc, A, Bm);
        double* out = wtile(ii, jj);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) out[(r0 + a) * CT + c0 + b] = -acc[a][b];
        __syncthreads();
    }
}

// Coupling blocks of the block-bidiagonal recurrence, 64x64 FP64 tiles:
//   F_K = D_K E_K      (K >= 1;  E_K = L_{K,K-1})
//   G_K = D_K^T E_{K+1}^T = (E_{K+1} D_K)^T   (K <= nK - 2)
// so that y_K = D_K c_K - F_K y_{K-1} and x_K = D_K^T y_K - G_K x_{K+1}.
// In tile terms E_K(m, J) is band tile (K Wt + m, Wt + m - J), nonzero for
// J >= m, and D_K(I, m) = W(K, I, m) for m <= I.  grid (Wt * Wt, nK, 2).
__global__ void __launch_bounds__(256) coupling_product_kernel(const double* band, const double* W, int Wt,
                                                               int nK, double* Ft, double* Gt) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Bm = sm + CT * CLD;
    const int K = blockIdx.y, I = blockIdx.x / Wt, J = blockIdx.x % Wt;
    const bool is_f = blockIdx.z == 0;
    if (is_f ? K == 0 : K >= nK - 1) return;
    const size_t Ptiles = (size_t)Wt * (Wt + 1) / 2;
    auto wtile = [&](int ii, int j2) { return W + ((size_t)K * Ptiles + (size_t)ii * (ii + 1) / 2 + j2) * CT * CT; };
    auto btile = [&](int R, int d) { return band + ((size_t)R * (Wt + 1) + d) * CT * CT; };
    double acc[4][4];
    acc_zero4(acc);
    if (is_f) {
        for (int m = 0; m <= min(I, J); ++m) {
            ct_load(A, wtile(I, m));
            ct_load(Bm, btile(K * Wt + m, Wt + m - J));
            __syncthreads();
            ct_mac<false>(acc, A, Bm);
            __syncthreads();
        }
    } else {
        // acc = H(J, I) = sum_m E_{K+1}(J, m) W(K, m, I)
        for (int m = max(I, J); m < Wt; ++m) {
            ct_load(A, btile((K + 1) * Wt + J, Wt + J - m));
            ct_load(Bm, wtile(m, I));
            __syncthreads();
            ct_mac<false>(acc, A, Bm);
            __syncthreads();
        }
    }
    const int r0 = (threadIdx.x >> 4) * 4, c0 = (threadIdx.x & 15) * 4;
    double* out = (is_f ? Ft : Gt) + (((size_t)K * Wt + I) * Wt + J) * CT * CT;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (is_f) out[(r0 + a) * CT + c0 + b] = acc[a][b];
            else out[(c0 + b) * CT + r0 + a] = acc[a][b];   // G tile = H tile transposed
        }
}

// profile-row fills (one warp per row)
enum { PM_D = 0, PM_DT = 1, PM_F = 2, PM_G = 3 };

template <int KIND>
__global__ void profile_fill_kernel(ProfileMat M, const int32_t* __restrict__ vlo,
                                    const int32_t* __restrict__ vhi, int rows, const double* W,
                                    const double* Tc, int Wt, int B) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= rows) return;
    const int i = wid;
    const int lo = M.lo[i], hi = M.hi[i];          // stored range (multiples of 4)
    const int tlo = vlo[i], thi = vhi[i];          // true nonzero range
    const int64_t rp = M.rowptr[i];
    const size_t Ptiles = (size_t)Wt * (Wt + 1) / 2;
    for (int jc = lo + lane; jc < hi; jc += 32) {
        double v = 0.0;
        if (jc >= tlo && jc < thi) {
            if (KIND == PM_D || KIND == PM_DT) {
                // D[a][b] with a >= b in super-block K: row-major W tiles
                const int a = KIND == PM_D ? i : jc, b = KIND == PM_D ? jc : i;
                const int K = a / B, la = a - K * B, lb = b - K * B;
                const int ti = la / CT, tj = lb / CT;
                v = W[((size_t)K * Ptiles + (size_t)ti * (ti + 1) / 2 + tj) * CT * CT + (la % CT) * CT + (lb % CT)];
            } else {
                // F_K (columns in super-block K-1) or G_K (columns in K+1) tiles
                const int K = i / B, li = i - K * B;
                const int lj = jc - (KIND == PM_F ? K - 1 : K + 1) * B;
                v = Tc[(((size_t)K * Wt + li / CT) * Wt + lj / CT) * CT * CT + (li % CT) * CT + (lj % CT)];
            }
        }
        M.v64[rp + (jc - lo)] = v;
        if (M.v32) M.v32[rp + (jc - lo)] = (float)v;
    }
}

// ---------------------------------------------------------------- apply
// out[i] = (a ? a[i] : 0) + sign * sum_{j in [lo_i, hi_i)} M[i][j] x[j], one warp
// per row.  Rows are stored on 4-aligned column ranges (zero padded), so each
// lane streams 16-byte chunks of the row and of x.
template <typename V> struct Vec4;
template <> struct Vec4<float> {
    using M = float4;
    static __device__ __forceinline__ M load(const float* m) {
        return __ldcs(reinterpret_cast<const float4*>(m));
    }
    static __device__ __forceinline__ float dot(const M& a, const float* x) {
        const float4 b = *reinterpret_cast<const float4*>(x);
        return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    }
    static __device__ __forceinline__ float dot(const float* m, const float* x) { return dot(load(m), x); }
};
template <> struct Vec4<double> {
    struct M {
        double2 a0, a1;
    };
    static __device__ __forceinline__ M load(const double* m) {
        return {__ldcs(reinterpret_cast<const double2*>(m)), __ldcs(reinterpret_cast<const double2*>(m + 2))};
    }
    static __device__ __forceinline__ double dot(const M& a, const double* x) {
        const double2 b0 = *reinterpret_cast<const double2*>(x);
        const double2 b1 = *reinterpret_cast<const double2*>(x + 2);
        return a.a0.x * b0.x + a.a0.y * b0.y + a.a1.x * b1.x + a.a1.y * b1.y;
    }
    static __device__ __forceinline__ double dot(const double* m, const double* x) { return dot(load(m), x); }
};

constexpr int GEMV_TPR = 64;    // threads per row (measured against 32, 128 and 256)
constexpr int GEMV_PF = 8;      // 16-byte chunks per thread loaded before the dependency wait

// Launched as a programmatic dependent of the previous step: the matrix row
// does not depend on that step, so it is read first; griddepcontrol.wait
// then orders the reads of x and a after the previous kernel's writes.
// Without the launch attribute both griddepcontrol instructions are no-ops.
// pf / pf_bytes: the next step's matrix rows, which every CTA's thread 0
// hands in equal 16-byte-multiple slices to the L2 prefetcher
// (cp.async.bulk.prefetch) before it reads its own row, so that the next
// step of the dependent chain finds its data in L2
template <typename V, typename MV>
__global__ void __launch_bounds__(GEMV_TPR) profile_gemv_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
    const MV* __restrict__ vals, int r0, const V* x, const V* a, V sign, V* out, const char* pf,
    unsigned long long pf_bytes) {
    __shared__ V sh[GEMV_TPR / 32];
    if (pf && threadIdx.x == 0) {
        const unsigned long long chunk = ((pf_bytes + gridDim.x - 1) / gridDim.x + 15) & ~15ull;
        const unsigned long long off = (unsigned long long)blockIdx.x * chunk;
        if (off < pf_bytes) {
            const unsigned sz = (unsigned)(chunk < pf_bytes - off ? chunk : pf_bytes - off);
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(pf + off), "r"(sz) : "memory");
        }
    }
    const int i = r0 + blockIdx.x;
    const int l = lo[i];
    const int nch = (hi[i] - l) >> 2;
    const MV* rv = vals + rowptr[i];
    typename Vec4<V>::M m[GEMV_PF];
#pragma unroll
    for (int k = 0; k < GEMV_PF; ++k) {
        const int c = threadIdx.x + k * GEMV_TPR;
        if (c < nch) m[k] = Vec4<V>::load(rv + 4 * c);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const V* xv = x + l;
    V s = 0;
#pragma unroll
    for (int k = 0; k < GEMV_PF; ++k) {
        const int c = threadIdx.x + k * GEMV_TPR;
        if (c < nch) s += Vec4<V>::dot(m[k], xv + 4 * c);
    }
    for (int c = threadIdx.x + GEMV_PF * GEMV_TPR; c < nch; c += GEMV_TPR)
        s += Vec4<V>::dot(Vec4<V>::load(rv + 4 * c), xv + 4 * c);
    s = ddgdev::warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        V t = 0;
#pragma unroll
        for (int w = 0; w < GEMV_TPR / 32; ++w) t += sh[w];
        out[i] = (a ? a[i] : (V)0) + sign * t;
    }
}

// c[coff_s + j] = sum_{g in Omega_s} Q[g, j] (r - A z)[g]   (z = 0 skips A z);
// the residual is matrix-free for the constant-coefficient Laplacians
template <int SK, int KC, typename V, typename AV>
__global__ void __launch_bounds__(256) coarse_restrict_kernel(
    const int64_t* __restrict__ sub_off, const int32_t* __restrict__ sub_nodes,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const AV* __restrict__ val,
    const V* __restrict__ r, const V* __restrict__ z, const V* __restrict__ Q, int kmax,
    const int32_t* __restrict__ coff, V* __restrict__ c, int residual, int nx, int ny, int nz) {
    __shared__ V red[32 * 8];
    __shared__ V out[KC];
    const int s = blockIdx.x;
    // launched as a programmatic dependent of the last local solve: the
    // subdomain's rows of Q (fixed at setup) go to L2 before the wait, r and
    // z are read after it
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    {
        const uintptr_t b = reinterpret_cast<uintptr_t>(Q + sub_off[s] * kmax);
        const uintptr_t e = reinterpret_cast<uintptr_t>(Q + sub_off[s + 1] * kmax);
        for (uintptr_t p = (b & ~(uintptr_t)127) + (uintptr_t)threadIdx.x * 128; p < e; p += (uintptr_t)blockDim.x * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    V acc[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] = 0;
    if constexpr (SK == ddgdev::SK_CSRW) {
        // a group of CSRW_G lanes per row computes its residual; the group's
        // first lane adds the row's Q contributions
        constexpr int G = ddgdev::CSRW_G;
        const int64_t a_end = sub_off[s + 1];
        for (int64_t base = sub_off[s]; base < a_end; base += blockDim.x / G) {
            const int64_t a = base + threadIdx.x / G;
            const bool live = a < a_end;
            const int g = live ? sub_nodes[a] : 0;
            V az = 0;
            if (residual) az = ddgdev::csr_row_dot_group<G>(g, live, rowptr, col, val, z);
            if (live && (threadIdx.x & (G - 1)) == 0) {
                const V w = r[g] - az;
                const V* qa = Q + a * kmax;
#pragma unroll
                for (int j = 0; j < KC; ++j)
                    if (j < kmax) acc[j] = fma(qa[j], w, acc[j]);
            }
        }
    } else {
        for (int64_t a = sub_off[s] + threadIdx.x; a < sub_off[s + 1]; a += blockDim.x) {
            const int g = sub_nodes[a];
            V w = r[g];
            if (residual) {
                if (SK == DDG_STENCIL_7PT_3D || SK == DDG_STENCIL_5PT_2D) {
                    const int i = g % nx, jj = (g / nx) % ny;
                    V az = (SK == DDG_STENCIL_7PT_3D ? (V)6 : (V)4) * z[g];
                    if (i > 0) az -= z[g - 1];
                    if (i < nx - 1) az -= z[g + 1];
                    if (jj > 0) az -= z[g - nx];
                    if (jj < ny - 1) az -= z[g + nx];
                    if (SK == DDG_STENCIL_7PT_3D) {
                        const int k = g / (nx * ny);
                        if (k > 0) az -= z[g - nx * ny];
                        if (k < nz - 1) az -= z[g + nx * ny];
                    }
                    w -= az;
                } else if (SK == ddgdev::SK_CSR8) {
                    w -= ddgdev::csr_row_dot_unrolled<8>(g, rowptr, col, val, z, 1, 0);
                } else if (SK == ddgdev::SK_CSR16) {
                    w -= ddgdev::csr_row_dot_unrolled<16>(g, rowptr, col, val, z, 1, 0);
                } else {
                    for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) w -= (V)val[e] * z[col[e]];
                }
            }
            const V* qa = Q + a * kmax;
#pragma unroll
            for (int j = 0; j < KC; ++j)
                if (j < kmax) acc[j] = fma(qa[j], w, acc[j]);
        }
    }
    ddgdev::block_sum_k<KC>(acc, red, out);
    const int ks = coff[s + 1] - coff[s];
    if (threadIdx.x < ks) c[coff[s] + threadIdx.x] = out[threadIdx.x];
}

// z[g] += sum_j Q[pos g, j] y[coff_{part g} + j]
template <typename V>
__global__ void coarse_prolong_kernel(int64_t n, const int32_t* __restrict__ part,
                                      const int32_t* __restrict__ pos, const V* __restrict__ Q,
                                      int kmax, const int32_t* __restrict__ coff,
                                      const V* __restrict__ y, V* __restrict__ z) {
    // a programmatic dependent of the coarse solve: the row of Q and the
    // indices (fixed at setup) are read before the wait, y and z after it
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;   // reads nothing the coarse solve writes
    const int s = part[g];
    const int c0 = coff[s], ks = coff[s + 1] - c0;
    const V* qa = Q + (int64_t)pos[g] * kmax;
    if (ks > 0) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(qa));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(qa + ks - 1));
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    V acc = 0;
    for (int j = 0; j < ks; ++j) acc = fma(qa[j], y[c0 + j], acc);
    z[g] += acc;
}

// Sec. 6, three-level V-cycle: the coarsened generators F0 = R0 F.  Row
// (I, s) of F0 is q_{I,s}^T F restricted to the subdomain I: one CTA per
// subdomain, one thread per (s, j), summing over the subdomain's nodes in
// position order.  F column-major [n][k], F0 column-major [n0][k].
__global__ void __launch_bounds__(256) coarse_generators_kernel(
    const int64_t* __restrict__ sub_off, const int32_t* __restrict__ sub_nodes,
    const int32_t* __restrict__ coff, const double* __restrict__ Q, int kmax,
    const double* __restrict__ F, int64_t n, int k, int n0, double* __restrict__ F0) {
    const int I = blockIdx.x;
    const int c0 = coff[I], kI = coff[I + 1] - c0;
    const int64_t a0 = sub_off[I], a1 = sub_off[I + 1];
    for (int e = threadIdx.x; e < kI * k; e += blockDim.x) {
        const int s = e % kI, j = e / kI;
        double acc = 0.0;
        for (int64_t a = a0; a < a1; ++a) acc = fma(Q[a * kmax + s], F[(int64_t)j * n + sub_nodes[a]], acc);
        F0[(int64_t)j * n0 + c0 + s] = acc;
    }
}

}  // namespace

namespace ddg {

void coarse_generators(ddg_handle h, const double* dF, int k, double* dF0) {
    coarse_generators_kernel<<<h->nsub, 256, 0, h->stream>>>(h->sub_off, h->sub_nodes, h->coff, h->Q64,
                                                             h->kmax, dF, h->n, k, h->n0, dF0);
    DDG_CHECK_LAUNCH();
}

void coarse_qr(ddg_handle h, int32_t* d_rank, const double* dF, int k) {
    auto qr = h->kmax <= 32 ? coarse_qr_kernel<32> : coarse_qr_kernel<DDG_KMAX>;
    qr<<<h->nsub, 256, 0, h->stream>>>(h->sub_off, h->sub_nodes, dF, h->n, k, h->kmax,
                                                     h->opt.rank_tol, h->Q64, d_rank);
    DDG_CHECK_LAUNCH();
}

void coarse_assemble_band(ddg_handle h, const std::vector<int>& bI, const std::vector<int>& bJ) {
    const size_t ntiles = (size_t)h->NT * (h->Wt + 1);
    DDG_CUDA(cudaMemsetAsync(h->bandL, 0, ntiles * CT * CT * sizeof(double), h->stream));
    if (!bI.empty()) {
        int32_t* dI = h->arena.alloc<int32_t>(bI.size());
        int32_t* dJ = h->arena.alloc<int32_t>(bJ.size());
        h2d(dI, bI.data(), bI.size(), h->stream);
        h2d(dJ, bJ.data(), bJ.size(), h->stream);
        coarse_assemble_kernel<<<(unsigned)bI.size(), 128, 0, h->stream>>>(
            dI, dJ, h->sub_off, h->sub_nodes, h->pos, h->part, h->rowptr, h->col, h->val64, h->Q64,
            h->kmax, h->coff, h->bandL, h->Wt, nullptr);
        DDG_CHECK_LAUNCH();
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        h->arena.release(dI);
        h->arena.release(dJ);
    }
    const int npad = h->n0p - h->n0;
    if (npad > 0) {
        band_identity_pad_kernel<<<(npad + 255) / 256, 256, 0, h->stream>>>(h->bandL, h->Wt, h->n0,
                                                                            h->n0p);
        DDG_CHECK_LAUNCH();
    }
}

void coarse_assemble_blocks(ddg_handle h, const std::vector<int>& bI, const std::vector<int>& bJ,
                            std::vector<double>& blocks) {
    const size_t per = (size_t)h->kmax * h->kmax;
    blocks.assign(bI.size() * per, 0.0);
    if (bI.empty()) return;
    int32_t* dI = h->arena.alloc<int32_t>(bI.size());
    int32_t* dJ = h->arena.alloc<int32_t>(bJ.size());
    double* dB = h->arena.alloc<double>(bI.size() * per);
    DDG_CUDA(cudaMemsetAsync(dB, 0, bI.size() * per * sizeof(double), h->stream));
    h2d(dI, bI.data(), bI.size(), h->stream);
    h2d(dJ, bJ.data(), bJ.size(), h->stream);
    coarse_assemble_kernel<<<(unsigned)bI.size(), 128, 0, h->stream>>>(
        dI, dJ, h->sub_off, h->sub_nodes, h->pos, h->part, h->rowptr, h->col, h->val64, h->Q64, h->kmax,
        h->coff, nullptr, 0, dB);
    DDG_CHECK_LAUNCH();
    d2h(blocks.data(), dB, blocks.size(), h->stream);
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    h->arena.release(dI);
    h->arena.release(dJ);
    h->arena.release(dB);
}

double* coarse_assemble_blocks_device(ddg_handle h, const std::vector<int>& bI, const std::vector<int>& bJ) {
    const size_t per = (size_t)h->kmax * h->kmax;
    double* dB = h->arena.alloc<double>(std::max<size_t>(1, bI.size() * per));
    if (bI.empty()) return dB;
    int32_t* dI = h->arena.alloc<int32_t>(bI.size());
    int32_t* dJ = h->arena.alloc<int32_t>(bJ.size());
    DDG_CUDA(cudaMemsetAsync(dB, 0, bI.size() * per * sizeof(double), h->stream));
    h2d(dI, bI.data(), bI.size(), h->stream);
    h2d(dJ, bJ.data(), bJ.size(), h->stream);
    coarse_assemble_kernel<<<(unsigned)bI.size(), 128, 0, h->stream>>>(
        dI, dJ, h->sub_off, h->sub_nodes, h->pos, h->part, h->rowptr, h->col, h->val64, h->Q64, h->kmax,
        h->coff, nullptr, 0, dB);
    DDG_CHECK_LAUNCH();
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    h->arena.release(dI);
    h->arena.release(dJ);
    return dB;
}

// the tile kernels take two 64 x 65 FP64 tiles of dynamic shared memory
static void configure_band_kernels() {
    static PerDeviceMax configured;
    const int sm2 = (int)(2 * CT * CLD * sizeof(double));
    int dev = -1;
    if (!configured.needs(sm2, dev)) return;
    DDG_CUDA(cudaFuncSetAttribute(band_potrf_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(band_trsm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(band_update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(superblock_inverse_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(band_potrf_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(band_trsm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(band_update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    DDG_CUDA(cudaFuncSetAttribute(superblock_inverse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    configured.commit(dev, sm2);
}

void coarse_band_cholesky(ddg_handle h) {
    const size_t sm2 = 2 * CT * CLD * sizeof(double);
    configure_band_kernels();
    double* dinv = h->arena.alloc<double>((size_t)h->NT * CT * CT);
    const int Wt = h->Wt, NT = h->NT;
    for (int k = 0; k < NT; ++k) {
        band_potrf_kernel<false><<<1, 256, sm2, h->stream>>>(h->bandL, Wt, k, dinv, h->errflags + E_COARSE_SPD,
                                                             nullptr, nullptr, nullptr, nullptr);
        DDG_CHECK_LAUNCH();
        const int m = std::min(Wt, NT - 1 - k);
        if (m > 0) {
            band_trsm_kernel<false><<<m, 256, sm2, h->stream>>>(h->bandL, Wt, k, dinv, nullptr, nullptr, nullptr,
                                                                nullptr);
            DDG_CHECK_LAUNCH();
            band_update_kernel<false><<<m * (m + 1) / 2, 256, sm2, h->stream>>>(h->bandL, Wt, k, nullptr, nullptr,
                                                                                nullptr);
            DDG_CHECK_LAUNCH();
        }
    }
    // super-block inverses D_K = L_KK^{-1}
    const size_t Ptiles = (size_t)Wt * (Wt + 1) / 2;
    double* W = h->arena.alloc<double>((size_t)h->nK * Ptiles * CT * CT);
    DDG_CUDA(cudaMemsetAsync(W, 0, (size_t)h->nK * Ptiles * CT * CT * sizeof(double), h->stream));
    superblock_inverse_kernel<false><<<dim3(Wt, h->nK), 256, sm2, h->stream>>>(h->bandL, Wt, dinv, W, NT, nullptr,
                                                                                nullptr, nullptr, nullptr, nullptr);
    DDG_CHECK_LAUNCH();
    h->coarseW = W;
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    h->arena.release(dinv);
}

// Band Cholesky of nb bands at once (the local band factors): band b holds
// nts[b] tile rows of Wt + 1 tiles at band + boff[b] (device offsets); the
// tile inverses L_kk^{-1} go to dinv + doff[b] and the super-block inverses
// D_K = L_KK^{-1} (lower tiles) to W + woff[b].  A non-positive pivot sets err.
void band_factor_batched(ddg_handle h, double* band, int Wt, int nb, int NTmax, const int64_t* boff,
                         const int32_t* nts, double* dinv, const int64_t* doff, double* W,
                         const int64_t* woff, int* err) {
    const size_t sm2 = 2 * CT * CLD * sizeof(double);
    configure_band_kernels();
    for (int k = 0; k < NTmax; ++k) {
        band_potrf_kernel<false><<<dim3(1, nb), 256, sm2, h->stream>>>(band, Wt, k, dinv, err, boff, doff, nts,
                                                                       nullptr);
        DDG_CHECK_LAUNCH();
        const int m = std::min(Wt, NTmax - 1 - k);
        if (m > 0) {
            band_trsm_kernel<false><<<dim3(m, nb), 256, sm2, h->stream>>>(band, Wt, k, dinv, boff, doff, nts,
                                                                          nullptr);
            DDG_CHECK_LAUNCH();
            band_update_kernel<false><<<dim3(m * (m + 1) / 2, nb), 256, sm2, h->stream>>>(band, Wt, k, boff, nts,
                                                                                          nullptr);
            DDG_CHECK_LAUNCH();
        }
    }
    superblock_inverse_kernel<false><<<dim3(Wt, NTmax / Wt, nb), 256, sm2, h->stream>>>(
        band, Wt, dinv, W, NTmax, boff, doff, woff, nts, nullptr);
    DDG_CHECK_LAUNCH();
}

// Partial Cholesky of the dense fronts of one level of the nested-dissection
// tree: front b (lower tiles at fronts + foff[b], nts[b] tile rows) has its
// first nss[b] tile columns eliminated, leaving L11, L21 and the Schur
// complement (the update matrix) in place; the inverse of L11 (packed lower
// tiles) goes to W + woff[b].
void front_factor_batched(ddg_handle h, double* fronts, int nb, int NTmax, int NSmax, const int64_t* foff,
                          const int32_t* nts, const int32_t* nss, double* dinv, const int64_t* doff, double* W,
                          const int64_t* woff, int* err) {
    const size_t sm2 = 2 * CT * CLD * sizeof(double);
    configure_band_kernels();
    for (int k = 0; k < NSmax; ++k) {
        band_potrf_kernel<true><<<dim3(1, nb), 256, sm2, h->stream>>>(fronts, 0, k, dinv, err, foff, doff, nts,
                                                                      nss);
        DDG_CHECK_LAUNCH();
        const int m = NTmax - 1 - k;
        if (m > 0) {
            band_trsm_kernel<true><<<dim3(m, nb), 256, sm2, h->stream>>>(fronts, 0, k, dinv, foff, doff, nts, nss);
            DDG_CHECK_LAUNCH();
            band_update_kernel<true><<<dim3(m * (m + 1) / 2, nb), 256, sm2, h->stream>>>(fronts, 0, k, foff, nts,
                                                                                         nss);
            DDG_CHECK_LAUNCH();
        }
    }
    superblock_inverse_kernel<true><<<dim3(NSmax, 1, nb), 256, sm2, h->stream>>>(fronts, 0, dinv, W, 0, foff, doff,
                                                                                woff, nts, nss);
    DDG_CHECK_LAUNCH();
}

// Rows are stored on [lo & ~3, (hi + 3) & ~3) so that every row starts on a
// 16-byte boundary; returns the true ranges (device) for the fill kernel.
static void alloc_profile(ddg_handle h, ProfileMat& M, const std::vector<int>& lo,
                          const std::vector<int>& hi, bool fp32, int32_t** vlo, int32_t** vhi) {
    const int rows = (int)lo.size();
    std::vector<int> lo4(rows), hi4(rows);
    std::vector<int64_t> rp(rows + 1, 0);
    for (int i = 0; i < rows; ++i) {
        if (hi[i] > lo[i]) {
            lo4[i] = lo[i] & ~3;
            hi4[i] = (hi[i] + 3) & ~3;
        } else {
            lo4[i] = hi4[i] = 0;
        }
        rp[i + 1] = rp[i] + (hi4[i] - lo4[i]);
    }
    M.nnz = rp[rows];
    M.h_rowptr = rp;
    M.rowptr = h->arena.alloc<int64_t>(rows + 1);
    M.lo = h->arena.alloc<int32_t>(rows);
    M.hi = h->arena.alloc<int32_t>(rows);
    M.v64 = h->arena.alloc<double>(M.nnz);
    M.v32 = fp32 ? h->arena.alloc<float>(M.nnz) : nullptr;
    *vlo = h->arena.alloc<int32_t>(rows);
    *vhi = h->arena.alloc<int32_t>(rows);
    h2d(M.rowptr, rp.data(), rows + 1, h->stream);
    h2d(M.lo, lo4.data(), rows, h->stream);
    h2d(M.hi, hi4.data(), rows, h->stream);
    h2d(*vlo, lo.data(), rows, h->stream);
    h2d(*vhi, hi.data(), rows, h->stream);
    DDG_CUDA(cudaStreamSynchronize(h->stream));
}

void coarse_build_apply(ddg_handle h) {
    const int n0p = h->n0p, B = h->B, Wt = h->Wt, nK = h->nK;
    const bool fp32 = true;
    // coupling blocks F_K, G_K (FP64 tiles, released after the fill)
    const size_t ntile = (size_t)nK * Wt * Wt * CT * CT;
    double* Ft = h->arena.alloc<double>(ntile);
    double* Gt = h->arena.alloc<double>(ntile);
    if (nK > 1) {
        const size_t sm2 = 2 * CT * CLD * sizeof(double);
        DDG_CUDA(cudaFuncSetAttribute(coupling_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
        coupling_product_kernel<<<dim3(Wt * Wt, nK, 2), 256, sm2, h->stream>>>(h->bandL, h->coarseW, Wt, nK, Ft, Gt);
        DDG_CHECK_LAUNCH();
    }
    std::vector<int> lo(n0p), hi(n0p);
    int32_t *vlo[4], *vhi[4];
    // D: lower triangle of the super-block
    for (int i = 0; i < n0p; ++i) {
        lo[i] = (i / B) * B;
        hi[i] = i + 1;
    }
    alloc_profile(h, h->Dm, lo, hi, fp32, &vlo[0], &vhi[0]);
    // D^T: upper triangle of the super-block
    for (int i = 0; i < n0p; ++i) {
        lo[i] = i;
        hi[i] = (i / B + 1) * B;
    }
    alloc_profile(h, h->Dt, lo, hi, fp32, &vlo[1], &vhi[1]);
    // F_K: rows of super-block K >= 1, all columns of K - 1
    for (int i = 0; i < n0p; ++i) {
        const int K = i / B;
        lo[i] = K == 0 ? 0 : (K - 1) * B;
        hi[i] = K == 0 ? 0 : K * B;
    }
    alloc_profile(h, h->Fm, lo, hi, fp32, &vlo[2], &vhi[2]);
    // G_K: rows of super-block K <= nK - 2, all columns of K + 1
    for (int i = 0; i < n0p; ++i) {
        const int K = i / B;
        lo[i] = K >= nK - 1 ? 0 : (K + 1) * B;
        hi[i] = K >= nK - 1 ? 0 : (K + 2) * B;
    }
    alloc_profile(h, h->Gm, lo, hi, fp32, &vlo[3], &vhi[3]);
    const unsigned blocks = (unsigned)((n0p * 32 + 255) / 256);
    profile_fill_kernel<PM_D><<<blocks, 256, 0, h->stream>>>(h->Dm, vlo[0], vhi[0], n0p, h->coarseW, nullptr, Wt, B);
    profile_fill_kernel<PM_DT><<<blocks, 256, 0, h->stream>>>(h->Dt, vlo[1], vhi[1], n0p, h->coarseW, nullptr, Wt, B);
    profile_fill_kernel<PM_F><<<blocks, 256, 0, h->stream>>>(h->Fm, vlo[2], vhi[2], n0p, nullptr, Ft, Wt, B);
    profile_fill_kernel<PM_G><<<blocks, 256, 0, h->stream>>>(h->Gm, vlo[3], vhi[3], n0p, nullptr, Gt, Wt, B);
    DDG_CHECK_LAUNCH();
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < 4; ++t) {
        h->arena.release(vlo[t]);
        h->arena.release(vhi[t]);
    }
    h->arena.release(Ft);
    h->arena.release(Gt);
    h->arena.release(h->coarseW);
    h->coarseW = nullptr;
    h->arena.release(h->bandL);
    h->bandL = nullptr;
}

template <int SK, int KC>
static void launch_restrict_k(ddg_handle h, int prec, bool residual) {
    if (prec == DDG_PREC_FP64)
        launch_pdl(h, coarse_restrict_kernel<SK, KC, double, double>, dim3(h->nsub), dim3(256), 0,
                   (const int64_t*)h->sub_off, (const int32_t*)h->sub_nodes, (const int64_t*)h->rowptr,
                   (const int32_t*)h->col, (const double*)h->val64, (const double*)h->rin64,
                   (const double*)h->z64, (const double*)h->Q64, h->kmax, (const int32_t*)h->coff, h->c64,
                   residual ? 1 : 0, h->nx, h->ny, h->nz);
    else
        launch_pdl(h, coarse_restrict_kernel<SK, KC, float, float>, dim3(h->nsub), dim3(256), 0,
                   (const int64_t*)h->sub_off, (const int32_t*)h->sub_nodes, (const int64_t*)h->rowptr,
                   (const int32_t*)h->col, (const float*)h->val32, (const float*)h->r32, (const float*)h->z32,
                   (const float*)h->Q32, h->kmax, (const int32_t*)h->coff, h->c32, residual ? 1 : 0, h->nx,
                   h->ny, h->nz);
    DDG_CHECK_LAUNCH();
}

template <int SK>
static void launch_restrict(ddg_handle h, int prec, bool residual) {
    if (h->kmax <= 32) launch_restrict_k<SK, 32>(h, prec, residual);
    else launch_restrict_k<SK, DDG_KMAX>(h, prec, residual);
}

void coarse_restrict(ddg_handle h, int prec, bool residual) {
#define CR_CALL(SK) launch_restrict<SK>(h, prec, residual)
    DDG_DISPATCH_SK(h, CR_CALL);
#undef CR_CALL
}

template <typename V>
static void gemv(ddg_handle h, const ProfileMat& M, int r0, int r1, const V* x, const V* a, V sign,
                 V* out, const ProfileMat* pfM = nullptr, int pf0 = 0, int pf1 = 0) {
    // the rows [pf0, pf1) of pfM go to L2 while this step runs (16-byte
    // multiples: every profile row is a multiple of four values)
    const char* pf = nullptr;
    unsigned long long pf_bytes = 0;
    if (pfM && pf1 > pf0 && !pfM->h_rowptr.empty()) {
        const size_t es = sizeof(V) == 8 ? 8 : 4;
        const char* base = sizeof(V) == 8 ? (const char*)pfM->v64 : (const char*)pfM->v32;
        pf = base + (size_t)pfM->h_rowptr[pf0] * es;
        pf_bytes = (unsigned long long)(pfM->h_rowptr[pf1] - pfM->h_rowptr[pf0]) * es;
        if (pf_bytes == 0) pf = nullptr;
    }
    if (r1 <= r0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(r1 - r0));
    cfg.blockDim = dim3(GEMV_TPR);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = h->use_pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (sizeof(V) == 8)
        DDG_CUDA(cudaLaunchKernelEx(&cfg, profile_gemv_kernel<double, double>, (const int64_t*)M.rowptr,
                                    (const int32_t*)M.lo, (const int32_t*)M.hi, (const double*)M.v64, r0,
                                    (const double*)x, (const double*)a, (double)sign, (double*)out, pf,
                                    pf_bytes));
    else
        DDG_CUDA(cudaLaunchKernelEx(&cfg, profile_gemv_kernel<float, float>, (const int64_t*)M.rowptr,
                                    (const int32_t*)M.lo, (const int32_t*)M.hi, (const float*)M.v32, r0,
                                    (const float*)x, (const float*)a, (float)sign, (float*)out, pf,
                                    pf_bytes));
}

// y = L^{-1} c and x = L^{-T} y on the block-bidiagonal factor:
//   y = D c (all super-blocks at once), then y_K -= F_K y_{K-1} for K = 1, 2, ...
//   x = D^T y, then x_K -= G_K x_{K+1} for K = nK-2, ..., 0
// 2 nK launches, of which 2 (nK - 1) form the dependent chain
// Each step of the two chains prefetches the next step's block of F or G
// into L2 (and the block-diagonal steps the chain's first block), so the
// chain reads from L2 while HBM streams the block after it.
template <typename V>
static void coarse_solve_t(ddg_handle h, V* c, V* y, V* x) {
    const int B = h->B, nK = h->nK, n0p = h->n0p;
    gemv<V>(h, h->Dm, 0, n0p, c, nullptr, (V)1, y, &h->Fm, B, std::min(2, nK) * B);
    for (int K = 1; K < nK; ++K)
        gemv<V>(h, h->Fm, K * B, (K + 1) * B, y, y, (V)-1, y, &h->Fm, (K + 1) * B, std::min(K + 2, nK) * B);
    gemv<V>(h, h->Dt, 0, n0p, y, nullptr, (V)1, x, &h->Gm, std::max(0, nK - 2) * B, std::max(0, nK - 1) * B);
    for (int K = nK - 2; K >= 0; --K)
        gemv<V>(h, h->Gm, K * B, (K + 1) * B, x, x, (V)-1, x, &h->Gm, std::max(0, K - 1) * B, K * B);
}

void coarse_solve(ddg_handle h, int prec) {
    if (h->nd.on) {
        nd_coarse_solve(h, prec);
        return;
    }
    if (prec == DDG_PREC_FP64) coarse_solve_t<double>(h, h->c64, h->y64, h->x64);
    else coarse_solve_t<float>(h, h->c32, h->y32, h->x32);
}

void coarse_prolong(ddg_handle h, int prec) {
    const unsigned blocks = (unsigned)((h->n + 255) / 256);
    if (prec == DDG_PREC_FP64)
        launch_pdl(h, coarse_prolong_kernel<double>, dim3(blocks), dim3(256), 0, h->n, (const int32_t*)h->part,
                   (const int32_t*)h->pos, (const double*)h->Q64, h->kmax, (const int32_t*)h->coff,
                   (const double*)h->x64, h->z64);
    else
        launch_pdl(h, coarse_prolong_kernel<float>, dim3(blocks), dim3(256), 0, h->n, (const int32_t*)h->part,
                   (const int32_t*)h->pos, (const float*)h->Q32, h->kmax, (const int32_t*)h->coff,
                   (const float*)h->x32, h->z32);
    DDG_CHECK_LAUNCH();
}

}  // namespace ddg
