// Exact coarse solve A0^{-1} (Sec. 4) through a nested-dissection Cholesky
// factor of A0 (coarse_order ND).
//
// The coarse dofs of one subdomain stay together: the graph is that of the
// subdomains that A0 couples, each weighted by its number of coarse dofs.
// Nested dissection (recursive bisection by BFS level sets from a
// pseudo-peripheral subdomain, the middle level the separator) orders the
// subdomains; each separator is a front of the multifrontal factorisation:
// its dense frontal matrix holds the front's own rows S and the rows U of
// the ancestors' subdomains that its subtree couples to.  Fronts are
// factorised level by level from the leaves (children's Schur complements
// added into the parent, original A0 blocks placed in the front of the
// earlier-eliminated subdomain), with the batched tile kernels in dense
// mode.  Per front the solve keeps D = L_SS^{-1} and G = L_US D (FP64 and
// FP32), since L_US y_S = L_US D w_S = G w_S and D^T L_US^T = G^T:
//   forward  (leaves first)  y_S = D w_S,  w_U -= G w_S
//   backward (root first)    x_S = D^T y_S - G^T x_U
// so each level is one launch per direction (its products read only data
// that earlier levels finished).  The solve runs on vectors permuted to the
// elimination order, where every front's S rows are one contiguous range;
// D, D^T, G and G^T are stored by rows, so every product is a row-per-warp
// dot product over contiguous data (only x_U is gathered).  The updates of
// w are summed per target in a fixed order, so the solve is deterministic.
#include <algorithm>
#include <cstdlib>
#include <deque>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "ddg_internal.cuh"
#include "dev_common.cuh"
#include "tile64.cuh"

namespace {

using namespace tile64;
constexpr int ND_LEAF_DOFS = 256;   // a part of at most this many coarse dofs is a leaf front

__host__ __device__ __forceinline__ int r4(int v) { return (v + 3) & ~3; }

// element offset of row i of a packed lower triangle whose row r holds the
// columns [0, r] padded to a multiple of 4: sum_{r < i} r4(r + 1)
__host__ __device__ __forceinline__ int64_t drow(int i) {
    const int64_t q = i / 4, rem = i % 4;
    return 4 * (2 * q * (q + 1) + rem * (q + 1));
}

// element offset of row j of a packed upper triangle of n columns whose row
// r holds the columns [r & ~3, n) padded to a multiple of 4
__host__ __device__ __forceinline__ int64_t dtrow(int j, int n) {
    const int64_t q = j / 4, rem = j % 4;
    return (int64_t)j * r4(n) - 8 * q * (q - 1) - 4 * q * rem;
}

// element (r, c), r >= c, of a front stored as lower 64 x 64 tiles in row order
__device__ __forceinline__ size_t dtile(int r, int c) {
    const int R = r / CT, C = c / CT;
    return ((size_t)R * (R + 1) / 2 + C) * CT * CT + (size_t)(r % CT) * CT + (c % CT);
}

struct NdPlace {
    int64_t foff, blk;
    int rpos, cpos, kr, kc, trans, diag;
};

// the blocks A0[(I,.),(J,.)] (I >= J, row stride kmax) into their fronts
__global__ void nd_scatter_kernel(const NdPlace* __restrict__ pl, const double* __restrict__ blocks, int kmax,
                                  double* fronts) {
    const NdPlace P = pl[blockIdx.x];
    for (int e = threadIdx.x; e < P.kr * P.kc; e += blockDim.x) {
        const int s = e / P.kc, t = e % P.kc;
        if (P.diag && t > s) continue;
        const double v = P.trans ? blocks[P.blk + (size_t)t * kmax + s] : blocks[P.blk + (size_t)s * kmax + t];
        fronts[P.foff + dtile(P.rpos + s, P.cpos + t)] = v;
    }
}

// unit diagonal on the padding rows of a front: [a0, a1) and [b0, b1)
__global__ void nd_pad_kernel(const int64_t* __restrict__ foff, const int4* __restrict__ pads, double* fronts) {
    const int4 p = pads[blockIdx.x];
    double* F = fronts + foff[blockIdx.x];
    for (int i = p.x + threadIdx.x; i < p.y; i += blockDim.x) F[dtile(i, i)] = 1.0;
    for (int i = p.z + threadIdx.x; i < p.w; i += blockDim.x) F[dtile(i, i)] = 1.0;
}

struct NdChild {
    int64_t cfoff, pfoff, map_off;
    int cbase;   // first row of the child's update matrix in its front
};

// parent[map a][map b] += child update[a][b], b <= a (one row a per CTA)
__global__ void nd_extend_kernel(const NdChild* __restrict__ ch, const int2* __restrict__ items,
                                 const int32_t* __restrict__ map, double* fronts) {
    const int2 it = items[blockIdx.x];
    const NdChild C = ch[it.x];
    const int a = it.y;
    const int pa = map[C.map_off + a];
    for (int b = threadIdx.x; b <= a; b += blockDim.x)
        fronts[C.pfoff + dtile(pa, map[C.map_off + b])] += fronts[C.cfoff + dtile(C.cbase + a, C.cbase + b)];
}

struct NdPack {
    int64_t foff, woff, goff, doff, loff, dtoff, ltoff;   // loff / ltoff: rows of G / G^T
    int nS, nU, nSt;
};

__device__ __forceinline__ double nd_dinv(const NdPack& P, const double* W, int i, int j) {
    const int ti = i / CT, tj = j / CT;
    return W[P.woff + ((size_t)ti * (ti + 1) / 2 + tj) * CT * CT + (size_t)(i % CT) * CT + (j % CT)];
}

// G = L_US D of one front, 64 x 64 tile (I, J) per CTA: the sum over the
// tiles m >= J of L_US(I, m) D(m, J) (D lower triangular); G stored as row
// tiles nUt x nSt at Gw + goff.  grid (nUt * nSt max, fronts of the level)
__global__ void __launch_bounds__(256) nd_gprod_kernel(const NdPack* __restrict__ fp,
                                                       const int32_t* __restrict__ flist,
                                                       const double* __restrict__ fronts,
                                                       const double* __restrict__ W, double* Gw) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Bm = sm + CT * CLD;
    const NdPack P = fp[flist[blockIdx.y]];
    const int nUt = (P.nU + CT - 1) / CT;
    if ((int)blockIdx.x >= nUt * P.nSt) return;
    const int I = blockIdx.x / P.nSt, J = blockIdx.x % P.nSt;
    double acc[4][4];
    acc_zero4(acc);
    for (int m = J; m < P.nSt; ++m) {
        const int R = P.nSt + I;
        ct_load(A, fronts + P.foff + ((size_t)R * (R + 1) / 2 + m) * CT * CT);
        ct_load(Bm, W + P.woff + ((size_t)m * (m + 1) / 2 + J) * CT * CT);
        __syncthreads();
        ct_mac<false>(acc, A, Bm);
        __syncthreads();
    }
    const int r0 = (threadIdx.x >> 4) * 4, c0 = (threadIdx.x & 15) * 4;
    double* out = Gw + P.goff + ((size_t)I * P.nSt + J) * CT * CT;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) out[(r0 + a) * CT + c0 + b] = acc[a][b];
}

__device__ __forceinline__ double nd_g(const NdPack& P, const double* Gw, int u, int s) {
    return Gw[P.goff + ((size_t)(u / CT) * P.nSt + s / CT) * CT * CT + (size_t)(u % CT) * CT + (s % CT)];
}

// rows of D = L_SS^{-1} (kind 0), G (kind 1), D^T (kind 2) and G^T (kind 3)
// of one front per item
__global__ void nd_pack_kernel(const NdPack* __restrict__ fp, const int4* __restrict__ items,
                               const double* __restrict__ Gw, const double* __restrict__ W, double* out64,
                               float* out32) {
    const int4 it = items[blockIdx.x];   // (front, kind, row, unused)
    const NdPack P = fp[it.x];
    const int i = it.z;
    int64_t o0;
    int c0, len;
    if (it.y == 0) {
        o0 = P.doff + drow(i), c0 = 0, len = r4(i + 1);
    } else if (it.y == 1) {
        o0 = P.loff + (int64_t)i * r4(P.nS), c0 = 0, len = r4(P.nS);
    } else if (it.y == 2) {
        o0 = P.dtoff + dtrow(i, P.nS), c0 = i & ~3, len = r4(P.nS) - c0;
    } else {
        o0 = P.ltoff + (int64_t)i * r4(P.nU), c0 = 0, len = r4(P.nU);
    }
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int c = c0 + e;
        double v = 0.0;
        if (it.y == 0) v = c <= i ? nd_dinv(P, W, i, c) : 0.0;
        else if (it.y == 1) v = c < P.nS ? nd_g(P, Gw, i, c) : 0.0;
        else if (it.y == 2) v = (c >= i && c < P.nS) ? nd_dinv(P, W, c, i) : 0.0;
        else v = c < P.nU ? nd_g(P, Gw, c, i) : 0.0;
        if (out64) out64[o0 + e] = v;
        if (out32) out32[o0 + e] = (float)v;
    }
}

// ---- solve kernels (one launch per level and direction) on vectors in
// elimination order
struct NdSolve {
    const int32_t *nS, *nU, *s0, *up;
    const int64_t *uoff, *doff, *goff, *dtoff, *gtoff;
};

// a factor row into L2, one 128-byte line per thread and step (every line
// it names holds part of the row, so the address is valid); t is the
// thread's index among the nt threads that share the row
template <typename T>
__device__ __forceinline__ void nd_prefetch_row(const T* row, int len, int t, int nt) {
    if (len <= 0) return;
    const uintptr_t b = reinterpret_cast<uintptr_t>(row), e = b + (uintptr_t)len * sizeof(T);
    for (uintptr_t a = (b & ~(uintptr_t)127) + (uintptr_t)t * 128; a < e; a += (uintptr_t)nt * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// WPR warps share one item (levels near the root have long rows and few of
// them); the WPR warp sums are added in warp order through shared memory,
// so the result depends on WPR (fixed per level at setup) and nothing else
template <typename V, int WPR>
__device__ __forceinline__ bool nd_combine(V& s, V* part) {
    if (WPR == 1) return (threadIdx.x & 31) == 0;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) part[warp] = s;
    __syncthreads();
    if (warp % WPR != 0 || (threadIdx.x & 31) != 0) return false;
    V t = part[warp];
#pragma unroll
    for (int u = 1; u < WPR; ++u) t += part[warp + u];
    s = t;
    return true;
}

// forward, one item per WPR warps: (front f, row i) gives y[s0 + i] =
// D[i] . w_S; (-1 - k, 0) gives target k of the level: w[tgt_k] -= the sum,
// in a fixed order, of G_f[u] . w_{S_f} over the (front, row) pairs listed
// for it.  The factor rows do not depend on the previous level, so the
// warps prefetch them before they wait for that level (programmatic
// dependent launch); the vectors are read after the wait.
template <typename V, int WPR>
__global__ void __launch_bounds__(256) nd_fwd_kernel(NdSolve F, const int2* __restrict__ items, int n,
                                                     const int32_t* __restrict__ tgt, const int64_t* __restrict__ ptr,
                                                     const int2* __restrict__ src, const V* __restrict__ data, V* w,
                                                     V* y, int pf) {
    __shared__ V part[8];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int wi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) / WPR, lane = threadIdx.x & 31;
    const int t = ((threadIdx.x >> 5) % WPR) * 32 + lane;   // thread's index within its item
    if (WPR == 1 && wi >= n) return;   // reads nothing the previous level writes
    const bool live = wi < n;
    const int2 it = live ? items[wi] : make_int2(0, 0);
    V s = 0;
    int out = -1;
    if (it.x >= 0) {
        const int f = it.x, i = it.y;
        const V* row = data + F.doff[f] + drow(i);
        if (live && pf) nd_prefetch_row(row, i + 1, t, 32 * WPR);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const V* v = w + F.s0[f];
        if (live) {
#pragma unroll 4
            for (int j = t; j <= i; j += 32 * WPR) s = fma(row[j], v[j], s);
        }
        s = ddgdev::warp_sum(s);
        out = F.s0[f] + i;
    } else {
        const int k = -1 - it.x;
        const int64_t e0 = ptr[k], e1 = ptr[k + 1];
        for (int64_t e = e0; pf && e < e1; ++e) {
            const int2 fu = src[e];
            const int nS = F.nS[fu.x];
            nd_prefetch_row(data + F.goff[fu.x] + (int64_t)fu.y * r4(nS), nS, t, 32 * WPR);
        }
        asm volatile("griddepcontrol.wait;" ::: "memory");
        for (int64_t e = e0; e < e1; ++e) {
            const int2 fu = src[e];
            const int f = fu.x, nS = F.nS[f];
            const V* row = data + F.goff[f] + (int64_t)fu.y * r4(nS);
            const V* v = w + F.s0[f];
            V tt = 0;
#pragma unroll 4
            for (int j = t; j < nS; j += 32 * WPR) tt = fma(row[j], v[j], tt);
            s += ddgdev::warp_sum(tt);
        }
    }
    if (!nd_combine<V, WPR>(s, part) || !live) return;
    if (out >= 0) y[out] = s;
    else w[tgt[-1 - it.x]] -= s;
}

// backward, one item per WPR warps (front f, row s): x[s0 + s] = D^T[s] . y_S
// - G^T[s] . x_U (the factor rows and the U positions prefetched before the
// wait, as forward)
template <typename V, int WPR>
__global__ void __launch_bounds__(256) nd_bwd_kernel(NdSolve F, const int2* __restrict__ items, int n,
                                                     const V* __restrict__ data, const V* y, V* x, int pf) {
    __shared__ V part[8];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int wi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) / WPR, lane = threadIdx.x & 31;
    const int t = ((threadIdx.x >> 5) % WPR) * 32 + lane;
    if (WPR == 1 && wi >= n) return;   // reads nothing the previous level writes
    const bool live = wi < n;
    const int2 it = live ? items[wi] : make_int2(0, 0);
    const int f = it.x, r = it.y;
    const int nS = live ? F.nS[f] : 0, nU = live ? F.nU[f] : 0, s0 = F.s0[f];
    const int c0 = r & ~3;
    const V* drow_ = data + F.dtoff[f] + dtrow(r, nS);
    const V* grow = data + F.gtoff[f] + (int64_t)r * r4(nU);
    const int32_t* up = F.up + F.uoff[f];
    if (pf) {
        nd_prefetch_row(drow_, nS - c0, t, 32 * WPR);
        nd_prefetch_row(grow, nU, t, 32 * WPR);
        nd_prefetch_row(up, nU, t, 32 * WPR);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const V* vy = y + s0 + c0;
    V s = 0;
#pragma unroll 4
    for (int j = t; j < nS - c0; j += 32 * WPR) s = fma(drow_[j], vy[j], s);
#pragma unroll 4
    for (int j = t; j < nU; j += 32 * WPR) s = fma(-grow[j], x[up[j]], s);
    s = ddgdev::warp_sum(s);
    if (!nd_combine<V, WPR>(s, part) || !live) return;
    x[s0 + r] = s;
}

__device__ __forceinline__ uint64_t nd_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned nd_load_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct NdPersist {
    NdSolve F;
    const int2 *fitems, *bitems, *rsrc;
    const int32_t *rtgt, *elim, *fwd_off, *bwd_off;   // level offsets (device, [nlevel + 1])
    const int64_t* rptr;
    int n0, nlevel;
    unsigned* bar;      // grid barrier counter, zero at launch
    int* err;           // set when a barrier wait runs out
    uint64_t limit_ns;
};

// The whole ND solve in one cooperative launch: the permutation, the forward
// levels, the backward levels and the inverse permutation are phases of a
// grid-stride loop over the same items as the per-level kernels, separated
// by grid barriers (a monotone counter; every wait bounded by limit_ns).
// Vectors written in one phase and read in a later one are read through L2
// (__ldcg), never from a possibly stale L1 line.
template <typename V>
__global__ void __launch_bounds__(256, 4) nd_persistent_kernel(NdPersist P, const V* __restrict__ data, const V* c,
                                                            V* w, V* y, V* xp, V* xout) {
    const NdSolve& F = P.F;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * 8 + (threadIdx.x >> 5), nw = gridDim.x * 8;
    unsigned phase = 0;
    auto barrier = [&]() {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(P.bar, 1u);
            const unsigned target = (phase + 1) * gridDim.x;
            const uint64_t t0 = nd_ns();
            for (uint32_t i = 0;; ++i) {
                if (nd_load_acquire(P.bar) >= target) break;
                if ((i & 63) == 63 && nd_ns() - t0 > P.limit_ns) {
                    atomicExch(P.err, 1);
                    break;
                }
            }
            __threadfence();
        }
        __syncthreads();
        ++phase;
    };
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n0; p += gridDim.x * blockDim.x)
        w[p] = c[P.elim[p]];
    barrier();
    for (int l = 0; l < P.nlevel; ++l) {
        const int a0 = P.fwd_off[l], a1 = P.fwd_off[l + 1];
        for (int wi = a0 + gw; wi < a1; wi += nw) {
            const int2 it = P.fitems[wi];
            if (it.x >= 0) {
                const int f = it.x, i = it.y;
                const V* row = data + F.doff[f] + drow(i);
                const V* v = w + F.s0[f];
                V s = 0;
#pragma unroll 4
                for (int j = lane; j <= i; j += 32) s = fma(row[j], __ldcg(v + j), s);
                s = ddgdev::warp_sum(s);
                if (lane == 0) y[F.s0[f] + i] = s;
            } else {
                const int k = -1 - it.x;
                V s = 0;
                for (int64_t e = P.rptr[k]; e < P.rptr[k + 1]; ++e) {
                    const int2 fu = P.rsrc[e];
                    const int f = fu.x, nS = F.nS[f];
                    const V* row = data + F.goff[f] + (int64_t)fu.y * r4(nS);
                    const V* v = w + F.s0[f];
                    V t = 0;
#pragma unroll 4
                    for (int j = lane; j < nS; j += 32) t = fma(row[j], __ldcg(v + j), t);
                    s += ddgdev::warp_sum(t);
                }
                if (lane == 0) w[P.rtgt[k]] = __ldcg(w + P.rtgt[k]) - s;
            }
        }
        barrier();
    }
    for (int l = P.nlevel - 1; l >= 0; --l) {
        const int a0 = P.bwd_off[l], a1 = P.bwd_off[l + 1];
        for (int wi = a0 + gw; wi < a1; wi += nw) {
            const int2 it = P.bitems[wi];
            const int f = it.x, r = it.y;
            const int nS = F.nS[f], nU = F.nU[f], s0 = F.s0[f];
            const int c0 = r & ~3;
            const V* drow_ = data + F.dtoff[f] + dtrow(r, nS);
            const V* vy = y + s0 + c0;
            V s = 0;
#pragma unroll 4
            for (int j = lane; j < nS - c0; j += 32) s = fma(drow_[j], __ldcg(vy + j), s);
            const V* grow = data + F.gtoff[f] + (int64_t)r * r4(nU);
            const int32_t* up = F.up + F.uoff[f];
#pragma unroll 4
            for (int j = lane; j < nU; j += 32) s = fma(-grow[j], __ldcg(xp + up[j]), s);
            s = ddgdev::warp_sum(s);
            if (lane == 0) xp[s0 + r] = s;
        }
        barrier();
    }
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n0; p += gridDim.x * blockDim.x)
        xout[P.elim[p]] = __ldcg(xp + p);
}

// ---- the same solve for m right-hand sides (FP32, dof-major n0 x m,
// m <= 64).  Every front product is a small dense matrix product with m
// columns, so a CTA takes a 32-row tile of one front's D, G, D^T or G^T and
// runs over K in 64-wide stages (A stage 32 x 64, vector stage 64 x m)
// copied into shared memory with cp.async, two stages in flight; each
// thread keeps 2 rows x 4 adjacent columns.  Where a level has few tiles, a
// cluster of KS CTAs splits each tile's stages and CTA 0 of the cluster sums
// the partial tiles from the others' shared memory in rank order.  The
// forward G products of a level go to per-front partial rows P (nU x m per
// front), which a second launch sums in the same fixed order as the
// one-column solve and subtracts from their targets.
static_assert(DDG_MCHUNK <= 64, "the multi-column ND tiles hold at most 64 columns");
constexpr int NDT = 32;                                 // rows per tile
constexpr int NDK = 64;                                 // K per stage
constexpr int ND_LDA = NDK + 4;                         // A stage row stride (16-byte rows)
constexpr int ND_AS = NDT * ND_LDA;
constexpr int ND_STAGE = ND_AS + NDK * 64;              // floats per stage
constexpr size_t ND_TILE_SMEM = 2 * ND_STAGE * sizeof(float);
constexpr int ND_MAX_KS = 8;                            // CTAs per cluster (portable limit)

struct NdTileAcc {
    float a[2][4];
};

// asynchronous copies global -> shared; a null source fills zeros
__device__ __forceinline__ void nd_cp16(float* dst, const float* src, const float* dummy) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src ? src : dummy),
                 "r"(src ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void nd_cp4(float* dst, const float* src, const float* dummy) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src ? src : dummy), "r"(src ? 4 : 0)
                 : "memory");
}

// acc += A[., k] B[k, :] over the stages [st0, st1) of the K range starting
// at kbeg (stage t covers kbeg + t NDK .. + NDK, cut at kend).
// aptr(rr, c): address of the 4 entries A(r0 + rr, c .. c + 3) (c a
// multiple of 4; rows are stored zero-padded to multiples of 4) or null for
// zeros; brow(k): row k of B (m floats, 16-byte aligned when m % 4 == 0).
template <class AP, class BR>
__device__ __forceinline__ void nd_tile_run(int kbeg, int kend, int st0, int st1, int m, AP aptr, BR brow,
                                            float* smem, const float* dummy, NdTileAcc& acc) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool vec = (m & 3) == 0;
    auto issue = [&](int buf, int k0) {
        float* As = smem + buf * ND_STAGE;
        float* Bs = As + ND_AS;
        for (int e = tid; e < NDT * NDK / 4; e += 256) {
            const int rr = e / (NDK / 4), c = k0 + 4 * (e - rr * (NDK / 4));
            nd_cp16(As + rr * ND_LDA + (c - k0), c < kend ? aptr(rr, c) : nullptr, dummy);
        }
        if (vec) {
            const int m4 = m >> 2;
            for (int e = tid; e < NDK * m4; e += 256) {
                const int kk = e / m4, col = 4 * (e - kk * m4), k = k0 + kk;
                nd_cp16(Bs + kk * 64 + col, k < kend ? brow(k) + col : nullptr, dummy);
            }
        } else {
            for (int e = tid; e < NDK * m; e += 256) {
                const int kk = e / m, col = e - kk * m, k = k0 + kk;
                nd_cp4(Bs + kk * 64 + col, k < kend ? brow(k) + col : nullptr, dummy);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (st1 > st0) issue(st0 & 1, kbeg + st0 * NDK);
    for (int st = st0; st < st1; ++st) {
        if (st + 1 < st1) {
            issue((st + 1) & 1, kbeg + (st + 1) * NDK);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float* As = smem + (st & 1) * ND_STAGE;
        const float* Bs = As + ND_AS;
#pragma unroll 4
        for (int kk = 0; kk < NDK; kk += 4) {
            const float4 a0 = *reinterpret_cast<const float4*>(As + ty * ND_LDA + kk);
            const float4 a1 = *reinterpret_cast<const float4*>(As + (ty + 16) * ND_LDA + kk);
            const float av0[4] = {a0.x, a0.y, a0.z, a0.w}, av1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 b = *reinterpret_cast<const float4*>(Bs + (kk + q) * 64 + 4 * tx);
                const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc.a[0][j] = fmaf(av0[q], bv[j], acc.a[0][j]);
                    acc.a[1][j] = fmaf(av1[q], bv[j], acc.a[1][j]);
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned nd_cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned nd_cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void nd_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float nd_ld_remote(const float* local, unsigned rank) {
    unsigned a = (unsigned)__cvta_generic_to_shared(local), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(r) : "memory");
    return v;
}

// the stages [st0, st1) of n that cluster CTA q of ks takes
__device__ __forceinline__ void nd_split(int n, int q, int ks, int& st0, int& st1) {
    const int per = (n + ks - 1) / ks;
    st0 = min(n, q * per);
    st1 = min(n, st0 + per);
}

// sums the cluster's partial tiles into CTA 0 (rank order); returns false
// on the other CTAs, which then have nothing to store
__device__ __forceinline__ bool nd_cluster_reduce(NdTileAcc* t, int nt, float* smem) {
    const unsigned ks = nd_cluster_size();
    if (ks == 1) return true;
    const unsigned q = nd_cluster_rank();
    const int tid = threadIdx.x;
    for (int u = 0; u < nt; ++u)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) smem[(u * 8 + i * 4 + j) * 256 + tid] = t[u].a[i][j];
    nd_cluster_sync();
    if (q == 0) {
        for (unsigned p = 1; p < ks; ++p)
            for (int u = 0; u < nt; ++u)
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) t[u].a[i][j] += nd_ld_remote(smem + (u * 8 + i * 4 + j) * 256 + tid, p);
    }
    nd_cluster_sync();   // the other CTAs keep their shared memory until CTA 0 has read it
    return q == 0;
}

__device__ __forceinline__ void nd_store_tile(const NdTileAcc& acc, const NdTileAcc* sub, float* out, int r0,
                                              int nrow, int m) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= nrow) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * tx + j;
            if (c < m) out[(int64_t)r * m + c] = sub ? acc.a[i][j] - sub->a[i][j] : acc.a[i][j];
        }
    }
}

// forward tile (f, r0, kind): kind 0 gives rows r0.. of y_S = D w_S, kind 1
// rows r0.. of the partial product P_f = G_f w_S; a cluster of KS CTAs per
// tile (grid = tiles x KS)
__global__ void __launch_bounds__(256) nd_fwd_tile_kernel(NdSolve F, const int4* __restrict__ items,
                                                          const float* __restrict__ data, const float* w, float* y,
                                                          float* P, int m) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) float nd_smem[];
    const int ks = (int)nd_cluster_size();
    const int4 it = items[blockIdx.x / ks];
    const int f = it.x, r0 = it.y, kind = it.z;
    const int nS = F.nS[f], s0 = F.s0[f];
    const int nrow = kind == 0 ? nS : F.nU[f];
    const int kend = kind == 0 ? min(r0 + NDT, nS) : nS;
    const float* base = data + (kind == 0 ? F.doff[f] : F.goff[f]);
    const float* W = w + (int64_t)s0 * m;
    const int ld = r4(nS);
    auto aptr = [&](int rr, int c) -> const float* {
        const int r = r0 + rr;
        if (kind == 0) return (r < nS && c <= r) ? base + drow(r) + c : nullptr;
        return r < nrow ? base + (int64_t)r * ld + c : nullptr;
    };
    auto brow = [&](int k) { return W + (int64_t)k * m; };
    NdTileAcc acc = {};
    int st0, st1;
    nd_split((kend + NDK - 1) / NDK, (int)nd_cluster_rank(), ks, st0, st1);
    {
        // the CTA's factor rows (fixed at setup) into L2 before waiting for
        // the previous level: 8 threads per row
        const int r = r0 + (threadIdx.x >> 3), t8 = threadIdx.x & 7;
        const int c_lo = st0 * NDK, c_hi = min(kend, st1 * NDK);
        if (r < nrow && c_hi > c_lo) {
            if (kind == 0) {
                const int ce = min(c_hi, r + 1);
                if (ce > c_lo) nd_prefetch_row(base + drow(r) + c_lo, ce - c_lo, t8, 8);
            } else {
                nd_prefetch_row(base + (int64_t)r * ld + c_lo, c_hi - c_lo, t8, 8);
            }
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    nd_tile_run(0, kend, st0, st1, m, aptr, brow, nd_smem, data, acc);
    if (!nd_cluster_reduce(&acc, 1, nd_smem)) return;
    float* out = kind == 0 ? y + (int64_t)s0 * m : P + F.uoff[f] * m;
    nd_store_tile(acc, nullptr, out, r0, nrow, m);
}

// one warp per target k of the level: w[tgt_k] -= the sum over its partial
// rows, in the listed order
__global__ void __launch_bounds__(256) nd_fwd_reduce_kernel(const int32_t* __restrict__ tgt,
                                                            const int64_t* __restrict__ ptr,
                                                            const int64_t* __restrict__ srcp, int t0, int nt,
                                                            const float* __restrict__ P, float* w, int m) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int wi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (wi >= nt) return;
    const int k = t0 + wi;
    float acc[2] = {0.f, 0.f};
    for (int64_t e = ptr[k]; e < ptr[k + 1]; ++e) {
        const float* p = P + srcp[e] * m;
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (lane + 32 * u < m) acc[u] += p[lane + 32 * u];
    }
    float* out = w + (int64_t)tgt[k] * m;
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (lane + 32 * u < m) out[lane + 32 * u] -= acc[u];
}

// backward tile (f, r0): rows r0.. of x_S = D^T y_S - G^T x_U (x_U gathered
// from the ancestors' rows, already solved); the D^T and G^T stages form
// one sequence that a cluster of KS CTAs splits
__global__ void __launch_bounds__(256) nd_bwd_tile_kernel(NdSolve F, const int2* __restrict__ items,
                                                          const float* __restrict__ data, const float* y, float* x,
                                                          int m) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) float nd_smem[];
    const int ks = (int)nd_cluster_size();
    const int2 it = items[blockIdx.x / ks];
    const int f = it.x, r0 = it.y;
    const int nS = F.nS[f], nU = F.nU[f], s0 = F.s0[f];
    const float* dt = data + F.dtoff[f];
    const float* gt = data + F.gtoff[f];
    const int32_t* up = F.up + F.uoff[f];
    const int ldu = r4(nU);
    NdTileAcc t[2] = {};   // D^T y_S and G^T x_U
    const int n1 = (nS - r0 + NDK - 1) / NDK, n2 = (nU + NDK - 1) / NDK;
    int a, b;
    nd_split(n1 + n2, (int)nd_cluster_rank(), ks, a, b);
    {
        // the CTA's D^T and G^T row segments (fixed at setup) into L2 before
        // waiting for the level above: 8 threads per row
        const int r = r0 + (threadIdx.x >> 3), t8 = threadIdx.x & 7;
        if (r < nS) {
            const int p1s = min(a, n1), p1e = min(b, n1);
            const int lo1 = max(r0 + p1s * NDK, r & ~3), hi1 = min(nS, r0 + p1e * NDK);
            if (hi1 > lo1) nd_prefetch_row(dt + dtrow(r, nS) + (lo1 - (r & ~3)), hi1 - lo1, t8, 8);
            const int p2s = max(a, n1) - n1, p2e = max(b, n1) - n1;
            const int lo2 = p2s * NDK, hi2 = min(nU, p2e * NDK);
            if (hi2 > lo2) nd_prefetch_row(gt + (int64_t)r * ldu + lo2, hi2 - lo2, t8, 8);
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    auto dptr = [&](int rr, int c) -> const float* {
        const int r = r0 + rr;
        return (r < nS && c >= (r & ~3)) ? dt + dtrow(r, nS) + (c - (r & ~3)) : nullptr;
    };
    auto yrow = [&](int k) { return y + (int64_t)(s0 + k) * m; };
    nd_tile_run(r0, nS, min(a, n1), min(b, n1), m, dptr, yrow, nd_smem, data, t[0]);
    auto gptr = [&](int rr, int c) -> const float* {
        const int r = r0 + rr;
        return r < nS ? gt + (int64_t)r * ldu + c : nullptr;
    };
    auto xrow = [&](int k) { return x + (int64_t)up[k] * m; };
    nd_tile_run(0, nU, max(a, n1) - n1, max(b, n1) - n1, m, gptr, xrow, nd_smem, data, t[1]);
    if (!nd_cluster_reduce(t, 2, nd_smem)) return;
    nd_store_tile(t[0], &t[1], x + (int64_t)s0 * m, r0, nS, m);
}

template <bool GATHER>
__global__ void nd_permute_multi_kernel(int64_t total, int m, const int32_t* __restrict__ idx, const float* src,
                                        float* dst) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t p = e / m, c = e - p * m;
    if (GATHER) dst[e] = src[(int64_t)idx[p] * m + c];
    else dst[(int64_t)idx[p] * m + c] = src[e];
}

// dst[p] = src[idx[p]] (into elimination order), or dst[idx[p]] = src[p] (back)
template <typename V, bool GATHER>
__global__ void nd_permute_kernel(int n, const int32_t* __restrict__ idx, const V* src, V* dst) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (GATHER) dst[p] = src[idx[p]];
    else dst[idx[p]] = src[p];
}

// ---- host symbolic analysis
struct FrontH {
    std::vector<int> S, U;
    int child[2] = {-1, -1};
    int nchild = 0, parent = -1, depth = 0;
};

struct NdBuilder {
    const std::vector<std::vector<int>>& adj;
    const std::vector<int>& rank;
    std::vector<FrontH> fronts;
    std::vector<int> stamp, level;
    int cur = 0;
    NdBuilder(const std::vector<std::vector<int>>& a, const std::vector<int>& r)
        : adj(a), rank(r), stamp(a.size(), -1), level(a.size(), -1) {}

    // BFS levels inside the set marked with `cur`; returns the visit order
    std::vector<int> bfs(int start) {
        std::vector<int> order{start};
        level[start] = 0;
        std::vector<int> seen{start};
        for (size_t h = 0; h < order.size(); ++h) {
            const int u = order[h];
            for (int w : adj[u])
                if (stamp[w] == cur && level[w] < 0) {
                    level[w] = level[u] + 1;
                    order.push_back(w);
                }
        }
        return order;
    }
    void clear_levels(const std::vector<int>& order) {
        for (int v : order) level[v] = -1;
    }

    int leaf(const std::vector<int>& nodes) {
        FrontH f;
        f.S = nodes;
        std::sort(f.S.begin(), f.S.end());
        fronts.push_back(f);
        return (int)fronts.size() - 1;
    }

    int build(std::vector<int> nodes) {
        int64_t weight = 0;
        for (int v : nodes) weight += rank[v];
        if (weight <= ND_LEAF_DOFS || nodes.size() <= 2) return leaf(nodes);
        const int mark = ++cur;
        for (int v : nodes) stamp[v] = mark;
        // pseudo-peripheral start: two sweeps to the farthest node
        int start = *std::min_element(nodes.begin(), nodes.end());
        for (int sweep = 0; sweep < 2; ++sweep) {
            std::vector<int> order = bfs(start);
            int far = start;
            for (int v : order)
                if (level[v] > level[far] || (level[v] == level[far] && v < far)) far = v;
            clear_levels(order);
            start = far;
        }
        std::vector<int> order = bfs(start);
        int maxl = 0;
        int64_t reached = 0;
        for (int v : order) {
            maxl = std::max(maxl, level[v]);
            reached += rank[v];
        }
        std::vector<int64_t> wl(maxl + 1, 0);
        for (int v : order) wl[level[v]] += rank[v];
        int k = 0;
        int64_t cum = 0;
        for (int l = 0; l <= maxl; ++l) {
            cum += wl[l];
            if (2 * cum >= reached) {
                k = l;
                break;
            }
        }
        if (k == 0 && maxl >= 1) k = 1;
        std::vector<int> S, V1, V2;
        for (int v : nodes) {
            const int l = level[v];
            if (l == k) S.push_back(v);
            else if (l >= 0 && l < k) V1.push_back(v);
            else V2.push_back(v);
        }
        clear_levels(order);
        for (int v : nodes) stamp[v] = -1;
        if (V1.empty() || V2.empty() || S.empty()) return leaf(nodes);
        const int c1 = build(V1);
        const int c2 = build(V2);
        FrontH f;
        f.S = S;
        std::sort(f.S.begin(), f.S.end());
        f.child[0] = c1;
        f.child[1] = c2;
        f.nchild = 2;
        fronts.push_back(f);
        const int id = (int)fronts.size() - 1;
        fronts[c1].parent = id;
        fronts[c2].parent = id;
        return id;
    }
};

template <typename T>
T* upload(ddg_handle h, const std::vector<T>& v) {
    T* d = h->arena.alloc<T>(v.size());
    h2d(d, v.data(), v.size(), h->stream);
    return d;
}

}  // namespace

namespace ddg {

// Symbolic analysis and numeric factorisation of the nested-dissection
// coarse factor; pairs bI >= bJ are the subdomain pairs that A0 couples
// (both with coarse dofs), blocks (device) their kmax x kmax blocks of A0.
void nd_coarse_setup(ddg_handle h, const std::vector<int>& bI, const std::vector<int>& bJ, const double* blocks) {
    NdCoarse& N = h->nd;
    const int nsub = h->nsub, kmax = h->kmax;
    const std::vector<int>& coff = h->h_coff;
    std::vector<int> rank(nsub);
    for (int v = 0; v < nsub; ++v) rank[v] = coff[v + 1] - coff[v];
    std::vector<std::vector<int>> adj(nsub);
    for (size_t p = 0; p < bI.size(); ++p)
        if (bI[p] != bJ[p]) {
            adj[bI[p]].push_back(bJ[p]);
            adj[bJ[p]].push_back(bI[p]);
        }
    std::vector<int> nodes;
    for (int v = 0; v < nsub; ++v)
        if (rank[v] > 0) nodes.push_back(v);
    NdBuilder nb(adj, rank);
    nb.build(nodes);
    std::vector<FrontH>& fr = nb.fronts;
    const int nf = (int)fr.size();
    // postorder = creation order; the root is the last front
    std::vector<int> fof(nsub, -1), eidx(nsub, -1);
    {
        int e = 0;
        for (int f = 0; f < nf; ++f)
            for (int v : fr[f].S) {
                fof[v] = f;
                eidx[v] = e++;
            }
    }
    int nlevel = 1;
    for (int f = nf - 1; f >= 0; --f) {
        if (fr[f].parent >= 0) fr[f].depth = fr[fr[f].parent].depth + 1;
        nlevel = std::max(nlevel, fr[f].depth + 1);
    }
    // U_f: subdomains of ancestors coupled to the subtree of f, in elimination order
    {
        std::vector<int> mark(nsub, -1);
        for (int f = 0; f < nf; ++f) {
            std::vector<int>& U = fr[f].U;
            auto take = [&](int w) {
                if (fof[w] > f && mark[w] != f) {
                    mark[w] = f;
                    U.push_back(w);
                }
            };
            for (int v : fr[f].S)
                for (int w : adj[v]) take(w);
            for (int c = 0; c < fr[f].nchild; ++c)
                for (int w : fr[fr[f].child[c]].U) take(w);
            std::sort(U.begin(), U.end(), [&](int a, int b) { return eidx[a] < eidx[b]; });
        }
    }
    // per front: dof counts, tiles, positions of its subdomains
    std::vector<int> nS(nf), nU(nf), nSt(nf), NT(nf);
    std::vector<std::unordered_map<int, int>> pos(nf);
    std::vector<int64_t> foff(nf + 1, 0), doff(nf + 1, 0), woff(nf + 1, 0);
    for (int f = 0; f < nf; ++f) {
        int a = 0;
        for (int v : fr[f].S) {
            pos[f][v] = a;
            a += rank[v];
        }
        nS[f] = a;
        nSt[f] = std::max(1, (a + CT - 1) / CT);
        int b = 0;
        for (int v : fr[f].U) {
            pos[f][v] = nSt[f] * CT + b;
            b += rank[v];
        }
        nU[f] = b;
        NT[f] = nSt[f] + (b + CT - 1) / CT;
        foff[f + 1] = foff[f] + (int64_t)NT[f] * (NT[f] + 1) / 2 * CT * CT;
        doff[f + 1] = doff[f] + (int64_t)nSt[f] * CT * CT;
        woff[f + 1] = woff[f] + (int64_t)nSt[f] * (nSt[f] + 1) / 2 * CT * CT;
    }
    N.nfront = nf;
    N.nlevel = nlevel;
    // placement of the original blocks: the front of the earlier-eliminated subdomain
    std::vector<NdPlace> place(bI.size());
    for (size_t p = 0; p < bI.size(); ++p) {
        const int I = bI[p], J = bJ[p];
        const bool i_later = eidx[I] >= eidx[J];
        const int L = i_later ? I : J, E = i_later ? J : I;
        const int f = fof[E];
        NdPlace P;
        P.foff = foff[f];
        P.blk = (int64_t)p * kmax * kmax;
        P.rpos = pos[f].at(L);
        P.cpos = pos[f].at(E);
        P.kr = rank[L];
        P.kc = rank[E];
        P.trans = (I != J && L == J) ? 1 : 0;
        P.diag = I == J ? 1 : 0;
        place[p] = P;
    }
    std::vector<int4> pads(nf);
    for (int f = 0; f < nf; ++f)
        pads[f] = make_int4(nS[f], nSt[f] * CT, nSt[f] * CT + nU[f], NT[f] * CT);
    // extend-add maps: child update row a -> parent front position
    std::vector<int32_t> maps;
    std::vector<NdChild> childs(nf);
    for (int c = 0; c < nf; ++c) {
        const int f = fr[c].parent;
        NdChild C{};
        C.cfoff = foff[c];
        C.cbase = nSt[c] * CT;
        C.map_off = (int64_t)maps.size();
        C.pfoff = f >= 0 ? foff[f] : 0;
        if (f >= 0)
            for (int w : fr[c].U)
                for (int t = 0; t < rank[w]; ++t) maps.push_back(pos[f].at(w) + t);
        childs[c] = C;
    }
    // solve layout, in elimination order: front f's S dofs are the positions
    // s0[f] .. s0[f] + nS[f]; per front the rows of D, G, D^T and G^T
    std::vector<int32_t> s0(nf, 0), upos, elim(h->n0, 0), pos_of(h->n0, 0);
    std::vector<int64_t> sdoff(nf + 1, 0), sgoff(nf + 1, 0), stoff(nf + 1, 0), sgtoff(nf + 1, 0), uoff(nf + 1, 0);
    {
        int p = 0;
        for (int f = 0; f < nf; ++f) {
            s0[f] = p;
            for (int v : fr[f].S)
                for (int t = 0; t < rank[v]; ++t) {
                    elim[p] = coff[v] + t;
                    pos_of[coff[v] + t] = p;
                    ++p;
                }
        }
    }
    int64_t cur = 0;
    for (int f = 0; f < nf; ++f) {
        sdoff[f] = cur;
        cur += drow(nS[f]);
        sgoff[f] = cur;
        cur += (int64_t)nU[f] * r4(nS[f]);
        stoff[f] = cur;
        cur += dtrow(nS[f], nS[f]);
        sgtoff[f] = cur;
        cur += (int64_t)nS[f] * r4(nU[f]);
        for (int v : fr[f].U)
            for (int t = 0; t < rank[v]; ++t) upos.push_back(pos_of[coff[v] + t]);
        uoff[f + 1] = (int64_t)upos.size();
    }
    N.elems = cur;
    // fronts by level, deepest first (the forward order); per level the
    // forward items (the fronts' D rows, then one item per target of G w_S)
    // and the backward items (the fronts' rows)
    std::vector<std::vector<int>> bylevel(nlevel);
    for (int f = 0; f < nf; ++f) bylevel[nlevel - 1 - fr[f].depth].push_back(f);
    std::vector<int2> fitems, bitems, rsrc, mbitems;
    std::vector<int4> mfitems;
    std::vector<int32_t> rtgt;
    std::vector<int64_t> rptr{0}, rsrcp;
    N.h_fwd_off.assign(nlevel + 1, 0);
    N.h_bwd_off.assign(nlevel + 1, 0);
    N.h_mf_off.assign(nlevel + 1, 0);
    N.h_mb_off.assign(nlevel + 1, 0);
    N.h_tgt_off.assign(nlevel + 1, 0);
    for (int l = 0; l < nlevel; ++l) {
        std::unordered_map<int, std::vector<int2>> contrib;
        std::vector<int> order;
        for (int f : bylevel[l]) {
            for (int i = 0; i < nS[f]; ++i) {
                fitems.push_back(make_int2(f, i));
                bitems.push_back(make_int2(f, i));
            }
            // multi-column tiles of 32 rows: D and G forward, D^T / G^T backward
            for (int i = 0; i < nS[f]; i += NDT) {
                mfitems.push_back(make_int4(f, i, 0, 0));
                mbitems.push_back(make_int2(f, i));
            }
            for (int u = 0; u < nU[f]; u += NDT) mfitems.push_back(make_int4(f, u, 1, 0));
            for (int u = 0; u < nU[f]; ++u) {
                const int t = upos[uoff[f] + u];
                auto it = contrib.find(t);
                if (it == contrib.end()) {
                    order.push_back(t);
                    contrib[t] = {make_int2(f, u)};
                } else {
                    it->second.push_back(make_int2(f, u));
                }
            }
        }
        std::sort(order.begin(), order.end());
        for (int t : order) {
            fitems.push_back(make_int2(-1 - (int)rtgt.size(), 0));
            rtgt.push_back(t);
            for (const int2& e : contrib[t]) {
                rsrc.push_back(e);
                rsrcp.push_back(uoff[e.x] + e.y);
            }
            rptr.push_back((int64_t)rsrc.size());
        }
        N.h_fwd_off[l + 1] = (int)fitems.size();
        N.h_bwd_off[l + 1] = (int)bitems.size();
        N.h_mf_off[l + 1] = (int)mfitems.size();
        N.h_mb_off[l + 1] = (int)mbitems.size();
        N.h_tgt_off[l + 1] = (int)rtgt.size();
    }
    N.urows = uoff[nf];
    // warps per item of the single-vector solve, per level and direction:
    // the largest of 1, 2, 4, 8 that leaves every lane at least 4 entries of
    // the level's mean row and keeps the level within one wave of warps
    {
        int dev = 0, sms = 0;
        DDG_CUDA(cudaGetDevice(&dev));
        DDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        auto pick = [&](int64_t items, double mean_len) {
            int wpr = 1;
            while (wpr < 8 && mean_len >= 32.0 * 4 * (2 * wpr) && items * 2 * wpr <= (int64_t)sms * 64) wpr *= 2;
            return wpr;
        };
        N.h_fwd_wpr.assign(nlevel, 1);
        N.h_bwd_wpr.assign(nlevel, 1);
        N.h_fwd_pf.assign(nlevel, 1);
        N.h_bwd_pf.assign(nlevel, 1);
        for (int l = 0; l < nlevel; ++l) {
            double fl = 0.0, bl = 0.0;
            for (int e = N.h_fwd_off[l]; e < N.h_fwd_off[l + 1]; ++e) {
                const int2 it = fitems[e];
                if (it.x >= 0) {
                    fl += it.y + 1;
                } else {
                    const int k = -1 - it.x;
                    for (int64_t q = rptr[k]; q < rptr[k + 1]; ++q) fl += nS[rsrc[q].x];
                }
            }
            for (int e = N.h_bwd_off[l]; e < N.h_bwd_off[l + 1]; ++e) {
                const int2 it = bitems[e];
                bl += (nS[it.x] - (it.y & ~3)) + nU[it.x];
            }
            const int64_t nfi = N.h_fwd_off[l + 1] - N.h_fwd_off[l], nbi = N.h_bwd_off[l + 1] - N.h_bwd_off[l];
            if (nfi > 0) N.h_fwd_wpr[l] = pick(nfi, fl / nfi);
            if (nbi > 0) N.h_bwd_wpr[l] = pick(nbi, bl / nbi);
            // prefetch a level's factor rows only while they fit well inside
            // L2 (12 M elements: 48 MB in FP32, 96 MB in FP64); larger levels
            // would evict their own prefetched lines before use
            N.h_fwd_pf[l] = fl <= 12e6 ? 1 : 0;
            N.h_bwd_pf[l] = bl <= 12e6 ? 1 : 0;
        }
    }
    // cluster size per level of the multi-column solve: split the stages of
    // each tile over up to 8 CTAs while the level has fewer tiles than four
    // per SM (the CTAs of a cluster take at most the tile's stage count)
    {
        int dev = 0, sms = 0;
        DDG_CUDA(cudaGetDevice(&dev));
        DDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        auto pick = [&](int ntiles, int maxst) {
            int ks = 1;
            while (ks * 2 <= ND_MAX_KS && ks * 2 <= maxst && ntiles * ks * 2 <= 4 * sms) ks *= 2;
            return ks;
        };
        N.h_mf_ks.assign(nlevel, 1);
        N.h_mb_ks.assign(nlevel, 1);
        for (int l = 0; l < nlevel; ++l) {
            int mf = 0, mb = 0;
            for (int e = N.h_mf_off[l]; e < N.h_mf_off[l + 1]; ++e) {
                const int4 t = mfitems[e];
                const int kend = t.z == 0 ? std::min(t.y + NDT, nS[t.x]) : nS[t.x];
                mf = std::max(mf, (kend + NDK - 1) / NDK);
            }
            for (int e = N.h_mb_off[l]; e < N.h_mb_off[l + 1]; ++e) {
                const int2 t = mbitems[e];
                mb = std::max(mb, (nS[t.x] - t.y + NDK - 1) / NDK + (nU[t.x] + NDK - 1) / NDK);
            }
            N.h_mf_ks[l] = pick(N.h_mf_off[l + 1] - N.h_mf_off[l], mf);
            N.h_mb_ks[l] = pick(N.h_mb_off[l + 1] - N.h_mb_off[l], mb);
        }
    }
    // device copies of the solve layout
    N.nS = upload(h, nS);
    N.nU = upload(h, nU);
    N.s0 = upload(h, s0);
    N.up = upload(h, upos.empty() ? std::vector<int32_t>{0} : upos);
    N.uoff = upload(h, uoff);
    N.doff = upload(h, sdoff);
    N.goff = upload(h, sgoff);
    N.dtoff = upload(h, stoff);
    N.gtoff = upload(h, sgtoff);
    N.elim = upload(h, elim.empty() ? std::vector<int32_t>{0} : elim);
    N.fitems = upload(h, fitems.empty() ? std::vector<int2>{make_int2(0, 0)} : fitems);
    N.bitems = upload(h, bitems.empty() ? std::vector<int2>{make_int2(0, 0)} : bitems);
    N.rtgt = upload(h, rtgt.empty() ? std::vector<int32_t>{0} : rtgt);
    N.rptr = upload(h, rptr);
    N.rsrc = upload(h, rsrc.empty() ? std::vector<int2>{make_int2(0, 0)} : rsrc);
    N.rsrcp = upload(h, rsrcp.empty() ? std::vector<int64_t>{0} : rsrcp);
    N.mfitems = upload(h, mfitems.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : mfitems);
    N.mbitems = upload(h, mbitems.empty() ? std::vector<int2>{make_int2(0, 0)} : mbitems);
    N.fwd_off = upload(h, N.h_fwd_off);
    N.bwd_off = upload(h, N.h_bwd_off);
    N.bar = h->arena.alloc<unsigned>(1);
    N.d64 = h->arena.alloc<double>(N.elems);
    N.d32 = h->arena.alloc<float>(N.elems);
    N.w64 = h->arena.alloc<double>(std::max(1, h->n0));
    N.w32 = h->arena.alloc<float>(std::max(1, h->n0));
    N.x64 = h->arena.alloc<double>(std::max(1, h->n0));
    N.x32 = h->arena.alloc<float>(std::max(1, h->n0));

    // ---- numeric factorisation (FP64 workspaces, released at the end)
    std::vector<int64_t> gwoff(nf + 1, 0);
    for (int f = 0; f < nf; ++f)
        gwoff[f + 1] = gwoff[f] + (int64_t)((nU[f] + CT - 1) / CT) * nSt[f] * CT * CT;
    double* fronts = h->arena.alloc<double>(foff[nf]);
    double* dinv = h->arena.alloc<double>(doff[nf]);
    double* W = h->arena.alloc<double>(woff[nf]);
    double* Gw = h->arena.alloc<double>(std::max<int64_t>(1, gwoff[nf]));
    DDG_CUDA(cudaMemsetAsync(fronts, 0, foff[nf] * sizeof(double), h->stream));
    DDG_CUDA(cudaMemsetAsync(W, 0, woff[nf] * sizeof(double), h->stream));
    std::vector<void*> tmp;
    auto up = [&](auto v) {
        auto* d = upload(h, v);
        tmp.push_back((void*)d);
        return d;
    };
    if (!place.empty()) {
        NdPlace* dpl = up(place);
        nd_scatter_kernel<<<(unsigned)place.size(), 128, 0, h->stream>>>(dpl, blocks, kmax, fronts);
        DDG_CHECK_LAUNCH();
    }
    {
        int64_t* dfo = up(std::vector<int64_t>(foff.begin(), foff.end() - 1));
        int4* dpads = up(pads);
        nd_pad_kernel<<<nf, 128, 0, h->stream>>>(dfo, dpads, fronts);
        DDG_CHECK_LAUNCH();
    }
    std::vector<NdPack> packs(nf);
    for (int f = 0; f < nf; ++f)
        packs[f] = NdPack{foff[f], woff[f], gwoff[f], sdoff[f], sgoff[f], stoff[f], sgtoff[f], nS[f], nU[f], nSt[f]};
    NdChild* dch = upload(h, childs);
    int32_t* dmaps = upload(h, maps.empty() ? std::vector<int32_t>{0} : maps);
    NdPack* dpk = upload(h, packs);
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    for (void* p : tmp) h->arena.release(p);
    tmp.clear();
    for (int l = 0; l < nlevel; ++l) {
        const std::vector<int>& fl = bylevel[l];
        // children's update matrices into the fronts of this level, first
        // children then second children (one writer per parent entry)
        for (int slot = 0; slot < 2; ++slot) {
            std::vector<int2> items;
            for (int f : fl)
                if (fr[f].nchild > slot) {
                    const int c = fr[f].child[slot];
                    for (int a = 0; a < nU[c]; ++a) items.push_back(make_int2(c, a));
                }
            if (items.empty()) continue;
            int2* di = up(items);
            nd_extend_kernel<<<(unsigned)items.size(), 256, 0, h->stream>>>(dch, di, dmaps, fronts);
            DDG_CHECK_LAUNCH();
        }
        // partial factorisation of the level's fronts
        std::vector<int64_t> bo, dof2, wo;
        std::vector<int32_t> nts, nss;
        int NTmax = 0, NSmax = 0;
        for (int f : fl) {
            bo.push_back(foff[f]);
            dof2.push_back(doff[f]);
            wo.push_back(woff[f]);
            nts.push_back(NT[f]);
            nss.push_back(nSt[f]);
            NTmax = std::max(NTmax, NT[f]);
            NSmax = std::max(NSmax, nSt[f]);
        }
        front_factor_batched(h, fronts, (int)fl.size(), NTmax, NSmax, up(bo), up(nts), up(nss), dinv, up(dof2), W,
                             up(wo), h->errflags + E_COARSE_SPD);
        // G = L_US D of the level's fronts
        {
            int gmax = 0;
            std::vector<int32_t> fls(fl.begin(), fl.end());
            for (int f : fl) gmax = std::max(gmax, ((nU[f] + CT - 1) / CT) * nSt[f]);
            if (gmax > 0) {
                const size_t sm2 = 2 * CT * CLD * sizeof(double);
                DDG_CUDA(cudaFuncSetAttribute(nd_gprod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
                nd_gprod_kernel<<<dim3(gmax, (unsigned)fl.size()), 256, sm2, h->stream>>>(dpk, up(fls), fronts, W, Gw);
                DDG_CHECK_LAUNCH();
            }
        }
        // D, G, D^T and G^T rows of the level into the solve arrays
        std::vector<int4> items;
        for (int f : fl) {
            for (int i = 0; i < nS[f]; ++i) {
                items.push_back(make_int4(f, 0, i, 0));
                items.push_back(make_int4(f, 2, i, 0));
                if (nU[f] > 0) items.push_back(make_int4(f, 3, i, 0));
            }
            for (int u = 0; u < nU[f]; ++u) items.push_back(make_int4(f, 1, u, 0));
        }
        if (!items.empty()) {
            int4* di = up(items);
            nd_pack_kernel<<<(unsigned)items.size(), 128, 0, h->stream>>>(dpk, di, Gw, W, N.d64, N.d32);
            DDG_CHECK_LAUNCH();
        }
        // the level's workspaces are needed until its launches have run
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        for (void* p : tmp) h->arena.release(p);
        tmp.clear();
    }
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    for (void* p : {(void*)dch, (void*)dmaps, (void*)dpk}) h->arena.release(p);
    h->arena.release(fronts);
    h->arena.release(dinv);
    h->arena.release(W);
    h->arena.release(Gw);
    N.on = true;
    // one launch per level and direction by default: on GB300 the grid
    // barriers of the cooperative variant cost more than the launch gaps
    // they replace (measured: 2.2 vs 1.7 ms of coarse work per solve at 128^3)
    N.persistent = false;
    if (const char* ev = std::getenv("DDG_ND_PERSISTENT")) N.persistent = ev[0] == '1';
}

// grid of the persistent solve: every CTA co-resident (a cooperative launch
// checks it), at most one CTA per eight items of the widest phase
template <typename V>
static int nd_persistent_grid(ddg_handle h) {
    int dev = 0, sms = 1, per = 0;
    DDG_CUDA(cudaGetDevice(&dev));
    DDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DDG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, nd_persistent_kernel<V>, 256, 0));
    const NdCoarse& N = h->nd;
    int widest = (h->n0 + 255) / 256;
    for (int l = 0; l < N.nlevel; ++l) {
        widest = std::max(widest, (N.h_fwd_off[l + 1] - N.h_fwd_off[l] + 7) / 8);
        widest = std::max(widest, (N.h_bwd_off[l + 1] - N.h_bwd_off[l] + 7) / 8);
    }
    return std::max(1, std::min(std::max(1, per) * sms, widest));
}

template <typename V>
static void nd_solve_t(ddg_handle h, const V* data, const V* c, V* y, V* xout, V* w, V* xp) {
    const NdCoarse& N = h->nd;
    const NdSolve F{N.nS, N.nU, N.s0, N.up, N.uoff, N.doff, N.goff, N.dtoff, N.gtoff};
    const int n0 = h->n0;
    if (N.persistent) {
        const NdPersist P{F, N.fitems, N.bitems, N.rsrc, N.rtgt, N.elim, N.fwd_off, N.bwd_off, N.rptr, n0,
                          N.nlevel, N.bar, h->errflags + E_TIMEOUT, (uint64_t)h->wait_ns};
        DDG_CUDA(cudaMemsetAsync(N.bar, 0, sizeof(unsigned), h->stream));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nd_persistent_grid<V>(h));
        cfg.blockDim = dim3(256);
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DDG_CUDA(cudaLaunchKernelEx(&cfg, nd_persistent_kernel<V>, P, data, c, w, y, xp, xout));
        return;
    }
    const unsigned pb = (unsigned)((n0 + 255) / 256);
    launch_pdl(h, nd_permute_kernel<V, true>, dim3(pb), dim3(256), 0, n0, (const int32_t*)N.elim, c, w);
    // forward, deepest level first; w is updated in place
    for (int l = 0; l < N.nlevel; ++l) {
        const int a0 = N.h_fwd_off[l], a1 = N.h_fwd_off[l + 1];
        if (a1 <= a0) continue;
        const int wpr = N.h_fwd_wpr[l];
        const dim3 grid((unsigned)(((int64_t)(a1 - a0) * wpr + 7) / 8));
#define ND_FWD(W)                                                                                            \
    launch_pdl(h, nd_fwd_kernel<V, W>, grid, dim3(256), 0, F, (const int2*)(N.fitems + a0), a1 - a0,          \
               (const int32_t*)N.rtgt, (const int64_t*)N.rptr, (const int2*)N.rsrc, data, w, y, N.h_fwd_pf[l])
        if (wpr == 8) ND_FWD(8);
        else if (wpr == 4) ND_FWD(4);
        else if (wpr == 2) ND_FWD(2);
        else ND_FWD(1);
#undef ND_FWD
    }
    // backward, root first
    for (int l = N.nlevel - 1; l >= 0; --l) {
        const int a0 = N.h_bwd_off[l], a1 = N.h_bwd_off[l + 1];
        if (a1 <= a0) continue;
        const int wpr = N.h_bwd_wpr[l];
        const dim3 grid((unsigned)(((int64_t)(a1 - a0) * wpr + 7) / 8));
#define ND_BWD(W)                                                                                            \
    launch_pdl(h, nd_bwd_kernel<V, W>, grid, dim3(256), 0, F, (const int2*)(N.bitems + a0), a1 - a0, data,    \
               (const V*)y, xp, N.h_bwd_pf[l])
        if (wpr == 8) ND_BWD(8);
        else if (wpr == 4) ND_BWD(4);
        else if (wpr == 2) ND_BWD(2);
        else ND_BWD(1);
#undef ND_BWD
    }
    launch_pdl(h, nd_permute_kernel<V, false>, dim3(pb), dim3(256), 0, n0, (const int32_t*)N.elim, (const V*)xp,
               xout);
}

int nd_solve_launches(ddg_handle h) {
    const NdCoarse& N = h->nd;
    if (N.persistent) return 1;
    int cnt = 2;
    for (int l = 0; l < N.nlevel; ++l) {
        if (N.h_fwd_off[l + 1] > N.h_fwd_off[l]) ++cnt;
        if (N.h_bwd_off[l + 1] > N.h_bwd_off[l]) ++cnt;
    }
    return cnt;
}

// a tile kernel over ntiles tiles, ks CTAs (one cluster) per tile
template <typename... KArgs, typename... Args>
static void launch_cluster(ddg_handle h, void (*kern)(KArgs...), int ks, int ntiles, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntiles * ks));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = ND_TILE_SMEM;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = h->use_pdl ? 1 : 0;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = (unsigned)ks;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    DDG_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

int nd_solve_multi_launches(ddg_handle h) {
    const NdCoarse& N = h->nd;
    int cnt = 2;
    for (int l = 0; l < N.nlevel; ++l) {
        if (N.h_mf_off[l + 1] > N.h_mf_off[l]) ++cnt;
        if (N.h_tgt_off[l + 1] > N.h_tgt_off[l]) ++cnt;
        if (N.h_mb_off[l + 1] > N.h_mb_off[l]) ++cnt;
    }
    return cnt;
}

// m right-hand sides: c, y, x as the batched path's coarse vectors (n0 x m,
// dof-major), w and xp work vectors of the same size in elimination order,
// P the partial rows (sum of the fronts' nU) x m
void nd_coarse_solve_multi(ddg_handle h, int m, const float* c, float* y, float* x, float* w, float* xp, float* P) {
    const NdCoarse& N = h->nd;
    static PerDeviceMax configured;   // the shared-memory attribute is per device
    int dev = -1;
    if (configured.needs((int)ND_TILE_SMEM, dev)) {
        DDG_CUDA(cudaFuncSetAttribute(nd_fwd_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ND_TILE_SMEM));
        DDG_CUDA(cudaFuncSetAttribute(nd_bwd_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ND_TILE_SMEM));
        configured.commit(dev, (int)ND_TILE_SMEM);
    }
    const NdSolve F{N.nS, N.nU, N.s0, N.up, N.uoff, N.doff, N.goff, N.dtoff, N.gtoff};
    const int64_t total = (int64_t)h->n0 * m;
    const unsigned pb = (unsigned)((total + 255) / 256);
    launch_pdl(h, nd_permute_multi_kernel<true>, dim3(pb), dim3(256), 0, total, m, (const int32_t*)N.elim, c, w);
    for (int l = 0; l < N.nlevel; ++l) {
        const int a0 = N.h_mf_off[l], a1 = N.h_mf_off[l + 1];
        if (a1 > a0)
            launch_cluster(h, nd_fwd_tile_kernel, N.h_mf_ks[l], a1 - a0, F, (const int4*)(N.mfitems + a0),
                           (const float*)N.d32, (const float*)w, y, P, m);
        const int t0 = N.h_tgt_off[l], t1 = N.h_tgt_off[l + 1];
        if (t1 > t0)
            launch_pdl(h, nd_fwd_reduce_kernel, dim3((unsigned)((t1 - t0 + 7) / 8)), dim3(256), 0,
                       (const int32_t*)N.rtgt, (const int64_t*)N.rptr, (const int64_t*)N.rsrcp, t0, t1 - t0,
                       (const float*)P, w, m);
    }
    for (int l = N.nlevel - 1; l >= 0; --l) {
        const int a0 = N.h_mb_off[l], a1 = N.h_mb_off[l + 1];
        if (a1 > a0)
            launch_cluster(h, nd_bwd_tile_kernel, N.h_mb_ks[l], a1 - a0, F, (const int2*)(N.mbitems + a0),
                           (const float*)N.d32, (const float*)y, xp, m);
    }
    launch_pdl(h, nd_permute_multi_kernel<false>, dim3(pb), dim3(256), 0, total, m, (const int32_t*)N.elim,
               (const float*)xp, x);
}

void nd_coarse_solve(ddg_handle h, int prec) {
    NdCoarse& N = h->nd;
    if (prec == DDG_PREC_FP64) nd_solve_t<double>(h, N.d64, h->c64, h->y64, h->x64, N.w64, N.x64);
    else nd_solve_t<float>(h, N.d32, h->c32, h->y32, h->x32, N.w32, N.x32);
}

}  // namespace ddg
