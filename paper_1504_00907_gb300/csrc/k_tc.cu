// Multi-RHS local solves on the 5th-generation tensor cores (tcgen05).
//
// For the batched solve the local step z[Omega~_i] += A_i^{-1} R~_i (r - A z)
// (Sec. 6) is a dense GEMM Y_i = A_i^{-1} X_i with X_i = n_i x m.  A_i^{-1} is
// kept as 128 x 32 slabs in BF16 or in TF32 (FP32 storage), K-major,
// SWIZZLE_NONE core-matrix order: core matrix (8 rows x 16 bytes) (mc, kc) at
// byte (mc * KC + kc) * 128 with KC = 4 core matrices along K for BF16 and 8
// for TF32; the local residual is written straight into X^T slabs of the same
// type (N x 32, same core order).  One CTA computes one 128-row block of Y_i:
//   thread 0      producer: cp.async.bulk of the A slab and the X slab of each
//                 K step into a STAGES-deep shared-memory ring (mbarrier
//                 transaction counts);
//   thread 32     issues tcgen05.mma kind::f16 (BF16 x BF16 -> FP32, M = 128,
//                 N = m rounded up to 16, K = 16, two per slab) or kind::tf32
//                 (TF32 x TF32 -> FP32, K = 8, four per slab) into a TMEM
//                 accumulator and commits each stage back to the producer;
//   warps 0-3     read their 32 TMEM lanes (tcgen05.ld 32x32b) and add the
//                 rows into z.
// Every wait is bounded by a time limit on the GPU's global timer (the
// handle's spin_budget_ms): a wait that runs out sets the error flag, the
// kernel drains the copies it has issued (each of them completes, since it
// reads valid global memory; the drain still has a limit of its own, four
// times the budget), frees its TMEM and returns.
#include <type_traits>

#include "ddg_internal.cuh"
#include "dev_common.cuh"

namespace {

constexpr int TC_M = 128;            // rows of Y per CTA (MMA M)
constexpr int TC_K = 32;             // K per slab (two K = 16 MMAs)
// ring depth TC_STAGES: a template parameter (3, 4 or 6), chosen per column
// count by the autotuner (4 when it is off)
constexpr int TC_THREADS = 128;
constexpr int A_SLAB = TC_M * TC_K;       // elements per A slab

template <bool TF32>
using TcElem = typename std::conditional<TF32, float, __nv_bfloat16>::type;

// round to TF32 (nearest, ties away from zero), kept in FP32 storage
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO (K-direction stride between
// core matrices), SBO (M/N-direction stride), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity to complete, for at most
// `limit_ns` nanoseconds of the global timer (checked every 64 polls; a
// poll count of 2^31 ends the wait as well, should the timer not advance).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    uint32_t ok = 0;
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < (1u << 31); ++i) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(sa(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if ((i & 63) == 0) {
            const uint64_t t = global_ns();
            if (i == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int N, int TC_STAGES, bool TF32>
__global__ void __launch_bounds__(TC_THREADS) local_solve_tc_kernel(
    const int2* __restrict__ items, int item_base, const int64_t* __restrict__ ov_off,
    const int32_t* __restrict__ ov_nodes, const int32_t* __restrict__ Tq,
    const int64_t* __restrict__ slab_off, const int64_t* __restrict__ xoff,
    const TcElem<TF32>* __restrict__ Aslab, const TcElem<TF32>* __restrict__ Xslab,
    float* __restrict__ z, int m, int* err, uint64_t limit_ns, int no_copies) {
    using E = TcElem<TF32>;
    constexpr int X_SLAB = N * TC_K;
    constexpr uint32_t A_BYTES = A_SLAB * sizeof(E), X_BYTES = X_SLAB * sizeof(E), STAGE = A_BYTES + X_BYTES;
    // MMAs per slab (each covers 32 bytes of K: two core matrices) and the
    // byte stride between 8-row core-matrix groups
    constexpr int KSTEPS = TF32 ? 4 : 2;
    constexpr uint32_t SBO = TF32 ? 1024 : 512;
    constexpr uint32_t TCOLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + TC_STAGES * STAGE);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* done = empty + TC_STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int failed;

    const int2 it = items[item_base + blockIdx.x];
    const int q = it.x, blk = it.y;
    const int T = Tq[q];
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    const E* Ab = Aslab + (slab_off[q] + (int64_t)blk * T) * A_SLAB;
    const E* Xb = Xslab + xoff[q] * X_SLAB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sa(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sa(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sa(done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(sa(tslot)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    int issued = 0;   // stages handed to the copy engine (producer only)
    if (threadIdx.x == 0 && !no_copies) {
        for (int J = 0; J < T; ++J) {
            const int s = J % TC_STAGES;
            if (J >= TC_STAGES && !mbar_wait(&empty[s], ((J / TC_STAGES) - 1) & 1, limit_ns)) {
                failed = 1;
                break;
            }
            unsigned char* st = smem + s * STAGE;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(sa(&full[s])), "r"(STAGE) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(sa(st)), "l"(Ab + (int64_t)J * A_SLAB), "r"(A_BYTES), "r"(sa(&full[s])) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(sa(st + A_BYTES)), "l"(Xb + (int64_t)J * X_SLAB), "r"(X_BYTES), "r"(sa(&full[s])) : "memory");
            issued = J + 1;
        }
    } else if (threadIdx.x == 32) {
        // D F32 (bits 4-5 = 1), A and B type at bits 7-9 and 10-12 (kind::f16:
        // BF16 = 1; kind::tf32: TF32 = 2), K-major A and B, N >> 3 at bit 17,
        // M >> 4 at bit 24
        constexpr uint32_t ab = TF32 ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
        bool ok = true;
        for (int J = 0; J < T; ++J) {
            const int s = J % TC_STAGES;
            if (!mbar_wait(&full[s], (J / TC_STAGES) & 1, limit_ns)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = sa(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < KSTEPS; ++kk) {
                const uint64_t ad = sdesc(a0 + kk * 256, 128, SBO);
                const uint64_t bd = sdesc(b0 + kk * 256, 128, SBO);
                const uint32_t acc = (J > 0 || kk > 0) ? 1u : 0u;
                if constexpr (TF32)
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                else
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(sa(&empty[s])) : "memory");
        }
        if (!ok) failed = 1;
        // arrives on `done` once every MMA issued above has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(sa(done)) : "memory");
    }
    // the other lanes of the producer and MMA warps park here instead of
    // polling `done` beside their role thread
    __syncwarp();
    // epilogue: TMEM lanes [32 w, 32 w + 32) hold rows blk * 128 + 32 w + lane
    const bool have = mbar_wait(done, 0, limit_ns);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!have) failed = 1;
    __syncthreads();
    if (!failed) {
        // TMEM -> shared tile [128][N + 1] (the stage ring is free: every
        // copy has been consumed by an MMA that completed before `done`)
        float* tile = reinterpret_cast<float*>(smem);
        constexpr int LDS = N + 1;
        const int rl = warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int cb = 0; cb < N / 16; ++cb) {
            float v[16];
            tmem_ld16(taddr + cb * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) tile[rl * LDS + cb * 16 + i] = v[i];
        }
        int* grow = reinterpret_cast<int*>(tile + TC_M * LDS);
        grow[rl] = (blk * TC_M + rl < n) ? ov_nodes[o + blk * TC_M + rl] : -1;
        __syncthreads();
        // z[rows of the block] += tile: consecutive threads take consecutive
        // columns of a row (coalesced), and each thread first loads the 8
        // distinct z entries it updates, then writes them back
        for (int e0 = threadIdx.x; e0 < TC_M * N; e0 += TC_THREADS * 8) {
            float zv[8];
            int64_t ad[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * TC_THREADS;
                const int rr = e / N, c = e % N;
                const int g = e < TC_M * N ? grow[rr] : -1;
                ad[u] = (g >= 0 && c < m) ? (int64_t)g * m + c : -1;
                zv[u] = ad[u] >= 0 ? z[ad[u]] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * TC_THREADS;
                if (ad[u] >= 0) z[ad[u]] = zv[u] + tile[(e / N) * LDS + e % N];
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
        // drain every copy this CTA has issued and that may still be in
        // flight (the last TC_STAGES stages: an earlier stage was consumed by
        // an MMA before its slot was refilled) before the shared memory goes
        // away; issued copies complete, the limit only guards the wait itself
        for (int J = (issued > TC_STAGES ? issued - TC_STAGES : 0); J < issued; ++J)
            mbar_wait(&full[J % TC_STAGES], (J / TC_STAGES) & 1, 4 * limit_ns);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS));
    }
}

// A_i^{-1} (FP64 workspace after local_factor_invert: inverse in the upper
// 32x32 tiles) -> BF16 or TF32 128 x 32 slabs in core-matrix order
template <bool TF32>
__global__ void tc_pack_kernel(int q0, const int32_t* __restrict__ qlist, const double* __restrict__ ws, int Np,
                               const int64_t* __restrict__ ov_off, const int32_t* __restrict__ Tq,
                               const int64_t* __restrict__ slab_off, TcElem<TF32>* __restrict__ out) {
    // elements per 16-byte core-matrix row, core matrices along K per slab
    constexpr int EPR = TF32 ? 4 : 8, KC = TC_K / EPR;
    const int b = blockIdx.x, q = qlist ? qlist[q0 + b] : q0 + b;
    const int n = (int)(ov_off[q + 1] - ov_off[q]);
    const int T = Tq[q];
    const int Mb = (n + TC_M - 1) / TC_M;
    const double* A = ws + (size_t)b * Np * Np;
    TcElem<TF32>* dst = out + slab_off[q] * A_SLAB;
    const int64_t total = (int64_t)Mb * T * A_SLAB;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int64_t slab = e / A_SLAB;
        const int w = (int)(e % A_SLAB);
        const int blk = (int)(slab / T), J = (int)(slab % T);
        // invert the layout: w = ((mc * KC + kc) * 8 * EPR) + (r % 8) * EPR + (k % EPR)
        const int core = w / (8 * EPR), within = w % (8 * EPR);
        const int mc = core / KC, kc = core % KC;
        const int row = blk * TC_M + mc * 8 + within / EPR;
        const int col = J * TC_K + kc * EPR + within % EPR;
        double v = 0.0;
        if (row < n && col < n)
            v = (row / DDG_LT <= col / DDG_LT) ? A[(size_t)row * Np + col] : A[(size_t)col * Np + row];
        if constexpr (TF32) dst[e] = to_tf32((float)v);
        else dst[e] = __float2bfloat16_rn((float)v);
    }
}

// (r - A z) at the colour's rows, all m columns, written as BF16 or TF32 X^T
// slabs: one CTA per (subdomain, 32-row slab); the residual is computed with
// coalesced reads (consecutive threads = consecutive columns), staged in
// shared memory and written out in core-matrix order with 16-byte stores.
template <int SK, bool TF32>
__global__ void __launch_bounds__(256) tc_residual_kernel(
    const int2* __restrict__ slabs, int slab_base, int m, int N, const int32_t* __restrict__ ov_nodes,
    const int64_t* __restrict__ ov_off, const int64_t* __restrict__ xoff,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
    const float* __restrict__ r, const float* __restrict__ z, TcElem<TF32>* __restrict__ X, int z_zero,
    int nx, int ny, int nz) {
    using E = TcElem<TF32>;
    __shared__ __align__(16) E sx[TC_K][DDG_MCHUNK + 8];
    // row metadata of the slab, shared by all m columns: node, and for the
    // CSR path up to 16 (column, value) pairs per row
    __shared__ int sg[TC_K], scnt[TC_K];
    __shared__ int scol[TC_K][16];
    __shared__ float sval[TC_K][16];
    const int2 sl = slabs[slab_base + blockIdx.x];
    const int q = sl.x, J = sl.y;
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    constexpr bool csr = SK == ddgdev::SK_CSR8 || SK == ddgdev::SK_CSR16;
    __shared__ int64_t se0[TC_K];
    if (threadIdx.x < TC_K) {
        const int la = J * TC_K + threadIdx.x;
        const int g = la < n ? ov_nodes[o + la] : -1;
        sg[threadIdx.x] = g;
        if (csr) {
            const int64_t e0 = g >= 0 ? rowptr[g] : 0;
            se0[threadIdx.x] = e0;
            scnt[threadIdx.x] = g >= 0 ? (int)(rowptr[g + 1] - e0) : 0;
        }
    }
    __syncthreads();
    if (csr) {
        // every (row, entry) pair of the slab by its own thread: one round of loads
        for (int e = threadIdx.x; e < TC_K * 16; e += blockDim.x) {
            const int kr = e >> 4, i = e & 15;
            if (i < scnt[kr]) {
                scol[kr][i] = col[se0[kr] + i];
                sval[kr][i] = val[se0[kr] + i];
            }
        }
        __syncthreads();
    }
    if ((m & 3) == 0) {
        // 4 adjacent columns per thread (16-byte z words); the row's stencil
        // or CSR entries and index arithmetic are shared by the 4 columns
        const int nq = N >> 2, cq = threadIdx.x % nq;
        const int c4 = 4 * cq;
        auto ld = [&](const float* v, int gg) { return *reinterpret_cast<const float4*>(v + (int64_t)gg * m + c4); };
        for (int kr = threadIdx.x / nq; kr < TC_K; kr += blockDim.x / nq) {
            const int g = sg[kr];
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g >= 0 && c4 < m) {
                s = ld(r, g);
                if (!z_zero) {
                    float4 az = make_float4(0.f, 0.f, 0.f, 0.f);
                    auto fma4 = [&](float a, const float4& b) {
                        az.x = fma(a, b.x, az.x);
                        az.y = fma(a, b.y, az.y);
                        az.z = fma(a, b.z, az.z);
                        az.w = fma(a, b.w, az.w);
                    };
                    if (SK == DDG_STENCIL_7PT_3D || SK == DDG_STENCIL_5PT_2D) {
                        const int i = g % nx, j = (g / nx) % ny;
                        fma4(SK == DDG_STENCIL_7PT_3D ? 6.f : 4.f, ld(z, g));
                        if (i > 0) fma4(-1.f, ld(z, g - 1));
                        if (i < nx - 1) fma4(-1.f, ld(z, g + 1));
                        if (j > 0) fma4(-1.f, ld(z, g - nx));
                        if (j < ny - 1) fma4(-1.f, ld(z, g + nx));
                        if (SK == DDG_STENCIL_7PT_3D) {
                            const int k = g / (nx * ny);
                            if (k > 0) fma4(-1.f, ld(z, g - nx * ny));
                            if (k < nz - 1) fma4(-1.f, ld(z, g + nx * ny));
                        }
                    } else if (csr) {
                        constexpr int NMAX = SK == ddgdev::SK_CSR8 ? 8 : 16;
                        const int cnt = scnt[kr];
#pragma unroll
                        for (int i2 = 0; i2 < NMAX; ++i2)
                            if (i2 < cnt) fma4(sval[kr][i2], ld(z, scol[kr][i2]));
                    } else {
                        for (int64_t p = rowptr[g]; p < rowptr[g + 1]; ++p) fma4(val[p], ld(z, col[p]));
                    }
                    s = make_float4(s.x - az.x, s.y - az.y, s.z - az.z, s.w - az.w);
                }
            }
            if constexpr (TF32) {
                *reinterpret_cast<float4*>(&sx[kr][c4]) =
                    make_float4(to_tf32(s.x), to_tf32(s.y), to_tf32(s.z), to_tf32(s.w));
            } else {
                __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(&sx[kr][c4]);
                d[0] = __floats2bfloat162_rn(s.x, s.y);
                d[1] = __floats2bfloat162_rn(s.z, s.w);
            }
        }
    } else {
    #pragma unroll 4
        for (int e = threadIdx.x; e < TC_K * N; e += blockDim.x) {
            const int kr = e / N, c = e % N;
            const int g = sg[kr];
            float s = 0.f;
            if (g >= 0 && c < m) {
                s = r[(int64_t)g * m + c];
                if (!z_zero) {
                    if (SK == DDG_STENCIL_7PT_3D || SK == DDG_STENCIL_5PT_2D) {
                        const int i = g % nx, j = (g / nx) % ny;
                        float az = (SK == DDG_STENCIL_7PT_3D ? 6.f : 4.f) * z[(int64_t)g * m + c];
                        if (i > 0) az -= z[(int64_t)(g - 1) * m + c];
                        if (i < nx - 1) az -= z[(int64_t)(g + 1) * m + c];
                        if (j > 0) az -= z[(int64_t)(g - nx) * m + c];
                        if (j < ny - 1) az -= z[(int64_t)(g + nx) * m + c];
                        if (SK == DDG_STENCIL_7PT_3D) {
                            const int k = g / (nx * ny);
                            if (k > 0) az -= z[(int64_t)(g - nx * ny) * m + c];
                            if (k < nz - 1) az -= z[(int64_t)(g + nx * ny) * m + c];
                        }
                        s -= az;
                    } else if (csr) {
                        constexpr int NMAX = SK == ddgdev::SK_CSR8 ? 8 : 16;
                        const int cnt = scnt[kr];
                        float acc = 0.f;
    #pragma unroll
                        for (int i2 = 0; i2 < NMAX; ++i2)
                            if (i2 < cnt) acc = fma(sval[kr][i2], z[(int64_t)scol[kr][i2] * m + c], acc);
                        s -= acc;
                    } else {
                        for (int64_t p = rowptr[g]; p < rowptr[g + 1]; ++p) s -= val[p] * z[(int64_t)col[p] * m + c];
                    }
                }
            }
            if constexpr (TF32) sx[kr][c] = to_tf32(s);
            else sx[kr][c] = __float2bfloat16_rn(s);
        }
    }
    __syncthreads();
    // core-matrix rows: (n, kc) holds k = kc*EPR .. kc*EPR+EPR-1 of column n,
    // 16 bytes (EPR = 8 BF16 or 4 TF32 elements, KC = 32 / EPR)
    constexpr int EPR = TF32 ? 4 : 8, KC = TC_K / EPR;
    uint4* dst = reinterpret_cast<uint4*>(X + (xoff[q] + J) * (int64_t)(N * TC_K));
    for (int e = threadIdx.x; e < N * KC; e += blockDim.x) {
        const int core_row = e;                   // ((nc * KC + kc) * 8 + n % 8)
        const int cm = core_row >> 3, nr = core_row & 7;
        const int nc = cm / KC, kc = cm % KC;
        const int nn = nc * 8 + nr;
        __align__(16) E v[EPR];
#pragma unroll
        for (int t = 0; t < EPR; ++t) v[t] = sx[kc * EPR + t][nn];
        dst[e] = *reinterpret_cast<const uint4*>(v);
    }
}

template <int N, int TC_STAGES, bool TF32>
constexpr int tc_smem() {
    return TC_STAGES * (A_SLAB + N * TC_K) * (int)sizeof(TcElem<TF32>) + (2 * TC_STAGES + 1) * 8 + 16;
}

template <int N, int TC_STAGES, bool TF32>
void configure_tc() {
    static PerDeviceMax configured;   // the attribute is per device
    constexpr int smem = tc_smem<N, TC_STAGES, TF32>();
    int dev = -1;
    if (!configured.needs(smem, dev)) return;
    DDG_CUDA(cudaFuncSetAttribute(local_solve_tc_kernel<N, TC_STAGES, TF32>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    configured.commit(dev, smem);
}

template <int N, int TC_STAGES, bool TF32>
void launch_tc_s(ddg_handle h, int i0, int i1, int m) {
    configure_tc<N, TC_STAGES, TF32>();
    constexpr int smem = tc_smem<N, TC_STAGES, TF32>();
    const TcElem<TF32>* A;
    const TcElem<TF32>* X;
    if constexpr (TF32) {
        A = h->tc.A32;
        X = h->tc.X32;
    } else {
        A = h->tc.A;
        X = h->tc.X;
    }
    local_solve_tc_kernel<N, TC_STAGES, TF32><<<i1 - i0, TC_THREADS, smem, h->stream>>>(
        h->tc.items, i0, h->ov_off, h->ov_nodes, h->Tq, h->tc.slab_off, h->tc.xoff, A, X,
        h->mw.z32, m, h->errflags + E_TIMEOUT, (uint64_t)h->wait_ns,
        (h->debug & DDG_DEBUG_TC_NO_COPIES) ? 1 : 0);
    DDG_CHECK_LAUNCH();
}

template <int N, bool TF32>
void launch_tc_k(ddg_handle h, int i0, int i1, int m) {
    if (h->tc_stages == 3) launch_tc_s<N, 3, TF32>(h, i0, i1, m);
    else if (h->tc_stages == 6) launch_tc_s<N, 6, TF32>(h, i0, i1, m);
    else launch_tc_s<N, 4, TF32>(h, i0, i1, m);
}

template <int N>
void launch_tc(ddg_handle h, int i0, int i1, int m) {
    if (h->tc.kind == DDG_TC_TF32) launch_tc_k<N, true>(h, i0, i1, m);
    else launch_tc_k<N, false>(h, i0, i1, m);
}

}  // namespace

namespace ddg {

int tc_n_for(int m) { return ((m + 15) / 16) * 16; }

void tc_pack(ddg_handle h, int q0, int q1, const int32_t* qlist, const double* ws) {
    const int nb = q1 - q0;
    if (nb <= 0 || h->tc.kind == DDG_TC_OFF) return;
    if (h->tc.kind == DDG_TC_TF32)
        tc_pack_kernel<true><<<nb, 256, 0, h->stream>>>(q0, qlist, ws, h->Tmax * DDG_LT, h->ov_off, h->Tq,
                                                        h->tc.slab_off, h->tc.A32);
    else
        tc_pack_kernel<false><<<nb, 256, 0, h->stream>>>(q0, qlist, ws, h->Tmax * DDG_LT, h->ov_off, h->Tq,
                                                         h->tc.slab_off, h->tc.A);
    DDG_CHECK_LAUNCH();
}

void tc_residual(ddg_handle h, int c, bool z_zero, int m) {
    const int s0 = h->tc.h_cslab_off[c], s1 = h->tc.h_cslab_off[c + 1];
    if (s1 <= s0) return;
    const int N = tc_n_for(m);
    MultiWork& w = h->mw;
#define TC_RES(SK)                                                                                          \
    do {                                                                                                     \
        if (h->tc.kind == DDG_TC_TF32)                                                                       \
            tc_residual_kernel<SK, true><<<s1 - s0, 256, 0, h->stream>>>(                                    \
                h->tc.slabs, s0, m, N, h->ov_nodes, h->ov_off, h->tc.xoff, h->rowptr, h->col, h->val32, w.r32, \
                w.z32, h->tc.X32, z_zero, h->nx, h->ny, h->nz);                                              \
        else                                                                                                 \
            tc_residual_kernel<SK, false><<<s1 - s0, 256, 0, h->stream>>>(                                   \
                h->tc.slabs, s0, m, N, h->ov_nodes, h->ov_off, h->tc.xoff, h->rowptr, h->col, h->val32, w.r32, \
                w.z32, h->tc.X, z_zero, h->nx, h->ny, h->nz);                                                \
    } while (0)
    DDG_DISPATCH_SK(h, TC_RES);
#undef TC_RES
    DDG_CHECK_LAUNCH();
}

void tc_local_solve(ddg_handle h, int c, int m) {
    const int i0 = h->tc.h_citem_off[c], i1 = h->tc.h_citem_off[c + 1];
    if (i1 <= i0) return;
    switch (tc_n_for(m)) {
        case 16: launch_tc<16>(h, i0, i1, m); break;
        case 32: launch_tc<32>(h, i0, i1, m); break;
        case 48: launch_tc<48>(h, i0, i1, m); break;
        default: launch_tc<64>(h, i0, i1, m); break;
    }
}

}  // namespace ddg
