// Exact local solves with banded Cholesky factors (Sec. 6: A_i^{-1} r_i),
// for overlapping subdomains too large for dense inverses.
//
// A_i (rows and columns in ascending dof order) has half-bandwidth b.  Its
// banded Cholesky factor L = chol(A_i) is computed in FP64 with the 64x64
// tile band kernels, batched over the subdomains, and rewritten in block form
// with super-blocks of B = 64 Wt >= b rows:
//   forward   y_K = D_K (r_K - C_K y_{K-1}),        D_K = L_KK^{-1}
//   backward  x_K = D_K^T (y_K - C_{K+1}^T x_{K+1})
// where C_K = L_{K,K-1} is nonzero only in its first b rows and, in row i,
// only in the columns B - b + i .. B - 1 of block K - 1.  Per super-block the
// stored data are C_K (row i: columns [(B - b + i) & ~3, B)) followed by D_K
// (row i: columns [0, i] padded to a multiple of 4), FP64 and FP32 copies.
//
// One CTA solves one subdomain: a producer warp streams the blocks' rows in
// the order the recurrence reads them (C_1, D_1, ..., then backwards) with
// cp.async.bulk into a ring of shared-memory stages; 16 consumer warps apply
// them to the subdomain's vector, which stays in shared memory from the
// residual to the correction.  The recurrence is sequential in K, but the
// matrix stream does not depend on it, so the CTA reads its factor at close
// to one SM's share of HBM bandwidth while the subdomains of a colour run in
// parallel.  Every wait is bounded by the handle's spin budget.
#include "ddg_internal.cuh"
#include "dev_common.cuh"

namespace {

constexpr int CT = DDG_CT;
constexpr int BL_CONSUMERS = 512;                 // 16 consumer warps
constexpr int BL_THREADS = BL_CONSUMERS + 32;     // + the producer warp
constexpr int BL_NW = BL_CONSUMERS / 32;

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase of `bar` with the given parity (global timer)
__device__ __forceinline__ bool bl_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
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

__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" :: "r"(BL_CONSUMERS) : "memory");
}

// barrier of the consumer warps that also returns whether any of them passed
// a non-zero `pred` (the same answer in every consumer thread)
__device__ __forceinline__ int consumers_any(int pred) {
    int r;
    asm volatile("{\n.reg .pred p;\nsetp.ne.s32 p, %1, 0;\nbar.red.or.pred p, 1, %2, p;\nselp.s32 %0, 1, 0, p;\n}\n"
                 : "=r"(r) : "r"(pred), "r"(BL_CONSUMERS) : "memory");
    return r;
}

__device__ __forceinline__ size_t band_index(int row, int col, int Wt) {
    const int R = row / CT, C = col / CT;
    return ((size_t)R * (Wt + 1) + (R - C)) * CT * CT + (row % CT) * CT + (col % CT);
}

// A_i into the band tiles: one CTA per subdomain of the batch, a thread per
// local row; columns found by binary search in the sorted local dof list.
// Padding rows (n_i .. 64 NT_i) get a unit diagonal.
__global__ void band_assemble_kernel(const int32_t* __restrict__ qlist, const int64_t* __restrict__ ov_off,
                                     const int32_t* __restrict__ ov_nodes, const int64_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ col, const double* __restrict__ val,
                                     const int64_t* __restrict__ boff, const int32_t* __restrict__ nts, int Wt,
                                     double* band) {
    const int b = blockIdx.x, q = qlist[b];
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    const int32_t* idx = ov_nodes + o;
    double* bd = band + boff[b];
    const int npad = nts[b] * CT;
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        if (i >= n) {
            bd[band_index(i, i, Wt)] = 1.0;
            continue;
        }
        const int g = idx[i];
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
            const int c = col[e];
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (idx[mid] < c) lo = mid + 1;
                else hi = mid;
            }
            if (lo < n && idx[lo] == c && lo <= i) bd[band_index(i, lo, Wt)] = val[e];
        }
    }
}

// Block form of each factor: grid (nK_max, nb); C_K then D_K rows as
// described above, into data + qoff[q] + K (sizeC + sizeD).
__global__ void band_pack_kernel(const int32_t* __restrict__ qlist, const int32_t* __restrict__ nkq,
                                 const int64_t* __restrict__ boff, const int64_t* __restrict__ woff,
                                 const double* __restrict__ band, const double* __restrict__ W, int Wt, int b,
                                 const int32_t* __restrict__ rowC, const int32_t* __restrict__ rowD, int sizeC,
                                 int sizeD, const int64_t* __restrict__ qoff, double* out64, float* out32) {
    const int K = blockIdx.x, bi = blockIdx.y, q = qlist[bi];
    if (K >= nkq[q]) return;
    const int B = Wt * CT;
    const double* bd = band + boff[bi];
    const double* Wq = W + woff[bi];
    const size_t Ptiles = (size_t)Wt * (Wt + 1) / 2;
    const int64_t base = qoff[q] + (int64_t)K * (sizeC + sizeD);
    // C_K = L_{K,K-1}: row i < b, stored columns [a_i, B) of block K-1
    for (int e = threadIdx.x; e < sizeC; e += blockDim.x) {
        int lo = 0, hi = b;   // the row of element e: rowC[i] <= e < rowC[i + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (rowC[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int i = lo;
        double v = 0.0;
        if (K > 0 && e < rowC[b]) {
            const int a = (B - b + i) & ~3;
            const int cl = a + (e - rowC[i]);
            const int row = K * B + i, colg = (K - 1) * B + cl;
            const int R = row / CT, C = colg / CT;
            if (cl >= B - b + i && R - C <= Wt) v = bd[band_index(row, colg, Wt)];
        }
        if (out64) out64[base + e] = v;
        if (out32) out32[base + e] = (float)v;
    }
    // D_K = L_KK^{-1}: row i, columns [0, i] (padded to a multiple of 4)
    for (int e = threadIdx.x; e < sizeD; e += blockDim.x) {
        int lo = 0, hi = B;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (rowD[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int i = lo, j = e - rowD[i];
        double v = 0.0;
        if (j <= i) {
            const int ti = i / CT, tj = j / CT;
            v = Wq[((size_t)K * Ptiles + (size_t)ti * (ti + 1) / 2 + tj) * CT * CT + (i % CT) * CT + (j % CT)];
        }
        if (out64) out64[base + sizeC + e] = v;
        if (out32) out32[base + sizeC + e] = (float)v;
    }
}

// One CTA per subdomain of a colour (sweep positions q_base + blockIdx.x):
// z[Omega~_q] += A_q^{-1} res_q through the block-form factor (see the file
// comment).  Shared memory: `stages` ring slots of stage_elems values, the
// subdomain vector (nK B values), a B-value work vector and the barriers.
template <typename V>
__global__ void __launch_bounds__(BL_THREADS) band_solve_kernel(
    int q_base, const int64_t* __restrict__ ov_off, const int32_t* __restrict__ ov_nodes,
    const int32_t* __restrict__ nkq, const int64_t* __restrict__ qoff, const V* __restrict__ data,
    const int32_t* __restrict__ rowC, const int32_t* __restrict__ rowD, const int2* __restrict__ chC, int nchC,
    const int2* __restrict__ chD, int nchD, int B, int b, int sizeC, int sizeD, int stages, int stage_elems,
    int vec_elems, const V* __restrict__ res, V* __restrict__ z, int* err, uint64_t limit_ns) {
    extern __shared__ __align__(128) unsigned char smraw[];
    V* ring = reinterpret_cast<V*>(smraw);
    V* vec = ring + (size_t)stages * stage_elems;
    V* tbuf = vec + vec_elems;
    uint64_t* full = reinterpret_cast<uint64_t*>(tbuf + ((B + 15) & ~15));
    uint64_t* empty = full + stages;

    const int q = q_base + blockIdx.x;
    const int64_t o = ov_off[q];
    const int n = (int)(ov_off[q + 1] - o);
    const int nK = nkq[q];
    const V* dq = data + qoff[q];
    const int tid = threadIdx.x;
    const bool producer = tid >= BL_CONSUMERS;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sa(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sa(&empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // launched as a programmatic dependent of the residual kernel
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();

    if (producer) {
        if (tid != BL_CONSUMERS) return;
        // the chunks in the order the consumers read them
        int seq = 0;
        bool ok = true;
        auto issue = [&](int K, bool isC, int c) {
            const int2 ch = isC ? chC[c] : chD[c];
            const int64_t e0 = (int64_t)K * (sizeC + sizeD) + (isC ? rowC[ch.x] : sizeC + rowD[ch.x]);
            const int elems = isC ? rowC[ch.y] - rowC[ch.x] : rowD[ch.y] - rowD[ch.x];
            const uint32_t bytes = (uint32_t)elems * sizeof(V);
            const int s = seq % stages;
            if (seq >= stages && !bl_wait(&empty[s], ((seq / stages) - 1) & 1, limit_ns)) {
                ok = false;
                return;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(sa(&full[s])), "r"(bytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(sa(ring + (size_t)s * stage_elems)), "l"(dq + e0), "r"(bytes), "r"(sa(&full[s]))
                         : "memory");
            ++seq;
        };
        for (int K = 0; K < nK && ok; ++K) {
            if (K > 0)
                for (int c = 0; c < nchC && ok; ++c) issue(K, true, c);
            for (int c = 0; c < nchD && ok; ++c) issue(K, false, c);
        }
        for (int K = nK - 1; K >= 0 && ok; --K) {
            if (K + 1 < nK)
                for (int c = 0; c < nchC && ok; ++c) issue(K + 1, true, c);
            for (int c = 0; c < nchD && ok; ++c) issue(K, false, c);
        }
        // every copy issued is complete before the CTA's shared memory goes
        // away (the consumers have waited for all of them unless they stopped)
        for (int t = (seq > stages ? seq - stages : 0); t < seq; ++t)
            bl_wait(&full[t % stages], (t / stages) & 1, 4 * limit_ns);
        if (!ok) atomicExch(err, 1);
        return;
    }

    // ---- consumers
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int npad = nK * B;
    for (int i = tid; i < npad; i += BL_CONSUMERS) vec[i] = i < n ? res[o + i] : (V)0;
    consumers_sync();
    const int warp = tid >> 5, lane = tid & 31;   // consumer warps 0..15
    int seq = 0;
    bool stop = false;   // the same in every consumer thread (a barrier vote)
    int bad = 0;         // this thread's wait for a chunk ran out
    // wait for chunk `seq` in its slot (bounded)
    auto acquire = [&](const V*& chunk) {
        const int s = seq % stages;
        if (!bl_wait(&full[s], (seq / stages) & 1, limit_ns)) bad = 1;
        chunk = ring + (size_t)s * stage_elems;
    };
    // after a chunk: every consumer is done with its slot; stop together if
    // any wait ran out
    auto release = [&]() {
        stop = consumers_any(bad) != 0;
        if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(sa(&empty[seq % stages])) : "memory");
        ++seq;
    };
    // forward: y_K = D_K (r_K - C_K y_{K-1})
    for (int K = 0; K < nK && !stop; ++K) {
        V* vK = vec + (size_t)K * B;
        for (int i = tid; i < B; i += BL_CONSUMERS) tbuf[i] = vK[i];
        consumers_sync();
        if (K > 0) {
            const V* yprev = vK - B;
            for (int c = 0; c < nchC && !stop; ++c) {
                const int2 ch = chC[c];
                const V* chunk;
                acquire(chunk);
                // four rows per warp, eight lanes per row: three shuffle steps
                // per row (the FP64 adds of a full-warp sum would cost half as
                // much again as the row's multiply-adds)
                for (int i0 = ch.x + warp * 4; i0 < ch.y; i0 += BL_NW * 4) {
                    const int i = i0 + (lane >> 3), l8 = lane & 7;
                    V s = 0;
                    if (i < ch.y) {
                        const int a = (B - b + i) & ~3;
                        const V* row = chunk + (rowC[i] - rowC[ch.x]);
                        for (int j = l8; j < B - a; j += 8) s = fma(row[j], yprev[a + j], s);
                    }
                    s += __shfl_xor_sync(0xffffffffu, s, 4);
                    s += __shfl_xor_sync(0xffffffffu, s, 2);
                    s += __shfl_xor_sync(0xffffffffu, s, 1);
                    if (l8 == 0 && i < ch.y) tbuf[i] -= s;
                }
                release();
            }
        }
        for (int c = 0; c < nchD && !stop; ++c) {
            const int2 ch = chD[c];
            const V* chunk;
            acquire(chunk);
            for (int i0 = ch.x + warp * 4; i0 < ch.y; i0 += BL_NW * 4) {
                const int i = i0 + (lane >> 3), l8 = lane & 7;
                V s = 0;
                if (i < ch.y) {
                    const V* row = chunk + (rowD[i] - rowD[ch.x]);
                    for (int j = l8; j <= i; j += 8) s = fma(row[j], tbuf[j], s);
                }
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                if (l8 == 0 && i < ch.y) vK[i] = s;
            }
            release();
        }
    }
    // backward: x_K = D_K^T (y_K - C_{K+1}^T x_{K+1}); thread tid owns the
    // columns tid and tid + 512 of the block (B <= 1024)
    for (int K = nK - 1; K >= 0 && !stop; --K) {
        V* vK = vec + (size_t)K * B;
        V acc[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = tid + u * BL_CONSUMERS;
            acc[u] = j < B ? vK[j] : (V)0;
        }
        if (K + 1 < nK) {
            const V* xnext = vK + B;
            for (int c = 0; c < nchC && !stop; ++c) {
                const int2 ch = chC[c];
                const V* chunk;
                acquire(chunk);
                for (int i = ch.x; i < ch.y; ++i) {
                    const int a = (B - b + i) & ~3;
                    const V* row = chunk + (rowC[i] - rowC[ch.x]);
                    const V xi = xnext[i];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = tid + u * BL_CONSUMERS;
                        if (j >= a && j < B) acc[u] = fma(-row[j - a], xi, acc[u]);
                    }
                }
                release();
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = tid + u * BL_CONSUMERS;
            if (j < B) tbuf[j] = acc[u];
            acc[u] = 0;
        }
        consumers_sync();
        for (int c = 0; c < nchD && !stop; ++c) {
            const int2 ch = chD[c];
            const V* chunk;
            acquire(chunk);
            for (int i = ch.x; i < ch.y; ++i) {
                const V* row = chunk + (rowD[i] - rowD[ch.x]);
                const V si = tbuf[i];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int j = tid + u * BL_CONSUMERS;
                    if (j <= i) acc[u] = fma(row[j], si, acc[u]);
                }
            }
            release();
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = tid + u * BL_CONSUMERS;
            if (j < B) vK[j] = acc[u];
        }
        consumers_sync();
    }
    if (stop) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    for (int i = tid; i < n; i += BL_CONSUMERS) z[ov_nodes[o + i]] += vec[i];
}

}  // namespace

namespace ddg {

void band_local_assemble(ddg_handle h, const int32_t* qlist, int nb, const int64_t* boff, const int32_t* nts,
                         double* band) {
    band_assemble_kernel<<<nb, 256, 0, h->stream>>>(qlist, h->ov_off, h->ov_nodes, h->rowptr, h->col, h->val64,
                                                    boff, nts, h->bl.Wt, band);
    DDG_CHECK_LAUNCH();
}

void band_local_pack(ddg_handle h, const int32_t* qlist, int nb, int nKmax, const int64_t* boff,
                     const int64_t* woff, const double* band, const double* W) {
    BandLocal& L = h->bl;
    band_pack_kernel<<<dim3(nKmax, nb), 256, 0, h->stream>>>(qlist, L.nk, boff, woff, band, W, L.Wt, L.b, L.rowC,
                                                             L.rowD, L.sizeC, L.sizeD, L.qoff, L.d64, L.d32);
    DDG_CHECK_LAUNCH();
}

size_t band_solve_smem(const BandLocal& L, int prec, int stages) {
    const size_t sv = prec == DDG_PREC_FP64 ? 8 : 4;
    return (size_t)stages * DDG_BAND_STAGE_BYTES + (size_t)L.vec_elems * sv + (size_t)((L.B + 15) & ~15) * sv +
           (size_t)2 * stages * 8;
}

template <typename V>
static void launch_band(ddg_handle h, int c, const V* data, const int2* chC, int nchC, const int2* chD, int nchD,
                        const V* res, V* z, int stages) {
    const BandLocal& L = h->bl;
    const int q0 = h->h_csub_off[c], q1 = h->h_csub_off[c + 1];
    if (q1 <= q0) return;
    const size_t smem = band_solve_smem(L, sizeof(V) == 8 ? DDG_PREC_FP64 : DDG_PREC_FP32, stages);
    launch_pdl(h, band_solve_kernel<V>, dim3(q1 - q0), dim3(BL_THREADS), smem, q0, (const int64_t*)h->ov_off,
               (const int32_t*)h->ov_nodes, (const int32_t*)L.nk, (const int64_t*)L.qoff, data,
               (const int32_t*)L.rowC, (const int32_t*)L.rowD, chC, nchC, chD, nchD, L.B, L.b, L.sizeC, L.sizeD,
               stages, (int)(DDG_BAND_STAGE_BYTES / sizeof(V)), L.vec_elems, res, z, h->errflags + E_TIMEOUT,
               (uint64_t)h->wait_ns);
}

void band_local_configure(ddg_handle h) {
    static PerDeviceMax conf64, conf32;
    const BandLocal& L = h->bl;
    int dev = -1;
    const int s64 = (int)band_solve_smem(L, DDG_PREC_FP64, L.stages64);
    if (conf64.needs(s64, dev)) {
        DDG_CUDA(cudaFuncSetAttribute(band_solve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64));
        conf64.commit(dev, s64);
    }
    const int s32 = (int)band_solve_smem(L, DDG_PREC_FP32, L.stages32);
    if (conf32.needs(s32, dev)) {
        DDG_CUDA(cudaFuncSetAttribute(band_solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
        conf32.commit(dev, s32);
    }
}

void band_local_solve_colour(ddg_handle h, int c, int prec) {
    const BandLocal& L = h->bl;
    if (prec == DDG_PREC_FP64)
        launch_band<double>(h, c, L.d64, L.ch64C, L.nch64C, L.ch64D, L.nch64D, h->res64, h->z64, L.stages64);
    else
        launch_band<float>(h, c, L.d32, L.ch32C, L.nch32C, L.ch32D, L.nch32D, h->res32, h->z32, L.stages32);
}

}  // namespace ddg
