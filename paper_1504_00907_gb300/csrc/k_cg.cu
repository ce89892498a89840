// Preconditioned CG recurrence (Sec. 7) in FP64: SpMV with the fused p^T A p,
// the u/r update with ||r||^2, the r^T z (and q^T z) dots that yield beta,
// and the p update.  Every reduction is deterministic: each block writes a
// partial, and the last block to finish (ticket counter) sums the partials
// in block order and derives the CG scalars on the device.
#include "ddg_internal.cuh"
#include "dev_common.cuh"

namespace {

constexpr int RT = 256;   // threads of the reduction kernels

// last-block epilogue: every block passes NV partial sums; the last block
// leaves the totals in tot[] and returns true
template <int NV>
__device__ bool reduce_last(double (&v)[NV], double* partials, unsigned* counter, double* tot) {
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double bs[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) bs[i] = ddgdev::block_sum(v[i], sh);
    if (threadIdx.x == 0)
        for (int i = 0; i < NV; ++i) partials[(size_t)blockIdx.x * NV + i] = bs[i];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s += __ldcg(partials + (size_t)b * NV + i);
        tot[i] = ddgdev::block_sum(s, sh);
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// y = A x over CSR rows; optionally dot = x^T y into scal[S_PQ] and
// alpha = rho / p^T A p into scal[S_ALPHA] (breakdown flag if p^T A p <= 0)
// G = 1: a thread per row; G > 1: a group of G lanes per row (long rows)
template <bool DOT, int G>
__global__ void __launch_bounds__(RT) spmv_csr64_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ y, double* partials,
                                                        unsigned* counter, double* scal) {
    double acc[1] = {0.0};
    if (G == 1) {
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
             g += (int64_t)gridDim.x * blockDim.x) {
            double s = 0.0;
            for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) s = fma(val[e], x[col[e]], s);
            y[g] = s;
            if (DOT) acc[0] = fma(x[g], s, acc[0]);
        }
    } else {
        // the trip count depends on the block only, so all lanes reach the shuffles
        constexpr int RPB = RT / G;
        for (int64_t base = (int64_t)blockIdx.x * RPB; base < n; base += (int64_t)gridDim.x * RPB) {
            const int64_t g = base + threadIdx.x / G;
            const bool live = g < n;
            const double s = ddgdev::csr_row_dot_group<G>((int)(live ? g : 0), live, rowptr, col, val, x);
            if (live && (threadIdx.x & (G - 1)) == 0) {
                y[g] = s;
                if (DOT) acc[0] = fma(x[g], s, acc[0]);
            }
        }
    }
    if (!DOT) return;
    double tot[1];
    if (reduce_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        scal[S_PQ] = pq;
        scal[S_ALPHA] = scal[S_RZ] / pq;
        if (!(pq > 0.0) || pq != pq) scal[S_FLAG] = 1.0;
    }
}

// matrix-free constant-coefficient Laplacians: [6,-1] (3D) / [4,-1] (2D)
template <bool DOT, int DIM>
__global__ void __launch_bounds__(RT) spmv_lap64_kernel(int nx, int ny, int nz,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ y, double* partials,
                                                        unsigned* counter, double* scal) {
    // n < 2^31 (checked at setup): 32-bit index arithmetic, two 32-bit
    // divisions per row instead of three 64-bit ones
    const int n = nx * ny * nz, sxy = nx * ny;
    double acc[1] = {0.0};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const int t = g / nx;
        const int i = g - t * nx, j = t % ny, k = t / ny;
        const double xc = x[g];
        // the neighbours' sum, then one FMA: one FP64 operation fewer per
        // row than subtracting the neighbours one by one (FP64 issue bound);
        // the sum starts from the first neighbour, not from an added zero
        double nb = i > 0 ? x[g - 1] : 0.0;
        if (i < nx - 1) nb += x[g + 1];
        if (j > 0) nb += x[g - nx];
        if (j < ny - 1) nb += x[g + nx];
        if (DIM == 3) {
            if (k > 0) nb += x[g - sxy];
            if (k < nz - 1) nb += x[g + sxy];
        }
        const double s = fma(DIM == 3 ? 6.0 : 4.0, xc, -nb);
        y[g] = s;
        if (DOT) acc[0] = fma(xc, s, acc[0]);
    }
    if (!DOT) return;
    double tot[1];
    if (reduce_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        scal[S_PQ] = pq;
        scal[S_ALPHA] = scal[S_RZ] / pq;
        if (!(pq > 0.0) || pq != pq) scal[S_FLAG] = 1.0;
    }
}

// u += alpha p; r -= alpha q; ||r||^2 -> scal[S_RR]
__global__ void __launch_bounds__(RT) cg_update_ur_kernel(int64_t n, double* __restrict__ u,
                                                          double* __restrict__ r,
                                                          const double* __restrict__ p,
                                                          const double* __restrict__ q,
                                                          double* partials, unsigned* counter,
                                                          double* scal) {
    const double alpha = scal[S_ALPHA];
    double acc[1] = {0.0};
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        u[g] = fma(alpha, p[g], u[g]);
        const double rg = fma(-alpha, q[g], r[g]);
        r[g] = rg;
        acc[0] = fma(rg, rg, acc[0]);
    }
    double tot[1];
    if (reduce_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        scal[S_RR] = tot[0];
        if (tot[0] != tot[0]) scal[S_FLAG] = 1.0;
    }
}

// rho' = r^T z, qz = q^T z; beta = rho'/rho (FR) or -alpha qz / rho (PR); rho <- rho'
// (first: a restart, beta = 0; read from *firstp when that is set, so that a
// graph-driven solve decides it on the device)
template <typename ZV>
__global__ void __launch_bounds__(RT) cg_dots_kernel(int64_t n, const double* __restrict__ r,
                                                     const double* __restrict__ q,
                                                     const ZV* __restrict__ z, int first, int pr,
                                                     double* partials, unsigned* counter,
                                                     double* scal, const int* firstp) {
    if (firstp) first = *firstp;
    double acc[2] = {0.0, 0.0};
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const double zg = (double)z[g];
        acc[0] = fma(r[g], zg, acc[0]);
        if (!first && pr) acc[1] = fma(q[g], zg, acc[1]);
    }
    double tot[2];
    if (reduce_last<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
        const double rz = tot[0];
        if (!first) {
            const double beta = pr ? (-scal[S_ALPHA] * tot[1] / scal[S_RZ]) : (rz / scal[S_RZ]);
            scal[S_BETA] = beta;
        } else {
            scal[S_BETA] = 0.0;
        }
        scal[S_QZ] = tot[1];
        scal[S_RZ] = rz;
        if (rz != rz) scal[S_FLAG] = 1.0;
    }
}

template <typename ZV>
__global__ void cg_update_p_kernel(int64_t n, double* __restrict__ p, const ZV* __restrict__ z,
                                   const double* __restrict__ scal, int first, const int* firstp) {
    if (firstp) first = *firstp;
    const double beta = first ? 0.0 : scal[S_BETA];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x)
        p[g] = first ? (double)z[g] : fma(beta, p[g], (double)z[g]);
}

// (gate: when set, every block returns at once unless *gate != 0)
__global__ void __launch_bounds__(RT) dot64_kernel(int64_t n, const double* __restrict__ a,
                                                   const double* __restrict__ b, double* partials,
                                                   unsigned* counter, double* scal, int slot,
                                                   const int* gate) {
    if (gate && !*gate) return;
    double acc[1] = {0.0};
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x)
        acc[0] = fma(a[g], b[g], acc[0]);
    double tot[1];
    if (reduce_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) scal[slot] = tot[0];
}

// r = f - A u (CSR)
__global__ void residual64_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                  const double* __restrict__ f, const double* __restrict__ u,
                                  double* __restrict__ r, const int* gate) {
    if (gate && !*gate) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    double s = f[g];
    for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) s = fma(-val[e], u[col[e]], s);
    r[g] = s;
}

__global__ void copy_gated_kernel(int64_t n, const double* __restrict__ a, double* __restrict__ b,
                                  const int* gate) {
    if (!*gate) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) b[g] = a[g];
}

__global__ void to_float_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) b[g] = (float)a[g];
}
__global__ void to_double_kernel(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) b[g] = (double)a[g];
}

__global__ void strided_gather_kernel(int64_t n, const double* __restrict__ src, int m, int j,
                                      double* __restrict__ dst) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dst[g] = src[g * m + j];
}
__global__ void strided_scatter_kernel(int64_t n, const double* __restrict__ src, int m, int j,
                                       double* __restrict__ dst) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dst[g * m + j] = src[g];
}
__global__ void cast_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) b[g] = (float)a[g];
}

__global__ void set_scalar_kernel(double* scal, int slot, double v) { scal[slot] = v; }

// dL/dkappa for the cell-centred variable-coefficient operator:
// A = sum_faces c_f (e_a - e_b)(e_a - e_b)^T (interior) + c_f e_a e_a^T (boundary),
// so dL/dc_f = -lambda^T (dA/dc_f) u = -(l_a - l_b)(u_a - u_b) (interior) or
// -l_a u_a (boundary); the chain rule through c_f = 2 ka kb / (ka + kb)
// (interior) or c_f = 2 ka (boundary) gives each cell's gradient.
__global__ void grad_var7_kernel(int nx, int ny, int nz, const double* __restrict__ kap, const double* __restrict__ lam,
                                 const double* __restrict__ u, double* __restrict__ dk) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int i = (int)(g % nx), j = (int)((g / nx) % ny), k = (int)(g / ((int64_t)nx * ny));
    const double ka = kap[g];
    double s = 0.0;
    const int64_t st[3] = {1, nx, (int64_t)nx * ny};
    const int cc[3] = {i, j, k}, nn[3] = {nx, ny, nz};
    for (int ax = 0; ax < 3; ++ax) {
        for (int side = -1; side <= 1; side += 2) {
            const int c2 = cc[ax] + side;
            if (c2 < 0 || c2 >= nn[ax]) {
                // boundary face: c = 2 ka, dc/dka = 2
                s += -lam[g] * u[g] * 2.0;
            } else {
                const int64_t gb = g + side * st[ax];
                const double kb = kap[gb];
                const double dcdka = 2.0 * kb * kb / ((ka + kb) * (ka + kb));
                s += -(lam[g] - lam[gb]) * (u[g] - u[gb]) * dcdka;
            }
        }
    }
    dk[g] = s;
}

// dL/dmu_e = -lambda_e^T K^mu u_e for Q1 elasticity: gather the 24 dofs of
// element e (clamped x = 0 nodes contribute zero) and contract with the
// element matrix dK_e / dmu_e
__global__ void grad_q1_kernel(int ne, const double* __restrict__ kmu, const double* __restrict__ lam,
                               const double* __restrict__ u, double* __restrict__ dmu) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ne * ne * ne) return;
    const int ei = (int)(e % ne), ej = (int)((e / ne) % ne), ek = (int)(e / ((int64_t)ne * ne));
    double lv[24], uv[24];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int I = ei + (a & 1), J = ej + ((a >> 1) & 1), K = ek + (a >> 2);
        const int64_t base = I >= 1 ? 3 * ((int64_t)(I - 1) + (int64_t)ne * (J + (int64_t)(ne + 1) * K)) : -1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            lv[3 * a + i] = base >= 0 ? lam[base + i] : 0.0;
            uv[3 * a + i] = base >= 0 ? u[base + i] : 0.0;
        }
    }
    double s = 0.0;
    for (int a = 0; a < 24; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < 24; ++b) t = fma(__ldg(kmu + a * 24 + b), uv[b], t);
        s = fma(lv[a], t, s);
    }
    dmu[e] = -s;
}

// ---- control of the graph-driven PCG (single thread each) ----
// Before the loop: ||f|| from scal[S_TMP]; the loop runs only for f != 0.
__global__ void loop_init_kernel(CgCtl* ctl, double* scal, double* hist, cudaGraphConditionalHandle cond) {
    const double fn = sqrt(scal[S_TMP]);
    ctl->fn = fn;
    ctl->it = 0;
    ctl->restarts = 0;
    ctl->check = 0;
    ctl->first = 1;
    ctl->restart_now = 0;
    ctl->need_final = 0;
    ctl->true_rel = 0.0;
    ctl->seg_start[0] = 0;
    scal[S_FLAG] = 0.0;
    ctl->state = fn > 0.0 ? CG_RUN : (fn == fn ? CG_ZERO : CG_NANRHS);
    hist[0] = fn > 0.0 ? 1.0 : 0.0;
    cudaGraphSetConditional(cond, ctl->state == CG_RUN ? 1u : 0u);
}

// After the u/r update: record alpha_j, beta_j and ||r|| / ||f||; breakdown
// ends the loop; a recurrence residual at or below tol asks for the true one.
__global__ void loop_decide_recurrence_kernel(CgCtl* ctl, const double* scal, double* hist, double* alpha,
                                              double* beta) {
    const int it = ++ctl->it;
    alpha[it - 1] = scal[S_ALPHA];
    beta[it - 1] = scal[S_BETA];     // 0 at the start of a segment
    ctl->first = 0;
    ctl->restart_now = 0;
    ctl->check = 0;
    if (scal[S_FLAG] != 0.0) {
        ctl->state = CG_BREAKDOWN;
        ctl->need_final = 1;
        return;
    }
    const double rel = sqrt(scal[S_RR]) / ctl->fn;
    hist[it] = rel;
    if (rel <= ctl->tol) ctl->check = 1;
    else if (it >= ctl->maxit) {
        ctl->state = CG_MAXIT;
        ctl->need_final = 1;
    }
}

// After the true residual (when asked for): accept, give up after the last
// restart, or restart CG from the true residual; then the loop condition.
__global__ void loop_decide_true_kernel(CgCtl* ctl, const double* scal, const int* errflag,
                                        cudaGraphConditionalHandle cond) {
    if (*errflag) {
        // a bounded wait of a local solve ran out: the iterate is not valid
        ctl->state = CG_TIMEOUT;
        cudaGraphSetConditional(cond, 0u);
        return;
    }
    if (ctl->check) {
        const double tr = sqrt(scal[S_TMP]) / ctl->fn;
        ctl->true_rel = tr;
        if (tr <= ctl->tol) {
            ctl->state = CG_CONV;
        } else if (ctl->restarts >= DDG_MAX_RESTARTS) {
            ctl->state = CG_STALLED;
        } else {
            ctl->seg_start[++ctl->restarts] = ctl->it;
            ctl->first = 1;
            ctl->restart_now = 1;
            if (ctl->it >= ctl->maxit) ctl->state = CG_MAXIT;
        }
    }
    cudaGraphSetConditional(cond, ctl->state == CG_RUN ? 1u : 0u);
}

__global__ void loop_final_kernel(CgCtl* ctl, const double* scal) {
    if (ctl->need_final) ctl->true_rel = sqrt(scal[S_TMP]) / ctl->fn;
}

inline unsigned red_grid(int64_t n) {
    int64_t b = (n + RT - 1) / RT;
    if (b > DDG_RED_BLOCKS) b = DDG_RED_BLOCKS;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

namespace ddg {

void spmv64(ddg_handle h, const double* x, double* y, bool dot, int /*slot*/) {
    const unsigned G = red_grid(h->n);
    const int sk = h->stencil_kind;
    if (sk == DDG_STENCIL_7PT_3D) {
        if (dot) spmv_lap64_kernel<true, 3><<<G, RT, 0, h->stream>>>(h->nx, h->ny, h->nz, x, y, h->red_partials, h->red_counter, h->scal);
        else spmv_lap64_kernel<false, 3><<<G, RT, 0, h->stream>>>(h->nx, h->ny, h->nz, x, y, h->red_partials, h->red_counter, h->scal);
    } else if (sk == DDG_STENCIL_5PT_2D) {
        if (dot) spmv_lap64_kernel<true, 2><<<G, RT, 0, h->stream>>>(h->nx, h->ny, 1, x, y, h->red_partials, h->red_counter, h->scal);
        else spmv_lap64_kernel<false, 2><<<G, RT, 0, h->stream>>>(h->nx, h->ny, 1, x, y, h->red_partials, h->red_counter, h->scal);
    } else {
        auto kern = h->wide_rows ? (dot ? spmv_csr64_kernel<true, ddgdev::CSRW_G> : spmv_csr64_kernel<false, ddgdev::CSRW_G>)
                                 : (dot ? spmv_csr64_kernel<true, 1> : spmv_csr64_kernel<false, 1>);
        kern<<<G, RT, 0, h->stream>>>(h->n, h->rowptr, h->col, h->val64, x, y, h->red_partials, h->red_counter, h->scal);
    }
    DDG_CHECK_LAUNCH();
}

void dot64(ddg_handle h, const double* a, const double* b, int slot, const int* gate) {
    dot64_kernel<<<red_grid(h->n), RT, 0, h->stream>>>(h->n, a, b, h->red_partials, h->red_counter,
                                                       h->scal, slot, gate);
    DDG_CHECK_LAUNCH();
}

void loop_init(ddg_handle h, cudaGraphConditionalHandle cond) {
    loop_init_kernel<<<1, 1, 0, h->stream>>>(h->ctl, h->scal, h->d_hist, cond);
    DDG_CHECK_LAUNCH();
}

void loop_decide_recurrence(ddg_handle h) {
    loop_decide_recurrence_kernel<<<1, 1, 0, h->stream>>>(h->ctl, h->scal, h->d_hist, h->d_alpha, h->d_beta);
    DDG_CHECK_LAUNCH();
}

void loop_decide_true(ddg_handle h, cudaGraphConditionalHandle cond) {
    loop_decide_true_kernel<<<1, 1, 0, h->stream>>>(h->ctl, h->scal, h->errflags + E_TIMEOUT, cond);
    DDG_CHECK_LAUNCH();
}

void loop_final(ddg_handle h) {
    loop_final_kernel<<<1, 1, 0, h->stream>>>(h->ctl, h->scal);
    DDG_CHECK_LAUNCH();
}

void copy_gated(ddg_handle h, const double* src, double* dst, const int* gate) {
    copy_gated_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->n, src, dst, gate);
    DDG_CHECK_LAUNCH();
}

void cg_update_ur(ddg_handle h) {
    cg_update_ur_kernel<<<red_grid(h->n), RT, 0, h->stream>>>(h->n, h->u, h->r, h->p, h->q,
                                                              h->red_partials, h->red_counter, h->scal);
    DDG_CHECK_LAUNCH();
}

void cg_dots_after_precond(ddg_handle h, int prec, bool first, int pr, const int* firstp) {
    if (prec == DDG_PREC_FP64)
        cg_dots_kernel<double><<<red_grid(h->n), RT, 0, h->stream>>>(h->n, h->r, h->q, h->z64, first, pr,
                                                                     h->red_partials, h->red_counter, h->scal,
                                                                     firstp);
    else
        cg_dots_kernel<float><<<red_grid(h->n), RT, 0, h->stream>>>(h->n, h->r, h->q, h->z32, first, pr,
                                                                    h->red_partials, h->red_counter, h->scal,
                                                                    firstp);
    DDG_CHECK_LAUNCH();
}

void cg_update_p(ddg_handle h, int prec, bool first, const int* firstp) {
    const unsigned G = red_grid(h->n);
    if (prec == DDG_PREC_FP64)
        cg_update_p_kernel<double><<<G, RT, 0, h->stream>>>(h->n, h->p, h->z64, h->scal, first, firstp);
    else
        cg_update_p_kernel<float><<<G, RT, 0, h->stream>>>(h->n, h->p, h->z32, h->scal, first, firstp);
    DDG_CHECK_LAUNCH();
}

void residual64(ddg_handle h, const double* f, const double* u, double* r, const int* gate) {
    residual64_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->n, h->rowptr, h->col,
                                                                             h->val64, f, u, r, gate);
    DDG_CHECK_LAUNCH();
}

void convert_to_float(ddg_handle h, const double* src, float* dst) {
    to_float_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->n, src, dst);
    DDG_CHECK_LAUNCH();
}

void convert_to_double(ddg_handle h, const float* src, double* dst) {
    to_double_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->n, src, dst);
    DDG_CHECK_LAUNCH();
}

void set_scalar(ddg_handle h, int slot, double v) {
    set_scalar_kernel<<<1, 1, 0, h->stream>>>(h->scal, slot, v);
    DDG_CHECK_LAUNCH();
}

void strided_gather(ddg_handle h, const double* src, int m, int j, double* dst) {
    strided_gather_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->n, src, m, j, dst);
    DDG_CHECK_LAUNCH();
}

void strided_scatter(ddg_handle h, const double* src, int m, int j, double* dst) {
    strided_scatter_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->n, src, m, j, dst);
    DDG_CHECK_LAUNCH();
}

void cast_q32(ddg_handle h) {
    const int64_t cnt = h->n * (int64_t)h->kmax;
    cast_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, h->stream>>>(cnt, h->Q64, h->Q32);
    DDG_CHECK_LAUNCH();
}

void grad_coeff_q1(ddg_handle h, const double* lambda, const double* u, double* dk) {
    const int ne = h->nx;
    const int64_t ncell = (int64_t)ne * ne * ne;
    grad_q1_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, h->stream>>>(ne, h->kmu, lambda, u, dk);
    DDG_CHECK_LAUNCH();
}

void grad_coeff_var7(ddg_handle h, const double* lambda, const double* u, double* dk) {
    grad_var7_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(
        h->nx, h->ny, h->nz, h->kappa, lambda, u, dk);
    DDG_CHECK_LAUNCH();
}

}  // namespace ddg
