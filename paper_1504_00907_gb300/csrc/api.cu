// C ABI entry points of the DDG solver: setup orchestration (host graph
// work + device numerics) and the PCG driver (Sec. 7).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <string>
#include <vector>

#include "ddg_internal.cuh"


namespace {

thread_local std::string g_setup_error;

void drop_graphs(ddg_handle h);

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------- host graph work
// Sec. 6: Omega~_i = all dofs within distance Delta of Omega_i, in the graph of
// A (GRAPH) or in the L-infinity neighbour graph of the grid nodes (BOX).
void grow_overlaps(const ddg_matrix* A, const std::vector<int64_t>& sub_off,
                   const std::vector<int32_t>& sub_nodes, int nsub, int delta, int mode,
                   std::vector<std::vector<int32_t>>& out) {
    const int64_t n = A->n;
    out.assign(nsub, {});
    std::vector<int32_t> stamp(n, -1);
    std::vector<int32_t> frontier, next;
    const int dpn = A->dofs_per_node > 0 ? A->dofs_per_node : 1;
    const int nx = A->nx, ny = A->ny, nz = A->dim == 3 ? A->nz : 1;
    for (int s = 0; s < nsub; ++s) {
        std::vector<int32_t>& om = out[s];
        frontier.clear();
        for (int64_t a = sub_off[s]; a < sub_off[s + 1]; ++a) {
            const int32_t g = sub_nodes[a];
            stamp[g] = s;
            om.push_back(g);
            frontier.push_back(g);
        }
        for (int layer = 0; layer < delta; ++layer) {
            next.clear();
            for (int32_t g : frontier) {
                if (mode == DDG_OVERLAP_GRAPH) {
                    for (int64_t e = A->rowptr[g]; e < A->rowptr[g + 1]; ++e) {
                        const int32_t c = A->col[e];
                        if (stamp[c] != s) {
                            stamp[c] = s;
                            om.push_back(c);
                            next.push_back(c);
                        }
                    }
                } else {
                    const int64_t node = g / dpn;
                    const int i = (int)(node % nx), j = (int)((node / nx) % ny), k = (int)(node / ((int64_t)nx * ny));
                    for (int dk = (A->dim == 3 ? -1 : 0); dk <= (A->dim == 3 ? 1 : 0); ++dk)
                        for (int dj = -1; dj <= 1; ++dj)
                            for (int di = -1; di <= 1; ++di) {
                                const int ii = i + di, jj = j + dj, kk = k + dk;
                                if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
                                const int64_t nb = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
                                for (int c = 0; c < dpn; ++c) {
                                    const int32_t d = (int32_t)(nb * dpn + c);
                                    if (stamp[d] != s) {
                                        stamp[d] = s;
                                        om.push_back(d);
                                        next.push_back(d);
                                    }
                                }
                            }
                }
            }
            frontier.swap(next);
        }
        std::sort(om.begin(), om.end());
    }
}

// Subdomains (in sweep position q) whose local matrices A[ov, ov] (rows and
// columns in ascending dof order) are equal entry for entry: rep[q] is the
// first such position, rep[q] == q for the ones that keep their own inverse.
std::vector<int32_t> identical_locals(const ddg_matrix* A, const std::vector<std::vector<int32_t>>& ov,
                                      const std::vector<int>& sid) {
    const int nsub = (int)sid.size();
    std::vector<int32_t> rep(nsub), loc(A->n, -1);
    std::vector<int64_t> ki, kr;
    std::vector<double> kv, kvr;
    // canonical form: size, then per row the (local column, value) pairs in CSR order
    auto key = [&](int q, std::vector<int64_t>& kidx, std::vector<double>& kval) {
        const std::vector<int32_t>& idx = ov[sid[q]];
        for (size_t r = 0; r < idx.size(); ++r) loc[idx[r]] = (int32_t)r;
        kidx.assign(1, (int64_t)idx.size());
        kval.clear();
        for (size_t r = 0; r < idx.size(); ++r) {
            for (int64_t e = A->rowptr[idx[r]]; e < A->rowptr[idx[r] + 1]; ++e) {
                const int32_t c = loc[A->col[e]];
                if (c < 0) continue;
                kidx.push_back(((int64_t)r << 32) | (uint32_t)c);
                kval.push_back(A->val[e]);
            }
            kidx.push_back(-1);
        }
        for (int32_t g : idx) loc[g] = -1;
        uint64_t hsh = 1469598103934665603ull;   // FNV-1a over the bytes of the key
        auto mix = [&](const void* p, size_t bytes) {
            const unsigned char* b = static_cast<const unsigned char*>(p);
            for (size_t i = 0; i < bytes; ++i) hsh = (hsh ^ b[i]) * 1099511628211ull;
        };
        mix(kidx.data(), kidx.size() * sizeof(int64_t));
        mix(kval.data(), kval.size() * sizeof(double));
        return hsh;
    };
    std::unordered_map<uint64_t, std::vector<int32_t>> seen;
    for (int q = 0; q < nsub; ++q) {
        const uint64_t hq = key(q, ki, kv);
        rep[q] = q;
        std::vector<int32_t>& cands = seen[hq];
        for (int32_t r : cands) {
            key(r, kr, kvr);
            if (kr == ki && kvr.size() == kv.size() &&
                std::memcmp(kvr.data(), kv.data(), kv.size() * sizeof(double)) == 0) {
                rep[q] = r;
                break;
            }
        }
        if (rep[q] == q) cands.push_back(q);
    }
    return rep;
}

// greedy colouring in id order: i and j conflict when Omega~_j meets the
// one-step neighbourhood of Omega~_i in the graph of A
std::vector<int> colour_subdomains(const ddg_matrix* A, const std::vector<std::vector<int32_t>>& ov) {
    const int64_t n = A->n;
    const int nsub = (int)ov.size();
    std::vector<int64_t> own_off(n + 1, 0);
    for (const auto& o : ov)
        for (int32_t g : o) own_off[g + 1]++;
    for (int64_t g = 0; g < n; ++g) own_off[g + 1] += own_off[g];
    std::vector<int32_t> owners(own_off[n]);
    std::vector<int64_t> fill(own_off.begin(), own_off.end() - 1);
    for (int s = 0; s < nsub; ++s)
        for (int32_t g : ov[s]) owners[fill[g]++] = s;
    std::vector<int> colour(nsub, -1), used;
    std::vector<int32_t> seen(nsub, -1);
    for (int i = 0; i < nsub; ++i) {
        std::vector<int> nbcol;
        auto visit = [&](int32_t c) {
            for (int64_t t = own_off[c]; t < own_off[c + 1]; ++t) {
                const int j = owners[t];
                if (j < i && seen[j] != i) {
                    seen[j] = i;
                    nbcol.push_back(colour[j]);
                }
            }
        };
        for (int32_t g : ov[i]) {
            visit(g);
            for (int64_t e = A->rowptr[g]; e < A->rowptr[g + 1]; ++e) visit(A->col[e]);
        }
        std::sort(nbcol.begin(), nbcol.end());
        int c = 0;
        for (int v : nbcol) {
            if (v == c) ++c;
            else if (v > c) break;
        }
        colour[i] = c;
    }
    return colour;
}

// dK_e / dmu_e of trilinear hexahedral elasticity on a cube of side h: the
// shear part of the bilinear form int lam div u div v + 2 mu eps(u):eps(v),
// i.e. h * int_[0,1]^3 (delta_ij grad N_a . grad N_b + d_j N_a d_i N_b),
// integrated exactly by 2x2x2 Gauss points; local dof 3 a + i, node
// a = (a & 1, (a >> 1) & 1, a >> 2)
std::vector<double> q1_dk_dmu(double h) {
    std::vector<double> K(576, 0.0);
    const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    for (double x : gp)
        for (double y : gp)
            for (double z : gp) {
                const double xi[3] = {x, y, z};
                double grad[8][3];
                for (int a = 0; a < 8; ++a) {
                    const int bits[3] = {a & 1, (a >> 1) & 1, a >> 2};
                    double f[3], df[3];
                    for (int d = 0; d < 3; ++d) {
                        f[d] = bits[d] ? xi[d] : 1.0 - xi[d];
                        df[d] = bits[d] ? 1.0 : -1.0;
                    }
                    grad[a][0] = df[0] * f[1] * f[2];
                    grad[a][1] = f[0] * df[1] * f[2];
                    grad[a][2] = f[0] * f[1] * df[2];
                }
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b) {
                        const double gg = grad[a][0] * grad[b][0] + grad[a][1] * grad[b][1] + grad[a][2] * grad[b][2];
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j)
                                K[(3 * a + i) * 24 + 3 * b + j] +=
                                    0.125 * h * ((i == j ? gg : 0.0) + grad[a][j] * grad[b][i]);
                    }
            }
    return K;
}

void validate(const ddg_matrix* A, const int32_t* part, const double* F, int k, int overlap,
              const ddg_options& o) {
    DDG_REQUIRE(A && A->rowptr && A->col && A->val, DDG_EINVAL, "A and its CSR arrays must be non-null");
    DDG_REQUIRE(A->n > 0 && A->n < (int64_t)INT32_MAX, DDG_EINVAL, "n must be in [1, 2^31)");
    DDG_REQUIRE(A->rowptr[0] == 0, DDG_EINVAL, "rowptr[0] must be 0");
    for (int64_t g = 0; g < A->n; ++g)
        DDG_REQUIRE(A->rowptr[g + 1] >= A->rowptr[g], DDG_EINVAL, "rowptr must be non-decreasing");
    const int64_t nnz = A->rowptr[A->n];
    for (int64_t e = 0; e < nnz; ++e)
        DDG_REQUIRE(A->col[e] >= 0 && A->col[e] < A->n, DDG_EINVAL, "column index out of range");
    DDG_REQUIRE(part, DDG_EINVAL, "partition must be non-null");
    for (int64_t g = 0; g < A->n; ++g)
        DDG_REQUIRE(part[g] >= 0 && part[g] < INT32_MAX, DDG_EINVAL, "partition ids must be >= 0");
    DDG_REQUIRE(overlap >= 0, DDG_EINVAL, "overlap must be >= 0");
    DDG_REQUIRE(o.precision >= DDG_PREC_FP64 && o.precision <= DDG_PREC_BF16, DDG_EINVAL, "bad precision");
    DDG_REQUIRE(o.overlap_mode == DDG_OVERLAP_GRAPH || o.overlap_mode == DDG_OVERLAP_BOX, DDG_EINVAL,
                "bad overlap_mode");
    if (o.overlap_mode == DDG_OVERLAP_BOX) {
        DDG_REQUIRE(A->dim == 2 || A->dim == 3, DDG_EINVAL, "BOX overlap needs dim 2 or 3");
        const int64_t nodes = (int64_t)A->nx * A->ny * (A->dim == 3 ? A->nz : 1);
        const int dpn = A->dofs_per_node > 0 ? A->dofs_per_node : 1;
        DDG_REQUIRE(nodes * dpn == A->n, DDG_EINVAL, "grid shape * dofs_per_node must equal n");
    }
    if (A->stencil_kind == DDG_STENCIL_7PT_3D || A->stencil_kind == DDG_STENCIL_VAR7_3D)
        DDG_REQUIRE((int64_t)A->nx * A->ny * A->nz == A->n, DDG_EINVAL, "3D stencil shape must match n");
    if (A->stencil_kind == DDG_STENCIL_5PT_2D || A->stencil_kind == DDG_STENCIL_13PT_2D)
        DDG_REQUIRE((int64_t)A->nx * A->ny == A->n, DDG_EINVAL, "2D stencil shape must match n");
    if (o.use_coarse) {
        DDG_REQUIRE(F, DDG_EINVAL, "F must be non-null for the two-level method");
        DDG_REQUIRE(k >= 1 && k <= DDG_KMAX, DDG_EINVAL, "k must be in [1, 96]");
    }
    DDG_REQUIRE(o.maxit >= 1, DDG_EINVAL, "maxit must be >= 1");
    DDG_REQUIRE(o.spin_budget_ms >= 0.0 && o.spin_budget_ms <= 3.6e6, DDG_EINVAL,
                "spin_budget_ms must be in [0, 3.6e6]");
    DDG_REQUIRE(o.local_repr >= DDG_LOCAL_AUTO && o.local_repr <= DDG_LOCAL_BAND, DDG_EINVAL, "bad local_repr");
    DDG_REQUIRE(o.tensor_cores >= DDG_TC_OFF && o.tensor_cores <= DDG_TC_TF32, DDG_EINVAL, "bad tensor_cores");
    DDG_REQUIRE(o.coarse_order == DDG_COARSE_BAND || o.coarse_order == DDG_COARSE_ND, DDG_EINVAL,
                "bad coarse_order");
}

// ---------------------------------------------------------------- preconditioner
void local_step(ddg_handle h, int c, bool z_zero, int prec) {
    {
        ProfScope ps(h, DDG_K_LOCAL_RESIDUAL, 1, 0.0);
        ddg::local_residual(h, c, z_zero, prec);
    }
    ProfScope ps(h, DDG_K_LOCAL_SOLVE, 1, h->colour_bytes[prec][c]);
    ddg::local_solve_colour(h, c, prec);
}

int64_t coarse_vcycle(ddg_handle h, int prec);

void coarse_step(ddg_handle h, int prec, bool residual) {
    ProfScope ps(h, DDG_K_COARSE, h->inner ? 2 : 2 + (h->nd.on ? ddg::nd_solve_launches(h) : 2 * h->nK), 0.0);
    ddg::coarse_restrict(h, prec, residual);
    if (h->inner) h->prof_launches[DDG_K_COARSE] += coarse_vcycle(h, prec);
    else ddg::coarse_solve(h, prec);
    ddg::coarse_prolong(h, prec);
}

// One symmetric two-level step from z = 0 on the input already in rin64
// (FP64) or r32, z already zeroed (Sec. 6).
void sweeps_and_coarse(ddg_handle h, int prec) {
    // pre-smoother: one multiplicative pass in sweep order
    for (int c = 0; c < h->ncol; ++c) local_step(h, c, c == 0, prec);
    // coarse correction of the current residual
    if (h->use_coarse) coarse_step(h, prec, true);
    // post-smoother: the same pass in reverse order
    for (int c = h->ncol - 1; c >= 0; --c) local_step(h, c, false, prec);
}

// Sec. 6, three-level V-cycle: x = B0 c, one application of the two-level
// preconditioner of A0 to the restricted residual c, enqueued on this
// handle's stream.  The inner handle reads c (c64 in place, c32 as its r32)
// and leaves B0 c in x (its z64 / z32).  Returns the inner kernel launches.
int64_t coarse_vcycle(ddg_handle h, int prec) {
    ddg_handle in = h->inner;
    int64_t before = 0, after = 0;
    for (int c = 0; c < DDG_K_COUNT; ++c) before += in->prof_launches[c];
    in->stream = h->stream;
    if (prec == DDG_PREC_FP64) {
        in->rin64 = h->c64;
        DDG_CUDA(cudaMemsetAsync(in->z64, 0, in->n * sizeof(double), h->stream));
    } else {
        DDG_CUDA(cudaMemsetAsync(in->z32, 0, in->n * sizeof(float), h->stream));
    }
    sweeps_and_coarse(in, prec);
    for (int c = 0; c < DDG_K_COUNT; ++c) after += in->prof_launches[c];
    return after - before;
}

void apply_prec(ddg_handle h, const double* rin) {
    const int prec = h->precision;
    if (prec == DDG_PREC_FP64) {
        h->rin64 = rin;
        DDG_CUDA(cudaMemsetAsync(h->z64, 0, h->n * sizeof(double), h->stream));
    } else {
        ProfScope ps(h, DDG_K_CG, 1, 0.0);
        ddg::convert_to_float(h, rin, h->r32);
        DDG_CUDA(cudaMemsetAsync(h->z32, 0, h->n * sizeof(float), h->stream));
    }
    sweeps_and_coarse(h, prec);
}

// The preconditioner of the PCG loop always reads h->r, so its launch
// sequence is fixed per precision: capture it once into a CUDA graph (on a
// private non-blocking stream: the caller's stream may be the legacy default
// stream, which cannot be captured) and replay it on the caller's stream.
// Per-kernel event timing (ddg_profile) needs the individual launches, so it
// bypasses the graph.
void apply_in_pcg(ddg_handle h) {
    const int p = h->precision;
    if (!h->use_graphs || h->prof_mask != 0) {
        apply_prec(h, h->r);
        return;
    }
    if (!h->apply_exec[p]) {
        if (!h->cap_stream) DDG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        int64_t saved_counts[DDG_K_COUNT];
        for (int c = 0; c < DDG_K_COUNT; ++c) saved_counts[c] = h->prof_launches[c];
        cudaStream_t saved = h->stream;
        // order the capture after earlier work of the handle
        DDG_CUDA(cudaStreamSynchronize(saved));
        h->stream = h->cap_stream;
        DDG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t g = nullptr;
        try {
            apply_prec(h, h->r);
        } catch (...) {
            cudaStreamEndCapture(h->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            h->stream = saved;
            throw;
        }
        const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        h->stream = saved;
        DDG_CUDA(e);
        const cudaError_t ei = cudaGraphInstantiate(&h->apply_exec[p], g, 0);
        cudaGraphDestroy(g);
        DDG_CUDA(ei);
        for (int c = 0; c < DDG_K_COUNT; ++c) {
            h->apply_launches[p][c] = h->prof_launches[c] - saved_counts[c];
            h->prof_launches[c] = saved_counts[c];
        }
    }
    DDG_CUDA(cudaGraphLaunch(h->apply_exec[p], h->stream));
    for (int c = 0; c < DDG_K_COUNT; ++c) h->prof_launches[c] += h->apply_launches[p][c];
}

// the CG scalars, and the timeout flag of the bounded waits of the local
// solves (a solve whose wait ran out stops with DDG_ETIMEOUT)
void read_scalars(ddg_handle h) {
    int32_t timed_out = 0;
    d2h(h->h_scal, h->scal, S_COUNT, h->stream);
    d2h(&timed_out, h->errflags + E_TIMEOUT, 1, h->stream);
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    if (timed_out) {
        DDG_CUDA(cudaMemsetAsync(h->errflags + E_TIMEOUT, 0, sizeof(int32_t), h->stream));
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        throw DdgError{DDG_ETIMEOUT, "a bounded wait of a local solve ran out"};
    }
}

// PCG from u = 0 (Sec. 7), driven from the host (two reads of the device
// scalars per iteration).  Returns the status; u, history, iters, relres set.
ddg_status pcg_host(ddg_handle h, const double* f, double* u, double tol, int* iters_out, double* relres_out) {
    const int prec = h->precision;
    const int beta = h->opt.beta == DDG_BETA_AUTO ? (prec == DDG_PREC_FP64 ? DDG_BETA_FR : DDG_BETA_PR)
                                                  : h->opt.beta;
    const int pr = beta == DDG_BETA_PR;
    h->history.clear();
    for (auto* v : {&h->cg_alpha, &h->cg_beta, &h->seg_alpha, &h->seg_beta}) v->clear();
    // a true-residual restart starts a new Lanczos sequence: keep the longest
    auto keep_segment = [&]() {
        if (h->seg_alpha.size() > h->cg_alpha.size()) {
            h->cg_alpha.swap(h->seg_alpha);
            h->cg_beta.swap(h->seg_beta);
        }
        h->seg_alpha.clear();
        h->seg_beta.clear();
    };
    {
        ProfScope ps(h, DDG_K_CG, 1, 0.0);
        ddg::dot64(h, f, f, S_TMP);
    }
    read_scalars(h);
    const double fn = std::sqrt(h->h_scal[S_TMP]);
    DDG_CUDA(cudaMemsetAsync(u, 0, h->n * sizeof(double), h->stream));
    if (!(fn > 0.0)) {
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = 0.0;
        h->history.push_back(0.0);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return fn == fn ? DDG_OK : DDG_EINVAL;
    }
    h->history.push_back(1.0);
    h->u = u;
    {
        ProfScope ps(h, DDG_K_CG, 1, 0.0);
        ddg::set_scalar(h, S_FLAG, 0.0);
    }
    DDG_CUDA(cudaMemcpyAsync(h->r, f, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    auto restart = [&]() {
        keep_segment();
        apply_in_pcg(h);
        ProfScope ps(h, DDG_K_CG, 2, 0.0);
        ddg::cg_dots_after_precond(h, prec, true, pr);
        ddg::cg_update_p(h, prec, true);
    };
    restart();
    int it = 0, restarts = 0;
    ddg_status st = DDG_ENOCONV;
    double true_rel = -1.0;
    while (it < h->opt.maxit) {
        {
            ProfScope ps(h, DDG_K_SPMV, 1, 0.0);
            ddg::spmv64(h, h->p, h->q, true, S_PQ);
        }
        {
            ProfScope ps(h, DDG_K_CG, 1, 0.0);
            ddg::cg_update_ur(h);
        }
        read_scalars(h);
        ++it;
        if (h->h_scal[S_FLAG] != 0.0) {
            st = DDG_EBREAKDOWN;
            break;
        }
        // Sec. 7: the coefficients of the Lanczos tridiagonal; the beta read
        // here formed the current p
        if (!h->seg_alpha.empty()) h->seg_beta.push_back(h->h_scal[S_BETA]);
        h->seg_alpha.push_back(h->h_scal[S_ALPHA]);
        const double rel = std::sqrt(h->h_scal[S_RR]) / fn;
        h->history.push_back(rel);
        if (rel <= tol) {
            // verify against the true residual; replace and restart if the
            // recurrence has drifted
            {
                ProfScope ps(h, DDG_K_CG, 2, 0.0);
                ddg::residual64(h, f, u, h->q);
                ddg::dot64(h, h->q, h->q, S_TMP);
            }
            read_scalars(h);
            true_rel = std::sqrt(h->h_scal[S_TMP]) / fn;
            if (true_rel <= tol || restarts >= 3) {
                st = true_rel <= tol ? DDG_OK : DDG_ENOCONV;
                if (st != DDG_OK)
                    h->err = "the recurrence residual met tol but the true residual stayed above it "
                             "after 3 restarts of CG from the true residual";
                break;
            }
            DDG_CUDA(cudaMemcpyAsync(h->r, h->q, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
            ++restarts;
            restart();
            true_rel = -1.0;
            continue;
        }
        apply_in_pcg(h);
        ProfScope ps(h, DDG_K_CG, 2, 0.0);
        ddg::cg_dots_after_precond(h, prec, false, pr);
        ddg::cg_update_p(h, prec, false);
    }
    if (st == DDG_ENOCONV && h->err.empty()) h->err = "maxit iterations reached";
    if (true_rel < 0.0) {
        ProfScope ps(h, DDG_K_CG, 2, 0.0);
        ddg::residual64(h, f, u, h->q);
        ddg::dot64(h, h->q, h->q, S_TMP);
        read_scalars(h);
        true_rel = std::sqrt(h->h_scal[S_TMP]) / fn;
    }
    keep_segment();
    h->u = nullptr;
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = true_rel;
    return st;
}

// ---------------------------------------------------------------- graph-driven PCG
// The whole solve of Sec. 7 as one CUDA graph: ||f|| and the start (u = 0,
// r = f), a conditional WHILE node whose body is one CG iteration (the
// preconditioner apply, the dots and p update, the SpMV and u/r update, and
// the control kernels that record alpha_j, beta_j and ||r_k||, check the
// true residual once the recurrence meets tol and restart CG from it), and
// the true residual after a loop that ended without one.  The graph reads
// f from h->fbuf and writes u to h->ubuf; the host reads the outcome once.

void ensure_loop_buffers(ddg_handle h) {
    if (h->ctl) return;
    h->ctl = h->arena.alloc<CgCtl>(1);
    DDG_CUDA(cudaMallocHost((void**)&h->h_ctl, sizeof(CgCtl)));
    std::memset(h->h_ctl, 0, sizeof(CgCtl));
    const size_t len = (size_t)h->opt.maxit + 1;
    h->d_hist = h->arena.alloc<double>(len);
    h->d_alpha = h->arena.alloc<double>(len);
    h->d_beta = h->arena.alloc<double>(len);
}

// one CG iteration (from the preconditioner apply to the loop condition),
// enqueued on h->stream
void loop_body(ddg_handle h, int prec, int pr, cudaGraphConditionalHandle cond) {
    const int* firstp = &h->ctl->first;
    apply_prec(h, h->r);
    {
        ProfScope ps(h, DDG_K_CG, 2, 0.0);
        ddg::cg_dots_after_precond(h, prec, false, pr, firstp);
        ddg::cg_update_p(h, prec, false, firstp);
    }
    {
        ProfScope ps(h, DDG_K_SPMV, 1, 0.0);
        ddg::spmv64(h, h->p, h->q, true, S_PQ);
    }
    ProfScope ps(h, DDG_K_CG, 6, 0.0);
    ddg::cg_update_ur(h);
    ddg::loop_decide_recurrence(h);
    ddg::residual64(h, h->fbuf, h->ubuf, h->q, &h->ctl->check);
    ddg::dot64(h, h->q, h->q, S_TMP, &h->ctl->check);
    ddg::loop_decide_true(h, cond);
    ddg::copy_gated(h, h->q, h->r, &h->ctl->restart_now);
}

// Append the whole solve of h (current precision) to graph g as one branch
// with no dependencies: captured on the handle's private streams.
void capture_solve_branch(ddg_handle h, cudaGraph_t g) {
    const int prec = h->precision;
    const int beta = h->opt.beta == DDG_BETA_AUTO ? (prec == DDG_PREC_FP64 ? DDG_BETA_FR : DDG_BETA_PR)
                                                  : h->opt.beta;
    const int pr = beta == DDG_BETA_PR;
    ensure_loop_buffers(h);
    if (!h->cap_stream) DDG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (!h->cap_stream2) DDG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream, bs = h->cap_stream2;
    cudaStream_t saved = h->stream;
    int64_t c0[DDG_K_COUNT], c1[DDG_K_COUNT], c2[DDG_K_COUNT];
    for (int c = 0; c < DDG_K_COUNT; ++c) c0[c] = h->prof_launches[c];
    bool in_main = false, in_body = false;
    try {
        DDG_CUDA(cudaStreamSynchronize(saved));
        h->stream = cs;
        h->u = h->ubuf;
        DDG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        in_main = true;
        {
            ProfScope ps(h, DDG_K_CG, 1, 0.0);
            ddg::dot64(h, h->fbuf, h->fbuf, S_TMP);
        }
        DDG_CUDA(cudaMemsetAsync(h->ubuf, 0, h->n * sizeof(double), cs));
        DDG_CUDA(cudaMemcpyAsync(h->r, h->fbuf, h->n * sizeof(double), cudaMemcpyDeviceToDevice, cs));
        cudaGraphConditionalHandle cond;
        DDG_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
        {
            ProfScope ps(h, DDG_K_CG, 1, 0.0);
            ddg::loop_init(h, cond);
        }
        cudaStreamCaptureStatus cst;
        cudaGraph_t capg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        DDG_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &nd));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        DDG_CUDA(cudaGraphAddNode(&wnode, capg, deps, nullptr, nd, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        for (int c = 0; c < DDG_K_COUNT; ++c) c1[c] = h->prof_launches[c];
        h->stream = bs;
        DDG_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        in_body = true;
        loop_body(h, prec, pr, cond);
        cudaGraph_t bout = nullptr;
        in_body = false;
        DDG_CUDA(cudaStreamEndCapture(bs, &bout));
        for (int c = 0; c < DDG_K_COUNT; ++c) c2[c] = h->prof_launches[c];
        h->stream = cs;
        DDG_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        {
            ProfScope ps(h, DDG_K_CG, 3, 0.0);
            ddg::residual64(h, h->fbuf, h->ubuf, h->q, &h->ctl->need_final);
            ddg::dot64(h, h->q, h->q, S_TMP, &h->ctl->need_final);
            ddg::loop_final(h);
        }
        cudaGraph_t gout = nullptr;
        in_main = false;
        DDG_CUDA(cudaStreamEndCapture(cs, &gout));
    } catch (...) {
        cudaGraph_t junk = nullptr;
        if (in_body) cudaStreamEndCapture(bs, &junk);
        if (in_main) cudaStreamEndCapture(cs, &junk);
        cudaGetLastError();
        h->stream = saved;
        h->u = nullptr;
        for (int c = 0; c < DDG_K_COUNT; ++c) h->prof_launches[c] = c0[c];
        throw;
    }
    h->stream = saved;
    h->u = nullptr;
    for (int c = 0; c < DDG_K_COUNT; ++c) {
        h->solve_body_launches[prec][c] = c2[c] - c1[c];
        h->solve_pre_launches[prec][c] = (h->prof_launches[c] - c0[c]) - (c2[c] - c1[c]);
        h->prof_launches[c] = c0[c];
    }
}

// the instantiated whole-solve graph of the current precision, or nullptr
// when conditional graphs are not available (the host loop runs instead)
cudaGraphExec_t solve_graph(ddg_handle h) {
    const int p = h->precision;
    if (h->solve_exec[p] || h->solve_graph_failed) return h->solve_exec[p];
    cudaGraph_t g = nullptr;
    try {
        DDG_CUDA(cudaGraphCreate(&g, 0));
        capture_solve_branch(h, g);
        DDG_CUDA(cudaGraphInstantiate(&h->solve_exec[p], g, 0));
        cudaGraphDestroy(g);
    } catch (DdgError& e) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->solve_exec[p] = nullptr;
        h->solve_graph_failed = true;
        h->solve_graph_error = e.msg;
    }
    return h->solve_exec[p];
}

// outcome of a graph-driven solve from the device control block: history,
// CG coefficients (the longest restart segment), iterations, true residual
ddg_status loop_outcome(ddg_handle h, int* iters_out, double* relres_out) {
    const CgCtl& c = *h->h_ctl;
    std::vector<double> hist(c.it + 1), al(std::max(1, c.it)), be(std::max(1, c.it));
    d2h(hist.data(), h->d_hist, (size_t)c.it + 1, h->stream);
    if (c.it > 0) {
        d2h(al.data(), h->d_alpha, (size_t)c.it, h->stream);
        d2h(be.data(), h->d_beta, (size_t)c.it, h->stream);
    }
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    h->history.assign(hist.begin(), hist.end());
    h->cg_alpha.clear();
    h->cg_beta.clear();
    for (int s = 0; s <= c.restarts; ++s) {
        const int a = c.seg_start[s], b = s < c.restarts ? c.seg_start[s + 1] : c.it;
        if (b - a > (int)h->cg_alpha.size()) {
            h->cg_alpha.assign(al.begin() + a, al.begin() + b);
            h->cg_beta.assign(be.begin() + a + 1, be.begin() + b);
        }
    }
    for (int k = 0; k < DDG_K_COUNT; ++k)
        h->prof_launches[k] += h->solve_pre_launches[h->precision][k] +
                               (int64_t)c.it * h->solve_body_launches[h->precision][k];
    if (iters_out) *iters_out = c.it;
    if (relres_out) *relres_out = c.true_rel;
    h->last_solve_graph = 1;
    switch (c.state) {
        case CG_CONV:
        case CG_ZERO: return DDG_OK;
        case CG_BREAKDOWN: return DDG_EBREAKDOWN;
        case CG_MAXIT: h->err = "maxit iterations reached"; return DDG_ENOCONV;
        case CG_STALLED:
            h->err = "the recurrence residual met tol but the true residual stayed above it "
                     "after 3 restarts of CG from the true residual";
            return DDG_ENOCONV;
        case CG_NANRHS: h->err = "f contains NaN"; return DDG_EINVAL;
        case CG_TIMEOUT:
            DDG_CUDA(cudaMemsetAsync(h->errflags + E_TIMEOUT, 0, sizeof(int32_t), h->stream));
            DDG_CUDA(cudaStreamSynchronize(h->stream));
            h->err = "a bounded wait of a local solve ran out";
            return DDG_ETIMEOUT;
    }
    h->err = "graph-driven solve ended in an unknown state";
    return DDG_ECUDA;
}

// write tol and maxit into the control block (enqueued before the graph)
void loop_params(ddg_handle h, double tol) {
    h->h_ctl->tol = tol;
    h->h_ctl->maxit = h->opt.maxit;
    DDG_CUDA(cudaMemcpyAsync(h->ctl, h->h_ctl, sizeof(CgCtl), cudaMemcpyHostToDevice, h->stream));
}

// PCG from u = 0 (Sec. 7): one graph launch when available, else the host loop
ddg_status pcg(ddg_handle h, const double* f, double* u, double tol, int* iters_out, double* relres_out) {
    h->last_solve_graph = 0;
    if (!h->use_graphs || h->prof_mask != 0) return pcg_host(h, f, u, tol, iters_out, relres_out);
    cudaGraphExec_t ge = solve_graph(h);
    if (!ge) {
        // conditional graphs unavailable: the same solve, driven by the host
        const ddg_status st = pcg_host(h, f, u, tol, iters_out, relres_out);
        if (st == DDG_OK) h->err = "graph-driven solve unavailable: " + h->solve_graph_error;
        return st;
    }
    if (f != h->fbuf)
        DDG_CUDA(cudaMemcpyAsync(h->fbuf, f, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    loop_params(h, tol);
    DDG_CUDA(cudaGraphLaunch(ge, h->stream));
    if (u != h->ubuf)
        DDG_CUDA(cudaMemcpyAsync(u, h->ubuf, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    DDG_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(CgCtl), cudaMemcpyDeviceToHost, h->stream));
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    return loop_outcome(h, iters_out, relres_out);
}

void prof_flush(ddg_handle h) {
    if (h->ev_used == 0) return;
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < h->ev_used; ++i) {
        float ms = 0.f;
        DDG_CUDA(cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
        h->prof_ms[h->ev_class[i]] += ms;
        h->prof_bytes[h->ev_class[i]] += h->ev_bytes[i];
        h->prof_timed[h->ev_class[i]] += 1;
    }
    h->ev_used = 0;
}

// Batched PCG on an n x m block (m <= DDG_MCHUNK), FP32/BF16 preconditioner:
// every column runs its own CG (alpha, beta, convergence, restarts); the
// preconditioner is applied to all columns at once.  Driven from the host.
ddg_status pcg_batch_host(ddg_handle h, const double* F, double* U, int m, double tol, int* iters,
                          double* relres) {
    ddg::multi_ensure(h, m);
    MultiWork& w = h->mw;
    const int64_t n = h->n;
    const int beta = h->opt.beta == DDG_BETA_AUTO ? DDG_BETA_PR : h->opt.beta;
    const int pr = beta == DDG_BETA_PR;
    std::vector<double> sc(S_COUNT * DDG_MCHUNK);
    int32_t timed_out = 0;
    // the scalars of every column, and the timeout flag of the bounded waits
    // of the tensor-core local solve: a solve whose wait ran out stops here
    auto read_sc = [&]() {
        d2h(sc.data(), w.scal, sc.size(), h->stream);
        d2h(&timed_out, h->errflags + E_TIMEOUT, 1, h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        if (timed_out) {
            DDG_CUDA(cudaMemsetAsync(h->errflags + E_TIMEOUT, 0, sizeof(int32_t), h->stream));
            DDG_CUDA(cudaStreamSynchronize(h->stream));
            throw DdgError{DDG_ETIMEOUT, "a bounded wait of the tensor-core local solve ran out"};
        }
    };
    auto at = [&](int slot, int c) { return sc[slot * DDG_MCHUNK + c]; };
    DDG_CUDA(cudaMemsetAsync(w.scal, 0, S_COUNT * DDG_MCHUNK * sizeof(double), h->stream));
    ddg::multi_resnorm(h, m, F, nullptr, nullptr, S_TMP);
    read_sc();
    std::vector<double> fn(m);
    std::vector<int> active(DDG_MCHUNK, 0), restart(DDG_MCHUNK, 0), nrest(m, 0), done_it(m, -1);
    std::vector<double> done_rel(m, -1.0);
    std::vector<ddg_status> st(m, DDG_OK);
    for (int j = 0; j < m; ++j) {
        fn[j] = std::sqrt(at(S_TMP, j));
        active[j] = fn[j] > 0.0;
        restart[j] = 1;
        if (!active[j]) {
            done_it[j] = 0;
            done_rel[j] = 0.0;
        }
    }
    DDG_CUDA(cudaMemsetAsync(U, 0, n * m * sizeof(double), h->stream));
    DDG_CUDA(cudaMemsetAsync(w.P, 0, n * m * sizeof(double), h->stream));
    DDG_CUDA(cudaMemcpyAsync(w.R, F, n * m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    w.r32_current = false;
    auto upload = [&]() {
        h2d(w.active, active.data(), DDG_MCHUNK, h->stream);
        h2d(w.restart, restart.data(), DDG_MCHUNK, h->stream);
    };
    upload();
    auto precond_and_p = [&]() {
        ddg::multi_apply(h, m);
        ProfScope ps(h, DDG_K_CG, 2, 0.0);
        ddg::multi_dots(h, m, pr);
        ddg::multi_update_p(h, m);
    };
    precond_and_p();
    std::fill(restart.begin(), restart.end(), 0);
    upload();
    int it = 0;
    auto any_active = [&]() {
        for (int j = 0; j < m; ++j)
            if (active[j]) return true;
        return false;
    };
    while (any_active() && it < h->opt.maxit) {
        {
            ProfScope ps(h, DDG_K_SPMV, 1, 0.0);
            ddg::multi_spmv_pq(h, m);
        }
        {
            ProfScope ps(h, DDG_K_CG, 1, 0.0);
            ddg::multi_update_ur(h, m, U);
        }
        read_sc();
        ++it;
        bool candidates = false;
        for (int j = 0; j < m; ++j) {
            if (!active[j]) continue;
            if (at(S_FLAG, j) != 0.0) {
                st[j] = DDG_EBREAKDOWN;
                active[j] = 0;
                done_it[j] = it;
                continue;
            }
            if (std::sqrt(at(S_RR, j)) / fn[j] <= tol) candidates = true;
        }
        bool any_restart = false;
        if (candidates) {
            ProfScope ps(h, DDG_K_CG, 1, 0.0);
            ddg::multi_resnorm(h, m, F, U, w.T, S_TMP);
            read_sc();
            for (int j = 0; j < m; ++j) {
                if (!active[j] || std::sqrt(at(S_RR, j)) / fn[j] > tol) continue;
                const double trel = std::sqrt(at(S_TMP, j)) / fn[j];
                if (trel <= tol || nrest[j] >= 3) {
                    active[j] = 0;
                    done_it[j] = it;
                    done_rel[j] = trel;
                    st[j] = trel <= tol ? DDG_OK : DDG_ENOCONV;
                } else {
                    restart[j] = 1;
                    ++nrest[j];
                    any_restart = true;
                }
            }
            upload();
            if (any_restart) ddg::multi_replace_cols(h, m, w.T, w.R, w.restart);
        }
        if (!any_active()) break;
        precond_and_p();
        if (any_restart) {
            std::fill(restart.begin(), restart.end(), 0);
            upload();
        }
    }
    // columns still running hit maxit: report their true residual
    bool unfinished = false;
    for (int j = 0; j < m; ++j)
        if (done_rel[j] < 0.0) unfinished = true;
    if (unfinished) {
        ddg::multi_resnorm(h, m, F, U, nullptr, S_TMP);
        read_sc();
        for (int j = 0; j < m; ++j)
            if (done_rel[j] < 0.0) {
                done_rel[j] = std::sqrt(at(S_TMP, j)) / fn[j];
                if (done_it[j] < 0) {
                    done_it[j] = it;
                    st[j] = DDG_ENOCONV;
                }
            }
    }
    ddg_status worst = DDG_OK;
    {
        int32_t flags[E_COUNT];
        d2h(flags, h->errflags, E_COUNT, h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        if (flags[E_TIMEOUT]) {
            DDG_CUDA(cudaMemsetAsync(h->errflags + E_TIMEOUT, 0, sizeof(int32_t), h->stream));
            h->err = "a bounded wait of the tensor-core local solve ran out";
            worst = DDG_ETIMEOUT;
        }
    }
    for (int j = 0; j < m; ++j) {
        if (iters) iters[j] = done_it[j];
        if (relres) relres[j] = done_rel[j];
        if (st[j] != DDG_OK && worst == DDG_OK) worst = st[j];
    }
    return worst;
}

// Makes `dev` the calling thread's current device for the lifetime of the
// object and restores the previous one afterwards (a handle's streams,
// kernels and memory belong to the device that was current at its setup).
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------- graph-driven batched PCG
// The batched solve as one CUDA graph, as for a single vector: every column
// keeps its own CG, and the per-column decisions of the host loop above
// (breakdown, true-residual check, restart, maxit) are taken by control
// kernels with one thread per column.  The graph reads F from mw.Fb and
// writes U to mw.Ub.
void capture_batch(ddg_handle h, int m, cudaGraph_t g, int64_t* pre, int64_t* body_launches) {
    MultiWork& w = h->mw;
    const int beta = h->opt.beta == DDG_BETA_AUTO ? DDG_BETA_PR : h->opt.beta;
    const int pr = beta == DDG_BETA_PR;
    const int64_t n = h->n;
    if (!h->cap_stream) DDG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (!h->cap_stream2) DDG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream, bs = h->cap_stream2;
    cudaStream_t saved = h->stream;
    int64_t c0[DDG_K_COUNT];
    for (int c = 0; c < DDG_K_COUNT; ++c) c0[c] = h->prof_launches[c];
    bool in_main = false, in_body = false;
    try {
        DDG_CUDA(cudaStreamSynchronize(saved));
        if (h->precision == h->tc.prec() && h->tc.last_m != m) {
            // padding rows/columns of the residual slabs must read as zero
            DDG_CUDA(cudaMemsetAsync(h->tc.x_ptr(), 0, h->tc.x_bytes(), saved));
            DDG_CUDA(cudaStreamSynchronize(saved));
            h->tc.last_m = m;
        }
        h->stream = cs;
        DDG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        in_main = true;
        DDG_CUDA(cudaMemsetAsync(w.scal, 0, S_COUNT * DDG_MCHUNK * sizeof(double), cs));
        ddg::multi_resnorm(h, m, w.Fb, nullptr, nullptr, S_TMP);
        DDG_CUDA(cudaMemsetAsync(w.Ub, 0, n * m * sizeof(double), cs));
        DDG_CUDA(cudaMemsetAsync(w.P, 0, n * m * sizeof(double), cs));
        DDG_CUDA(cudaMemcpyAsync(w.R, w.Fb, n * m * sizeof(double), cudaMemcpyDeviceToDevice, cs));
        ddg::multi_to_float(h, m, nullptr);
        cudaGraphConditionalHandle cond;
        DDG_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
        ddg::mloop_init(h, m, cond);
        cudaStreamCaptureStatus cst;
        cudaGraph_t capg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        DDG_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &nd));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        DDG_CUDA(cudaGraphAddNode(&wnode, capg, deps, nullptr, nd, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        int64_t c1[DDG_K_COUNT];
        for (int c = 0; c < DDG_K_COUNT; ++c) c1[c] = h->prof_launches[c];
        h->stream = bs;
        DDG_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        in_body = true;
        // one iteration: r32 is current (converted after the u/r update, or
        // after a restart replaced columns of R)
        w.r32_current = true;
        ddg::multi_apply(h, m);
        ddg::multi_dots(h, m, pr);
        ddg::multi_update_p(h, m);
        ddg::multi_spmv_pq(h, m);
        ddg::multi_update_ur(h, m, w.Ub);
        ddg::mloop_decide_recurrence(h, m);
        ddg::multi_resnorm_gated(h, m, w.Fb, w.Ub, w.T, S_TMP, &w.ctl->any_cand);
        ddg::mloop_decide_true(h, m, cond);
        ddg::multi_replace_cols_gated(h, m, w.T, w.R, w.restart, &w.ctl->any_restart);
        ddg::multi_to_float(h, m, &w.ctl->any_restart);
        h->prof_launches[DDG_K_CG] += 9;   // the control, dot, update and gated kernels above
        cudaGraph_t bout = nullptr;
        in_body = false;
        DDG_CUDA(cudaStreamEndCapture(bs, &bout));
        for (int c = 0; c < DDG_K_COUNT; ++c) {
            body_launches[c] = h->prof_launches[c] - c1[c];
            pre[c] = c1[c] - c0[c];
        }
        pre[DDG_K_CG] += 9;   // norms, conversion, control kernels and the final residual
        h->stream = cs;
        DDG_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        ddg::mloop_final_prep(h, m);
        ddg::multi_resnorm_gated(h, m, w.Fb, w.Ub, nullptr, S_TMP, &w.ctl->any_unfinished);
        ddg::mloop_final(h, m);
        cudaGraph_t gout = nullptr;
        in_main = false;
        DDG_CUDA(cudaStreamEndCapture(cs, &gout));
    } catch (...) {
        cudaGraph_t junk = nullptr;
        if (in_body) cudaStreamEndCapture(bs, &junk);
        if (in_main) cudaStreamEndCapture(cs, &junk);
        cudaGetLastError();
        h->stream = saved;
        w.r32_current = false;
        for (int c = 0; c < DDG_K_COUNT; ++c) h->prof_launches[c] = c0[c];
        throw;
    }
    h->stream = saved;
    w.r32_current = false;
    for (int c = 0; c < DDG_K_COUNT; ++c) h->prof_launches[c] = c0[c];
}

const ddg_handle_s::BatchGraph* batch_graph(ddg_handle h, int m) {
    const int p = h->precision;
    if (h->batch_gen != h->mw.gen) {
        // the workspace was reallocated: the captured graphs point at the old one
        for (auto& pe : h->batch_exec)
            for (auto& e : pe) cudaGraphExecDestroy(e.exec);
        for (auto& pe : h->batch_exec) pe.clear();
        h->batch_gen = h->mw.gen;
    }
    for (auto& e : h->batch_exec[p])
        if (e.m == m) return &e;
    if (h->solve_graph_failed) return nullptr;
    cudaGraph_t g = nullptr;
    ddg_handle_s::BatchGraph bg{};
    bg.m = m;
    try {
        DDG_CUDA(cudaGraphCreate(&g, 0));
        capture_batch(h, m, g, bg.pre, bg.body);
        DDG_CUDA(cudaGraphInstantiate(&bg.exec, g, 0));
        cudaGraphDestroy(g);
    } catch (DdgError& e) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->solve_graph_failed = true;
        h->solve_graph_error = e.msg;
        return nullptr;
    }
    h->batch_exec[p].push_back(bg);
    return &h->batch_exec[p].back();
}

ddg_status pcg_batch(ddg_handle h, const double* F, double* U, int m, double tol, int* iters, double* relres) {
    ddg::multi_ensure(h, m);
    if (h->opt.autotune && h->precision == h->tc.prec()) {
        // the ring depth is a launch shape: tune it before a graph bakes it in
        const int before = h->tc_stages;
        if (h->tc.last_m != m) {
            DDG_CUDA(cudaMemsetAsync(h->tc.x_ptr(), 0, h->tc.x_bytes(), h->stream));
            h->tc.last_m = m;
        }
        ddg::autotune_tc(h, m);
        if (h->tc_stages != before) drop_graphs(h);
    }
    if (!h->use_graphs || h->prof_mask != 0) return pcg_batch_host(h, F, U, m, tol, iters, relres);
    const ddg_handle_s::BatchGraph* bg = batch_graph(h, m);
    if (!bg) return pcg_batch_host(h, F, U, m, tol, iters, relres);
    cudaGraphExec_t ge = bg->exec;
    MultiWork& w = h->mw;
    const int64_t n = h->n;
    if (F != w.Fb)
        DDG_CUDA(cudaMemcpyAsync(w.Fb, F, n * m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    w.h_ctl->tol = tol;
    w.h_ctl->maxit = h->opt.maxit;
    DDG_CUDA(cudaMemcpyAsync(w.ctl, w.h_ctl, sizeof(MultiCtl), cudaMemcpyHostToDevice, h->stream));
    DDG_CUDA(cudaGraphLaunch(ge, h->stream));
    if (U != w.Ub)
        DDG_CUDA(cudaMemcpyAsync(U, w.Ub, n * m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    DDG_CUDA(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(MultiCtl), cudaMemcpyDeviceToHost, h->stream));
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    const MultiCtl& c = *w.h_ctl;
    for (int k = 0; k < DDG_K_COUNT; ++k) h->prof_launches[k] += bg->pre[k] + (int64_t)c.it * bg->body[k];
    if (c.timed_out) {
        DDG_CUDA(cudaMemsetAsync(h->errflags + E_TIMEOUT, 0, sizeof(int32_t), h->stream));
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        throw DdgError{DDG_ETIMEOUT, "a bounded wait of the tensor-core local solve ran out"};
    }
    ddg_status worst = DDG_OK;
    for (int j = 0; j < m; ++j) {
        if (iters) iters[j] = c.done_it[j];
        if (relres) relres[j] = c.done_rel[j];
        if (c.cstat[j] != DDG_OK && worst == DDG_OK) worst = (ddg_status)c.cstat[j];
    }
    return worst;
}

template <typename Fn>
ddg_status guarded(ddg_handle h, Fn&& fn);

// ---------------------------------------------------------------- many problems, one graph
// Combined whole-solve graphs of handle lists (ddg_solve_many), kept until a
// handle of the list changes (precision, generators, batched workspace) or
// is destroyed.  Problem p is a single-vector solve (m = 1) or a batched
// solve of m columns; each is one branch of the graph.
struct ManyGraph {
    std::vector<ddg_handle> hs;
    std::vector<int> precs, versions, ms, gens;
    std::vector<std::vector<int64_t>> pre, body;   // launches per problem: once / per iteration
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_many_mu;
std::list<ManyGraph> g_many;   // a list: references stay valid

void drop_many_graphs(ddg_handle h) {
    std::lock_guard<std::mutex> lock(g_many_mu);
    for (auto it = g_many.begin(); it != g_many.end();) {
        if (std::find(it->hs.begin(), it->hs.end(), h) != it->hs.end()) {
            if (it->exec) cudaGraphExecDestroy(it->exec);
            it = g_many.erase(it);
        } else {
            ++it;
        }
    }
}

// the combined graph of these problems (built on first use)
const ManyGraph& many_graph(ddg_handle* hs, int nprob, const int* m) {
    std::lock_guard<std::mutex> lock(g_many_mu);
    for (ManyGraph& mg : g_many) {
        if ((int)mg.hs.size() != nprob) continue;
        bool same = true;
        for (int p = 0; p < nprob && same; ++p)
            same = mg.hs[p] == hs[p] && mg.precs[p] == hs[p]->precision && mg.versions[p] == hs[p]->version &&
                   mg.ms[p] == m[p] && mg.gens[p] == hs[p]->mw.gen;
        if (same) return mg;
    }
    ManyGraph mg;
    cudaGraph_t g = nullptr;
    DDG_CUDA(cudaGraphCreate(&g, 0));
    try {
        for (int p = 0; p < nprob; ++p) {
            ddg_handle h = hs[p];
            std::vector<int64_t> pre(DDG_K_COUNT, 0), body(DDG_K_COUNT, 0);
            if (m[p] == 1) {
                capture_solve_branch(h, g);
                for (int c = 0; c < DDG_K_COUNT; ++c) {
                    pre[c] = h->solve_pre_launches[h->precision][c];
                    body[c] = h->solve_body_launches[h->precision][c];
                }
            } else {
                ddg::multi_ensure(h, m[p]);
                capture_batch(h, m[p], g, pre.data(), body.data());
            }
            mg.pre.push_back(pre);
            mg.body.push_back(body);
        }
        DDG_CUDA(cudaGraphInstantiate(&mg.exec, g, 0));
    } catch (...) {
        cudaGraphDestroy(g);
        throw;
    }
    cudaGraphDestroy(g);
    for (int p = 0; p < nprob; ++p) {
        mg.hs.push_back(hs[p]);
        mg.precs.push_back(hs[p]->precision);
        mg.versions.push_back(hs[p]->version);
        mg.ms.push_back(m[p]);
        mg.gens.push_back(hs[p]->mw.gen);
    }
    g_many.push_back(mg);
    return g_many.back();
}

// ddg_solve_many as one graph launch when every handle can run graph-driven
// solves, the batched ones (m > 1) take the batched path (FP32/BF16
// preconditioner, two-level handle, at most 32 generators, m <= 64) and all
// handles are on one device; returns false (nothing done) otherwise.  The
// launch runs on hs[0]'s stream, ordered after and before the work on every
// handle's stream by events.
bool solve_many_graph(ddg_handle* hs, int nprob, const double* const* F, double* const* U, const int* m,
                      double tol, int* iters, double* relres, ddg_status& worst) {
    for (int p = 0; p < nprob; ++p) {
        ddg_handle h = hs[p];
        if (!h->use_graphs || h->prof_mask != 0 || h->solve_graph_failed || h->device != hs[0]->device ||
            (const void*)F[p] == (const void*)U[p])
            return false;
        if (m[p] > 1 && (m[p] > DDG_MCHUNK || h->precision == DDG_PREC_FP64 || h->inner || h->kmax > 32 ||
                         h->bl.on))
            return false;
    }
    DeviceScope scope(hs[0]->device);
    bool built = false;
    std::vector<cudaEvent_t> ev(nprob + 1, nullptr);
    try {
        for (int p = 0; p < nprob; ++p) {
            hs[p]->err.clear();
            if (m[p] == 1) ensure_loop_buffers(hs[p]);
            else ddg::multi_ensure(hs[p], m[p]);
        }
        const ManyGraph& mg = many_graph(hs, nprob, m);
        built = true;
        for (auto& e : ev) DDG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaStream_t L = hs[0]->stream;
        for (int p = 0; p < nprob; ++p) {
            ddg_handle h = hs[p];
            if (m[p] == 1) {
                DDG_CUDA(cudaMemcpyAsync(h->fbuf, F[p], h->n * sizeof(double), cudaMemcpyDeviceToDevice,
                                         h->stream));
                loop_params(h, tol);
            } else {
                MultiWork& w = h->mw;
                DDG_CUDA(cudaMemcpyAsync(w.Fb, F[p], h->n * m[p] * sizeof(double), cudaMemcpyDeviceToDevice,
                                         h->stream));
                w.h_ctl->tol = tol;
                w.h_ctl->maxit = h->opt.maxit;
                DDG_CUDA(cudaMemcpyAsync(w.ctl, w.h_ctl, sizeof(MultiCtl), cudaMemcpyHostToDevice, h->stream));
            }
            DDG_CUDA(cudaEventRecord(ev[p], h->stream));
            DDG_CUDA(cudaStreamWaitEvent(L, ev[p], 0));
        }
        DDG_CUDA(cudaGraphLaunch(mg.exec, L));
        DDG_CUDA(cudaEventRecord(ev[nprob], L));
        for (int p = 0; p < nprob; ++p) {
            ddg_handle h = hs[p];
            DDG_CUDA(cudaStreamWaitEvent(h->stream, ev[nprob], 0));
            if (m[p] == 1) {
                DDG_CUDA(cudaMemcpyAsync(U[p], h->ubuf, h->n * sizeof(double), cudaMemcpyDeviceToDevice,
                                         h->stream));
                DDG_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(CgCtl), cudaMemcpyDeviceToHost, h->stream));
            } else {
                MultiWork& w = h->mw;
                DDG_CUDA(cudaMemcpyAsync(U[p], w.Ub, h->n * m[p] * sizeof(double), cudaMemcpyDeviceToDevice,
                                         h->stream));
                DDG_CUDA(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(MultiCtl), cudaMemcpyDeviceToHost, h->stream));
            }
        }
        for (int p = 0; p < nprob; ++p) DDG_CUDA(cudaStreamSynchronize(hs[p]->stream));
        worst = DDG_OK;
        int64_t off = 0;
        for (int p = 0; p < nprob; ++p) {
            ddg_handle h = hs[p];
            ddg_status st = DDG_OK;
            if (m[p] == 1) {
                st = loop_outcome(h, iters ? iters + off : nullptr, relres ? relres + off : nullptr);
            } else {
                const MultiCtl& c = *h->mw.h_ctl;
                for (int k = 0; k < DDG_K_COUNT; ++k)
                    h->prof_launches[k] += mg.pre[p][k] + (int64_t)c.it * mg.body[p][k];
                if (c.timed_out) {
                    DDG_CUDA(cudaMemsetAsync(h->errflags + E_TIMEOUT, 0, sizeof(int32_t), h->stream));
                    DDG_CUDA(cudaStreamSynchronize(h->stream));
                    h->err = "a bounded wait of the tensor-core local solve ran out";
                    st = DDG_ETIMEOUT;
                }
                for (int j = 0; j < m[p]; ++j) {
                    if (iters) iters[off + j] = c.done_it[j];
                    if (relres) relres[off + j] = c.done_rel[j];
                    if (st == DDG_OK && c.cstat[j] != DDG_OK) st = (ddg_status)c.cstat[j];
                }
            }
            if (st != DDG_OK && worst == DDG_OK) worst = st;
            off += m[p];
        }
    } catch (DdgError& e) {
        for (auto& x : ev)
            if (x) cudaEventDestroy(x);
        hs[0]->err = e.msg;
        if (!built) return false;   // the graph could not be built: solve the problems one by one
        worst = e.st;
        return true;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    return true;
}

// Destroy every captured graph of h (preconditioner applies, whole solves,
// batched solves, combined graphs that include h): their kernels carry
// arguments that a change of the handle makes stale.
void drop_graphs(ddg_handle h) {
    for (cudaGraphExec_t& g : h->apply_exec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (cudaGraphExec_t& g : h->solve_exec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (auto& pe : h->batch_exec) {
        for (auto& e : pe) cudaGraphExecDestroy(e.exec);
        pe.clear();
    }
    ++h->version;
    drop_many_graphs(h);
}

template <typename Fn>
ddg_status guarded(ddg_handle h, Fn&& fn) {
    if (!h) return DDG_EINVAL;
    DeviceScope scope(h->device);
    try {
        h->err.clear();
        return fn();
    } catch (DdgError& e) {
        h->err = e.msg;
        return e.st;
    } catch (std::exception& e) {
        h->err = e.what();
        return DDG_EINVAL;
    }
}

}  // namespace

namespace ddg {
// message for ddg_last_error(NULL) from calls that have no handle
void set_handleless_error(const char* msg) { g_setup_error = msg ? msg : ""; }
}  // namespace ddg

ProfScope::ProfScope(ddg_handle hh, int c, int nlaunch, double bytes) : h(hh), cls(c), pair(-1) {
    h->prof_launches[c] += nlaunch;
    if (!(h->prof_mask & (1 << c))) return;
    if (h->ev_used * 2 + 2 > h->ev_pool.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            DDG_CUDA(cudaEventCreate(&e));
            h->ev_pool.push_back(e);
        }
    }
    pair = (int)h->ev_used++;
    if (h->ev_class.size() < h->ev_used) {
        h->ev_class.resize(h->ev_used);
        h->ev_bytes.resize(h->ev_used);
    }
    h->ev_class[pair] = c;
    h->ev_bytes[pair] = bytes;
    DDG_CUDA(cudaEventRecord(h->ev_pool[2 * pair], h->stream));
}

ProfScope::~ProfScope() {
    if (pair >= 0) cudaEventRecord(h->ev_pool[2 * pair + 1], h->stream);
}

extern "C" {

void ddg_default_options(ddg_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = DDG_PREC_FP64;
    o->keep_precisions = 0;
    o->overlap_mode = DDG_OVERLAP_GRAPH;
    o->beta = DDG_BETA_AUTO;
    o->maxit = 1000;
    o->use_coarse = 1;
    o->rank_tol = 1e-10;
    o->chunk_tiles = 0;
    o->spin_budget_ms = 1000.0;
    o->coarse_order = DDG_COARSE_ND;
}

}  // extern "C"

namespace {
void setup_vcycle(ddg_handle h, const double* F, int k, int overlap, const ddg_options& o,
                  const int32_t* groups, const std::vector<int>& bI, const std::vector<int>& bJ,
                  const std::vector<int64_t>& sub_off, const std::vector<int32_t>& sub_nodes);

// pairs of subdomains (I >= J, ascending) that A couples: an entry of a row of
// Omega_I lies in a column of Omega_J
void subdomain_pairs(const ddg_matrix* A, const int32_t* partition, const std::vector<int64_t>& sub_off,
                     const std::vector<int32_t>& sub_nodes, int nsub, std::vector<int>& pI,
                     std::vector<int>& pJ) {
    pI.clear();
    pJ.clear();
    std::vector<int> mark(nsub, -1), js;
    for (int I = 0; I < nsub; ++I) {
        js.clear();
        for (int64_t a = sub_off[I]; a < sub_off[I + 1]; ++a) {
            const int g = sub_nodes[a];
            for (int64_t e = A->rowptr[g]; e < A->rowptr[g + 1]; ++e) {
                const int J = partition[A->col[e]];
                if (J <= I && mark[J] != I) {
                    mark[J] = I;
                    js.push_back(J);
                }
            }
        }
        std::sort(js.begin(), js.end());
        for (int J : js) {
            pI.push_back(I);
            pJ.push_back(J);
        }
    }
}

// Sec. 4: R0 from the generators (per-subdomain QR and rank drop), then A0 and
// its block-bidiagonal factor, or the coarse level of the V-cycle when groups
// is set.  Leaves use_coarse = 0 when every subdomain drops every generator.
// The device memory it keeps is listed in h->coarse_allocs.
void build_coarse(ddg_handle h, const double* F, int k, int overlap, const ddg_options& o,
                  const int32_t* groups) {
    const size_t mark_allocs = h->arena.ptrs.size();
    const int64_t n = h->n;
    const int nsub = h->nsub;
    h->kmax = k;
    double* dF = h->arena.alloc<double>((size_t)n * k);
    h2d(dF, F, (size_t)n * k, h->stream);
    h->Q64 = h->arena.alloc<double>((size_t)n * k);
    int32_t* d_rank = h->arena.alloc<int32_t>(nsub);
    ddg::coarse_qr(h, d_rank, dF, k);
    std::vector<int32_t> rank(nsub);
    d2h(rank.data(), d_rank, nsub, h->stream);
    DDG_CUDA(cudaStreamSynchronize(h->stream));
    h->arena.release(dF);
    h->arena.release(d_rank);
    h->h_coff.assign(nsub + 1, 0);
    for (int s = 0; s < nsub; ++s) h->h_coff[s + 1] = h->h_coff[s] + rank[s];
    h->n0 = h->h_coff[nsub];
    if (h->n0 == 0) h->use_coarse = 0;
    if (h->use_coarse) {
        h->coff = h->arena.alloc<int32_t>(nsub + 1);
        h2d(h->coff, h->h_coff.data(), nsub + 1, h->stream);
        // coupled pairs with coarse dofs on both sides, and the half-bandwidth of A0
        std::vector<int> bI, bJ;
        int64_t band = 0;
        for (size_t p = 0; p < h->h_adjI.size(); ++p) {
            const int I = h->h_adjI[p], J = h->h_adjJ[p];
            if (h->h_coff[I + 1] == h->h_coff[I] || h->h_coff[J + 1] == h->h_coff[J]) continue;
            bI.push_back(I);
            bJ.push_back(J);
            band = std::max<int64_t>(band, (int64_t)h->h_coff[I + 1] - 1 - h->h_coff[J]);
        }
        h->band = (int)band;
        if (groups) {
            setup_vcycle(h, F, k, overlap, o, groups, bI, bJ, h->h_sub_off, h->h_sub_nodes);
        } else if (o.coarse_order == DDG_COARSE_ND) {
            // nested-dissection factor of A0 (multifrontal, dense fronts)
            const int n0 = h->n0;
            h->n0p = n0;
            h->nK = 0;
            double* blocks = ddg::coarse_assemble_blocks_device(h, bI, bJ);
            ddg::nd_coarse_setup(h, bI, bJ, blocks);
            h->arena.release(blocks);
            h->c64 = h->arena.alloc<double>(n0);
            h->y64 = h->arena.alloc<double>(n0);
            h->x64 = h->arena.alloc<double>(n0);
            h->c32 = h->arena.alloc<float>(n0);
            h->y32 = h->arena.alloc<float>(n0);
            h->x32 = h->arena.alloc<float>(n0);
        } else {
            h->Wt = std::max(1, (int)((band + DDG_CT - 1) / DDG_CT));
            const int NT0 = (h->n0 + DDG_CT - 1) / DDG_CT;
            h->nK = (NT0 + h->Wt - 1) / h->Wt;
            h->NT = h->nK * h->Wt;
            h->n0p = h->NT * DDG_CT;
            h->B = h->Wt * DDG_CT;
            h->bandL = h->arena.alloc<double>((size_t)h->NT * (h->Wt + 1) * DDG_CT * DDG_CT);
            ddg::coarse_assemble_band(h, bI, bJ);
            ddg::coarse_band_cholesky(h);
            ddg::coarse_build_apply(h);
            const int n0p = h->n0p;
            h->c64 = h->arena.alloc<double>(n0p);
            h->y64 = h->arena.alloc<double>(n0p);
            h->x64 = h->arena.alloc<double>(n0p);
            h->c32 = h->arena.alloc<float>(n0p);
            h->y32 = h->arena.alloc<float>(n0p);
            h->x32 = h->arena.alloc<float>(n0p);
            for (void* p : {(void*)h->c64, (void*)h->y64, (void*)h->x64})
                DDG_CUDA(cudaMemsetAsync(p, 0, n0p * sizeof(double), h->stream));
            for (void* p : {(void*)h->c32, (void*)h->y32, (void*)h->x32})
                DDG_CUDA(cudaMemsetAsync(p, 0, n0p * sizeof(float), h->stream));
        }
        h->Q32 = h->arena.alloc<float>((size_t)n * k);
        ddg::cast_q32(h);
    }
    h->coarse_allocs.clear();
    for (size_t i = mark_allocs; i < h->arena.ptrs.size(); ++i)
        if (h->arena.ptrs[i]) h->coarse_allocs.push_back(h->arena.ptrs[i]);
}
}  // namespace

namespace {
// Work items of the single-vector local solve: bands of whole tile rows of
// each packed upper triangle, about `chunk` tiles and at most `band` tile
// rows each (a row joins the band only if it brings it closer to `chunk`).
std::vector<int4> local_items(const ddg_handle h, int chunk, int band) {
    std::vector<int4> items;
    for (int c = 0; c < h->ncol; ++c)
        for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q) {
            const int T = h->h_Tq[q];
            int I = 0;
            while (I < T) {
                const int I0 = I;
                int cnt = 0;
                while (I < T && I - I0 < band) {
                    const int len = T - I;
                    if (cnt > 0 && cnt + len - chunk > chunk - cnt) break;
                    cnt += len;
                    ++I;
                }
                items.push_back(make_int4(q, I0, I, 0));
            }
        }
    return items;
}

// (Re)build the work items and their metadata on the device; the partial
// buffers are left to the caller (they hold nitems * Tmax * 32 values).
void build_local_items(ddg_handle h, int chunk, int band) {
    for (void* p : {(void*)h->items, (void*)h->nchunks, (void*)h->first_item, (void*)h->counters,
                    (void*)h->ov_sub, (void*)h->row_nchunks})
        if (p) h->arena.release(p);
    const int nsub = h->nsub;
    const std::vector<int4> items = local_items(h, chunk, band);
    std::vector<int32_t> nch(nsub, 0), first(nsub, 0);
    h->h_citem_off.assign(h->ncol + 1, 0);
    for (size_t i = 0; i < items.size(); ++i) {
        const int q = items[i].x;
        if (nch[q]++ == 0) first[q] = (int)i;
    }
    for (int c = 0; c < h->ncol; ++c) {
        int cnt = 0;
        for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q) cnt += nch[q];
        h->h_citem_off[c + 1] = h->h_citem_off[c] + cnt;
    }
    h->nitems = (int)items.size();
    h->items = h->arena.alloc<int4>(items.size());
    h->nchunks = h->arena.alloc<int32_t>(nsub);
    h->first_item = h->arena.alloc<int32_t>(nsub);
    h->counters = h->arena.alloc<unsigned>(nsub);
    h2d(h->items, items.data(), items.size(), h->stream);
    h2d(h->nchunks, nch.data(), nsub, h->stream);
    h2d(h->first_item, first.data(), nsub, h->stream);
    DDG_CUDA(cudaMemsetAsync(h->counters, 0, nsub * sizeof(unsigned), h->stream));
    const std::vector<int64_t>& ov_off = h->h_ov_off;
    std::vector<int32_t> ovs(h->sum_local), rnc(h->sum_local);
    for (int q = 0; q < nsub; ++q)
        for (int64_t a = ov_off[q]; a < ov_off[q + 1]; ++a) {
            ovs[a] = q;
            const int row_tile = (int)((a - ov_off[q]) / DDG_LT);
            int c = 0;
            while (c < nch[q] && items[first[q] + c].y <= row_tile) ++c;
            rnc[a] = c;
        }
    h->ov_sub = h->arena.alloc<int32_t>(h->sum_local);
    h->row_nchunks = h->arena.alloc<int32_t>(h->sum_local);
    h2d(h->ov_sub, ovs.data(), h->sum_local, h->stream);
    h2d(h->row_nchunks, rnc.data(), h->sum_local, h->stream);
    h->split_gather = *std::max_element(nch.begin(), nch.end()) > DDG_GATHER_SPLIT_CHUNKS;
    h->ls_chunk = chunk;
    h->ls_band_rows = band;
    DDG_CUDA(cudaStreamSynchronize(h->stream));
}

// ---------------------------------------------------------------- autotuner
// Launch shapes of the local solves chosen by timing candidates on the
// handle's own data (CUDA events on its stream, median of three launches of
// the colour with the most local rows), keyed on the local-block class (the
// largest block, the number of subdomains and colours), the column count m
// and the precision; a choice is kept process-wide, so a second handle of
// the same class reuses it (and computes the same bits) without timing.
struct TuneKey {
    int max_local, nsub, ncol, m, prec;
    bool operator<(const TuneKey& o) const {
        return std::tie(max_local, nsub, ncol, m, prec) < std::tie(o.max_local, o.nsub, o.ncol, o.m, o.prec);
    }
};
struct TuneChoice {
    int warps = 8, chunk = 96, band = DDG_BAND_ROWS, stages = 4;
    double ms = 0.0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

int largest_colour(ddg_handle h) {
    int best = 0;
    for (int c = 1; c < h->ncol; ++c)
        if (h->h_crow_off[c + 1] - h->h_crow_off[c] > h->h_crow_off[best + 1] - h->h_crow_off[best]) best = c;
    return best;
}

// median of three timed runs of `launch` after one warm-up, in ms
template <typename Fn>
double time_launches(ddg_handle h, Fn&& launch) {
    cudaEvent_t e0, e1;
    DDG_CUDA(cudaEventCreate(&e0));
    DDG_CUDA(cudaEventCreate(&e1));
    launch();
    std::vector<float> t;
    for (int r = 0; r < 3; ++r) {
        DDG_CUDA(cudaEventRecord(e0, h->stream));
        launch();
        DDG_CUDA(cudaEventRecord(e1, h->stream));
        DDG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        DDG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    return t[1];
}

void alloc_partials(ddg_handle h, int nitems) {
    if (h->partial64) h->arena.release(h->partial64);
    if (h->partial32) h->arena.release(h->partial32);
    h->partial64 = nullptr;
    h->partial32 = nullptr;
    const size_t pslots = (size_t)nitems * h->Tmax * DDG_LT;
    const int keep = h->opt.keep_precisions;
    if (keep & (1 << DDG_PREC_FP64)) h->partial64 = h->arena.alloc<double>(pslots);
    if (keep & ((1 << DDG_PREC_FP32) | (1 << DDG_PREC_BF16))) h->partial32 = h->arena.alloc<float>(pslots);
}

// warps per CTA {8, 4} x tiles per item {48, 96, 192} x tile rows per item
// {8, 16} for the single-vector local solve in the handle's precision (the
// tiles per item stay fixed when chunk_tiles was given)
void autotune_local(ddg_handle h) {
    const int prec = h->precision;
    const TuneKey key{h->max_local, h->nsub, h->ncol, 1, prec};
    TuneChoice best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        std::vector<int> chunks = {48, 96, 192};
        if (h->opt.chunk_tiles > 0) chunks = {h->opt.chunk_tiles};
        int max_items = 0;
        for (int ch : chunks)
            for (int band : {8, DDG_BAND_ROWS})
                max_items = std::max(max_items, (int)local_items(h, ch, band).size());
        alloc_partials(h, max_items);
        const int c = largest_colour(h);
        if (prec == DDG_PREC_FP64) {
            DDG_CUDA(cudaMemsetAsync(h->res64, 0, h->sum_local * sizeof(double), h->stream));
            DDG_CUDA(cudaMemsetAsync(h->z64, 0, h->n * sizeof(double), h->stream));
        } else {
            DDG_CUDA(cudaMemsetAsync(h->res32, 0, h->sum_local * sizeof(float), h->stream));
            DDG_CUDA(cudaMemsetAsync(h->z32, 0, h->n * sizeof(float), h->stream));
        }
        best.ms = 1e30;
        for (int ch : chunks)
            for (int band : {DDG_BAND_ROWS, 8}) {
                build_local_items(h, ch, band);
                for (int w : {8, 4}) {
                    h->ls_warps = w;
                    const double ms = time_launches(h, [&]() { ddg::local_solve_colour(h, c, prec); });
                    // a candidate replaces the incumbent only when more than 2% faster
                    if (ms < best.ms * 0.98) {
                        best.ms = ms;
                        best.warps = w;
                        best.chunk = ch;
                        best.band = band;
                    }
                }
            }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune.emplace(key, best);
    }
    h->ls_warps = best.warps;
    build_local_items(h, best.chunk, best.band);
    alloc_partials(h, h->nitems);
    h->tuned = 1;
    h->tune_ms = best.ms;
}
}  // namespace

namespace ddg {
// tensor-core ring depth {3, 4, 6} for m columns (called before the batched
// solve is captured or run; cached per class and m)
void autotune_tc(ddg_handle h, int m) {
    // keyed on the operand type: BF16 and TF32 slabs differ in bytes per stage
    const TuneKey key{h->max_local, h->nsub, h->ncol, m, h->tc.kind == DDG_TC_TF32 ? 100 + DDG_PREC_FP32 : DDG_PREC_BF16};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            h->tc_stages = it->second.stages;
            return;
        }
    }
    const int c = largest_colour(h);
    TuneChoice best;
    best.ms = 1e30;
    for (int st : {4, 3, 6}) {
        h->tc_stages = st;
        const double ms = time_launches(h, [&]() { ddg::tc_local_solve(h, c, m); });
        if (ms < best.ms * 0.98) {
            best.ms = ms;
            best.stages = st;
        }
    }
    DDG_CUDA(cudaMemsetAsync(h->mw.z32, 0, h->n * m * sizeof(float), h->stream));
    h->tc_stages = best.stages;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.emplace(key, best);
}
}  // namespace ddg

namespace {
// half-bandwidth max |i - j| of each A_i = A[ov, ov] in ascending dof order
std::vector<int> local_bandwidths(const ddg_matrix* A, const std::vector<std::vector<int32_t>>& ov,
                                  const std::vector<int>& sid) {
    std::vector<int> bq(sid.size(), 0);
    std::vector<int32_t> loc(A->n, -1);
    for (size_t q = 0; q < sid.size(); ++q) {
        const std::vector<int32_t>& idx = ov[sid[q]];
        for (size_t r = 0; r < idx.size(); ++r) loc[idx[r]] = (int32_t)r;
        int b = 0;
        for (size_t r = 0; r < idx.size(); ++r)
            for (int64_t e = A->rowptr[idx[r]]; e < A->rowptr[idx[r] + 1]; ++e) {
                const int32_t c = loc[A->col[e]];
                if (c >= 0) b = std::max(b, std::abs((int)r - c));
            }
        bq[q] = b;
        for (int32_t g : idx) loc[g] = -1;
    }
    return bq;
}

// row chunks of a block for one element size: consecutive whole rows of at
// most DDG_BAND_STAGE_BYTES
std::vector<int2> band_chunks(const std::vector<int32_t>& row, size_t elem) {
    std::vector<int2> ch;
    const int rows = (int)row.size() - 1;
    int r = 0;
    while (r < rows) {
        int e = r + 1;
        while (e < rows && (size_t)(row[e + 1] - row[r]) * elem <= DDG_BAND_STAGE_BYTES) ++e;
        ch.push_back(make_int2(r, e));
        r = e;
    }
    return ch;
}

// Banded local factors (Sec. 6, exact local solves): Cholesky of every A_i
// in FP64 with the tile band kernels, batched over subdomains, rewritten in
// block form (C_K, D_K per super-block of B rows) in FP64 and/or FP32.
void setup_band_local(ddg_handle h, const std::vector<int>& bq) {
    BandLocal& L = h->bl;
    const int nsub = h->nsub;
    const int keep = h->opt.keep_precisions;
    L.b = std::max(1, *std::max_element(bq.begin(), bq.end()));
    L.Wt = (L.b + DDG_CT - 1) / DDG_CT;
    L.B = L.Wt * DDG_CT;
    DDG_REQUIRE(L.B <= 1024, DDG_EINVAL, "banded local factors take half-bandwidths of at most 1024");
    const int B = L.B, b = L.b, Wt = L.Wt;
    std::vector<int32_t> rowC(b + 1, 0), rowD(B + 1, 0);
    for (int i = 0; i < b; ++i) rowC[i + 1] = rowC[i] + (B - ((B - b + i) & ~3));
    for (int i = 0; i < B; ++i) rowD[i + 1] = rowD[i] + ((i + 4) & ~3);
    L.sizeC = rowC[b];
    L.sizeD = rowD[B];
    std::vector<int32_t> nts(nsub);
    L.h_nk.assign(nsub, 0);
    L.h_qoff.assign(nsub + 1, 0);
    int nKmax = 0;
    for (int q = 0; q < nsub; ++q) {
        const int nq = (int)(h->h_ov_off[q + 1] - h->h_ov_off[q]);
        const int nk = std::max(1, (nq + B - 1) / B);
        L.h_nk[q] = nk;
        nts[q] = nk * Wt;
        nKmax = std::max(nKmax, nk);
        L.h_qoff[q + 1] = L.h_qoff[q] + (int64_t)nk * (L.sizeC + L.sizeD);
    }
    L.vec_elems = nKmax * B;
    L.elems = L.h_qoff[nsub];
    // shared-memory ring depth: what is left of 220 KB after the vectors
    auto stages_for = [&](size_t sv) {
        const size_t fixed = (size_t)L.vec_elems * sv + (size_t)((B + 15) & ~15) * sv + 256;
        const size_t budget = (size_t)220 << 10;
        return fixed >= budget ? 0 : (int)std::min<size_t>(4, (budget - fixed) / DDG_BAND_STAGE_BYTES);
    };
    L.stages64 = stages_for(8);
    L.stages32 = stages_for(4);
    if (keep & (1 << DDG_PREC_FP64))
        DDG_REQUIRE(L.stages64 >= 2, DDG_EINVAL, "local block too large for the FP64 banded solve");
    DDG_REQUIRE(L.stages32 >= 2, DDG_EINVAL, "local block too large for the banded solve");
    L.nk = h->arena.alloc<int32_t>(nsub);
    L.qoff = h->arena.alloc<int64_t>(nsub + 1);
    L.rowC = h->arena.alloc<int32_t>(b + 1);
    L.rowD = h->arena.alloc<int32_t>(B + 1);
    h2d(L.nk, L.h_nk.data(), nsub, h->stream);
    h2d(L.qoff, L.h_qoff.data(), nsub + 1, h->stream);
    h2d(L.rowC, rowC.data(), b + 1, h->stream);
    h2d(L.rowD, rowD.data(), B + 1, h->stream);
    auto upload_chunks = [&](const std::vector<int32_t>& row, size_t elem, int2*& d, int& cnt) {
        const std::vector<int2> ch = band_chunks(row, elem);
        cnt = (int)ch.size();
        d = h->arena.alloc<int2>(ch.size());
        h2d(d, ch.data(), ch.size(), h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
    };
    upload_chunks(rowC, 8, L.ch64C, L.nch64C);
    upload_chunks(rowD, 8, L.ch64D, L.nch64D);
    upload_chunks(rowC, 4, L.ch32C, L.nch32C);
    upload_chunks(rowD, 4, L.ch32D, L.nch32D);
    if (keep & (1 << DDG_PREC_FP64)) L.d64 = h->arena.alloc<double>(L.elems);
    if (keep & ((1 << DDG_PREC_FP32) | (1 << DDG_PREC_BF16))) L.d32 = h->arena.alloc<float>(L.elems);
    // FP64 workspaces per batch of subdomains (about 2 GB): band tiles, tile
    // inverses and super-block inverses
    const size_t tile = (size_t)DDG_CT * DDG_CT;
    const size_t Ptiles = (size_t)Wt * (Wt + 1) / 2;
    auto per_sub = [&](int q) {
        return (size_t)nts[q] * (Wt + 1) * tile + (size_t)nts[q] * tile + (size_t)L.h_nk[q] * Ptiles * tile;
    };
    const size_t budget = (size_t)1 << 28;   // doubles
    int q0 = 0;
    while (q0 < nsub) {
        int q1 = q0;
        size_t used = 0;
        while (q1 < nsub && (q1 == q0 || used + per_sub(q1) <= budget)) used += per_sub(q1++);
        const int nb = q1 - q0;
        std::vector<int32_t> ql(nb), nt(nb);
        std::vector<int64_t> bo(nb), dof(nb), wo(nb);
        size_t ob = 0, od = 0, ow = 0;
        int NTmax = 0;
        for (int t = 0; t < nb; ++t) {
            const int q = q0 + t;
            ql[t] = q;
            nt[t] = nts[q];
            NTmax = std::max(NTmax, nts[q]);
            bo[t] = (int64_t)ob;
            dof[t] = (int64_t)od;
            wo[t] = (int64_t)ow;
            ob += (size_t)nts[q] * (Wt + 1) * tile;
            od += (size_t)nts[q] * tile;
            ow += (size_t)L.h_nk[q] * Ptiles * tile;
        }
        double* band = h->arena.alloc<double>(ob);
        double* dinv = h->arena.alloc<double>(od);
        double* W = h->arena.alloc<double>(ow);
        int32_t* dql = h->arena.alloc<int32_t>(nb);
        int32_t* dnt = h->arena.alloc<int32_t>(nb);
        int64_t* dbo = h->arena.alloc<int64_t>(nb);
        int64_t* ddo = h->arena.alloc<int64_t>(nb);
        int64_t* dwo = h->arena.alloc<int64_t>(nb);
        h2d(dql, ql.data(), nb, h->stream);
        h2d(dnt, nt.data(), nb, h->stream);
        h2d(dbo, bo.data(), nb, h->stream);
        h2d(ddo, dof.data(), nb, h->stream);
        h2d(dwo, wo.data(), nb, h->stream);
        DDG_CUDA(cudaMemsetAsync(band, 0, ob * sizeof(double), h->stream));
        DDG_CUDA(cudaMemsetAsync(W, 0, ow * sizeof(double), h->stream));
        ddg::band_local_assemble(h, dql, nb, dbo, dnt, band);
        ddg::band_factor_batched(h, band, Wt, nb, NTmax, dbo, dnt, dinv, ddo, W, dwo, h->errflags + E_LOCAL_SPD);
        ddg::band_local_pack(h, dql, nb, NTmax / Wt, dbo, dwo, band, W);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        for (void* p : {(void*)band, (void*)dinv, (void*)W, (void*)dql, (void*)dnt, (void*)dbo, (void*)ddo,
                        (void*)dwo})
            h->arena.release(p);
        q0 = q1;
    }
    ddg::band_local_configure(h);
}
}  // namespace

static ddg_status setup_impl(const ddg_matrix* A, const int32_t* partition, const int32_t* groups,
                             const double* F, int k, int overlap, const ddg_options* opt, void* stream,
                             ddg_handle* out) {
    g_setup_error.clear();
    if (!out) {
        g_setup_error = "out must be non-null";
        return DDG_EINVAL;
    }
    *out = nullptr;
    const double t0 = now_ms();
    ddg_handle h = new ddg_handle_s;
    try {
        ddg_options o;
        if (opt) o = *opt;
        else ddg_default_options(&o);
        validate(A, partition, F, k, overlap, o);
        if (groups) {
            int nsub_ids = 0;
            for (int64_t g = 0; g < A->n; ++g) nsub_ids = std::max(nsub_ids, partition[g] + 1);
            for (int s = 0; s < nsub_ids; ++s)
                DDG_REQUIRE(groups[s] >= 0, DDG_EINVAL, "coarse_partition ids must be >= 0");
        }
        h->opt = o;
        h->precision = o.precision;
        DDG_CUDA(cudaGetDevice(&h->device));
        h->wait_ns = (unsigned long long)((o.spin_budget_ms > 0.0 ? o.spin_budget_ms : 1000.0) * 1e6);
        if (const char* ev = std::getenv("DDG_NO_GRAPHS")) h->use_graphs = ev[0] == '0';
        if (const char* ev = std::getenv("DDG_PDL")) h->use_pdl = ev[0] != '0';
        h->use_coarse = o.use_coarse;
        h->stream = (cudaStream_t)stream;
        const int64_t n = A->n;
        h->n = n;
        h->nnz = A->rowptr[n];
        for (int64_t g = 0; g < n; ++g)
            h->max_row_nnz = std::max<int>(h->max_row_nnz, (int)(A->rowptr[g + 1] - A->rowptr[g]));
        h->wide_rows = h->nnz >= 32 * n;
        h->stencil_kind = A->stencil_kind;
        h->dim = A->dim;
        h->nx = A->nx > 0 ? A->nx : 1;
        h->ny = A->ny > 0 ? A->ny : 1;
        h->nz = A->nz > 0 ? A->nz : 1;
        h->dpn = A->dofs_per_node > 0 ? A->dofs_per_node : 1;
        const int keep = (o.keep_precisions ? o.keep_precisions : 0) | (1 << o.precision);
        h->opt.keep_precisions = keep;

        // ---- fine matrix
        h->rowptr = h->arena.alloc<int64_t>(n + 1);
        h->col = h->arena.alloc<int32_t>(h->nnz);
        h->val64 = h->arena.alloc<double>(h->nnz);
        h->val32 = h->arena.alloc<float>(h->nnz);
        h2d(h->rowptr, A->rowptr, n + 1, h->stream);
        h2d(h->col, A->col, h->nnz, h->stream);
        h2d(h->val64, A->val, h->nnz, h->stream);
        {
            std::vector<float> v32(A->val, A->val + h->nnz);
            h2d(h->val32, v32.data(), h->nnz, h->stream);
            DDG_CUDA(cudaStreamSynchronize(h->stream));
        }
        if (A->stencil_kind == DDG_STENCIL_VAR7_3D && A->coef) {
            h->ncoef = n;
            h->kappa = h->arena.alloc<double>(n);
            h2d(h->kappa, A->coef, n, h->stream);
        }
        if (A->stencil_kind == DDG_STENCIL_Q1_ELASTIC) {
            const int ne = A->nx;
            DDG_REQUIRE(ne >= 1 && A->ny == ne + 1 && A->nz == ne + 1 && A->dofs_per_node == 3 &&
                            (int64_t)3 * ne * (ne + 1) * (ne + 1) == n,
                        DDG_EINVAL, "Q1 elasticity needs nx = ne, ny = nz = ne + 1, 3 dofs per node");
            const std::vector<double> K = q1_dk_dmu(1.0 / ne);
            h->kmu = h->arena.alloc<double>(576);
            h2d(h->kmu, K.data(), 576, h->stream);
            if (A->coef) {
                h->ncoef = (int64_t)ne * ne * ne;
                h->kappa = h->arena.alloc<double>(h->ncoef);
                h2d(h->kappa, A->coef, h->ncoef, h->stream);
            }
            DDG_CUDA(cudaStreamSynchronize(h->stream));
        }

        // ---- partition (Sec. 4)
        int nsub = 0;
        for (int64_t g = 0; g < n; ++g) {
            DDG_REQUIRE(partition[g] >= 0, DDG_EINVAL, "partition ids must be >= 0");
            nsub = std::max(nsub, partition[g] + 1);
        }
        h->nsub = nsub;
        std::vector<int64_t> sub_off(nsub + 1, 0);
        for (int64_t g = 0; g < n; ++g) sub_off[partition[g] + 1]++;
        for (int s = 0; s < nsub; ++s) {
            DDG_REQUIRE(sub_off[s + 1] > 0, DDG_EINVAL, "every subdomain id in [0, nsub) must own a node");
            sub_off[s + 1] += sub_off[s];
        }
        std::vector<int32_t> sub_nodes(n), pos(n);
        {
            std::vector<int64_t> fill(sub_off.begin(), sub_off.end() - 1);
            for (int64_t g = 0; g < n; ++g) {
                const int64_t a = fill[partition[g]]++;
                sub_nodes[a] = (int32_t)g;
                pos[g] = (int32_t)a;
            }
        }
        h->h_sub_off = sub_off;
        h->part = h->arena.alloc<int32_t>(n);
        h->sub_off = h->arena.alloc<int64_t>(nsub + 1);
        h->sub_nodes = h->arena.alloc<int32_t>(n);
        h->pos = h->arena.alloc<int32_t>(n);
        h2d(h->part, partition, n, h->stream);
        h2d(h->sub_off, sub_off.data(), nsub + 1, h->stream);
        h2d(h->sub_nodes, sub_nodes.data(), n, h->stream);
        h2d(h->pos, pos.data(), n, h->stream);

        // ---- overlapping subdomains, colouring, sweep order (Sec. 6)
        std::vector<std::vector<int32_t>> ov;
        grow_overlaps(A, sub_off, sub_nodes, nsub, overlap, o.overlap_mode, ov);
        h->h_colour = colour_subdomains(A, ov);
        h->ncol = 1 + *std::max_element(h->h_colour.begin(), h->h_colour.end());
        h->h_csub_off.assign(h->ncol + 1, 0);
        h->h_sid.clear();
        for (int c = 0; c < h->ncol; ++c) {
            for (int s = 0; s < nsub; ++s)
                if (h->h_colour[s] == c) h->h_sid.push_back(s);
            h->h_csub_off[c + 1] = (int)h->h_sid.size();
        }
        std::vector<int64_t> ov_off(nsub + 1, 0);
        std::vector<int32_t> Tq(nsub);
        std::vector<int64_t> tile_off(nsub + 1, 0);
        // representation of the local solves: dense inverses while every block
        // fits them, else (or on request) banded Cholesky factors
        int largest = 0;
        for (const auto& om : ov) largest = std::max(largest, (int)om.size());
        const bool band_local = o.local_repr == DDG_LOCAL_BAND ||
                                (o.local_repr == DDG_LOCAL_AUTO && largest > 96 * DDG_LT);
        DDG_REQUIRE(!(band_local && (o.tensor_cores || o.dedup_local)), DDG_EINVAL,
                    "tensor_cores and dedup_local need dense local inverses (local_repr INV)");
        h->bl.on = band_local;
        std::vector<int> bq;   // half-bandwidth of each A_i (band), sweep order
        if (band_local) bq = local_bandwidths(A, ov, h->h_sid);
        // subdomains with equal local matrices share the stored inverse of the
        // first of them (opt.dedup_local); rep[q] == q keeps its own
        std::vector<int32_t> rep(nsub);
        if (o.dedup_local) rep = identical_locals(A, ov, h->h_sid);
        else std::iota(rep.begin(), rep.end(), 0);
        std::vector<int32_t> reps;
        int64_t tile_cursor = 0;
        h->max_local = 0;
        for (int q = 0; q < nsub; ++q) {
            const int nq = (int)ov[h->h_sid[q]].size();
            ov_off[q + 1] = ov_off[q] + nq;
            Tq[q] = (nq + DDG_LT - 1) / DDG_LT;
            if (band_local) {
                tile_off[q] = 0;
            } else if (rep[q] == q) {
                reps.push_back(q);
                tile_off[q] = tile_cursor;
                tile_cursor += (int64_t)ddgdev::packed_elems(Tq[q], ddgdev::packed_narrow_width(nq, Tq[q]));
            } else {
                tile_off[q] = tile_off[rep[q]];
            }
            h->max_local = std::max(h->max_local, nq);
        }
        tile_off[nsub] = tile_cursor;
        h->nrep_local = (int)reps.size();
        h->sum_local = ov_off[nsub];
        h->inv_elems = tile_cursor;
        h->Tmax = (h->max_local + DDG_LT - 1) / DDG_LT;
        DDG_REQUIRE(band_local || h->Tmax <= 96, DDG_EINVAL,
                    "dense local inverses take overlapping subdomains of at most 3072 dofs (local_repr BAND "
                    "takes larger ones)");
        if (band_local) {
            h->Tmax = 1;   // no packed inverses and no dense work items
            h->nrep_local = nsub;
        }
        h->h_ov_off = ov_off;
        h->h_crow_off.assign(h->ncol + 1, 0);
        for (int c = 0; c < h->ncol; ++c) h->h_crow_off[c + 1] = ov_off[h->h_csub_off[c + 1]];
        {
            std::vector<int32_t> ov_nodes(h->sum_local);
            for (int q = 0; q < nsub; ++q)
                std::copy(ov[h->h_sid[q]].begin(), ov[h->h_sid[q]].end(), ov_nodes.begin() + ov_off[q]);
            h->ov_off = h->arena.alloc<int64_t>(nsub + 1);
            h->ov_nodes = h->arena.alloc<int32_t>(h->sum_local);
            h->Tq = h->arena.alloc<int32_t>(nsub);
            h->tile_off = h->arena.alloc<int64_t>(nsub + 1);
            h2d(h->ov_off, ov_off.data(), nsub + 1, h->stream);
            h2d(h->ov_nodes, ov_nodes.data(), h->sum_local, h->stream);
            h2d(h->Tq, Tq.data(), nsub, h->stream);
            h2d(h->tile_off, tile_off.data(), nsub + 1, h->stream);
            DDG_CUDA(cudaStreamSynchronize(h->stream));
        }
        ov.clear();
        ov.shrink_to_fit();

        // ---- local-solve work items: bands of whole tile rows of the packed
        // upper triangle, about `chunk` tiles and at most ls_band_rows rows each
        h->h_Tq = Tq;
        if (o.chunk_tiles > 0) h->ls_chunk = o.chunk_tiles;
        if (!band_local) build_local_items(h, h->ls_chunk, h->ls_band_rows);

        // algorithmic bytes of one local-solve launch per colour and precision:
        // packed triangle of A_i^{-1} + residual read + z read and write
        for (int p = 0; p < 3; ++p) {
            const double se = p == DDG_PREC_FP64 ? 8.0 : (p == DDG_PREC_FP32 ? 4.0 : 2.0);
            const double sv = p == DDG_PREC_FP64 ? 8.0 : 4.0;
            h->colour_bytes[p].assign(h->ncol, 0.0);
            for (int c = 0; c < h->ncol; ++c)
                for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q) {
                    const double nq = (double)(ov_off[q + 1] - ov_off[q]);
                    h->colour_bytes[p][c] += nq * (nq + 1.0) / 2.0 * se + 3.0 * nq * sv;
                }
        }

        // ---- tensor-core slabs and residual layout for the batched solve
        if (o.tensor_cores) {
            std::vector<int64_t> soff(nsub + 1, 0), xo(nsub + 1, 0);
            std::vector<int2> tit;
            h->tc.h_citem_off.assign(h->ncol + 1, 0);
            for (int c = 0; c < h->ncol; ++c) {
                for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q) {
                    const int nq = (int)(ov_off[q + 1] - ov_off[q]);
                    const int Mb = (nq + 127) / 128;
                    for (int b = 0; b < Mb; ++b) tit.push_back(make_int2(q, b));
                }
                h->tc.h_citem_off[c + 1] = (int)tit.size();
            }
            int64_t slab_cursor = 0;
            for (int q = 0; q < nsub; ++q) {
                const int nq = (int)(ov_off[q + 1] - ov_off[q]);
                if (rep[q] == q) {
                    soff[q] = slab_cursor;
                    slab_cursor += (int64_t)((nq + 127) / 128) * Tq[q];
                } else {
                    soff[q] = soff[rep[q]];
                }
                xo[q + 1] = xo[q] + Tq[q];
            }
            soff[nsub] = slab_cursor;
            std::vector<int2> tsl;
            h->tc.h_cslab_off.assign(h->ncol + 1, 0);
            for (int c = 0; c < h->ncol; ++c) {
                for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q)
                    for (int J = 0; J < Tq[q]; ++J) tsl.push_back(make_int2(q, J));
                h->tc.h_cslab_off[c + 1] = (int)tsl.size();
            }
            h->tc.slabs = h->arena.alloc<int2>(tsl.size());
            h2d(h->tc.slabs, tsl.data(), tsl.size(), h->stream);
            h->tc.slab_off = h->arena.alloc<int64_t>(nsub + 1);
            h->tc.xoff = h->arena.alloc<int64_t>(nsub + 1);
            h->tc.items = h->arena.alloc<int2>(tit.size());
            h2d(h->tc.slab_off, soff.data(), nsub + 1, h->stream);
            h2d(h->tc.xoff, xo.data(), nsub + 1, h->stream);
            h2d(h->tc.items, tit.data(), tit.size(), h->stream);
            h->tc.kind = o.tensor_cores;
            h->tc.x_elems = xo[nsub] * (int64_t)DDG_MCHUNK * 32;
            if (o.tensor_cores == DDG_TC_TF32) {
                h->tc.A32 = h->arena.alloc<float>((size_t)soff[nsub] * 128 * 32);
                h->tc.X32 = h->arena.alloc<float>(h->tc.x_elems);
            } else {
                h->tc.A = h->arena.alloc<__nv_bfloat16>((size_t)soff[nsub] * 128 * 32);
                h->tc.X = h->arena.alloc<__nv_bfloat16>(h->tc.x_elems);
            }
            DDG_CUDA(cudaStreamSynchronize(h->stream));
        }

        // ---- local inverses (FP64 factorisation, packed copies)
        h->errflags = h->arena.alloc<int32_t>(E_COUNT);
        DDG_CUDA(cudaMemsetAsync(h->errflags, 0, E_COUNT * sizeof(int32_t), h->stream));
        const size_t tile_elems = (size_t)h->inv_elems;
        if (!band_local) {
            if (keep & (1 << DDG_PREC_FP64)) h->inv64 = h->arena.alloc<double>(tile_elems);
            if (keep & (1 << DDG_PREC_FP32)) h->inv32 = h->arena.alloc<float>(tile_elems);
            if (keep & (1 << DDG_PREC_BF16)) h->inv16 = h->arena.alloc<__nv_bfloat16>(tile_elems);
        }
        if (band_local) {
            setup_band_local(h, bq);
            for (int p = 0; p < 3; ++p) {
                // the block-form factor is read twice (forward, backward) plus
                // the residual read and z read + write
                const double se = p == DDG_PREC_FP64 ? 8.0 : 4.0;
                for (int c = 0; c < h->ncol; ++c) {
                    h->colour_bytes[p][c] = 0.0;
                    for (int q = h->h_csub_off[c]; q < h->h_csub_off[c + 1]; ++q)
                        h->colour_bytes[p][c] += 2.0 * (double)(h->bl.h_qoff[q + 1] - h->bl.h_qoff[q]) * se +
                                                 3.0 * (double)(ov_off[q + 1] - ov_off[q]) * se;
                }
            }
        } else {
            const size_t Np = (size_t)h->Tmax * DDG_LT;
            const size_t per = Np * Np * sizeof(double);
            // chunks of whole waves (a multiple of the SM count), about 3 GB of workspace
            int dev = 0, sms = 1;
            DDG_CUDA(cudaGetDevice(&dev));
            DDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            const size_t budget = (size_t)3 << 30;
            size_t waves = std::max<size_t>(1, budget / (per * (size_t)sms));
            const int nrep = (int)reps.size();
            const int nb = (int)std::min<size_t>((size_t)nrep, waves * (size_t)sms);
            double* ws = h->arena.alloc<double>((size_t)nb * Np * Np);
            double* invdiag = h->arena.alloc<double>((size_t)nb * h->Tmax * DDG_LT * DDG_LT);
            int32_t* qlist = nullptr;
            if (nrep < nsub) {
                qlist = h->arena.alloc<int32_t>(nrep);
                h2d(qlist, reps.data(), nrep, h->stream);
            }
            for (int q0 = 0; q0 < nrep; q0 += nb) {
                const int q1 = std::min(nrep, q0 + nb);
                ddg::local_extract_factor_invert(h, q0, q1, qlist, ws, invdiag);
                ddg::local_pack(h, q0, q1, qlist, ws);
                ddg::tc_pack(h, q0, q1, qlist, ws);
            }
            DDG_CUDA(cudaStreamSynchronize(h->stream));
            h->arena.release(ws);
            h->arena.release(invdiag);
            if (qlist) h->arena.release(qlist);
        }
        if (!band_local) ddg::local_configure(h);
        h->res64 = h->arena.alloc<double>(h->sum_local);
        h->res32 = h->arena.alloc<float>(h->sum_local);
        alloc_partials(h, h->nitems);

        // ---- coarse space (Sec. 4): pairs of subdomains that A couples, then
        // R0, A0 and its factor (or the coarse level of the V-cycle)
        subdomain_pairs(A, partition, sub_off, sub_nodes, nsub, h->h_adjI, h->h_adjJ);
        h->h_sub_nodes = sub_nodes;
        if (h->use_coarse) build_coarse(h, F, k, overlap, o, groups);

        // ---- CG workspace
        h->r = h->arena.alloc<double>(n);
        h->p = h->arena.alloc<double>(n);
        h->q = h->arena.alloc<double>(n);
        h->zc = h->arena.alloc<double>(n);
        h->z64 = h->arena.alloc<double>(n);
        h->fbuf = h->arena.alloc<double>(n);
        h->ubuf = h->arena.alloc<double>(n);
        h->r32 = h->arena.alloc<float>(n);
        h->z32 = h->arena.alloc<float>(n);
        h->scal = h->arena.alloc<double>(S_COUNT);
        DDG_CUDA(cudaMemsetAsync(h->scal, 0, S_COUNT * sizeof(double), h->stream));
        DDG_CUDA(cudaMallocHost((void**)&h->h_scal, S_COUNT * sizeof(double)));
        h->red_partials = h->arena.alloc<double>((size_t)DDG_RED_BLOCKS * 4);
        h->red_counter = h->arena.alloc<unsigned>(1);
        DDG_CUDA(cudaMemsetAsync(h->red_counter, 0, sizeof(unsigned), h->stream));

        if (o.autotune && !band_local) autotune_local(h);

        int32_t flags[E_COUNT];
        d2h(flags, h->errflags, E_COUNT, h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        DDG_REQUIRE(!flags[E_LOCAL_SPD], DDG_ENOTSPD, "a local matrix A_i is not positive definite");
        DDG_REQUIRE(!flags[E_COARSE_SPD], DDG_ENOTSPD, "the coarse matrix A0 is not positive definite");
        h->setup_ms = now_ms() - t0;
        *out = h;
        return DDG_OK;
    } catch (DdgError& e) {
        g_setup_error = e.msg;
        ddg_destroy(h);
        return e.st;
    } catch (std::exception& e) {
        g_setup_error = e.what();
        ddg_destroy(h);
        return DDG_EINVAL;
    }
}

namespace {
// Sec. 6, three-level V-cycle: the two-level method applied again to A0, with
// the coarsened generators F0 = R0 F, on coarse-level subdomains that group
// the fine ones (coarse dof (I, s) belongs to group groups[I]; groups without
// coarse dofs are dropped and the rest numbered in ascending id order).  The
// coarse level's overlap is the same Delta, grown in the graph of A0.
void setup_vcycle(ddg_handle h, const double* F, int k, int overlap, const ddg_options& o,
                  const int32_t* groups, const std::vector<int>& bI, const std::vector<int>& bJ,
                  const std::vector<int64_t>& sub_off, const std::vector<int32_t>& sub_nodes) {
    const int nsub = h->nsub, kmax = h->kmax, n0 = h->n0;
    const int64_t n = h->n;
    const std::vector<int>& coff = h->h_coff;

    // A0 in CSR, both triangles, columns ascending (diagonal blocks taken
    // from their lower triangle, so that the matrix is exactly symmetric)
    std::vector<double> blk;
    ddg::coarse_assemble_blocks(h, bI, bJ, blk);
    struct Nb {
        int J;
        size_t p;
        bool tr;
    };
    std::vector<std::vector<Nb>> nb(nsub);
    for (size_t p = 0; p < bI.size(); ++p) {
        nb[bI[p]].push_back({bJ[p], p, false});
        if (bI[p] != bJ[p]) nb[bJ[p]].push_back({bI[p], p, true});
    }
    for (auto& v : nb) std::sort(v.begin(), v.end(), [](const Nb& a, const Nb& b) { return a.J < b.J; });
    const size_t per = (size_t)kmax * kmax;
    std::vector<int64_t> rp(n0 + 1, 0);
    std::vector<int32_t> cols;
    std::vector<double> vals;
    for (int I = 0; I < nsub; ++I)
        for (int s = 0; s < coff[I + 1] - coff[I]; ++s) {
            for (const Nb& e : nb[I]) {
                const double* B = blk.data() + e.p * per;
                for (int t = 0; t < coff[e.J + 1] - coff[e.J]; ++t) {
                    double v;
                    if (e.J == I) v = B[(size_t)std::max(s, t) * kmax + std::min(s, t)];
                    else if (e.tr) v = B[(size_t)t * kmax + s];
                    else v = B[(size_t)s * kmax + t];
                    cols.push_back(coff[e.J] + t);
                    vals.push_back(v);
                }
            }
            rp[coff[I] + s + 1] = (int64_t)cols.size();
        }
    blk.clear();
    blk.shrink_to_fit();

    // F0 = R0 F: row (I, s) is q_{I,s}^T F on the non-overlapping subdomain I
    // (computed on the device; the coarse level's setup reads it on the host)
    std::vector<double> F0((size_t)n0 * k, 0.0);
    {
        double* dF = h->arena.alloc<double>((size_t)n * k);
        double* dF0 = h->arena.alloc<double>((size_t)n0 * k);
        h2d(dF, F, (size_t)n * k, h->stream);
        ddg::coarse_generators(h, dF, k, dF0);
        d2h(F0.data(), dF0, F0.size(), h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        h->arena.release(dF);
        h->arena.release(dF0);
    }

    // coarse dof -> coarse-level subdomain, ids compacted in ascending order
    std::vector<int32_t> ids;
    for (int I = 0; I < nsub; ++I)
        if (coff[I + 1] > coff[I]) ids.push_back(groups[I]);
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    std::vector<int32_t> part0(n0);
    for (int I = 0; I < nsub; ++I) {
        const int32_t gid = (int32_t)(std::lower_bound(ids.begin(), ids.end(), groups[I]) - ids.begin());
        for (int s = coff[I]; s < coff[I + 1]; ++s) part0[s] = gid;
    }

    ddg_matrix A0{};
    A0.n = n0;
    A0.rowptr = rp.data();
    A0.col = cols.data();
    A0.val = vals.data();
    A0.dofs_per_node = 1;
    A0.stencil_kind = DDG_STENCIL_NONE;
    ddg_options oi = o;
    oi.overlap_mode = DDG_OVERLAP_GRAPH;
    oi.tensor_cores = 0;
    oi.keep_precisions = h->opt.keep_precisions;
    ddg_handle in = nullptr;
    const ddg_status st = setup_impl(&A0, part0.data(), nullptr, F0.data(), k, overlap, &oi, h->stream, &in);
    if (st != DDG_OK) throw DdgError{st, "coarse level of the V-cycle: " + g_setup_error};
    h->inner = in;
    in->use_graphs = false;
    h->n0p = n0;
    h->nK = 0;
    h->c64 = h->arena.alloc<double>(n0);
    DDG_CUDA(cudaMemsetAsync(h->c64, 0, (size_t)n0 * sizeof(double), h->stream));
    h->x64 = in->z64;
    h->c32 = in->r32;
    h->x32 = in->z32;
}
}  // namespace

extern "C" {

ddg_status ddg_setup(const ddg_matrix* A, const int32_t* partition, const double* F, int k,
                     int overlap, const ddg_options* opt, void* stream, ddg_handle* out) {
    return setup_impl(A, partition, nullptr, F, k, overlap, opt, stream, out);
}

ddg_status ddg_setup_vcycle(const ddg_matrix* A, const int32_t* partition, const int32_t* coarse_partition,
                            const double* F, int k, int overlap, const ddg_options* opt, void* stream,
                            ddg_handle* out) {
    ddg_options o;
    if (opt) o = *opt;
    else ddg_default_options(&o);
    if (!coarse_partition || !o.use_coarse) {
        g_setup_error = "the V-cycle needs coarse_partition and use_coarse = 1";
        if (out) *out = nullptr;
        return DDG_EINVAL;
    }
    return setup_impl(A, partition, coarse_partition, F, k, overlap, &o, stream, out);
}

ddg_status ddg_set_generators(ddg_handle h, const double* F, int k) {
    return guarded(h, [&]() {
        DDG_REQUIRE(!h->inner, DDG_EINVAL, "a V-cycle handle keeps the generators it was built with");
        DDG_REQUIRE(F && k >= 1 && k <= DDG_KMAX, DDG_EINVAL, "F must be non-null and k in [1, 96]");
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        // the captured graphs hold launches of the old coarse space
        drop_graphs(h);
        for (void* p : h->coarse_allocs) h->arena.release(p);
        h->coarse_allocs.clear();
        h->Q64 = nullptr;
        h->Q32 = nullptr;
        h->coff = nullptr;
        h->c64 = h->y64 = h->x64 = nullptr;
        h->c32 = h->y32 = h->x32 = nullptr;
        h->Dm = h->Dt = h->Fm = h->Gm = ProfileMat{};
        h->nd = NdCoarse{};
        h->band = 0;
        h->Wt = 1;
        h->NT = h->nK = h->B = h->n0p = 0;
        h->mw.m_alloc = 0;   // the batched workspace is sized by the coarse dimension
        h->use_coarse = 1;
        h->opt.use_coarse = 1;
        DDG_CUDA(cudaMemsetAsync(h->errflags + E_COARSE_SPD, 0, sizeof(int32_t), h->stream));
        build_coarse(h, F, k, 0, h->opt, nullptr);
        int32_t bad = 0;
        d2h(&bad, h->errflags + E_COARSE_SPD, 1, h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        DDG_REQUIRE(!bad, DDG_ENOTSPD, "the coarse matrix A0 is not positive definite");
        return DDG_OK;
    });
}

ddg_status ddg_solve(ddg_handle h, const double* f, double* u, double tol, int* iters, double* relres) {
    return guarded(h, [&]() {
        DDG_REQUIRE(f && u, DDG_EINVAL, "f and u must be non-null device pointers");
        DDG_REQUIRE((const void*)f != (const void*)u, DDG_EINVAL,
                    "f and u must not alias (u is cleared before f is read)");
        DDG_REQUIRE(tol > 0.0, DDG_EINVAL, "tol must be > 0");
        return pcg(h, f, u, tol, iters, relres);
    });
}

ddg_status ddg_solve_host(ddg_handle h, const double* f_host, double* u_host, double tol, int* iters,
                          double* relres) {
    return guarded(h, [&]() {
        DDG_REQUIRE(f_host && u_host, DDG_EINVAL, "f and u must be non-null host pointers");
        DDG_REQUIRE(tol > 0.0, DDG_EINVAL, "tol must be > 0");
        h2d(h->fbuf, f_host, h->n, h->stream);
        const ddg_status st = pcg(h, h->fbuf, h->ubuf, tol, iters, relres);
        d2h(u_host, h->ubuf, h->n, h->stream);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return st;
    });
}

ddg_status ddg_solve_batch(ddg_handle h, const double* F, double* U, int m, double tol, int* iters,
                           double* relres) {
    return guarded(h, [&]() {
        DDG_REQUIRE(F && U && m >= 1, DDG_EINVAL, "F, U must be non-null and m >= 1");
        DDG_REQUIRE(tol > 0.0, DDG_EINVAL, "tol must be > 0");
        ddg_status worst = DDG_OK;
        if (h->precision == DDG_PREC_FP64 || h->inner || h->kmax > 32 || h->bl.on) {
            // the FP64 and the V-cycle preconditioners, and coarse spaces of
            // more than 32 generators per subdomain, run one column at a time
            for (int j = 0; j < m; ++j) {
                ddg::strided_gather(h, F, m, j, h->fbuf);
                int it = 0;
                double rr = 0.0;
                const ddg_status st = pcg(h, h->fbuf, h->ubuf, tol, &it, &rr);
                ddg::strided_scatter(h, h->ubuf, m, j, U);
                if (iters) iters[j] = it;
                if (relres) relres[j] = rr;
                if (st != DDG_OK && worst == DDG_OK) worst = st;
            }
        } else if (m <= DDG_MCHUNK) {
            worst = pcg_batch(h, F, U, m, tol, iters, relres);
        } else {
            // groups of DDG_MCHUNK columns through staging blocks
            ddg::multi_ensure(h, DDG_MCHUNK);
            for (int j0 = 0; j0 < m; j0 += DDG_MCHUNK) {
                const int mg = std::min(DDG_MCHUNK, m - j0);
                ddg::copy_cols(h, F, m, j0, h->mw.Fb, mg, 0, mg);
                const ddg_status st = pcg_batch(h, h->mw.Fb, h->mw.Ub, mg, tol, iters ? iters + j0 : nullptr,
                                                relres ? relres + j0 : nullptr);
                ddg::copy_cols(h, h->mw.Ub, mg, 0, U, m, j0, mg);
                if (st != DDG_OK && worst == DDG_OK) worst = st;
            }
        }
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return worst;
    });
}

ddg_status ddg_solve_many(ddg_handle* hs, int nprob, const double* const* F, double* const* U,
                          const int* m, double tol, int* iters, double* relres) {
    if (!hs || !F || !U || !m || nprob < 1) return DDG_EINVAL;
    for (int p = 0; p < nprob; ++p) {
        if (!hs[p] || !F[p] || !U[p] || m[p] < 1) return DDG_EINVAL;
        for (int q = 0; q < p; ++q)
            if (hs[q] == hs[p]) return DDG_EINVAL;   // a handle serves one thread
    }
    if (!(tol > 0.0)) return DDG_EINVAL;
    std::vector<int64_t> off(nprob + 1, 0);
    for (int p = 0; p < nprob; ++p) off[p + 1] = off[p] + m[p];
    {
        // single right-hand sides on one device: every problem's whole solve
        // is a branch of one CUDA graph, launched once
        ddg_status st = DDG_OK;
        if (solve_many_graph(hs, nprob, F, U, m, tol, iters, relres, st)) return st;
    }
    std::vector<ddg_status> st(nprob, DDG_OK);
    std::vector<std::thread> th;
    th.reserve(nprob);
    for (int p = 0; p < nprob; ++p)
        th.emplace_back([&, p]() {
            int* it = iters ? iters + off[p] : nullptr;
            double* rr = relres ? relres + off[p] : nullptr;
            if (m[p] == 1) st[p] = ddg_solve(hs[p], F[p], U[p], tol, it, rr);
            else st[p] = ddg_solve_batch(hs[p], F[p], U[p], m[p], tol, it, rr);
        });
    for (auto& t : th) t.join();
    for (int p = 0; p < nprob; ++p)
        if (st[p] != DDG_OK) return st[p];
    return DDG_OK;
}

ddg_status ddg_adjoint(ddg_handle h, const double* dLdu, double* lambda, double tol, int* iters,
                       double* relres) {
    return ddg_solve(h, dLdu, lambda, tol, iters, relres);
}

ddg_status ddg_grad_coeff(ddg_handle h, const double* lambda, const double* u, double* dcoef) {
    return guarded(h, [&]() {
        DDG_REQUIRE(lambda && u && dcoef, DDG_EINVAL, "null pointer");
        if (h->stencil_kind == DDG_STENCIL_Q1_ELASTIC && h->kmu) {
            ddg::grad_coeff_q1(h, lambda, u, dcoef);
        } else {
            DDG_REQUIRE(h->stencil_kind == DDG_STENCIL_VAR7_3D && h->kappa, DDG_EINVAL,
                        "ddg_grad_coeff needs a VAR7 or Q1 handle set up with its coefficients");
            ddg::grad_coeff_var7(h, lambda, u, dcoef);
        }
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return DDG_OK;
    });
}

ddg_status ddg_apply_preconditioner(ddg_handle h, const double* r, double* z) {
    return guarded(h, [&]() {
        DDG_REQUIRE(r && z, DDG_EINVAL, "null pointer");
        apply_prec(h, r);
        if (h->precision == DDG_PREC_FP64)
            DDG_CUDA(cudaMemcpyAsync(z, h->z64, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        else
            ddg::convert_to_double(h, h->z32, z);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return DDG_OK;
    });
}

ddg_status ddg_coarse_correction(ddg_handle h, const double* r, double* z) {
    return guarded(h, [&]() {
        DDG_REQUIRE(r && z, DDG_EINVAL, "null pointer");
        DDG_REQUIRE(h->use_coarse, DDG_EINVAL, "the handle has no coarse space");
        const int prec = h->precision;
        if (prec == DDG_PREC_FP64) {
            h->rin64 = r;
            DDG_CUDA(cudaMemsetAsync(h->z64, 0, h->n * sizeof(double), h->stream));
        } else {
            ddg::convert_to_float(h, r, h->r32);
            DDG_CUDA(cudaMemsetAsync(h->z32, 0, h->n * sizeof(float), h->stream));
        }
        coarse_step(h, prec, false);
        if (prec == DDG_PREC_FP64)
            DDG_CUDA(cudaMemcpyAsync(z, h->z64, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        else
            ddg::convert_to_double(h, h->z32, z);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return DDG_OK;
    });
}

ddg_status ddg_spmv(ddg_handle h, const double* x, double* y) {
    return guarded(h, [&]() {
        DDG_REQUIRE(x && y, DDG_EINVAL, "null pointer");
        ddg::spmv64(h, x, y, false, 0);
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        return DDG_OK;
    });
}

ddg_status ddg_set_debug(ddg_handle h, int flags) {
    return guarded(h, [&]() {
        DDG_REQUIRE((flags & ~DDG_DEBUG_TC_NO_COPIES) == 0, DDG_EINVAL, "unknown debug flag");
        DDG_CUDA(cudaStreamSynchronize(h->stream));
        if (flags != h->debug) drop_graphs(h);   // the flags are launch arguments of captured kernels
        h->debug = flags;
        return DDG_OK;
    });
}

ddg_status ddg_set_precision(ddg_handle h, int precision) {
    return guarded(h, [&]() {
        DDG_REQUIRE(precision >= DDG_PREC_FP64 && precision <= DDG_PREC_BF16, DDG_EINVAL, "bad precision");
        DDG_REQUIRE(h->opt.keep_precisions & (1 << precision), DDG_EINVAL,
                    "that precision was not kept at setup (keep_precisions)");
        h->precision = precision;
        return DDG_OK;
    });
}

ddg_status ddg_set_stream(ddg_handle h, void* stream) {
    return guarded(h, [&]() {
        h->stream = (cudaStream_t)stream;
        if (h->inner) h->inner->stream = h->stream;
        return DDG_OK;
    });
}

ddg_status ddg_get_info(ddg_handle h, ddg_info* info) {
    return guarded(h, [&]() {
        DDG_REQUIRE(info, DDG_EINVAL, "null pointer");
        info->n = h->n;
        info->nsub = h->nsub;
        info->ncolours = h->ncol;
        info->n0 = h->use_coarse ? h->n0 : 0;
        info->kmax = h->kmax;
        info->max_local = h->max_local;
        info->sum_local = h->sum_local;
        info->local_tiles = (h->inv_elems + 1023) / 1024;
        info->coarse_band = h->band;
        info->coarse_blocks = h->nK;
        info->setup_ms = h->setup_ms;
        info->precision = h->precision;
        info->local_inverses = h->nrep_local;
        info->graph_solve = h->solve_graph_failed ? -1 : h->last_solve_graph;
        info->ls_warps = h->ls_warps;
        info->ls_chunk_tiles = h->ls_chunk;
        info->ls_band_rows = h->ls_band_rows;
        info->tc_stages = h->tc_stages;
        info->tuned = h->tuned;
        info->local_repr = h->bl.on ? DDG_LOCAL_BAND : DDG_LOCAL_INV;
        info->local_band = h->bl.on ? h->bl.b : 0;
        info->local_elems = h->bl.on ? h->bl.elems : h->inv_elems;
        info->coarse_order = h->nd.on ? DDG_COARSE_ND : DDG_COARSE_BAND;
        info->coarse_fronts = h->nd.on ? h->nd.nfront : 0;
        info->coarse_levels = h->nd.on ? h->nd.nlevel : 0;
        info->coarse_elems = h->nd.on ? h->nd.elems : (h->use_coarse ? h->Dm.nnz + h->Dt.nnz + h->Fm.nnz + h->Gm.nnz : 0);
        return DDG_OK;
    });
}

ddg_status ddg_get_colouring(ddg_handle h, int32_t* colour) {
    return guarded(h, [&]() {
        DDG_REQUIRE(colour, DDG_EINVAL, "null pointer");
        for (int s = 0; s < h->nsub; ++s) colour[s] = h->h_colour[s];
        return DDG_OK;
    });
}

ddg_status ddg_get_coarse_offsets(ddg_handle h, int32_t* offsets) {
    return guarded(h, [&]() {
        DDG_REQUIRE(offsets, DDG_EINVAL, "null pointer");
        for (int s = 0; s <= h->nsub; ++s) offsets[s] = h->use_coarse ? h->h_coff[s] : 0;
        return DDG_OK;
    });
}

ddg_status ddg_get_history(ddg_handle h, double* hist, int max_len, int* len) {
    return guarded(h, [&]() {
        const int cnt = (int)h->history.size();
        if (len) *len = cnt;
        if (hist)
            for (int i = 0; i < std::min(cnt, max_len); ++i) hist[i] = h->history[i];
        return DDG_OK;
    });
}

ddg_status ddg_get_cg_coefficients(ddg_handle h, double* alpha, double* beta, int max_len, int* len) {
    return guarded(h, [&]() {
        const int cnt = (int)h->cg_alpha.size();
        if (len) *len = cnt;
        for (int i = 0; i < std::min(cnt, max_len); ++i) {
            if (alpha) alpha[i] = h->cg_alpha[i];
            if (beta && i + 1 < cnt) beta[i] = h->cg_beta[i];
        }
        return DDG_OK;
    });
}

ddg_status ddg_condition_estimate(const double* alpha, const double* beta, int m, double tol,
                                  double* lambda_min, double* lambda_max, double* iter_bound) {
    if (!alpha || (m > 1 && !beta) || m < 1 || !lambda_min || !lambda_max || !(tol > 0.0 && tol < 1.0)) {
        ddg::set_handleless_error("alpha, beta, lambda_min, lambda_max must be non-null, m >= 1, 0 < tol < 1");
        return DDG_EINVAL;
    }
    for (int j = 0; j < m; ++j)
        if (!(alpha[j] > 0.0) || (j + 1 < m && !(beta[j] >= 0.0))) {
            ddg::set_handleless_error("alpha must be > 0 and beta >= 0");
            return DDG_EINVAL;
        }
    // T = tridiag(e, d, e): d_0 = 1/alpha_0, d_j = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    // e_j = sqrt(beta_j)/alpha_j
    std::vector<double> d(m), e2(m > 1 ? m - 1 : 1, 0.0);
    for (int j = 0; j < m; ++j) d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    for (int j = 0; j + 1 < m; ++j) e2[j] = beta[j] / (alpha[j] * alpha[j]);
    // Gershgorin interval
    double lo = d[0], hi = d[0];
    for (int j = 0; j < m; ++j) {
        const double r = (j > 0 ? std::sqrt(e2[j - 1]) : 0.0) + (j + 1 < m ? std::sqrt(e2[j]) : 0.0);
        lo = std::min(lo, d[j] - r);
        hi = std::max(hi, d[j] + r);
    }
    // Sturm count: the number of eigenvalues of T below x (LDL^T pivots)
    auto below = [&](double x) {
        int cnt = 0;
        double q = d[0] - x;
        const double tiny = 1e-300;
        for (int j = 0;; ++j) {
            if (q == 0.0) q = -tiny;
            if (q < 0.0) ++cnt;
            if (j + 1 == m) break;
            q = d[j + 1] - x - e2[j] / q;
        }
        return cnt;
    };
    // the k-th smallest eigenvalue (k = 1..m) by bisection
    auto kth = [&](int k) {
        double a = lo, b = hi;
        for (int it = 0; it < 400 && b - a > 1e-14 * std::max(std::fabs(a), std::fabs(b)); ++it) {
            const double mid = 0.5 * (a + b);
            if (below(mid) >= k) b = mid;
            else a = mid;
        }
        return 0.5 * (a + b);
    };
    *lambda_min = kth(1);
    *lambda_max = kth(m);
    if (iter_bound) {
        const double kappa = *lambda_max / *lambda_min;
        if (!(kappa > 1.0)) {
            *iter_bound = 0.0;
        } else {
            const double sk = std::sqrt(kappa);
            *iter_bound = std::log(2.0 / tol) / std::log((sk + 1.0) / (sk - 1.0));
        }
    }
    return DDG_OK;
}

ddg_status ddg_profile(ddg_handle h, int timed_mask) {
    return guarded(h, [&]() {
        prof_flush(h);
        h->prof_mask = timed_mask;
        for (int c = 0; c < DDG_K_COUNT; ++c) {
            h->prof_launches[c] = h->prof_timed[c] = 0;
            h->prof_ms[c] = h->prof_bytes[c] = 0.0;
        }
        return DDG_OK;
    });
}

ddg_status ddg_get_kernel_stats(ddg_handle h, ddg_kernel_stat* st) {
    return guarded(h, [&]() {
        DDG_REQUIRE(st, DDG_EINVAL, "null pointer");
        prof_flush(h);
        for (int c = 0; c < DDG_K_COUNT; ++c) {
            st[c].launches = h->prof_launches[c];
            st[c].timed = h->prof_timed[c];
            st[c].ms = h->prof_ms[c];
            st[c].bytes = h->prof_bytes[c];
        }
        return DDG_OK;
    });
}

ddg_status ddg_destroy(ddg_handle h) {
    if (!h) return DDG_OK;
    DeviceScope scope(h->device);
    drop_many_graphs(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->inner) ddg_destroy(h->inner);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (cudaGraphExec_t g : h->apply_exec)
        if (g) cudaGraphExecDestroy(g);
    for (cudaGraphExec_t g : h->solve_exec)
        if (g) cudaGraphExecDestroy(g);
    for (auto& pe : h->batch_exec)
        for (auto& e : pe) cudaGraphExecDestroy(e.exec);
    if (h->mw.h_ctl) cudaFreeHost(h->mw.h_ctl);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    h->arena.free_all();
    if (h->h_scal) cudaFreeHost(h->h_scal);
    delete h;
    return DDG_OK;
}

const char* ddg_last_error(ddg_handle h) {
    if (!h) return g_setup_error.c_str();
    return h->err.c_str();
}

const char* ddg_status_string(ddg_status s) {
    switch (s) {
        case DDG_OK: return "DDG_OK";
        case DDG_EINVAL: return "DDG_EINVAL";
        case DDG_ENOMEM: return "DDG_ENOMEM";
        case DDG_ENOTSPD: return "DDG_ENOTSPD";
        case DDG_EBREAKDOWN: return "DDG_EBREAKDOWN";
        case DDG_ENOCONV: return "DDG_ENOCONV";
        case DDG_ETIMEOUT: return "DDG_ETIMEOUT";
        case DDG_ECUDA: return "DDG_ECUDA";
    }
    return "unknown status";
}

}  // extern "C"
