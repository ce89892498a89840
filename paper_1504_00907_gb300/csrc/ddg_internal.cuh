// Internal declarations of the DDG solver library (not part of the C ABI).
//
// Data layout in HBM (all device arrays are owned by the handle):
//   * fine matrix A: CSR (int64 rowptr, int32 col, FP64 and FP32 values);
//   * non-overlapping subdomains (Sec. 4) in id order: sub_off[nsub+1],
//     sub_nodes[n] (ascending per subdomain), pos[g] = index of g in
//     sub_nodes; the coarse basis Q is stored per such position, kmax values
//     per node (row-major), FP64 and FP32;
//   * overlapping subdomains (Sec. 6) in *sweep order* q (colour-major, ids
//     ascending inside a colour): ov_off[nsub+1], ov_nodes (sorted per
//     subdomain); colour c owns sweep positions csub_off[c]..csub_off[c+1]
//     and local rows crow_off[c]..crow_off[c+1];
//   * local inverses A_i^{-1}: zero-padded to T_q = ceil(n_q/32) tiles per
//     side, upper-triangular 32x32 tiles (I <= J) in row-major tile order,
//     each tile row-major; the diagonal tiles hold the full symmetric tile;
//   * coarse factor: A0 = L L^T in 64x64 tiles inside the band, regrouped
//     into super-blocks of Wt tiles: y_K = D_K (c_K - E_K y_{K-1}) forward
//     and x_K = D_K^T (y_K - E_{K+1}^T x_{K+1}) backward, with D_K = L_KK^{-1};
//     D, E, D^T, E^T are stored as "profile rows" (contiguous column range
//     per row) in FP64 and FP32.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "ddg.h"
#include "dev_common.cuh"

#define DDG_LT 32        // local-inverse tile edge
#define DDG_CT 64        // coarse factor tile edge
#define DDG_KMAX 96      // largest supported number of generators (a multiple of 32)
#define DDG_RED_BLOCKS 1216  // blocks of the deterministic reductions (8 x 152 SMs)
#define DDG_BAND_ROWS 16     // tile rows per local-solve work item at most
#define DDG_GATHER_SPLIT_CHUNKS 8  // chunks per subdomain above which the gather is a kernel of its own
#define DDG_MCHUNK 64        // right-hand sides per batched PCG group

// ---------------------------------------------------------------- errors
struct DdgError {
    ddg_status st;
    std::string msg;
};

#define DDG_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t _e = (call);                                                    \
        if (_e != cudaSuccess)                                                      \
            throw DdgError{_e == cudaErrorMemoryAllocation ? DDG_ENOMEM : DDG_ECUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(_e)};      \
    } while (0)

#define DDG_CHECK_LAUNCH() DDG_CUDA(cudaGetLastError())

#define DDG_REQUIRE(cond, status, text)                \
    do {                                               \
        if (!(cond)) throw DdgError{status, (text)};   \
    } while (0)

// A kernel attribute (cudaFuncSetAttribute) is set per device: the largest
// value set so far on each device, so that every device is configured once
// and a value is never lowered.
struct PerDeviceMax {
    std::mutex mu;
    int value[64] = {};
    // true when `want` exceeds the value recorded for the current device (the
    // caller then sets the attribute and calls commit)
    bool needs(int want, int& dev) {
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = -1;
        std::lock_guard<std::mutex> lock(mu);
        return dev < 0 || want > value[dev];
    }
    void commit(int dev, int want) {
        if (dev < 0) return;
        std::lock_guard<std::mutex> lock(mu);
        if (want > value[dev]) value[dev] = want;
    }
};

// device allocation helper: every allocation is recorded for ddg_destroy
struct DevArena {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    template <typename T>
    T* alloc(size_t count) {
        if (count == 0) count = 1;
        void* p = nullptr;
        DDG_CUDA(cudaMalloc(&p, count * sizeof(T)));
        ptrs.push_back(p);
        bytes += count * sizeof(T);
        return static_cast<T*>(p);
    }
    void release(void* p) {
        for (auto& q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
    void free_all() {
        for (void* p : ptrs)
            if (p) cudaFree(p);
        ptrs.clear();
    }
};

template <typename T>
static inline void h2d(T* dst, const T* src, size_t count, cudaStream_t s) {
    if (count) DDG_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
}
template <typename T>
static inline void d2h(T* dst, const T* src, size_t count, cudaStream_t s) {
    if (count) DDG_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToHost, s));
}

// Launch a kernel that may start before its predecessor in the stream ends
// (programmatic dependent launch, when h->use_pdl): the kernel itself
// executes griddepcontrol.wait before it reads anything the predecessor
// writes.  Kernels after a memset or a copy keep the ordinary dependency.
template <typename... KArgs, typename... Args>
static inline void launch_pdl(ddg_handle h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              Args&&... args);

// kernel flavour of the A z products: the matrix-free Laplacians, or the CSR
// path with rows unrolled when they are short (see dev_common.cuh)
#define DDG_DISPATCH_SK(h, CALL)                                                  \
    do {                                                                          \
        if ((h)->stencil_kind == DDG_STENCIL_7PT_3D) { CALL(DDG_STENCIL_7PT_3D); } \
        else if ((h)->stencil_kind == DDG_STENCIL_5PT_2D) { CALL(DDG_STENCIL_5PT_2D); } \
        else if ((h)->max_row_nnz <= 8) { CALL(100); }                             \
        else if ((h)->max_row_nnz <= 16) { CALL(101); }                            \
        else if ((h)->wide_rows) { CALL(102); }                                    \
        else { CALL(DDG_STENCIL_NONE); }                                           \
    } while (0)

// device scalar slots of the CG recurrence (FP64)
enum {
    S_RZ = 0,      // rho_k = r_k^T z_k
    S_PQ = 1,      // p^T A p
    S_RR = 2,      // ||r||^2
    S_ALPHA = 3,
    S_BETA = 4,
    S_QZ = 5,      // q_k^T z_{k+1} (Polak-Ribiere)
    S_RZNEW = 6,
    S_TMP = 7,
    S_FLAG = 8,    // breakdown flag (1.0 when p^T A p <= 0 or NaN)
    S_COUNT = 16
};

// Device-side state of a graph-driven PCG solve (one CUDA graph whose
// conditional WHILE node repeats the CG iteration; the control kernels
// decide convergence, breakdown, the true-residual check and restarts).
enum { CG_RUN = 0, CG_CONV = 1, CG_BREAKDOWN = 2, CG_MAXIT = 3, CG_STALLED = 4, CG_ZERO = 5, CG_NANRHS = 6,
       CG_TIMEOUT = 7 };
#define DDG_MAX_RESTARTS 3
struct CgCtl {
    int it;            // iterations done
    int restarts;      // true-residual restarts done
    int state;         // CG_*
    int check;         // the recurrence met tol this iteration: check the true residual
    int first;         // the next p update starts a segment (beta = 0)
    int restart_now;   // copy the true residual into r before the next iteration
    int need_final;    // the loop ended without a true residual: compute it after the loop
    int maxit;
    int seg_start[DDG_MAX_RESTARTS + 1];   // first iteration of each restart segment
    double tol, fn, true_rel, pad;
};

// error flags written by kernels (int32)
enum { E_LOCAL_SPD = 0, E_COARSE_SPD = 1, E_TIMEOUT = 2, E_COUNT = 4 };

// ---------------------------------------------------------------- handle
struct ProfileMat {         // rows with one contiguous column range each
    int64_t* rowptr = nullptr;  // [rows + 1]
    int32_t* lo = nullptr;      // [rows], global column of the first entry
    int32_t* hi = nullptr;      // [rows], one past the last column
    double* v64 = nullptr;
    float* v32 = nullptr;
    int64_t nnz = 0;
    std::vector<int64_t> h_rowptr;   // host copy of rowptr
};

// Device-side state of a graph-driven batched PCG (per column: its own CG)
struct MultiCtl {
    int it, maxit, any_cand, any_restart, any_unfinished, timed_out, pad0, pad1;
    double tol;
    int done_it[DDG_MCHUNK], cstat[DDG_MCHUNK], nrest[DDG_MCHUNK], cand[DDG_MCHUNK];
    double fn[DDG_MCHUNK], done_rel[DDG_MCHUNK];
};

// workspace of the batched (multi-RHS) PCG, grown on first use
struct MultiWork {
    bool r32_current = false;   // r32 holds (float)R (written by update_ur)
    int m_alloc = 0;
    double *R = nullptr, *P = nullptr, *Q = nullptr, *T = nullptr;   // n x m FP64
    double *Fb = nullptr, *Ub = nullptr;                              // column-group staging
    float *r32 = nullptr, *z32 = nullptr, *res32 = nullptr;
    float *c32 = nullptr, *y32 = nullptr, *x32 = nullptr;
    double* scal = nullptr;       // [S_COUNT][DDG_MCHUNK]
    double* partials = nullptr;   // [DDG_RED_BLOCKS][2][DDG_MCHUNK]
    int* active = nullptr;        // [DDG_MCHUNK]
    int* restart = nullptr;       // [DDG_MCHUNK]
    int2* items = nullptr;        // (sweep position, tile row) per colour
    std::vector<int> h_citem_off;
    float* gpart = nullptr;       // split partials of the coarse GEMMs
    unsigned* gtick = nullptr;    // one ticket per 32-row tile
    float *ndw = nullptr, *ndx = nullptr;   // nested-dissection coarse solve: vectors in elimination order
    float* ndp = nullptr;                   // and its partial G rows
    int gen = 0;                  // bumped when the workspace is reallocated
    MultiCtl* ctl = nullptr;      // graph-driven batched solves
    MultiCtl* h_ctl = nullptr;    // pinned
};

// banded local factors (local_repr BAND): the Cholesky factor of every A_i in
// block form, super-blocks of B = 64 Wt rows; per super-block K the stored
// rows of C_K = L_{K,K-1} (rows i < b, columns [(B - b + i) & ~3, B)) and of
// D_K = L_KK^{-1} (row i: columns [0, i] padded to a multiple of 4)
#define DDG_BAND_STAGE_BYTES 32768
struct BandLocal {
    bool on = false;
    int Wt = 0, B = 0, b = 0;          // tiles per super-block, its rows, half-bandwidth
    int sizeC = 0, sizeD = 0;          // stored elements of one C_K / D_K
    int vec_elems = 0;                 // largest nK_q * B
    int stages64 = 0, stages32 = 0;    // shared-memory ring depth per precision
    std::vector<int> h_nk;             // [nsub] super-blocks per subdomain (sweep position)
    std::vector<int64_t> h_qoff;       // [nsub + 1] element offsets of each subdomain's blocks
    int32_t* nk = nullptr;
    int64_t* qoff = nullptr;
    int32_t *rowC = nullptr, *rowD = nullptr;   // [b + 1], [B + 1] row offsets inside a block
    int2 *ch64C = nullptr, *ch64D = nullptr, *ch32C = nullptr, *ch32D = nullptr;   // row chunks
    int nch64C = 0, nch64D = 0, nch32C = 0, nch32D = 0;
    double* d64 = nullptr;
    float* d32 = nullptr;
    int64_t elems = 0;
};

// nested-dissection coarse factor (coarse_order ND): per front the rows of
// D = L_SS^{-1} (row i: columns [0, i] padded to 4) and of L_US (row u: nS
// columns padded to 4), work lists per level (deepest first)
struct NdCoarse {
    bool on = false;
    int nfront = 0, nlevel = 0;
    int64_t elems = 0;                 // stored elements (one precision): D, G, D^T, G^T
    int32_t *nS = nullptr, *nU = nullptr, *s0 = nullptr;   // front sizes, first S position
    int32_t *up = nullptr;             // positions of the fronts' U dofs (elimination order)
    int32_t* elim = nullptr;           // [n0] coarse dof at each elimination position
    int64_t *uoff = nullptr, *doff = nullptr, *goff = nullptr, *dtoff = nullptr, *gtoff = nullptr;
    int2 *fitems = nullptr, *bitems = nullptr;   // forward / backward items per level
    int32_t* rtgt = nullptr;           // targets of the forward updates, per level
    int64_t* rptr = nullptr;
    int2* rsrc = nullptr;              // (front, G row) pairs per target, in a fixed order
    std::vector<int> h_fwd_off, h_bwd_off;   // [nlevel + 1], levels deepest first
    // multi-column solve: 32-row tiles (front, first row, D or G) forward and
    // (front, first row) backward, targets per level, partial-row index of
    // every listed (front, G row) pair, total G rows
    int4* mfitems = nullptr;
    int2* mbitems = nullptr;
    int64_t* rsrcp = nullptr;
    std::vector<int> h_mf_off, h_mb_off, h_tgt_off;
    std::vector<int> h_mf_ks, h_mb_ks;   // CTAs per tile (one cluster) per level
    std::vector<int> h_fwd_wpr, h_bwd_wpr;   // warps per item of the single-vector solve, per level
    std::vector<int> h_fwd_pf, h_bwd_pf;     // whether a level prefetches its factor rows into L2
    int64_t urows = 0;
    int32_t *fwd_off = nullptr, *bwd_off = nullptr;   // device copies
    unsigned* bar = nullptr;           // grid barrier of the persistent solve
    bool persistent = false;           // one cooperative launch (DDG_ND_PERSISTENT=1) or one per level
    double *d64 = nullptr, *w64 = nullptr, *x64 = nullptr;
    float *d32 = nullptr, *w32 = nullptr, *x32 = nullptr;
};

// tensor-core (tcgen05) multi-RHS local solves: BF16 slabs of every A_i^{-1}
struct TcData {
    int kind = 0;                  // DDG_TC_*: the operand type of the slabs below
    __nv_bfloat16* A = nullptr;    // 128 x 32 slabs, core-matrix order (BF16)
    __nv_bfloat16* X = nullptr;    // residual slabs N x 32 per subdomain (BF16)
    float* A32 = nullptr;          // the same slabs in TF32 (FP32 storage)
    float* X32 = nullptr;
    int64_t* slab_off = nullptr;   // [nsub + 1] in A slabs
    int64_t* xoff = nullptr;       // [nsub + 1] in X slabs
    int2* items = nullptr;         // (sweep position, 128-row block) per colour
    std::vector<int> h_citem_off;
    int2* slabs = nullptr;         // (sweep position, 32-row K slab) per colour
    std::vector<int> h_cslab_off;
    int64_t x_elems = 0;
    int last_m = -1;
    // the precision whose batched local solves run on the tensor cores
    int prec() const { return kind == DDG_TC_BF16 ? DDG_PREC_BF16 : (kind == DDG_TC_TF32 ? DDG_PREC_FP32 : -1); }
    size_t x_bytes() const { return (size_t)x_elems * (kind == DDG_TC_TF32 ? 4 : 2); }
    void* x_ptr() const { return kind == DDG_TC_TF32 ? (void*)X32 : (void*)X; }
};

struct ddg_handle_s {
    DevArena arena;
    cudaStream_t stream = nullptr;
    ddg_options opt{};
    std::string err;
    int precision = DDG_PREC_FP64;
    double setup_ms = 0.0;
    int device = 0;                 // CUDA device current at setup; made current by every call
    // launch shapes (autotuned when opt.autotune is set): warps per local-solve
    // CTA, tiles and tile rows per local-solve work item, tensor-core ring depth
    int ls_warps = 8, ls_chunk = 96, ls_band_rows = DDG_BAND_ROWS, tc_stages = 4;
    int tuned = 0;                  // 1: ls_* chosen by timing candidates (or a cached choice)
    double tune_ms = 0.0;           // local-solve time of one colour phase with the choice
    int debug = 0;                  // DDG_DEBUG_* test hooks (ddg_set_debug)
    unsigned long long wait_ns = 1000000000ull;   // limit of every device-side wait

    // ---- fine problem
    int64_t n = 0, nnz = 0;
    int max_row_nnz = 0;        // longest CSR row (selects the unrolled row kernels)
    bool wide_rows = false;     // rows average >= 32 entries: a lane group per row
    int stencil_kind = 0, dim = 0, nx = 1, ny = 1, nz = 1, dpn = 1;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val64 = nullptr;
    float* val32 = nullptr;
    double* kappa = nullptr;    // VAR7 cell coefficients / Q1 shear moduli (device)
    double* kmu = nullptr;      // Q1: 24 x 24 element matrix dK_e / dmu_e (device)
    int64_t ncoef = 0;

    // ---- partition (Sec. 4) in id order
    int nsub = 0;
    int32_t* part = nullptr;       // [n]
    int64_t* sub_off = nullptr;    // [nsub + 1]
    int32_t* sub_nodes = nullptr;  // [n]
    int32_t* pos = nullptr;        // [n]
    std::vector<int64_t> h_sub_off;

    // ---- overlapping subdomains in sweep order (Sec. 6)
    int ncol = 0;
    std::vector<int> h_colour;     // [nsub] colour of each id
    std::vector<int> h_sid;        // [nsub] sweep position -> id
    std::vector<int> h_csub_off;   // [ncol + 1]
    std::vector<int64_t> h_crow_off;
    std::vector<int64_t> h_ov_off;
    int64_t sum_local = 0;
    int max_local = 0, Tmax = 0;
    int64_t* ov_off = nullptr;
    int32_t* ov_nodes = nullptr;
    int32_t* Tq = nullptr;
    std::vector<int32_t> h_Tq;     // [nsub] tile rows of each packed inverse (host)
    int64_t* tile_off = nullptr;   // [nsub + 1] element offset of each packed inverse
    int64_t inv_elems = 0;         // elements of all packed inverses
    // local-solve work items per colour: {q, tile_begin, tile_end, unused}
    std::vector<int> h_citem_off;
    int nitems = 0;
    int4* items = nullptr;
    int32_t* nchunks = nullptr;
    int32_t* first_item = nullptr;
    unsigned* counters = nullptr;
    int32_t* ov_sub = nullptr;      // [sum_local] sweep position of each local row
    int32_t* row_nchunks = nullptr; // [sum_local] chunks whose band starts at or above the row
    // subdomains cut into many chunks sum their chunk partials in a separate
    // row-parallel kernel instead of in the CTA that finishes last
    bool split_gather = false;
    // dependent launches of chained kernels may start before their predecessor
    // ends (programmatic dependent launch); DDG_PDL=0 turns it off
    bool use_pdl = true;
    double* inv64 = nullptr;
    float* inv32 = nullptr;
    __nv_bfloat16* inv16 = nullptr;
    // partial results of the local GEMV: [nitems][Tmax * 32]
    double* partial64 = nullptr;
    float* partial32 = nullptr;
    double* res64 = nullptr;       // [sum_local]
    float* res32 = nullptr;

    // ---- coarse space (Sec. 4)
    int use_coarse = 1;
    int kmax = 0, n0 = 0;
    std::vector<int> h_coff;
    int32_t* coff = nullptr;       // [nsub + 1]
    double* Q64 = nullptr;         // [n * kmax] by position
    float* Q32 = nullptr;
    int band = 0, Wt = 1, NT = 0, nK = 0, B = 0, n0p = 0;
    double* bandL = nullptr;       // [NT][Wt+1][64*64] (setup only)
    double* coarseW = nullptr;     // super-block inverses (setup only)
    // block-bidiagonal factor: D_K = L_KK^{-1} (Dm) and its transpose (Dt);
    // coupling blocks F_K = D_K L_{K,K-1} (Fm) and G_K = D_K^T L_{K+1,K}^T (Gm)
    ProfileMat Dm, Dt, Fm, Gm;
    double *c64 = nullptr, *y64 = nullptr, *x64 = nullptr;
    float *c32 = nullptr, *y32 = nullptr, *x32 = nullptr;
    // three-level V-cycle (Sec. 6): the two-level preconditioner of A0 that
    // replaces A0^{-1}.  Its input r32 and outputs z32, z64 are this handle's
    // c32, x32 and x64 (owned by the inner handle); it reads c64 in place.
    ddg_handle_s* inner = nullptr;
    // subdomain pairs that A couples (I >= J), the partition's node lists and
    // the device memory of the coarse space (released when it is rebuilt)
    std::vector<int> h_adjI, h_adjJ;
    std::vector<int32_t> h_sub_nodes;
    std::vector<void*> coarse_allocs;

    // ---- CG workspace (FP64) and preconditioner vectors
    const double* rin64 = nullptr;  // input of the FP64 preconditioner apply
    double *r = nullptr, *zc = nullptr, *p = nullptr, *q = nullptr, *u = nullptr;
    double *fbuf = nullptr, *ubuf = nullptr;   // staging for host solves
    float *r32 = nullptr, *z32 = nullptr;      // preconditioner-precision copies
    double* z64 = nullptr;
    double* scal = nullptr;        // [S_COUNT]
    double* h_scal = nullptr;      // pinned
    double* red_partials = nullptr;   // [DDG_RED_BLOCKS * 4]
    unsigned* red_counter = nullptr;
    int32_t* errflags = nullptr;
    int nrep_local = 0;            // distinct stored local inverses (dedup_local)
    std::vector<double> history;
    // CG coefficients of the longest restart segment of the last solve, and
    // of the segment in progress
    std::vector<double> cg_alpha, cg_beta, seg_alpha, seg_beta;

    MultiWork mw;
    TcData tc;
    BandLocal bl;
    NdCoarse nd;

    // ---- graph-driven PCG (whole solve in one graph launch, one per precision)
    CgCtl* ctl = nullptr;          // device
    CgCtl* h_ctl = nullptr;        // pinned host copy
    double *d_hist = nullptr, *d_alpha = nullptr, *d_beta = nullptr;   // [maxit + 1] each
    cudaGraphExec_t solve_exec[3] = {nullptr, nullptr, nullptr};
    // whole batched solves per precision and column count (m <= DDG_MCHUNK)
    struct BatchGraph {
        int m;
        cudaGraphExec_t exec;
        int64_t pre[DDG_K_COUNT], body[DDG_K_COUNT];   // launches once / per iteration
    };
    std::vector<BatchGraph> batch_exec[3];
    int batch_gen = 0;                 // MultiWork::gen the batched graphs were captured with
    int64_t solve_pre_launches[3][DDG_K_COUNT] = {};    // launched once per solve
    int64_t solve_body_launches[3][DDG_K_COUNT] = {};   // launched once per iteration
    bool solve_graph_failed = false;   // conditional graphs unavailable: host-driven loop
    std::string solve_graph_error;
    int last_solve_graph = 0;          // 1 when the last solve ran as one graph launch
    int version = 0;                   // bumped when a change invalidates captured graphs

    // ---- CUDA graphs of the preconditioner apply inside PCG (one per precision)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;   // body of a conditional node, captured beside cap_stream
    cudaGraphExec_t apply_exec[3] = {nullptr, nullptr, nullptr};
    int64_t apply_launches[3][DDG_K_COUNT] = {};
    bool use_graphs = true;

    // ---- tracing (ddg_profile)
    int prof_mask = 0;
    int64_t prof_launches[DDG_K_COUNT] = {0};
    int64_t prof_timed[DDG_K_COUNT] = {0};
    double prof_ms[DDG_K_COUNT] = {0};
    double prof_bytes[DDG_K_COUNT] = {0};
    std::vector<cudaEvent_t> ev_pool;          // created lazily, reused
    std::vector<int> ev_class;                 // class of each recorded pair
    std::vector<double> ev_bytes;
    size_t ev_used = 0;                        // pairs recorded since the last flush
    std::vector<double> colour_bytes[3];       // per precision: local-solve bytes per colour
};

// Scope of one or more kernel launches of class `cls`: counts the launches
// and, when that class is timed, brackets them with a CUDA event pair.
struct ProfScope {
    ddg_handle h;
    int cls, pair;
    ProfScope(ddg_handle hh, int c, int nlaunch, double bytes);
    ~ProfScope();
};

// ---------------------------------------------------------------- kernels
// (declared here, defined in the k_*.cu files; every launcher enqueues on
// the handle's stream and throws DdgError on a launch failure)
namespace ddg {

// k_local.cu
// setup of the subdomains q0..q1-1, or of qlist[q0..q1-1] when qlist (device) is set
void local_extract_factor_invert(ddg_handle h, int q0, int q1, const int32_t* qlist, double* ws,
                                 double* invdiag);
void local_pack(ddg_handle h, int q0, int q1, const int32_t* qlist, const double* ws);
void local_configure(ddg_handle h);
void local_residual(ddg_handle h, int colour, bool z_zero, int prec);
void local_solve_colour(ddg_handle h, int colour, int prec);

// k_band.cu (banded local factors)
void band_local_assemble(ddg_handle h, const int32_t* qlist, int nb, const int64_t* boff, const int32_t* nts,
                         double* band);
void band_local_pack(ddg_handle h, const int32_t* qlist, int nb, int nKmax, const int64_t* boff,
                     const int64_t* woff, const double* band, const double* W);
size_t band_solve_smem(const BandLocal& L, int prec, int stages);
void band_local_configure(ddg_handle h);
void band_local_solve_colour(ddg_handle h, int c, int prec);

// k_coarse.cu
void band_factor_batched(ddg_handle h, double* band, int Wt, int nb, int NTmax, const int64_t* boff,
                         const int32_t* nts, double* dinv, const int64_t* doff, double* W,
                         const int64_t* woff, int* err);
void front_factor_batched(ddg_handle h, double* fronts, int nb, int NTmax, int NSmax, const int64_t* foff,
                          const int32_t* nts, const int32_t* nss, double* dinv, const int64_t* doff, double* W,
                          const int64_t* woff, int* err);
void coarse_qr(ddg_handle h, int32_t* d_rank, const double* dF, int k);
void coarse_assemble_band(ddg_handle h, const std::vector<int>& blk_I, const std::vector<int>& blk_J);
// the kmax x kmax blocks A0[(I,.),(J,.)] of the listed pairs, copied to the host
void coarse_assemble_blocks(ddg_handle h, const std::vector<int>& blk_I, const std::vector<int>& blk_J,
                            std::vector<double>& blocks);
void coarse_band_cholesky(ddg_handle h);
// F0 = R0 F (device, column-major [n0][k]) from F (device, column-major [n][k])
void coarse_generators(ddg_handle h, const double* dF, int k, double* dF0);
void coarse_build_apply(ddg_handle h);
// the blocks of the listed pairs on the device (caller releases)
double* coarse_assemble_blocks_device(ddg_handle h, const std::vector<int>& blk_I, const std::vector<int>& blk_J);
// k_nd.cu: nested-dissection coarse factor and its solve
void nd_coarse_setup(ddg_handle h, const std::vector<int>& bI, const std::vector<int>& bJ, const double* blocks);
void nd_coarse_solve(ddg_handle h, int prec);
int nd_solve_multi_launches(ddg_handle h);
void nd_coarse_solve_multi(ddg_handle h, int m, const float* c, float* y, float* x, float* w, float* xp, float* P);
int nd_solve_launches(ddg_handle h);
void coarse_restrict(ddg_handle h, int prec, bool residual);
void coarse_solve(ddg_handle h, int prec);
void coarse_prolong(ddg_handle h, int prec);

// k_cg.cu
// gate / firstp: device flags read by the kernels themselves (graph-driven
// solves decide them on the device); nullptr = always run / use `first`
void spmv64(ddg_handle h, const double* x, double* y, bool dot_with_x, int slot);
void dot64(ddg_handle h, const double* a, const double* b, int slot, const int* gate = nullptr);
void copy_gated(ddg_handle h, const double* src, double* dst, const int* gate);
void cg_update_ur(ddg_handle h);
void cg_dots_after_precond(ddg_handle h, int prec, bool first, int pr, const int* firstp = nullptr);
void cg_update_p(ddg_handle h, int prec, bool first, const int* firstp = nullptr);
void convert_to_float(ddg_handle h, const double* src, float* dst);
void convert_to_double(ddg_handle h, const float* src, double* dst);
void residual64(ddg_handle h, const double* f, const double* u, double* r, const int* gate = nullptr);
void grad_coeff_var7(ddg_handle h, const double* lambda, const double* u, double* dk);
void grad_coeff_q1(ddg_handle h, const double* lambda, const double* u, double* dk);
void set_scalar(ddg_handle h, int slot, double v);
void strided_gather(ddg_handle h, const double* src, int m, int j, double* dst);
void strided_scatter(ddg_handle h, const double* src, int m, int j, double* dst);
void cast_q32(ddg_handle h);

// k_multi.cu (batched PCG on n x m blocks, m <= DDG_MCHUNK)
void multi_ensure(ddg_handle h, int m);
void multi_apply(ddg_handle h, int m);
void multi_spmv_pq(ddg_handle h, int m);
void multi_update_ur(ddg_handle h, int m, double* U);
void multi_dots(ddg_handle h, int m, int pr);
void multi_update_p(ddg_handle h, int m);
void multi_resnorm(ddg_handle h, int m, const double* a, const double* b, double* out, int slot);
void multi_replace_cols(ddg_handle h, int m, const double* src, double* dst, const int* replace);
void copy_cols(ddg_handle h, const double* src, int ms, int j0, double* dst, int md, int k0, int cnt);
// graph-driven batched PCG: gated variants and control kernels
void multi_resnorm_gated(ddg_handle h, int m, const double* a, const double* b, double* out, int slot,
                         const int* gate);
void multi_replace_cols_gated(ddg_handle h, int m, const double* src, double* dst, const int* replace,
                              const int* gate);
void multi_to_float(ddg_handle h, int m, const int* gate);
void mloop_init(ddg_handle h, int m, cudaGraphConditionalHandle cond);
void mloop_decide_recurrence(ddg_handle h, int m);
void mloop_decide_true(ddg_handle h, int m, cudaGraphConditionalHandle cond);
void mloop_final_prep(ddg_handle h, int m);
void mloop_final(ddg_handle h, int m);

// k_cg.cu: control kernels of the graph-driven PCG
void loop_init(ddg_handle h, cudaGraphConditionalHandle cond);
void loop_decide_recurrence(ddg_handle h);
void loop_decide_true(ddg_handle h, cudaGraphConditionalHandle cond);
void loop_final(ddg_handle h);

// k_tc.cu (tcgen05 local solves of the batched path)
int tc_n_for(int m);
void tc_pack(ddg_handle h, int q0, int q1, const int32_t* qlist, const double* ws);
void tc_residual(ddg_handle h, int colour, bool z_zero, int m);
void tc_local_solve(ddg_handle h, int colour, int m);

// api.cu: autotuner of the tensor-core ring depth for m columns
void autotune_tc(ddg_handle h, int m);

// api.cu: error message of a handle-less call, read by ddg_last_error(NULL)
void set_handleless_error(const char* msg);

}  // namespace ddg

template <typename... KArgs, typename... Args>
static inline void launch_pdl(ddg_handle h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = h->use_pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DDG_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}
