"""Plain CPU FP64 oracle of the DDG two-level Schwarz preconditioned CG.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this module: it is used by ``tests/``, by ``__graft_entry__.smoke()``
to check one GPU result, and by ``bench.py``'s timed CPU baseline.  It shares
no code with the CUDA library; both take their inputs from ``ddg_inputs``.

Every function restates one step of Edwards & Bridson, "The Discretely-
Discontinuous Galerkin Coarse Grid for Domain Decomposition", in the paper's
order and notation, in plain numpy / scipy (library primitives: sparse
products, QR, Cholesky, triangular solves).  Nothing is blocked, fused or
reordered beyond what the paper states.

Readings where the paper is silent (each one is also listed in the design
notes):

* Overlap (Sec. 6): ``mode="graph"`` grows each partition by all nodes within
  graph distance Delta in the graph of A (the paper's definition);
  ``mode="box"`` grows by L-infinity grid distance Delta (graph distance in
  the 9-/27-point neighbour graph), which is what "8^3 boxes with overlap 1
  -> 10^3-dof blocks" means.
* Subdomain order (Sec. 6 gives none): subdomains are coloured greedily in
  id order so that no two subdomains of one colour interact (the one-step
  neighbourhood of one overlapping subdomain misses the other).  The
  pre-smoother runs colour 0, 1, ..., C-1 (ids ascending inside a colour),
  the post-smoother the exact reverse.  Inside a colour the result does not
  depend on the order, in exact or floating-point arithmetic.
* Orthogonalisation and rank drop (Sec. 4, Fig. 1): column-pivoted
  Householder QR of F restricted to each subdomain; column j is kept while
  |R_jj| > 1e-10 |R_00|.  Coarse dofs are numbered subdomain-major,
  generator-minor (Fig. 1: column partition(i)*k + j), surviving columns
  compacted.
* Stopping (Sec. 7): u0 = 0, stop when the recurrence residual satisfies
  ||r_k||_2 <= tol ||f||_2; the true residual is reported beside it; at most
  1000 iterations.
* beta: Fletcher-Reeves (textbook CG) by default; Polak-Ribiere
  (flexible) on request.
* Three-level V-cycle (Sec. 6): the exact coarse solve A0^{-1} is replaced
  by one application of the two-level method to A0 with the coarsened
  generators F0 = R0 F.  The coarse-level subdomains are given as groups of
  fine subdomains (a coarse dof belongs to the group of its subdomain; groups
  without coarse dofs are dropped and the ids compacted); their overlap is
  the same Delta, grown in the graph of A0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

RANK_TOL = 1e-10


# --------------------------------------------------------------------------
# Sec. 6: overlapping subdomains
# --------------------------------------------------------------------------
def _pattern(M):
    P = sp.csr_matrix(M, copy=True)
    P.data = np.ones_like(P.data)
    return P


def neighbour_graph_box(shape, reach=1):
    """Adjacency (with self loops) of the L-infinity neighbour graph of a grid."""
    shape = tuple(shape)
    n = int(np.prod(shape))
    idx = np.arange(n)
    coord = []
    stride = 1
    strides = []
    for s in shape:
        coord.append((idx // stride) % s)
        strides.append(stride)
        stride *= s
    rows, cols = [], []
    offs = np.array(np.meshgrid(*[np.arange(-reach, reach + 1)] * len(shape), indexing="ij"))
    offs = offs.reshape(len(shape), -1).T
    for off in offs:
        ok = np.ones(n, dtype=bool)
        shift = 0
        for d, o in enumerate(off):
            c = coord[d] + o
            ok &= (c >= 0) & (c < shape[d])
            shift += int(o) * strides[d]
        r = idx[ok]
        rows.append(r)
        cols.append(r + shift)
    r = np.concatenate(rows)
    return sp.csr_matrix((np.ones(r.size), (r, np.concatenate(cols))), shape=(n, n))


def grow_overlap(A, part, delta, mode="graph", shape=None, dpn=1):
    """Overlapping subdomains: Omega~_i = nodes within distance Delta of Omega_i.

    Sec. 6: "expanding the partition to include nodes within graph distance
    Delta in the graph defined by A".  In box mode the distance is measured
    between grid nodes, and all ``dpn`` interleaved dofs of a node move
    together.  Returns a list of sorted int64 index arrays, one per subdomain.
    """
    n = A.shape[0]
    nsub = int(part.max()) + 1
    S = sp.csr_matrix((np.ones(n), (np.arange(n), part)), shape=(n, nsub))
    if mode == "graph":
        G = _pattern(A) + sp.identity(n, format="csr")
    elif mode == "box":
        G = sp.kron(neighbour_graph_box(shape, 1), np.ones((dpn, dpn)), format="csr")
    else:
        raise ValueError(mode)
    G = _pattern(G)
    for _ in range(delta):
        S = _pattern(G @ S)
    S = S.tocsc()
    S.sort_indices()
    return [S.indices[S.indptr[i]:S.indptr[i + 1]].astype(np.int64) for i in range(nsub)]


def colour_subdomains(A, overlapping):
    """Greedy colouring in subdomain-id order (the order reading above).

    Subdomains i and j conflict when Omega~_j meets the one-step
    neighbourhood of Omega~_i in the graph of A (or vice versa); each
    subdomain takes the smallest colour no earlier conflicting subdomain has.
    """
    n = A.shape[0]
    nsub = len(overlapping)
    rows = np.concatenate(overlapping)
    cols = np.concatenate([np.full(len(o), i) for i, o in enumerate(overlapping)])
    S = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(n, nsub))
    NS = _pattern(_pattern(A) @ S + S)
    C = (NS.T @ S).tocsr()
    C = _pattern(C + C.T)
    colour = np.full(nsub, -1, dtype=np.int64)
    for i in range(nsub):
        nb = C.indices[C.indptr[i]:C.indptr[i + 1]]
        used = {int(colour[j]) for j in nb if j != i and colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def sweep_order(colour):
    """Pre-smoother order: colour-major, ids ascending inside a colour."""
    return [int(i) for c in range(int(colour.max()) + 1) for i in np.flatnonzero(colour == c)]


# --------------------------------------------------------------------------
# Sec. 4: the DDG coarse space
# --------------------------------------------------------------------------
def coarse_basis(F, part, rank_tol=RANK_TOL):
    """R0 from the generators (Sec. 4 and Fig. 1).

    phi_i = R_i^T R_i F: column j of F restricted to subdomain i is one
    coarse basis vector; each subdomain's block is orthonormalised on its
    own (the subdomains do not overlap), and rank-deficient columns are
    discarded.  Returns (R0 as sparse n0 x n, coarse offsets[nsub+1]).
    """
    n, k = F.shape
    nsub = int(part.max()) + 1
    rows, cols, vals = [], [], []
    offs = [0]
    for i in range(nsub):
        dofs = np.flatnonzero(part == i)
        Fi = F[dofs, :]
        if dofs.size == 0:
            offs.append(offs[-1])
            continue
        Q, R, _ = sla.qr(Fi, mode="economic", pivoting=True)
        d = np.abs(np.diag(R))
        rank = 0
        if d.size and d[0] > 0:
            rank = int(np.sum(d > rank_tol * d[0]))
        for j in range(rank):
            rows.append(np.full(dofs.size, offs[-1] + j))
            cols.append(dofs)
            vals.append(Q[:, j])
        offs.append(offs[-1] + rank)
    n0 = offs[-1]
    if n0 == 0:
        return sp.csr_matrix((0, n)), np.array(offs)
    R0 = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n0, n))
    return R0, np.array(offs)


def galerkin_coarse(A, R0):
    """A0 = R0 A R0^T (Sec. 4, Galerkin projection)."""
    return (R0 @ A @ R0.T).tocsr()


class CoarseSolver:
    """Exact solve with A0 through its Cholesky factor (dense or banded)."""

    def __init__(self, A0, dense_limit=6000):
        self.n0 = A0.shape[0]
        if self.n0 == 0:
            self.kind = "empty"
        elif self.n0 <= dense_limit:
            self.kind = "dense"
            self.cf = sla.cho_factor(A0.toarray(), lower=True)
        else:
            self.kind = "banded"
            C = A0.tocoo()
            b = int(np.max(C.row - C.col))
            ab = np.zeros((b + 1, self.n0))
            low = C.row >= C.col
            ab[C.row[low] - C.col[low], C.col[low]] = C.data[low]
            self.cb = sla.cholesky_banded(ab, lower=True)

    def solve(self, c):
        if self.kind == "empty":
            return c.copy()
        if self.kind == "dense":
            return sla.cho_solve(self.cf, c)
        return sla.cho_solve_banded((self.cb, True), c)


# --------------------------------------------------------------------------
# Sec. 6: two-level symmetric multiplicative Schwarz
# --------------------------------------------------------------------------
class DDGOracle:
    """Setup and application of the DDG two-level Schwarz preconditioner."""

    def __init__(self, A, part, F, overlap, mode="graph", shape=None, rank_tol=RANK_TOL,
                 coarse=True, dpn=1, coarse_groups=None):
        self.A = sp.csr_matrix(A, dtype=np.float64)
        self.n = self.A.shape[0]
        self.part = np.asarray(part, dtype=np.int64)
        self.nsub = int(self.part.max()) + 1
        # Sec. 6: overlapping subdomains and the processing order
        self.omega = grow_overlap(self.A, self.part, overlap, mode, shape, dpn)
        self.colour = colour_subdomains(self.A, self.omega)
        self.order = sweep_order(self.colour)
        # Sec. 6: local matrices A_i = R~_i A R~_i^T, solved exactly (Cholesky)
        self.rows = []
        self.local = []
        for idx in self.omega:
            Ai_rows = self.A[idx, :]
            self.rows.append(Ai_rows)
            Ai = Ai_rows[:, idx].toarray()
            self.local.append(sla.cho_factor(Ai, lower=True))
        # Sec. 4: coarse space and Galerkin coarse matrix
        self.use_coarse = coarse
        if coarse:
            self.R0, self.coarse_offsets = coarse_basis(np.asarray(F, dtype=np.float64),
                                                         self.part, rank_tol)
            self.A0 = galerkin_coarse(self.A, self.R0)
            self.inner = None
            if coarse_groups is not None and self.A0.shape[0] > 0:
                # Sec. 6: the three-level method applies the two-level
                # method to A0, with generators F0 = R0 F
                sub_of_dof = np.repeat(np.arange(self.nsub), np.diff(self.coarse_offsets))
                group = np.asarray(coarse_groups, dtype=np.int64)[sub_of_dof]
                _, part0 = np.unique(group, return_inverse=True)
                F0 = self.R0 @ np.asarray(F, dtype=np.float64)
                self.inner = DDGOracle(self.A0, part0, F0, overlap, "graph", rank_tol=rank_tol)
            else:
                self.coarse = CoarseSolver(self.A0)

    # one subdomain step of Sec. 6: u <- u + R~_i^T A_i^{-1} R~_i (f - A u)
    def _subdomain_step(self, i, r, z):
        idx = self.omega[i]
        res = r[idx] - self.rows[i] @ z
        z[idx] += sla.cho_solve(self.local[i], res)

    def coarse_correction(self, r):
        """R0^T A0^{-1} R0 r (Sec. 4: coarse approximation R0^T u0, A0 u0 = R0 f).

        In the three-level method A0^{-1} is replaced by one application of
        the two-level preconditioner of A0 (Sec. 6).
        """
        c = self.R0 @ r
        x = self.inner.apply(c) if self.inner is not None else self.coarse.solve(c)
        return self.R0.T @ x

    def apply(self, r):
        """z = M^{-1} r: one two-level symmetric multiplicative step from z = 0.

        Pre-smoother: one pass over the subdomains; coarse correction of the
        current residual; post-smoother: the same pass in reverse order
        (Sec. 6), which makes M symmetric.
        """
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        for i in self.order:
            self._subdomain_step(i, r, z)
        if self.use_coarse:
            w = r - self.A @ z
            z += self.coarse_correction(w)
        for i in reversed(self.order):
            self._subdomain_step(i, r, z)
        return z

    # ---- dense helpers for tiny problems (pins) ----
    def dense_preconditioner(self):
        """M^{-1} as a dense matrix, one column per unit vector."""
        I = np.eye(self.n)
        return np.stack([self.apply(I[:, j]) for j in range(self.n)], axis=1)

    def dense_projections(self):
        """P_i = R~_i^T A_i^{-1} R~_i A (dense), and P_0 = R0^T A0^{-1} R0 A."""
        Ad = self.A.toarray()
        P = []
        for i in range(self.nsub):
            idx = self.omega[i]
            Ai = Ad[np.ix_(idx, idx)]
            Pi = np.zeros((self.n, self.n))
            Pi[idx, :] = np.linalg.solve(Ai, Ad[idx, :])
            P.append(Pi)
        P0 = None
        if self.use_coarse:
            R0 = self.R0.toarray()
            A0 = R0 @ Ad @ R0.T
            P0 = R0.T @ np.linalg.solve(A0, R0 @ Ad)
        return P, P0


# --------------------------------------------------------------------------
# Sec. 7: preconditioned conjugate gradient and its reporting
# --------------------------------------------------------------------------
class PCGResult:
    def __init__(self, u, iters, history, alphas, betas, converged, true_relres):
        self.u = u
        self.iters = iters
        self.history = history          # ||r_k|| / ||f|| for k = 0..iters
        self.alphas = alphas
        self.betas = betas
        self.converged = converged
        self.true_relres = true_relres


def pcg(A, f, apply_m, tol=1e-8, maxit=1000, beta="FR"):
    """Preconditioned CG from u0 = 0 (Sec. 7 protocol).

    Stops when ||r_k||_2 <= tol ||f||_2 for the recurrence residual; caps
    at ``maxit`` iterations (the paper stops at 1000).  ``beta`` is
    "FR" (r_{k+1}^T z_{k+1} / r_k^T z_k) or "PR"
    ((r_{k+1} - r_k)^T z_{k+1} / r_k^T z_k).
    """
    f = np.asarray(f, dtype=np.float64)
    u = np.zeros_like(f)
    r = f.copy()
    fn = np.linalg.norm(f)
    hist = [1.0 if fn > 0 else 0.0]
    if fn == 0:
        return PCGResult(u, 0, hist, [], [], True, 0.0)
    z = apply_m(r)
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    converged = False
    k = 0
    while k < maxit:
        q = A @ p
        pq = p @ q
        alpha = rz / pq
        u = u + alpha * p
        r_old = r
        r = r - alpha * q
        k += 1
        alphas.append(alpha)
        hist.append(np.linalg.norm(r) / fn)
        if hist[-1] <= tol:
            converged = True
            break
        z = apply_m(r)
        rz_new = r @ z
        if beta == "FR":
            b = rz_new / rz
        else:
            b = (rz_new - r_old @ z) / rz
        betas.append(b)
        p = z + b * p
        rz = rz_new
    true_rel = np.linalg.norm(f - A @ u) / fn
    return PCGResult(u, k, np.array(hist), np.array(alphas), np.array(betas), converged, true_rel)


def fractional_iterations(history, tol):
    """Sec. 7: where the straight line through log residuals meets tol.

    Linear interpolation of log(residual) between the last iterate above
    the tolerance and the first one at or below it.
    """
    h = np.asarray(history, dtype=np.float64)
    below = np.flatnonzero(h <= tol)
    if below.size == 0:
        return float("nan")
    k = int(below[0])
    if k == 0:
        return 0.0
    a, b = np.log(h[k - 1]), np.log(h[k])
    return (k - 1) + (a - np.log(tol)) / (a - b)


def lanczos_extremes(alphas, betas):
    """Sec. 7: eigenvalue estimates of M^{-1} A from the CG coefficients.

    The Lanczos tridiagonal of CG has diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}
    and off-diagonal sqrt(beta_j)/alpha_j; its extreme eigenvalues estimate
    those of the preconditioned operator.  Returns (lambda_min, lambda_max).
    """
    a = np.asarray(alphas, dtype=np.float64)
    b = np.asarray(betas, dtype=np.float64)
    m = a.size
    if m == 0:
        return float("nan"), float("nan")
    d = 1.0 / a
    d[1:] += b[:m - 1] / a[:m - 1]
    e = np.sqrt(np.abs(b[:m - 1])) / a[:m - 1]
    w = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(w[0]), float(w[-1])


def cg_iteration_bound(kappa, tol):
    """Sec. 7: iterations that CG needs for a tol reduction of the A-norm
    error given the condition number kappa (the Chebyshev bound
    2 ((sqrt k - 1)/(sqrt k + 1))^j <= tol solved for j)."""
    if kappa <= 1.0:
        return 0.0
    sk = np.sqrt(kappa)
    return float(np.log(2.0 / tol) / np.log((sk + 1.0) / (sk - 1.0)))


def solve(A, part, F, f, overlap, mode="graph", shape=None, tol=1e-8, maxit=1000, beta="FR"):
    """Setup plus PCG in one call; returns (PCGResult, DDGOracle)."""
    M = DDGOracle(A, part, F, overlap, mode, shape)
    return pcg(M.A, f, M.apply, tol, maxit, beta), M
