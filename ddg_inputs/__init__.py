"""Seeded synthetic inputs for the DDG two-level Schwarz PCG solver.

This module builds the *problems* the solver is run on: a sparse SPD matrix
``A`` (CSR, FP64), a non-overlapping node partition, the generating vectors
``F`` (monomials in the nodal coordinates) and right-hand sides.  It contains
none of the method's arithmetic (no coarse space, no Schwarz sweep, no CG):
both the CPU oracle and the CUDA library consume what it produces, and
neither shares any other code with the other.

Problem families (structured grids, natural lexicographic order, x fastest):

* 2D Poisson, 5-point FD, homogeneous Dirichlet, integer stencil [4, -1]
  (the paper's scaling is unstated; relative residuals are scale invariant).
* 3D Poisson, 7-point FD, homogeneous Dirichlet, integer stencil [6, -1]
  (paper Sec. 7, problem A uses a 7-point stencil; the boundary conditions
  here are all-Dirichlet).
* 2D biharmonic, 13-point FD, clamped (Dirichlet + Neumann) boundary
  (paper Sec. 7, problem F): interior stencil = square of the 5-point
  Laplacian [20, -8, 2, 1]; u = 0 on the boundary nodes and the Neumann
  condition by the ghost reflection u(-2) = u(0), which adds 1 to the
  diagonal per adjacent boundary edge.
* 3D variable-coefficient diffusion -div(kappa grad u), cell-centred FD,
  harmonic-mean face coefficients, Dirichlet faces at half-cell distance
  (coefficient 2*kappa), operator scaled by h^2.
* 3D linear elasticity, trilinear (Q1) hexahedral finite elements on ne^3
  elements of the unit cube, Lame lambda constant and shear modulus mu per
  element, 2x2x2 Gauss quadrature, the x = 0 face clamped; 3 interleaved
  displacement dofs per node (analogue of the paper's vector problem E).
* Gaussian random field g with squared-exponential covariance
  sigma^2 exp(-r^2 / (2 l^2)), sampled exactly through the separable
  (Kronecker) factorisation, kappa = exp(g).

Generators ``F`` (paper Sec. 4: "a small set of input vectors that span a
low-degree polynomial space", built from nodal coordinates): all monomials
of total degree <= p, ordered by total degree, then by descending exponent
of x, then y (1, x, y, z, x^2, xy, xz, y^2, yz, z^2, ...).  Vector-valued
problems take the monomials once per component.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem", "poisson5_2d", "poisson7_3d", "biharmonic13_2d",
    "varcoef7_3d", "gaussian_random_field", "box_partition", "monomials",
    "fd_node_coords", "cell_centre_coords", "uniform_rhs", "normal_rhs",
    "make_poisson2d", "make_poisson3d", "make_biharmonic2d",
    "make_varcoef3d", "csr_arrays", "monomial_exponents", "q1_reference_stiffness",
    "elasticity_q1_3d", "make_elasticity3d",
]

# stencil kinds understood by the library's matrix-free SpMV (the CSR is
# always supplied; the kind only enables a faster SpMV for the same matrix)
STENCIL_NONE = 0
STENCIL_5PT_2D = 1
STENCIL_7PT_3D = 2
STENCIL_13PT_2D = 3
STENCIL_VAR7_3D = 4
STENCIL_Q1_ELASTIC = 5


@dataclasses.dataclass
class Problem:
    """One SPD system plus everything the DDG preconditioner needs."""
    name: str
    A: sp.csr_matrix            # n x n, FP64, symmetric positive definite
    shape: tuple                # grid shape (nx, ny[, nz]) of nodes/cells
    part: np.ndarray            # int32[n], node -> non-overlapping subdomain
    box: tuple                  # subdomain box size per axis (box partitions)
    F: np.ndarray               # float64[n, k] generating vectors
    f: np.ndarray               # float64[n] or [n, m] right-hand side(s)
    overlap: int                # overlap layers Delta
    overlap_mode: str           # "box" (L-inf growth) or "graph" (graph of A)
    p: int                      # polynomial degree of F
    stencil_kind: int = STENCIL_NONE
    face_coef: Optional[np.ndarray] = None   # VAR7: float64[3, nz, ny, nx+1..]
    kappa: Optional[np.ndarray] = None       # VAR7: cell coefficients; Q1: mu per element
    dofs_per_node: int = 1
    target: Optional[np.ndarray] = None      # Q1 workload: u_t of the loss

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def nsub(self) -> int:
        return int(self.part.max()) + 1


# --------------------------------------------------------------------------
# grids and coordinates
# --------------------------------------------------------------------------
def _grid_index(shape):
    """Per-axis integer coordinates of every node, x fastest."""
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    out = []
    stride = 1
    for s in shape:
        out.append((idx // stride) % s)
        stride *= s
    return out


def fd_node_coords(shape):
    """Interior FD nodes of the unit box: x_i = (i + 1) / (N + 1)."""
    ax = _grid_index(shape)
    return np.stack([(a + 1.0) / (s + 1.0) for a, s in zip(ax, shape)], axis=1)


def cell_centre_coords(shape):
    """Cell centres of a uniform grid on the unit box: x_i = (i + 1/2) / N."""
    ax = _grid_index(shape)
    return np.stack([(a + 0.5) / s for a, s in zip(ax, shape)], axis=1)


def _stencil_csr(shape, offsets, weights, diag_extra=None):
    """Assemble a constant stencil with homogeneous Dirichlet elimination.

    ``offsets`` are integer tuples per axis; entries whose neighbour lies
    outside the grid are dropped (the boundary value is zero).
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    ax = _grid_index(shape)
    strides = np.cumprod((1,) + shape[:-1])
    rows, cols, vals = [], [], []
    idx = np.arange(n, dtype=np.int64)
    for off, w in zip(offsets, weights):
        ok = np.ones(n, dtype=bool)
        shift = 0
        for d, o in enumerate(off):
            if o:
                c = ax[d] + o
                ok &= (c >= 0) & (c < shape[d])
                shift += o * int(strides[d])
        r = idx[ok]
        rows.append(r)
        cols.append(r + shift)
        vals.append(np.full(r.size, float(w)))
    if diag_extra is not None:
        rows.append(idx)
        cols.append(idx)
        vals.append(diag_extra.astype(np.float64))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    A.eliminate_zeros()
    return A


def poisson5_2d(nx, ny=None):
    """5-point Laplacian [4, -1] on an nx x ny interior grid, Dirichlet."""
    ny = nx if ny is None else ny
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    return _stencil_csr((nx, ny), offs, [4, -1, -1, -1, -1])


def poisson7_3d(nx, ny=None, nz=None):
    """7-point Laplacian [6, -1] on an nx x ny x nz interior grid, Dirichlet."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return _stencil_csr((nx, ny, nz), offs, [6, -1, -1, -1, -1, -1, -1])


def biharmonic13_2d(nx, ny=None):
    """13-point h^4 * biharmonic, clamped boundary (Sec. 7, problem F).

    Interior weights: centre 20, face neighbours -8, diagonal neighbours 2,
    distance-two axial neighbours 1.  u = 0 on the boundary ring; the
    Neumann condition reflects the ghost two steps out onto the first
    interior node (u(-2) = u(0)), adding 1 to the diagonal per adjacent edge.
    """
    ny = nx if ny is None else ny
    offs = [(0, 0),
            (-1, 0), (1, 0), (0, -1), (0, 1),
            (-1, -1), (1, -1), (-1, 1), (1, 1),
            (-2, 0), (2, 0), (0, -2), (0, 2)]
    w = [20, -8, -8, -8, -8, 2, 2, 2, 2, 1, 1, 1, 1]
    i, j = _grid_index((nx, ny))
    extra = ((i == 0).astype(int) + (i == nx - 1) + (j == 0) + (j == ny - 1))
    return _stencil_csr((nx, ny), offs, w, diag_extra=extra)


def varcoef7_3d(kappa):
    """Cell-centred FD of -div(kappa grad u) on the unit cube, scaled by h^2.

    ``kappa`` has shape (nz, ny, nx) (x fastest when raveled).  Interior
    face coefficient: harmonic mean 2 ka kb / (ka + kb); Dirichlet boundary
    face at half-cell distance: 2 kappa_cell.  Returns (A, face) where
    ``face`` = (cx[nz,ny,nx+1], cy[nz,ny+1,nx], cz[nz+1,ny,nx]) are the face
    coefficients including boundary faces.
    """
    kap = np.asarray(kappa, dtype=np.float64)
    nz, ny, nx = kap.shape
    n = kap.size

    def faces(axis):
        k = np.moveaxis(kap, axis, 0)
        m = k.shape[0]
        c = np.empty((m + 1,) + k.shape[1:])
        c[1:-1] = 2.0 * k[:-1] * k[1:] / (k[:-1] + k[1:])
        c[0] = 2.0 * k[0]
        c[-1] = 2.0 * k[-1]
        return np.moveaxis(c, 0, axis)

    cz, cy, cx = faces(0), faces(1), faces(2)
    idx = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    diag = (cx[:, :, :-1] + cx[:, :, 1:] + cy[:, :-1, :] + cy[:, 1:, :]
            + cz[:-1, :, :] + cz[1:, :, :])
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [diag.ravel()]
    # interior faces couple the two cells with -c
    for a, b, c in ((idx[:, :, :-1], idx[:, :, 1:], cx[:, :, 1:-1]),
                    (idx[:, :-1, :], idx[:, 1:, :], cy[:, 1:-1, :]),
                    (idx[:-1, :, :], idx[1:, :, :], cz[1:-1, :, :])):
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
        vals += [-c.ravel(), -c.ravel()]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A, (cx, cy, cz)


def q1_reference_stiffness():
    """Element matrices of trilinear (Q1) linear elasticity on the unit cube.

    Local dof 3 a + i = component i of node a = (a & 1, (a >> 1) & 1, a >> 2).
    With N_a the trilinear shape functions and 2x2x2 Gauss quadrature (exact
    here): K_lam[ai, bj] = int d_i N_a d_j N_b and
    K_mu[ai, bj] = int (delta_ij grad N_a . grad N_b + d_j N_a d_i N_b), so
    that the element stiffness of lam, mu on a cube of side h is
    h (lam K_lam + mu K_mu) (bilinear form int lam div u div v + 2 mu eps:eps).
    """
    g = 0.5 + np.array([-0.5, 0.5]) / np.sqrt(3.0)
    Kl = np.zeros((24, 24))
    Km = np.zeros((24, 24))
    for x in g:
        for y in g:
            for z in g:
                xi = (x, y, z)
                grad = np.zeros((8, 3))
                for a in range(8):
                    bits = (a & 1, (a >> 1) & 1, (a >> 2) & 1)
                    f = [xi[d] if bits[d] else 1.0 - xi[d] for d in range(3)]
                    df = [1.0 if bits[d] else -1.0 for d in range(3)]
                    grad[a] = [df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]]
                w = 1.0 / 8.0
                for a in range(8):
                    for b in range(8):
                        gg = grad[a] @ grad[b]
                        for i in range(3):
                            for j in range(3):
                                Kl[3 * a + i, 3 * b + j] += w * grad[a, i] * grad[b, j]
                                Km[3 * a + i, 3 * b + j] += w * ((i == j) * gg + grad[a, j] * grad[b, i])
    return Kl, Km


def elasticity_q1_3d(mu, lam=1.0):
    """Q1 hexahedral linear elasticity on ne^3 elements of the unit cube.

    ``mu`` has shape (ne, ne, ne) (x fastest when raveled), one shear modulus
    per element; ``lam`` is constant.  The nodes of the x = 0 face are clamped
    (their dofs eliminated); the remaining nodes (i = 1..ne, j, k = 0..ne) are
    numbered x fastest with 3 interleaved displacement dofs each.  Returns
    (A, node_shape) with node_shape = (ne, ne + 1, ne + 1).
    """
    mu = np.asarray(mu, dtype=np.float64)
    ne = mu.shape[0]
    h = 1.0 / ne
    Kl, Km = q1_reference_stiffness()
    Kl = Kl * h
    Km = Km * h
    E = np.arange(ne ** 3, dtype=np.int64)
    ei, ej, ek = E % ne, (E // ne) % ne, E // (ne * ne)
    dofs = np.empty((ne ** 3, 24), dtype=np.int64)
    for a in range(8):
        I, J, K = ei + (a & 1), ej + ((a >> 1) & 1), ek + (a >> 2)
        base = np.where(I >= 1, 3 * ((I - 1) + ne * (J + (ne + 1) * K)), -1)
        for i in range(3):
            dofs[:, 3 * a + i] = np.where(base >= 0, base + i, -1)
    n = 3 * ne * (ne + 1) ** 2
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    vals = (lam * Kl[None, :, :] + mu.ravel()[:, None, None] * Km[None, :, :]).ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A, (ne, ne + 1, ne + 1)


def gaussian_random_field(shape, length, sigma, seed, coords="cell"):
    """Exact sample of a squared-exponential Gaussian random field.

    Covariance sigma^2 exp(-|x - y|^2 / (2 length^2)) on the grid points of
    ``shape`` = (nx, ny, nz) (cell centres by default).  The kernel is a
    product over axes, so g = sigma (S_z (x) S_y (x) S_x) xi with S the
    symmetric square root of each 1D correlation matrix (eigenvalues below
    zero from rounding are clipped to zero) and xi ~ N(0, 1) i.i.d. from
    numpy's PCG64 generator seeded with ``seed``.  Returns an array of shape
    (nz, ny, nx).
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    roots = []
    for m in (nx, ny, nz):
        x = (np.arange(m) + 0.5) / m if coords == "cell" else (np.arange(m) + 1.0) / (m + 1.0)
        K = np.exp(-(x[:, None] - x[None, :]) ** 2 / (2.0 * length ** 2))
        w, V = np.linalg.eigh(K)
        w = np.clip(w, 0.0, None)
        roots.append((V * np.sqrt(w)) @ V.T)
    xi = rng.standard_normal((nz, ny, nx))
    Sx, Sy, Sz = roots
    g = np.einsum("ai,kji->kja", Sx, xi)
    g = np.einsum("bj,kja->kba", Sy, g)
    g = np.einsum("ck,kba->cba", Sz, g)
    return sigma * g


# --------------------------------------------------------------------------
# partitions, generators, right-hand sides
# --------------------------------------------------------------------------
def box_partition(shape, box):
    """Node -> subdomain id for a regular box partition (x-fastest boxes).

    A trailing partial box along an axis (shape not divisible by box) is a
    box of its own.
    """
    ax = _grid_index(shape)
    nb = [(s + b - 1) // b for s, b in zip(shape, box)]
    sid = np.zeros(ax[0].shape, dtype=np.int64)
    stride = 1
    for a, b, m in zip(ax, box, nb):
        sid += (a // b) * stride
        stride *= m
    return sid.astype(np.int32)


def subdomain_groups(shape, box, group):
    """Subdomain -> coarse-level subdomain for the three-level method.

    The subdomains of ``box_partition(shape, box)`` form a grid of boxes (x
    fastest); the coarse-level subdomains are boxes of ``group`` subdomains
    per axis of that grid, numbered the same way.
    """
    nb = tuple((s + b - 1) // b for s, b in zip(shape, box))
    g = group if isinstance(group, (tuple, list)) else (group,) * len(nb)
    return box_partition(nb, tuple(g))


def monomial_exponents(d, p):
    """Exponent tuples of all monomials of total degree <= p in d variables,
    ordered by total degree, then descending exponent lexicographically."""
    out = []
    for deg in range(p + 1):
        cur = []

        def rec(prefix, left, dims):
            if dims == 1:
                cur.append(tuple(prefix + [left]))
                return
            for e in range(left, -1, -1):
                rec(prefix + [e], left - e, dims - 1)
        rec([], deg, d)
        out += cur
    return out


def monomials(coords, p, components=1):
    """Generating vectors: monomials of degree <= p in the nodal coordinates.

    For ``components`` > 1 (vector problems, dofs interleaved per node) the
    scalar monomials are placed once per component.
    """
    coords = np.asarray(coords, dtype=np.float64)
    nn, d = coords.shape
    ex = monomial_exponents(d, p)
    S = np.empty((nn, len(ex)))
    for c, e in enumerate(ex):
        v = np.ones(nn)
        for a in range(d):
            if e[a]:
                v = v * coords[:, a] ** e[a]
        S[:, c] = v
    if components == 1:
        return S
    F = np.zeros((nn * components, len(ex) * components))
    for comp in range(components):
        F[comp::components, comp * len(ex):(comp + 1) * len(ex)] = S
    return F


def local_monomials(coords, part, p):
    """Monomials of degree <= p in coordinates centred and scaled per
    subdomain: column j on the nodes of subdomain i is m_j((x - c_i) / s_i),
    with c_i the centre and s_i the half-width of the subdomain's bounding box
    (per axis; 1 where the box is flat).

    The coarse space uses only each generator's restriction to each
    subdomain (Sec. 4), and on one subdomain these columns span the same
    polynomials as the global monomials, so the coarse space is the same; the
    per-subdomain blocks are far better conditioned at high degree.
    """
    coords = np.asarray(coords, dtype=np.float64)
    part = np.asarray(part, dtype=np.int64)
    nsub = int(part.max()) + 1
    d = coords.shape[1]
    lo = np.full((nsub, d), np.inf)
    hi = np.full((nsub, d), -np.inf)
    np.minimum.at(lo, part, coords)
    np.maximum.at(hi, part, coords)
    centre = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo)
    half[half == 0.0] = 1.0
    return monomials((coords - centre[part]) / half[part], p)


def aggregate_generators(shape, box, agg, p=1):
    """Generators for aggregation on subdomains smaller than the smoothing
    ones (the comparison of Fig. 3): each box x box subdomain is cut into
    aggregates of agg x agg nodes (box % agg == 0), and column
    (slot * nm + j) holds the j-th local monomial of degree <= p on the
    aggregate at position ``slot`` inside every subdomain, zero elsewhere.
    Restricted to a subdomain these columns span the piecewise polynomials
    on its aggregates."""
    if any(b % agg for b in box):
        raise ValueError("aggregates must tile the subdomain boxes")
    ax = _grid_index(shape)
    apart = box_partition(shape, (agg,) * len(shape))
    per = [b // agg for b in box]
    slot = np.zeros(ax[0].shape, dtype=np.int64)
    stride = 1
    for a, b, q in zip(ax, box, per):
        slot += ((a % b) // agg) * stride
        stride *= q
    L = local_monomials(fd_node_coords(shape), apart, p)
    nm = L.shape[1]
    F = np.zeros((L.shape[0], nm * stride))
    for sl in range(stride):
        rows = slot == sl
        F[rows, sl * nm:(sl + 1) * nm] = L[rows]
    return F


def uniform_rhs(n, seed, m=None):
    """f ~ U(-1, 1) i.i.d. (PCG64 seeded)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n if m is None else (n, m))


def normal_rhs(n, seed, m=None):
    """f ~ N(0, 1) i.i.d. (PCG64 seeded)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n if m is None else (n, m))


def csr_arrays(A):
    """(rowptr int64, col int32, val float64) of a scipy CSR matrix."""
    A = A.tocsr()
    return (np.ascontiguousarray(A.indptr, dtype=np.int64),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64))


# --------------------------------------------------------------------------
# ready-made workloads
# --------------------------------------------------------------------------
def make_poisson2d(N=64, box=16, overlap=2, p=2, seed=0, m=None, mode="box"):
    """2D Poisson 5-point on N x N, box partition, U(-1,1) right-hand side."""
    shape = (N, N)
    A = poisson5_2d(N)
    return Problem(name=f"poisson2d_{N}", A=A, shape=shape,
                   part=box_partition(shape, (box, box)), box=(box, box),
                   F=monomials(fd_node_coords(shape), p), f=uniform_rhs(A.shape[0], seed, m),
                   overlap=overlap, overlap_mode=mode, p=p, stencil_kind=STENCIL_5PT_2D)


def make_poisson3d(N=128, box=8, overlap=1, p=2, seed=1, m=None, mode="box"):
    """3D Poisson 7-point on N^3, box partition, U(-1,1) right-hand side."""
    shape = (N, N, N)
    A = poisson7_3d(N)
    return Problem(name=f"poisson3d_{N}", A=A, shape=shape,
                   part=box_partition(shape, (box,) * 3), box=(box,) * 3,
                   F=monomials(fd_node_coords(shape), p), f=uniform_rhs(A.shape[0], seed, m),
                   overlap=overlap, overlap_mode=mode, p=p, stencil_kind=STENCIL_7PT_3D)


def make_biharmonic2d(N=256, box=16, overlap=2, p=3, seed=100, m=None, mode="box", local=False):
    """2D clamped biharmonic 13-point on N x N, box partition; ``local``
    takes the generators centred and scaled per subdomain (same coarse
    space, better conditioned at high p)."""
    shape = (N, N)
    A = biharmonic13_2d(N)
    part = box_partition(shape, (box, box))
    coords = fd_node_coords(shape)
    F = local_monomials(coords, part, p) if local else monomials(coords, p)
    return Problem(name=f"biharmonic2d_{N}", A=A, shape=shape,
                   part=part, box=(box, box),
                   F=F, f=uniform_rhs(A.shape[0], seed, m),
                   overlap=overlap, overlap_mode=mode, p=p, stencil_kind=STENCIL_13PT_2D)


def make_elasticity3d(ne=64, box=8, overlap=1, p=2, lam=1.0, length=0.15, sigma=1.0,
                      field_seed=4, body_seed=5, target_seed=6, mode="box"):
    """Q1 elasticity on ne^3 elements, mu = exp(GRF) per element, clamped x = 0,
    body force ~ N(0, 1) per dof, target displacement u_t ~ N(0, 1); node
    partition by boxes of ``box`` node layers (node index // box, the last
    box absorbing the end layer); generators: monomials of degree <= p in the
    node coordinates, once per displacement component."""
    g = gaussian_random_field((ne, ne, ne), length, sigma, field_seed)
    mu = np.exp(g)
    A, nshape = elasticity_q1_3d(mu, lam)
    nx, ny, nz = nshape
    nn = nx * ny * nz
    node = np.arange(nn)
    I = node % nx + 1
    J = (node // nx) % ny
    K = node // (nx * ny)
    nb = ne // box
    sid = (np.minimum(I // box, nb - 1) + nb * (np.minimum(J // box, nb - 1)
           + nb * np.minimum(K // box, nb - 1)))
    part = np.repeat(sid, 3).astype(np.int32)
    h = 1.0 / ne
    coords = np.stack([I * h, J * h, K * h], axis=1)
    F = monomials(coords, p, components=3)
    n = A.shape[0]
    return Problem(name=f"elasticity3d_{ne}", A=A, shape=nshape, part=part, box=(box,) * 3, F=F,
                   f=normal_rhs(n, body_seed), overlap=overlap, overlap_mode=mode, p=p,
                   stencil_kind=STENCIL_Q1_ELASTIC, kappa=mu, dofs_per_node=3,
                   target=normal_rhs(n, target_seed))


def make_varcoef3d(N=96, box=8, overlap=1, p=2, field_seed=2, rhs_seed=3, m=64,
                   length=0.1, sigma=1.0, mode="box"):
    """3D cell-centred -div(exp(g) grad u) with g a GRF; N(0,1) right-hand sides."""
    shape = (N, N, N)
    g = gaussian_random_field(shape, length, sigma, field_seed)
    kappa = np.exp(g)
    A, face = varcoef7_3d(kappa)
    return Problem(name=f"varcoef3d_{N}", A=A, shape=shape,
                   part=box_partition(shape, (box,) * 3), box=(box,) * 3,
                   F=monomials(cell_centre_coords(shape), p), f=normal_rhs(A.shape[0], rhs_seed, m),
                   overlap=overlap, overlap_mode=mode, p=p, stencil_kind=STENCIL_VAR7_3D,
                   face_coef=face, kappa=kappa)


def two_material_coefficient(coords):
    """Sec. 7 problem C's coefficient on cell centres: D = S + 100 J with the
    smooth S = exp(1 + sin(pi (x + y))) and the material indicator
    J = H(0.25 + cos(pi x) cos(2 pi y)) (H the Heaviside step); returns (D, J).
    On the unit cube the fields do not depend on z."""
    x, y = coords[:, 0], coords[:, 1]
    S = np.exp(1.0 + np.sin(np.pi * (x + y)))
    J = (0.25 + np.cos(np.pi * x) * np.cos(2.0 * np.pi * y) > 0.0).astype(np.float64)
    return S + 100.0 * J, J


def material_aware_generators(F, J):
    """Generators that are piecewise in the materials (Sec. 7, problem C):
    every column of F once times the indicator of each material, [F(1-J), FJ]."""
    J = np.asarray(J, dtype=np.float64)[:, None]
    return np.hstack([F * (1.0 - J), F * J])


def varcoef5_2d(kappa):
    """Cell-centred FD of -div(kappa grad u) on the unit square, scaled by
    h^2 (the 2D analogue of ``varcoef7_3d``): interior faces take the
    harmonic mean of the two cells, Dirichlet boundary faces 2 kappa_cell.
    ``kappa`` has shape (ny, nx), x fastest when raveled."""
    kap = np.asarray(kappa, dtype=np.float64)
    ny, nx = kap.shape
    n = kap.size
    cx = np.empty((ny, nx + 1))
    cx[:, 1:-1] = 2.0 * kap[:, :-1] * kap[:, 1:] / (kap[:, :-1] + kap[:, 1:])
    cx[:, 0], cx[:, -1] = 2.0 * kap[:, 0], 2.0 * kap[:, -1]
    cy = np.empty((ny + 1, nx))
    cy[1:-1] = 2.0 * kap[:-1] * kap[1:] / (kap[:-1] + kap[1:])
    cy[0], cy[-1] = 2.0 * kap[0], 2.0 * kap[-1]
    idx = np.arange(n, dtype=np.int64).reshape(ny, nx)
    diag = cx[:, :-1] + cx[:, 1:] + cy[:-1, :] + cy[1:, :]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
    for a, b, c in ((idx[:, :-1], idx[:, 1:], cx[:, 1:-1]), (idx[:-1, :], idx[1:, :], cy[1:-1, :])):
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
        vals += [-c.ravel(), -c.ravel()]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A


def make_twomaterial2d(N=1024, box=16, overlap=0, p=3, material_aware=False, rhs_seed=8, m=None,
                       mode="graph"):
    """2D cell-centred -div(D grad u) with the two-material coefficient of
    Sec. 7 problem C, D = S + 100 J, on an N x N grid (a structured stand-in
    for the paper's annulus mesh); box partitions that do not follow the
    material boundary; monomials of degree <= p, or their material-aware
    split; N(0,1) right-hand side.  General CSR (no matrix-free stencil)."""
    shape = (N, N)
    coords = cell_centre_coords(shape)
    D, J = two_material_coefficient(coords)
    A = varcoef5_2d(D.reshape(N, N))
    F = monomials(coords, p)
    if material_aware:
        F = material_aware_generators(F, J)
    return Problem(name=f"twomaterial2d_{N}" + ("_aware" if material_aware else ""), A=A, shape=shape,
                   part=box_partition(shape, (box, box)), box=(box, box), F=F,
                   f=normal_rhs(A.shape[0], rhs_seed, m), overlap=overlap, overlap_mode=mode, p=p)


def make_twomaterial3d(N=128, box=8, overlap=1, p=2, material_aware=False, rhs_seed=7, m=None,
                       mode="box"):
    """3D cell-centred -div(D grad u) with the two-material coefficient
    D = S + 100 J of Sec. 7 problem C (extruded in z); box partitions that do
    not follow the material boundary; monomial generators, or their
    material-aware split (twice the columns); N(0,1) right-hand side."""
    shape = (N, N, N)
    coords = cell_centre_coords(shape)
    D, J = two_material_coefficient(coords)
    kappa = D.reshape(N, N, N)
    A, face = varcoef7_3d(kappa)
    F = monomials(coords, p)
    if material_aware:
        F = material_aware_generators(F, J)
    return Problem(name=f"twomaterial3d_{N}" + ("_aware" if material_aware else ""), A=A, shape=shape,
                   part=box_partition(shape, (box,) * 3), box=(box,) * 3, F=F,
                   f=normal_rhs(A.shape[0], rhs_seed, m), overlap=overlap, overlap_mode=mode, p=p,
                   stencil_kind=STENCIL_VAR7_3D, face_coef=face, kappa=kappa)
