"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants the paper states, textbook special cases, brute force on
tiny inputs, or the paper's printed numbers.  No GPU is used here.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ddg_inputs as di
from oracle import ddg_oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle(prob, **kw):
    return orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode,
                         prob.shape, **kw)


# ---------------------------------------------------------------- inputs
def test_poisson5_eigenvalues_closed_form():
    N = 7
    A = di.poisson5_2d(N).toarray()
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    lam = (4 - 2 * np.cos(j[:, None] * np.pi * h) - 2 * np.cos(j[None, :] * np.pi * h)).ravel()
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(lam), atol=1e-12)


def test_poisson7_row_sums_count_boundary_neighbours():
    N = 5
    A = di.poisson7_3d(N)
    i, j, k = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    nb = sum(((a == 0) | (a == N - 1)).astype(int) for a in (i, j, k))
    # Dirichlet elimination drops one -1 per boundary neighbour
    np.testing.assert_array_equal(A @ np.ones(N ** 3), nb.transpose(2, 1, 0).ravel())


def test_biharmonic_interior_rows_are_squared_laplacian_and_clamped_diagonal():
    N = 9
    A = di.biharmonic13_2d(N).toarray()
    L = di.poisson5_2d(N).toarray()
    L2 = L @ L
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    i, j = i.ravel(), j.ravel()
    deep = (i >= 2) & (i <= N - 3) & (j >= 2) & (j <= N - 3)
    np.testing.assert_array_equal(A[deep], L2[deep])
    edges = (i == 0).astype(int) + (i == N - 1) + (j == 0) + (j == N - 1)
    np.testing.assert_array_equal(np.diag(A), 20 + edges)
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_varcoef_unit_kappa_is_cell_centred_laplacian():
    N = 4
    A, _ = di.varcoef7_3d(np.ones((N, N, N)))
    A = A.toarray()
    assert np.allclose(A, A.T)
    c = np.arange(N)
    bf = ((c == 0).astype(int) + (c == N - 1))
    faces = bf[None, None, :] + bf[None, :, None] + bf[:, None, None]
    # each boundary face is a Dirichlet face at half-cell distance: weight 2
    np.testing.assert_allclose(A @ np.ones(N ** 3), 2.0 * faces.ravel())
    np.testing.assert_allclose(np.diag(A), 6.0 + faces.ravel())


def test_grf_separable_covariance():
    # covariance of g = sigma * (Sz x Sy x Sx) xi is sigma^2 Kz x Ky x Kx
    shape = (5, 4, 3)
    n = np.prod(shape)
    G = np.stack([di.gaussian_random_field(shape, 0.3, 1.5, s).ravel() for s in range(4000)])
    emp = np.cov(G.T)
    x = [(np.arange(m) + 0.5) / m for m in shape]
    K = [np.exp(-(a[:, None] - a[None, :]) ** 2 / (2 * 0.3 ** 2)) for a in x]
    full = 1.5 ** 2 * np.kron(K[2], np.kron(K[1], K[0]))
    assert emp.shape == (n, n)
    assert np.max(np.abs(emp - full)) < 0.25


# ---------------------------------------------------------------- overlap
def test_box_overlap_sizes_and_graph_overlap_sizes():
    N, b = 24, 8
    A = di.poisson7_3d(N)
    part = di.box_partition((N,) * 3, (b,) * 3)
    om = orc.grow_overlap(A, part, 1, "box", (N,) * 3)
    sizes = np.array([len(o) for o in om]).reshape(3, 3, 3)
    assert sizes[1, 1, 1] == 10 ** 3            # interior box grows to 10^3
    assert sizes[0, 0, 0] == 9 ** 3             # corner box clipped on 3 faces
    assert sizes[1, 1, 0] == 10 * 10 * 9
    og = orc.grow_overlap(A, part, 1, "graph")
    assert len(og[13]) == 8 ** 3 + 6 * 8 ** 2  # 7-point graph distance 1


def test_greedy_colouring_is_lattice_colouring_and_valid():
    N, b = 24, 6
    A = di.poisson7_3d(N)
    part = di.box_partition((N,) * 3, (b,) * 3)
    om = orc.grow_overlap(A, part, 1, "box", (N,) * 3)
    col = orc.colour_subdomains(A, om)
    nb = N // b
    ix, iy, iz = np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij")
    lattice = (ix % 2 + 2 * (iy % 2) + 4 * (iz % 2)).transpose(2, 1, 0).ravel()
    np.testing.assert_array_equal(col, lattice)
    # validity by brute force: same colour => no A-coupling between the sets
    Ad = A.tocsr()
    for i in range(len(om)):
        for j in range(len(om)):
            if i != j and col[i] == col[j]:
                assert Ad[om[i], :][:, om[j]].nnz == 0
                assert np.intersect1d(om[i], om[j]).size == 0


# ---------------------------------------------------------------- R0
def test_R0_orthonormal_and_reproduces_generators():
    prob = di.make_poisson2d(N=24, box=8, overlap=1, p=2)
    R0, offs = orc.coarse_basis(prob.F, prob.part)
    assert R0.shape == (9 * 6, prob.n)
    np.testing.assert_allclose((R0 @ R0.T).toarray(), np.eye(R0.shape[0]), atol=1e-12)
    # every generator restricted to every subdomain lies in span(R0^T)
    np.testing.assert_allclose(R0.T @ (R0 @ prob.F), prob.F, atol=1e-12)


def test_R0_p0_is_normalised_aggregation():
    # Sec. 2: with only the constant generator the method is non-smoothed
    # aggregation: one basis vector per subdomain, 1/sqrt(|Omega_i|) on it.
    prob = di.make_poisson2d(N=20, box=6, overlap=1, p=0)
    R0, _ = orc.coarse_basis(prob.F, prob.part)
    R = np.abs(R0.toarray())
    for i in range(prob.nsub):
        members = prob.part == i
        np.testing.assert_allclose(R[i, members], 1 / np.sqrt(members.sum()), rtol=1e-14)
        assert np.all(R[i, ~members] == 0)


def test_R0_rank_drop_on_degenerate_subdomain():
    # a subdomain that is one grid line x = const: of the six quadratics only
    # 1, y, y^2 stay independent there, so its block keeps rank 3.
    N = 8
    coords = di.fd_node_coords((N, N))
    F = di.monomials(coords, 2)
    i = np.arange(N * N) % N
    part = np.where(i == 0, 0, 1).astype(np.int32)
    R0, offs = orc.coarse_basis(F, part)
    assert offs[1] - offs[0] == 3
    assert offs[2] - offs[1] == 6


# ---------------------------------------------------------------- A0 / coarse
def test_coarse_reproduces_exact_polynomial_solution():
    # u = x(1-x)y(1-y) is degree 2 in each variable, so the 5-point stencil
    # is exact for it and (with homogeneous Dirichlet data) the discrete
    # solution of A u = h^2 * 2(x(1-x) + y(1-y)) is u itself.  With p = 4 the
    # coarse space contains u, and Galerkin projection must reproduce it.
    N = 31
    prob = di.make_poisson2d(N=N, box=8, overlap=1, p=4)
    x, y = di.fd_node_coords((N, N)).T
    u = x * (1 - x) * y * (1 - y)
    h = 1.0 / (N + 1)
    f = h * h * 2 * (x * (1 - x) + y * (1 - y))
    np.testing.assert_allclose(prob.A @ u, f, atol=1e-15)
    M = _oracle(prob)
    np.testing.assert_allclose(M.coarse_correction(f), u, atol=1e-11 * np.abs(u).max())


def test_coarse_galerkin_invariants():
    prob = di.make_poisson2d(N=24, box=8, overlap=1, p=2)
    M = _oracle(prob)
    A0 = M.A0.toarray()
    assert np.allclose(A0, A0.T, rtol=0, atol=1e-14 * np.abs(A0).max())
    assert np.linalg.eigvalsh(A0).min() > 0
    rng = np.random.default_rng(0)
    # reproduction of any coarse-space vector
    c = rng.standard_normal(M.R0.shape[0])
    ustar = M.R0.T @ c
    np.testing.assert_allclose(M.coarse_correction(prob.A @ ustar), ustar, atol=1e-11)
    # Galerkin optimality (Sec. 5): the coarse solution is A-norm best, so it
    # beats the l2 projection R0^T R0 u
    u = rng.standard_normal(prob.n)
    uc = M.coarse_correction(prob.A @ u)
    v = M.R0.T @ (M.R0 @ u)
    an = lambda e: np.sqrt(e @ (prob.A @ e))
    assert an(uc - u) <= an(v - u) * (1 + 1e-12)


def test_coarse_solver_banded_branch_matches_sparse_direct_solve():
    # CoarseSolver factorises A0 in LAPACK's lower band storage (ab[i - j, j]
    # = A0[i, j]) once n0 exceeds its dense limit.  The 256^2 Poisson problem
    # with 32^2 subdomains of 8^2 and p <= 2 has n0 = 1024 * 6 = 6144, so the
    # band branch is chosen by size; its solves are compared with scipy's
    # sparse LU (a different factorisation of the same A0), and the coarse
    # correction built on it must reproduce coarse-space vectors (Galerkin).
    from scipy.sparse.linalg import spsolve
    prob = di.make_poisson2d(N=256, box=8, overlap=1, p=2, seed=3)
    M = _oracle(prob)
    assert M.A0.shape[0] == 6144 and M.coarse.kind == "banded"
    rng = np.random.default_rng(4)
    c = rng.standard_normal(M.A0.shape[0])
    ref = spsolve(M.A0.tocsc(), c)
    np.testing.assert_allclose(M.coarse.solve(c), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    ustar = M.R0.T @ rng.standard_normal(M.A0.shape[0])
    np.testing.assert_allclose(M.coarse_correction(prob.A @ ustar), ustar, rtol=0,
                               atol=1e-10 * np.abs(ustar).max())
    # the same branch forced on a small A0 agrees with the dense branch
    small = _oracle(di.make_biharmonic2d(N=48, box=16, overlap=2, p=3, seed=5))
    band = orc.CoarseSolver(small.A0, dense_limit=0)
    assert band.kind == "banded" and small.coarse.kind == "dense"
    c = rng.standard_normal(small.A0.shape[0])
    x_dense = small.coarse.solve(c)
    np.testing.assert_allclose(band.solve(c), x_dense, rtol=0, atol=1e-10 * np.abs(x_dense).max())


def test_coarse_error_non_increasing_in_p():
    # Sec. 5, "Proof vs. Practice": raising p grows the coarse space and
    # Galerkin is optimal in it, so the A-norm error never increases.
    N = 32
    x, y = di.fd_node_coords((N, N)).T
    u = np.sin(3 * x) * np.exp(y) * x * (1 - x) * y * (1 - y)
    errs = []
    for p in range(5):
        prob = di.make_poisson2d(N=N, box=8, overlap=1, p=p)
        M = _oracle(prob)
        e = M.coarse_correction(prob.A @ u) - u
        errs.append(np.sqrt(e @ (prob.A @ e)))
    assert all(b <= a * (1 + 1e-10) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.05 * errs[0]


# ---------------------------------------------------------------- local solves
def test_local_solve_matches_dense_solve():
    prob = di.make_poisson2d(N=24, box=8, overlap=2, p=2)
    M = _oracle(prob)
    Ad = prob.A.toarray()
    rng = np.random.default_rng(1)
    r = rng.standard_normal(prob.n)
    i = 4
    idx = M.omega[i]
    z = np.zeros(prob.n)
    M._subdomain_step(i, r, z)
    np.testing.assert_allclose(z[idx], np.linalg.solve(Ad[np.ix_(idx, idx)], r[idx]), rtol=1e-12)


# ---------------------------------------------------------------- apply_M
@pytest.mark.parametrize("maker", [
    lambda: di.make_poisson2d(N=14, box=5, overlap=1, p=1),
    lambda: di.make_biharmonic2d(N=12, box=6, overlap=1, p=2),
])
def test_preconditioner_symmetric_positive_and_product_form(maker):
    prob = maker()
    M = _oracle(prob)
    Minv = M.dense_preconditioner()
    assert np.max(np.abs(Minv - Minv.T)) <= 1e-12 * np.abs(Minv).max()
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0
    # Sec. 6: error propagation of the symmetric multiplicative method is
    # E = (I-P_1)...(I-P_N)(I-P_0)(I-P_N)...(I-P_1) in the sweep order,
    # and M^{-1} = (I - E) A^{-1}.
    P, P0 = M.dense_projections()
    n = prob.n
    I = np.eye(n)
    E = I.copy()
    for i in M.order:                       # pre-smoother, first subdomain first
        E = (I - P[i]) @ E
    E = (I - P0) @ E
    for i in reversed(M.order):             # post-smoother, reverse order
        E = (I - P[i]) @ E
    Ad = prob.A.toarray()
    ref = (I - E) @ np.linalg.inv(Ad)
    np.testing.assert_allclose(Minv, ref, atol=1e-10 * np.abs(ref).max())


def test_order_inside_a_colour_is_irrelevant_bitwise():
    prob = di.make_poisson2d(N=40, box=8, overlap=2, p=2)
    M = _oracle(prob)
    r = np.random.default_rng(2).standard_normal(prob.n)
    z1 = M.apply(r)
    rng = np.random.default_rng(3)
    order = []
    for c in range(int(M.colour.max()) + 1):
        ids = np.flatnonzero(M.colour == c)
        order += list(rng.permutation(ids))
    M.order = order
    z2 = M.apply(r)
    assert np.array_equal(z1, z2)


# ---------------------------------------------------------------- PCG
def test_pcg_matches_direct_solve():
    prob = di.make_poisson2d(N=32, box=8, overlap=2, p=2)
    res, M = orc.solve(prob.A, prob.part, prob.F, prob.f, 2, "box", prob.shape, tol=1e-12)
    assert res.converged
    exact = np.linalg.solve(prob.A.toarray(), prob.f)
    assert np.linalg.norm(res.u - exact) <= 1e-9 * np.linalg.norm(exact)
    assert res.true_relres <= 1e-11


def test_unpreconditioned_cg_converges_in_at_most_n_steps():
    A = di.poisson5_2d(6)
    f = di.uniform_rhs(36, 5)
    res = orc.pcg(A, f, lambda r: r.copy(), tol=1e-10)
    assert res.converged and res.iters <= 36


def test_iterations_flat_in_h_at_fixed_H_over_h():
    # Sec. 7 / Table 1: at fixed H/h the two-level iteration count does not
    # grow with the problem size.
    its = []
    for N in (32, 64, 128):
        prob = di.make_poisson2d(N=N, box=8, overlap=1, p=2)
        res, _ = orc.solve(prob.A, prob.part, prob.F, prob.f, 1, "box", prob.shape, tol=1e-8)
        its.append(res.iters)
    assert max(its) - min(its) <= 2, its


def test_iterations_non_increasing_in_p():
    its = []
    for p in range(4):
        prob = di.make_poisson2d(N=64, box=16, overlap=1, p=p)
        res, _ = orc.solve(prob.A, prob.part, prob.F, prob.f, 1, "box", prob.shape, tol=1e-8)
        its.append(res.iters)
    assert all(b <= a for a, b in zip(its, its[1:])), its
    assert its[-1] < its[0]


def test_lanczos_estimates_match_dense_spectrum():
    prob = di.make_poisson2d(N=16, box=4, overlap=1, p=1)
    M = _oracle(prob)
    res = orc.pcg(M.A, prob.f, M.apply, tol=1e-14)
    lo, hi = orc.lanczos_extremes(res.alphas, res.betas)
    Minv = M.dense_preconditioner()
    ev = np.sort(np.linalg.eigvals(Minv @ prob.A.toarray()).real)
    # Ritz values interlace: they lie inside [lambda_min, lambda_max] of
    # M^{-1}A and approach both ends as CG converges.  The symmetric
    # multiplicative method has lambda_max = 1 (I - M^{-1}A = E >= 0 in the
    # A inner product).
    assert abs(ev[-1] - 1.0) < 1e-10
    assert ev[0] * (1 - 1e-10) <= lo and hi <= ev[-1] * (1 + 1e-10)
    assert hi >= 0.999 * ev[-1]
    assert lo <= 1.01 * ev[0]


def test_fractional_iterations_geometric_history():
    h = 10.0 ** -np.arange(8)          # straight log-residual line
    assert abs(orc.fractional_iterations(h, 10 ** -3.5) - 3.5) < 1e-12
    assert orc.fractional_iterations(h, 1e-9) != orc.fractional_iterations(h, 1e-9)  # nan


@pytest.mark.slow
def test_table1_plausibility_poisson3d():
    # Table 1 (Sec. 7): 3D Poisson, n^(1/3) = 40, H/h = 10, Delta = 0.
    # The paper's boundary conditions (one Dirichlet face) and irregular
    # partitions make its problem harder than this all-Dirichlet box
    # version, so the counts here may not exceed the paper's by more than 2,
    # and they must fall as p grows.
    gold = json.load(open(os.path.join(GOLDEN, "table1_poisson3d.json")))
    N = gold["n_1d"]
    its = []
    for p in range(4):
        prob = di.make_poisson3d(N=N, box=gold["H_over_h"], overlap=0, p=p, mode="graph")
        res, _ = orc.solve(prob.A, prob.part, prob.F, di.normal_rhs(prob.n, 7), 0, "graph",
                           tol=1e-9)
        its.append(res.iters)
    paper = [gold["cg_iterations"][f"P{p}"] for p in range(4)]
    assert all(a <= b + 2 for a, b in zip(its, paper)), (its, paper)
    assert all(b <= a for a, b in zip(its, its[1:])), its


def test_q1_elasticity_patch_test_and_rigid_modes():
    # element matrices annihilate rigid motions; the assembled operator with
    # constant coefficients maps any linear displacement field (constant
    # strain, an exact FE solution of the homogeneous equations) to zero at
    # the interior nodes -- the FEM patch test
    Kl, Km = di.q1_reference_stiffness()
    pts = np.array([[a & 1, (a >> 1) & 1, a >> 2] for a in range(8)], float)
    for fn in (lambda p: [1, 0, 0], lambda p: [0, 0, 1], lambda p: [-p[1], p[0], 0],
               lambda p: [p[2], 0, -p[0]]):
        v = np.concatenate([fn(p) for p in pts])
        assert np.abs(Kl @ v).max() < 1e-14 and np.abs(Km @ v).max() < 1e-14
    ne = 5
    A, (nx, ny, nz) = di.elasticity_q1_3d(np.full((ne, ne, ne), 1.3), lam=0.7)
    node = np.arange(nx * ny * nz)
    I, J, K = node % nx + 1, (node // nx) % ny, node // (nx * ny)
    x, y, z = I / ne, J / ne, K / ne
    u = np.stack([0.3 * x + 0.2 * y - 0.1 * z, -0.4 * x + 0.5 * z, 0.25 * y + 0.6 * z], axis=1).ravel()
    r = (A @ u).reshape(-1, 3)
    # interior: every neighbouring node carries the linear field (nodes at
    # I = 1 touch the clamped, eliminated x = 0 layer)
    interior = (I > 1) & (I < ne) & (J > 0) & (J < ne) & (K > 0) & (K < ne)
    assert np.abs(r[interior]).max() < 1e-13
    assert np.abs(r[~interior]).max() > 1e-3          # boundary rows carry tractions
    assert np.linalg.eigvalsh(A.toarray()).min() > 0  # clamped: SPD
