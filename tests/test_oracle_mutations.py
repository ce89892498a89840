"""Planted mistakes in the oracle (CPU only) must fail the pins.

Each test copies the oracle's behaviour with one plausible error (wrong
sweep order, dropped term, wrong sign, transposed operand) and checks that
the corresponding pin of test_oracle_pins.py would reject it.  This shows
the pins constrain the oracle rather than restate it.
"""
import numpy as np
import scipy.linalg as sla

import ddg_inputs as di
from oracle import ddg_oracle as orc


def _setup():
    prob = di.make_poisson2d(N=14, box=5, overlap=1, p=1)
    M = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape, dpn=prob.dofs_per_node)
    return prob, M


def _dense(apply, n):
    I = np.eye(n)
    return np.stack([apply(I[:, j]) for j in range(n)], axis=1)


def _product_form(M, prob):
    P, P0 = M.dense_projections()
    I = np.eye(prob.n)
    E = I.copy()
    for i in M.order:
        E = (I - P[i]) @ E
    E = (I - P0) @ E
    for i in reversed(M.order):
        E = (I - P[i]) @ E
    return (I - E) @ np.linalg.inv(prob.A.toarray())


def test_forward_post_smoother_breaks_symmetry():
    prob, M = _setup()

    def wrong(r):
        z = np.zeros_like(r)
        for i in M.order:
            M._subdomain_step(i, r, z)
        z += M.coarse_correction(r - M.A @ z)
        for i in M.order:                      # mistake: not reversed
            M._subdomain_step(i, r, z)
        return z

    W = _dense(wrong, prob.n)
    assert np.max(np.abs(W - W.T)) > 1e-6 * np.abs(W).max()


def test_dropped_coarse_residual_update_fails_product_form():
    prob, M = _setup()

    def wrong(r):
        z = np.zeros_like(r)
        for i in M.order:
            M._subdomain_step(i, r, z)
        z += M.coarse_correction(r)            # mistake: residual of z dropped
        for i in reversed(M.order):
            M._subdomain_step(i, r, z)
        return z

    ref = _product_form(M, prob)
    assert np.linalg.norm(_dense(wrong, prob.n) - ref) > 1e-6 * np.linalg.norm(ref)


def test_residual_sign_error_fails_local_and_product_pins():
    prob, M = _setup()

    def step(i, r, z):
        idx = M.omega[i]
        res = r[idx] + M.rows[i] @ z          # mistake: wrong sign
        z[idx] += sla.cho_solve(M.local[i], res)

    def wrong(r):
        z = np.zeros_like(r)
        for i in M.order:
            step(i, r, z)
        z += M.coarse_correction(r - M.A @ z)
        for i in reversed(M.order):
            step(i, r, z)
        return z

    ref = _product_form(M, prob)
    assert np.linalg.norm(_dense(wrong, prob.n) - ref) > 1e-6 * np.linalg.norm(ref)


def test_off_by_one_local_factor_fails_product_form():
    prob, M = _setup()

    def step(i, r, z):
        idx = M.omega[i]
        j = (i + 1) % M.nsub                   # mistake: neighbouring subdomain's factor
        res = r[idx] - M.rows[i] @ z
        if len(M.omega[j]) == len(idx):
            z[idx] += sla.cho_solve(M.local[j], res)
        else:
            z[idx] += res / np.diag(M.local[i][0]) ** 2

    def wrong(r):
        z = np.zeros_like(r)
        for i in M.order:
            step(i, r, z)
        z += M.coarse_correction(r - M.A @ z)
        for i in reversed(M.order):
            step(i, r, z)
        return z

    ref = _product_form(M, prob)
    assert np.linalg.norm(_dense(wrong, prob.n) - ref) > 1e-6 * np.linalg.norm(ref)


def test_unorthogonalised_basis_fails_orthonormality_pin():
    prob = di.make_poisson2d(N=24, box=8, overlap=1, p=2)
    # mistake: raw restricted generators used as rows of R0 (no QR)
    rows = []
    for i in range(prob.nsub):
        dofs = np.flatnonzero(prob.part == i)
        for j in range(prob.F.shape[1]):
            v = np.zeros(prob.n)
            v[dofs] = prob.F[dofs, j]
            rows.append(v)
    R = np.array(rows)
    assert np.max(np.abs(R @ R.T - np.eye(R.shape[0]))) > 1e-3


def test_transposed_band_storage_fails_sparse_direct_solve():
    # The band branch of CoarseSolver with the upper band layout
    # ab[b + j - i, i] (what LAPACK expects for lower=False) handed to the
    # lower-band factorisation: the comparison with scipy's sparse LU
    # (test_coarse_solver_banded_branch_matches_sparse_direct_solve) rejects it.
    from scipy.sparse.linalg import spsolve
    prob = di.make_biharmonic2d(N=48, box=16, overlap=2, p=3, seed=5)
    M = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape)
    C = M.A0.tocoo()
    b = int(np.max(C.row - C.col))
    ab = np.zeros((b + 1, M.A0.shape[0]))
    up = C.row <= C.col
    ab[b + C.row[up] - C.col[up], C.col[up]] = C.data[up]   # mistake: upper layout
    c = np.random.default_rng(4).standard_normal(M.A0.shape[0])
    ref = spsolve(M.A0.tocsc(), c)
    try:
        x = sla.cho_solve_banded((sla.cholesky_banded(ab, lower=True), True), c)
    except np.linalg.LinAlgError:
        return   # not even positive definite in that layout
    assert np.abs(x - ref).max() > 1e-6 * np.abs(ref).max()
