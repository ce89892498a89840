"""Pins of the oracle's three-level V-cycle (Sec. 6), CPU only.

The three-level method replaces the exact coarse solve A0^{-1} by one
application B0 of the two-level method to A0 with generators F0 = R0 F.
What fixes it independently of the sweep code:

* with a single coarse-level subdomain, the inner pre-smoother solves A0
  exactly, so the three-level method is the two-level method;
* its error propagation is the product of projections
  E = (I-P_N)...(I-P_1) (I - R0^T B0 R0 A) (I-P_1)...(I-P_N), with
  B0 = (I - E_0) A0^{-1} and E_0 the same product on A0 (Sec. 6);
* the paper states that coarsening the coarse problem is the same as
  coarsening the original problem directly with larger subdomains: the
  level-2 correction R0^T R1^T A1^{-1} R1 R0 A equals the A-orthogonal
  projection onto the DDG space of the grouped partition;
* the preconditioner is symmetric and positive definite.

Each pin is followed by a planted mistake that it rejects.
"""
import numpy as np

import ddg_inputs as di
from oracle import ddg_oracle as orc


def _problem(N=16, box=4, overlap=1, p=1):
    return di.make_poisson2d(N=N, box=box, overlap=overlap, p=p)


def _oracle(prob, groups=None):
    return orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape,
                         coarse_groups=groups)


def _dense(apply, n):
    I = np.eye(n)
    return np.stack([apply(I[:, j]) for j in range(n)], axis=1)


def _sweep_product(M, P, I):
    """(I-P_N)...(I-P_1) in the sweep order (first subdomain first)."""
    E = I.copy()
    for i in M.order:
        E = (I - P[i]) @ E
    return E


def _vcycle_product_form(M, prob):
    """(I - E) A^{-1} with E the error propagation of the V-cycle (Sec. 6)."""
    inner = M.inner
    # level 1: B0 = (I - E_0) A0^{-1}, E_0 the two-level product on A0
    P0s, P01 = inner.dense_projections()
    n0 = inner.n
    I0 = np.eye(n0)
    pre0 = _sweep_product(inner, P0s, I0)
    post0 = I0.copy()
    for i in reversed(inner.order):
        post0 = (I0 - P0s[i]) @ post0
    E0 = post0 @ (I0 - P01) @ pre0
    A0 = M.A0.toarray()
    B0 = (I0 - E0) @ np.linalg.inv(A0)
    # level 0
    P, _ = M.dense_projections()
    I = np.eye(prob.n)
    Ad = prob.A.toarray()
    R0 = M.R0.toarray()
    E = _sweep_product(M, P, I)
    E = (I - R0.T @ B0 @ R0 @ Ad) @ E
    for i in reversed(M.order):
        E = (I - P[i]) @ E
    return (I - E) @ np.linalg.inv(Ad)


def test_single_coarse_subdomain_reduces_to_two_level():
    prob = di.make_poisson2d(N=24, box=6, overlap=1, p=2)
    M2 = _oracle(prob)
    M3 = _oracle(prob, groups=np.zeros(prob.nsub, dtype=np.int32))
    assert M3.inner is not None and M3.inner.nsub == 1
    r = np.random.default_rng(40).standard_normal(prob.n)
    z2, z3 = M2.apply(r), M3.apply(r)
    assert np.linalg.norm(z3 - z2) <= 1e-12 * np.linalg.norm(z2)


def test_vcycle_matches_error_propagation_product():
    prob = _problem()
    groups = di.subdomain_groups(prob.shape, prob.box, 2)
    M = _oracle(prob, groups)
    assert M.inner.nsub == 4 and M.A0.shape[0] == 16 * 3
    ref = _vcycle_product_form(M, prob)
    got = M.dense_preconditioner()
    np.testing.assert_allclose(got, ref, atol=1e-10 * np.abs(ref).max())


def test_level2_correction_is_direct_coarsening_with_grouped_subdomains():
    prob = di.make_poisson2d(N=24, box=4, overlap=1, p=2)
    groups = di.subdomain_groups(prob.shape, prob.box, 3)
    M = _oracle(prob, groups)
    Ad = prob.A.toarray()
    R0 = M.R0.toarray()
    R1 = M.inner.R0.toarray()
    A1 = M.inner.A0.toarray()
    composite = R0.T @ R1.T @ np.linalg.solve(A1, R1 @ R0 @ Ad)
    direct = orc.DDGOracle(prob.A, groups[prob.part], prob.F, prob.overlap, prob.overlap_mode,
                           prob.shape)
    _, P_direct = direct.dense_projections()
    np.testing.assert_allclose(composite, P_direct, atol=1e-9)
    # the grouped coarse dimension: 2 x 2 groups x 6 monomials of degree <= 2
    assert A1.shape == (4 * 6, 4 * 6)


def test_vcycle_is_symmetric_positive_definite():
    prob = _problem(N=18, box=3, overlap=1, p=1)
    M = _oracle(prob, di.subdomain_groups(prob.shape, prob.box, 2))
    W = M.dense_preconditioner()
    assert np.max(np.abs(W - W.T)) <= 1e-12 * np.abs(W).max()
    assert np.linalg.eigvalsh(0.5 * (W + W.T)).min() > 0


def test_vcycle_pcg_converges_and_groups_without_coarse_dofs_are_dropped():
    prob = di.make_poisson3d(N=12, box=3, overlap=1, p=1, mode="box")
    groups = di.subdomain_groups(prob.shape, prob.box, 2)
    res = orc.pcg(prob.A, prob.f, _oracle(prob, groups).apply)
    assert res.converged and res.true_relres <= 1e-8
    # unused group ids are compacted away: ids with gaps (same order) give
    # the same coarse-level subdomains, bit for bit
    g2 = 2 * groups + 5
    M1, M2 = _oracle(prob, groups), _oracle(prob, g2)
    r = np.random.default_rng(41).standard_normal(prob.n)
    np.testing.assert_array_equal(M1.apply(r), M2.apply(r))


# ---------------------------------------------------------------- planted mistakes
def test_planted_exact_inner_coarse_solve_fails_product_form():
    prob = _problem()
    M = _oracle(prob, di.subdomain_groups(prob.shape, prob.box, 2))
    ref = _vcycle_product_form(M, prob)
    A0 = M.A0.toarray()

    def wrong(r):                              # mistake: exact A0^{-1} (two-level)
        z = np.zeros_like(r)
        for i in M.order:
            M._subdomain_step(i, r, z)
        w = r - M.A @ z
        z += M.R0.T @ np.linalg.solve(A0, M.R0 @ w)
        for i in reversed(M.order):
            M._subdomain_step(i, r, z)
        return z

    assert np.linalg.norm(_dense(wrong, prob.n) - ref) > 1e-6 * np.linalg.norm(ref)


def test_planted_wrong_coarse_generators_fail_direct_coarsening():
    prob = di.make_poisson2d(N=24, box=4, overlap=1, p=2)
    groups = di.subdomain_groups(prob.shape, prob.box, 3)
    M = _oracle(prob, groups)
    # mistake: F0 taken as the first k rows pattern of F instead of R0 F
    sub_of_dof = np.repeat(np.arange(M.nsub), np.diff(M.coarse_offsets))
    _, part0 = np.unique(groups[sub_of_dof], return_inverse=True)
    F0_wrong = np.asarray(prob.F)[: M.A0.shape[0], :]
    R1, _ = orc.coarse_basis(F0_wrong, part0)
    R1 = R1.toarray()
    Ad = prob.A.toarray()
    R0 = M.R0.toarray()
    A1 = R1 @ (R0 @ Ad @ R0.T) @ R1.T
    composite = R0.T @ R1.T @ np.linalg.solve(A1, R1 @ R0 @ Ad)
    direct = orc.DDGOracle(prob.A, groups[prob.part], prob.F, prob.overlap, prob.overlap_mode,
                           prob.shape)
    _, P_direct = direct.dense_projections()
    assert np.abs(composite - P_direct).max() > 1e-3
