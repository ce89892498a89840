"""Sec. 7 condition estimates from the CG coefficients, on the CPU.

The oracle's ``lanczos_extremes`` and ``cg_iteration_bound`` are pinned to
closed forms; the library's host-only ``ddg_condition_estimate`` (its own
bisection on Sturm counts) is checked against them and against the same
closed forms.  No GPU is used.
"""
import numpy as np
import pytest

import ddg_inputs as di
from oracle import ddg_oracle as orc


@pytest.fixture(scope="module")
def ddg():
    from paper_1504_00907_gb300 import build, ddg as mod
    import os
    if not os.path.exists(mod.LIB_PATH):
        build.build()
    mod.load()
    return mod


def _plain_cg_on_diagonal(m):
    # unpreconditioned CG on diag(1..m) from a vector with every eigen-
    # component present ends after m steps with Ritz values = eigenvalues
    A = np.diag(np.arange(1.0, m + 1))
    res = orc.pcg(A, np.ones(m), lambda r: r.copy(), tol=1e-15, maxit=m)
    return res


def test_oracle_bound_closed_form():
    # kappa = 9: (sqrt k + 1)/(sqrt k - 1) = 2, so the bound is log2(2/tol)
    assert abs(orc.cg_iteration_bound(9.0, 2.0 ** -10) - 11.0) < 1e-12
    assert orc.cg_iteration_bound(1.0, 1e-8) == 0.0


def test_oracle_lanczos_on_diagonal_recovers_spectrum_ends():
    res = _plain_cg_on_diagonal(10)
    lo, hi = orc.lanczos_extremes(res.alphas, res.betas)
    assert abs(lo - 1.0) < 1e-8 and abs(hi - 10.0) < 1e-8


def test_library_estimate_matches_closed_forms(ddg):
    res = _plain_cg_on_diagonal(10)
    lo, hi, bound = ddg.condition_estimate(res.alphas, res.betas, 2.0 ** -10)
    assert abs(lo - 1.0) < 1e-8 and abs(hi - 10.0) < 1e-8
    assert abs(bound - orc.cg_iteration_bound(hi / lo, 2.0 ** -10)) <= 1e-12 * bound
    # one step: the 1x1 tridiagonal 1/alpha_0
    lo1, hi1, _ = ddg.condition_estimate(np.array([0.25]), np.array([]), 1e-8)
    assert lo1 == pytest.approx(4.0, rel=1e-14) and hi1 == pytest.approx(4.0, rel=1e-14)


@pytest.mark.parametrize("make", [
    lambda: di.make_poisson2d(N=24, box=6, overlap=1, p=1),
    lambda: di.make_biharmonic2d(N=32, box=8, overlap=2, p=3),
    lambda: di.make_poisson3d(N=12, box=4, overlap=1, p=2),
])
def test_library_estimate_matches_oracle_on_ddg_cg(ddg, make):
    prob = make()
    M = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape)
    res = orc.pcg(M.A, prob.f, M.apply, tol=1e-10)
    lo_o, hi_o = orc.lanczos_extremes(res.alphas, res.betas)
    lo, hi, bound = ddg.condition_estimate(res.alphas, res.betas, 1e-8)
    assert abs(lo - lo_o) <= 1e-10 * hi_o and abs(hi - hi_o) <= 1e-10 * hi_o
    assert abs(bound - orc.cg_iteration_bound(hi_o / lo_o, 1e-8)) <= 1e-8 * bound
    # symmetric multiplicative Schwarz: lambda_max(M^{-1}A) <= 1
    assert hi <= 1.0 + 1e-10


def test_library_estimate_rejects_bad_input(ddg):
    with pytest.raises(ddg.DDGError):
        ddg.condition_estimate(np.array([1.0, -1.0]), np.array([0.5]), 1e-8)
    with pytest.raises(ddg.DDGError):
        ddg.condition_estimate(np.array([1.0]), np.array([]), 2.0)


def test_planted_dropped_beta_term_fails_the_diagonal_pin():
    # mistake: diagonal 1/alpha_j without beta_{j-1}/alpha_{j-1}
    import scipy.linalg as sla
    res = _plain_cg_on_diagonal(10)
    a, b = np.asarray(res.alphas), np.asarray(res.betas)
    d = 1.0 / a
    e = np.sqrt(b) / a[:-1]
    w = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    assert abs(w[0] - 1.0) > 1e-3 or abs(w[-1] - 10.0) > 1e-3


def test_planted_swapped_offdiagonal_scale_fails_the_diagonal_pin():
    # mistake: off-diagonal sqrt(beta_j) / alpha_{j+1} instead of / alpha_j
    import scipy.linalg as sla
    res = _plain_cg_on_diagonal(10)
    a, b = np.asarray(res.alphas), np.asarray(res.betas)
    d = 1.0 / a
    d[1:] += b / a[:-1]
    e = np.sqrt(b) / a[1:]
    w = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    assert abs(w[0] - 1.0) > 1e-3 or abs(w[-1] - 10.0) > 1e-3
