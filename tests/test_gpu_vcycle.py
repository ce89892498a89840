"""Parity of the three-level V-cycle (Sec. 6) on the GPU with the oracle.

The library builds the coarse level as a second two-level handle on A0 with
generators F0 = R0 F (``ddg_setup_vcycle``); the oracle composes its own
two-level oracle on A0.  Tolerances as in test_gpu_parity.py: FP64 building
blocks 1e-11, FP64 PCG solution 1e-10 with iterations within 1, FP32 / BF16
preconditioner: true residual <= tol and 1e-7 against the oracle's solution.
"""
import numpy as np
import pytest

import ddg_inputs as di
from oracle import ddg_oracle as orc
from closeness import assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    # 6 x 6 subdomains in 3 x 3 groups
    "poisson2d_48": (lambda: di.make_poisson2d(N=48, box=8, overlap=1, p=2, seed=20), 2),
    # 5^3 subdomains in 3^3 groups, the last group one subdomain wide
    "poisson3d_20_ragged": (lambda: di.make_poisson3d(N=20, box=4, overlap=1, p=2, seed=21), 2),
    # 13-point stencil: A0 couples diagonal neighbours; overlap 2 on both levels
    "biharmonic_64": (lambda: di.make_biharmonic2d(N=64, box=16, overlap=2, p=3, seed=22), 2),
    "varcoef_16": (lambda: di.make_varcoef3d(N=16, box=4, overlap=1, p=2, m=None), 2),
    # rank-deficient boundary subdomains (p = 2 on 2-wide boxes) and graph overlap
    "poisson3d_graph_rankdrop": (lambda: di.make_poisson3d(N=10, box=2, overlap=1, p=2, seed=23,
                                                           mode="graph"), 3),
}

_cache = {}


def setup_case(name):
    if name not in _cache:
        from paper_1504_00907_gb300 import ddg
        make, g = CASES[name]
        prob = make()
        groups = di.subdomain_groups(prob.shape, prob.box, g)
        solver = ddg.Solver.from_problem(prob, precision="fp64", keep=("fp64", "fp32", "bf16"),
                                         coarse_groups=groups)
        oracle = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape,
                               coarse_groups=groups)
        _cache[name] = (prob, solver, oracle, groups)
    return _cache[name]


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rhs(prob):
    return prob.f if prob.f.ndim == 1 else prob.f[:, 0]


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_colouring_and_ranks_match_oracle(name):
    prob, solver, oracle, _ = setup_case(name)
    np.testing.assert_array_equal(solver.colouring(), oracle.colour)
    np.testing.assert_array_equal(solver.coarse_offsets(), oracle.coarse_offsets)
    assert solver.info()["n0"] == oracle.A0.shape[0]


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_coarse_correction_matches_oracle(name):
    prob, solver, oracle, _ = setup_case(name)
    solver.set_precision("fp64")
    r = np.random.default_rng(50).standard_normal(prob.n)
    z = solver.coarse_correction(dev(r)).cpu().numpy()
    assert_close(z, oracle.coarse_correction(r), 1e-11)


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_preconditioner_matches_oracle_fp64(name):
    prob, solver, oracle, _ = setup_case(name)
    solver.set_precision("fp64")
    r = np.random.default_rng(51).standard_normal(prob.n)
    z = solver.apply(dev(r)).cpu().numpy()
    assert_close(z, oracle.apply(r), 1e-11)


# FP32 tolerance: the normwise error of a solve with an FP32 inverse is about
# cond(block) * 2^-24.  The coarse-level blocks of the 13-point operator have
# cond(A0[i, i]) = 8.8e4 (8.8e3 on the fine level), so 8.8e4 * 2^-24 = 5e-3;
# the second-order cases stay below 1e-5.
@pytest.mark.parametrize("name,prec,tol", [("poisson2d_48", "fp32", 1e-5), ("poisson3d_20_ragged", "fp32", 1e-5),
                                           ("varcoef_16", "fp32", 1e-5), ("biharmonic_64", "fp32", 5e-3),
                                           ("poisson3d_20_ragged", "bf16", 3e-2)])
def test_vcycle_preconditioner_reduced_precision(name, prec, tol):
    prob, solver, oracle, _ = setup_case(name)
    solver.set_precision(prec)
    r = np.random.default_rng(52).standard_normal(prob.n)
    z = solver.apply(dev(r)).cpu().numpy()
    solver.set_precision("fp64")
    assert_close(z, oracle.apply(r), tol)


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_solve_fp64_matches_oracle(name):
    prob, solver, oracle, _ = setup_case(name)
    solver.set_precision("fp64")
    f = rhs(prob)
    ref = orc.pcg(oracle.A, f, oracle.apply, tol=1e-8)
    u, iters, relres, st = solver.solve(dev(f), tol=1e-8)
    assert st == 0 and relres <= 1e-8
    assert_close(u.cpu().numpy(), ref.u, 1e-10)
    assert abs(iters - ref.iters) <= 1
    hist = solver.history()
    m = min(hist.size, ref.history.size)
    np.testing.assert_allclose(hist[:m], ref.history[:m], rtol=1e-6, atol=1e-13)


@pytest.mark.parametrize("name,prec", [("poisson2d_48", "fp32"), ("poisson3d_20_ragged", "fp32"),
                                       ("varcoef_16", "fp32"), ("biharmonic_64", "fp32"),
                                       ("poisson3d_20_ragged", "bf16")])
def test_vcycle_solve_mixed_precision(name, prec):
    prob, solver, oracle, _ = setup_case(name)
    f = rhs(prob)
    ref = orc.pcg(oracle.A, f, oracle.apply, tol=1e-8)
    solver.set_precision(prec)
    u, iters, relres, st = solver.solve(dev(f), tol=1e-8)
    solver.set_precision("fp64")
    assert st == 0
    un = u.cpu().numpy()
    assert np.linalg.norm(f - prob.A @ un) / np.linalg.norm(f) <= 1e-8
    assert_close(un, ref.u, 1e-7)
    assert iters <= ref.iters + 3


def test_vcycle_is_slower_to_converge_than_two_level_but_converges():
    # Table 1: the V-cycle needs more iterations than the exact coarse solve
    prob, solver, oracle, _ = setup_case("poisson3d_20_ragged")
    two = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape)
    f = rhs(prob)
    ref2 = orc.pcg(two.A, f, two.apply, tol=1e-8)
    solver.set_precision("fp64")
    _, iters, _, st = solver.solve(dev(f), tol=1e-8)
    assert st == 0 and ref2.iters <= iters <= 3 * ref2.iters


def test_vcycle_one_group_equals_two_level_on_gpu():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson2d(N=40, box=8, overlap=1, p=2, seed=24)
    s2 = ddg.Solver.from_problem(prob, precision="fp64")
    s3 = ddg.Solver.from_problem(prob, precision="fp64",
                                 coarse_groups=np.zeros(prob.nsub, dtype=np.int32))
    r = dev(np.random.default_rng(53).standard_normal(prob.n))
    z2, z3 = s2.apply(r).cpu().numpy(), s3.apply(r).cpu().numpy()
    s2.close()
    s3.close()
    assert_close(z3, z2, 1e-11)


def test_vcycle_batch_solves_columns_one_at_a_time():
    prob, solver, oracle, _ = setup_case("poisson2d_48")
    F = di.normal_rhs(prob.n, 60, 3)
    solver.set_precision("fp32")
    U, its, rrs, st = solver.solve_batch(dev(F), tol=1e-8)
    assert st == 0 and np.all(rrs <= 1e-8)
    for j in range(3):
        u, it, rr, st1 = solver.solve(dev(F[:, j]), tol=1e-8)
        assert st1 == 0 and it == its[j]
        assert_close(U[:, j].cpu().numpy(), u.cpu().numpy(), 1e-14)
    solver.set_precision("fp64")


def test_vcycle_counts_coarse_level_launches():
    prob, solver, _, _ = setup_case("poisson2d_48")
    solver.set_precision("fp32")
    solver.profile(())
    solver.apply(dev(rhs(prob)))
    st = solver.kernel_stats()
    solver.set_precision("fp64")
    # restrict + prolong, then the coarse level's residual and solve
    # launches per colour and sweep, and its own coarse step
    assert st["coarse"]["launches"] > 2 + 4 * 4
