"""The two orderings of the exact coarse factor against the oracle: nested
dissection (coarse_order ND, the default) and the natural-order band.

The exact coarse solve A0^{-1} of Sec. 4 runs through a multifrontal
Cholesky factor of A0 ordered by nested dissection of the subdomain graph
(the oracle factorises A0 densely, or banded above 6000 coarse dofs).  The
coarse correction does not depend on the ordering, so FP64 results agree to
rounding: two backward-stable Cholesky solves of A0 differ by about
cond(A0) 2^-52, so the bound for the coarse correction and the
preconditioner is max(1e-11, cond(A0) 2^-52) and for PCG solutions
max(1e-10, cond(A0) 2^-52) (iterations within 1).  cond(A0) was computed
once with numpy eigvalsh: 1.56e6 for the biharmonic case (3.5e-10), 1.09e4
for elasticity, 217 for the Poisson case; the others are smaller problems of
the same kinds.  FP32 factors: mixed solves reach the true residual 1e-8 and
stay within 1e-7 of the oracle's solution.

Cases: 3D Poisson with 8^3 subdomains of 4^3 (a dissection tree of several
levels), the 13-point biharmonic (A0 couples diagonal neighbours), Q1
elasticity (30 generators per subdomain), graph overlap with rank-deficient
subdomains, and a single-front case.
"""
import numpy as np
import pytest

import ddg_inputs as di
from closeness import assert_close
from oracle import ddg_oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "poisson3d_32_box4": lambda: di.make_poisson3d(N=32, box=4, overlap=1, p=2, seed=41),
    "biharmonic_128_box16": lambda: di.make_biharmonic2d(N=128, box=16, overlap=2, p=3, seed=42),
    "elasticity_q1_12": lambda: di.make_elasticity3d(ne=12, box=3, overlap=1, p=2),
    "poisson3d_graph_rankdrop": lambda: di.make_poisson3d(N=10, box=2, overlap=1, p=2, seed=43, mode="graph"),
    "poisson2d_single_front": lambda: di.make_poisson2d(N=40, box=10, overlap=1, p=2, seed=44),
}

COND_A0 = {"biharmonic_128_box16": 1.56e6, "elasticity_q1_12": 1.09e4, "poisson3d_32_box4": 217.0}


def tol64(name, floor):
    return max(floor, COND_A0.get(name, 0.0) * 2.0 ** -52)


_cache = {}
ORDERS = ("nd", "band")


def setup(name, order="nd"):
    if (name, order) not in _cache:
        from paper_1504_00907_gb300 import ddg
        prob = CASES[name]()
        s = ddg.Solver.from_problem(prob, precision="fp64", keep=("fp64", "fp32"), coarse_order=order)
        oracle = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape,
                               dpn=prob.dofs_per_node)
        _cache[(name, order)] = (prob, s, oracle)
    return _cache[(name, order)]


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rhs(prob):
    return prob.f if prob.f.ndim == 1 else prob.f[:, 0]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", list(CASES))
def test_coarse_structure(name, order):
    prob, nd, oracle = setup(name, order)
    info = nd.info()
    assert info["n0"] == oracle.A0.shape[0]
    if order == "nd":
        assert info["coarse_order"] == 1
        assert info["coarse_fronts"] >= 1 and info["coarse_levels"] >= 1
        if name == "poisson3d_32_box4":
            assert info["coarse_levels"] >= 3
        # the default options take the ND ordering
        from paper_1504_00907_gb300 import ddg
        assert ddg.default_options().coarse_order == 1
    else:
        assert info["coarse_order"] == 0 and info["coarse_fronts"] == 0
    np.testing.assert_array_equal(nd.coarse_offsets(), oracle.coarse_offsets)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", list(CASES))
def test_coarse_correction_matches_oracle(name, order):
    prob, nd, oracle = setup(name, order)
    nd.set_precision("fp64")
    r = np.random.default_rng(45).standard_normal(prob.n)
    z = nd.coarse_correction(dev(r)).cpu().numpy()
    assert_close(z, oracle.coarse_correction(r), tol64(name, 1e-11))
    # and it is deterministic
    z2 = nd.coarse_correction(dev(r)).cpu().numpy()
    assert np.array_equal(z, z2)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", list(CASES))
def test_preconditioner_and_solve_match_oracle(name, order):
    prob, nd, oracle = setup(name, order)
    nd.set_precision("fp64")
    r = np.random.default_rng(46).standard_normal(prob.n)
    assert_close(nd.apply(dev(r)).cpu().numpy(), oracle.apply(r), tol64(name, 1e-11))
    f = rhs(prob)
    ref = orc.pcg(oracle.A, f, oracle.apply, tol=1e-8)
    u, iters, relres, st = nd.solve(dev(f), tol=1e-8)
    assert st == 0 and relres <= 1e-8 and abs(iters - ref.iters) <= 1
    assert_close(u.cpu().numpy(), ref.u, tol64(name, 1e-10))


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", ["poisson3d_32_box4", "biharmonic_128_box16", "elasticity_q1_12"])
def test_mixed_solve_matches_oracle(name, order):
    prob, nd, oracle = setup(name, order)
    f = rhs(prob)
    ref = orc.pcg(oracle.A, f, oracle.apply, tol=1e-8)
    nd.set_precision("fp32")
    u, iters, relres, st = nd.solve(dev(f), tol=1e-8)
    nd.set_precision("fp64")
    un = u.cpu().numpy()
    assert st == 0 and relres <= 1e-8
    assert np.linalg.norm(f - prob.A @ un) / np.linalg.norm(f) <= 1e-8
    assert_close(un, ref.u, 1e-7)
    assert iters <= ref.iters + 3


def test_nd_reproduces_generators_and_rebuilds_with_new_generators():
    # F restricted to each subdomain spans part of the coarse space, so the
    # coarse correction reproduces every generator column; ddg_set_generators
    # rebuilds the dissection for the new coarse space
    prob, nd, _ = setup("poisson3d_32_box4")
    nd.set_precision("fp64")
    for j in (0, 5, 9):
        Fj = prob.F[:, j]
        assert_close(nd.coarse_correction(dev(prob.A @ Fj)).cpu().numpy(), Fj, 1e-10)
    F1 = di.monomials(di.fd_node_coords(prob.shape), 1)
    nd.set_generators(F1)
    M1 = orc.DDGOracle(prob.A, prob.part, F1, prob.overlap, prob.overlap_mode, prob.shape)
    r = np.random.default_rng(47).standard_normal(prob.n)
    assert_close(nd.coarse_correction(dev(r)).cpu().numpy(), M1.coarse_correction(r), 1e-11)
    nd.set_generators(prob.F)
    _cache.pop(("poisson3d_32_box4", "nd"))


def test_persistent_and_per_level_nd_solves_agree():
    # the ND solve as one cooperative launch (grid barriers between levels)
    # and as one launch per level and direction: the same products, but the
    # per-level launches let several warps share a long row near the root
    # (their partial sums added in warp order), so the two agree to rounding
    # (FP64 1e-13, FP32 1e-6) and each is deterministic
    import os
    from paper_1504_00907_gb300 import ddg
    prob = CASES["poisson3d_32_box4"]()
    os.environ["DDG_ND_PERSISTENT"] = "1"
    try:
        a = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32"), coarse_order="nd")
    finally:
        del os.environ["DDG_ND_PERSISTENT"]
    b = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32"), coarse_order="nd")
    r = dev(np.random.default_rng(48).standard_normal(prob.n))
    for prec, tol in (("fp64", 1e-13), ("fp32", 1e-6)):
        a.set_precision(prec)
        b.set_precision(prec)
        za, zb = a.coarse_correction(r), b.coarse_correction(r)
        assert_close(za.cpu().numpy(), zb.cpu().numpy(), tol, label=prec)
        assert torch.equal(zb, b.coarse_correction(r)), prec
    ua, ita, _, sta = a.solve(dev(prob.f), tol=1e-8)
    ub, itb, _, stb = b.solve(dev(prob.f), tol=1e-8)
    assert sta == stb == 0 and abs(ita - itb) <= 1
    assert_close(ua.cpu().numpy(), ub.cpu().numpy(), 1e-7)
    a.close()
    b.close()


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name,m", [("poisson3d_32_box4", 8), ("biharmonic_128_box16", 5),
                                    ("elasticity_q1_12", 64), ("poisson3d_graph_rankdrop", 33)])
def test_batched_solve_matches_oracle_per_column(name, m, order):
    # the batched FP32 preconditioner runs the coarse solve on all m columns
    # at once (dof-major n0 x m vectors); m = 5 and 33 take the scalar
    # restriction, m = 64 fills both column halves of every ND lane
    prob, nd, oracle = setup(name, order)
    F = di.normal_rhs(prob.n, 60 + m, m)
    nd.set_precision("fp32")
    U, its, rrs, st = nd.solve_batch(dev(F), tol=1e-8)
    u0, it0, _, st0 = nd.solve(dev(F[:, 0]), tol=1e-8)
    nd.set_precision("fp64")
    assert st == 0 and st0 == 0 and np.all(rrs <= 1e-8)
    Un = U.cpu().numpy()
    for j in range(m):
        f = F[:, j]
        assert np.linalg.norm(f - prob.A @ Un[:, j]) / np.linalg.norm(f) <= 1e-8, j
    for j in sorted({0, m // 2, m - 1}):
        ref = orc.pcg(oracle.A, F[:, j], oracle.apply, tol=1e-8)
        assert_close(Un[:, j], ref.u, 1e-7, label=str(j))
        assert its[j] <= ref.iters + 3, (j, its[j], ref.iters)
    assert abs(int(its[0]) - it0) <= 1
    assert_close(Un[:, 0], u0.cpu().numpy(), 1e-7)


def test_nd_solve_many_batches_columns():
    # ddg_solve_many over ND handles: a multi-column problem goes through
    # the batched branch, a single column through the one-column branch
    from paper_1504_00907_gb300 import ddg
    probs = [CASES["poisson3d_32_box4"](), CASES["biharmonic_128_box16"]()]
    streams = [torch.cuda.Stream() for _ in probs]
    solvers = [ddg.Solver.from_problem(p, precision="fp32", keep=("fp32",), coarse_order="nd",
                                       stream=s.cuda_stream) for p, s in zip(probs, streams)]
    rhss = [dev(di.normal_rhs(probs[0].n, 71, 4)), dev(rhs(probs[1]))]
    torch.cuda.synchronize()
    outs, its, rrs, st = ddg.solve_many(solvers, rhss, tol=1e-8)
    torch.cuda.synchronize()
    assert st == 0 and np.all(rrs <= 1e-8) and len(its) == 5
    for p, f, u in zip(probs, rhss, outs):
        F = f.cpu().numpy().reshape(p.n, -1)
        Un = u.cpu().numpy().reshape(p.n, -1)
        M = orc.DDGOracle(p.A, p.part, p.F, p.overlap, p.overlap_mode, p.shape, dpn=p.dofs_per_node)
        for j in range(F.shape[1]):
            ref = orc.pcg(M.A, F[:, j], M.apply, tol=1e-8)
            assert_close(Un[:, j], ref.u, 1e-7, label=str(j))
    for s in solvers:
        s.close()

