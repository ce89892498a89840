"""Banded local factors (exact local solves of Sec. 6 for large blocks).

Local blocks of more than 3072 dofs are solved through the banded Cholesky
factor of A_i in block form (local_repr BAND, chosen automatically there);
the same path can be forced on small blocks.  The oracle solves each local
block by a dense Cholesky factorisation, so the comparison checks the band
assembly, the batched band factorisation, the block-form rewrite and the
streamed recurrences together.

Tolerances: FP64 preconditioner 1e-11 (the blocks here have cond(A_i) up to
1.1e4, so rounding stays near cond u = 2.5e-12); FP64 PCG solution 1e-10
with iterations within 1.  FP32 factors: solving A_i x = r through FP32 L
and L^T carries a relative error of order cond(A_i) 2^-24, so the FP32
preconditioner bound is max(1e-5, cond_max 2^-24) with cond_max the largest
condition number of the case's local blocks (numpy eigvalsh of the blocks;
for the two large cases computed once: 1818.7 for the 66^2 Poisson blocks,
130.6 for the 17^3 ones).  Mixed solves reach the true residual 1e-8 with
solutions within 1e-7 of the oracle's.
"""
import numpy as np
import pytest

import ddg_inputs as di
from closeness import assert_close
from oracle import ddg_oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# blocks above the dense-inverse limit: 2D 128^2 with 64^2 boxes + overlap 2
# (66^2 = 4356 dofs, half-bandwidth 66) and 3D 32^3 with 16^3 boxes +
# overlap 1 (17^3 = 4913 dofs, half-bandwidth 289: five tiles per super-block)
LARGE = {
    "poisson2d_band_4356": lambda: di.make_poisson2d(N=128, box=64, overlap=2, p=2, seed=8),
    "poisson3d_band_4913": lambda: di.make_poisson3d(N=32, box=16, overlap=1, p=2, seed=9),
}
# small blocks with the band path forced: 5-point, 13-point (overlap 2, two
# rows of coupling), variable-coefficient 7-point and Q1 elasticity (3 dofs
# per node interleaved)
SMALL = {
    "poisson2d_64": lambda: di.make_poisson2d(N=64, box=16, overlap=2, p=2, seed=0),
    "biharmonic_64": lambda: di.make_biharmonic2d(N=64, box=16, overlap=2, p=3, seed=100),
    "varcoef_16": lambda: di.make_varcoef3d(N=16, box=8, overlap=1, p=2, m=None),
    "elasticity_q1_6": lambda: di.make_elasticity3d(ne=6, box=3, overlap=1, p=2),
}

_cache = {}


def setup(name):
    if name not in _cache:
        from paper_1504_00907_gb300 import ddg
        make = LARGE.get(name) or SMALL[name]
        prob = make()
        repr_ = "auto" if name in LARGE else "band"
        solver = ddg.Solver.from_problem(prob, precision="fp64", keep=("fp64", "fp32"), local_repr=repr_)
        oracle = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape,
                               dpn=prob.dofs_per_node)
        _cache[name] = (prob, solver, oracle)
    return _cache[name]


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rhs(prob):
    return prob.f if prob.f.ndim == 1 else prob.f[:, 0]


@pytest.mark.parametrize("name", list(LARGE))
def test_large_blocks_choose_the_band(name):
    prob, solver, oracle = setup(name)
    info = solver.info()
    assert info["local_repr"] == 2 and info["max_local"] > 3072
    # the half-bandwidth of the largest block in ascending dof order
    idx = max(oracle.omega, key=len)
    Ai = prob.A[idx][:, idx].tocoo()
    assert info["local_band"] == int(np.max(np.abs(Ai.row - Ai.col)))
    np.testing.assert_array_equal(solver.colouring(), oracle.colour)


LARGE_COND = {"poisson2d_band_4356": 1818.7, "poisson3d_band_4913": 130.6}


def cond_max(name, prob, oracle):
    if name in LARGE_COND:
        return LARGE_COND[name]
    worst = 0.0
    for idx in oracle.omega:
        w = np.linalg.eigvalsh(prob.A[idx][:, idx].toarray())
        worst = max(worst, w[-1] / w[0])
    return worst


@pytest.mark.parametrize("name", list(LARGE) + list(SMALL))
def test_band_preconditioner_matches_oracle(name):
    prob, solver, oracle = setup(name)
    r = np.random.default_rng(21).standard_normal(prob.n)
    ref = oracle.apply(r)
    solver.set_precision("fp64")
    assert_close(solver.apply(dev(r)).cpu().numpy(), ref, 1e-11, "fp64")
    solver.set_precision("fp32")
    tol32 = max(1e-5, cond_max(name, prob, oracle) * 2.0 ** -24)
    assert_close(solver.apply(dev(r)).cpu().numpy(), ref, tol32, "fp32")
    solver.set_precision("fp64")


@pytest.mark.parametrize("name", ["poisson2d_band_4356", "biharmonic_64", "elasticity_q1_6"])
def test_band_solve_fp64_matches_oracle(name):
    prob, solver, oracle = setup(name)
    f = rhs(prob)
    ref = orc.pcg(oracle.A, f, oracle.apply, tol=1e-8)
    solver.set_precision("fp64")
    u, iters, relres, st = solver.solve(dev(f), tol=1e-8)
    assert st == 0 and relres <= 1e-8 and abs(iters - ref.iters) <= 1
    assert_close(u.cpu().numpy(), ref.u, 1e-10)


@pytest.mark.parametrize("name", list(LARGE) + ["biharmonic_64"])
def test_band_solve_mixed_matches_oracle(name):
    prob, solver, oracle = setup(name)
    f = rhs(prob)
    ref = orc.pcg(oracle.A, f, oracle.apply, tol=1e-8)
    solver.set_precision("fp32")
    u, iters, relres, st = solver.solve(dev(f), tol=1e-8)
    solver.set_precision("fp64")
    un = u.cpu().numpy()
    assert st == 0 and relres <= 1e-8
    assert np.linalg.norm(f - prob.A @ un) / np.linalg.norm(f) <= 1e-8
    assert_close(un, ref.u, 1e-7)
    assert iters <= ref.iters + 3


def test_band_equals_inverse_path_to_rounding_and_is_deterministic():
    from paper_1504_00907_gb300 import ddg
    prob, band, _ = setup("poisson2d_64")
    inv = ddg.Solver.from_problem(prob, precision="fp64", keep=("fp64",), local_repr="inv")
    r = dev(np.random.default_rng(22).standard_normal(prob.n))
    band.set_precision("fp64")
    za, zb = band.apply(r), band.apply(r)
    assert torch.equal(za, zb)
    assert_close(za.cpu().numpy(), inv.apply(r).cpu().numpy(), 1e-12)
    assert inv.info()["local_repr"] == 1
    inv.close()


def test_band_batch_runs_column_by_column():
    prob, solver, oracle = setup("biharmonic_64")
    solver.set_precision("fp32")
    F = di.normal_rhs(prob.n, 23, 3)
    U, its, rrs, st = solver.solve_batch(dev(F), tol=1e-8)
    solver.set_precision("fp64")
    assert st == 0 and np.all(rrs <= 1e-8)
    for j in range(3):
        f = F[:, j]
        assert np.linalg.norm(f - prob.A @ U[:, j].cpu().numpy()) / np.linalg.norm(f) <= 1e-8


def test_band_rejects_dense_only_options():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson2d(N=32, box=16, overlap=1, p=1)
    with pytest.raises(ddg.DDGError) as e:
        ddg.Solver.from_problem(prob, local_repr="band", tensor_cores=True, precision="bf16", keep=("bf16",))
    assert e.value.status == ddg.DDG_EINVAL
    with pytest.raises(ddg.DDGError):
        ddg.Solver.from_problem(di.make_poisson2d(N=128, box=64, overlap=2, p=2), local_repr="inv")
