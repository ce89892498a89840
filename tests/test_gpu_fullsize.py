"""Checks at the benchmark's full sizes, in the benchmark's launch configuration.

The CPU oracle cannot run these sizes in seconds, so every check here is a
property that holds at any size, evaluated independently of the CUDA path
(scipy sparse products on the CPU, closed forms):

* 3D Poisson 128^3 (8^3 boxes + overlap 1, p <= 2, coarse dimension 40960):
  the greedy colouring is the lattice colouring; every subdomain keeps all
  10 generators; the coarse correction R0^T A0^{-1} R0 A reproduces every
  generator column (it is the A-orthogonal projection onto span R0^T); the
  FP64 preconditioner is symmetric and positive; FP32, BF16 and FP64 solves
  reach a true relative residual of 1e-8 measured with scipy.
* variable-coefficient 96^3 with 64 right-hand sides on the tensor-core
  path: every column reaches 1e-8 (scipy residual) and matches the
  single-column FP32 solve.
* Q1 elasticity on 64^3 elements: forward and adjoint solves reach 1e-8
  (scipy residuals); sampled entries of dL/dmu equal -lambda_e^T K^mu u_e
  recomputed on the CPU from the element matrices.
* the three-level V-cycle on Poisson 128^3 (4^3 subdomains per
  coarse-level subdomain) reaches 1e-8 (scipy residual).
"""
import numpy as np
import pytest

import ddg_inputs as di
from closeness import assert_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def true_rel(A, u, f):
    return np.linalg.norm(f - A @ u) / np.linalg.norm(f)


@pytest.fixture(scope="module")
def poisson128():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson3d(N=128, box=8, overlap=1, p=2, seed=1)
    s = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32", "bf16"))
    yield prob, s
    s.close()


def test_poisson128_colouring_and_coarse_ranks(poisson128):
    prob, s = poisson128
    nb = 16
    ix, iy, iz = np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij")
    lattice = (ix % 2 + 2 * (iy % 2) + 4 * (iz % 2)).transpose(2, 1, 0).ravel()
    np.testing.assert_array_equal(s.colouring(), lattice)
    np.testing.assert_array_equal(s.coarse_offsets(), 10 * np.arange(nb ** 3 + 1))


def test_poisson128_coarse_correction_reproduces_generators(poisson128):
    prob, s = poisson128
    s.set_precision("fp64")
    for j in (0, 3, 9):
        Fj = prob.F[:, j]
        z = s.coarse_correction(dev(prob.A @ Fj)).cpu().numpy()
        assert_close(z, Fj, 1e-9, label=str(j))
    s.set_precision("fp32")


def test_poisson128_preconditioner_symmetric_positive(poisson128):
    prob, s = poisson128
    s.set_precision("fp64")
    rng = np.random.default_rng(30)
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    Mx, My = s.apply(dev(x)).cpu().numpy(), s.apply(dev(y)).cpu().numpy()
    assert abs(x @ My - y @ Mx) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(My)
    assert x @ Mx > 0 and y @ My > 0
    s.set_precision("fp32")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64"])
def test_poisson128_solve_reaches_true_residual(poisson128, prec):
    from paper_1504_00907_gb300 import ddg
    prob, s = poisson128
    s.set_precision(prec)
    u, it, rr, st = s.solve(dev(prob.f), tol=1e-8)
    s.set_precision("fp32")
    assert st == ddg.DDG_OK and it <= 8
    r = true_rel(prob.A, u.cpu().numpy(), prob.f)
    assert r <= 1e-8 and abs(r - rr) <= 1e-3 * r


def test_varcoef96_batched_tensor_core_all_columns():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_varcoef3d(N=96, box=8, overlap=1, p=2, m=64)
    s = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp32", "bf16"), tensor_cores=True)
    F = dev(prob.f)
    s.set_precision("bf16")
    U, its, rrs, st = s.solve_batch(F, 1e-8)
    assert st == ddg.DDG_OK and its.max() <= 8
    Uc = U.cpu().numpy()
    R = prob.f - prob.A @ Uc
    col_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(prob.f, axis=0)
    assert col_rel.max() <= 1e-8
    s.set_precision("fp32")
    for j in (0, 37):
        u, it, rr, st1 = s.solve(F[:, j].contiguous(), 1e-8)
        assert st1 == ddg.DDG_OK and rel(Uc[:, j], u.cpu().numpy()) <= 1e-6
    s.close()


def test_elasticity64_forward_adjoint_and_sampled_gradient():
    from paper_1504_00907_gb300 import ddg
    ne = 64
    prob = di.make_elasticity3d(ne=ne)
    s = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32"))
    u, it, rr, st = s.solve(dev(prob.f), 1e-8)
    assert st == ddg.DDG_OK
    uc = u.cpu().numpy()
    assert true_rel(prob.A, uc, prob.f) <= 1e-8
    g = uc - prob.target
    lam, ita, rra, _ = s.adjoint(dev(g), 1e-8)
    lc = lam.cpu().numpy()
    assert true_rel(prob.A, lc, g) <= 1e-8
    dmu = s.grad_coeff(lam, u).cpu().numpy()
    s.close()
    # -lambda_e^T K^mu u_e for sampled elements, clamped dofs (x = 0 face) as 0
    _, Km = di.q1_reference_stiffness()
    Km = Km / ne
    rng = np.random.default_rng(31)
    sample = np.concatenate([rng.integers(0, ne ** 3, 40), [0, ne - 1, ne ** 3 - 1]])
    for e in sample:
        ei, ej, ek = e % ne, (e // ne) % ne, e // (ne * ne)
        le, ue = np.zeros(24), np.zeros(24)
        for a in range(8):
            I, J, K = ei + (a & 1), ej + ((a >> 1) & 1), ek + (a >> 2)
            if I >= 1:
                base = 3 * ((I - 1) + ne * (J + (ne + 1) * K))
                le[3 * a:3 * a + 3] = lc[base:base + 3]
                ue[3 * a:3 * a + 3] = uc[base:base + 3]
        ref = -le @ Km @ ue
        assert abs(dmu[e] - ref) <= 1e-10 * max(abs(ref), 1e-300) + 1e-14 * np.abs(dmu).max(), e


def test_poisson128_vcycle_reaches_true_residual():
    # three-level V-cycle with 4^3 subdomains per coarse-level subdomain
    # (64 of them, about 1600 coarse dofs each with their overlap)
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson3d(N=128, box=8, overlap=1, p=2, seed=1)
    groups = di.subdomain_groups(prob.shape, prob.box, 4)
    s = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp32",), coarse_groups=groups)
    u, it, rr, st = s.solve(dev(prob.f), tol=1e-8)
    s.close()
    assert st == ddg.DDG_OK and it <= 12
    r = true_rel(prob.A, u.cpu().numpy(), prob.f)
    assert r <= 1e-8 and abs(r - rr) <= 1e-3 * r
