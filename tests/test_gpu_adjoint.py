"""Adjoint solve and coefficient gradient (the differentiation workload) on the GPU.

Loss L(u) = 0.5 ||u - u_t||^2 with u = A(kappa)^{-1} f for the cell-centred
variable-coefficient operator.  The GPU gradient (adjoint PCG through the
library + ddg_grad_coeff) is checked against central finite differences of
dense direct solves (numpy, no GPU) and against the dense adjoint formula;
the torch autograd wrapper must give the same numbers.
"""
import numpy as np
import pytest

import ddg_inputs as di

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 6


def _problem():
    kappa = np.exp(di.gaussian_random_field((N, N, N), 0.15, 1.0, 4))
    A, _ = di.varcoef7_3d(kappa)
    f = di.normal_rhs(A.shape[0], 5)
    ut = di.normal_rhs(A.shape[0], 6)
    return kappa, A, f, ut


def _loss_dense(kappa, f, ut):
    A, _ = di.varcoef7_3d(kappa)
    u = np.linalg.solve(A.toarray(), f)
    return 0.5 * np.sum((u - ut) ** 2)


def _solver(kappa, A, precision="fp64"):
    from paper_1504_00907_gb300 import ddg
    shape = (N, N, N)
    part = di.box_partition(shape, (3, 3, 3))
    F = di.monomials(di.cell_centre_coords(shape), 1)
    return ddg.Solver(A, part, F, 1, mode="box", shape=shape, stencil_kind=di.STENCIL_VAR7_3D,
                      coef=kappa, precision=precision, keep=("fp64", "fp32"))


def test_gradient_matches_central_differences():
    kappa, A, f, ut = _problem()
    s = _solver(kappa, A)
    fd_ = torch.tensor(f, dtype=torch.float64, device="cuda")
    u, it, rr, st = s.solve(fd_, tol=1e-13)
    assert st == 0
    g = u - torch.tensor(ut, dtype=torch.float64, device="cuda")
    lam, _, _, _ = s.adjoint(g.contiguous(), tol=1e-13)
    dk = s.grad_coeff(lam, u).cpu().numpy()
    # central differences of the dense-solve loss, relative step 1e-6
    fd = np.zeros(kappa.size)
    kf = kappa.ravel()
    for j in range(kappa.size):
        h = 1e-6 * kf[j]
        kp = kf.copy(); kp[j] += h
        km = kf.copy(); km[j] -= h
        fd[j] = (_loss_dense(kp.reshape(kappa.shape), f, ut)
                 - _loss_dense(km.reshape(kappa.shape), f, ut)) / (2 * h)
    assert np.linalg.norm(dk - fd) <= 1e-5 * np.linalg.norm(fd)
    # dL/df = lambda, against the dense adjoint A^{-1} (u - u_t)
    Ad = A.toarray()
    lam_ref = np.linalg.solve(Ad, np.linalg.solve(Ad, f) - ut)
    assert np.linalg.norm(lam.cpu().numpy() - lam_ref) <= 1e-10 * np.linalg.norm(lam_ref)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autograd_function(precision):
    from paper_1504_00907_gb300 import ddg
    kappa, A, f, ut = _problem()
    s = _solver(kappa, A, precision)
    k_t = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
    f_t = torch.tensor(f, dtype=torch.float64, device="cuda", requires_grad=True)
    u = ddg.solve_autograd(s, k_t, f_t, tol=1e-12)
    loss = 0.5 * ((u - torch.tensor(ut, dtype=torch.float64, device="cuda")) ** 2).sum()
    loss.backward()
    Ad = A.toarray()
    u_ref = np.linalg.solve(Ad, f)
    lam_ref = np.linalg.solve(Ad, u_ref - ut)
    assert np.linalg.norm(f_t.grad.cpu().numpy() - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    # dense adjoint formula for dL/dkappa on the same discretisation
    kf = kappa.ravel()
    ref = np.zeros(kf.size)
    h = 1e-6
    for j in range(kf.size):
        kp = kf.copy(); kp[j] *= 1 + h
        km = kf.copy(); km[j] *= 1 - h
        dA = (di.varcoef7_3d(kp.reshape(kappa.shape))[0] - di.varcoef7_3d(km.reshape(kappa.shape))[0]) / (2 * h * kf[j])
        ref[j] = -lam_ref @ (dA @ u_ref)
    got = k_t.grad.cpu().numpy().ravel()
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    s.close()


def test_q1_elasticity_mu_gradient_matches_central_differences():
    # the Q1 elasticity differentiation workload on a 6^3-element copy: loss
    # L = 0.5 ||u - u_t||^2, u = A(mu)^{-1} b; dL/dmu_e by the adjoint solve
    # and ddg_grad_coeff against central differences of dense solves
    from paper_1504_00907_gb300 import ddg
    prob = di.make_elasticity3d(ne=6, box=3, overlap=1, p=2)
    mu = prob.kappa
    s = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32"))
    b = torch.tensor(prob.f, dtype=torch.float64, device="cuda")
    ut = torch.tensor(prob.target, dtype=torch.float64, device="cuda")
    u, it, rr, st = s.solve(b, tol=1e-13)
    assert st == 0
    lam, _, _, _ = s.adjoint((u - ut).contiguous(), tol=1e-13)
    dmu = s.grad_coeff(lam, u).cpu().numpy()

    def loss(m):
        A, _ = di.elasticity_q1_3d(m)
        x = np.linalg.solve(A.toarray(), prob.f)
        return 0.5 * np.sum((x - prob.target) ** 2)

    fd = np.zeros(mu.size)
    mf = mu.ravel()
    for e in range(mu.size):
        h = 1e-6 * mf[e]
        mp = mf.copy(); mp[e] += h
        mm = mf.copy(); mm[e] -= h
        fd[e] = (loss(mp.reshape(mu.shape)) - loss(mm.reshape(mu.shape))) / (2 * h)
    assert np.linalg.norm(dmu - fd) <= 1e-5 * np.linalg.norm(fd)
    # torch autograd through the same solver: d loss / d log mu = mu * dL/dmu
    mu_t = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    b_t = b.clone().requires_grad_(True)
    uu = ddg.solve_autograd(s, mu_t, b_t, tol=1e-13)
    (0.5 * ((uu - ut) ** 2).sum()).backward()
    g = mu_t.grad.cpu().numpy().ravel()
    assert np.linalg.norm(g - fd) <= 1e-5 * np.linalg.norm(fd)
    dlogmu = mf * g
    assert np.linalg.norm(dlogmu - mf * fd) <= 1e-5 * np.linalg.norm(mf * fd)
    s.close()


def test_autograd_rejects_coefficients_that_differ_from_the_handle():
    # the handle's matrix is built from the coefficients given at setup: a
    # kappa with other values must not silently get the old matrix's answer
    from paper_1504_00907_gb300 import ddg
    kappa, A, f, _ = _problem()
    s = _solver(kappa, A)
    f_t = torch.tensor(f, dtype=torch.float64, device="cuda", requires_grad=True)
    changed = torch.tensor(kappa * 1.01, dtype=torch.float64, device="cuda", requires_grad=True)
    with pytest.raises(ValueError):
        ddg.solve_autograd(s, changed, f_t)
    same = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
    u = ddg.solve_autograd(s, same, f_t, tol=1e-10)
    assert u.shape == f_t.shape
    s.close()


def test_autograd_backward_raises_when_the_adjoint_does_not_converge():
    # a failing adjoint solve is planted on the host (the binding's adjoint
    # returns DDG_ENOCONV): the backward must raise, not return the
    # unconverged lambda as dL/df
    from paper_1504_00907_gb300 import ddg
    kappa, A, f, _ = _problem()
    s = _solver(kappa, A)
    real = s.adjoint

    def unconverged(g, tol=1e-8):
        lam, it, rr, _ = real(g, tol)
        return lam, it, rr, ddg.DDG_ENOCONV

    s.adjoint = unconverged
    k_t = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
    f_t = torch.tensor(f, dtype=torch.float64, device="cuda", requires_grad=True)
    u = ddg.solve_autograd(s, k_t, f_t, tol=1e-10)
    with pytest.raises(ddg.DDGError) as e:
        (u * u).sum().backward()
    assert e.value.status == ddg.DDG_ENOCONV
    s.close()
