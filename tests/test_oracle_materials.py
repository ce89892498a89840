"""Material-aware generators (Sec. 7, problem C), oracle pins on the CPU.

The generators [F(1-J), FJ] split every monomial at the material boundary
(J the indicator of the second material).  What fixes the resulting coarse
space independently of the QR code:

* a subdomain inside one material keeps exactly the k plain generators;
  a subdomain that meets both materials gains at least one more and at most
  k more (each material's part contributes its own polynomials);
* the split space contains the plain one (F(1-J) + FJ = F), so the coarse
  correction reproduces every plain generator column;
* the paper reports fewer iterations with the material-aware space for
  piecewise cubics; the structured stand-in (minimal overlap, p = 3) shows
  the same direction.
"""
import numpy as np

import ddg_inputs as di
from oracle import ddg_oracle as orc


def _oracle(prob):
    return orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape)


def test_two_material_coefficient_values():
    coords = np.array([[0.0, 0.0, 0.3], [0.5, 0.25, 0.9], [1.0, 0.0, 0.1]])
    D, J = di.two_material_coefficient(coords)
    # cos(0) cos(0) = 1 -> J = 1; cos(pi/2) = 0 -> 0.25 > 0 -> J = 1;
    # cos(pi) cos(0) = -1 -> J = 0
    np.testing.assert_array_equal(J, [1.0, 1.0, 0.0])
    S = np.exp(1.0 + np.sin(np.pi * (coords[:, 0] + coords[:, 1])))
    np.testing.assert_allclose(D, S + 100.0 * J, rtol=1e-15)


def test_ranks_follow_the_material_count_per_subdomain():
    prob = di.make_twomaterial3d(N=16, box=4, overlap=0, p=2, material_aware=True, mode="graph")
    k = 10
    assert prob.F.shape[1] == 2 * k
    M = _oracle(prob)
    ranks = np.diff(M.coarse_offsets)
    _, J = di.two_material_coefficient(di.cell_centre_coords(prob.shape))
    mixed = 0
    for s in range(prob.nsub):
        mats = np.unique(J[prob.part == s])
        if mats.size == 1:
            assert ranks[s] == k, s
        else:
            mixed += 1
            assert k < ranks[s] <= 2 * k, (s, ranks[s])
    assert 0 < mixed < prob.nsub


def test_split_space_reproduces_plain_generators():
    plain = di.make_twomaterial3d(N=16, box=4, overlap=1, p=2, material_aware=False, mode="graph")
    aware = di.make_twomaterial3d(N=16, box=4, overlap=1, p=2, material_aware=True, mode="graph")
    np.testing.assert_array_equal(aware.F[:, :10] + aware.F[:, 10:], plain.F)
    M = _oracle(aware)
    for j in (0, 4, 9):
        Fj = plain.F[:, j]
        z = M.coarse_correction(aware.A @ Fj)
        assert np.linalg.norm(z - Fj) <= 1e-9 * np.linalg.norm(Fj), j


def test_material_aware_cubics_need_fewer_iterations():
    # 2D as in the paper's problem C: 128^2 cells, 16^2 boxes, overlap 0
    its = []
    for aware in (False, True):
        prob = di.make_twomaterial2d(N=128, box=16, overlap=0, p=3, material_aware=aware)
        assert prob.F.shape[1] == (20 if aware else 10)
        res = orc.pcg(prob.A, prob.f, _oracle(prob).apply, tol=1e-8)
        assert res.converged
        its.append(res.iters)
    assert its[1] < its[0], its


def test_varcoef5_unit_coefficient_is_cell_centred_laplacian():
    N = 5
    A = di.varcoef5_2d(np.ones((N, N))).toarray()
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    i, j = i.ravel(), j.ravel()
    # interior faces 1, boundary faces 2 (half-cell distance to the wall)
    nb = ((i == 0).astype(int) + (i == N - 1) + (j == 0) + (j == N - 1))
    np.testing.assert_array_equal(np.diag(A), 4 + nb)
    assert np.allclose(A, A.T)
    np.testing.assert_array_equal(A[0, 1], -1.0)
