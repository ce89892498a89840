"""Rebuilding the coarse space of a built handle (``ddg_set_generators``).

A handle whose generators are replaced must behave exactly like a handle
set up with the new generators from the start: the coarse build is the same
code on the same inputs, and the local inverses do not depend on the
generators.  So results are compared bitwise, and the original generators,
put back, reproduce the original results bitwise.
"""
import numpy as np
import pytest

import ddg_inputs as di

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _solver(prob, F, **kw):
    from paper_1504_00907_gb300 import ddg
    return ddg.Solver(prob.A, prob.part, F, prob.overlap, mode=prob.overlap_mode, shape=prob.shape,
                      stencil_kind=prob.stencil_kind, keep=("fp64", "fp32"), **kw)


def test_set_generators_equals_a_fresh_handle_and_round_trips():
    prob = di.make_poisson3d(N=24, box=8, overlap=1, p=2, seed=80)
    coords = di.fd_node_coords(prob.shape)
    F1 = di.monomials(coords, 1)
    s = _solver(prob, prob.F)
    r = dev(np.random.default_rng(81).standard_normal(prob.n))
    f = dev(prob.f)
    before = {p: (s.set_precision(p), s.apply(r))[1] for p in ("fp64", "fp32")}
    u_before, it_before, _, _ = s.solve(f, 1e-8)
    s.set_generators(F1)
    fresh = _solver(prob, F1)
    np.testing.assert_array_equal(s.coarse_offsets(), fresh.coarse_offsets())
    assert s.info()["n0"] == fresh.info()["n0"] == 27 * 4
    for p in ("fp64", "fp32"):
        s.set_precision(p)
        fresh.set_precision(p)
        assert torch.equal(s.apply(r), fresh.apply(r)), p
        ua, ita, rra, sta = s.solve(f, 1e-8)
        ub, itb, rrb, stb = fresh.solve(f, 1e-8)
        assert sta == stb == 0 and ita == itb and torch.equal(ua, ub), p
    # batched FP32 path: its workspace is resized for the new coarse space
    s.set_precision("fp32")
    fresh.set_precision("fp32")
    Fb = dev(di.normal_rhs(prob.n, 82, 4))
    Ua, ia, _, sa = s.solve_batch(Fb, 1e-8)
    Ub, ib, _, sb = fresh.solve_batch(Fb, 1e-8)
    assert sa == sb == 0 and np.array_equal(ia, ib) and torch.equal(Ua, Ub)
    fresh.close()
    # back to the original generators
    s.set_generators(prob.F)
    for p in ("fp64", "fp32"):
        s.set_precision(p)
        assert torch.equal(s.apply(r), before[p]), p
    s.set_precision("fp32")
    u_after, it_after, _, _ = s.solve(f, 1e-8)
    assert it_after == it_before and torch.equal(u_after, u_before)
    s.close()


def test_set_generators_turns_on_the_coarse_level():
    prob = di.make_poisson2d(N=48, box=12, overlap=1, p=2, seed=83)
    one = _solver(prob, prob.F, use_coarse=False)
    two = _solver(prob, prob.F)
    r = dev(np.random.default_rng(84).standard_normal(prob.n))
    one.set_precision("fp64")
    two.set_precision("fp64")
    z1 = one.apply(r)
    one.set_generators(prob.F)
    assert not torch.equal(one.apply(r), z1)
    assert torch.equal(one.apply(r), two.apply(r))
    one.close()
    two.close()


def test_set_generators_is_refused_on_a_vcycle_handle():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson2d(N=48, box=8, overlap=1, p=2, seed=85)
    s = ddg.Solver.from_problem(prob, precision="fp64",
                                coarse_groups=di.subdomain_groups(prob.shape, prob.box, 2))
    with pytest.raises(ddg.DDGError):
        s.set_generators(prob.F)
    s.close()
