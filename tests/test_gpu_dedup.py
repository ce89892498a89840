"""Shared inverses of identical local matrices (``dedup_local``) on the GPU.

Sharing changes where an inverse is stored, not what is computed: equal
local matrices give equal inverses (the factorisation is deterministic), so
every result must be bitwise equal to the handle without sharing.  The
number of distinct local matrices is counted independently here by
comparing the dense blocks A[ov_i, ov_i] of the oracle's overlapping
subdomains.
"""
import numpy as np
import pytest

import ddg_inputs as di
from oracle import ddg_oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def distinct_local_matrices(prob):
    M = orc.DDGOracle(prob.A, prob.part, prob.F, prob.overlap, prob.overlap_mode, prob.shape)
    Ad = prob.A.tocsr()
    keys = set()
    for idx in M.omega:
        blk = Ad[idx, :][:, idx].toarray()
        keys.add((blk.shape, blk.tobytes()))
    return len(keys)


CASES = {
    # 5^3 boxes of 8^3 + overlap 1: per axis a 9-wide block at either end and
    # 10-wide ones inside, so 2^3 distinct local matrices
    "poisson3d_40": lambda: di.make_poisson3d(N=40, box=8, overlap=1, p=2, seed=70),
    "poisson2d_ragged": lambda: di.make_poisson2d(N=50, box=16, overlap=2, p=2, seed=71),
    # variable coefficients: no two local matrices agree
    "varcoef_16": lambda: di.make_varcoef3d(N=16, box=4, overlap=1, p=2, m=None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dedup_is_bitwise_neutral(name):
    from paper_1504_00907_gb300 import ddg
    prob = CASES[name]()
    a = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32"))
    b = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp64", "fp32"), dedup_local=True)
    ia, ib = a.info(), b.info()
    assert ia["local_inverses"] == prob.nsub
    assert ib["local_inverses"] == distinct_local_matrices(prob)
    if name == "poisson3d_40":
        assert ib["local_inverses"] == 8 and ib["local_tiles"] < ia["local_tiles"] / 10
    r = dev(np.random.default_rng(72).standard_normal(prob.n))
    f = dev(prob.f if prob.f.ndim == 1 else prob.f[:, 0])
    for prec in ("fp64", "fp32"):
        a.set_precision(prec)
        b.set_precision(prec)
        assert torch.equal(a.apply(r), b.apply(r)), prec
        ua, ita, rra, sta = a.solve(f, 1e-8)
        ub, itb, rrb, stb = b.solve(f, 1e-8)
        assert sta == stb == 0 and ita == itb and rra == rrb
        assert torch.equal(ua, ub), prec
    a.close()
    b.close()


def test_dedup_tensor_core_batch_is_bitwise_neutral():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson3d(N=40, box=8, overlap=1, p=2, seed=73)
    F = dev(di.normal_rhs(prob.n, 74, 16))
    out = []
    for dd in (False, True):
        s = ddg.Solver.from_problem(prob, precision="bf16", keep=("bf16",), tensor_cores=True,
                                    dedup_local=dd)
        U, its, rrs, st = s.solve_batch(F, 1e-8)
        assert st == 0
        out.append((U, its))
        s.close()
    assert torch.equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
