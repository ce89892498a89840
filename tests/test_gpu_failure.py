"""Failure detection on the GPU, without a GPU fault.

* The tensor-core local solve's waits are bounded by the handle's
  spin_budget_ms.  With the DDG_DEBUG_TC_NO_COPIES hook its producer issues
  no copies, so the MMA thread waits on a barrier that nothing completes;
  the wait runs out, the kernel records the timeout, frees its tensor memory
  and returns, and the batched solve reports DDG_ETIMEOUT.  The same handle
  then solves normally.
* Calls from another host thread run on the handle's device.
* In-place solves (f and u the same buffer) are rejected.
"""
import threading

import numpy as np
import pytest

import ddg_inputs as di
from closeness import assert_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("kind", ["bf16", "tf32"])
def test_tensor_core_wait_runs_out_and_the_handle_recovers(kind):
    import time
    from paper_1504_00907_gb300 import ddg
    prob = di.make_varcoef3d(N=16, box=8, overlap=1, p=2, m=None)
    prec = "bf16" if kind == "bf16" else "fp32"
    s = ddg.Solver.from_problem(prob, precision=prec, keep=(prec,), tensor_cores=kind,
                                spin_budget_ms=20.0)
    F = dev(di.normal_rhs(prob.n, 70, 16))
    U_ref, its, rrs, st = s.solve_batch(F, tol=1e-8)
    assert st == ddg.DDG_OK and np.all(rrs <= 1e-8)
    s.set_debug(ddg.DDG_DEBUG_TC_NO_COPIES)
    t0 = time.perf_counter()
    with pytest.raises(ddg.DDGError) as e:
        s.solve_batch(F, tol=1e-8)
    elapsed = time.perf_counter() - t0
    assert e.value.status == ddg.DDG_ETIMEOUT
    assert "bounded wait" in str(e.value)
    # the first sweep's launches wait 20 ms each, then the solve stops
    assert elapsed < 30.0
    s.set_debug(0)
    U, its2, rrs2, st2 = s.solve_batch(F, tol=1e-8)
    assert st2 == ddg.DDG_OK and np.all(rrs2 <= 1e-8)
    assert np.array_equal(its, its2) and torch.equal(U, U_ref)
    s.close()


def test_calls_from_another_host_thread_use_the_handle_device():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson3d(N=16, box=8, overlap=1, p=2, seed=31)
    s = ddg.Solver.from_problem(prob, precision="fp32", keep=("fp32",))
    f = dev(prob.f)
    u0, it0, rr0, st0 = s.solve(f, tol=1e-8)
    torch.cuda.synchronize()
    out = {}

    def work():
        out["res"] = s.solve(f, tol=1e-8)

    t = threading.Thread(target=work)
    t.start()
    t.join()
    u1, it1, rr1, st1 = out["res"]
    torch.cuda.synchronize()
    assert st0 == st1 == ddg.DDG_OK and it0 == it1 and torch.equal(u0, u1)
    s.close()


def test_in_place_solve_is_rejected():
    from paper_1504_00907_gb300 import ddg
    prob = di.make_poisson2d(N=24, box=8, overlap=1, p=1, seed=32)
    s = ddg.Solver.from_problem(prob)
    f = dev(prob.f)
    with pytest.raises(ddg.DDGError) as e:
        s.solve(f, tol=1e-8, u=f)
    assert e.value.status == ddg.DDG_EINVAL and "alias" in str(e.value)
    u, it, rr, st = s.solve(f, tol=1e-8)
    assert st == ddg.DDG_OK
    assert_close(prob.A @ u.cpu().numpy(), prob.f, 1e-7)
    s.close()
