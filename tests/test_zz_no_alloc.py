"""ddg_spmv_dot_noalloc: the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc (a host framework's caching allocator
owns all device memory, a memory budget fixed at start-up, a caller inside
another library's critical section).  ddg_spmv_dot_noalloc computes y = A x
and x^T A x for a caller-owned CSR matrix with its scratch in a static
device array.  Here it is called through the C ABI twice in a row and
compared with the handle-based ddg_spmv (same arithmetic, so y must be
bit-identical) and with x . y for the reduction; the device's free memory
must not change across the two calls.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import ddg_inputs as di

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_handle_spmv_on_two_calls():
    from paper_1504_00907_gb300 import ddg
    lib = ddg.load()
    shape = (40, 40, 40)
    kappa = np.exp(di.gaussian_random_field(shape, 0.1, 1.0, 2))
    A, _ = di.varcoef7_3d(kappa)
    n = A.shape[0]
    assert n <= ddg_max_rows()
    # handle-based reference on the generic CSR path (no stencil kind)
    part = di.box_partition(shape, (8, 8, 8))
    F = di.monomials(di.cell_centre_coords(shape), 1)
    solver = ddg.Solver(A, part, F, 1, mode="box", shape=shape, stencil_kind=0)
    rowptr, col, val = di.csr_arrays(A)
    dev = "cuda"
    d_rowptr = torch.tensor(rowptr, device=dev)
    d_col = torch.tensor(col, device=dev)
    d_val = torch.tensor(val, device=dev)
    rng = np.random.default_rng(31)
    xs = [torch.tensor(rng.standard_normal(n), dtype=torch.float64, device=dev) for _ in range(2)]
    ys = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    dots = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in range(2)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(x, y, d):
        return lib.ddg_spmv_dot_noalloc(n, _ptr(d_rowptr), _ptr(d_col), _ptr(d_val), _ptr(x),
                                        _ptr(y), _ptr(d), stream)

    # the first call on a device looks up the scratch array (module load)
    assert call(xs[0], ys[0], dots[0]) == ddg.DDG_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for x, y, d in zip(xs, ys, dots):
        assert call(x, y, d) == ddg.DDG_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for x, y, d in zip(xs, ys, dots):
        y_ref = solver.spmv(x)
        assert torch.equal(y, y_ref)
        ref = torch.dot(x, y_ref).item()
        assert abs(d.item() - ref) <= 1e-12 * abs(ref)
    solver.close()


def ddg_max_rows():
    import re
    from paper_1504_00907_gb300 import ddg
    text = open(ddg.HEADER).read()
    return int(re.search(r"#define DDG_NOALLOC_MAX_ROWS (\d+)", text).group(1))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1504_00907_gb300 import ddg
    lib = ddg.load()
    big = ddg_max_rows() + 1
    st = lib.ddg_spmv_dot_noalloc(big, None, None, None, None, None, None, None)
    assert st == ddg.DDG_EINVAL
    assert b"DDG_NOALLOC_MAX_ROWS" in lib.ddg_last_error(None)
