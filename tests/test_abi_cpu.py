"""The C-ABI library loads, exports every declared symbol, and its structs
match the binding; argument validation works without a GPU."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_00907_gb300 import build, ddg
    if not os.path.exists(ddg.LIB_PATH):
        build.build()
    return ddg.load()


def test_every_declared_function_is_exported(lib):
    from paper_1504_00907_gb300 import ddg
    names = ddg.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(ddg._SIGS), "binding and header disagree"


def test_struct_layouts_match_header(tmp_path):
    from paper_1504_00907_gb300 import ddg
    src = tmp_path / "lay.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "ddg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(ddg_options), offsetof(ddg_options, rank_tol),
         offsetof(ddg_options, chunk_tiles), offsetof(ddg_options, tensor_cores), sizeof(ddg_matrix));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(ddg_matrix, coef), sizeof(ddg_info), offsetof(ddg_info, setup_ms),
         offsetof(ddg_info, local_inverses), offsetof(ddg_options, dedup_local),
         offsetof(ddg_options, spin_budget_ms), offsetof(ddg_info, graph_solve));
  printf("%zu %zu %zu %zu\\n", offsetof(ddg_options, autotune), offsetof(ddg_info, tuned),
         offsetof(ddg_options, local_repr), offsetof(ddg_info, local_elems));
  printf("%zu %zu\\n", offsetof(ddg_options, coarse_order), offsetof(ddg_info, coarse_elems));
  return 0;
}
""")
    exe = tmp_path / "lay"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    got = [int(x) for x in out]
    exp = [ctypes.sizeof(ddg.Options), ddg.Options.rank_tol.offset, ddg.Options.chunk_tiles.offset,
           ddg.Options.tensor_cores.offset, ctypes.sizeof(ddg.Matrix), ddg.Matrix.coef.offset, ctypes.sizeof(ddg.Info),
           ddg.Info.setup_ms.offset, ddg.Info.local_inverses.offset, ddg.Options.dedup_local.offset,
           ddg.Options.spin_budget_ms.offset, ddg.Info.graph_solve.offset,
           ddg.Options.autotune.offset, ddg.Info.tuned.offset, ddg.Options.local_repr.offset,
           ddg.Info.local_elems.offset, ddg.Options.coarse_order.offset, ddg.Info.coarse_elems.offset]
    assert got == exp


def test_defaults_and_status_strings(lib):
    from paper_1504_00907_gb300 import ddg
    o = ddg.default_options()
    assert (o.precision, o.maxit, o.use_coarse, o.rank_tol) == (0, 1000, 1, 1e-10)
    assert o.spin_budget_ms == 1000.0
    assert o.coarse_order == ddg.COARSE["nd"]
    assert lib.ddg_status_string(ddg.DDG_ENOTSPD) == b"DDG_ENOTSPD"


def _matrix(rowptr, col, val):
    from paper_1504_00907_gb300 import ddg
    m = ddg.Matrix()
    m.n = len(rowptr) - 1
    m.rowptr = rowptr.ctypes.data_as(ctypes.c_void_p)
    m.col = col.ctypes.data_as(ctypes.c_void_p)
    m.val = val.ctypes.data_as(ctypes.c_void_p)
    return m


@pytest.mark.parametrize("case", ["neg_part", "col_range", "k_zero", "box_shape", "tc_kind"])
def test_setup_rejects_bad_arguments_before_touching_the_gpu(lib, case):
    from paper_1504_00907_gb300 import ddg
    import ddg_inputs as di
    A = di.poisson5_2d(4)
    rowptr, col, val = di.csr_arrays(A)
    part = np.zeros(16, dtype=np.int32)
    F = np.ones(16)
    k = 1
    o = ddg.default_options()
    if case == "neg_part":
        part[3] = -1
    if case == "col_range":
        col = col.copy()
        col[5] = 99
    if case == "k_zero":
        k = 0
    m = _matrix(rowptr, col, val)
    if case == "box_shape":
        o.overlap_mode = 1
        m.dim, m.nx, m.ny, m.nz = 2, 5, 4, 1
    if case == "tc_kind":
        o.tensor_cores = 3
    h = ctypes.c_void_p()
    st = lib.ddg_setup(ctypes.byref(m), part.ctypes.data_as(ctypes.c_void_p),
                       F.ctypes.data_as(ctypes.c_void_p), k, 1, ctypes.byref(o), None, ctypes.byref(h))
    assert st == ddg.DDG_EINVAL
    assert h.value is None
    assert len(lib.ddg_last_error(None)) > 0


@pytest.mark.parametrize("case", ["no_groups", "one_level", "neg_group"])
def test_vcycle_setup_rejects_bad_arguments_before_touching_the_gpu(lib, case):
    from paper_1504_00907_gb300 import ddg
    import ddg_inputs as di
    A = di.poisson5_2d(4)
    rowptr, col, val = di.csr_arrays(A)
    part = np.repeat(np.arange(4, dtype=np.int32), 4)
    groups = np.array([0, 0, 1, 1], dtype=np.int32)
    F = np.ones(16)
    o = ddg.default_options()
    if case == "one_level":
        o.use_coarse = 0
    if case == "neg_group":
        groups[2] = -1
    p_groups = None if case == "no_groups" else groups.ctypes.data_as(ctypes.c_void_p)
    m = _matrix(rowptr, col, val)
    h = ctypes.c_void_p()
    st = lib.ddg_setup_vcycle(ctypes.byref(m), part.ctypes.data_as(ctypes.c_void_p), p_groups,
                              F.ctypes.data_as(ctypes.c_void_p), 1, 1, ctypes.byref(o), None,
                              ctypes.byref(h))
    assert st == ddg.DDG_EINVAL
    assert h.value is None
    assert len(lib.ddg_last_error(None)) > 0


def test_set_generators_rejects_a_null_handle(lib):
    from paper_1504_00907_gb300 import ddg
    F = np.ones(4)
    assert lib.ddg_set_generators(None, F.ctypes.data_as(ctypes.c_void_p), 1) == ddg.DDG_EINVAL


def test_product_path_has_no_cpu_fallback():
    # the binding never imports the oracle and refuses to run without a GPU
    src = open(os.path.join(ROOT, "paper_1504_00907_gb300", "ddg.py")).read()
    assert "import oracle" not in src and "from oracle" not in src
    import torch
    if not torch.cuda.is_available():
        import ddg_inputs as di
        from paper_1504_00907_gb300 import ddg
        prob = di.make_poisson2d(N=16, box=8, overlap=1, p=1)
        with pytest.raises(RuntimeError):
            ddg.Solver.from_problem(prob)
