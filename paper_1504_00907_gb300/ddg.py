"""Python binding of the C ABI in include/ddg.h (argument marshalling only).

Every numerical step runs inside ``libddg.so`` (hand-written sm_103a
kernels).  PyTorch provides device memory and the CUDA stream; numpy arrays
carry the host-side setup inputs.  There is no CPU fallback: if the library
is missing or no GPU is present, the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ddg.h")

# status codes and enums (mirror include/ddg.h)
DDG_OK, DDG_EINVAL, DDG_ENOMEM, DDG_ENOTSPD, DDG_EBREAKDOWN, DDG_ENOCONV, DDG_ETIMEOUT, DDG_ECUDA = range(8)
DDG_DEBUG_TC_NO_COPIES = 1
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
LOCAL = {"auto": 0, "inv": 1, "band": 2}
COARSE = {"band": 0, "nd": 1}
TC = {"off": 0, "bf16": 1, "tf32": 2}
OVERLAP = {"graph": 0, "box": 1}
BETA = {"fr": 0, "pr": 1, "auto": 2}


class DDGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("keep_precisions", ctypes.c_int),
                ("overlap_mode", ctypes.c_int), ("beta", ctypes.c_int), ("maxit", ctypes.c_int),
                ("use_coarse", ctypes.c_int), ("rank_tol", ctypes.c_double),
                ("chunk_tiles", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("dedup_local", ctypes.c_int), ("spin_budget_ms", ctypes.c_double),
                ("autotune", ctypes.c_int), ("local_repr", ctypes.c_int), ("coarse_order", ctypes.c_int)]


class Matrix(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("dim", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dofs_per_node", ctypes.c_int),
                ("stencil_kind", ctypes.c_int), ("coef", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nsub", ctypes.c_int), ("ncolours", ctypes.c_int),
                ("n0", ctypes.c_int), ("kmax", ctypes.c_int), ("max_local", ctypes.c_int),
                ("sum_local", ctypes.c_int64), ("local_tiles", ctypes.c_int64),
                ("coarse_band", ctypes.c_int), ("coarse_blocks", ctypes.c_int),
                ("setup_ms", ctypes.c_double), ("precision", ctypes.c_int),
                ("local_inverses", ctypes.c_int), ("graph_solve", ctypes.c_int),
                ("ls_warps", ctypes.c_int), ("ls_chunk_tiles", ctypes.c_int), ("ls_band_rows", ctypes.c_int),
                ("tc_stages", ctypes.c_int), ("tuned", ctypes.c_int), ("local_repr", ctypes.c_int),
                ("local_band", ctypes.c_int), ("local_elems", ctypes.c_int64), ("coarse_order", ctypes.c_int),
                ("coarse_fronts", ctypes.c_int), ("coarse_levels", ctypes.c_int), ("coarse_elems", ctypes.c_int64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("timed", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


KERNEL_CLASSES = ("local_solve", "local_residual", "coarse", "spmv", "cg")

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "ddg_default_options": (None, [ctypes.POINTER(Options)]),
    "ddg_setup": (_I, [ctypes.POINTER(Matrix), _P, _P, _I, _I, ctypes.POINTER(Options), _P, ctypes.POINTER(_P)]),
    "ddg_setup_vcycle": (_I, [ctypes.POINTER(Matrix), _P, _P, _P, _I, _I, ctypes.POINTER(Options), _P,
                              ctypes.POINTER(_P)]),
    "ddg_set_generators": (_I, [_P, _P, _I]),
    "ddg_solve": (_I, [_P, _P, _P, _D, _PI, _PD]),
    "ddg_solve_host": (_I, [_P, _P, _P, _D, _PI, _PD]),
    "ddg_solve_batch": (_I, [_P, _P, _P, _I, _D, _P, _P]),
    "ddg_solve_many": (_I, [_P, _I, _P, _P, _P, _D, _P, _P]),
    "ddg_adjoint": (_I, [_P, _P, _P, _D, _PI, _PD]),
    "ddg_grad_coeff": (_I, [_P, _P, _P, _P]),
    "ddg_apply_preconditioner": (_I, [_P, _P, _P]),
    "ddg_coarse_correction": (_I, [_P, _P, _P]),
    "ddg_spmv": (_I, [_P, _P, _P]),
    "ddg_set_precision": (_I, [_P, _I]),
    "ddg_set_debug": (_I, [_P, _I]),
    "ddg_set_stream": (_I, [_P, _P]),
    "ddg_get_info": (_I, [_P, ctypes.POINTER(Info)]),
    "ddg_get_colouring": (_I, [_P, _P]),
    "ddg_get_coarse_offsets": (_I, [_P, _P]),
    "ddg_get_history": (_I, [_P, _P, _I, _PI]),
    "ddg_get_cg_coefficients": (_I, [_P, _P, _P, _I, _PI]),
    "ddg_condition_estimate": (_I, [_P, _P, _I, _D, _PD, _PD, _PD]),
    "ddg_profile": (_I, [_P, _I]),
    "ddg_get_kernel_stats": (_I, [_P, _P]),
    "ddg_spmv_dot_noalloc": (_I, [ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "ddg_destroy": (_I, [_P]),
    "ddg_last_error": (ctypes.c_char_p, [_P]),
    "ddg_status_string": (ctypes.c_char_p, [_I]),
}


def header_functions():
    """Names of the functions declared in include/ddg.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ddg_[a-z_0-9]+)\s*\(", text)))


def load():
    """Load the in-tree libddg.so (built by ``build.py``); no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           f"`python -m paper_1504_00907_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_options():
    o = Options()
    load().ddg_default_options(ctypes.byref(o))
    return o


def _check(st, handle=None):
    if st != DDG_OK:
        lib = load()
        msg = lib.ddg_last_error(handle).decode() or lib.ddg_status_string(st).decode()
        raise DDGError(st, msg)


def _dev(t, n=None, name="vector"):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def torch_empty_like_host(t):
    """An output buffer like the host tensor ``t`` (page-locked if ``t`` is)."""
    import torch
    out = torch.empty_like(t)
    return out.pin_memory() if t.is_pinned() else out


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def condition_estimate(alpha, beta, tol=1e-8):
    """Sec. 7: (lambda_min, lambda_max, iteration bound) from CG coefficients
    (``ddg_condition_estimate``; host only, needs no GPU)."""
    a, pa = _host(alpha, np.float64)
    b, pb = _host(beta if len(beta) else np.zeros(1), np.float64)
    lo, hi, it = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().ddg_condition_estimate(pa, pb, int(a.size), tol, ctypes.byref(lo), ctypes.byref(hi),
                                         ctypes.byref(it)), None)
    return lo.value, hi.value, it.value


class Solver:
    """DDG two-level Schwarz PCG for one SPD matrix (wraps a ddg_handle)."""

    def __init__(self, A, part, F, overlap, *, mode="graph", shape=None, stencil_kind=0,
                 coef=None, dofs_per_node=1, precision="fp64", keep=None, beta="auto",
                 maxit=1000, use_coarse=True, rank_tol=1e-10, chunk_tiles=0, tensor_cores=False,
                 stream=None, coarse_groups=None, dedup_local=False, spin_budget_ms=1000.0,
                 autotune=False, local_repr="auto", coarse_order="nd"):
        """Set up the preconditioner for the CSR matrix ``A`` (scipy), the
        partition ``part`` (subdomain id per dof) and the generators ``F``
        (n x k) with ``overlap`` layers (``ddg_setup``).

        precision: "fp64" | "fp32" | "bf16" (preconditioner; CG is FP64);
        keep: the precisions whose local inverses are stored (set_precision
        switches among them); tensor_cores: False | "bf16" | "tf32" (True
        means "bf16"): operands of the tcgen05 local solves of solve_batch
        at precision "bf16" or "fp32" respectively; coarse_order: "nd" |
        "band"; local_repr: "auto" | "inv" | "band"; coarse_groups: group id
        per subdomain for the three-level V-cycle (``ddg_setup_vcycle``).
        The remaining keywords mirror the fields of ``ddg_options``."""
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("the DDG solver needs a CUDA GPU")
        A = A.tocsr()
        self.n = A.shape[0]
        rowptr, p_rowptr = _host(A.indptr, np.int64)
        col, p_col = _host(A.indices, np.int32)
        val, p_val = _host(A.data, np.float64)
        m = Matrix()
        m.n = self.n
        m.rowptr, m.col, m.val = p_rowptr, p_col, p_val
        shape = tuple(shape) if shape is not None else ()
        m.dim = len(shape)
        m.nx = shape[0] if len(shape) > 0 else 0
        m.ny = shape[1] if len(shape) > 1 else 1
        m.nz = shape[2] if len(shape) > 2 else 1
        m.dofs_per_node = dofs_per_node
        m.stencil_kind = stencil_kind
        self._coef = None
        if coef is not None:
            self._coef, m.coef = _host(np.asarray(coef).ravel(), np.float64)
        part_a, p_part = _host(part, np.int32)
        F = np.asarray(F, dtype=np.float64)
        if F.ndim == 1:
            F = F[:, None]
        k = F.shape[1]
        Fc, p_F = _host(F.T.ravel(), np.float64)      # column-major
        o = default_options()
        o.precision = PREC[precision]
        o.keep_precisions = sum(1 << PREC[p] for p in (keep or (precision,)))
        o.overlap_mode = OVERLAP[mode]
        o.beta = BETA[beta]
        o.maxit = maxit
        o.use_coarse = 1 if use_coarse else 0
        o.rank_tol = rank_tol
        o.chunk_tiles = chunk_tiles
        o.tensor_cores = TC[tensor_cores] if isinstance(tensor_cores, str) else (1 if tensor_cores else 0)
        o.dedup_local = 1 if dedup_local else 0
        o.spin_budget_ms = spin_budget_ms
        o.autotune = 1 if autotune else 0
        o.local_repr = LOCAL[local_repr]
        o.coarse_order = COARSE[coarse_order]
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = ctypes.c_void_p()
        if coarse_groups is None:
            st = lib.ddg_setup(ctypes.byref(m), p_part, p_F, k, overlap, ctypes.byref(o),
                               ctypes.c_void_p(stream), ctypes.byref(h))
        else:
            # three-level V-cycle: coarse_groups maps each subdomain to its
            # coarse-level subdomain
            groups, p_groups = _host(coarse_groups, np.int32)
            st = lib.ddg_setup_vcycle(ctypes.byref(m), p_part, p_groups, p_F, k, overlap,
                                      ctypes.byref(o), ctypes.c_void_p(stream), ctypes.byref(h))
        _check(st, None)
        self.h = h
        self.precision = precision

    @classmethod
    def from_problem(cls, prob, **kw):
        """Build from a ``ddg_inputs.Problem``."""
        kw.setdefault("mode", prob.overlap_mode)
        kw.setdefault("shape", prob.shape)
        kw.setdefault("stencil_kind", prob.stencil_kind)
        kw.setdefault("dofs_per_node", getattr(prob, "dofs_per_node", 1))
        if prob.kappa is not None:
            kw.setdefault("coef", prob.kappa)
        return cls(prob.A, prob.part, prob.F, prob.overlap, **kw)

    def set_generators(self, F):
        """Rebuild the coarse space from new generators F (n x k host array),
        keeping the local inverses (``ddg_set_generators``)."""
        F = np.asarray(F, dtype=np.float64)
        if F.ndim == 1:
            F = F[:, None]
        Fc, p_F = _host(F.T.ravel(), np.float64)
        _check(load().ddg_set_generators(self.h, p_F, F.shape[1]), self.h)

    # ---- solves
    def solve(self, f, tol=1e-8, u=None):
        import torch
        pf = _dev(f, self.n, "f")
        if u is None:
            u = torch.empty_like(f)
        pu = _dev(u, self.n, "u")
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        st = load().ddg_solve(self.h, pf, pu, tol, ctypes.byref(it), ctypes.byref(rr))
        if st not in (DDG_OK, DDG_ENOCONV):
            _check(st, self.h)
        return u, it.value, rr.value, st

    def solve_host(self, f, tol=1e-8, u=None):
        """Solve from and into host memory (the copies happen inside the call).
        ``f`` is a numpy array or a CPU float64 torch tensor; page-locked
        tensors (``pin_memory()``) let the copies run at link speed.  ``u``
        is an optional output of the same kind."""
        if hasattr(f, "data_ptr"):
            if f.device.type != "cpu" or not f.is_contiguous() or f.numel() != self.n:
                raise ValueError(f"f must be a contiguous CPU tensor of {self.n} entries")
            if u is None:
                u = torch_empty_like_host(f)
            pf, pu = ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr())
        else:
            f, pf = _host(f, np.float64)
            if u is None:
                u = np.empty_like(f)
            pu = u.ctypes.data_as(ctypes.c_void_p)
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        st = load().ddg_solve_host(self.h, pf, pu, tol, ctypes.byref(it), ctypes.byref(rr))
        if st not in (DDG_OK, DDG_ENOCONV):
            _check(st, self.h)
        return u, it.value, rr.value, st

    def solve_batch(self, F, tol=1e-8):
        import torch
        n, m = F.shape
        pF = _dev(F.contiguous(), None, "F")
        U = torch.empty_like(F)
        its = np.zeros(m, dtype=np.int32)
        rr = np.zeros(m, dtype=np.float64)
        st = load().ddg_solve_batch(self.h, pF, _dev(U, None, "U"), m, tol,
                                    its.ctypes.data_as(ctypes.c_void_p),
                                    rr.ctypes.data_as(ctypes.c_void_p))
        if st not in (DDG_OK, DDG_ENOCONV):
            _check(st, self.h)
        return U, its, rr, st

    def adjoint(self, g, tol=1e-8):
        """lambda = A^{-1} g; returns (lambda, iterations, true relative
        residual, status) like ``solve`` (DDG_ENOCONV is returned, not raised)."""
        import torch
        lam = torch.empty_like(g)
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        st = load().ddg_adjoint(self.h, _dev(g, self.n, "g"), _dev(lam, self.n), tol,
                                ctypes.byref(it), ctypes.byref(rr))
        if st not in (DDG_OK, DDG_ENOCONV):
            _check(st, self.h)
        return lam, it.value, rr.value, st

    def grad_coeff(self, lam, u):
        """dL/dc for the coefficient array c given at setup (kappa per cell
        for VAR7, mu per element for Q1 elasticity)."""
        import torch
        ncoef = self._coef.size if self._coef is not None else u.numel()
        dk = torch.empty(ncoef, dtype=torch.float64, device=u.device)
        _check(load().ddg_grad_coeff(self.h, _dev(lam, self.n), _dev(u, self.n), _dev(dk, ncoef)), self.h)
        return dk

    # ---- building blocks (parity tests)
    def apply(self, r):
        import torch
        z = torch.empty_like(r)
        _check(load().ddg_apply_preconditioner(self.h, _dev(r, self.n, "r"), _dev(z, self.n)), self.h)
        return z

    def coarse_correction(self, r):
        import torch
        z = torch.empty_like(r)
        _check(load().ddg_coarse_correction(self.h, _dev(r, self.n, "r"), _dev(z, self.n)), self.h)
        return z

    def spmv(self, x):
        import torch
        y = torch.empty_like(x)
        _check(load().ddg_spmv(self.h, _dev(x, self.n, "x"), _dev(y, self.n)), self.h)
        return y

    def set_debug(self, flags):
        """Test hooks of the bounded device waits (DDG_DEBUG_*; 0 = off)."""
        _check(load().ddg_set_debug(self.h, int(flags)), self.h)

    def set_precision(self, precision):
        _check(load().ddg_set_precision(self.h, PREC[precision]), self.h)
        self.precision = precision

    def set_stream(self, stream):
        _check(load().ddg_set_stream(self.h, ctypes.c_void_p(stream)), self.h)
        self.stream = stream

    def info(self):
        inf = Info()
        _check(load().ddg_get_info(self.h, ctypes.byref(inf)), self.h)
        return {f: getattr(inf, f) for f, _ in Info._fields_}

    def colouring(self):
        c = np.zeros(self.info()["nsub"], dtype=np.int32)
        _check(load().ddg_get_colouring(self.h, c.ctypes.data_as(ctypes.c_void_p)), self.h)
        return c

    def coarse_offsets(self):
        c = np.zeros(self.info()["nsub"] + 1, dtype=np.int32)
        _check(load().ddg_get_coarse_offsets(self.h, c.ctypes.data_as(ctypes.c_void_p)), self.h)
        return c

    def history(self):
        ln = ctypes.c_int(0)
        load().ddg_get_history(self.h, None, 0, ctypes.byref(ln))
        buf = np.zeros(max(1, ln.value))
        load().ddg_get_history(self.h, buf.ctypes.data_as(ctypes.c_void_p), ln.value, ctypes.byref(ln))
        return buf[:ln.value]

    def cg_coefficients(self):
        """(alpha, beta) of the last single-vector solve (Sec. 7)."""
        ln = ctypes.c_int(0)
        _check(load().ddg_get_cg_coefficients(self.h, None, None, 0, ctypes.byref(ln)), self.h)
        a = np.zeros(max(1, ln.value))
        b = np.zeros(max(1, ln.value))
        _check(load().ddg_get_cg_coefficients(self.h, a.ctypes.data_as(ctypes.c_void_p),
                                              b.ctypes.data_as(ctypes.c_void_p), ln.value,
                                              ctypes.byref(ln)), self.h)
        return a[:ln.value], b[:max(0, ln.value - 1)]

    def condition_estimate(self, tol=1e-8):
        """(lambda_min, lambda_max, CG iteration bound for tol) of M^{-1}A
        from the last solve's Lanczos tridiagonal (Sec. 7)."""
        a, b = self.cg_coefficients()
        return condition_estimate(a, b, tol)

    def profile(self, classes=()):
        """Reset the launch counters; time the named kernel classes with events."""
        mask = sum(1 << KERNEL_CLASSES.index(c) for c in classes)
        _check(load().ddg_profile(self.h, mask), self.h)

    def kernel_stats(self):
        st = (KernelStat * len(KERNEL_CLASSES))()
        _check(load().ddg_get_kernel_stats(self.h, ctypes.cast(st, ctypes.c_void_p)), self.h)
        return {c: {"launches": st[i].launches, "timed": st[i].timed, "ms": st[i].ms,
                    "bytes": st[i].bytes} for i, c in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "h", None):
            load().ddg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_many(solvers, rhs, tol=1e-8):
    """Solve independent problems of uneven sizes concurrently.

    ``solvers``: distinct Solver objects (give each its own CUDA stream so the
    problems overlap); ``rhs``: one CUDA float64 tensor per problem, [n] or
    [n, m].  Returns (solutions, iterations per column, true relative
    residual per column, status).
    """
    import torch
    lib = load()
    nprob = len(solvers)
    hs = (ctypes.c_void_p * nprob)(*[s.h for s in solvers])
    outs, fptr, uptr, ms = [], [], [], []
    for s, f in zip(solvers, rhs):
        if f.dim() == 1:
            _dev(f, s.n, "f")
            ms.append(1)
        else:
            _dev(f, None, "F")
            ms.append(f.shape[1])
        u = torch.empty_like(f)
        outs.append(u)
        fptr.append(f.data_ptr())
        uptr.append(u.data_ptr())
    tot = sum(ms)
    its = np.zeros(tot, dtype=np.int32)
    rr = np.zeros(tot, dtype=np.float64)
    F = (ctypes.c_void_p * nprob)(*fptr)
    U = (ctypes.c_void_p * nprob)(*uptr)
    M = (ctypes.c_int * nprob)(*ms)
    st = lib.ddg_solve_many(hs, nprob, F, U, M, tol, its.ctypes.data_as(ctypes.c_void_p),
                            rr.ctypes.data_as(ctypes.c_void_p))
    if st not in (DDG_OK, DDG_ENOCONV):
        raise DDGError(st, "ddg_solve_many failed")
    return outs, its, rr, st


def solve_autograd(solver, kappa, f, tol=1e-10):
    """u = A(c)^{-1} f with gradients for the coefficient array c and for f.

    ``solver`` must have been set up with coefficients ``c`` (the cell
    conductivities kappa of a variable-coefficient handle, or the element
    shear moduli mu of a Q1-elasticity handle), and ``kappa`` must hold those
    same values: the handle's matrix and preconditioner are built from them,
    so a different ``kappa`` (after an optimiser step, say) raises ValueError
    instead of returning the solution and gradient of the old matrix; set up
    a new Solver for new coefficients.  The forward solve and the adjoint
    solve both run through the library; the backward returns dL/df = lambda
    and dL/dc = -lambda^T (dA/dc) u (``ddg_grad_coeff``).  Both directions
    raise DDGError unless their solve converged.
    """
    import torch

    if solver._coef is None:
        raise ValueError("the solver was set up without coefficients (coef=None)")
    given = kappa.detach().to("cpu", torch.float64).reshape(-1)
    if given.numel() != solver._coef.size or not torch.equal(given, torch.from_numpy(solver._coef)):
        raise ValueError("kappa differs from the coefficients the solver was set up with")

    class _DDGSolve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, kappa_t, f_t):
            u, _, _, st = solver.solve(f_t.detach().contiguous(), tol)
            if st != DDG_OK:
                raise DDGError(st, "forward solve did not converge")
            ctx.save_for_backward(u)
            return u

        @staticmethod
        def backward(ctx, gu):
            (u,) = ctx.saved_tensors
            lam, _, _, st = solver.adjoint(gu.contiguous(), tol)
            if st != DDG_OK:
                raise DDGError(st, "adjoint solve did not converge")
            dk = solver.grad_coeff(lam, u)
            return dk.view_as(kappa), lam

    return _DDGSolve.apply(kappa, f)
