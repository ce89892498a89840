"""Comparison of a GPU result with the oracle's, normwise and element by element.

``assert_close(got, ref, tol)`` asserts both
  * ||got - ref||_2 <= tol ||ref||_2   (the normwise bound), and
  * max_i |got_i - ref_i| <= tol max_i |ref_i|   (the element-wise bound),
so that a few wrong entries (a clipped boundary subdomain, a ragged tile)
cannot hide under the norm of a long vector.
"""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def max_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b), initial=0.0)) / max(float(np.max(np.abs(b), initial=0.0)), 1e-300)


def assert_close(got, ref, tol, label=""):
    nr, mr = rel(got, ref), max_rel(got, ref)
    assert nr <= tol, f"{label} normwise {nr:.3e} > {tol:.1e}"
    assert mr <= tol, f"{label} element-wise {mr:.3e} > {tol:.1e}"
