"""Closeness checks shared by the GPU parity tests.

A result passes only if it is close both as a whole and entry by entry:
  rel  = ||a - b||_F / ||b||_F          (the norm-wise relative error)
  elem = max_i |a_i - b_i| / max_i |b_i|  (the worst single entry against the largest one)
A norm-wise bound alone hides isolated wrong entries: one wrong value of typical size among
m entries moves `rel` by only about 1/sqrt(m).
"""
import numpy as np


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def elem(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def assert_close(a, b, tol: float, what: str = ""):
    """Both rel(a, b) and elem(a, b) must be <= tol."""
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, f"{what} shape {a.shape} != {b.shape}"
    r, e = rel(a, b), elem(a, b)
    maxabs = float(np.max(np.abs(a - b))) if b.size else 0.0
    assert r <= tol and e <= tol, (f"{what} rel {r:.3e}, elementwise {e:.3e} (max |diff| {maxabs:.3e}), "
                                   f"bound {tol:.1e}")
