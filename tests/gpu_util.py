"""Helpers shared by the GPU tests (no transform arithmetic here)."""
import numpy as np


def rel_errors(z, ref):
    """(E_2, E_inf): normwise and max-norm relative errors (eq:Einf for the latter)."""
    z = np.asarray(z, np.float64)
    ref = np.asarray(ref, np.float64)
    d = z - ref
    n2 = np.linalg.norm(ref)
    ninf = np.abs(ref).max()
    e2 = np.linalg.norm(d) / n2 if n2 > 0 else np.linalg.norm(d)
    einf = np.abs(d).max() / ninf if ninf > 0 else np.abs(d).max()
    return float(e2), float(einf)
