"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_l2(got, ref):
    """max over batch items of ||got - ref||_2 / ||ref||_2."""
    got = np.atleast_2d(np.asarray(got))
    ref = np.atleast_2d(np.asarray(ref))
    num = np.linalg.norm(got - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


# Tolerances of the parity bar: relative L2 error against the FP64 oracle.
TOL = {"c64": 1e-5, "c128": 1e-12}
