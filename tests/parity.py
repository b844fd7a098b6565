"""Comparison used by the GPU parity tests."""
import numpy as np


def rel(a, b):
    """Error of ``a`` against the reference ``b``: the larger of the relative
    2-norm ||a - b|| / ||b|| and the element-wise max|a - b| / max|b| (a
    single wrong entry can hide under a norm bound on large vectors, but not
    under the element-wise one).  numpy arrays or torch tensors."""
    a = a.detach().cpu().double().numpy() if hasattr(a, "detach") else np.asarray(a, dtype=np.float64)
    b = b.detach().cpu().double().numpy() if hasattr(b, "detach") else np.asarray(b, dtype=np.float64)
    nb, mb = np.linalg.norm(b), np.abs(b).max(initial=0.0)
    diff = a - b
    return max(np.linalg.norm(diff) / (nb if nb > 0 else 1.0), np.abs(diff).max(initial=0.0) / (mb if mb > 0 else 1.0))
