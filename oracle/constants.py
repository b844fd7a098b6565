"""Damping factors the paper leaves open, computed from their definitions.

Reading for the Jacobi damping on p-level p (§2.2 and §3.2 name a damped
Jacobi smoother but give no omega):

    omega_J(d, p) = 4 / (3 lambda_max(D^{-1} A_{j,p})),

with lambda_max from a dense symmetric eigen-solve of D^{-1/2} A D^{-1/2} on
the Cartesian patch (the ratio is invariant under the cell size h).

Reading for the additive patch damping (the paper's smoother is
multiplicative and needs none): omega_AS = theta / 2^d.  Every free DoF away
from the boundary lies in 2^d patches, so lambda_max(B_AS A) <= 2^d for
local solves with lambda(V_j A_j) <= 1, and theta < 2 keeps the smoother
convergent.  theta = 1.5: the oracle measured lambda_max(B_AS A) / 2^d between
0.94 and 0.999 on Cartesian test meshes, and among theta in {0.75, 1, 1.25,
1.5, 1.75} the value 1.5 gave the fewest (or within one of the fewest) CG
iterations on the 2D and 3D cases tried.

Parity unpinned: these numbers are the oracle's readings, not the paper's.
"""
import functools

import numpy as np

from .fem import Mesh
from .patch import PatchSolver, p_hierarchy, patch_matrix

THETA_PATCH = 1.5


@functools.lru_cache(maxsize=None)
def lambda_max_jacobi(d, p):
    """lambda_max(D^{-1} A_{j,p}) on a unit Cartesian patch (n = 2, v = centre)."""
    if p == 1:
        return 1.0
    mesh = Mesh(d, 2, p)
    A = patch_matrix(mesh, (1,) * d, p)
    s = 1.0 / np.sqrt(np.diag(A))
    return float(np.linalg.eigvalsh(s[:, None] * A * s[None, :])[-1])


def omega_jacobi(d, k):
    """Per p-level damping list (index 0 = the p = 1 level, unused)."""
    return [1.0 if p == 1 else 4.0 / (3.0 * lambda_max_jacobi(d, p)) for p in p_hierarchy(k)]


def omega_patch(d, theta=THETA_PATCH):
    return theta / 2 ** d
