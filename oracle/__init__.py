"""CPU oracle for the matrix-free p-multigrid vertex-patch method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import, call or execute it.  It shares no code, headers,
tables or constant generators with the CUDA library; the two meet only in
the seeded input vectors that the tests feed to both.

Everything here is plain, slow and written to be checked by eye against the
paper (arXiv 2512.02577, "Multigrid p-Robustness at Jacobi Speeds"):

* ``quadrature`` -- 1D Gauss-Lobatto nodes, Gauss-Legendre rules, Lagrange
  basis (the nodal Q_k basis and quadrature of §3 and the sum-factorised
  operator of Eq. (3)).
* ``fem`` -- the structured mesh hierarchy of Eq. (1), the geometry, the
  assembled sparse stiffness A_l of Eq. (4) built from the bilinear form
  Eq. (3), the transfer operators of Eq. (2), right-hand sides and L2 error.
* ``patch`` -- vertex patches (§2.1), the p-level hierarchy, p-transfers and
  rediscretised patch operators (§2.2, §3.2), the local p-multigrid V-cycle
  (Algorithm 3) inside the local Richardson iteration (Algorithm 2), and the
  exact dense patch solve.
* ``solver`` -- the additive vertex-patch smoother (Algorithm 1 with the
  sequential update replaced by a sum), the geometric V-cycle, PCG and
  flexible GMRES (the outer solver for the half local V-cycle, §3.2.2).
* ``constants`` -- the damping factors the paper leaves open (readings).

All arithmetic is float64.  Where the deformed-geometry operator stores its
quadrature-point tensors in float32, the oracle rounds them the same way
(``geom_fp32``) so that the discrete operator is the same one.

Parity status of each function is stated in its docstring; functions whose
result is pinned only by the oracle itself say "parity unpinned".
"""
