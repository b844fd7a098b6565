"""The library's default damping against the oracle's (CPU, no GPU).

The paper leaves the local Jacobi damping omega_J and the additive-Schwarz
damping omega_AS open (§2.2, §3.2).  Both sides take the same reading,
omega_J(p) = 4 / (3 lambda_max(D^{-1} A_{j,p})) on the Cartesian patch and
omega_AS = 1.5 / 2^d, but compute lambda_max independently: the oracle by a
dense symmetric eigen-solve, the library by Lanczos on the Kronecker-form
patch operator.  pmg_default_damping is host arithmetic, so this runs
without a GPU; the GPU tests check that contexts built with the default
damping run with exactly these values and match the oracle.
"""
import pytest

import paper_2512_02577_gb300 as p
from oracle import constants

try:
    p.load_library()
except OSError:  # not built in this checkout
    pytest.skip("libpmg.so not built", allow_module_level=True)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("k", range(1, 9))
def test_default_damping_matches_oracle(d, k):
    wp, wj = p.default_damping(d, k)
    assert wp == constants.omega_patch(d)
    ref = constants.omega_jacobi(d, k)
    for l, w in enumerate(ref):
        assert abs(wj[l] - w) <= 1e-12 * w, (l, wj[l], w)
    assert all(x == 1.0 for x in wj[len(ref):])


def test_default_damping_rejects_bad_arguments():
    with pytest.raises(p.PmgError):
        p.default_damping(4, 2)
    with pytest.raises(p.PmgError):
        p.default_damping(3, 9)
