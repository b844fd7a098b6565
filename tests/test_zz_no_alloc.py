"""The allocation-free apply (pmg_apply_cartesian_noalloc) against the
context apply (pmg_apply).

The allocation-free entry point serves callers that cannot allocate device
memory (another framework's memory pool, a hard memory cap, real-time loops
that may not call cudaMalloc).  Its scratch is a device array shared by all
calls, so each case is called twice in a row, and cases of different sizes
follow one another, to show that a call does not depend on what the previous
call left in the array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from paper_2512_02577_gb300.inputs import random_vector

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


from tests.parity import rel  # noqa: E402  (max of norm-relative and element-wise error)


@pytest.mark.parametrize("d,n,k", [(3, 8, 3), (2, 16, 2), (3, 24, 5), (3, 4, 8), (2, 5, 1)])
def test_noalloc_apply_matches_context_apply_on_two_calls(d, n, k):
    cfg = p.make_config(dim=d, n_cells=n, degree=k)   # automatic coarsening keeps the coarse problem small
    ctx = p.Context(cfg, device=DEV)
    x = torch.tensor(random_vector(d, n, k, seed=100 + n + k), device=DEV)
    x[0] = 5.0  # a boundary entry: ignored by both
    y_ref = torch.empty_like(x)
    ctx.apply(x, y_ref)
    torch.cuda.synchronize()
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        p.apply_cartesian_noalloc(d, n, k, x, y)
        torch.cuda.synchronize()
        assert rel(y, y_ref) <= 1e-12
    ctx.close()


def test_noalloc_rejects_grids_above_the_limit():
    d, n, k = 3, 32, 4                      # 129^3 = 2,146,689 > 2,097,152
    N = (k * n + 1) ** d
    assert N > p.NOALLOC_MAX_DOFS
    x = torch.zeros(N, dtype=torch.float64, device=DEV)
    with pytest.raises(p.PmgError) as e:
        p.apply_cartesian_noalloc(d, n, k, x, torch.empty_like(x))
    assert e.value.code == p.PMG_ERR_UNSUPPORTED and "limit" in str(e.value)
