"""Table 1 (§3.2.2): outer GMRES iterations of the multigrid preconditioner
with the multiplicative vertex-patch smoother on randomly distorted meshes,
for four local solvers, against the counts the paper prints
(tests/golden/table1_gmres_iterations.txt).  The paper states neither the
mesh sizes nor the tolerance; here rtol = 1e-8, 2D n = 32 (p = 3) or 16
(p = 7), 3D n = 16, distortion seed 2512.  Degree 3 reproduces every count
within 2; at degree 7 the counts keep the table's order and trends but run
higher (the local Jacobi damping is this build's reading, not the paper's)."""
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from paper_2512_02577_gb300.inputs import vertex_displacements
from tests.conftest import golden_rows

pytestmark = pytest.mark.gpu
DELTAS = {2: (0.0, 0.10, 0.25, 0.35), 3: (0.0, 0.10, 0.25, 0.30)}
SOLVERS = {"1V": (0, 1), "1H": (1, 1), "2H": (1, 2), "25V": (0, 25)}


def paper_counts():
    return {(int(r[0]), int(r[1]), r[2]): [int(v) for v in r[3:]] for r in golden_rows("table1_gmres_iterations.txt")}


def our_counts(dim, k, n):
    out = {}
    for name, (half, cycles) in SOLVERS.items():
        its = []
        for delta in DELTAS[dim]:
            cfg = p.make_config(dim=dim, n_cells=n, degree=k, geometry=p.DISTORTED,
                                vertex_disp=vertex_displacements(dim, n, delta, 2512), smoother=p.MULTIPLICATIVE,
                                local_half=half, local_cycles=cycles, outer_solver=p.OUTER_GMRES)
            ctx = p.Context(cfg, device="cuda:0")
            b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device="cuda:0")
            ctx.rhs_manufactured(b)
            x = torch.zeros_like(b)
            info = ctx.solve(b, x, rtol=1e-8)
            assert info.status == 0
            its.append(info.iterations)
            ctx.close()
        out[name] = its
    return out


@pytest.mark.parametrize("dim,k,n", [(2, 3, 32), (3, 3, 16), (2, 7, 16)])
def test_table1_iterations(dim, k, n):
    ours = our_counts(dim, k, n)
    paper = paper_counts()
    for i in range(4):
        # the table's order at every distortion
        assert ours["25V"][i] <= ours["1V"][i] <= ours["1H"][i], ours
        assert ours["2H"][i] <= ours["1H"][i], ours
    for name, its in ours.items():
        # counts do not fall as the distortion grows (one iteration of slack)
        assert all(b >= a - 1 for a, b in zip(its, its[1:])), (name, its)
        ref = paper[(dim, k, name)]
        if k == 3:
            assert all(abs(a - b) <= 2 for a, b in zip(its, ref)), (name, its, ref)
        else:
            assert all(0 <= a - b <= 6 for a, b in zip(its, ref)), (name, its, ref)
