"""Grouped solves: several systems of one method, any mesh sizes, solved in
lockstep with every launch covering all of them (pmg_solve_group, and the
server's grouping).  Each system's iterations and solution must be bitwise
those of its own pmg_solve; one grouped solve is also checked against the
oracle directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from oracle import constants, fem, solver
from paper_2512_02577_gb300 import serve
from paper_2512_02577_gb300.inputs import random_vector

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _ctx(d, n, k, **kw):
    return p.Context(p.make_config(dim=d, n_cells=n, degree=k, **kw), device=DEV)


def _rhs(d, n, k, seed):
    return torch.from_numpy(random_vector(d, n, k, seed=seed)).to(DEV)


def _levels(n):
    """levels of the library's automatic coarsening (halve while even)"""
    L = 1
    while n % 2 == 0:
        n //= 2
        L += 1
    return L


def _solo(ctxs, bs, rtol, maxit):
    out = []
    for c, b in zip(ctxs, bs):
        x = torch.full_like(b, 7.0)  # the solve overwrites x
        info = c.solve(b, x, rtol=rtol, maxit=maxit)
        out.append((info.iterations, info.status, x))
    return out


def _check_group_equals_solo(ctxs, bs, rtol=1e-8, maxit=300):
    solo = _solo(ctxs, bs, rtol, maxit)
    xs = [torch.full_like(b, -3.0) for b in bs]
    before = p.launch_count()
    infos = p.solve_group(ctxs, bs, xs, rtol=rtol, maxit=maxit)
    launches = p.launch_count() - before
    for (it, st, xa), info, x in zip(solo, infos, xs):
        assert info.iterations == it and info.status == st
        assert torch.equal(x, xa)
    return infos, launches


@pytest.mark.parametrize("d,k,ns,kw", [
    (3, 2, (8, 12, 16, 4), dict(mg_precision=p.FP32)),
    (3, 4, (8, 16, 6), dict(mg_precision=p.FP32)),
    (3, 4, (8, 4, 16), dict(mg_precision=p.FP64)),
    (3, 3, (8, 16, 12), dict(mg_precision=p.FP32, outer_apply=p.APPLY_FLOAT_FLOAT)),
    (3, 2, (8, 4, 16), dict(mg_precision=p.FP64, outer_apply=p.APPLY_FLOAT_FLOAT)),
    (3, 3, (8, 16, 4), dict(mg_precision=p.FP32, smoother=p.MULTIPLICATIVE)),
    (3, 2, (8, 16), dict(mg_precision=p.FP32, smooth_steps=2, local_cycles=2)),
    (3, 7, (8, 4), dict(mg_precision=p.FP32)),
    (2, 5, (16, 32, 64, 8, 24), dict(mg_precision=p.FP64)),
    (2, 3, (16, 8), dict(mg_precision=p.FP32, smoother=p.MULTIPLICATIVE, smooth_steps=2)),
])
def test_grouped_solve_is_bitwise_the_solo_solve(d, k, ns, kw):
    ctxs = [_ctx(d, n, k, **kw) for n in ns]
    bs = [_rhs(d, n, k, 900 + i) for i, n in enumerate(ns)]
    infos, launches = _check_group_equals_solo(ctxs, bs)
    assert all(i.status == 0 and i.rel_residual <= 1e-8 for i in infos)
    for c in ctxs:
        c.close()


def test_grouped_launches_cover_all_members():
    # eight systems of one size: a round launches what one system's
    # iteration does (plus the per-system residual copies), not eight times that
    d, k, n = 3, 3, 8
    ctxs = [_ctx(d, n, k, mg_precision=p.FP32) for _ in range(8)]
    bs = [_rhs(d, n, k, 40 + i) for i in range(8)]
    b1 = [_rhs(d, n, k, 40)]
    x1 = [torch.zeros_like(b1[0])]
    before = p.launch_count()
    one = p.solve_group(ctxs[:1], b1, x1)
    single = p.launch_count() - before
    infos, launches = _check_group_equals_solo(ctxs, bs)
    its = max(i.iterations for i in infos)
    assert launches <= single * (its + 1) / (one[0].iterations + 1) * 1.3
    for c in ctxs:
        c.close()


def test_members_with_different_damping_and_levels():
    d, k = 3, 3
    ctxs = [_ctx(d, 16, k, mg_precision=p.FP32),
            _ctx(d, 16, k, mg_precision=p.FP32, omega_patch=0.1),
            _ctx(d, 8, k, mg_precision=p.FP32, n_levels=2),
            _ctx(d, 16, k, mg_precision=p.FP32, omega_jacobi=[0.9, 0.7, 0.7, 0.7])]
    bs = [_rhs(d, c.cfg.n_cells, k, 60 + i) for i, c in enumerate(ctxs)]
    _check_group_equals_solo(ctxs, bs)


def test_edge_members_single_cell_zero_rhs_and_maxit():
    d, k = 3, 2
    ctxs = [_ctx(d, 1, k), _ctx(d, 8, k), _ctx(d, 2, k), _ctx(d, 8, k)]
    bs = [_rhs(d, 1, k, 1), torch.zeros(ctxs[1].num_dofs(), dtype=torch.float64, device=DEV),
          _rhs(d, 2, k, 3), _rhs(d, 8, k, 4)]
    infos, _ = _check_group_equals_solo(ctxs, bs, rtol=1e-12)
    assert infos[1].iterations == 0
    # stopped at maxit: status reported per system, still bitwise the solo solve
    infos, _ = _check_group_equals_solo(ctxs[2:], bs[2:], rtol=1e-14, maxit=2)
    assert [i.status for i in infos] == [p.PMG_NOT_CONVERGED] * 2


def test_grouped_solve_matches_the_oracle():
    d, k, ns = 2, 3, (8, 4)
    wj, wp = constants.omega_jacobi(d, k), constants.omega_patch(d)
    ctxs = [_ctx(d, n, k, omega_jacobi=wj, omega_patch=wp) for n in ns]
    bs = []
    for c in ctxs:
        b = torch.empty(c.num_dofs(), dtype=torch.float64, device=DEV)
        c.rhs_manufactured(b)
        bs.append(b)
    xs = [torch.zeros_like(b) for b in bs]
    infos = p.solve_group(ctxs, bs, xs, rtol=1e-8)
    for n, c, b, x, info in zip(ns, ctxs, bs, xs, infos):
        m = fem.Mesh(d, n, k)
        h = solver.Hierarchy(m, _levels(n), wj, wp)
        fine = h.levels[-1]
        b_ref = fem.rhs_manufactured(m)
        x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8)
        assert abs(info.iterations - it_ref) <= 1
        xf = np.zeros(m.n_dofs)
        xf[fine.I] = x_ref
        xh = x.cpu().numpy()
        assert np.abs(xh - xf).max() <= 1e-6 * np.abs(xf).max()


def test_grouped_solve_rejects_mismatches():
    a = _ctx(3, 8, 2)
    b_ = _ctx(3, 8, 3)
    c = _ctx(3, 4, 2, geometry=p.DEFORMED)
    g = _ctx(3, 8, 2, local_half=1, outer_solver=p.OUTER_GMRES)
    va, vb, vc, vg = (torch.zeros(x.num_dofs(), dtype=torch.float64, device=DEV) for x in (a, b_, c, g))
    with pytest.raises(p.PmgError) as e:
        p.solve_group([a, b_], [va, vb], [va.clone(), vb.clone()])
    assert e.value.code == p.PMG_ERR_ARG
    with pytest.raises(p.PmgError) as e:
        p.solve_group([a, a], [va, va], [va.clone(), va.clone()])
    assert e.value.code == p.PMG_ERR_ARG
    for other, v in ((c, vc), (g, vg)):
        with pytest.raises(p.PmgError) as e:
            p.solve_group([other], [v], [v.clone()])
        assert e.value.code == p.PMG_ERR_UNSUPPORTED
    # contexts are usable after a refused group
    x = torch.zeros_like(va)
    assert a.solve(_rhs(3, 8, 2, 5), x).status == 0


def test_server_grouping_same_alone_and_in_the_mix():
    from paper_2512_02577_gb300.inputs import serving_requests
    reqs = serving_requests(n_requests=24, rate=2000.0, arrival_seed=3, size_seed=5, n_lo=4, n_hi=16, k_lo=2, k_hi=4)
    before = p.launch_count()
    mix, summary = serve.run(reqs, precision=p.FP32, max_active=12, group_work=1e12, max_group=8)
    grouped_launches = p.launch_count() - before
    assert summary["failed"] == 0
    before = p.launch_count()
    plain, _ = serve.run(reqs, precision=p.FP32, max_active=12)
    plain_launches = p.launch_count() - before
    for a, b in zip(mix, plain):
        assert a["iterations"] == b["iterations"]
        assert torch.equal(a["x"], b["x"])
    assert grouped_launches < plain_launches


def test_solve_group_limits():
    ctxs = [_ctx(3, 1, 2) for _ in range(33)]
    bs = [_rhs(3, 1, 2, i) for i in range(33)]
    with pytest.raises(p.PmgError) as e:
        p.solve_group(ctxs, bs, [b.clone() for b in bs])
    assert e.value.code == p.PMG_ERR_ARG
    infos = p.solve_group(ctxs[:32], bs[:32], [torch.zeros_like(b) for b in bs[:32]])
    assert all(i.status == 0 for i in infos)


def test_server_closed_while_groups_run():
    # closing the server cancels the rounds in flight; the device stays usable
    from paper_2512_02577_gb300.inputs import serving_requests
    srv = p.Server(0, 8, group_work=1e18, max_group=8)
    keep = []
    for r in serving_requests(n_requests=8, rate=1e6, arrival_seed=1, size_seed=2, n_lo=8, n_hi=16, k_lo=3, k_hi=3):
        cfg = p.make_config(dim=3, n_cells=r["n"], degree=r["k"], mg_precision=p.FP32)
        b = serve._rhs(3, r["n"], r["k"], r["rhs_seed"])
        x = torch.zeros_like(b).pin_memory()
        keep.append((cfg, b, x, srv.submit(cfg, b, x)))
    for _ in range(3):
        srv.poll()
    srv.close()
    ctx = _ctx(3, 8, 3, mg_precision=p.FP32)
    b = _rhs(3, 8, 3, 9)
    x = torch.zeros_like(b)
    assert ctx.solve(b, x).status == 0
