"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/pmg.h, and validates configurations on the host."""
import ctypes
import os
import re

import pytest

import paper_2512_02577_gb300 as p
from tests.conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "pmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = p.load_library()
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(p.EXPORTED) == names


def test_status_strings():
    lib = p.load_library()
    assert lib.pmg_status_string(0) == b"ok"
    assert lib.pmg_status_string(p.PMG_ERR_UNSUPPORTED) == b"unsupported configuration"


@pytest.mark.parametrize("kw,code", [
    (dict(degree=9), p.PMG_ERR_UNSUPPORTED),
    (dict(degree=0), p.PMG_ERR_UNSUPPORTED),
    (dict(dim=4), p.PMG_ERR_UNSUPPORTED),
    (dict(n_cells=0), p.PMG_ERR_ARG),
    (dict(n_cells=12, n_levels=4), p.PMG_ERR_UNSUPPORTED),   # 12 not divisible by 8
    (dict(local_cycles=0), p.PMG_ERR_ARG),
    (dict(local_half=1, outer_solver=p.OUTER_CG), p.PMG_ERR_UNSUPPORTED),  # nonsymmetric under CG
    (dict(local_half=2), p.PMG_ERR_ARG),
    (dict(outer_solver=p.OUTER_GMRES, gmres_restart=0), p.PMG_ERR_ARG),
    (dict(outer_solver=p.OUTER_GMRES, gmres_restart=65), p.PMG_ERR_ARG),
    (dict(outer_solver=7), p.PMG_ERR_ARG),
    (dict(smoother=2), p.PMG_ERR_ARG),
    (dict(geometry=p.DISTORTED), p.PMG_ERR_ARG),            # no vertex displacements
    (dict(patch_persistent=2), p.PMG_ERR_ARG),
    (dict(patch_persistent=-2), p.PMG_ERR_ARG),
])
def test_bytes_required_rejects(kw, code):
    with pytest.raises(p.PmgError) as e:
        p.bytes_required(p.make_config(**kw))
    assert e.value.code == code


def test_bytes_required_grows_with_size():
    small = p.bytes_required(p.make_config(dim=3, n_cells=8, degree=2))
    big = p.bytes_required(p.make_config(dim=3, n_cells=16, degree=2))
    assert 6 * small < big < 10 * small
    fp32 = p.bytes_required(p.make_config(dim=3, n_cells=16, degree=2, mg_precision=p.FP32))
    assert 0.5 * big < fp32 < 1.5 * big  # FP32 MG halves the hierarchy, keeps FP64 CG vectors
    # 3D n=32 Q4 (2.1M DoFs): a few hundred MB
    assert 1e8 < p.bytes_required(p.make_config(dim=3, n_cells=32, degree=4)) < 1e9


def test_gmres_workspace_holds_its_krylov_vectors():
    # 2m + 1 extra FP64 vectors of the finest grid (plus small state)
    cg = p.bytes_required(p.make_config(dim=3, n_cells=16, degree=2))
    for m in (1, 10, 30):
        gm = p.bytes_required(p.make_config(dim=3, n_cells=16, degree=2, local_half=1, gmres_restart=m))
        small = gm - cg - (2 * m + 1) * 33 ** 3 * 8   # Hessenberg, state, multi-dot partials
        assert 0 <= small <= (m + 1) * (320 + m) * 8 + 2048
    # local_half selects GMRES by default in the binding
    assert p.make_config(local_half=1).outer_solver == p.OUTER_GMRES
    assert p.make_config().outer_solver == p.OUTER_CG


def test_large_coarse_level_is_accepted_for_apply_only_contexts():
    # 5 cells (odd): one level whose (39)^3 free DoFs exceed the dense coarse
    # limit; the plan exists (apply/smooth), the V-cycle is refused at run time
    assert p.bytes_required(p.make_config(n_cells=5, degree=8)) > 0


def test_create_null_out_is_rejected():
    lib = p.load_library()
    cfg = p.make_config()
    assert lib.pmg_create(ctypes.byref(cfg), None, None, 0, None) == p.PMG_ERR_ARG


def test_distorted_config_keeps_its_displacements():
    import numpy as np
    d = np.zeros((5 ** 3, 3))
    cfg = p.make_config(dim=3, n_cells=4, degree=2, geometry=p.DISTORTED, vertex_disp=d)
    assert cfg.vertex_disp == cfg._vertex_disp_ref.ctypes.data
    assert p.bytes_required(cfg) > p.bytes_required(p.make_config(dim=3, n_cells=4, degree=2, geometry=p.DEFORMED))
    with pytest.raises(ValueError):
        p.make_config(dim=3, n_cells=4, degree=2, geometry=p.DISTORTED, vertex_disp=np.zeros((10, 3)))


def test_coarse_dofs_stops_automatic_coarsening():
    # 32^3 Q4: free DoFs per level 127^3, 63^3, 31^3, 15^3 = 3375, 7^3, 3^3;
    # coarse_dofs = 4096 stops at 4^3 cells, whose dense inverse the plan holds
    small = p.bytes_required(p.make_config(dim=3, n_cells=32, degree=4))
    big = p.bytes_required(p.make_config(dim=3, n_cells=32, degree=4, coarse_dofs=4096))
    assert big > small + 3375 * 3375 * 8      # the dense FP64 coarse inverse of 3375 free DoFs
    with pytest.raises(p.PmgError) as e:
        p.bytes_required(p.make_config(dim=3, n_cells=32, degree=4, coarse_dofs=5000))
    assert e.value.code == p.PMG_ERR_ARG
