"""Python binding of the GB300 p-multigrid vertex-patch library (libpmg.so).

Argument marshalling only: every numerical step runs in the CUDA kernels of
the in-tree shared library, whose C ABI is declared in include/pmg.h.  PyTorch
supplies device memory (the context workspace and the vectors) and the CUDA
stream.  If libpmg.so is missing or fails to load, importing the library
raises: there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmg.so")

PMG_OK = 0
PMG_NOT_CONVERGED = 1
PMG_ERR_ARG = -1
PMG_ERR_UNSUPPORTED = -2
PMG_ERR_OOM = -3
PMG_ERR_CUDA = -4
PMG_ERR_DEVICE_TIMEOUT = -5
PMG_ERR_STATE = -6
CARTESIAN, DEFORMED, DISTORTED = 0, 1, 2
FP64, FP32 = 0, 1
OUTER_CG, OUTER_GMRES = 0, 1
ADDITIVE, MULTIPLICATIVE = 0, 1
PATCH_AUTO, PATCH_MAJOR, PATCH_INTERLEAVED = 0, 1, 2
SERVE_FIFO, SERVE_SHORTEST_FIRST = 0, 1
APPLY_FP64, APPLY_FLOAT_FLOAT = 0, 1

# Every entry point declared in include/pmg.h.
EXPORTED = [
    "pmg_config_default", "pmg_bytes_required", "pmg_create", "pmg_destroy", "pmg_num_levels",
    "pmg_num_dofs", "pmg_apply", "pmg_residual", "pmg_smooth", "pmg_vcycle", "pmg_solve",
    "pmg_solve_host", "pmg_rhs_manufactured", "pmg_l2_error_manufactured", "pmg_synchronize",
    "pmg_launch_count", "pmg_status_string", "pmg_last_error", "pmg_apply_cartesian_noalloc",
    "pmg_patches_per_block", "pmg_solve_start", "pmg_solve_progress", "pmg_server_create",
    "pmg_server_destroy", "pmg_server_submit", "pmg_server_poll", "pmg_server_result", "pmg_server_stats",
    "pmg_smoother_phase_times", "pmg_damping", "pmg_default_damping", "pmg_server_release", "pmg_patch_layout",
    "pmg_server_set_policy", "pmg_apply_cells_per_block", "pmg_patch_persistent", "pmg_solve_group",
    "pmg_server_set_grouping",
]
NOALLOC_MAX_DOFS = 2097152


class PmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pmg error %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n_cells", ctypes.c_int), ("degree", ctypes.c_int),
        ("n_levels", ctypes.c_int), ("geometry", ctypes.c_int), ("deform_amp", ctypes.c_double),
        ("mg_precision", ctypes.c_int), ("omega_patch", ctypes.c_double),
        ("omega_jacobi", ctypes.c_double * 4), ("local_cycles", ctypes.c_int),
        ("smooth_steps", ctypes.c_int), ("patches_per_block", ctypes.c_int),
        ("local_half", ctypes.c_int), ("outer_solver", ctypes.c_int), ("gmres_restart", ctypes.c_int),
        ("smoother", ctypes.c_int), ("vertex_disp", ctypes.c_void_p),
        ("patch_layout", ctypes.c_int), ("patch_threads", ctypes.c_int), ("outer_apply", ctypes.c_int),
        ("geom_precision", ctypes.c_int), ("apply_cells_per_block", ctypes.c_int),
        ("patch_persistent", ctypes.c_int), ("coarse_dofs", ctypes.c_int),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("status", ctypes.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libpmg.so (raises OSError if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libpmg.so not found at %s; run __graft_entry__.build() or "
                      "python paper_2512_02577_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    vp, i64, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    sigs = {
        "pmg_config_default": (None, [ctypes.POINTER(Config)]),
        "pmg_bytes_required": (cint, [ctypes.POINTER(Config), ctypes.POINTER(i64)]),
        "pmg_create": (cint, [ctypes.POINTER(Config), vp, vp, i64, ctypes.POINTER(vp)]),
        "pmg_destroy": (cint, [vp]),
        "pmg_num_levels": (cint, [vp, ctypes.POINTER(cint)]),
        "pmg_num_dofs": (cint, [vp, cint, ctypes.POINTER(i64)]),
        "pmg_apply": (cint, [vp, cint, cint, vp, vp]),
        "pmg_residual": (cint, [vp, cint, cint, vp, vp, vp]),
        "pmg_smooth": (cint, [vp, cint, cint, vp, vp, cint]),
        "pmg_vcycle": (cint, [vp, vp, vp]),
        "pmg_solve": (cint, [vp, vp, vp, dbl, cint, ctypes.POINTER(SolveInfo)]),
        "pmg_solve_host": (cint, [vp, vp, vp, dbl, cint, ctypes.POINTER(SolveInfo)]),
        "pmg_rhs_manufactured": (cint, [vp, vp]),
        "pmg_l2_error_manufactured": (cint, [vp, vp, ctypes.POINTER(dbl)]),
        "pmg_synchronize": (cint, [vp]),
        "pmg_launch_count": (i64, []),
        "pmg_status_string": (ctypes.c_char_p, [cint]),
        "pmg_last_error": (ctypes.c_char_p, []),
        "pmg_apply_cartesian_noalloc": (cint, [cint, cint, cint, vp, vp, vp]),
        "pmg_patches_per_block": (cint, [vp, ctypes.POINTER(cint)]),
        "pmg_solve_start": (cint, [vp, vp, cint, vp, cint, dbl, cint]),
        "pmg_solve_progress": (cint, [vp, ctypes.POINTER(cint), ctypes.POINTER(SolveInfo)]),
        "pmg_server_create": (cint, [i64, cint, ctypes.POINTER(vp)]),
        "pmg_server_destroy": (cint, [vp]),
        "pmg_server_submit": (cint, [vp, ctypes.POINTER(Config), vp, vp, dbl, cint, ctypes.POINTER(i64)]),
        "pmg_server_poll": (cint, [vp, ctypes.POINTER(cint), ctypes.POINTER(cint)]),
        "pmg_server_result": (cint, [vp, i64, ctypes.POINTER(cint), ctypes.POINTER(SolveInfo),
                                     ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "pmg_server_stats": (cint, [vp, ctypes.POINTER(i64), ctypes.POINTER(cint), ctypes.POINTER(i64)]),
        "pmg_smoother_phase_times": (cint, [vp, cint, cint, ctypes.POINTER(dbl)]),
        "pmg_damping": (cint, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "pmg_default_damping": (cint, [cint, cint, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "pmg_server_release": (cint, [vp, i64]),
        "pmg_server_set_policy": (cint, [vp, cint, dbl, dbl]),
        "pmg_server_set_grouping": (cint, [vp, cint, dbl, cint]),
        "pmg_solve_group": (cint, [vp, cint, vp, vp, dbl, cint, vp]),
        "pmg_apply_cells_per_block": (cint, [vp, ctypes.POINTER(cint)]),
        "pmg_patch_persistent": (cint, [vp, ctypes.POINTER(cint)]),
        "pmg_patch_layout": (cint, [vp, ctypes.POINTER(cint), ctypes.POINTER(cint), ctypes.POINTER(cint)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code):
    if code < 0:
        raise PmgError(code, _lib.pmg_last_error().decode())
    return code


def make_config(dim=3, n_cells=8, degree=2, n_levels=0, geometry=CARTESIAN, deform_amp=0.05,
                mg_precision=FP64, omega_patch=0.0, omega_jacobi=None, local_cycles=1,
                smooth_steps=1, patches_per_block=0, local_half=0, outer_solver=None, gmres_restart=30,
                smoother=ADDITIVE, vertex_disp=None, patch_layout=PATCH_AUTO, patch_threads=0, outer_apply=APPLY_FP64,
                geom_precision=FP32, apply_cells_per_block=0, patch_persistent=0, coarse_dofs=0):
    """A pmg_config; outer_solver defaults to GMRES for the half local
    V-cycle (local_half=1) and to CG otherwise."""
    lib = load_library()
    c = Config()
    lib.pmg_config_default(ctypes.byref(c))
    c.dim, c.n_cells, c.degree, c.n_levels = dim, n_cells, degree, n_levels
    c.geometry, c.deform_amp, c.mg_precision = geometry, deform_amp, mg_precision
    c.omega_patch = omega_patch
    for i, w in enumerate(omega_jacobi or []):
        c.omega_jacobi[i] = w
    c.local_cycles, c.smooth_steps, c.patches_per_block = local_cycles, smooth_steps, patches_per_block
    c.local_half = local_half
    c.outer_solver = (OUTER_GMRES if local_half else OUTER_CG) if outer_solver is None else outer_solver
    c.gmres_restart = gmres_restart
    c.smoother = smoother
    c.patch_layout, c.patch_threads = patch_layout, patch_threads
    c.outer_apply = outer_apply
    c.geom_precision = geom_precision
    c.apply_cells_per_block = apply_cells_per_block
    c.patch_persistent = patch_persistent
    c.coarse_dofs = coarse_dofs
    if vertex_disp is not None:
        # ((n+1)^d, d) float64 displacements of the finest mesh's vertices;
        # the config keeps a reference so the array outlives it
        d = np.ascontiguousarray(vertex_disp, dtype=np.float64)
        if d.shape != ((n_cells + 1) ** dim, dim):
            raise ValueError("vertex_disp must have shape ((n_cells + 1)^dim, dim)")
        c._vertex_disp_ref = d
        c.vertex_disp = d.ctypes.data
    return c


def bytes_required(cfg):
    lib = load_library()
    n = ctypes.c_int64()
    _check(lib.pmg_bytes_required(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def launch_count():
    return load_library().pmg_launch_count()


def apply_cartesian_noalloc(dim, n_cells, degree, x, y, stream=None):
    """y = A x (FP64, Cartesian) through the allocation-free entry point, for
    callers that cannot allocate device memory; see include/pmg.h.  x and y
    must be on one device; the call runs with that device current, on
    ``stream`` (default: that device's current stream)."""
    lib = load_library()
    n = (degree * n_cells + 1) ** dim
    px, py = _ptr(x, torch.float64, n), _ptr(y, torch.float64, n)
    if x.device != y.device:
        raise ValueError("x and y must be on the same device, got %s and %s" % (x.device, y.device))
    if stream is not None and stream.device != x.device:
        raise ValueError("stream is on %s, the vectors on %s" % (stream.device, x.device))
    with torch.cuda.device(x.device):
        sh = (stream if stream is not None else torch.cuda.current_stream(x.device)).cuda_stream
        _check(lib.pmg_apply_cartesian_noalloc(dim, n_cells, degree, px, py, ctypes.c_void_p(sh or None)))


def default_damping(dim, degree):
    """(omega_patch, [omega_J per p-level]) the library uses when a config
    leaves the damping at its default; host arithmetic, no GPU needed."""
    lib = load_library()
    wp, wj = ctypes.c_double(), (ctypes.c_double * 4)()
    _check(lib.pmg_default_damping(dim, degree, ctypes.byref(wp), wj))
    return wp.value, list(wj)


def _ptr(t, dtype, n):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError("expected a contiguous %s tensor of %d elements, got %s %s" % (dtype, n, t.dtype,
                                                                                     tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One hierarchy on the current CUDA device; workspace owned by torch."""

    def __init__(self, cfg, stream=None, device=None):
        lib = load_library()
        self.cfg = cfg
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = bytes_required(cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            sh = self.stream.cuda_stream   # 0 (legacy default) -> the library makes its own stream
            _check(lib.pmg_create(ctypes.byref(cfg), ctypes.c_void_p(sh or None),
                                  ctypes.c_void_p(self.workspace.data_ptr()), nbytes, ctypes.byref(h)))
        self.handle = h
        self.n_levels = self._num_levels()
        self.mg_dtype = torch.float32 if cfg.mg_precision == FP32 else torch.float64

    def _num_levels(self):
        n = ctypes.c_int()
        _check(_lib.pmg_num_levels(self.handle, ctypes.byref(n)))
        return n.value

    def num_dofs(self, level=-1):
        level = self.n_levels - 1 if level < 0 else level
        n = ctypes.c_int64()
        _check(_lib.pmg_num_dofs(self.handle, level, ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.pmg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dt(self, prec):
        return torch.float64 if prec == FP64 else torch.float32

    def apply(self, x, y, level=-1, prec=FP64):
        level = self.n_levels - 1 if level < 0 else level
        n, dt = self.num_dofs(level), self._dt(prec)
        _check(_lib.pmg_apply(self.handle, level, prec, _ptr(x, dt, n), _ptr(y, dt, n)))

    def residual(self, b, u, r, level=-1, prec=FP64):
        level = self.n_levels - 1 if level < 0 else level
        n, dt = self.num_dofs(level), self._dt(prec)
        _check(_lib.pmg_residual(self.handle, level, prec, _ptr(b, dt, n), _ptr(u, dt, n), _ptr(r, dt, n)))

    def smooth(self, b, u, sweeps=1, level=-1):
        level = self.n_levels - 1 if level < 0 else level
        prec = self.cfg.mg_precision
        n, dt = self.num_dofs(level), self._dt(prec)
        _check(_lib.pmg_smooth(self.handle, level, prec, _ptr(b, dt, n), _ptr(u, dt, n), sweeps))

    def vcycle(self, r, z):
        n = self.num_dofs()
        _check(_lib.pmg_vcycle(self.handle, _ptr(r, torch.float64, n), _ptr(z, torch.float64, n)))

    def solve(self, b, x, rtol=1e-8, maxit=500):
        n = self.num_dofs()
        info = SolveInfo()
        _check(_lib.pmg_solve(self.handle, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n), rtol, maxit,
                              ctypes.byref(info)))
        return info

    def solve_host(self, b_host, x_host, rtol=1e-8, maxit=500):
        """b_host, x_host: CPU float64 tensors (pinned for asynchronous copies)."""
        n = self.num_dofs()
        for t in (b_host, x_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
                raise ValueError("expected contiguous CPU float64 tensors of %d elements" % n)
        info = SolveInfo()
        _check(_lib.pmg_solve_host(self.handle, ctypes.c_void_p(b_host.data_ptr()),
                                   ctypes.c_void_p(x_host.data_ptr()), rtol, maxit, ctypes.byref(info)))
        return info

    def rhs_manufactured(self, b):
        _check(_lib.pmg_rhs_manufactured(self.handle, _ptr(b, torch.float64, self.num_dofs())))

    def l2_error_manufactured(self, x):
        e = ctypes.c_double()
        _check(_lib.pmg_l2_error_manufactured(self.handle, _ptr(x, torch.float64, self.num_dofs()),
                                              ctypes.byref(e)))
        return e.value

    def smoother_phase_times(self, level=-1, reps=10):
        """Mean ms of (residual, patch launch, gather) of one smoothing step."""
        level = self.n_levels - 1 if level < 0 else level
        out = (ctypes.c_double * 3)()
        _check(_lib.pmg_smoother_phase_times(self.handle, level, reps, out))
        return tuple(out)

    def damping(self):
        """(omega_patch, [omega_J per p-level]) this context runs with."""
        wp, wj = ctypes.c_double(), (ctypes.c_double * 4)()
        _check(_lib.pmg_damping(self.handle, ctypes.byref(wp), wj))
        return wp.value, list(wj)

    def patch_persistent(self):
        """True if the Cartesian patch launches run as persistent grids."""
        v = ctypes.c_int()
        _check(_lib.pmg_patch_persistent(self.handle, ctypes.byref(v)))
        return bool(v.value)

    def apply_cells_per_block(self):
        """Cells per block of the deformed apply (0: the kernel's rule)."""
        v = ctypes.c_int()
        _check(_lib.pmg_apply_cells_per_block(self.handle, ctypes.byref(v)))
        return v.value

    def patch_layout(self):
        """(layout, patches per block, threads per block) of the finest level."""
        lay, ppc, thr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.pmg_patch_layout(self.handle, ctypes.byref(lay), ctypes.byref(ppc), ctypes.byref(thr)))
        return lay.value, ppc.value, thr.value

    def patches_per_block(self):
        n = ctypes.c_int()
        _check(_lib.pmg_patches_per_block(self.handle, ctypes.byref(n)))
        return n.value

    def synchronize(self):
        _check(_lib.pmg_synchronize(self.handle))


def solve_group(ctxs, bs, xs, rtol=1e-8, maxit=500):
    """Solve several systems at once, every launch covering all of them
    (pmg_solve_group): contexts of one method, any mesh sizes; bs, xs: CUDA
    float64 vectors of each context's finest level.  Returns a SolveInfo per
    system; raises on an error (PMG_NOT_CONVERGED is reported in the infos)."""
    m = len(ctxs)
    if not (len(bs) == len(xs) == m) or m < 1:
        raise ValueError("one b and one x per context")
    H = (ctypes.c_void_p * m)(*[c.handle.value for c in ctxs])
    B = (ctypes.c_void_p * m)(*[_ptr(b, torch.float64, c.num_dofs()).value for c, b in zip(ctxs, bs)])
    X = (ctypes.c_void_p * m)(*[_ptr(x, torch.float64, c.num_dofs()).value for c, x in zip(ctxs, xs)])
    infos = (SolveInfo * m)()
    with torch.cuda.device(ctxs[0].device):
        rc = _lib.pmg_solve_group(H, m, B, X, rtol, maxit, infos)
    if rc < 0:
        _check(rc)
    return list(infos)


class Server:
    """Serving loop over resident contexts (native, see include/pmg.h).

    submit() takes CPU float64 tensors (pinned for overlapped copies) for b
    and x; poll() never blocks; result() reports state, solve info and the
    submit/admit/done host times."""

    def __init__(self, memory_budget_bytes=0, max_active=8, policy=SERVE_FIFO, max_wait_s=2.0, small_work=0.0,
                 group_work=0.0, max_group=8):
        """group_work > 0: requests of estimated work (finest-grid nodes x
        (degree + 2)) up to group_work run in groups of up to max_group
        (pmg_server_set_grouping)."""
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.pmg_server_create(int(memory_budget_bytes), int(max_active), ctypes.byref(h)))
        self.handle = h
        self._keep = {}
        if policy != SERVE_FIFO:
            _check(lib.pmg_server_set_policy(h, policy, float(max_wait_s), float(small_work)))
        if group_work > 0:
            _check(lib.pmg_server_set_grouping(h, 1, float(group_work), int(max_group)))

    def submit(self, cfg, b_host, x_host, rtol=1e-8, maxit=500):
        for t in (b_host, x_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("expected contiguous CPU float64 tensors")
        rid = ctypes.c_int64()
        _check(_lib.pmg_server_submit(self.handle, ctypes.byref(cfg), ctypes.c_void_p(b_host.data_ptr()),
                                      ctypes.c_void_p(x_host.data_ptr()), rtol, maxit, ctypes.byref(rid)))
        self._keep[rid.value] = (cfg, b_host, x_host)
        return rid.value

    def poll(self):
        nr, nq = ctypes.c_int(), ctypes.c_int()
        _check(_lib.pmg_server_poll(self.handle, ctypes.byref(nr), ctypes.byref(nq)))
        return nr.value, nq.value

    def result(self, rid):
        st = ctypes.c_int()
        info = SolveInfo()
        ts, ta, td = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        code = _lib.pmg_server_result(self.handle, rid, ctypes.byref(st), ctypes.byref(info), ctypes.byref(ts),
                                      ctypes.byref(ta), ctypes.byref(td))
        return dict(state=st.value, code=code, iterations=info.iterations, rel_residual=info.rel_residual,
                    device_ms=info.time_ms, status=info.status, t_submit=ts.value, t_start=ta.value,
                    t_done=td.value)

    def release(self, rid):
        """Forget a finished request (its buffers may then be reused)."""
        _check(_lib.pmg_server_release(self.handle, rid))
        self._keep.pop(rid, None)

    def stats(self):
        used, res, created = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        _check(_lib.pmg_server_stats(self.handle, ctypes.byref(used), ctypes.byref(res), ctypes.byref(created)))
        return dict(used_bytes=used.value, resident_contexts=res.value, created_contexts=created.value)

    def close(self):
        if getattr(self, "handle", None):
            _lib.pmg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
