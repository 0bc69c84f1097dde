"""Python binding of the GB300 matrix-free finite element Poisson library.

Argument marshalling only: every function forwards to the C ABI declared in
``include/fe.h`` (same names), passing raw pointers of torch tensors (device
or host) or numpy arrays (host).  All arithmetic runs in the CUDA library; if
it has not been built (``paper_2104_08012_gb300.build.build()``) every call
raises ``FeError`` -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FE_OK = 0
FE_ERR_ARG, FE_ERR_CUDA, FE_ERR_NOMEM, FE_ERR_NO_CONVERGENCE, FE_ERR_NAN, FE_ERR_TIMEOUT, FE_ERR_UNSUPPORTED = range(-1, -8, -1)
FE_F64, FE_F32, FE_BF16 = 0, 1, 2
FE_F64_NATIVE, FE_F64_DOUBLE_FLOAT, FE_F64_DOUBLE_FLOAT_TET, FE_F64_DOUBLE_FLOAT_CUBE, FE_F64_DOUBLE_FLOAT_PAIR = \
    0, 1, 2, 3, 4
FE_PC_JACOBI, FE_PC_GMG, FE_PC_FMG = 0, 1, 2
FE_SMOOTHER_JACOBI, FE_SMOOTHER_PATCH = 0, 1
FE_COARSE_AUTO, FE_COARSE_DENSE, FE_COARSE_BLOCKED = 0, 1, 2
FE_GEOMETRY_AUTO, FE_GEOMETRY_PER_CELL = 0, 1
FE_QUAD_POINTS = 27
FE_PREC_F64, FE_PREC_MIXED_F32, FE_PREC_MIXED_BF16 = 0, 1, 2
FE_RHS_LOAD, FE_RHS_NODAL_F, FE_RHS_QUAD_F = 0, 1, 2
FE_MAX_LEVELS = 9
FE_PHASE_APPLY, FE_PHASE_SMOOTH, FE_PHASE_TRANSFER, FE_PHASE_COARSE, FE_PHASE_BLAS1 = range(5)
FE_NUM_PHASES = 5

# every symbol include/fe.h declares
EXPORTED = (
    "fe_default_opts", "fe_last_error", "fe_device_count", "fe_kernel_launches", "fe_mesh_create", "fe_mesh_destroy",
    "fe_hierarchy_refine", "fe_hierarchy_destroy", "fe_num_levels", "fe_level_sizes", "fe_dof_coordinates",
    "fe_cell_centroids", "fe_boundary_mask", "fe_set_coefficient", "fe_apply_operator", "fe_apply_mass",
    "fe_diagonal", "fe_lambda_max", "fe_prolong", "fe_restrict", "fe_smooth", "fe_coarse_solve", "fe_vcycle",
    "fe_load_vector", "fe_quadrature_points", "fe_load_vector_quadrature", "fe_solve_poisson", "fe_adjoint_gradient",
    "fe_objective", "fe_dot_noalloc", "fe_set_coarse_solver", "fe_coarse_info", "fe_set_geometry_form",
    "fe_set_f64_mode", "fe_set_smoother_fusion", "fe_set_smoother", "fe_batch_create", "fe_batch_destroy", "fe_batch_hierarchy", "fe_solve_batched", "fe_batch_schedule",
)


class FeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class SolverOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_it", ctypes.c_int), ("precond", ctypes.c_int),
                ("precision", ctypes.c_int), ("cheb_steps", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("inner_rtol", ctypes.c_double), ("inner_max_it", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("profile", ctypes.c_int), ("wait_timeout_us", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("solve_ms", ctypes.c_double), ("fine_applies_f64", ctypes.c_int),
                ("fine_applies_low", ctypes.c_int), ("apply_ms", ctypes.c_double), ("apply_timed", ctypes.c_int),
                ("levels_timed", ctypes.c_int),
                ("phase_ms", (ctypes.c_double * FE_MAX_LEVELS) * FE_NUM_PHASES)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_ms"}
        d["phase_ms"] = [list(row) for row in self.phase_ms]
        return d


_LIB = None


def lib_path():
    return _build.lib_path()


def load():
    """Load the built library (raises FeError if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise FeError(FE_ERR_UNSUPPORTED, f"CUDA library not built ({path}); run paper_2104_08012_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "fe_default_opts": (None, [ctypes.POINTER(SolverOpts)]),
        "fe_last_error": (ctypes.c_char_p, []),
        "fe_device_count": (i, []),
        "fe_kernel_launches": (ll, []),
        "fe_mesh_create": (i, [i, i, i, ctypes.POINTER(vp)]),
        "fe_mesh_destroy": (None, [vp]),
        "fe_hierarchy_refine": (i, [vp, i, i, ctypes.POINTER(vp)]),
        "fe_hierarchy_destroy": (None, [vp]),
        "fe_num_levels": (i, [vp]),
        "fe_level_sizes": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(ll), ctypes.POINTER(ll)]),
        "fe_dof_coordinates": (i, [vp, i, vp]),
        "fe_cell_centroids": (i, [vp, i, vp]),
        "fe_boundary_mask": (i, [vp, i, vp]),
        "fe_set_coefficient": (i, [vp, vp, vp]),
        "fe_apply_operator": (i, [vp, i, vp, vp, i, vp]),
        "fe_apply_mass": (i, [vp, i, vp, vp, vp]),
        "fe_diagonal": (i, [vp, i, vp, vp]),
        "fe_lambda_max": (i, [vp, i, ctypes.POINTER(d)]),
        "fe_prolong": (i, [vp, i, vp, vp, i, vp]),
        "fe_restrict": (i, [vp, i, vp, vp, i, vp]),
        "fe_smooth": (i, [vp, i, vp, vp, i, d, d, i, vp]),
        "fe_coarse_solve": (i, [vp, vp, vp, vp]),
        "fe_vcycle": (i, [vp, vp, vp, i, vp]),
        "fe_load_vector": (i, [vp, vp, vp, vp]),
        "fe_quadrature_points": (i, [vp, vp]),
        "fe_load_vector_quadrature": (i, [vp, vp, vp, vp]),
        "fe_solve_poisson": (i, [vp, vp, i, vp, ctypes.POINTER(SolverOpts), vp, ctypes.POINTER(SolveStats), vp]),
        "fe_adjoint_gradient": (i, [vp, vp, i, vp, vp, ctypes.POINTER(SolverOpts), vp, ctypes.POINTER(d), vp, vp]),
        "fe_objective": (i, [vp, vp, vp, ctypes.POINTER(d), vp]),
        "fe_dot_noalloc": (i, [vp, vp, ll, vp, vp]),
        "fe_set_f64_mode": (i, [vp, i]),
        "fe_set_smoother_fusion": (i, [vp, i]),
        "fe_set_smoother": (i, [vp, i]),
        "fe_set_coarse_solver": (i, [vp, i]),
        "fe_set_geometry_form": (i, [vp, i]),
        "fe_coarse_info": (i, [vp, ctypes.POINTER(ll), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ll),
                               ctypes.POINTER(d)]),
        "fe_batch_create": (i, [i, vp, vp, vp, ctypes.POINTER(vp)]),
        "fe_batch_destroy": (None, [vp]),
        "fe_batch_hierarchy": (i, [vp, i, ctypes.POINTER(vp)]),
        "fe_solve_batched": (i, [vp, vp, vp, ctypes.POINTER(SolverOpts), vp, vp]),
        "fe_batch_schedule": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _check(rc):
    if rc != FE_OK:
        raise FeError(rc, load().fe_last_error().decode())
    return rc


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise FeError(FE_ERR_ARG, "tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise FeError(FE_ERR_ARG, "arrays must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise FeError(FE_ERR_ARG, f"unsupported vector type {type(a)}")


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def default_opts(**kw):
    o = SolverOpts()
    load().fe_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise FeError(FE_ERR_ARG, f"unknown option {k}")
        setattr(o, k, v)
    return o


# ---- thin wrappers with the C names ----------------------------------------
def fe_device_count():
    return load().fe_device_count()


def fe_kernel_launches():
    return load().fe_kernel_launches()


def fe_mesh_create(nx, ny=None, nz=None):
    h = ctypes.c_void_p()
    _check(load().fe_mesh_create(nx, ny or nx, nz or nx, ctypes.byref(h)))
    return h


def fe_mesh_destroy(mesh):
    load().fe_mesh_destroy(mesh)


def fe_hierarchy_refine(mesh, nrefine, degree):
    h = ctypes.c_void_p()
    _check(load().fe_hierarchy_refine(mesh, nrefine, degree, ctypes.byref(h)))
    return h


def fe_hierarchy_destroy(h):
    load().fe_hierarchy_destroy(h)


def fe_set_coefficient(h, kappa, stream=None):
    _check(load().fe_set_coefficient(h, _ptr(kappa), _stream(stream)))


def fe_apply_operator(h, level, x, y, dtype=FE_F64, stream=None):
    _check(load().fe_apply_operator(h, level, _ptr(x), _ptr(y), dtype, _stream(stream)))


def fe_solve_poisson(h, rhs, rhs_kind, opts, u, stream=None, bc_values=None):
    st = SolveStats()
    rc = load().fe_solve_poisson(h, _ptr(rhs), rhs_kind, _ptr(bc_values), ctypes.byref(opts), _ptr(u),
                                 ctypes.byref(st), _stream(stream))
    _check(rc)
    return st


def fe_adjoint_gradient(h, rhs, rhs_kind, u_d, u_ckpt, opts, dJ, u_out=None, stream=None):
    J = ctypes.c_double()
    _check(load().fe_adjoint_gradient(h, _ptr(rhs), rhs_kind, _ptr(u_d), _ptr(u_ckpt), ctypes.byref(opts), _ptr(dJ),
                                      ctypes.byref(J), _ptr(u_out), _stream(stream)))
    return J.value


def _torch_float64():
    import torch  # only reached for tensor arguments, so torch is already imported by the caller
    return torch.float64


def fe_dot_noalloc(x, y, n=None, out=None, stream=None):
    """sum_i x[i] y[i] of two device vectors without any device allocation (see include/fe.h).

    ``out``: optional device tensor / host array of one double; returns the value when ``out`` is None.
    """
    def count(a, name):
        # the kernel reads n doubles from x and y and writes one to out: check what each buffer holds
        if hasattr(a, "data_ptr"):
            if a.dtype != _torch_float64() or not a.is_contiguous():
                raise FeError(FE_ERR_ARG, f"{name} must be a contiguous float64 tensor")
            return a.numel(), (a.device.type, a.device.index if a.device.type == "cuda" else None)
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise FeError(FE_ERR_ARG, f"{name} must be a C-contiguous float64 array")
            return a.size, ("cpu", None)
        raise FeError(FE_ERR_ARG, f"unsupported vector type {type(a)}")

    nx, dx = count(x, "x")
    ny, dy = count(y, "y")
    if n is None:
        n = nx
    n = int(n)
    if n < 0 or n > nx or n > ny:
        raise FeError(FE_ERR_ARG, f"n = {n} exceeds the length of x ({nx}) or y ({ny})")
    if dx != dy:
        raise FeError(FE_ERR_ARG, "x and y must be on the same device")
    if out is not None:
        no, do = count(out, "out")
        if no < 1:
            raise FeError(FE_ERR_ARG, "out must hold at least one float64")
        if do[0] == "cuda" and do != dx:
            raise FeError(FE_ERR_ARG, "a device out must be on the device of x and y")
    if out is None:
        res = np.zeros(1)
        _check(load().fe_dot_noalloc(_ptr(x), _ptr(y), n, _ptr(res), _stream(stream)))
        return float(res[0])
    _check(load().fe_dot_noalloc(_ptr(x), _ptr(y), n, _ptr(out), _stream(stream)))
    return out


class Batch:
    """Owning wrapper of an ``fe_batch``: independent problems solved by one persistent launch."""

    def __init__(self, sizes):
        """sizes: list of (N0, nrefine, degree)."""
        self._L = load()
        P = len(sizes)
        arr = lambda k: (ctypes.c_int * P)(*[int(s[k]) for s in sizes])
        self.b = ctypes.c_void_p()
        _check(self._L.fe_batch_create(P, arr(0), arr(1), arr(2), ctypes.byref(self.b)))
        self.nprob = P
        self.problems = []
        for p in range(P):
            hp = ctypes.c_void_p()
            _check(self._L.fe_batch_hierarchy(self.b, p, ctypes.byref(hp)))
            h = Hierarchy.__new__(Hierarchy)
            h._L, h.h, h.mesh, h.degree = self._L, hp, None, int(sizes[p][2])
            h.nlev = self._L.fe_num_levels(hp)
            h._borrowed = True
            self.problems.append(h)

    def close(self):
        if getattr(self, "b", None):
            for h in self.problems:
                h.h = None
            self._L.fe_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, f_list, u_list, opts=None, stream=None, **kw):
        o = opts if opts is not None else default_opts(**kw)
        P = self.nprob
        fp = (ctypes.c_void_p * P)(*[t.data_ptr() for t in f_list])
        up = (ctypes.c_void_p * P)(*[t.data_ptr() for t in u_list])
        st = (SolveStats * P)()
        _check(self._L.fe_solve_batched(self.b, fp, up, ctypes.byref(o), st, _stream(stream)))
        return [st[p] for p in range(P)]

    def schedule(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._L.fe_batch_schedule(self.b, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"cell_block": a.value, "dof_block": b.value, "ctas_per_sm": c.value}


class Hierarchy:
    """Owning wrapper of an ``fe_hierarchy`` (UnitCubeMesh(N0) refined ``nrefine`` times, P``degree``)."""

    def __init__(self, N0, nrefine, degree):
        self._L = load()
        self.h = None
        self.mesh = fe_mesh_create(N0)
        try:
            self.h = fe_hierarchy_refine(self.mesh, nrefine, degree)
        except Exception:
            fe_mesh_destroy(self.mesh)
            self.mesh = None
            raise
        self.degree = degree
        self.nlev = self._L.fe_num_levels(self.h)

    def close(self):
        if getattr(self, "_borrowed", False):
            self.h = None
            return
        if getattr(self, "h", None):
            fe_hierarchy_destroy(self.h)
            self.h = None
        if getattr(self, "mesh", None):
            fe_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- sizes and mesh queries (numpy, host)
    def sizes(self, level=-1):
        level = level % self.nlev
        N, n, c = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._L.fe_level_sizes(self.h, level, ctypes.byref(N), ctypes.byref(n), ctypes.byref(c)))
        return N.value, n.value, c.value

    def n_dofs(self, level=-1):
        return self.sizes(level)[1]

    def n_cells(self, level=-1):
        return self.sizes(level)[2]

    def dof_coordinates(self, level=-1):
        level = level % self.nlev
        out = np.empty((self.n_dofs(level), 3))
        _check(self._L.fe_dof_coordinates(self.h, level, _ptr(out)))
        return out

    def cell_centroids(self, level=-1):
        level = level % self.nlev
        out = np.empty((self.n_cells(level), 3))
        _check(self._L.fe_cell_centroids(self.h, level, _ptr(out)))
        return out

    def boundary_mask(self, level=-1):
        level = level % self.nlev
        out = np.empty(self.n_dofs(level), dtype=np.uint8)
        _check(self._L.fe_boundary_mask(self.h, level, _ptr(out)))
        return out.astype(bool)

    def lambda_max(self, level=-1):
        v = ctypes.c_double()
        _check(self._L.fe_lambda_max(self.h, level % self.nlev, ctypes.byref(v)))
        return v.value

    # -- operations on caller-owned vectors (torch tensors or numpy arrays)
    def set_f64_mode(self, mode):
        _check(self._L.fe_set_f64_mode(self.h, mode))

    def set_smoother(self, smoother):
        """FE_SMOOTHER_JACOBI (default) or FE_SMOOTHER_PATCH (vertex-star patches) as the Chebyshev preconditioner."""
        _check(self._L.fe_set_smoother(self.h, smoother))

    def set_geometry_form(self, form):
        """FE_GEOMETRY_AUTO (one value per cell when every G = c M) or FE_GEOMETRY_PER_CELL (six stored factors)."""
        _check(self._L.fe_set_geometry_form(self.h, form))

    def set_coarse_solver(self, mode):
        """FE_COARSE_AUTO (default), FE_COARSE_DENSE (explicit inverse factor) or FE_COARSE_BLOCKED (band factor)."""
        _check(self._L.fe_set_coarse_solver(self.h, mode))

    def coarse_info(self):
        n, w, blk, byt, ms = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_double()
        _check(self._L.fe_coarse_info(self.h, ctypes.byref(n), ctypes.byref(w), ctypes.byref(blk), ctypes.byref(byt),
                                      ctypes.byref(ms)))
        return {"n_interior": n.value, "bandwidth": w.value, "blocked": bool(blk.value), "bytes": byt.value,
                "setup_ms": ms.value}

    def set_smoother_fusion(self, on):
        """Chebyshev update fused into the operator launch (True) or a separate vector kernel (False, default)."""
        _check(self._L.fe_set_smoother_fusion(self.h, 1 if on else 0))

    def set_coefficient(self, kappa=None, stream=None):
        fe_set_coefficient(self.h, kappa, stream)

    def apply_operator(self, x, y, level=-1, dtype=FE_F64, stream=None):
        fe_apply_operator(self.h, level % self.nlev, x, y, dtype, stream)
        return y

    def apply_mass(self, x, y, level=-1, stream=None):
        _check(self._L.fe_apply_mass(self.h, level % self.nlev, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def diagonal(self, out, level=-1, stream=None):
        _check(self._L.fe_diagonal(self.h, level % self.nlev, _ptr(out), _stream(stream)))
        return out

    def prolong(self, xc, xf, level_fine, accumulate=False, stream=None):
        _check(self._L.fe_prolong(self.h, level_fine, _ptr(xc), _ptr(xf), int(accumulate), _stream(stream)))
        return xf

    def restrict(self, rf, rc, level_fine, zero_boundary=False, stream=None):
        _check(self._L.fe_restrict(self.h, level_fine, _ptr(rf), _ptr(rc), int(zero_boundary), _stream(stream)))
        return rc

    def smooth(self, b, x, level=-1, steps=2, lo=0.1, hi=1.1, dtype=FE_F64, stream=None):
        _check(self._L.fe_smooth(self.h, level % self.nlev, _ptr(b), _ptr(x), steps, lo, hi, dtype, _stream(stream)))
        return x

    def coarse_solve(self, b, x, stream=None):
        _check(self._L.fe_coarse_solve(self.h, _ptr(b), _ptr(x), _stream(stream)))
        return x

    def vcycle(self, b, x, dtype=FE_F64, stream=None):
        _check(self._L.fe_vcycle(self.h, _ptr(b), _ptr(x), dtype, _stream(stream)))
        return x

    def load_vector(self, f, b, stream=None):
        _check(self._L.fe_load_vector(self.h, _ptr(f), _ptr(b), _stream(stream)))
        return b

    def quadrature_points(self):
        """Physical quadrature points of the finest level's cells, shape (n_cells, FE_QUAD_POINTS, 3)."""
        out = np.empty((self.n_cells(), FE_QUAD_POINTS, 3))
        _check(self._L.fe_quadrature_points(self.h, _ptr(out)))
        return out

    def load_vector_quadrature(self, f_qp, b, stream=None):
        _check(self._L.fe_load_vector_quadrature(self.h, _ptr(f_qp), _ptr(b), _stream(stream)))
        return b

    def objective(self, u, u_d, stream=None):
        J = ctypes.c_double()
        _check(self._L.fe_objective(self.h, _ptr(u), _ptr(u_d), ctypes.byref(J), _stream(stream)))
        return J.value

    def solve(self, rhs, u, rhs_kind=FE_RHS_NODAL_F, opts=None, stream=None, bc_values=None, **kw):
        """Solve with Dirichlet data ``bc_values`` on the boundary dofs (None: homogeneous)."""
        o = opts if opts is not None else default_opts(**kw)
        return fe_solve_poisson(self.h, rhs, rhs_kind, o, u, stream, bc_values)

    def adjoint_gradient(self, rhs, u_d, dJ, rhs_kind=FE_RHS_NODAL_F, u_ckpt=None, u_out=None, opts=None,
                         stream=None, **kw):
        o = opts if opts is not None else default_opts(**kw)
        return fe_adjoint_gradient(self.h, rhs, rhs_kind, u_d, u_ckpt, o, dJ, u_out, stream)
