"""Python binding of the crhyb C interface (include/crhyb.h), by ctypes.

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions carry the names of the C entry points.  Arrays may
be torch tensors (on the GPU or pinned/pageable host memory) or numpy
arrays; device memory and streams come from torch.

The library must have been built (``paper_2101_03777_gb300.build``); loading
fails with an ImportError otherwise.  There is no CPU fallback.
"""

import atexit
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrhyb.so")

CR_OK = 0
CR_ERR = {
    -1: "CR_ERR_ARG", -2: "CR_ERR_MESH", -3: "CR_ERR_SINGULAR", -4: "CR_ERR_NOT_CONVERGED",
    -5: "CR_ERR_BREAKDOWN", -6: "CR_ERR_TIMEOUT", -7: "CR_ERR_CUDA", -8: "CR_ERR_OOM",
}
CONV = {"none": 0, "newton": 1, "oseen": 2}
PREC = {"fp64": 0, "mixed": 1, "mixed_fp32": 1, "mixed_bf16": 2, "ff": 3, "ff_bf16": 4}
METHOD = {"pcg": 0, "gmres": 1, "bicgstab": 2}
PRECOND = {"jacobi": 0, "chebyshev": 1}
POLY_PREC = {"same": 0, "fp32": 1, "bf16": 2}
CR_MAX_RESTART = 64


class CrError(RuntimeError):
    """A crhyb call returned an error status."""

    def __init__(self, code, msg):
        self.code = code
        self.name = CR_ERR.get(code, str(code))
        super().__init__(f"{self.name}: {msg}")


class cr_mesh_opts(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_int32), ("need_mis", ctypes.c_int32)]


class cr_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("mu", ctypes.c_double), ("conv", ctypes.c_int32),
                ("lambda_scale", ctypes.c_double)]


class cr_hyb_opts(ctypes.Structure):
    _fields_ = [("keep_fp32", ctypes.c_int32), ("keep_bf16", ctypes.c_int32),
                ("keep_lo_fp32", ctypes.c_int32), ("keep_lo_bf16", ctypes.c_int32)]


class cr_solve_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("prec", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("restart", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("use_x0", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("profile", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("poly_degree", ctypes.c_int32), ("poly_ratio", ctypes.c_double),
                ("poly_prec", ctypes.c_int32), ("deflation", ctypes.c_void_p)]


class cr_batch_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("autotune", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("rhs_grouping", ctypes.c_int32)]


class cr_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("relres", ctypes.c_double),
                ("status", ctypes.c_int32), ("spmv_launches", ctypes.c_int32), ("spmv_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64)]


class cr_newton_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("linear_steps", ctypes.c_int32),
                ("inner_iterations", ctypes.c_int64), ("increment", ctypes.c_double),
                ("residual", ctypes.c_double), ("first_residual", ctypes.c_double), ("status", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
# name: (restype, argtypes)
_SIGS = {
    "cr_mesh_load": (_i32, [ctypes.c_int, _vp, _i64, _vp, _i64, ctypes.POINTER(cr_mesh_opts), _vp, ctypes.POINTER(_vp)]),
    "cr_mesh_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "cr_mesh_faces": (_i32, [_vp, _vp]),
    "cr_mesh_face_elements": (_i32, [_vp, _vp, _vp]),
    "cr_mesh_mis": (_i32, [_vp, _vp]),
    "cr_destroy_mesh": (None, [_vp]),
    "cr_assemble_coupled": (_i32, [_vp, ctypes.POINTER(cr_params), _vp, ctypes.c_int, _vp, ctypes.POINTER(_vp), _vp]),
    "cr_destroy_system": (None, [_vp]),
    "cr_hybridise": (_i32, [_vp, ctypes.POINTER(cr_hyb_opts), ctypes.POINTER(_vp)]),
    "cr_hybrid_export": (_i32, [_vp, _vp, _vp, _vp]),
    "cr_solve": (_i32, [_vp, ctypes.c_int, ctypes.POINTER(cr_solve_opts), _vp, ctypes.POINTER(cr_solve_stats)]),
    "cr_system_set_previous": (_i32, [_vp, _vp]),
    "cr_coupled_create": (_i32, [_vp, ctypes.POINTER(_vp)]),
    "cr_solve_coupled": (_i32, [_vp, ctypes.c_int, ctypes.POINTER(cr_solve_opts), _vp, _vp,
                                ctypes.POINTER(cr_solve_stats)]),
    "cr_destroy_coupled": (None, [_vp]),
    "cr_solve_steady": (_i32, [_vp, _vp, ctypes.c_int, ctypes.POINTER(cr_solve_opts), _vp, _vp,
                                ctypes.POINTER(cr_solve_stats)]),
    "cr_solve_newton": (_i32, [_vp, ctypes.c_double, _vp, _vp, ctypes.POINTER(cr_solve_opts), ctypes.c_double,
                                ctypes.c_int, _vp, _vp, ctypes.POINTER(cr_newton_stats)]),
    "cr_solve_preconditioned": (_i32, [_vp, ctypes.c_int, _vp, ctypes.POINTER(cr_solve_opts), _vp,
                                       ctypes.POINTER(cr_solve_stats)]),
    "cr_apply_G": (_i32, [_vp, _vp, _vp]),
    "cr_recover_up": (_i32, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "cr_destroy_hybrid": (None, [_vp]),
    "cr_batch_create": (_i32, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(cr_batch_opts), ctypes.POINTER(_vp)]),
    "cr_batch_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "cr_solve_batched": (_i32, [_vp, ctypes.POINTER(cr_solve_opts), ctypes.POINTER(_vp), ctypes.POINTER(cr_solve_stats)]),
    "cr_destroy_batch": (None, [_vp]),
    "cr_residual_noalloc": (_i32, [ctypes.c_int, _i64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "cr_residual_noalloc_max_rows": (_i64, []),
    "cr_chebyshev_step_form": (_i32, [ctypes.c_int, ctypes.c_int]),
    "cr_deflation_create": (_i32, [_vp, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "cr_deflation_lanczos": (_i32, [_vp, ctypes.c_int, ctypes.POINTER(cr_solve_opts), ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_vp)]),
    "cr_solve_ritz": (_i32, [_vp, ctypes.c_int, ctypes.POINTER(cr_solve_opts), _vp, ctypes.POINTER(cr_solve_stats),
                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_vp)]),
    "cr_deflation_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "cr_deflation_export": (_i32, [_vp, _vp]),
    "cr_destroy_deflation": (None, [_vp]),
    "cr_last_error": (ctypes.c_char_p, []),
}
EXPORTED = tuple(_SIGS)

_lib = None
_closing = False


@atexit.register
def _at_exit():
    # Handles still alive at interpreter exit are left to process teardown:
    # module teardown order is arbitrary and the CUDA runtime may already be gone.
    global _closing
    _closing = True


def _alive():
    return _lib is not None and not _closing


def load_library(path=LIB_PATH):
    """Load libcrhyb.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"crhyb CUDA library not built: {path} is missing "
                          "(run paper_2101_03777_gb300.build.build_library())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != CR_OK:
        raise CrError(rc, load_library().cr_last_error().decode())


def _ptr(a, dtype, size=None, name="array"):
    """Address of a contiguous torch tensor or numpy array of the given dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name}: need a C-contiguous numpy array of {np.dtype(dtype)}")
        if size is not None and a.size != size:
            raise ValueError(f"{name}: expected {size} elements, got {a.size}")
        return a.ctypes.data
    import torch
    tmap = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8, np.float32: torch.float32}
    if not isinstance(a, torch.Tensor):
        raise TypeError(f"{name}: need a torch tensor or numpy array")
    if a.dtype != tmap[dtype] or not a.is_contiguous():
        raise TypeError(f"{name}: need a contiguous tensor of {tmap[dtype]}")
    if size is not None and a.numel() != size:
        raise ValueError(f"{name}: expected {size} elements, got {a.numel()}")
    return a.data_ptr()


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Mesh:
    """Owner of a cr_mesh handle."""

    def __init__(self, handle, dim, ne, nf, nf_ext):
        self.handle, self.dim, self.ne, self.nf, self.nf_ext = handle, dim, ne, nf, nf_ext

    def __del__(self):
        if getattr(self, "handle", None) and _alive():
            _lib.cr_destroy_mesh(self.handle)
            self.handle = None


class System:
    """Owner of a cr_system handle (keeps its mesh alive)."""

    def __init__(self, handle, mesh, nrhs):
        self.handle, self.mesh, self.nrhs = handle, mesh, nrhs

    def __del__(self):
        if getattr(self, "handle", None) and _alive():
            _lib.cr_destroy_system(self.handle)
            self.handle = None


class Hybrid:
    """Owner of a cr_hybrid handle (keeps its system alive)."""

    def __init__(self, handle, system):
        self.handle, self.system, self.mesh = handle, system, system.mesh

    @property
    def n(self):
        return self.mesh.nf * self.mesh.dim

    def __del__(self):
        if getattr(self, "handle", None) and _alive():
            _lib.cr_destroy_hybrid(self.handle)
            self.handle = None


def cr_mesh_load(coords, elems, k0=0, need_mis=False, stream=None):
    """Load a simplicial mesh (host arrays: coords float64 [nv, d], elems int32 [ne, d+1])."""
    lib = load_library()
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    nv, dim = coords.shape
    ne = elems.shape[0]
    if elems.shape[1] != dim + 1:
        raise ValueError("elems must have dim+1 columns")
    opts = cr_mesh_opts(int(k0), int(bool(need_mis)))
    h = _vp()
    _check(lib.cr_mesh_load(dim, coords.ctypes.data, nv, elems.ctypes.data, ne, ctypes.byref(opts),
                            _stream_handle(stream), ctypes.byref(h)))
    d, n_e, nf, nx = _i32(), _i64(), _i64(), _i64()
    _check(lib.cr_mesh_info(h, ctypes.byref(d), ctypes.byref(n_e), ctypes.byref(nf), ctypes.byref(nx)))
    return Mesh(h, d.value, n_e.value, nf.value, nx.value)


def cr_mesh_faces(mesh):
    out = np.empty((mesh.nf, mesh.dim), dtype=np.int32)
    _check(load_library().cr_mesh_faces(mesh.handle, out.ctypes.data))
    return out


def cr_mesh_face_elements(mesh):
    fe = np.empty((mesh.nf, 2), dtype=np.int32)
    fl = np.empty((mesh.nf, 2), dtype=np.int32)
    _check(load_library().cr_mesh_face_elements(mesh.handle, fe.ctypes.data, fl.ctypes.data))
    return fe, fl


def cr_mesh_mis(mesh):
    out = np.empty(mesh.ne, dtype=np.uint8)
    _check(load_library().cr_mesh_mis(mesh.handle, out.ctypes.data))
    return out.astype(bool)


def cr_assemble_coupled(mesh, nu, mu, fbar, conv="none", w=None, lambda_scale=0.0, blocks_out=None):
    """Record the coupled system; fbar [nrhs, ne, d] float64 (host or device)."""
    lib = load_library()
    nrhs = int(fbar.shape[0]) if len(fbar.shape) == 3 else 1
    p = cr_params(float(nu), float(mu), CONV[conv], float(lambda_scale))
    h = _vp()
    _check(lib.cr_assemble_coupled(mesh.handle, ctypes.byref(p), _ptr(fbar, np.float64, nrhs * mesh.ne * mesh.dim, "fbar"),
                                   nrhs, _ptr(w, np.float64, mesh.nf * mesh.dim, "w"), ctypes.byref(h),
                                   _ptr(blocks_out, np.float64, None, "blocks_out")))
    return System(h, mesh, nrhs)


def cr_system_set_previous(system, u_prev):
    """Implicit Euler: later hybridisations and recoveries of `system` add the lumped
    mass term of the previous time level u_prev [nrhs, nf, d] (host or device) to the
    right-hand side; None turns it off."""
    n = system.nrhs * system.mesh.nf * system.mesh.dim
    _check(load_library().cr_system_set_previous(system.handle, _ptr(u_prev, np.float64, n, "u_prev")))


def cr_hybridise(system, keep_fp32=True, keep_bf16=False, keep_ff=False, keep_ff_bf16=False):
    """G and S; keep_* select the extra value planes the low-precision solves need."""
    lib = load_library()
    o = cr_hyb_opts(int(bool(keep_fp32)), int(bool(keep_bf16)), int(bool(keep_ff)), int(bool(keep_ff_bf16)))
    h = _vp()
    _check(lib.cr_hybridise(system.handle, ctypes.byref(o), ctypes.byref(h)))
    return Hybrid(h, system)


def cr_hybrid_export(hyb):
    """Block ELL of G (cols [nslot, nf], vals [nslot, d, d, nf]) and S [nrhs, nf, d], as numpy."""
    m = hyb.mesh
    d, nf = m.dim, m.nf
    ns = 2 * d + 1
    cols = np.empty((ns, nf), dtype=np.int32)
    vals = np.empty((ns, d, d, nf), dtype=np.float64)
    S = np.empty((hyb.system.nrhs, nf, d), dtype=np.float64)
    _check(load_library().cr_hybrid_export(hyb.handle, cols.ctypes.data, vals.ctypes.data, S.ctypes.data))
    return cols, vals, S


def make_solve_opts(method="pcg", prec="fp64", tol=1e-10, max_iter=100000, restart=30, inner_tol=0.0,
                    max_outer=60, use_x0=False, check_every=16, use_graph=False, profile=False, persistent=False,
                    precond="jacobi", poly_degree=0, poly_ratio=0.0, poly_prec="same", deflation=None):
    return cr_solve_opts(METHOD[method], PREC[prec], float(tol), int(max_iter), int(restart), float(inner_tol),
                         int(max_outer), int(bool(use_x0)), int(check_every), int(bool(use_graph)),
                         int(bool(profile)), int(bool(persistent)), PRECOND[precond], int(poly_degree),
                         float(poly_ratio), POLY_PREC[poly_prec], deflation.handle if deflation is not None else None)


class Deflation:
    """Owner of a cr_deflation handle (keeps the mesh of the system it was built
    from alive): k vectors of length n."""

    def __init__(self, handle, hyb):
        self.handle, self.mesh = handle, hyb.mesh
        k, n = _i32(), _i64()
        _check(load_library().cr_deflation_info(handle, ctypes.byref(k), ctypes.byref(n)))
        self.k, self.n = int(k.value), int(n.value)

    def vectors(self):
        """The space's vectors (rounded to FP32), float64 [k, n] on the host."""
        V = np.empty((self.k, self.n), dtype=np.float64)
        _check(load_library().cr_deflation_export(self.handle, _ptr(V, np.float64, self.k * self.n, "V")))
        return V

    def __del__(self):
        if getattr(self, "handle", None) and _alive():
            _lib.cr_destroy_deflation(self.handle)
            self.handle = None


def cr_deflation_create(hyb, V):
    """A deflation space of the G of `hyb` from the rows of V (float64 [k, n], host or device)."""
    k = int(V.shape[0])
    h = _vp()
    _check(load_library().cr_deflation_create(hyb.handle, k, _ptr(V, np.float64, k * hyb.n, "V"), ctypes.byref(h)))
    return Deflation(h, hyb)


def cr_deflation_lanczos(hyb, m, k, rhs=0, **opts):
    """A deflation space of k Ritz vectors from m FP64 PCG steps on right-hand side `rhs`
    of `hyb` (preconditioner from opts: precond, poly_degree, poly_ratio).
    Returns (Deflation, Ritz values of the vectors kept)."""
    o = make_solve_opts(**opts)
    theta = (ctypes.c_double * int(k))()
    h = _vp()
    _check(load_library().cr_deflation_lanczos(hyb.handle, int(rhs), ctypes.byref(o), int(m), int(k), theta,
                                               ctypes.byref(h)))
    d = Deflation(h, hyb)
    return d, np.array(theta[:d.k])


def cr_solve(hyb, W, rhs=0, raise_on_error=True, **opts):
    """Solve G W = S for right-hand side `rhs`; W float64 [nf, d] (host or device).

    Returns a dict of statistics (iterations, outer, relres, status)."""
    o = make_solve_opts(**opts)
    st = cr_solve_stats()
    rc = load_library().cr_solve(hyb.handle, int(rhs), ctypes.byref(o), _ptr(W, np.float64, hyb.n, "W"),
                                 ctypes.byref(st))
    stats = {"iterations": st.iterations, "outer": st.outer, "relres": st.relres, "status": st.status,
             "status_name": "CR_OK" if rc == 0 else CR_ERR.get(rc, str(rc)),
             "spmv_launches": st.spmv_launches, "spmv_ms": st.spmv_ms, "kernel_launches": st.kernel_launches}
    if rc != CR_OK:
        stats["error"] = load_library().cr_last_error().decode()
        if raise_on_error:
            _check(rc)
    return stats


def cr_solve_ritz(hyb, W, m, k, rhs=0, raise_on_error=True, **opts):
    """cr_solve that also returns a deflation space of k Ritz vectors from the Lanczos
    record of its first m iterations.  Returns (statistics, Deflation or None, Ritz values)."""
    o = make_solve_opts(**opts)
    st = cr_solve_stats()
    theta = (ctypes.c_double * int(k))()
    h = _vp()
    rc = load_library().cr_solve_ritz(hyb.handle, int(rhs), ctypes.byref(o), _ptr(W, np.float64, hyb.n, "W"),
                                      ctypes.byref(st), int(m), int(k), theta, ctypes.byref(h))
    stats = {"iterations": st.iterations, "outer": st.outer, "relres": st.relres, "status": st.status,
             "status_name": "CR_OK" if rc == 0 else CR_ERR.get(rc, str(rc)),
             "spmv_launches": st.spmv_launches, "spmv_ms": st.spmv_ms, "kernel_launches": st.kernel_launches}
    if rc != CR_OK:
        stats["error"] = load_library().cr_last_error().decode()
        if raise_on_error:
            _check(rc)
    d = Deflation(h, hyb) if h.value else None
    return stats, d, np.array(theta[:d.k]) if d is not None else np.zeros(0)


def cr_solve_preconditioned(hyb, pre, W, rhs=0, raise_on_error=True, **opts):
    """Flexible GMRES on G W = S of `hyb`, preconditioned by inner PCG solves with
    the SPD G of `pre` (same mesh).  opts as for cr_solve; method defaults to
    "gmres" and prec (the inner PCG's precision) to "ff".  Returns the statistics
    (iterations = inner PCG iterations, outer = GMRES steps)."""
    opts.setdefault("method", "gmres")
    opts.setdefault("prec", "ff")
    o = make_solve_opts(**opts)
    st = cr_solve_stats()
    rc = load_library().cr_solve_preconditioned(hyb.handle, int(rhs), pre.handle, ctypes.byref(o),
                                                _ptr(W, np.float64, hyb.n, "W"), ctypes.byref(st))
    stats = {"iterations": st.iterations, "outer": st.outer, "relres": st.relres, "status": st.status,
             "status_name": "CR_OK" if rc == 0 else CR_ERR.get(rc, str(rc)),
             "spmv_launches": st.spmv_launches, "spmv_ms": st.spmv_ms, "kernel_launches": st.kernel_launches}
    if rc != CR_OK and raise_on_error:
        _check(rc)
    return stats


def cr_solve_steady(system, pre, U, P, rhs=0, raise_on_error=True, **opts):
    """The steady problem (system assembled with mu = 0) by flexible GMRES on its
    coupled system, preconditioned by transient Stokes solves with the SPD G of
    `pre` (same mesh, mu > 0).  U float64 [nf*d], P float64 [ne] on the device
    (P_{K_0} = 0).  opts as for cr_solve; method defaults to "gmres", prec (the
    inner PCG's precision) to "ff".  Returns the statistics (iterations = inner
    PCG iterations, outer = GMRES steps, relres = the coupled residual)."""
    opts.setdefault("method", "gmres")
    opts.setdefault("prec", "ff")
    o = make_solve_opts(**opts)
    st = cr_solve_stats()
    n = system.mesh.nf * system.mesh.dim
    rc = load_library().cr_solve_steady(system.handle, pre.handle, int(rhs), ctypes.byref(o),
                                        _ptr(U, np.float64, n, "U"), _ptr(P, np.float64, system.mesh.ne, "P"),
                                        ctypes.byref(st))
    stats = {"iterations": st.iterations, "outer": st.outer, "relres": st.relres, "status": st.status,
             "status_name": "CR_OK" if rc == 0 else CR_ERR.get(rc, str(rc)),
             "spmv_launches": st.spmv_launches, "spmv_ms": st.spmv_ms, "kernel_launches": st.kernel_launches}
    if rc != CR_OK:
        stats["error"] = load_library().cr_last_error().decode()
        if raise_on_error:
            _check(rc)
    return stats


def cr_solve_newton(mesh, nu, fbar, pre, U, P, newton_tol=5e-7, max_newton=20, raise_on_error=True, **opts):
    """Newton's method for the steady Navier-Stokes problem (2D), each step a
    cr_solve_steady solve of the system linearised about the current U.  U and P
    (device) hold the start on entry and the last iterate on exit; fbar
    float64 [ne, 2] host or device.  opts: the linear solves' options (as for
    cr_solve_steady).  Returns the Newton statistics."""
    opts.setdefault("method", "gmres")
    opts.setdefault("prec", "ff")
    o = make_solve_opts(**opts)
    st = cr_newton_stats()
    rc = load_library().cr_solve_newton(mesh.handle, float(nu), _ptr(fbar, np.float64, mesh.ne * mesh.dim, "fbar"),
                                        pre.handle, ctypes.byref(o), float(newton_tol), int(max_newton),
                                        _ptr(U, np.float64, mesh.nf * mesh.dim, "U"), _ptr(P, np.float64, mesh.ne, "P"),
                                        ctypes.byref(st))
    stats = {k: getattr(st, k) for k, _ in cr_newton_stats._fields_}
    stats["status_name"] = "CR_OK" if rc == 0 else CR_ERR.get(rc, str(rc))
    if rc != CR_OK:
        stats["error"] = load_library().cr_last_error().decode()
        if raise_on_error:
            _check(rc)
    return stats


class Coupled:
    """Owner of a cr_coupled handle (keeps its system alive)."""

    def __init__(self, handle, system):
        self.handle, self.system, self.mesh = handle, system, system.mesh

    def __del__(self):
        if getattr(self, "handle", None) and _alive():
            _lib.cr_destroy_coupled(self.handle)
            self.handle = None


def cr_coupled_create(system):
    """A, D_K, R and the diagonal preconditioner of the coupled system (no hybridisation)."""
    h = _vp()
    _check(load_library().cr_coupled_create(system.handle, ctypes.byref(h)))
    return Coupled(h, system)


def cr_solve_coupled(cpl, U, P, rhs=0, raise_on_error=True, **opts):
    """MINRES on the coupled system; U [nf, d] and P [ne] device float64 (P_{K_0} = 0)."""
    opts.setdefault("method", "pcg")
    o = make_solve_opts(**opts)
    st = cr_solve_stats()
    m = cpl.mesh
    rc = load_library().cr_solve_coupled(cpl.handle, int(rhs), ctypes.byref(o), _ptr(U, np.float64, m.nf * m.dim, "U"),
                                         _ptr(P, np.float64, m.ne, "P"), ctypes.byref(st))
    stats = {"iterations": st.iterations, "outer": st.outer, "relres": st.relres, "status": st.status,
             "status_name": "CR_OK" if rc == 0 else CR_ERR.get(rc, str(rc)), "kernel_launches": st.kernel_launches}
    if rc != CR_OK and raise_on_error:
        _check(rc)
    return stats


def cr_apply_G(hyb, x, y):
    _check(load_library().cr_apply_G(hyb.handle, _ptr(x, np.float64, hyb.n, "x"), _ptr(y, np.float64, hyb.n, "y")))


def cr_recover_up(hyb, W, U, P, rhs=0, normalise_p=True, jump=False):
    """Recover U [nf, d] and P [ne] from W; returns max |Û_K - Û_L| when jump is set."""
    j = ctypes.c_double(0.0)
    _check(load_library().cr_recover_up(hyb.handle, int(rhs), _ptr(W, np.float64, hyb.n, "W"),
                                        _ptr(U, np.float64, hyb.n, "U"), _ptr(P, np.float64, hyb.mesh.ne, "P"),
                                        int(bool(normalise_p)), ctypes.byref(j) if jump else None))
    return j.value if jump else None


class Batch:
    """Owner of a cr_batch handle (keeps its problems alive)."""

    def __init__(self, handle, probs):
        self.handle, self.probs = handle, list(probs)

    def info(self):
        v = [_i32() for _ in range(4)]
        _check(load_library().cr_batch_info(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(("nsys", "ntiles", "grid", "blocks_per_sm"), (x.value for x in v)))

    def __del__(self):
        if getattr(self, "handle", None) and _alive():
            _lib.cr_destroy_batch(self.handle)
            self.handle = None


def cr_batch_create(probs, prec="ff", autotune=False, blocks_per_sm=0, rhs_grouping=0):
    """Plan one persistent batched PCG over the hybridised problems `probs`
    (rhs_grouping 1: right-hand sides of a problem share G; 2: one system per pair; 3: one system
    per two right-hand sides)."""
    arr = (_vp * len(probs))(*[h.handle for h in probs])
    o = cr_batch_opts(PREC[prec], int(bool(autotune)), int(blocks_per_sm), int(rhs_grouping))
    h = _vp()
    _check(load_library().cr_batch_create(arr, len(probs), ctypes.byref(o), ctypes.byref(h)))
    return Batch(h, probs)


def cr_solve_batched(batch, Ws, raise_on_error=True, **opts):
    """Solve all (problem, rhs) pairs; Ws: one device tensor [nrhs*nf*d] per problem.
    Returns a list of per-pair statistics (problem-major)."""
    o = make_solve_opts(**opts)
    npairs = sum(h.system.nrhs for h in batch.probs)
    st = (cr_solve_stats * npairs)()
    ptrs = (_vp * len(Ws))(*[_ptr(W, np.float64, h.system.nrhs * h.n, "W") for W, h in zip(Ws, batch.probs)])
    rc = load_library().cr_solve_batched(batch.handle, ctypes.byref(o), ptrs, st)
    out = [{"iterations": s.iterations, "outer": s.outer, "relres": s.relres, "status": s.status,
            "spmv_launches": s.spmv_launches, "spmv_ms": s.spmv_ms, "kernel_launches": s.kernel_launches}
           for s in st]
    if rc != CR_OK and raise_on_error:
        _check(rc)
    return out


CHEB_STEP_FORMS = ("rows1", "rows2", "staged")


def cr_chebyshev_step_form(dim, poly_prec):
    """Name of the Chebyshev step kernel form cr_solve runs for FP32/BF16 steps:
    'rows1' (one face row per thread), 'rows2' (two) or 'staged' (slices staged in
    shared memory by TMA bulk copies)."""
    rc = load_library().cr_chebyshev_step_form(int(dim), POLY_PREC[poly_prec])
    _check(rc if rc < 0 else 0)
    return CHEB_STEP_FORMS[rc]


def cr_residual_noalloc_max_rows():
    return int(load_library().cr_residual_noalloc_max_rows())


def cr_residual_noalloc(dim, nf, cols, vals, b, x, r=None, stream=None, check_sizes=True):
    """r = b - G x and (||r||^2, ||b||^2) without any device allocation.

    For callers that cannot allocate device memory: the library's only scratch
    is a fixed device array.  cols int32 [nslot, nf] and vals float64
    [nslot, dim, dim, nf] in the layout of cr_hybrid_export; b, x, r float64
    [nf*dim]; all on the device.  Returns the two squared norms."""
    nslot = int(cols.shape[0]) if len(cols.shape) == 2 else 2 * dim + 1
    ns = (lambda k: k) if check_sizes else (lambda k: None)
    norms = np.zeros(2, dtype=np.float64)
    rc = load_library().cr_residual_noalloc(
        int(dim), int(nf), nslot, _ptr(cols, np.int32, ns(nslot * nf), "cols"),
        _ptr(vals, np.float64, ns(nslot * dim * dim * nf), "vals"), _ptr(b, np.float64, ns(nf * dim), "b"),
        _ptr(x, np.float64, ns(nf * dim), "x"), _ptr(r, np.float64, ns(nf * dim), "r"), norms.ctypes.data,
        _stream_handle(stream))
    _check(rc)
    return float(norms[0]), float(norms[1])


def ell_to_csr(cols, vals):
    """Scalar CSR matrix (scipy) of a block ELL export, zero entries dropped."""
    import scipy.sparse as sp
    ns, d, _, nf = vals.shape
    di = np.arange(d)
    rows = np.broadcast_to(np.arange(nf)[None, None, None, :] * d + di[None, :, None, None], vals.shape)
    colsx = np.broadcast_to(cols[:, None, None, :].astype(np.int64) * d + di[None, None, :, None], vals.shape)
    keep = vals != 0.0
    return sp.coo_matrix((vals[keep], (rows[keep], colsx[keep])), shape=(nf * d, nf * d)).tocsr()
