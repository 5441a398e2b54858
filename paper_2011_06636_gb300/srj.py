"""ctypes binding of libsrj.so (include/srj.h), same names as the C ABI.

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device arrays are passed as raw pointers (``tensor.data_ptr()``);
PyTorch is used by callers for device memory and streams only.  Importing
this module loads the library and raises if it is missing -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

SRJ_OK, SRJ_EINVAL, SRJ_ENOMEM, SRJ_ECUDA, SRJ_ENOTCONV, SRJ_EDIVERGED, SRJ_ETIMEOUT, \
    SRJ_EUNSUPPORTED = range(8)
STATUS_NAMES = ["SRJ_OK", "SRJ_EINVAL", "SRJ_ENOMEM", "SRJ_ECUDA", "SRJ_ENOTCONV",
                "SRJ_EDIVERGED", "SRJ_ETIMEOUT", "SRJ_EUNSUPPORTED"]
SRJ_SEL_HEURISTIC, SRJ_SEL_INCREASING, SRJ_SEL_FIXED, SRJ_SEL_MLP, SRJ_SEL_JACOBI = range(5)
SRJ_PREC_F64, SRJ_PREC_F32, SRJ_PREC_MIXED = range(3)
SRJ_TOL_REL, SRJ_TOL_ABS, SRJ_TOL_DINF = range(3)
SRJ_BC_DIRICHLET, SRJ_BC_NEUMANN = range(2)

# every entry point include/srj.h declares
EXPORTS = ["srj_version", "srj_level_m", "srj_scheme_omegas", "srj_create", "srj_solve",
           "srj_solve_host", "srj_run_levels", "srj_residual_norm", "srj_get_trace",
           "srj_create_batched", "srj_solve_batched", "srj_mlp_set_weights", "srj_mlp_forward",
           "srj_mlp_train", "srj_residual_norm_noalloc", "srj_mg_create", "srj_mg_solve",
           "srj_collect_moves", "srj_set_wait_limit", "srj_last_error", "srj_destroy"]


class srj_move_record(C.Structure):
    _fields_ = [("prev_ratio", C.c_double), ("r_before", C.c_double), ("r_after", C.c_double),
                ("level", C.c_int32), ("action", C.c_int32)]


# numpy view of an array of srj_move_record (same layout)
MOVE_RECORD_DTYPE = [("prev_ratio", "<f8"), ("r_before", "<f8"), ("r_after", "<f8"),
                     ("level", "<i4"), ("action", "<i4")]


class srj_grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int64 * 3), ("h", C.c_double * 3),
                ("bc", C.c_int32 * 3)]


class srj_stencil(C.Structure):
    _fields_ = [("eps", C.c_double * 3), ("k", C.c_void_p), ("a_diag", C.c_void_p),
                ("a_off", C.c_void_p * 3)]


class srj_opts(C.Structure):
    _fields_ = [("selector", C.c_int32), ("precision", C.c_int32), ("tol_kind", C.c_int32),
                ("level0", C.c_int32), ("fixed_level", C.c_int32), ("max_level", C.c_int32),
                ("temporal_depth", C.c_int32), ("trace_capacity", C.c_int32),
                ("max_sweeps", C.c_int64), ("inner_tol", C.c_double)]


class srj_mg_opts(C.Structure):
    _fields_ = [("smoother_level", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("max_cycles", C.c_int32)]


class srj_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("final_level", C.c_int32), ("sweeps", C.c_int64),
                ("cycles", C.c_int64), ("outer", C.c_int64), ("passes", C.c_int64),
                ("r0", C.c_double), ("rn", C.c_double), ("seconds", C.c_double),
                ("inner_seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsrj.so (building it in-tree with nvcc if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError("libsrj.so is not built: run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(path)
    H = C.c_void_p
    L.srj_version.restype = C.c_char_p
    L.srj_level_m.argtypes = [C.c_int32]
    L.srj_level_m.restype = C.c_int32
    L.srj_scheme_omegas.argtypes = [C.c_int32, C.POINTER(C.c_double), C.c_int32]
    L.srj_scheme_omegas.restype = C.c_int32
    L.srj_create.argtypes = [C.POINTER(srj_grid), C.POINTER(srj_stencil), C.POINTER(srj_opts),
                             C.c_void_p, C.POINTER(H)]
    L.srj_create.restype = C.c_int
    L.srj_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(srj_stats)]
    L.srj_solve.restype = C.c_int
    L.srj_solve_host.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(srj_stats)]
    L.srj_solve_host.restype = C.c_int
    L.srj_run_levels.argtypes = [H, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_int64,
                                 C.POINTER(C.c_double)]
    L.srj_run_levels.restype = C.c_int
    L.srj_residual_norm.argtypes = [H, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    L.srj_residual_norm.restype = C.c_int
    L.srj_get_trace.argtypes = [H, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_int64]
    L.srj_get_trace.restype = C.c_int64
    L.srj_create_batched.argtypes = [C.c_int32, C.POINTER(srj_grid), C.POINTER(srj_stencil),
                                     C.POINTER(srj_opts), C.c_void_p, C.POINTER(H)]
    L.srj_create_batched.restype = C.c_int
    L.srj_solve_batched.argtypes = [H, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double,
                                    C.POINTER(srj_stats)]
    L.srj_solve_batched.restype = C.c_int
    L.srj_mlp_set_weights.argtypes = [H, C.c_void_p, C.c_int64]
    L.srj_mlp_set_weights.restype = C.c_int
    L.srj_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    L.srj_mlp_forward.restype = C.c_int
    L.srj_mlp_train.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                C.c_int32, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]
    L.srj_mlp_train.restype = C.c_int
    L.srj_last_error.argtypes = [H]
    L.srj_last_error.restype = C.c_char_p
    L.srj_mg_create.argtypes = [C.POINTER(srj_grid), C.POINTER(srj_stencil),
                                C.POINTER(srj_mg_opts), C.c_void_p, C.POINTER(H)]
    L.srj_mg_create.restype = C.c_int
    L.srj_mg_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(srj_stats)]
    L.srj_mg_solve.restype = C.c_int
    L.srj_collect_moves.argtypes = [C.c_int64, C.c_void_p, C.c_double, C.c_int32, C.c_uint64,
                                    C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_void_p]
    L.srj_collect_moves.restype = C.c_int
    L.srj_set_wait_limit.argtypes = [H, C.c_int64]
    L.srj_set_wait_limit.restype = C.c_int
    L.srj_destroy.argtypes = [H]
    L.srj_destroy.restype = C.c_int
    _lib = L
    return L


class SrjError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s%s" % (name, (": " + msg) if msg else ""))


def srj_version() -> str:
    return load().srj_version().decode()


def srj_level_m(level: int) -> int:
    return load().srj_level_m(level)


def srj_scheme_omegas(level: int):
    import numpy as np
    out = np.zeros(2362)
    m = load().srj_scheme_omegas(level, out.ctypes.data_as(C.POINTER(C.c_double)), 2362)
    if m < 0:
        raise SrjError(SRJ_EINVAL, "bad level")
    return out[:m].copy()


def _grid(n, h=None, bc=None):
    g = srj_grid()
    g.dim = len(n)
    for a in range(3):
        g.n[a] = int(n[a]) if a < len(n) else 1
        g.h[a] = float(h[a]) if (h is not None and a < len(n)) else 0.0
        g.bc[a] = int(bc[a]) if (bc is not None and a < len(n)) else SRJ_BC_DIRICHLET
    return g


def srj_create(n, h=None, eps=None, k_ptr=None, selector=SRJ_SEL_HEURISTIC,
               precision=SRJ_PREC_F64, tol_kind=SRJ_TOL_REL, level0=0, fixed_level=0,
               max_level=0, temporal_depth=0, trace_capacity=0, max_sweeps=0, inner_tol=0.0,
               stream=None, bc=None, a_diag_ptr=None, a_off_ptrs=None):
    """Returns an opaque handle (int).  ``k_ptr`` is a device pointer (int) or None;
    ``bc`` lists SRJ_BC_* per axis (None: Dirichlet); ``a_diag_ptr`` and
    ``a_off_ptrs`` (device pointers) give an explicit symmetric operator."""
    L = load()
    g = _grid(n, h, bc)
    st = srj_stencil()
    for a in range(3):
        st.eps[a] = float(eps[a]) if (eps is not None and a < len(eps)) else 0.0
    st.k = k_ptr
    st.a_diag = a_diag_ptr
    for a, p in enumerate(a_off_ptrs or []):
        st.a_off[a] = p
    o = srj_opts(selector, precision, tol_kind, level0, fixed_level, max_level, temporal_depth,
                 trace_capacity, max_sweeps, inner_tol)
    hnd = C.c_void_p()
    rc = L.srj_create(C.byref(g), C.byref(st), C.byref(o), stream, C.byref(hnd))
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_create")
    return hnd.value


def _check(h, rc, what):
    if rc not in (SRJ_OK,):
        raise SrjError(rc, "%s: %s" % (what, load().srj_last_error(h).decode()))


def srj_solve(h, f_ptr, u_ptr, tol, raise_on_notconv=False):
    s = srj_stats()
    rc = load().srj_solve(h, f_ptr, u_ptr, float(tol), C.byref(s))
    if rc in (SRJ_ENOTCONV, SRJ_EDIVERGED) and not raise_on_notconv:
        return s.as_dict()
    _check(h, rc, "srj_solve")
    return s.as_dict()


def srj_solve_host(h, f_host_ptr, u_host_ptr, tol, raise_on_notconv=False):
    s = srj_stats()
    rc = load().srj_solve_host(h, f_host_ptr, u_host_ptr, float(tol), C.byref(s))
    if rc in (SRJ_ENOTCONV, SRJ_EDIVERGED) and not raise_on_notconv:
        return s.as_dict()
    _check(h, rc, "srj_solve_host")
    return s.as_dict()


def srj_run_levels(h, f_ptr, u_ptr, levels):
    import numpy as np
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    rn = np.zeros(len(lv))
    rc = load().srj_run_levels(h, f_ptr, u_ptr, lv.ctypes.data_as(C.POINTER(C.c_int32)), len(lv),
                               rn.ctypes.data_as(C.POINTER(C.c_double)))
    _check(h, rc, "srj_run_levels")
    return rn


def srj_residual_norm(h, f_ptr, u_ptr) -> float:
    out = C.c_double()
    rc = load().srj_residual_norm(h, f_ptr, u_ptr, C.byref(out))
    _check(h, rc, "srj_residual_norm")
    return out.value


def srj_get_trace(h, capacity=100000):
    import numpy as np
    lv = np.zeros(capacity, dtype=np.int32)
    rn = np.zeros(capacity)
    n = load().srj_get_trace(h, lv.ctypes.data_as(C.POINTER(C.c_int32)),
                             rn.ctypes.data_as(C.POINTER(C.c_double)), capacity)
    if n < 0:
        raise SrjError(SRJ_EINVAL, "srj_get_trace")
    m = min(n, capacity)
    return lv[:m].copy(), rn[:m].copy()


def srj_create_batched(ns, eps=None, selector=SRJ_SEL_HEURISTIC, tol_kind=SRJ_TOL_REL,
                       level0=0, max_level=0, temporal_depth=0, max_sweeps=0, inner_tol=0.0,
                       stream=None):
    """ns: list of [nx, ny]; eps: list of [eps_x, eps_y] or None.  Mixed precision."""
    L = load()
    n = len(ns)
    grids = (srj_grid * n)(*[_grid(v) for v in ns])
    sts = (srj_stencil * n)()
    for i in range(n):
        for a in range(2):
            sts[i].eps[a] = float(eps[i][a]) if eps is not None else 0.0
        sts[i].k = None
    o = srj_opts(selector, SRJ_PREC_MIXED, tol_kind, level0, 0, max_level, temporal_depth, 0,
                 max_sweeps, inner_tol)
    hnd = C.c_void_p()
    rc = L.srj_create_batched(n, grids, sts, C.byref(o), stream, C.byref(hnd))
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_create_batched")
    return hnd.value


def srj_solve_batched(h, f_ptrs, u_ptrs, tol):
    """f_ptrs, u_ptrs: lists of device pointers.  Returns (status, [stats dict])."""
    n = len(f_ptrs)
    fa = (C.c_void_p * n)(*f_ptrs)
    ua = (C.c_void_p * n)(*u_ptrs)
    st = (srj_stats * n)()
    rc = load().srj_solve_batched(h, fa, ua, float(tol), st)
    if rc not in (SRJ_OK, SRJ_ENOTCONV, SRJ_EDIVERGED):
        _check(h, rc, "srj_solve_batched")
    return rc, [st[i].as_dict() for i in range(n)]


def srj_mlp_set_weights(h, w_bits):
    """w_bits: numpy uint16 array of 6617 BF16 bit patterns."""
    import numpy as np
    w = np.ascontiguousarray(w_bits, dtype=np.uint16)
    rc = load().srj_mlp_set_weights(h, w.ctypes.data, w.size)
    _check(h, rc, "srj_mlp_set_weights")


def srj_mlp_forward(w_bits, X):
    """Device inference on host features X (n x 12): (picks, logits)."""
    import numpy as np
    w = np.ascontiguousarray(w_bits, dtype=np.uint16)
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    pick = np.zeros(n, dtype=np.int32)
    logits = np.zeros((n, 25), dtype=np.float32)
    rc = load().srj_mlp_forward(w.ctypes.data, X.ctypes.data, n, pick.ctypes.data,
                                logits.ctypes.data)
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_mlp_forward")
    return pick, logits


def srj_mlp_train(x_ptr, y_ptr, n, order_ptr, steps, batch, lr, theta_ptr, stream=None):
    """Device pointers in; returns the per-step minibatch losses (numpy)."""
    import numpy as np
    loss = np.zeros(max(int(steps), 1), dtype=np.float32)
    rc = load().srj_mlp_train(x_ptr, y_ptr, n, order_ptr, steps, batch, lr, theta_ptr,
                              loss.ctypes.data, stream)
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_mlp_train")
    return loss[:steps]


def srj_collect_moves(n, f_ptr, tol, max_level, seed, trial0, ntrials, max_steps, out_ptr,
                      counts_ptr, stream=None):
    """Sec. 3 data collection (see include/srj.h); out_ptr / counts_ptr are
    caller-owned device buffers."""
    rc = load().srj_collect_moves(int(n), f_ptr, float(tol), int(max_level), int(seed),
                                  int(trial0), int(ntrials), int(max_steps), out_ptr, counts_ptr,
                                  stream)
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_collect_moves")


def srj_set_wait_limit(h, polls):
    """Polls a bounded device-side wait makes before the solve ends with
    SRJ_ETIMEOUT (negative: the library default)."""
    rc = load().srj_set_wait_limit(h, int(polls))
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_set_wait_limit")


def srj_last_error(h) -> str:
    return load().srj_last_error(h).decode()


def srj_mg_create(n, h=None, eps=None, smoother_level=1, nu1=1, nu2=1, max_cycles=0,
                  stream=None):
    """Multigrid with SRJ smoothing (FP64).  Returns an opaque handle (int)."""
    L = load()
    g = _grid(n, h)
    st = srj_stencil()
    for a in range(3):
        st.eps[a] = float(eps[a]) if (eps is not None and a < len(eps)) else 0.0
    o = srj_mg_opts(smoother_level, nu1, nu2, max_cycles)
    hnd = C.c_void_p()
    rc = L.srj_mg_create(C.byref(g), C.byref(st), C.byref(o), stream, C.byref(hnd))
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_mg_create")
    return hnd.value


def srj_mg_solve(h, f_ptr, u_ptr, tol, raise_on_notconv=False):
    s = srj_stats()
    rc = load().srj_mg_solve(h, f_ptr, u_ptr, float(tol), C.byref(s))
    if rc in (SRJ_ENOTCONV, SRJ_EDIVERGED) and not raise_on_notconv:
        return s.as_dict()
    _check(h, rc, "srj_mg_solve")
    return s.as_dict()


def srj_destroy(h):
    rc = load().srj_destroy(h)
    if rc != SRJ_OK:
        raise SrjError(rc, "srj_destroy")
