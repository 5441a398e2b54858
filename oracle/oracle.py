"""Python wrapper around the plain-C FP64 oracle (``srj_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the correctness reference for the
CUDA library; it shares no code with it.  Only ``tests/``, the smoke check in
``__graft_entry__.py`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It compiles the C file with the host ``gcc`` on first use
(``-O2``, no ``-march``/``-ffast-math``, so it builds and rounds identically on
x86_64 and aarch64).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsrj_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVEL = 24


_OMP_PATH = os.path.join(_BUILD, "libsrj_oracle_omp.so")
_lib_omp = None


def _compile(out, extra):
    with _lock:
        stale = (not os.path.exists(out)) or (os.path.getmtime(out) < os.path.getmtime(_SRC))
        if stale:
            os.makedirs(_BUILD, exist_ok=True)
            tmp = out + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                                   "-D_DEFAULT_SOURCE"] + extra + ["-o", tmp, _SRC, "-lm"])
            os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsrj_oracle.so``."""
    if force and os.path.exists(_LIB_PATH):
        os.unlink(_LIB_PATH)
    return _compile(_LIB_PATH, [])


def build_omp() -> str:
    """The same source compiled with ``-fopenmp`` (only the sweep's row loop
    carries a pragma; every result is the same as the plain build's).  Used
    to time the CPU baseline on all host cores."""
    return _compile(_OMP_PATH, ["-fopenmp"])


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_long * 3), ("h", C.c_double * 3),
                ("eps", C.c_double * 3), ("k", C.POINTER(C.c_double)), ("bc", C.c_int * 3),
                ("adiag", C.POINTER(C.c_double)), ("aoff", C.POINTER(C.c_double) * 3)]


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def omp_lib():
    """The OpenMP build (see build_omp); its thread count follows
    OMP_NUM_THREADS, default all host cores."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _declare(C.CDLL(build_omp()))
    return _lib_omp


def _declare(L):
    """Argument and result types of the oracle's C functions."""
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    lp = C.POINTER(C.c_long)
    pp = C.POINTER(_Problem)
    L.oracle_level_m.argtypes = [C.c_int]
    L.oracle_level_m.restype = C.c_int
    L.oracle_lambda_star.argtypes = [C.c_int]
    L.oracle_lambda_star.restype = C.c_double
    L.oracle_scheme_root_order.argtypes = [C.c_int, dp, dp]
    L.oracle_leja_order.argtypes = [C.c_int, dp, ip]
    L.oracle_level_omegas.argtypes = [C.c_int, dp]
    L.oracle_level_omegas.restype = C.c_int
    L.oracle_amplification.argtypes = [C.c_int, dp, C.c_double]
    L.oracle_amplification.restype = C.c_double
    L.oracle_apply_A.argtypes = [pp, dp, dp]
    L.oracle_diagonal.argtypes = [pp, dp]
    L.oracle_residual_norm.argtypes = [pp, dp, dp]
    L.oracle_residual_norm.restype = C.c_double
    L.oracle_sweep.argtypes = [pp, dp, dp, C.c_double, dp]
    L.oracle_sweeps.argtypes = [pp, dp, dp, dp, C.c_long]
    L.oracle_next_level.argtypes = [C.c_int, C.c_double, C.c_int]
    L.oracle_next_level.restype = C.c_int
    L.oracle_srj_solve.argtypes = [pp, dp, dp, C.c_double, C.c_int, C.c_int,
                                   C.c_int, C.c_long, lp, lp, dp, dp, ip,
                                   dp, C.c_long]
    L.oracle_srj_solve.restype = C.c_int
    L.oracle_srj_run_levels.argtypes = [pp, dp, dp, ip, C.c_long, dp]
    L.oracle_jacobi_solve.argtypes = [pp, dp, dp, C.c_double, C.c_int,
                                      C.c_long, C.c_long, lp, dp]
    L.oracle_jacobi_solve.restype = C.c_int
    L.oracle_thomas.argtypes = [C.c_long, dp, dp, dp, dp, dp]
    L.oracle_mg_restrict.argtypes = [pp, dp, pp, dp]
    L.oracle_mg_prolong_add.argtypes = [pp, dp, pp, dp]
    L.oracle_mg_vcycle.argtypes = [pp, dp, dp, C.c_int, C.c_int, C.c_int]
    L.oracle_mg_solve.argtypes = [pp, dp, dp, C.c_double, C.c_int, C.c_int, C.c_int,
                                  C.c_long, lp, dp, dp, dp]
    L.oracle_mg_solve.restype = C.c_int
    L.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    L.oracle_splitmix64.restype = C.c_uint64
    L.oracle_pick.argtypes = [C.c_uint64, C.c_long, C.c_long, C.c_int]
    L.oracle_pick.restype = C.c_int
    L.oracle_collect_moves.argtypes = [pp, dp, C.c_double, C.c_int, C.c_uint64, C.c_long,
                                       C.c_long, dp, ip, ip, dp, dp, lp, ip]
    L.oracle_collect_moves.restype = C.c_long
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Structured-grid problem A u = f.

    ``n`` lists sizes per axis with x first (x varies fastest in the flattened
    arrays).  ``adiag`` / ``aoff`` (one array per axis), when given, define an
    explicit symmetric operator instead (A_pp = adiag[p], A_{p,p+e_a} =
    A_{p+e_a,p} = aoff[a][p]; Sec. 4.1's random tridiagonal systems).  ``bc`` per axis: 0 zero Dirichlet (n interior points), 1
    homogeneous Neumann by a mirrored ghost node (n nodes including both ends,
    Sec. 4.2.2); default all Dirichlet.  ``h`` defaults to the unit domain,
    1/(n+1) on a Dirichlet axis and 1/(n-1) on a Neumann axis, ``eps`` to 1 per
    axis, ``k`` (cell coefficient with one ghost layer, shape reversed from
    ``n`` i.e. (..., n1+2, n0+2)) to None (constant).
    """

    def __init__(self, n, h=None, eps=None, k=None, bc=None, adiag=None, aoff=None):
        n = [int(v) for v in n]
        # explicit symmetric operator: A_pp = adiag[p], A_{p,p+e_a} = aoff[a][p]
        self.adiag = None if adiag is None else _f64(adiag).ravel()
        self.aoff = None if aoff is None else [_f64(v).ravel() for v in aoff]
        self.dim = len(n)
        self.n = n
        self.bc = [0] * self.dim if bc is None else [int(v) for v in bc]
        if h is None:  # unit domain: interior points (Dirichlet) or all nodes (Neumann)
            self.h = [1.0 / (v - 1) if b == 1 else 1.0 / (v + 1) for v, b in zip(n, self.bc)]
        else:
            self.h = [float(v) for v in h]
        self.eps = [1.0] * self.dim if eps is None else [float(v) for v in eps]
        self.k = None if k is None else _f64(k)
        self.size = int(np.prod(n))

    def _c(self):
        s = _Problem()
        s.dim = self.dim
        for a in range(3):
            s.n[a] = self.n[a] if a < self.dim else 1
            s.h[a] = self.h[a] if a < self.dim else 1.0
            s.eps[a] = self.eps[a] if a < self.dim else 0.0
        s.k = _dp(self.k) if self.k is not None else C.POINTER(C.c_double)()
        for a in range(3):
            s.bc[a] = self.bc[a] if a < self.dim else 0
        if self.adiag is not None:
            s.adiag = _dp(self.adiag)
            for a in range(self.dim):
                s.aoff[a] = _dp(self.aoff[a])
        self._keep = s
        return C.byref(s)


def level_m(level: int) -> int:
    return lib().oracle_level_m(level)


def lambda_star(M: int) -> float:
    return lib().oracle_lambda_star(M)


def scheme_root_order(M: int):
    x = np.zeros(M)
    w = np.zeros(M)
    lib().oracle_scheme_root_order(M, _dp(x), _dp(w))
    return x, w


def leja_order(M: int, x) -> np.ndarray:
    x = _f64(x)
    o = np.zeros(M, dtype=np.int32)
    lib().oracle_leja_order(M, _dp(x), o.ctypes.data_as(C.POINTER(C.c_int)))
    return o


def level_omegas(level: int) -> np.ndarray:
    w = np.zeros(2362)
    M = lib().oracle_level_omegas(level, _dp(w))
    return w[:M].copy()


def amplification(omega, lam: float) -> float:
    omega = _f64(omega)
    return lib().oracle_amplification(len(omega), _dp(omega), float(lam))


def apply_A(P: Problem, u):
    u = _f64(u).ravel()
    out = np.zeros(P.size)
    lib().oracle_apply_A(P._c(), _dp(u), _dp(out))
    return out


def diagonal(P: Problem):
    out = np.zeros(P.size)
    lib().oracle_diagonal(P._c(), _dp(out))
    return out


def residual_norm(P: Problem, u, f) -> float:
    u = _f64(u).ravel()
    f = _f64(f).ravel()
    return lib().oracle_residual_norm(P._c(), _dp(u), _dp(f))


def sweep(P: Problem, u, f, omega: float):
    u = _f64(u).ravel()
    f = _f64(f).ravel()
    out = np.zeros(P.size)
    lib().oracle_sweep(P._c(), _dp(u), _dp(f), float(omega), _dp(out))
    return out


def sweeps(P: Problem, u, f, omegas, parallel=False):
    """Apply the factors in order.  parallel=True runs the OpenMP build
    (same arithmetic, rows shared among the host threads)."""
    u = _f64(u).ravel().copy()
    f = _f64(f).ravel()
    w = _f64(omegas)
    (omp_lib() if parallel else lib()).oracle_sweeps(P._c(), _dp(u), _dp(f), _dp(w), len(w))
    return u


def next_level(rule: int, ratio: float, level: int) -> int:
    return lib().oracle_next_level(rule, float(ratio), level)


RULES = {"heuristic": 0, "increasing": 1, "fixed": 2}
TOL_KINDS = {"rel": 0, "abs": 1, "dinf": 2}


def srj_solve(P: Problem, f, u0=None, tol=1e-8, tol_kind="rel",
              rule="heuristic", level0=0, max_sweeps=10**7, trace_cap=100000):
    f = _f64(f).ravel()
    u = np.zeros(P.size) if u0 is None else _f64(u0).ravel().copy()
    sw = C.c_long()
    cy = C.c_long()
    r0 = C.c_double()
    rn = C.c_double()
    tl = np.zeros(trace_cap, dtype=np.int32)
    tr = np.zeros(trace_cap)
    st = lib().oracle_srj_solve(P._c(), _dp(f), _dp(u), float(tol),
                                TOL_KINDS[tol_kind], RULES[rule],
                                int(level0), int(max_sweeps), C.byref(sw),
                                C.byref(cy), C.byref(r0), C.byref(rn),
                                tl.ctypes.data_as(C.POINTER(C.c_int)), _dp(tr),
                                trace_cap)
    nc = min(cy.value, trace_cap)
    return dict(u=u, status=st, sweeps=sw.value, cycles=cy.value, r0=r0.value,
                rn=rn.value, levels=tl[:nc].copy(), rns=tr[:nc].copy())


def run_levels(P: Problem, f, u0, levels):
    f = _f64(f).ravel()
    u = _f64(u0).ravel().copy()
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    rns = np.zeros(len(lv))
    lib().oracle_srj_run_levels(P._c(), _dp(f), _dp(u),
                                lv.ctypes.data_as(C.POINTER(C.c_int)), len(lv),
                                _dp(rns))
    return u, rns


def jacobi_solve(P: Problem, f, u0=None, tol=1e-8, tol_kind="rel",
                 check_every=1, max_sweeps=10**7):
    f = _f64(f).ravel()
    u = np.zeros(P.size) if u0 is None else _f64(u0).ravel().copy()
    sw = C.c_long()
    rn = C.c_double()
    st = lib().oracle_jacobi_solve(P._c(), _dp(f), _dp(u), float(tol), TOL_KINDS[tol_kind],
                                   int(check_every), int(max_sweeps),
                                   C.byref(sw), C.byref(rn))
    return dict(u=u, status=st, sweeps=sw.value, rn=rn.value)


def thomas(a, b, c, d):
    a, b, c, d = (_f64(v) for v in (a, b, c, d))
    x = np.zeros(len(b))
    lib().oracle_thomas(len(b), _dp(a), _dp(b), _dp(c), _dp(d), _dp(x))
    return x


def mg_coarse(P: Problem) -> Problem:
    """The next coarser multigrid problem: (n - 1) / 2 points, twice the spacing."""
    return Problem([(v - 1) // 2 for v in P.n], h=[2 * v for v in P.h], eps=P.eps)


def mg_restrict(P: Problem, r):
    Pc = mg_coarse(P)
    r = _f64(r).ravel()
    out = np.zeros(Pc.size)
    lib().oracle_mg_restrict(P._c(), _dp(r), Pc._c(), _dp(out))
    return out


def mg_prolong_add(Pc: Problem, ec, P: Problem, u):
    ec = _f64(ec).ravel()
    u = _f64(u).ravel().copy()
    lib().oracle_mg_prolong_add(Pc._c(), _dp(ec), P._c(), _dp(u))
    return u


def mg_vcycle(P: Problem, u, f, level=0, nu1=1, nu2=1):
    u = _f64(u).ravel().copy()
    f = _f64(f).ravel()
    lib().oracle_mg_vcycle(P._c(), _dp(u), _dp(f), int(level), int(nu1), int(nu2))
    return u


def mg_solve(P: Problem, f, u0=None, tol=1e-8, level=0, nu1=1, nu2=1, max_cycles=200):
    f = _f64(f).ravel()
    u = np.zeros(P.size) if u0 is None else _f64(u0).ravel().copy()
    cy = C.c_long()
    r0 = C.c_double()
    rn = C.c_double()
    tr = np.zeros(max_cycles)
    st = lib().oracle_mg_solve(P._c(), _dp(f), _dp(u), float(tol), int(level), int(nu1), int(nu2),
                               int(max_cycles), C.byref(cy), C.byref(r0), C.byref(rn), _dp(tr))
    return dict(u=u, status=st, cycles=cy.value, r0=r0.value, rn=rn.value,
                rns=tr[:cy.value].copy())


def splitmix64(seed: int, index: int) -> int:
    return lib().oracle_splitmix64(seed, index)


def pick(seed: int, trial: int, step: int, ncand: int) -> int:
    return lib().oracle_pick(seed, trial, step, ncand)


def collect_moves(P: Problem, f, tol=1e-8, max_level=24, seed=0, trial=0, max_steps=100000):
    """One trial of the Sec. 3 data collection (see oracle_collect_moves).
    Returns the records (prev_ratio, level, action, r_before, r_after) and
    the levels taken (level 0 of the first cycle, then one per step)."""
    f = _f64(f).ravel()
    cap = 3 * max_steps
    pr = np.zeros(cap)
    lv = np.zeros(cap, dtype=np.int32)
    ac = np.zeros(cap, dtype=np.int32)
    rb = np.zeros(cap)
    ra = np.zeros(cap)
    taken = np.zeros(max_steps + 1, dtype=np.int32)
    nrec = C.c_long()
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    steps = lib().oracle_collect_moves(P._c(), _dp(f), float(tol), int(max_level), int(seed),
                                       int(trial), int(max_steps), _dp(pr), ip(lv), ip(ac),
                                       _dp(rb), _dp(ra), C.byref(nrec), ip(taken))
    n = nrec.value
    return dict(prev_ratio=pr[:n], level=lv[:n], action=ac[:n], r_before=rb[:n],
                r_after=ra[:n], steps=steps, taken=taken[:steps + 1])
