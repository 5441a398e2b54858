"""Pins of the oracle's operator, sweep and SRJ driver against closed forms,
library routines (scipy) and the iteration counts the paper prints."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from conftest import read_golden
from paper_2011_06636_gb300 import inputs


# ---------------------------------------------------------------- operator
def _lap1d(n, h, eps=1.0):
    e = np.ones(n)
    return sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) * (eps / h ** 2)


def _sparse_A(n, h, eps):
    """Kronecker-sum construction of the constant-coefficient operator
    (x is the fastest axis)."""
    dim = len(n)
    A = None
    for a in range(dim):
        mats = []
        for b in reversed(range(dim)):
            mats.append(_lap1d(n[b], h[b], eps[b]) if b == a else sp.identity(n[b]))
        term = mats[0]
        for m in mats[1:]:
            term = sp.kron(term, m)
        A = term if A is None else A + term
    return A.tocsr()


def _sparse_A_vark(n, h, eps, k):
    """-div(k grad u) as G^T K G: G = one-sided differences over every face
    (boundary faces included, zero Dirichlet outside), K = face coefficients
    (harmonic mean of the two cells, the outer one a ghost cell)."""
    dim = len(n)
    N = int(np.prod(n))
    idx = np.arange(N).reshape(tuple(reversed(n)))
    rows_G, cols_G, vals_G, kf = [], [], [], []
    face = 0
    kk = k  # shape reversed(n) + 2
    for a in range(dim):
        ax = dim - 1 - a  # numpy axis of grid axis a
        c = eps[a] / h[a] ** 2
        # faces between cell i-1 and i for i = 0..n[a] (n[a]+1 faces per line)
        shp = list(reversed(n))
        it = np.ndindex(*[shp[t] if t != ax else shp[ax] + 1 for t in range(dim)])
        for pos in it:
            i = pos[ax]
            left = list(pos); left[ax] = i - 1
            right = list(pos)
            kl = kk[tuple(v + 1 for v in left)]
            kr = kk[tuple(v + 1 for v in right)]
            coef = c * 2 * kl * kr / (kl + kr)
            if i - 1 >= 0:
                rows_G.append(face); cols_G.append(idx[tuple(left)]); vals_G.append(-1.0)
            if i < shp[ax]:
                rows_G.append(face); cols_G.append(idx[tuple(right)]); vals_G.append(1.0)
            kf.append(coef)
            face += 1
    G = sp.csr_matrix((vals_G, (rows_G, cols_G)), shape=(face, N))
    return (G.T @ sp.diags(kf) @ G).tocsr()


@pytest.mark.parametrize("n,eps", [([37], [1.0]), ([19, 23], [1.0, 1.0]),
                                   ([21, 17], [0.03, 1.0]), ([7, 9, 11], [1.0, 0.5, 2.0])])
def test_apply_A_matches_sparse_kron(orc, n, eps):
    h = [1.0 / (v + 1) for v in n]
    P = orc.Problem(n, h=h, eps=eps)
    A = _sparse_A(n, h, eps)
    u = np.random.default_rng(1).standard_normal(P.size)
    ref = A @ u
    got = orc.apply_A(P, u)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.allclose(orc.diagonal(P), A.diagonal(), rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [[29], [11, 13], [5, 6, 7]])
def test_apply_A_variable_k_matches_GtKG(orc, n):
    rng = np.random.default_rng(7)
    h = [1.0 / (v + 1) for v in n]
    eps = [1.0, 0.7, 1.3][:len(n)]
    k = np.exp(rng.standard_normal(tuple(v + 2 for v in reversed(n))))
    P = orc.Problem(n, h=h, eps=eps, k=k)
    A = _sparse_A_vark(n, h, eps, k)
    u = rng.standard_normal(P.size)
    ref = A @ u
    got = orc.apply_A(P, u)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.allclose(orc.diagonal(P), A.diagonal(), rtol=1e-13, atol=0)
    # constant k reduces to the constant operator scaled by k
    k3 = np.full_like(k, 3.0)
    P3 = orc.Problem(n, h=h, eps=eps, k=k3)
    Pc = orc.Problem(n, h=h, eps=eps)
    assert np.allclose(orc.apply_A(P3, u), 3.0 * orc.apply_A(Pc, u), rtol=1e-13, atol=1e-9)


def test_sweep_matches_definition_with_sparse_diagonal(orc):
    """Eq. (relaxed-jacobi): x' = omega (B_J x + D^-1 b) + (1 - omega) x with
    B_J = -D^-1 (L+U), built from the scipy matrix."""
    n, eps = [15, 12], [0.2, 1.0]
    h = [1.0 / 16, 1.0 / 13]
    P = orc.Problem(n, h=h, eps=eps)
    A = _sparse_A(n, h, eps)
    D = A.diagonal()
    LU = A - sp.diags(D)
    rng = np.random.default_rng(3)
    x, b = rng.standard_normal(P.size), rng.standard_normal(P.size)
    for w in (0.5, 1.0, 17.8):
        ref = w * (-(LU @ x) / D + b / D) + (1 - w) * x
        got = orc.sweep(P, x, b, w)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_residual_norm_matches_sparse(orc):
    n = [9, 8, 7]
    P = orc.Problem(n)
    A = _sparse_A(n, P.h, P.eps)
    rng = np.random.default_rng(4)
    u, f = rng.standard_normal(P.size), rng.standard_normal(P.size)
    assert abs(orc.residual_norm(P, u, f) - np.linalg.norm(f - A @ u)) <= 1e-12 * np.linalg.norm(f)


# ------------------------------------------------ eigenmode closed form
def _T(M, y):
    return math.cos(M * math.acos(y)) if abs(y) <= 1 else math.cosh(M * math.acosh(y))


def _G_closed(M, lam):
    ls = math.cosh(math.acosh(3.0) / M)
    return _T(M, ((ls + 1) * lam + (ls - 1)) / 2) / 3


@pytest.mark.parametrize("level", [0, 3, 8, 12, 16])
@pytest.mark.parametrize("kmode", [1, 5, 32, 63])
def test_single_eigenmode_decays_by_closed_form_1d(orc, level, kmode):
    """Sec. 2, Eq. (eigen-srj-1/2, amplification-M-scheme): with f = 0 and u0
    a discrete sine mode of the 1D Poisson matrix (Sec. 3), one cycle
    multiplies the mode by G_M(lambda_J), lambda_J = cos(k pi/(N+1))."""
    N = 64
    P = orc.Problem([N])
    i = np.arange(1, N + 1)
    u0 = np.sin(kmode * math.pi * i / (N + 1))
    u, _ = orc.run_levels(P, np.zeros(N), u0, [level])
    g = _G_closed(orc.level_m(level), math.cos(kmode * math.pi / (N + 1)))
    assert np.max(np.abs(u - g * u0)) <= 1e-10 * max(1.0, orc.level_m(level) ** 2 * 1e-3)


@pytest.mark.parametrize("n,eps,modes", [([24, 20], [1.0, 1.0], (3, 17)),
                                         ([24, 20], [0.01, 1.0], (1, 2)),
                                         ([10, 12, 9], [1.0, 0.5, 2.0], (2, 7, 4))])
def test_single_eigenmode_decays_by_closed_form_nd(orc, n, eps, modes):
    P = orc.Problem(n, eps=eps)
    grids = np.meshgrid(*[np.arange(1, v + 1) for v in reversed(n)], indexing="ij")
    u0 = np.ones(tuple(reversed(n)))
    num = den = 0.0
    for a in range(len(n)):
        g = grids[len(n) - 1 - a]
        u0 = u0 * np.sin(modes[a] * math.pi * g / (n[a] + 1))
        c = eps[a] / P.h[a] ** 2
        num += c * math.cos(modes[a] * math.pi / (n[a] + 1))
        den += c
    lam = num / den
    for level in (2, 7, 11):
        u, _ = orc.run_levels(P, np.zeros(P.size), u0.ravel(), [level])
        g = _G_closed(orc.level_m(level), lam)
        assert np.max(np.abs(u - g * u0.ravel())) <= 1e-10


# --------------------------------------------- manufactured / direct solves
def test_manufactured_16_sine_modes_1d(orc):
    """1D N=1024 with f a sum of 16 discrete sine modes: the exact discrete
    solution divides each amplitude by mu_k = (4/h^2) sin^2(k pi h / 2); an SRJ
    solve to relative residual 1e-8 must lie within ||r|| / mu_min of it."""
    N = 1024
    f = inputs.poisson1d_sines(N, seed=0)
    rng = np.random.default_rng(0)
    ks = rng.choice(np.arange(1, N + 1), size=16, replace=False)
    amps = rng.standard_normal(16)
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    ustar = np.zeros(N)
    for a, k in zip(amps, ks):
        ustar += a / (4 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2) * np.sin(k * math.pi * i * h)
    P = orc.Problem([N])
    res = orc.srj_solve(P, f, tol=1e-8)
    assert res["status"] == 0
    assert res["rn"] / res["r0"] < 1e-8
    mu_min = 4 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    assert np.linalg.norm(res["u"] - ustar) <= res["rn"] / mu_min * (1 + 1e-6)


def test_thomas_matches_scipy_banded(orc):
    rng = np.random.default_rng(11)
    N = 50
    a, c = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    b = np.abs(a) + np.abs(c) + rng.uniform(0.5, 1.5, N)
    d = rng.standard_normal(N)
    x = orc.thomas(a, b, c, d)
    ab = np.zeros((3, N))
    ab[0, 1:] = c[:-1]
    ab[1] = b
    ab[2, :-1] = a[1:]
    ref = sla.solve_banded((1, 1), ab, d)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [2, 5, 17, 48])
def test_srj_converges_to_direct_solution(orc, N):
    f = np.random.default_rng(N).standard_normal(N)
    h = 1.0 / (N + 1)
    e = np.ones(N)
    xd = orc.thomas(-e / h ** 2, 2 * e / h ** 2, -e / h ** 2, f)
    res = orc.srj_solve(orc.Problem([N]), f, tol=1e-13)
    assert res["status"] == 0
    assert np.max(np.abs(res["u"] - xd)) <= 1e-10 * np.max(np.abs(xd))


# ------------------------------------------------- the paper's iteration pins
def _golden_kv(name):
    return {r[0]: r[1:] for r in read_golden(name)}


def test_n100_heuristic_pattern_and_counts(orc):
    """Sec. 4.1: N=100, b=1, abs tol 1e-7 -- approximately 1000 iterations,
    levels climb to 11 then alternate 10/11; increasing rule over 3000."""
    g = _golden_kv("sec4_1d_poisson_n100.txt")
    N = int(g["N"][0])
    tol = float(g["tol_abs"][0])
    P = orc.Problem([N])
    res = orc.srj_solve(P, np.ones(N), tol=tol, tol_kind="abs")
    assert res["status"] == 0
    approx = float(g["heuristic_iterations_approx"][0])
    assert 0.9 * approx <= res["sweeps"] <= 1.1 * approx
    lv = list(res["levels"])
    top = int(g["heuristic_max_level"][0])
    assert max(lv) == top
    first_top = lv.index(top)
    assert lv[:first_top + 1] == list(range(top + 1))
    alt = set(int(v) for v in g["heuristic_alternating_levels"])
    assert set(lv[first_top:]) == alt
    assert all(a != b for a, b in zip(lv[first_top:], lv[first_top + 1:]))
    inc = orc.srj_solve(P, np.ones(N), tol=tol, tol_kind="abs", rule="increasing")
    assert inc["status"] == 0
    assert inc["sweeps"] > float(g["increasing_iterations_min"][0])
    assert res["sweeps"] <= 0.5 * inc["sweeps"]


def test_in_sample_heuristic_beats_increasing(orc):
    """Sec. 4.1: over the in-sample sizes the heuristic generally needs at most
    half the iterations of the increasing rule (checked for N >= 50)."""
    for N in (50, 100, 200, 400):
        P = orc.Problem([N])
        a = orc.srj_solve(P, np.ones(N), tol=1e-7, tol_kind="abs")
        b = orc.srj_solve(P, np.ones(N), tol=1e-7, tol_kind="abs", rule="increasing")
        assert a["status"] == 0 and b["status"] == 0
        assert a["sweeps"] <= 0.5 * b["sweeps"], (N, a["sweeps"], b["sweeps"])


def _jacobi_sweeps_closed_form(n, tol):
    """Exact plain-Jacobi sweep count for -lap u = 1 (constant coefficients,
    zero Dirichlet, u0 = 0, relative residual < tol).  With D a multiple of I,
    r_n = B_J^n r_0 and r_0 = f = 1; in the discrete sine basis B_J is diagonal
    with lambda_k = sum_a c_a cos(k_a pi h_a) / sum_a c_a, c_a = 1/h_a^2, and
    the coefficients of 1 come
    from scipy's type-I DST.  Returns the smallest n with ||r_n|| < tol ||r_0||."""
    from scipy.fft import dst
    dim = len(n)
    lam, w = None, None
    ca = [(v + 1.0) ** 2 for v in n]
    for a in range(dim):
        c = dst(np.ones(n[a]), type=1) / (n[a] + 1)
        l1 = np.cos(np.arange(1, n[a] + 1) * math.pi / (n[a] + 1)) * ca[a] / sum(ca)
        shape = [1] * dim
        shape[a] = n[a]
        lam = l1.reshape(shape) if lam is None else lam + l1.reshape(shape)
        w = (c ** 2).reshape(shape) if w is None else w * (c ** 2).reshape(shape)
    lam, w = np.broadcast_arrays(lam, w)
    keep = w > 1e-300
    lam, w = lam[keep], w[keep] / w[keep].sum()
    logl = np.log(np.maximum(np.abs(lam), 1e-300))
    ratio2 = lambda k: np.sum(w * np.exp(2 * k * logl))
    lo, hi = 0, 1
    while ratio2(hi) >= tol * tol:
        hi *= 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if ratio2(mid) >= tol * tol:
            lo = mid
        else:
            hi = mid
    return hi


@pytest.mark.parametrize("n", [[50], [12, 9], [8, 8, 8]])
def test_oracle_jacobi_matches_spectral_count(orc, n):
    P = orc.Problem(n)
    j = orc.jacobi_solve(P, np.ones(P.size), tol=1e-8, check_every=1)
    assert j["status"] == 0
    assert j["sweeps"] == _jacobi_sweeps_closed_form(n, 1e-8)


@pytest.mark.parametrize("side", [32, 48, 64])
def test_table3_3d_speedup_over_jacobi(orc, side):
    """Sec. 4.2.3, Table 3: Jacobi / SRJ+heuristic iteration ratio for 3D
    Poisson, f = 1, relative residual 1e-8, within 15 %.  SRJ from the oracle;
    the Jacobi count from its exact spectral closed form (pinned above)."""
    table = {int(r[0]): float(r[1]) for r in read_golden("table3_speedup.txt")}
    n = [side] * 3
    P = orc.Problem(n)
    s = orc.srj_solve(P, np.ones(P.size), tol=1e-8)
    assert s["status"] == 0
    jac = _jacobi_sweeps_closed_form(n, 1e-8)
    ratio = jac / s["sweeps"]
    assert abs(ratio / table[side] - 1) <= 0.15, (side, jac, s["sweeps"], ratio)


def test_selection_rule_thresholds(orc):
    """Alg. 1 with the strict comparisons as printed: > 0.4 up, in (0.2, 0.4)
    down, otherwise keep; clamped to [0, 24]."""
    nl = orc.next_level
    assert nl(0, 0.41, 5) == 6 and nl(0, 0.4, 5) == 5 and nl(0, 0.3, 5) == 4
    assert nl(0, 0.2, 5) == 5 and nl(0, 0.1, 5) == 5 and nl(0, 0.3, 0) == 0
    assert nl(0, 0.9, 24) == 24 and nl(1, 0.0, 3) == 4 and nl(2, 0.9, 3) == 3


def test_openmp_build_gives_identical_sweeps(orc):
    """The all-cores build that times the CPU baseline runs the same
    arithmetic: every sweep result is bit-identical to the plain build's
    (2D and 3D, several cycles, a ragged grid)."""
    for n in ([97, 61], [23, 17, 29]):
        P = orc.Problem(n)
        f = inputs.uniform_rhs(n, seed=3).ravel()
        u0 = np.random.default_rng(2).standard_normal(f.size)
        w = np.concatenate([orc.level_omegas(l) for l in (0, 3, 6, 9)])
        a = orc.sweeps(P, u0, f, w)
        b = orc.sweeps(P, u0, f, w, parallel=True)
        assert np.array_equal(a, b)
