"""Pins of the oracle's explicit symmetric operator (A_pp = adiag[p],
A_(p,p+e_a) = A_(p+e_a,p) = aoff[a][p]) used for Sec. 4.1's random symmetric
diagonally dominant tridiagonal systems, against scipy and an eigen-
decomposition of the Jacobi iteration, and of the input recipe."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from paper_2011_06636_gb300 import inputs


def _sparse_explicit(n, adiag, aoff):
    N = int(np.prod(n))
    A = sp.diags(adiag).tolil()
    stride = 1
    for a in range(len(n)):
        coords = np.unravel_index(np.arange(N), tuple(reversed(n)))  # (z, y, x)
        ca = coords[len(n) - 1 - a]
        for p in np.nonzero(ca + 1 < n[a])[0]:
            A[p, p + stride] = aoff[a][p]
            A[p + stride, p] = aoff[a][p]
        stride *= n[a]
    return A.tocsr()


@pytest.mark.parametrize("n", [[9], [7, 5], [4, 3, 5]])
def test_explicit_apply_matches_scipy(orc, n):
    rng = np.random.default_rng(len(n))
    N = int(np.prod(n))
    adiag = rng.uniform(1, 2, N)
    aoff = [rng.uniform(-1, 1, N) for _ in n]
    P = orc.Problem(n, adiag=adiag, aoff=aoff)
    u = rng.standard_normal(N)
    A = _sparse_explicit(n, adiag, aoff)
    np.testing.assert_allclose(orc.apply_A(P, u), A @ u, rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(orc.diagonal(P), adiag)
    f = rng.standard_normal(N)
    assert orc.residual_norm(P, u, f) == pytest.approx(np.linalg.norm(f - A @ u), rel=1e-13)


def test_poisson_coefficients_reproduce_constant_operator(orc):
    n = [20, 13]
    h = [1 / 21, 1 / 14]
    c = [1 / h[0] ** 2, 1 / h[1] ** 2]
    N = 20 * 13
    P0 = orc.Problem(n)
    P1 = orc.Problem(n, adiag=np.full(N, 2 * (c[0] + c[1])),
                     aoff=[np.full(N, -c[0]), np.full(N, -c[1])])
    f = inputs.uniform_rhs(n, seed=1).ravel()
    r0 = orc.srj_solve(P0, f, tol=1e-8)
    r1 = orc.srj_solve(P1, f, tol=1e-8)
    np.testing.assert_array_equal(r0["levels"], r1["levels"])
    np.testing.assert_allclose(r1["u"], r0["u"], rtol=0, atol=1e-11 * np.abs(r0["u"]).max())


def _spectral(d, e):
    """S = D^-1/2 A D^-1/2 = Q diag(lam) Q^T for the symmetric tridiagonal A."""
    s = 1 / np.sqrt(d)
    lam, Q = sla.eigh_tridiagonal(d * s * s, e[:-1] * s[:-1] * s[1:])
    return lam, Q, s


def _residual_after(omegas, lam, Q, s, b):
    # u0 = 0: e0 = -x*, r_k = D^1/2 Q [lam prod(1 - w lam)] Q^T D^1/2 e0 and
    # D^1/2 e0 = -Q lam^-1 Q^T D^-1/2 b, so r_k = D^1/2 Q prod(1 - w lam) Q^T D^-1/2 b
    c = Q.T @ (s * b)
    for w in omegas:
        c = c * (1 - w * lam)
    return (Q @ c) / s


def test_random_tridiagonal_jacobi_count_spectral(orc):
    N = 60
    d, e = inputs.random_sdd_tridiagonal(N, seed=4)
    b = np.ones(N)
    lam, Q, s = _spectral(d, e)
    assert lam.min() > 0 and lam.max() < 2  # Jacobi converges
    c = Q.T @ (s * b)
    g = 1 - lam
    k, tol = 0, 1e-7
    while np.linalg.norm((Q @ c) / s) >= tol:
        c = c * g
        k += 1
    P = orc.Problem([N], adiag=d, aoff=[e])
    r = orc.jacobi_solve(P, b, tol=tol, tol_kind="abs")
    assert r["status"] == 0 and r["sweeps"] == k


def test_random_tridiagonal_srj_cycle_residuals_spectral(orc):
    N = 80
    d, e = inputs.random_sdd_tridiagonal(N, seed=9)
    b = np.ones(N)
    lam, Q, s = _spectral(d, e)
    P = orc.Problem([N], adiag=d, aoff=[e])
    levels = [0, 1, 2, 3, 4, 5, 4, 6]
    _, rns = orc.run_levels(P, b, np.zeros(N), levels)
    om = []
    for i, lv in enumerate(levels):
        om += list(orc.level_omegas(lv))
        ref = np.linalg.norm(_residual_after(om, lam, Q, s, b))
        assert rns[i] == pytest.approx(ref, rel=1e-9, abs=1e-12 * np.linalg.norm(b))


@pytest.mark.parametrize("N", [1, 2, 3, 50])
def test_random_tridiagonal_recipe(N):
    d, e = inputs.random_sdd_tridiagonal(N, seed=N)
    assert d.shape == (N,) and e.shape == (N,) and e[N - 1] == 0.0
    off = np.abs(e)
    left = np.concatenate([[0.0], off[:-1]])
    assert np.all(d >= left + off - 1e-15)  # diagonally dominant
    assert np.all(e <= 0)
    if N >= 2:
        assert d[0] == 2 * off[0] and d[N - 1] == 2 * off[N - 2]
    again = inputs.random_sdd_tridiagonal(N, seed=N)
    np.testing.assert_array_equal(again[0], d)


@pytest.mark.slow
def test_sec41_random_tridiagonal_claims(orc):
    # Sec. 4.1: the heuristic beats the increasing rule for every matrix; for
    # large N plain Jacobi needs many times the sweeps of SRJ, for very small
    # N it beats the increasing rule (abs 1e-7, b = 1, 20 matrices per N)
    means = {}
    for N in (10, 500):
        heur, inc, jac = [], [], []
        for s in range(20):
            d, e = inputs.random_sdd_tridiagonal(N, seed=1000 * N + s)
            P = orc.Problem([N], adiag=d, aoff=[e])
            b = np.ones(N)
            h = orc.srj_solve(P, b, tol=1e-7, tol_kind="abs")
            i = orc.srj_solve(P, b, tol=1e-7, tol_kind="abs", rule="increasing")
            assert h["status"] == 0 and i["status"] == 0
            assert h["sweeps"] < i["sweeps"]
            heur.append(h["sweeps"])
            inc.append(i["sweeps"])
            if s < 3:
                j = orc.jacobi_solve(P, b, tol=1e-7, tol_kind="abs")
                assert j["status"] == 0
                jac.append(j["sweeps"])
        means[N] = (np.mean(heur), np.mean(inc), np.mean(jac))
    assert means[10][2] < means[10][1]        # small N: Jacobi beats increasing
    assert means[500][2] > 10 * means[500][0]  # large N: an order of magnitude
