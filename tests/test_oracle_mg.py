"""Pins of the oracle's multigrid with SRJ smoothing (an adjacent use named in
Sec. 1 and Sec. 5) against closed forms of full weighting, linear
interpolation and the exact two-grid operator, and against direct solves."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2011_06636_gb300 import inputs


def _sin(n, k):
    j = np.arange(1, n + 1)
    return np.sin(math.pi * k * j / (n + 1))


@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_full_weighting_of_a_sine_mode(orc, k):
    # R s_k = cos^2(k pi h / 2) s_k on the coarse grid (1D), products in 2D
    n = 31
    P = orc.Problem([n])
    th = math.pi * k / (n + 1)
    np.testing.assert_allclose(orc.mg_restrict(P, _sin(n, k)), math.cos(th / 2) ** 2 * _sin(15, k),
                               atol=1e-14)
    P2 = orc.Problem([n, n])
    v = np.outer(_sin(n, 2), _sin(n, k)).ravel()
    th2 = math.pi * 2 / (n + 1)
    ref = math.cos(th / 2) ** 2 * math.cos(th2 / 2) ** 2 * np.outer(_sin(15, 2), _sin(15, k)).ravel()
    np.testing.assert_allclose(orc.mg_restrict(P2, v), ref, atol=1e-14)


@pytest.mark.parametrize("k", [1, 4, 9, 15])
def test_linear_interpolation_of_a_coarse_mode(orc, k):
    # P s^c_k = cos^2(k pi h / 2) s_k - sin^2(k pi h / 2) s_(n+1-k)
    n, nc = 31, 15
    P, Pc = orc.Problem([n]), orc.Problem([nc])
    th = math.pi * k / (n + 1)
    got = orc.mg_prolong_add(Pc, _sin(nc, k), P, np.zeros(n))
    ref = math.cos(th / 2) ** 2 * _sin(n, k) - math.sin(th / 2) ** 2 * _sin(n, n + 1 - k)
    np.testing.assert_allclose(got, ref, atol=1e-14)


def test_interpolation_reproduces_linear_functions(orc):
    # away from the zero boundary, a linear coarse function is interpolated
    # exactly (3D, tensor product)
    nc = 7
    Pc, P = orc.Problem([nc] * 3), orc.Problem([15] * 3)
    zc, yc, xc = np.meshgrid(*[np.arange(1, nc + 1) * 2.0] * 3, indexing="ij")
    ec = (1.0 + 0.5 * xc - 0.25 * yc + 2.0 * zc).ravel()
    got = orc.mg_prolong_add(Pc, ec, P, np.zeros(15 ** 3)).reshape(15, 15, 15)
    z, y, x = np.meshgrid(*[np.arange(1, 16) * 1.0] * 3, indexing="ij")
    ref = 1.0 + 0.5 * x - 0.25 * y + 2.0 * z
    np.testing.assert_allclose(got[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1], atol=1e-12)


def _two_grid_matrix(n, k, omegas_pre, omegas_post):
    """Exact two-grid error propagation on the pair (s_k, s_(n+1-k)) of the 1D
    Poisson problem with the rediscretised coarse operator (textbook Fourier
    analysis of smoothing, full weighting and linear interpolation)."""
    h = 1.0 / (n + 1)
    kk = [k, n + 1 - k]
    th = [math.pi * q * h for q in kk]
    mu = [1 - math.cos(t) for t in th]  # eigenvalues of D^-1 A
    lam = [2 * (1 - math.cos(t)) / h ** 2 for t in th]
    c2, s2 = math.cos(th[0] / 2) ** 2, math.sin(th[0] / 2) ** 2
    # R maps s_k -> c2 s^c_k and s_(n+1-k) -> -s2 s^c_k; P maps s^c_k -> (c2, -s2)
    R = np.array([[c2, -s2]])
    Pm = np.array([[c2], [-s2]])
    lam_c = 2 * (1 - math.cos(2 * th[0])) / (2 * h) ** 2
    Ainv_c = 1.0 / lam_c
    A = np.diag(lam)
    CGC = np.eye(2) - Pm @ (Ainv_c * R) @ A
    S_pre = np.eye(2)
    for w in omegas_pre:
        S_pre = np.diag([1 - w * m for m in mu]) @ S_pre
    S_post = np.eye(2)
    for w in omegas_post:
        S_post = np.diag([1 - w * m for m in mu]) @ S_post
    return S_post @ CGC @ S_pre


@pytest.mark.parametrize("level", [0, 1, 2, 4])
@pytest.mark.parametrize("k", [1, 3])
def test_two_grid_cycle_matches_fourier_analysis(orc, level, k):
    # n = 3 coarsens to the one-point grid, where the coarse solve is exact:
    # the V-cycle is a true two-grid cycle.  With f = 0 the iterate is the
    # error, mapped by the closed-form 2 x 2 operator on the mode pair (k, 4-k).
    n = 3
    P = orc.Problem([n])
    om = list(orc.level_omegas(level))
    got = orc.mg_vcycle(P, _sin(n, k), np.zeros(n), level=level, nu1=1, nu2=1)
    G = _two_grid_matrix(n, 1, om, om)
    col = 0 if k == 1 else 1
    ref = G[0, col] * _sin(n, 1) + G[1, col] * _sin(n, 3)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_vcycle_matches_direct_solve_2d(orc):
    n = [31, 31]
    P = orc.Problem(n, eps=[1.0, 0.5])
    f = inputs.uniform_rhs(n, seed=3).ravel()
    r = orc.mg_solve(P, f, tol=1e-11, level=1)
    assert r["status"] == 0
    h = 1 / 32
    e = np.ones(31)
    T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) / h ** 2
    A = sp.kron(sp.identity(31), T) + 0.5 * sp.kron(T, sp.identity(31))
    x = spla.spsolve(A.tocsc(), f)
    np.testing.assert_allclose(r["u"], x, rtol=0, atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("n", [[63, 63], [127, 127], [15, 15, 15], [31, 31, 31]])
def test_vcycle_rate_independent_of_h(orc, n):
    # textbook multigrid property: the V(1,1) rate stays bounded as h -> 0
    P = orc.Problem(n)
    f = inputs.uniform_rhs(n, seed=5).ravel()
    r = orc.mg_solve(P, f, tol=1e-8, level=1)
    rate = (r["rn"] / r["r0"]) ** (1.0 / r["cycles"])
    assert r["status"] == 0 and rate < 0.2
