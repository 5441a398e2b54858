"""Pins of the oracle's Neumann boundary (mirrored ghost node, Sec. 4.2.2) and
of the per-sweep stopping test ||x^n - x^(n-1)||_inf < tol (Sec. 4.2.2, Eq.
relative_residual_solution) against closed forms and invariants.

With n nodes per Neumann axis (both boundary nodes included, h = 1/(n-1)) and
the ghost u_{-1} = u_1, u_n = u_{n-2}, the 1D operator is
    (A u)_0 = 2 (u_0 - u_1) / h^2,  (A u)_j = (2 u_j - u_{j-1} - u_{j+1}) / h^2,
its eigenvectors are cos(pi k j / (n-1)) with eigenvalues
2 (1 - cos(pi k / (n-1))) / h^2, and the trapezoid weights
w = (1/2, 1, ..., 1, 1/2) span its left null space, so w . u is invariant under
every relaxed Jacobi sweep of A u = 0.  A ghost placed wrongly (u_{-1} = u_0,
or a zero) breaks all three.
"""
import math

import numpy as np
import pytest

from paper_2011_06636_gb300 import inputs


def _cos_mode(n, k):
    j = np.arange(n)
    return np.cos(math.pi * k * j / (n - 1))


def _sin_mode(n, k):
    j = np.arange(n)
    return np.sin(math.pi * k * (j + 1) / (n + 1))


def _trap(n):
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    return w


@pytest.mark.parametrize("n", [2, 3, 9, 16])
def test_neumann_1d_cosines_are_eigenvectors(orc, n):
    P = orc.Problem([n], bc=[1])
    h = 1.0 / (n - 1)
    assert P.h[0] == pytest.approx(h)
    for k in range(n):
        v = _cos_mode(n, k)
        lam = 2.0 * (1.0 - math.cos(math.pi * k / (n - 1))) / h ** 2
        np.testing.assert_allclose(orc.apply_A(P, v), lam * v, rtol=0, atol=1e-12 * (1 + lam))


def test_mixed_bc_2d_products_are_eigenvectors(orc):
    # x Dirichlet (sines over interior points), y Neumann (cosines over nodes)
    nx, ny = 7, 6
    P = orc.Problem([nx, ny], bc=[0, 1], eps=[1.0, 0.3])
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny - 1)
    for i in (1, 4, 7):
        for k in (0, 2, 5):
            v = np.outer(_cos_mode(ny, k), _sin_mode(nx, i)).ravel()  # x fastest
            lam = (2 * (1 - math.cos(math.pi * i / (nx + 1))) / hx ** 2
                   + 0.3 * 2 * (1 - math.cos(math.pi * k / (ny - 1))) / hy ** 2)
            np.testing.assert_allclose(orc.apply_A(P, v), lam * v, rtol=0, atol=1e-10 * lam)


def test_neumann_3d_constants_span_null_space(orc):
    P = orc.Problem([5, 4, 3], bc=[1, 1, 1])
    np.testing.assert_array_equal(orc.apply_A(P, np.ones(P.size)), 0.0)
    # Dirichlet on one axis: the constant is no longer in the null space
    Q = orc.Problem([5, 4, 3], bc=[1, 0, 1])
    assert np.abs(orc.apply_A(Q, np.ones(Q.size))).max() > 1.0


def test_neumann_diagonal_is_interior_diagonal(orc):
    P = orc.Problem([6, 5], bc=[1, 1], eps=[2.0, 1.0])
    d = orc.diagonal(P)
    hx, hy = 1 / 5, 1 / 4
    np.testing.assert_allclose(d, 2 * (2.0 / hx ** 2 + 1.0 / hy ** 2), rtol=1e-15)


def test_sweep_of_a_mode_is_scaled_by_one_minus_omega_mu(orc):
    n = 11
    P = orc.Problem([n, n], bc=[1, 1])
    v = np.outer(_cos_mode(n, 3), _cos_mode(n, 7)).ravel()
    mu = 1 - (math.cos(3 * math.pi / (n - 1)) + math.cos(7 * math.pi / (n - 1))) / 2
    for omega in (0.3, 1.0, 4.5):
        out = orc.sweep(P, v, np.zeros(P.size), omega)
        np.testing.assert_allclose(out, (1 - omega * mu) * v, rtol=0, atol=1e-12 * (1 + omega))


def test_trapezoid_weighted_sum_is_invariant(orc):
    n0, n1 = 13, 9
    P = orc.Problem([n0, n1], bc=[1, 1])
    w = np.outer(_trap(n1), _trap(n0)).ravel()
    u0 = inputs.uniform_rhs([n0, n1], seed=5).ravel()
    u = orc.sweeps(P, u0, np.zeros(P.size), orc.level_omegas(6))
    assert abs(w @ u - w @ u0) < 1e-12 * np.abs(w @ np.abs(u0))


def test_checkerboard_jacobi_stagnates_and_srj_does_not(orc):
    # the checkerboard has mu = 2: Jacobi multiplies it by -1 every sweep, so
    # the largest change stays 2 (Sec. 4.2.2: Jacobi stagnates on this problem)
    n = 8
    P = orc.Problem([n, n], bc=[1, 1])
    v = np.outer(_cos_mode(n, n - 1), _cos_mode(n, n - 1)).ravel()
    f = np.zeros(P.size)
    u1 = orc.sweep(P, v, f, 1.0)
    np.testing.assert_allclose(u1, -v, atol=1e-13)
    r = orc.jacobi_solve(P, f, v, tol=1e-10, tol_kind="dinf", max_sweeps=500)
    assert r["status"] != 0 and r["sweeps"] == 500
    s = orc.srj_solve(P, f, v, tol=1e-10, tol_kind="dinf", rule="heuristic")
    assert s["status"] == 0


def _first_sweep_below(omegas, mu, tol, amp=1.0):
    """Closed form of the per-sweep stop for a single mode of amplitude amp:
    the change of sweep s is |omega_s mu prod_{i<s}(1 - omega_i mu)| amp."""
    g = amp
    margin = math.inf
    for s, w in enumerate(omegas, start=1):
        d = abs(w * mu * g)
        margin = min(margin, abs(d - tol) / tol)
        if d < tol:
            return s, margin
        g *= 1 - w * mu
    return None, margin


@pytest.mark.parametrize("level,k,tol", [(4, 3, 1e-6), (9, 1, 1e-8), (12, 2, 1e-10)])
def test_dinf_stop_matches_closed_form(orc, level, k, tol):
    n = 17
    P = orc.Problem([n], bc=[1])
    v = _cos_mode(n, k)
    mu = 1 - math.cos(math.pi * k / (n - 1))
    om = orc.level_omegas(level)
    cycles = 40
    s_exp, margin = _first_sweep_below(np.tile(om, cycles), mu, tol)
    assert s_exp is not None and margin > 1e-6
    r = orc.srj_solve(P, np.zeros(n), v, tol=tol, tol_kind="dinf", rule="fixed", level0=level)
    assert r["status"] == 0
    assert r["sweeps"] == s_exp
    # a stop inside a cycle records only the cycles that completed
    assert r["cycles"] == (s_exp - 1) // len(om)


def test_dinf_zero_start_on_null_space_stops_after_one_sweep(orc):
    P = orc.Problem([6, 6], bc=[1, 1])
    u0 = np.full(P.size, 3.0)
    r = orc.srj_solve(P, np.zeros(P.size), u0, tol=1e-10, tol_kind="dinf")
    assert r["status"] == 0 and r["sweeps"] == 1
    np.testing.assert_array_equal(r["u"], u0)


def test_laplace_neumann_converges_to_weighted_mean(orc):
    # Sec. 4.2.2: A x = 0 from a random start; the limit is the constant with
    # the trapezoid-weighted mean of the start
    n = 24
    P = orc.Problem([n, n], bc=[1, 1])
    u0 = inputs.uniform_rhs([n, n], seed=11).ravel()
    w = np.outer(_trap(n), _trap(n)).ravel()
    c = (w @ u0) / w.sum()
    r = orc.srj_solve(P, np.zeros(P.size), u0, tol=1e-10, tol_kind="dinf", rule="heuristic")
    assert r["status"] == 0
    assert np.abs(r["u"] - c).max() < 1e-7
    assert abs(w @ r["u"] - w @ u0) < 1e-11 * w.sum()


@pytest.mark.slow
def test_laplace_neumann_heuristic_beats_increasing(orc):
    # Sec. 4.2.2: the heuristic needs fewer sweeps than the increasing rule
    n = 64
    P = orc.Problem([n, n], bc=[1, 1])
    u0 = inputs.uniform_rhs([n, n], seed=3).ravel()
    f = np.zeros(P.size)
    heur = orc.srj_solve(P, f, u0, tol=1e-10, tol_kind="dinf", rule="heuristic")
    inc = orc.srj_solve(P, f, u0, tol=1e-10, tol_kind="dinf", rule="increasing")
    assert heur["status"] == 0 and inc["status"] == 0
    assert heur["sweeps"] < inc["sweeps"]
