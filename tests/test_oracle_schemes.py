"""Pins of the oracle's scheme family (Sec. 2, App. A, App. B) against values
the paper prints and against closed forms / library routines that share
nothing with the oracle's code."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from conftest import read_golden


def _decimals(s):
    return len(s.split(".")[1]) if "." in s else 0


def test_appB_level_table(orc):
    rows = read_golden("appB_levels.txt")
    assert len(rows) == 25
    for lv, M in rows:
        assert orc.level_m(int(lv)) == int(M)
    assert orc.level_m(25) == -1 and orc.level_m(-1) == -1


@pytest.mark.parametrize("row", read_golden("table2_omegas.txt"), ids=lambda r: "M%s" % r[0])
def test_table2_omegas_as_set(orc, row):
    """Table 2: the printed factors, as a set, to the printed digits."""
    M = int(row[0])
    printed = row[1:]
    assert len(printed) == M
    _, w = orc.scheme_root_order(M)
    got = sorted(w)
    for s, g in zip(sorted(printed, key=float), got):
        tol = 0.5 * 10.0 ** (-_decimals(s)) + 1e-15
        assert abs(float(s) - g) <= tol, (M, s, g)


@pytest.mark.parametrize("row", read_golden("table1_chebyshev.txt"), ids=lambda r: "M%s" % r[0])
def test_table1_affine_map_and_lambda_max(orc, row):
    """Table 1: G_M(lambda) = T_M(c1 lambda + c0)/3 with the printed c1, c0,
    and the printed lambda_max (largest lambda with |G_M| <= 1/3), found by
    bisection on the oracle's product form of G_M (Eq. amplification-M-scheme)."""
    M = int(row[0])
    c1p, c0p, lmaxp = row[1], row[2], row[3]
    ls = orc.lambda_star(M)
    c1, c0 = (ls + 1) / 2, (ls - 1) / 2
    assert abs(c1 - float(c1p)) <= 0.5 * 10 ** (-_decimals(c1p)) + 1e-12
    assert abs(c0 - float(c0p)) <= 0.5 * 10 ** (-_decimals(c0p)) + 1e-12
    w = orc.level_omegas([1, 2, 3, 5].index(M) if M != 5 else 3)
    assert len(w) == M
    G = lambda lam: orc.amplification(w, lam)
    # |G| <= 1/3 on [-1, lmax] and G(1) = 1: bisection for the crossing G = 1/3
    lo, hi = -1.0 if M > 1 else -0.5, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if G(mid) > 1.0 / 3.0 + 1e-15:
            hi = mid
        else:
            lo = mid
    assert abs(lo - float(lmaxp)) <= 0.5 * 10 ** (-_decimals(lmaxp)) + 1e-9, (M, lo)


def _T(M, y):
    """Chebyshev T_M by its trigonometric / hyperbolic closed form."""
    y = np.asarray(y, dtype=np.float64)
    out = np.empty_like(y)
    inside = np.abs(y) <= 1
    out[inside] = np.cos(M * np.arccos(y[inside]))
    big = y > 1
    out[big] = np.cosh(M * np.arccosh(y[big]))
    small = y < -1
    out[small] = (-1) ** M * np.cosh(M * np.arccosh(-y[small]))
    return out


@pytest.mark.parametrize("level", range(25))
def test_amplification_is_scaled_chebyshev(orc, level):
    """Eq. (transformation) / App. A: G_M(lambda) = T_M(f(lambda))/3 with
    f(-1) = -1 and f(1) = lambda*, T_M(lambda*) = 3; hence G_M(1) = 1,
    G_M(-1) = (-1)^M / 3, |G_M| <= 1/3 on [-1, lambda_max]."""
    M = orc.level_m(level)
    w = orc.level_omegas(level)
    ls = orc.lambda_star(M)
    assert abs(_T(M, np.array([ls]))[0] - 3.0) < 1e-9 * M * M
    G = lambda lam: orc.amplification(w, lam)
    assert abs(G(1.0) - 1.0) < 1e-9
    assert abs(G(-1.0) - (-1) ** M / 3.0) < 1e-9
    lmax = (3 - ls) / (ls + 1)
    lam = np.concatenate([np.cos(np.linspace(0, math.pi, 257)) * 0.5 * (1 + lmax) - 0.5 * (1 - lmax)])
    ref = _T(M, ((ls + 1) * lam + (ls - 1)) / 2) / 3
    got = np.array([G(v) for v in lam])
    assert np.max(np.abs(got)) <= 1.0 / 3.0 + 1e-9
    assert np.max(np.abs(got - ref)) < 1e-9
    if M <= 40:  # library Chebyshev evaluation (Clenshaw) as a second check
        cheb = npcheb.Chebyshev.basis(M)
        lam2 = np.linspace(-1, 1, 101)
        ref2 = cheb(((ls + 1) * lam2 + (ls - 1)) / 2) / 3
        got2 = np.array([G(v) for v in lam2])
        assert np.max(np.abs(got2 - ref2)) < 1e-9


@pytest.mark.parametrize("level", range(25))
def test_roots_map_to_chebyshev_nodes(orc, level):
    """Eq. (optimal-relaxed) and Eq. (transformation-inverse): the root of each
    factor, lambda_j = 1 - 1/omega_j, maps under f to a root of T_M; the set
    of mapped roots equals numpy's Chebyshev points of the first kind."""
    M = orc.level_m(level)
    w = orc.level_omegas(level)
    ls = orc.lambda_star(M)
    lam_r = 1.0 - 1.0 / w
    x = np.sort(((ls + 1) * lam_r + (ls - 1)) / 2)
    ref = np.sort(npcheb.chebpts1(M))
    assert np.max(np.abs(x - ref)) < 1e-12


@pytest.mark.parametrize("level", range(25))
def test_application_order_is_permutation_starting_largest(orc, level):
    M = orc.level_m(level)
    w = orc.level_omegas(level)
    _, wr = orc.scheme_root_order(M)
    assert np.array_equal(np.sort(w), np.sort(wr))
    assert w[0] == wr.max()


@pytest.mark.parametrize("M", [2, 3, 5, 7, 10, 14])
def test_leja_order_brute_force(orc, M):
    """Brute force on tiny inputs: each next root maximises the plain product
    of distances to the roots already applied (the Leja property)."""
    x, _ = orc.scheme_root_order(M)
    order = list(orc.leja_order(M, x))
    assert order[0] == 0
    for step in range(1, M):
        chosen = order[:step]
        prods = {j: np.prod([abs(x[j] - x[i]) for i in chosen])
                 for j in range(M) if j not in chosen}
        best = max(prods.values())
        assert prods[order[step]] >= best * (1 - 1e-12)


@pytest.mark.parametrize("level", [4, 8, 12, 16, 20, 24])
def test_cycle_is_order_independent_and_growth_bounded(orc, level):
    """In exact arithmetic a cycle's amplification does not depend on the
    order of its factors (Eq. amplification-M-scheme is a product); the chosen
    order keeps every partial product below M^2 on [-1, 1] (roundoff control,
    Sec. 2 last paragraph)."""
    M = orc.level_m(level)
    w = orc.level_omegas(level)
    _, wr = orc.scheme_root_order(M)
    lam = np.cos(np.linspace(0, math.pi, 4001))
    P = np.ones_like(lam)
    worst = 0.0
    for wi in w:
        P *= (1 - wi) + wi * lam
        worst = max(worst, np.abs(P).max())
    assert worst <= M * M
    if M <= 63:
        Q = np.ones_like(lam)
        for wi in wr:
            Q *= (1 - wi) + wi * lam
        assert np.max(np.abs(P - Q)) < 1e-9


def test_one_minus_omega_is_exact_in_fp32(orc):
    """The fused FP32-pair relaxation forms (1 - omega) u + omega q with
    1 - omega computed in FP32: exact for every factor of the 25 levels,
    because each lies in (0.5, 2^24) (Sterbenz's lemma up to 2, a multiple of
    omega's last place above)."""
    import numpy as np
    for level in range(25):
        w32 = orc.level_omegas(level).astype(np.float32)
        assert np.all(w32 > 0.5) and np.all(w32 < 2.0 ** 24)
        one_minus = np.float32(1.0) - w32
        assert np.array_equal(one_minus.astype(np.float64), 1.0 - w32.astype(np.float64))
