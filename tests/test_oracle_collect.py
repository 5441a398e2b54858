"""Pins of the oracle's Sec. 3 data collection (oracle_collect_moves) and of
its counter-based move generator, against what the paper and the
mathematics fix:

 * the generator is SplitMix64's output function: from state 0 its first
   outputs are the published reference values; the moves it draws are
   uniform over the allowed candidates and independent step to step;
 * the first state is the ratio of one level-0 cycle (omega = 2/3) from x = 0
   with b = 1, which has a closed form;
 * every step tries exactly the allowed moves (decrease / keep / increase
   inside [0, max_level]), takes the drawn one, and its ratio becomes the next
   state; a trial ends at the first taken residual below tol;
 * every recorded residual equals the one the plain solver's cycles
   (oracle_srj_run_levels, a separate code path) reach on the same levels;
 * on a 1 x 1 system each cycle multiplies the residual by |G_M(0)|, the
   amplification polynomial at lambda_J = 0 (Sec. 2, Eq. amplification-M-scheme).
"""
import math

import numpy as np
import pytest


def test_splitmix64_reference_outputs(orc):
    # SplitMix64 from state 0: the first three outputs of the published generator
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert orc.splitmix64(0, 2) == 0x06C45D188009454F


@pytest.mark.parametrize("ncand", [2, 3])
def test_pick_is_uniform_and_independent(orc, ncand):
    n = 30000
    draws = np.array([orc.pick(7, t, s, ncand) for t in range(30) for s in range(n // 30)])
    assert draws.min() == 0 and draws.max() == ncand - 1
    counts = np.bincount(draws, minlength=ncand)
    exp = len(draws) / ncand
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    assert chi2 < 20.0  # ncand - 1 degrees of freedom: far beyond the 99.9 % point
    pairs = draws[:-1] * ncand + draws[1:]
    pc = np.bincount(pairs, minlength=ncand * ncand)
    pexp = len(pairs) / ncand ** 2
    assert float(np.sum((pc - pexp) ** 2 / pexp)) < 40.0
    # another seed gives another sequence
    other = np.array([orc.pick(8, 0, s, ncand) for s in range(200)])
    assert not np.array_equal(other, draws[:200])


@pytest.mark.parametrize("N", [1, 2, 5, 100, 400])
def test_first_state_is_one_level0_cycle(orc, N):
    """From x = 0 with b = 1 one cycle at level 0 (M = 1, omega = 2/3) gives
    x = (2/3) D^-1 b and r = b - (1/3) (e_1 + e_N) (A 1 is 2/h^2 at both ends
    and 0 inside; for N = 1, r = b / 3): ratio sqrt((N - 2 + 8/9) / N)."""
    r = orc.collect_moves(orc.Problem([N]), np.ones(N), seed=3, max_steps=3)
    want = 1.0 / 3.0 if N == 1 else math.sqrt((N - 2 + 8.0 / 9.0) / N)
    assert abs(r["prev_ratio"][0] - want) <= 1e-14
    assert r["level"][0] == 0 and r["taken"][0] == 0


def _steps(rec):
    """Group the records of one trial by step (consecutive records sharing
    r_before and level)."""
    out, i = [], 0
    n = len(rec["action"])
    while i < n:
        j = i + 1
        while (j < n and rec["r_before"][j] == rec["r_before"][i]
               and rec["level"][j] == rec["level"][i] and rec["action"][j] > rec["action"][j - 1]):
            j += 1
        out.append(list(range(i, j)))
        i = j
    return out


@pytest.mark.parametrize("N,max_level,seed", [(60, 24, 1), (200, 24, 2), (40, 3, 5), (5, 24, 9)])
def test_walk_structure_and_stop_rule(orc, N, max_level, seed):
    tol = 1e-8
    rec = orc.collect_moves(orc.Problem([N]), np.ones(N), tol=tol, max_level=max_level,
                            seed=seed, trial=4)
    steps = _steps(rec)
    assert len(steps) == rec["steps"]
    taken = rec["taken"]
    for k, idx in enumerate(steps):
        L = taken[k]
        allowed = [a for a in (-1, 0, 1) if 0 <= L + a <= max_level]
        assert [int(rec["action"][i]) for i in idx] == allowed
        assert all(rec["level"][i] == L for i in idx)
        pick = orc.pick(seed, 4, k, len(allowed))
        chosen = idx[pick]
        assert taken[k + 1] == L + allowed[pick]
        # the taken cycle's ratio is the next state; its residual the next r_before
        if k + 1 < len(steps):
            nxt = steps[k + 1][0]
            assert rec["prev_ratio"][nxt] == rec["r_after"][chosen] / rec["r_before"][chosen]
            assert rec["r_before"][nxt] == rec["r_after"][chosen]
            assert rec["r_after"][chosen] >= tol
        else:
            assert rec["r_after"][chosen] < tol
    assert max(taken) <= max_level


@pytest.mark.parametrize("N,seed", [(30, 11), (100, 12)])
def test_records_match_the_plain_solver_cycles(orc, N, seed):
    """Every record's r_after is what the plain solver reaches when it runs
    the levels taken so far and then the record's own level."""
    P = orc.Problem([N])
    f = np.ones(N)
    rec = orc.collect_moves(P, f, seed=seed, trial=0)
    steps = _steps(rec)
    taken = list(rec["taken"])
    for k in list(range(min(6, len(steps)))) + [len(steps) - 1]:
        for i in steps[k]:
            levels = taken[:k + 1] + [int(rec["level"][i] + rec["action"][i])]
            _, rn = orc.run_levels(P, f, np.zeros(N), levels)
            assert rn[-1] == rec["r_after"][i], (k, i)
            assert rn[-2] == rec["r_before"][i]


def test_one_by_one_system_follows_the_amplification_polynomial(orc):
    """N = 1: D^-1 A = 1 and B_J = 0, so a cycle at level c multiplies the
    residual by |G_M(0)| = |prod (1 - omega_j)|.  The residual 1 - A x is
    formed near 1, so each norm carries an absolute error of a few eps64:
    the ratio is compared within 1e-12 relative plus 1e-14 / r_before."""
    rec = orc.collect_moves(orc.Problem([1]), np.ones(1), tol=1e-300, seed=2, max_steps=12)
    assert len(rec["action"]) >= 20
    for i in range(len(rec["action"])):
        c = int(rec["level"][i] + rec["action"][i])
        g = abs(orc.amplification(orc.level_omegas(c), 0.0))
        got = rec["r_after"][i] / rec["r_before"][i]
        assert abs(got - g) <= 1e-12 * g + 1e-14 / rec["r_before"][i], (i, got, g)
