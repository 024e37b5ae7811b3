"""Pins of the cost-model formulas (oracle/costmodel.py) to the paper's printed
numbers (tests/golden/paper_examples.json) and to direct minimisation."""
import json
import math
import os

import numpy as np
import pytest

from oracle import costmodel as cm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _round_sig(x, digits):
    return float(f"{x:.{digits - 1}e}")


def test_example1_sizes():
    e = GOLD["example1_sizes"]
    assert e["users"] * e["friends_per_user"] == e["F_tuples"]
    # friends of friends: each of the 6e11 tuples extends by ~300 friends
    assert e["F_tuples"] * e["friends_per_user"] == e["FF_tuples"]


def test_example3_linear_crossover():
    e = GOLD["example3_linear_friends"]
    F, I = e["F_tuples"], e["intermediate_tuples"]
    assert F * F == pytest.approx(e["T_term_numerator"])
    assert cm.cascade_tuples_moved(I) == pytest.approx(e["cascade_tuples_moved"])
    M = cm.linear_crossover_M(F, F, F, I)
    assert _round_sig(M, e["crossover_M_printed_digits"]) == e["crossover_M"]
    # at the crossover both plans move the same number of tuples
    assert cm.linear_tuples_read(F, F, F, M) == pytest.approx(cm.cascade_tuples_moved(I))
    assert cm.linear_tuples_read(F, F, F, 1.01 * M) < cm.cascade_tuples_moved(I)


def test_example4_cyclic_crossover_both_readings():
    e = GOLD["example4_cyclic_friends"]
    F, I = e["F_tuples"], e["intermediate_tuples_in_condition"]
    printed = cm.cyclic_crossover_M(F, I, factor=1.0)
    assert _round_sig(printed, e["crossover_M_printed_digits"]) == e["crossover_M_printed"]
    with_two = cm.cyclic_crossover_M(F, I, factor=2.0)
    assert with_two == pytest.approx(4 * printed)
    # the factor-2 crossover is where the optimal cyclic cost meets the intermediate
    assert cm.cyclic_optimal_cost(F, F, F, with_two) == pytest.approx(I)


@pytest.mark.parametrize("nR,nS,nT,M", [(1e6, 4e6, 9e6, 1e4), (5e8, 2e8, 3e8, 1.6e7),
                                        (7.0, 3.0, 11.0, 0.5)])
def test_cyclic_optimum_by_direct_minimisation(nR, nS, nT, M):
    H_star = cm.cyclic_optimal_H(nR, nS, nT, M)
    Hs = H_star * np.exp(np.linspace(-3, 3, 20001))
    costs = np.array([cm.cyclic_tuples_read_H(nR, nS, nT, M, h) for h in Hs])
    assert Hs[np.argmin(costs)] == pytest.approx(H_star, rel=1e-3)
    assert costs.min() == pytest.approx(cm.cyclic_optimal_cost(nR, nS, nT, M), rel=1e-9)
    # G H = |R| / M: the same cost through the (H, G) form
    G = nR / (M * H_star)
    assert cm.cyclic_tuples_read(nR, nS, nT, H_star, G) == pytest.approx(
        cm.cyclic_optimal_cost(nR, nS, nT, M))


def test_cyclic_cost_prefers_smallest_R():
    sizes = [2e6, 5e6, 9e6]
    costs = {perm: cm.cyclic_optimal_cost(*perm, 1e4)
             for perm in [(2e6, 5e6, 9e6), (5e6, 2e6, 9e6), (9e6, 5e6, 2e6)]}
    assert min(costs, key=costs.get)[0] == min(sizes)


def test_linear_prefers_smaller_R_first_term():
    # the T term is symmetric in R and T, the first term is not (Section 4.2)
    a = cm.linear_tuples_read(1e6, 5e6, 9e6, 1e4)
    b = cm.linear_tuples_read(9e6, 5e6, 1e6, 1e4)
    assert a < b


def test_branch_probability_and_intermediate():
    for g3, d in [(64, 1e6), (1024, 7e5), (1, 10)]:
        assert cm.branch_probability(g3, d) == pytest.approx(g3 / d)
    # uniform keys: |R join S| ~ |R||S|/d; check against an exact count on random data
    rng = np.random.default_rng(0)
    d = 500
    rb = rng.integers(0, d, 200000)
    sb = rng.integers(0, d, 200000)
    exact = int(np.sum(np.bincount(rb, minlength=d).astype(np.int64) *
                       np.bincount(sb, minlength=d).astype(np.int64)))
    assert exact == pytest.approx(cm.intermediate_estimate(2e5, 2e5, d), rel=0.02)


def test_branch_probability_by_loop_nest():
    """Appendix A's branch probability counted in the loop nest itself: S and T
    with uniform C values in [0, d) hashed into g3 buckets (c mod g3); every
    (s, t) pair of a bucket is one comparison, an equal pair is one match.
    Over many draws matches / comparisons approaches g3 / d."""
    rng = np.random.default_rng(3)
    for g3, d in [(4, 64), (8, 40), (1, 10)]:
        comps = matches = 0
        for _ in range(200):
            sc = rng.integers(0, d, 120)
            tc = rng.integers(0, d, 90)
            for k in range(g3):
                sk, tk = sc[sc % g3 == k], tc[tc % g3 == k]
                for s in sk:           # the nested loop of one bucket pair
                    for t in tk:
                        comps += 1
                        matches += int(s == t)
        assert matches / comps == pytest.approx(cm.branch_probability(g3, d), rel=0.05)
