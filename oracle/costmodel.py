"""The paper's tuple-count cost analysis, written out -- TEST INFRASTRUCTURE ONLY.

Each function restates one formula of the paper in its own notation and is
pinned by the tests to the numbers the paper prints (Examples 3 and 4) and to
direct minimisation.  M is the on-chip memory capacity in tuples, H, G, h, g
the bucket counts of the hash functions of the same names (Section 3.1).
"""
from __future__ import annotations

import math


def linear_tuples_read(nR: float, nS: float, nT: float, M: float) -> float:
    """Section 4.2: R and S are read once, T once per R partition (|R|/M of them)."""
    return nR + nS + nR * nT / M


def cascade_tuples_moved(nI: float) -> float:
    """Example 3: the cascade writes the intermediate I = R join S and reads it back."""
    return 2.0 * nI


def linear_crossover_M(nR: float, nS: float, nT: float, nI: float) -> float:
    """Smallest M for which the 3-way join reads fewer tuples than the cascade moves
    (Example 3): nR + nS + nR nT / M < 2 nI."""
    return nR * nT / (cascade_tuples_moved(nI) - nR - nS)


def cyclic_tuples_read(nR: float, nS: float, nT: float, H: float, G: float) -> float:
    """Section 5.2: R once, each S partition H times, each T partition G times."""
    return nR + H * nS + G * nT


def cyclic_tuples_read_H(nR: float, nS: float, nT: float, M: float, H: float) -> float:
    """Section 5.2 with GH = |R|/M substituted."""
    return nR + H * nS + nR * nT / (M * H)


def cyclic_optimal_H(nR: float, nS: float, nT: float, M: float) -> float:
    """Section 5.2: the H that zeroes the derivative of cyclic_tuples_read_H."""
    return math.sqrt(nR * nT / (M * nS))


def cyclic_optimal_cost(nR: float, nS: float, nT: float, M: float) -> float:
    """Section 5.2: the cost at the optimal H, |R| + 2 sqrt(|R||S||T|/M)."""
    return nR + 2.0 * math.sqrt(nR * nS * nT / M)


def cyclic_crossover_M(nF: float, nI: float, factor: float = 2.0) -> float:
    """Example 4 with R = S = T = F: the M above which nF (1 + factor sqrt(nF/M)) < nI.

    factor = 2 is the optimal-H cost of Section 5.2; factor = 1 is the
    expression Example 4 prints, which drops that factor 2 (its printed
    crossover, about seven million tuples, follows from factor = 1).
    """
    root = (nI / nF - 1.0) / factor
    return nF / (root * root)


def intermediate_estimate(nR: float, nS: float, d: float) -> float:
    """Section 6.3: |R join S| <= |R||S|/d under uniform keys with d distinct values."""
    return nR * nS / d


def branch_probability(g3: float, d: float) -> float:
    """Appendix A: P(S.C == T.C) inside the 3-way loop nest.

    Expected |S join T| = |S||T|/d matches over H3 h3 g3 (|T|/g3)(|S|/(H3 g3 h3))
    = |S||T|/g3 comparisons.
    """
    nS = nT = 1.0
    matches = nS * nT / d
    comparisons = nS * nT / g3
    return matches / comparisons
