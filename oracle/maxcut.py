"""Brute-force maximum cut of a tiny weighted graph (a pin for the MaxCut SDP bound).

With C = -(1/4) L and diag(X) = 1, the SDP value -<C, X*> is an upper bound
on the maximum cut: every cut vector z in {-1,1}^n gives a feasible X = z z^T
with (1/4) z^T L z = cut weight.
"""
from __future__ import annotations

import itertools

import numpy as np


def max_cut_brute_force(n: int, edges: np.ndarray, weights: np.ndarray) -> float:
    best = -np.inf
    for bits in itertools.product((0, 1), repeat=n - 1):
        side = np.array((0,) + bits)
        cut = float(np.sum(weights[side[edges[:, 0]] != side[edges[:, 1]]]))
        best = max(best, cut)
    return best
