"""The support-recovery score against hand-counted cases."""
import math

import numpy as np

from paper_2205_10027_gb300 import metrics


def _sym(n, pairs, val=0.5):
    A = np.eye(n)
    for i, j in pairs:
        A[i, j] = A[j, i] = val
    return A


def test_perfect_and_inverted_patterns():
    T = _sym(5, [(0, 1), (1, 2), (3, 4)])
    assert metrics.support_mcc(T, T * 3.0) == 1.0
    # the estimate is nonzero exactly where the truth is zero (off the diagonal)
    H = np.ones((5, 5)) - (T != 0) + np.eye(5)
    assert metrics.support_mcc(T, H) == -1.0


def test_hand_counted_case():
    # 4 x 4: 6 pairs.  truth {01, 12}; estimate {01, 23, 03}
    T = _sym(4, [(0, 1), (1, 2)])
    H = _sym(4, [(0, 1), (2, 3), (0, 3)], val=-0.2)
    assert metrics.support_counts(T, H) == (1, 2, 2, 1)     # TP {01}; TN {02, 13}; FP {23, 03}; FN {12}
    assert math.isclose(metrics.support_mcc(T, H), (1 * 2 - 2 * 1) / math.sqrt(3 * 2 * 4 * 3))


def test_diagonal_is_not_counted_and_degenerate_is_zero():
    T = _sym(3, [(0, 1)])
    H = np.diag([1.0, 2.0, 3.0])          # no off-diagonal support: TP + FP = 0
    assert metrics.support_counts(T, H) == (0, 2, 0, 1)
    assert metrics.support_mcc(T, H) == 0.0
