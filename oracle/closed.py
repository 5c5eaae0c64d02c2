"""Closed-form graphical-lasso results derived by hand.  TEST INFRASTRUCTURE ONLY.

Each follows from the optimality condition of Sec. 5.1 (0 in dF(A*), i.e.
W* - S = lam G* with G* in the sub-differential of ||A*||_1 and W* = (A*)^{-1}), or from
eqs. c, b and d_sol applied by hand to a diagonal start point.  None of them calls the
pISTA oracle; they pin it.
"""
from __future__ import annotations

import numpy as np


def _st(v, c):
    return np.sign(v) * np.maximum(np.abs(v) - c, 0.0)


def diagonal_solution(S, lam):
    """If lam >= max_{i != j} |S_ij| the minimiser is diag(1/(S_ii + lam)).

    With W = diag(S_ii + lam): the diagonal residual is W_ii - S_ii - lam = 0, and every
    off-diagonal entry has |W_ij - S_ij| = |S_ij| <= lam, so 0 is a sub-gradient."""
    S = np.asarray(S, dtype=np.float64)
    off = S - np.diag(np.diag(S))
    if np.max(np.abs(off), initial=0.0) > lam:
        raise ValueError("the diagonal closed form needs lam >= max off-diagonal |S_ij|")
    return np.diag(1.0 / (np.diag(S) + lam))


def scalar_solution(s, lam):
    """n = 1: F(a) = -log a + s a + lam a, minimised at a = 1/(s + lam)."""
    return 1.0 / (s + lam)


def two_by_two_solution(S, lam):
    """n = 2: W*_ii = S_ii + lam, W*_12 = ST(S_12, lam), A* = (W*)^{-1}.

    For a 2x2 SPD matrix sign(A_12) = -sign(W_12), so W_12 = S_12 + lam sign(A_12) becomes
    W_12 = S_12 - lam sign(W_12), whose solution is ST(S_12, lam); when |S_12| <= lam the
    off-diagonal of A* vanishes and |W_12 - S_12| = |S_12| <= lam holds."""
    S = np.asarray(S, dtype=np.float64)
    w11, w22 = S[0, 0] + lam, S[1, 1] + lam
    w12 = float(_st(S[0, 1], lam))
    det = w11 * w22 - w12 * w12
    return np.array([[w22, -w12], [-w12, w11]]) / det


def first_iterate(S, lam, t):
    """The first pISTA trial point from A0 = diag(a), a_i = 1/(S_ii + lam), at step t.

    Worked from eqs. G+, c, b and d_sol: W0 = diag(S_ii + lam), g_ii = -lam, g_ij = S_ij.
    On the diagonal G = 1, X_ii = 0, C_ii = lam a_i^2, B_ii = -lam a_i^2, so the trial keeps
    a_i.  Off the diagonal A_ij = 0, G_ij = -sign(S_ij), X_ij = ST(S_ij, lam),
    C_ij = lam a_i a_j and B_ij = a_i a_j S_ij on the free set |S_ij| > lam, so the trial
    entry is ST(-t a_i a_j S_ij, t lam a_i a_j) = -t a_i a_j ST(S_ij, lam)."""
    S = np.asarray(S, dtype=np.float64)
    a = 1.0 / (np.diag(S) + lam)
    T = -t * np.outer(a, a) * _st(S, lam)
    np.fill_diagonal(T, a)
    return T
