"""Independent brute-force checker: plain proximal gradient (G-ISTA) for the graphical lasso.

TEST INFRASTRUCTURE ONLY.  Sec. 2.2 of the paper: with H = I in eq. proximal_gen the
proximal method is plain ISTA,  A <- ST(A - t grad f(A), t lam).  The graphical-lasso
objective is strictly convex, so its minimiser is unique (Sec. 5.1) and any convergent
method reaches the same point; this solver reaches it by a different route from pISTA
(no preconditioner, no free set, no sign guess, eigenvalue-based log det) and so pins
the pISTA oracle's final answer at small n.  It deliberately imports nothing from
``oracle.pista``.
"""
from __future__ import annotations

import numpy as np


def _soft(v, c):
    return np.sign(v) * np.maximum(np.abs(v) - c, 0.0)


def _smooth(S, A):
    """(pd, f(A) = -log det A + tr(SA)) from the eigenvalues of A."""
    ev = np.linalg.eigvalsh(A)
    if ev[0] <= 0.0:
        return False, np.inf
    return True, float(-np.sum(np.log(ev)) + np.sum(S * A))


def _residual(A, g, lam):
    z = np.where(A != 0.0, g + lam * np.sign(A), _soft(g, lam))
    return float(np.sum(np.abs(z)) / np.sum(np.abs(A)))


def gista(S, lam, tol=1e-13, max_iter=400000, A0=None):
    """Proximal gradient with backtracking on the smooth part's quadratic upper bound.

    Far from the optimum the usual sufficient-decrease test picks the step.  Near it, that
    test is decided by rounding, so the step never drops below t_safe = lambda_min(A)^2 / 2,
    for which the gradient of f = -log det + tr(S .) is Lipschitz with constant at most
    1/lambda_min^2 around A (the bound behind Lemma 5.2 of the paper); at such a step the
    proximal map is a contraction towards the unique minimiser.

    Returns (theta, relative l1 residual, iterations)."""
    S = np.asarray(S, dtype=np.float64)
    A = np.diag(1.0 / (np.diag(S) + lam)) if A0 is None else np.array(A0, dtype=np.float64)
    t = 1.0
    r = np.inf
    for it in range(max_iter):
        W = np.linalg.inv(A)
        W = 0.5 * (W + W.T)
        g = S - W
        r = _residual(A, g, lam)
        if r <= tol:
            return A, r, it
        ev = np.linalg.eigvalsh(A)
        t_safe = 0.5 * ev[0] ** 2
        f = float(-np.sum(np.log(ev)) + np.sum(S * A))
        t = min(1.0, max(2.0 * t, t_safe))
        An = None
        while t > t_safe:
            cand = _soft(A - t * g, t * lam)
            cand = 0.5 * (cand + cand.T)
            okn, fn = _smooth(S, cand)
            D = cand - A
            bound = f + float(np.sum(g * D)) + float(np.sum(D * D)) / (2.0 * t)
            if okn and fn <= bound:
                An = cand
                break
            t *= 0.5
        if An is None:
            t = t_safe
            while True:
                cand = _soft(A - t * g, t * lam)
                cand = 0.5 * (cand + cand.T)
                if np.linalg.eigvalsh(cand)[0] > 0.0:
                    An = cand
                    break
                t *= 0.5
        A = An
    return A, r, max_iter
