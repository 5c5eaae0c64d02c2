"""Pins for the FP64 oracle: each check ties it to something the paper or the mathematics
fixes, not to itself.  CPU only.

  * App. A.1 scalar lemma                 -> soft_threshold
  * App. A.2 per-entry sub-gradient eq.   -> coupling_C, direction_B, trial (brute force)
  * hand-derived first iterate            -> sign_guess, free set, B, C, d_sol (golden file)
  * Sec. 5.1 optimality, closed forms     -> the whole solve (golden file, n = 1, 2, 3)
  * independent proximal-gradient solver  -> the whole solve at n <= 8
  * KKT certificate, monotone decrease, fixed point (Sec. 5) -> the whole solve at n = 100
  * planted mistakes in the oracle must fail at least one pin
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import closed, gista, pista
from paper_2205_10027_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _mat(rows):
    return np.array([[float(Fraction(x)) for x in r] for r in rows])


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _random_problem(n, m, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, m)) * rng.uniform(0.5, 2.0, (n, 1))
    Y[1:] += 0.6 * Y[:-1]
    Y -= Y.mean(axis=1, keepdims=True)
    return (Y @ Y.T) / m


def _rel_frob(A, B):
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


# ----------------------------------------------------------------------------------------
# App. A.1: x + b + c T(x + a) = 0 is solved by x = -a + ST(a - b, c)
# ----------------------------------------------------------------------------------------
def test_scalar_lemma():
    vals = np.array([-2.0, -1.0, -0.5, -0.25, 0.0, 0.3, 0.5, 1.0, 1.7])
    for a in vals:
        for b in vals:
            for c in (0.1, 0.25, 0.5, 1.0, 2.0):
                x = -a + pista.soft_threshold(a - b, c)
                y = x + a
                if y != 0.0:
                    assert abs(x + b + c * np.sign(y)) <= 1e-12
                else:  # T(0) may be any value in [-1, 1]
                    assert abs(x + b) <= c + 1e-12


def test_objective_pins():
    rng = np.random.default_rng(3)
    S = _random_problem(6, 9, 3)
    lam = 0.2
    assert pista.objective(S, np.eye(6), lam) == pytest.approx(np.trace(S) + lam * 6, rel=1e-14)
    a = rng.uniform(0.5, 2.0, 6)
    want = float(np.sum(-np.log(a) + np.diag(S) * a + lam * a))
    assert pista.objective(S, np.diag(a), lam) == pytest.approx(want, rel=1e-13)
    Q = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    ev = rng.uniform(0.3, 3.0, 6)
    A = (Q * ev) @ Q.T
    A = 0.5 * (A + A.T)
    want = -float(np.sum(np.log(ev))) + float(np.sum(S * A)) + lam * float(np.sum(np.abs(A)))
    assert pista.objective(S, A, lam) == pytest.approx(want, rel=1e-12)
    assert pista.objective(S, A - 4.0 * np.eye(6), lam) == np.inf


def test_inverse_and_logdet_pins():
    S = _random_problem(12, 40, 4)
    A = S + 0.3 * np.eye(12)
    W = pista.inverse(A)
    assert np.max(np.abs(A @ W - np.eye(12))) < 1e-12
    assert np.array_equal(W, W.T)
    pd, ld = pista.logdet(A)
    assert pd and ld == pytest.approx(float(np.sum(np.log(np.linalg.eigvalsh(A)))), rel=1e-12)


def test_min_norm_subgradient_brute_force():
    rng = np.random.default_rng(5)
    n, lam = 7, 0.3
    A = rng.standard_normal((n, n))
    A[rng.random((n, n)) < 0.5] = 0.0
    g = rng.standard_normal((n, n)) * 0.5
    Z = pista.min_norm_subgradient(A, g, lam)
    zgrid = np.linspace(-1.0, 1.0, 200001)
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0:
                want = g[i, j] + lam * np.sign(A[i, j])
            else:
                cand = g[i, j] + lam * zgrid
                want = cand[np.argmin(np.abs(cand))]
            assert abs(Z[i, j] - want) <= 1e-5


def _sign_guess_gives_min_norm_subgradient(mod, seed):
    """Sec. 4.3.1: G of eq. G+ together with the mask M gives the minimum-norm sub-gradient,
    (g + lam G).M = Z, with Z found by brute force over the sub-differential."""
    rng = np.random.default_rng(seed)
    n, lam = 7, 0.3
    A = rng.standard_normal((n, n))
    A[rng.random((n, n)) < 0.5] = 0.0
    g = rng.standard_normal((n, n)) * 0.5
    X = (g + lam * mod.sign_guess(A, g)) * mod.free_set_mask(A, g, lam)
    zgrid = np.linspace(-1.0, 1.0, 20001)
    worst = 0.0
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0:
                want = g[i, j] + lam * np.sign(A[i, j])
            else:
                cand = g[i, j] + lam * zgrid
                want = cand[np.argmin(np.abs(cand))]
            worst = max(worst, abs(X[i, j] - want))
    return worst


@pytest.mark.parametrize("seed", [0, 1])
def test_sign_guess_and_mask_give_min_norm_subgradient(seed):
    assert _sign_guess_gives_min_norm_subgradient(pista, seed) <= 1e-4


# ----------------------------------------------------------------------------------------
# App. A.2: with the other entries of G held fixed, D_ij solves
#   x/t + [A(g.M)A]_ij + lam [A(G^{-i,-j}.M)A]_ij + C_ij T(A_ij + x) = 0
# where G^{-i,-j} zeroes the (i,j) and (j,i) entries (eq. G_comp).  Checked by brute force.
# ----------------------------------------------------------------------------------------
def _entry_equation_violations(mod, seed, n=6, t=0.7):
    rng = np.random.default_rng(seed)
    S = _random_problem(n, 4, seed)
    lam = 0.15
    A = pista.initial_point(S, lam)
    # a PD start with chain couplings of both signs (normalised by the diagonal)
    for (i, j, v) in ((0, 1, 0.3), (1, 2, -0.3), (2, 3, 0.25), (3, 4, -0.3), (4, 5, 0.3)):
        A[i, j] = A[j, i] = v * np.sqrt(A[i, i] * A[j, j])
    assert pista.cholesky(A) is not None
    W = mod.inverse(A)
    g = mod.gradient(S, W)
    M = mod.free_set_mask(A, g, lam)
    G = mod.sign_guess(A, g)
    B = mod.direction_B(A, g, M, G, lam)
    C = mod.coupling_C(A, lam)
    At = mod.trial(A, B, C, M, t)
    D = At - A
    gm = A @ (g * M) @ A
    bad = 0
    for i in range(n):
        for j in range(n):
            if not M[i, j]:
                bad += 0 if D[i, j] == 0.0 else 1   # masked update (reading R2)
                continue
            Gm = (G * M).copy()
            Gm[i, j] = 0.0
            Gm[j, i] = 0.0
            rest = D[i, j] / t + gm[i, j] + lam * (A @ Gm @ A)[i, j]
            cij = lam * (A[i, i] * A[j, j] + (A[i, j] * A[j, i] if i != j else 0.0))
            y = A[i, j] + D[i, j]
            if y != 0.0:
                ok = abs(rest + cij * np.sign(y)) <= 1e-10
            else:
                ok = abs(rest) <= cij + 1e-10
            bad += 0 if ok else 1
    return bad


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_direction_solves_entry_equation(seed):
    assert _entry_equation_violations(pista, seed) == 0


# ----------------------------------------------------------------------------------------
# hand-derived first iterate and closed-form optima (golden file)
# ----------------------------------------------------------------------------------------
def test_golden_first_iterate():
    for case in _golden()["first_iterate_cases"]:
        S, lam, t = _mat(case["S"]), float(Fraction(case["lam"])), float(Fraction(case["t"]))
        want = _mat(case["theta1"])
        res = pista.pista(S, lam, tol=0.0, max_iter=1, trace=True)
        assert res["trace"][0]["t"] == t
        assert np.max(np.abs(res["theta"] - want)) <= 1e-15
        assert np.max(np.abs(closed.first_iterate(S, lam, t) - want)) <= 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_first_iterate_random(seed):
    S = _random_problem(10, 6, 10 + seed)
    lam = 0.2
    res = pista.pista(S, lam, tol=0.0, max_iter=1, trace=True)
    t = res["trace"][0]["t"]
    assert np.max(np.abs(res["theta"] - closed.first_iterate(S, lam, t))) <= 1e-14


def test_golden_optima():
    for case in _golden()["optimum_cases"]:
        S, lam = _mat(case["S"]), float(Fraction(case["lam"]))
        want = _mat(case["theta"])
        res = pista.pista(S, lam, tol=1e-14, max_iter=200)
        assert res["status"] == "converged", case["name"]
        assert _rel_frob(res["theta"], want) <= 1e-12, case["name"]


def test_diagonal_regime_returns_start_point():
    S = _random_problem(30, 60, 7)
    lam = float(np.max(np.abs(S - np.diag(np.diag(S))))) * 1.01
    res = pista.pista(S, lam, tol=1e-12)
    assert res["iterations"] == 0 and res["status"] == "converged"
    assert res["r"] <= 1e-13   # W = A^-1 carries rounding only
    assert np.array_equal(res["theta"], closed.diagonal_solution(S, lam))


def test_two_by_two_random():
    rng = np.random.default_rng(11)
    for _ in range(20):
        s12 = rng.uniform(-1, 1)
        S = np.array([[1.0 + rng.random(), s12], [s12, 1.0 + rng.random()]])
        lam = rng.uniform(0.02, 0.6)
        res = pista.pista(S, lam, tol=1e-14, max_iter=500)
        assert _rel_frob(res["theta"], closed.two_by_two_solution(S, lam)) <= 1e-11


# ----------------------------------------------------------------------------------------
# an independent solver reaches the same unique optimum (n <= 8)
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,lam,seed", [(4, 3, 0.1, 0), (6, 4, 0.05, 1), (8, 5, 0.1, 2),
                                          (8, 20, 0.2, 3), (5, 50, 0.02, 4)])
def test_agrees_with_proximal_gradient(n, m, lam, seed):
    S = _random_problem(n, m, seed)
    ref, r_ref, _ = gista.gista(S, lam, tol=1e-13)
    assert r_ref <= 1e-13
    res = pista.pista(S, lam, tol=1e-12, max_iter=2000)
    assert res["status"] == "converged"
    assert res["r"] <= 1e-12
    assert _rel_frob(res["theta"], ref) <= 1e-9
    Fa, Fb = pista.objective(S, res["theta"], lam), pista.objective(S, ref, lam)
    assert abs(Fa - Fb) / abs(Fb) <= 1e-10


# ----------------------------------------------------------------------------------------
# Sec. 5 invariants on the n = 100 chain workload
# ----------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def chain_solution():
    p = inputs.chain_n100()
    return p, pista.pista(p.S, p.lam, tol=1e-12, max_iter=500, trace=True)


def test_kkt_certificate(chain_solution):
    p, res = chain_solution
    A = res["theta"]
    assert pista.cholesky(A) is not None
    W = np.linalg.inv(A)
    R = W - p.S
    on = A != 0.0
    tau = 1e-9
    assert np.max(np.abs(R[on] - p.lam * np.sign(A[on]))) <= tau
    assert np.max(np.abs(R[~on])) <= p.lam + tau


def test_monotone_and_positive_definite(chain_solution):
    _, res = chain_solution
    # every accepted step decreases F (eq. t_cond_min); the F values themselves agree with
    # that up to their rounding
    assert all(h["dF"] < 0.0 for h in res["trace"])
    Fs = [h["F"] for h in res["trace"]] + [res["F"]]
    assert all(b < a + h["delta"] for a, b, h in zip(Fs, Fs[1:], res["trace"]))
    assert res["status"] == "converged"


def test_fixed_point(chain_solution):
    p, res = chain_solution
    A = res["theta"]
    W = pista.inverse(A)
    g = pista.gradient(p.S, W)
    M = pista.free_set_mask(A, g, p.lam)
    B = pista.direction_B(A, g, M, pista.sign_guess(A, g), p.lam)
    At = pista.trial(A, B, pista.coupling_C(A, p.lam), M, 1.0)
    assert np.max(np.abs(At - A)) <= 1e-9 * np.max(np.abs(A))


def test_block_diagonal_decouples():
    S1 = _random_problem(5, 8, 21)
    S2 = _random_problem(4, 8, 22)
    lam = 0.15
    S = np.zeros((9, 9))
    S[:5, :5], S[5:, 5:] = S1, S2
    S[:5, 5:] = 0.5 * lam
    S[5:, :5] = 0.5 * lam
    full = pista.pista(S, lam, tol=1e-13, max_iter=2000)["theta"]
    b1 = pista.pista(S1, lam, tol=1e-13, max_iter=2000)["theta"]
    b2 = pista.pista(S2, lam, tol=1e-13, max_iter=2000)["theta"]
    assert np.max(np.abs(full[:5, 5:])) == 0.0
    assert _rel_frob(full[:5, :5], b1) <= 1e-10 and _rel_frob(full[5:, 5:], b2) <= 1e-10


# ----------------------------------------------------------------------------------------
# planted mistakes: each must fail at least one pin
# ----------------------------------------------------------------------------------------
class _Mutant:
    """A copy of the oracle's step functions with one of them replaced."""

    def __init__(self, **over):
        for name in ("inverse", "gradient", "free_set_mask", "sign_guess", "direction_B",
                     "coupling_C", "trial"):
            setattr(self, name, over.get(name, getattr(pista, name)))


def _c_without_square(A, lam):
    d = np.diag(A)
    C = lam * np.outer(d, d)
    return C


def _c_without_lam(A, lam):
    return pista.coupling_C(A, lam) / lam


def _guess_wrong_sign(A, g):
    return np.where(A != 0.0, np.sign(A), np.sign(g))


def _b_dropped_l1_term(A, g, M, G, lam):
    return pista.mirror_lower(A @ (g * M) @ A - pista.coupling_C(A, lam) * (G * M))


def _b_transposed_outer(A, g, M, G, lam):
    GM = G * M
    P = A @ (g * M + lam * GM)
    return pista.mirror_lower(P @ np.triu(A) - pista.coupling_C(A, lam) * GM)


def _trial_unmasked(A, B, C, M, t):
    return pista.soft_threshold(A - t * B, t * C)


@pytest.mark.parametrize("over", [
    dict(coupling_C=_c_without_square), dict(coupling_C=_c_without_lam),
    dict(sign_guess=_guess_wrong_sign), dict(direction_B=_b_dropped_l1_term),
    dict(direction_B=_b_transposed_outer), dict(trial=_trial_unmasked),
], ids=["C_no_square", "C_no_lam", "G_wrong_sign", "B_no_l1", "B_bad_operand", "unmasked"])
def test_planted_mistake_is_caught(over):
    mutant = _Mutant(**over)
    bad = sum(_entry_equation_violations(mutant, s) for s in range(4))
    bad += int(_sign_guess_gives_min_norm_subgradient(mutant, 0) > 1e-4)
    if bad == 0:
        # the sign-guess mutant changes which D is built, not the entry equation: it must
        # move the hand-derived first iterate instead
        case = _golden()["first_iterate_cases"][0]
        S, lam = _mat(case["S"]), float(Fraction(case["lam"]))
        A = pista.initial_point(S, lam)
        W = mutant.inverse(A)
        g = mutant.gradient(S, W)
        M = mutant.free_set_mask(A, g, lam)
        B = mutant.direction_B(A, g, M, mutant.sign_guess(A, g), lam)
        At = mutant.trial(A, B, mutant.coupling_C(A, lam), M, 1.0)
        bad = int(np.max(np.abs(At - _mat(case["theta1"]))) > 1e-12)
    assert bad > 0
