"""Pins for the two line-search pieces of the oracle that a converged answer cannot see: the
fallback step of Sec. 6 and the rounding-proof objective difference of reading R6.  Both
only decide how the path runs, so the final-answer pins (closed forms, the independent
proximal-gradient solver, the KKT certificate) would pass with either of them wrong.  CPU
only.

  * fallback step t_f = (0.9 / cond_2 A)^2 (Sec. 6; Lemma 4.1's t < (beta / gamma)^2)
      -> pista.fallback_step, and its use in pista(): a start point whose eigenvalues are
         fixed by construction, and t_min above 1 so that halving never runs and every
         iteration takes t_f; the next steps against cond_2 from singular values.
  * objective difference of eq. t_cond_min (reading R6)
      -> pista.objective_difference against F(A_t) - F(A) evaluated with 50-digit
         determinants, inside the rounding band (tier 2, eigenvalues of E) and outside it
         (tier 1, the two Cholesky log-dets).
  * planted mistakes in either piece must fail these pins.
"""
import numpy as np
import pytest

from oracle import pista

mp = pytest.importorskip("mpmath")


def _problem(n, m, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, m)) * rng.uniform(0.5, 2.0, (n, 1))
    Y[1:] += 0.5 * Y[:-1]
    Y -= Y.mean(axis=1, keepdims=True)
    return (Y @ Y.T) / m


def _spd_with_spectrum(ev, seed):
    """Q diag(ev) Q^T with Q orthogonal (QR of a Gaussian matrix): its eigenvalues are ev."""
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((len(ev), len(ev))))[0]
    A = (Q * np.asarray(ev, dtype=np.float64)) @ Q.T
    return 0.5 * (A + A.T)


# ----------------------------------------------------------------------------------------
# fallback step (Sec. 6)
# ----------------------------------------------------------------------------------------
FALLBACK_CASES = [
    # (eigenvalues of the start point, n samples, lambda, seed)
    ([0.5, 1.0, 2.0, 4.0], 6, 0.1, 0),          # cond 8:  t_f = (0.9 / 8)^2
    ([0.25, 0.5, 0.75, 1.0, 1.5], 8, 0.2, 1),    # cond 6
    ([1.0, 1.0, 2.0, 3.0, 3.0, 5.0], 4, 0.05, 2),  # cond 5, repeated eigenvalues
]


def _fallback_violations(case, iters=4):
    """Count the ways pista() with t_min = 2 departs from what Sec. 6 fixes."""
    ev, m, lam, seed = case
    n = len(ev)
    S = _problem(n, m, 100 + seed)
    A0 = _spd_with_spectrum(ev, seed)
    bad = 0
    # the first step: its eigenvalues are known exactly, so t_f is a closed form
    want0 = (0.9 * min(ev) / max(ev)) ** 2
    res = pista.pista(S, lam, tol=0.0, A0=A0, max_iter=iters, t_min=2.0, trace=True)
    tr = res["trace"]
    if len(tr) != iters:   # a step was refused: the path stopped early
        return 1 + iters - len(tr)
    bad += int(abs(tr[0]["t"] - want0) > 1e-12 * want0)
    # every step is taken at t_f, is positive definite and decreases F (Lemma 4.1)
    for h in tr:
        bad += int(not h["accepted"]) + int(h["trials"] != 1) + int(not (h["dF"] < 0.0))
    # later steps: t_f from the iterate's singular values (a route independent of eigvalsh)
    for k in range(1, iters):
        Ak = pista.pista(S, lam, tol=0.0, A0=A0, max_iter=k, t_min=2.0)["theta"]
        bad += int(pista.cholesky(Ak) is None)
        sv = np.linalg.svd(Ak, compute_uv=False)
        want = (0.9 * sv[-1] / sv[0]) ** 2
        bad += int(abs(tr[k]["t"] - want) > 1e-10 * want)
    return bad


@pytest.mark.parametrize("case", FALLBACK_CASES, ids=["cond8", "cond6", "cond5_repeated"])
def test_fallback_step_is_sec6_closed_form(case):
    assert _fallback_violations(case) == 0


def test_fallback_replay_hook_takes_the_given_steps():
    """pista(fallback=...) replays given step sizes; with t_f itself it is the plain run."""
    ev, m, lam, seed = FALLBACK_CASES[0]
    S = _problem(len(ev), m, 100 + seed)
    A0 = _spd_with_spectrum(ev, seed)
    plain = pista.pista(S, lam, tol=0.0, A0=A0, max_iter=3, t_min=2.0, trace=True)
    same = pista.pista(S, lam, tol=0.0, A0=A0, max_iter=3, t_min=2.0, trace=True,
                       fallback=lambda k, A: pista.fallback_step(A))
    assert np.array_equal(plain["theta"], same["theta"])
    ts = [0.01, 0.02, 0.005]
    given = pista.pista(S, lam, tol=0.0, A0=A0, max_iter=3, t_min=2.0, trace=True,
                        fallback=lambda k, A: ts[k])
    assert [h["t"] for h in given["trace"]] == ts


def _fb_no_square(A):
    return pista.FALLBACK_FACTOR / pista.cond2(A)


def _fb_factor_outside(A):
    return pista.FALLBACK_FACTOR / pista.cond2(A) ** 2


def _fb_lambda_max_only(A):
    return (pista.FALLBACK_FACTOR / np.linalg.eigvalsh(A)[-1]) ** 2


def _fb_frobenius_cond(A):
    return (pista.FALLBACK_FACTOR / (np.linalg.norm(A) * np.linalg.norm(np.linalg.inv(A)))) ** 2


@pytest.mark.parametrize("mutant", [_fb_no_square, _fb_factor_outside, _fb_lambda_max_only,
                                    _fb_frobenius_cond],
                         ids=["no_square", "factor_outside", "lambda_max_only", "frobenius_cond"])
def test_planted_fallback_mistake_is_caught(mutant, monkeypatch):
    monkeypatch.setattr(pista, "fallback_step", mutant)
    assert sum(_fallback_violations(c, iters=2) for c in FALLBACK_CASES) > 0


# ----------------------------------------------------------------------------------------
# objective difference (eq. t_cond_min, reading R6)
# ----------------------------------------------------------------------------------------
def _dF_exact(S, A, At, lam):
    """F(At) - F(A) in 50-digit arithmetic from the FP64 entries (each converts exactly)."""
    mp.mp.dps = 50
    n = A.shape[0]
    MA = mp.matrix([[mp.mpf(float(x)) for x in row] for row in A])
    MAt = mp.matrix([[mp.mpf(float(x)) for x in row] for row in At])
    dld = mp.log(mp.det(MAt)) - mp.log(mp.det(MA))
    lin = mp.mpf(0)
    l1 = mp.mpf(0)
    for i in range(n):
        for j in range(n):
            a, at = mp.mpf(float(A[i, j])), mp.mpf(float(At[i, j]))
            lin += mp.mpf(float(S[i, j])) * (at - a)
            l1 += abs(at) - abs(a)
    return -dld + lin + mp.mpf(lam) * l1


def _difference_case(n, seed, eps):
    """(S, A, L, At, lam, delta): A sparse SPD, At = A + eps P, P symmetric on the support of
    A plus two new entries (so the l1 term changes too)."""
    rng = np.random.default_rng(seed)
    S = _problem(n, n + 3, 200 + seed)
    lam = 0.1
    A = np.diag(rng.uniform(1.0, 2.0, n))
    for i in range(n - 1):
        A[i, i + 1] = A[i + 1, i] = rng.uniform(-0.3, 0.3)
    P = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1):
            if A[i, j] != 0.0:
                P[i, j] = P[j, i] = rng.uniform(-1.0, 1.0)
    P[n - 1, 0] = P[0, n - 1] = 0.7
    P[n - 1, 1] = P[1, n - 1] = -0.4
    At = A + eps * P
    L = pista.cholesky(A)
    return S, A, L, At, lam, pista.decrease_slack(S, A, lam)


DIFF_CASES = [(3, 0), (5, 1), (8, 2), (8, 3)]


def _difference_violations(objective_difference):
    bad = 0
    for n, seed in DIFF_CASES:
        # inside the band: the Cholesky difference cannot resolve dF; tier 2 must, to 1e-6
        S, A, L, At, lam, delta = _difference_case(n, seed, 1e-13)
        dF, tier = objective_difference(S, A, L, At, lam, delta)
        exact = float(_dF_exact(S, A, At, lam))
        bad += int(abs(exact) > pista.DIFF_BAND * delta)   # the case is inside the band
        bad += int(tier != 2)
        bad += int(not (abs(dF - exact) <= 1e-6 * abs(exact)))
        # outside the band: the two Cholesky log-dets decide, accurate to rounding
        S, A, L, At, lam, delta = _difference_case(n, seed, 1e-3)
        dF, tier = objective_difference(S, A, L, At, lam, delta)
        exact = float(_dF_exact(S, A, At, lam))
        bad += int(tier != 1)
        bad += int(not (abs(dF - exact) <= 1e-10 * abs(exact)))
    return bad


def test_objective_difference_matches_50_digit_determinants():
    assert _difference_violations(pista.objective_difference) == 0


def test_objective_difference_not_pd_is_infinite():
    S, A, L, At, lam, delta = _difference_case(5, 0, 1e-13)
    dF, tier = pista.objective_difference(S, A, L, A - 10.0 * np.eye(5), lam, delta)
    assert dF == np.inf and tier == 1


# planted mistakes: each replaces one piece of reading R6
def _od_mutant(one_sided=False, plain_log=False, no_band=False, drop_l1=False):
    import scipy.linalg

    def od(S, A, L, At, lam, delta):
        Lt = pista.cholesky(At)
        if Lt is None:
            return np.inf, 1
        dA = At - A
        l1 = 0.0 if drop_l1 else lam * float(np.sum(np.abs(At) - np.abs(A)))
        lin = float(np.sum(S * dA)) + l1
        dld = 2.0 * float(np.sum(np.log(np.diag(Lt)))) - 2.0 * float(np.sum(np.log(np.diag(L))))
        dF = -dld + lin
        if no_band or abs(dF) > pista.DIFF_BAND * delta:
            return dF, 1
        X = scipy.linalg.solve_triangular(L, dA, lower=True)
        E = X if one_sided else scipy.linalg.solve_triangular(L, X.T, lower=True)
        mu = np.linalg.eigvalsh(0.5 * (E + E.T))
        logs = np.log(1.0 + mu) if plain_log else np.log1p(mu)
        return -float(np.sum(logs)) + lin, 2
    return od


def test_mutant_harness_reproduces_the_oracle():
    assert _difference_violations(_od_mutant()) == 0


@pytest.mark.parametrize("kw", [dict(one_sided=True), dict(plain_log=True), dict(no_band=True),
                                dict(drop_l1=True)],
                         ids=["E_one_sided", "log_not_log1p", "no_tier2", "dropped_l1"])
def test_planted_difference_mistake_is_caught(kw):
    assert _difference_violations(_od_mutant(**kw)) > 0
