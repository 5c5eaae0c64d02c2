"""The line search's two rarely-taken branches on the GPU, against the oracle.

Fallback step (Sec. 6; reading R5).  With t_min = 2 the halving loop never runs, so every
iteration takes t_f = (0.9 / cond_2 Theta)^2.  The GPU estimates cond_2 = lambda_max(Theta)
lambda_max(W) by 300 power iterations; its t_f agrees with the oracle's eigenvalue-based one
to 1e-2 (t_f is the square of 1/cond).  Given the GPU's own t, everything else of the step is
fixed, and the oracle replays the GPU's step sizes (pista(fallback=...)) to check the
iterates themselves:
  * first step from the diagonal start: Theta^1 = the hand-derived first iterate at the GPU's
    t (Theta^1_ii = a_i, Theta^1_ij = -t a_i a_j ST(S_ij, lam)) to 1e-13 of max|Theta^1| in
    FP64, 1e-8 in the split-precision forms (their W is refined to max|I - Theta W| <= 1e-9);
  * eight fallback steps: the oracle, replaying the GPU's t, reaches the same iterate: FP64
    to 1e-11 relative Frobenius; split-precision forms to 1e-4 of the distance travelled
    (once Theta fills in, the sandwich of eq. b runs as BF16x3 products, relative error
    <= 1e-4) plus 1e-8 of |Theta|.

Tier-2 objective difference (eq. t_cond_min; reading R6).  Near convergence the accept test
cannot resolve dF from two Cholesky log-dets, and the GPU evaluates
log det Theta_t - log det Theta = tr E - tr E^2 / 2 (E similar to dTheta W), where the
oracle takes sum log1p(mu), mu the eigenvalues of E.  On every iteration of the n = 100
chain solve where both sides used tier 2, the two dF agree within the series' truncation,
sum |mu|^3 / (3 (1 - max|mu|)), plus the rounding of the terms, and have the same sign
wherever the truncation cannot flip it.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import closed, pista
from paper_2205_10027_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "bf16x3"]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _grid400():
    return inputs.grid_n10000(side=20, m=80, seed=3)


@pytest.fixture(scope="module", params=PRECISIONS)
def fb_handle(request, glasso):
    h = glasso.Handle(precision=request.param, t_min=2.0)
    yield request.param, h
    h.close()


def _fallback_steps(h, p, k):
    """k step-wise iterations on the GPU; returns (the iterate, per-step result dicts)."""
    n = p.S.shape[0]
    h.begin(np.ascontiguousarray(p.S, dtype=np.float64), p.lam)
    steps = []
    for _ in range(k):
        st, res = h.step(0.0)
        steps.append(dict(res, status=st))
        if st != 11:   # GLASSO_PENDING: a step was accepted
            break
    out = np.empty((n, n), np.float64)
    h.end(out)
    return out, steps


@pytest.mark.parametrize("workload", ["chain100", "grid400"])
def test_first_fallback_step(fb_handle, workload):
    prec, h = fb_handle
    p = inputs.chain_n100() if workload == "chain100" else _grid400()
    S = np.asarray(p.S, dtype=np.float64)
    theta, steps = _fallback_steps(h, p, 1)
    s = steps[0]
    assert s["status"] == 11 and s["step_fallback"] == 1 and s["trials"] == 1
    t_gpu = s["step_t"]
    t_or = pista.fallback_step(pista.initial_point(S, p.lam))
    assert abs(t_gpu / t_or - 1.0) <= 1e-2, (t_gpu, t_or)
    want = closed.first_iterate(S, p.lam, t_gpu)
    tol = 1e-13 if prec == "fp64" else 1e-8
    assert np.max(np.abs(theta - want)) <= tol * np.max(np.abs(want))
    assert s["step_dF"] < 0.0


@pytest.mark.parametrize("workload", ["chain100", "grid400"])
def test_fallback_path_replayed_by_oracle(fb_handle, workload):
    prec, h = fb_handle
    p = inputs.chain_n100() if workload == "chain100" else _grid400()
    S = np.asarray(p.S, dtype=np.float64)
    K = 8
    theta, steps = _fallback_steps(h, p, K)
    assert len(steps) == K
    assert all(s["status"] == 11 and s["step_fallback"] == 1 and s["trials"] == 1 for s in steps)
    ts = [s["step_t"] for s in steps]
    ref = pista.pista(S, p.lam, tol=0.0, max_iter=K, t_min=2.0, trace=True, trace_iterates=True,
                      fallback=lambda k, A: ts[k])
    assert ref["iterations"] == K
    assert all(h_["accepted"] and h_["trials"] == 1 for h_ in ref["trace"])
    # the GPU's t_f against the oracle's own estimate at the same iterate
    for k, rec in enumerate(ref["trace"]):
        t_or = pista.fallback_step(rec["theta"])
        assert abs(ts[k] / t_or - 1.0) <= 1e-2, (k, ts[k], t_or)
    if prec == "fp64":
        assert _rel(theta, ref["theta"]) <= 1e-11
    else:
        travelled = np.linalg.norm(ref["theta"] - pista.initial_point(S, p.lam))
        assert np.linalg.norm(theta - ref["theta"]) <= 1e-4 * travelled + 1e-8 * np.linalg.norm(ref["theta"])
    # the decreases the accept test saw agree with the oracle's, within the rounding band of
    # the form (delta of reading R6 with u = 2^-53, or 2^-21 for the split-precision factor)
    band = 1e3 * (1.0 if prec == "fp64" else 2.0 ** 32)
    rel = 1e-6 if prec == "fp64" else 1e-3
    for k, rec in enumerate(ref["trace"]):
        assert steps[k]["step_dF"] < 0.0
        assert abs(steps[k]["step_dF"] - rec["dF"]) <= rel * abs(rec["dF"]) + band * rec["delta"]


@pytest.mark.parametrize("prec", PRECISIONS)
def test_tier2_difference_against_exact_eigenvalues(glasso, prec):
    p = inputs.chain_n100()
    S = np.asarray(p.S, dtype=np.float64)
    tol = 1e-10
    ref = pista.pista(S, p.lam, tol=tol, trace=True, trace_iterates=True)
    with glasso.Handle(precision=prec) as h:
        h.begin(S, p.lam)
        steps = []
        while True:
            st, res = h.step(tol)
            if st != 11:
                break
            steps.append(res)
        h.end(None)
    compared = 0
    for k, (g, rec) in enumerate(zip(steps, ref["trace"])):
        # compare while both sides walk the same path: same iterate support and step size
        if g["nnz"] != rec["nnz"] or g["step_t"] != rec["t"]:
            break
        if not (g["step_tier"] == 2 and rec["tier"] == 2):
            continue
        A, At = rec["theta"], rec["trial"]
        Lc = np.linalg.cholesky(A)
        X = scipy.linalg.solve_triangular(Lc, At - A, lower=True)
        E = scipy.linalg.solve_triangular(Lc, X.T, lower=True)
        mu = np.linalg.eigvalsh(0.5 * (E + E.T))
        trunc = float(np.sum(np.abs(mu) ** 3) / (3.0 * (1.0 - np.max(np.abs(mu)))))
        # rounding of the terms: tr E and tr E^2 carry the relative error of W (FP64
        # rounding, or about 1e-9 after the refinement of the split-precision forms), the
        # linear terms FP64 rounding of their entrywise sums
        w_err = 2.0 ** -53 if prec == "fp64" else 1e-8
        dA = At - A
        lin_mag = float(np.sum(np.abs(S * dA)) + p.lam * np.sum(np.abs(dA)))
        round_err = 64.0 * (w_err * float(np.sum(np.abs(mu)) + np.sum(mu * mu)) + 2.0 ** -53 * lin_mag)
        assert abs(g["step_dF"] - rec["dF"]) <= 2.0 * trunc + round_err, (k, g["step_dF"], rec["dF"], trunc)
        if abs(rec["dF"]) > 10.0 * (trunc + round_err):
            assert np.sign(g["step_dF"]) == np.sign(rec["dF"]), k
        compared += 1
    assert compared >= 5, compared
