"""Batched lambda paths and the continuous-batching server against the FP64 oracle, and the
serving identity: a request gives the same result alone and in a mix of concurrent requests.
"""
import time

import numpy as np
import pytest

from oracle import pista
from paper_2205_10027_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batch_paths_match_oracle(glasso):
    probs = inputs.batch_path_problems(count=5, nmin=32, nmax=160, n_lambda=3, seed=40)
    for p in probs:
        p["lambdas"] = [0.5, 0.35, 0.25]
        p["tol"] = 1e-9
    with glasso.Handle(precision="fp64", serve_slots=3) as h:
        thetas, results = h.solve_batch(probs)
    for p, th, rs in zip(probs, thetas, results):
        S = p["S"].astype(np.float64)
        for j, lam in enumerate(p["lambdas"]):
            assert rs[j]["status"] == 0
            ref = pista.pista(S, lam, tol=1e-9)
            # warm-started path vs a cold oracle solve: both at KKT 1e-9 of the same optimum
            assert _rel(th[j], ref["theta"]) <= 1e-6
            assert abs(rs[j]["objective"] - ref["F"]) <= 1e-9 * abs(ref["F"])


def test_batch_path_is_warm_started(glasso):
    """Each lambda of a path starts from the previous solution: repeating a lambda therefore
    takes no iteration, and a nearby lambda starts close to its optimum."""
    p = inputs.batch_path_problems(count=1, nmin=200, nmax=200, n_lambda=3, seed=41)[0]
    p["lambdas"] = [0.3, 0.3, 0.29]
    p["tol"] = 1e-8
    with glasso.Handle(precision="fp64") as h:
        th, res = h.solve_batch([p])
        cold = h.solve(p["S"], 0.29, 1e-8)[1]["iterations"]
    its = [r["iterations"] for r in res[0]]
    assert its[0] > 0 and its[1] == 0
    assert np.array_equal(th[0][0], th[0][1])
    assert its[2] < cold


def _drain(h, tickets, ns, timeout=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t, n in zip(tickets, ns):
            if t in out:
                continue
            st, res, theta = h.poll(t, n)
            if st != 11:  # not pending
                out[t] = (st, res, theta)
        assert time.time() - t0 < timeout
        time.sleep(0.002)
    return [out[t] for t in tickets]


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_served_alone_equals_in_the_mix(glasso, precision):
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(8):
        n = int(rng.integers(64, 400))
        if i % 2:
            S = inputs.sample_covariance(inputs.theta_chain(n), n, np.random.default_rng(100 + i))
        else:
            side = int(np.ceil(np.sqrt(n)))
            S = inputs.sample_covariance(inputs.theta_grid(side, n=n), n, np.random.default_rng(100 + i))
        reqs.append((S, float(rng.uniform(0.05, 0.3))))
    alone = []
    with glasso.Handle(precision=precision, serve_slots=1) as h:
        for S, lam in reqs:
            t = h.submit(S, lam, 1e-8)
            alone.append(_drain(h, [t], [S.shape[0]])[0])
    with glasso.Handle(precision=precision, serve_slots=4) as h:
        tickets = [h.submit(S, lam, 1e-8) for S, lam in reqs]
        mixed = _drain(h, tickets, [S.shape[0] for S, _ in reqs])
    for (S, lam), a, m in zip(reqs, alone, mixed):
        assert a[0] == 0 and m[0] == 0
        # same kernels, same inputs, fixed-order reductions: bit-identical alone and in the mix
        assert np.array_equal(a[2], m[2])
        assert a[1]["iterations"] == m[1]["iterations"]
        assert m[1]["t_done"] >= m[1]["t_start"] >= m[1]["t_submit"] > 0
    # and each result is the oracle's optimum
    for (S, lam), m in list(zip(reqs, mixed))[:3]:
        ref = pista.pista(S, lam, tol=1e-8)
        assert _rel(m[2], ref["theta"]) <= 1e-8


def test_served_warm_start_from_nearest_lambda(glasso):
    n = 150
    S = inputs.sample_covariance(inputs.theta_chain(n), n, np.random.default_rng(3))
    with glasso.Handle(precision="fp64", serve_slots=1) as h:
        t1 = h.submit(S, 0.2, 1e-8, dataset_id=5)
        r1 = _drain(h, [t1], [n])[0]
        t2 = h.submit(S, 0.19, 1e-8, dataset_id=5)
        r2 = _drain(h, [t2], [n])[0]
        t3 = h.submit(S, 0.19, 1e-8, dataset_id=-1)
        r3 = _drain(h, [t3], [n])[0]
    assert r1[0] == r2[0] == r3[0] == 0
    assert r2[1]["iterations"] < r3[1]["iterations"]
    assert _rel(r2[2], r3[2]) <= 1e-6


def test_served_budget_rejects_oversized(glasso):
    with glasso.Handle(precision="fp64", hbm_budget_bytes=1 << 20) as h:
        with pytest.raises(glasso.GlassoError) as e:
            h.submit(np.eye(300), 0.1, 1e-6)
        assert e.value.status == 6


def test_served_budget_admits_after_high_water(glasso):
    """Three slots each keep a workspace from a medium request; a larger request that fits the
    budget alone, but not beside those high-water workspaces, must still be admitted (idle
    slots give their workspaces back while a queued request waits)."""
    mid, big = 2000, 3000
    w_mid, w_big = glasso.workspace_bytes(mid), glasso.workspace_bytes(big)
    budget = int(1.5 * w_big)
    assert 3 * w_mid <= budget < 2 * w_mid + w_big   # the blocked configuration
    Sm = inputs.sample_covariance(inputs.theta_chain(mid), mid, np.random.default_rng(11))
    Sb = inputs.sample_covariance(inputs.theta_chain(big), big, np.random.default_rng(12))
    with glasso.Handle(precision="bf16x3", serve_slots=3, hbm_budget_bytes=budget) as h:
        ts = [h.submit(Sm, 0.2, 1e-5) for _ in range(3)]
        out = _drain(h, ts, [mid] * 3)
        assert all(o[0] == 0 for o in out)
        t = h.submit(Sb, 0.2, 1e-5)
        st, res, _ = _drain(h, [t], [big], timeout=120.0)[0]
    assert st == 0 and res["iterations"] > 0


def test_served_slot_failure_is_reported(glasso, monkeypatch):
    """A slot whose engine cannot be built (failure injected on the host) leaves the others
    serving; with every slot failed, queued requests end with the failure's status instead of
    staying pending, and further submits are refused."""
    n = 120
    S = inputs.sample_covariance(inputs.theta_chain(n), n, np.random.default_rng(13))
    monkeypatch.setenv("GLASSO_TEST_FAIL_SLOTS", "1")
    with glasso.Handle(precision="fp64", serve_slots=2) as h:
        ts = [h.submit(S, 0.2, 1e-8) for _ in range(3)]
        assert all(o[0] == 0 for o in _drain(h, ts, [n] * 3))
    monkeypatch.setenv("GLASSO_TEST_FAIL_SLOTS", "8")
    with glasso.Handle(precision="fp64", serve_slots=2) as h:
        t = h.submit(S, 0.2, 1e-8)
        t0 = time.time()
        while True:
            try:
                st = h.poll(t)[0]
            except glasso.GlassoError as e:   # a finished request with an error status
                st = e.status
            if st != 11:
                break
            assert time.time() - t0 < 30.0, "request left pending with no slot alive"
            time.sleep(0.01)
        assert st == 5   # GLASSO_ERR_OOM, the injected failure
        with pytest.raises(glasso.GlassoError) as e:
            h.submit(S, 0.2, 1e-8)
        assert e.value.status == 5


def test_served_resident_warm_start(glasso):
    """Solutions stay on the device: a request warm-started from the resident state of the
    same dataset (its Theta, inverse factor and W) reaches the same optimum as a cold solve in
    fewer iterations, in every form, and repeating a lambda takes no iteration."""
    n = 300
    S = inputs.sample_covariance(inputs.theta_grid(18, n=n), n, np.random.default_rng(14))
    for prec in ("fp64", "bf16x3"):
        with glasso.Handle(precision=prec, serve_slots=2) as h:
            r1 = _drain(h, [h.submit(S, 0.2, 1e-8, dataset_id=9)], [n])[0]
            r2 = _drain(h, [h.submit(S, 0.18, 1e-8, dataset_id=9)], [n])[0]
            r3 = _drain(h, [h.submit(S, 0.18, 1e-8, dataset_id=9)], [n])[0]
            cold = _drain(h, [h.submit(S, 0.18, 1e-8)], [n])[0]
        assert r1[0] == r2[0] == r3[0] == cold[0] == 0
        assert r2[1]["iterations"] < cold[1]["iterations"]
        assert r3[1]["iterations"] == 0
        assert _rel(r2[2], cold[2]) <= 1e-6
        ref = pista.pista(S, 0.18, tol=1e-8)
        assert _rel(r2[2], ref["theta"]) <= 1e-6
