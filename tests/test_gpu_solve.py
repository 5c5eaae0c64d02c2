"""Whole-solve parity of the FP64 form against the FP64 oracle, closed forms through the
GPU, error statuses, and the invariants that hold at any size."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import closed, pista
from paper_2205_10027_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _mat(rows):
    return np.array([[float(Fraction(x)) for x in r] for r in rows])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _same_path(gpu_res, theta, ref, frob=1e-9, gap=1e-10):
    assert gpu_res["status"] == 0 and ref["status"] == "converged"
    assert gpu_res["iterations"] == ref["iterations"]
    assert _rel(theta, ref["theta"]) <= frob
    assert abs(gpu_res["objective"] - ref["F"]) <= gap * abs(ref["F"])


def test_chain_n100_tight(fp64):
    p = inputs.chain_n100()
    theta, res = fp64.solve(p.S, p.lam, 1e-12)
    ref = pista.pista(p.S, p.lam, tol=1e-12)
    _same_path(res, theta, ref)
    assert res["rel_kkt_l1"] <= 1e-12


def test_chain_n100_workload_tolerance(fp64):
    p = inputs.chain_n100()
    theta, res = fp64.solve(p.S, p.lam, p.tol)
    ref = pista.pista(p.S, p.lam, tol=p.tol)
    _same_path(res, theta, ref)


def test_er_small_tight(fp64):
    p = inputs.er_n2000(lam=0.1, n=150, seed=11)
    theta, res = fp64.solve(p.S, p.lam, 1e-10)
    ref = pista.pista(p.S.astype(np.float64), p.lam, tol=1e-10)
    _same_path(res, theta, ref)


@pytest.mark.parametrize("side", [15, 20])
def test_grid_small(fp64, side):
    p = inputs.grid_n10000(side=side, m=side * side // 5, seed=3)
    theta, res = fp64.solve(p.S, p.lam, 1e-8)
    ref = pista.pista(p.S, p.lam, tol=1e-8)
    _same_path(res, theta, ref)


@pytest.mark.slow
def test_er_n2000_fp32_storage(fp64):
    p = inputs.er_n2000(lam=0.1)
    assert p.S.dtype == np.float32
    theta, res = fp64.solve(p.S, p.lam, p.tol)
    ref = pista.pista(p.S.astype(np.float64), p.lam, tol=p.tol)
    _same_path(res, theta, ref)


def test_golden_closed_forms(fp64):
    gold = json.load(open(GOLDEN))
    for case in gold["optimum_cases"]:
        S, lam = _mat(case["S"]), float(Fraction(case["lam"]))
        theta, res = fp64.solve(S, lam, 1e-14)
        assert res["status"] == 0, case["name"]
        assert _rel(theta, _mat(case["theta"])) <= 1e-12, case["name"]
    case = gold["first_iterate_cases"][0]
    S, lam = _mat(case["S"]), float(Fraction(case["lam"]))
    with fp64_handle_max_iter(1) as h:
        theta, res = h.solve(S, lam, 0.0)
    assert res["iterations"] == 1
    assert np.max(np.abs(theta - _mat(case["theta1"]))) <= 1e-15


class fp64_handle_max_iter:
    def __init__(self, k):
        from paper_2205_10027_gb300 import binding
        self.h = binding.Handle(precision="fp64", max_iter=k)

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        self.h.close()


def test_diagonal_regime_returns_at_iteration_zero(fp64):
    p = inputs.chain_n100()
    lam = float(np.max(np.abs(p.S - np.diag(np.diag(p.S))))) * 1.01
    theta, res = fp64.solve(p.S, lam, 1e-12)
    assert res["iterations"] == 0 and res["status"] == 0
    assert np.array_equal(theta, closed.diagonal_solution(p.S, lam))


def test_max_iter_returns_last_pd_iterate():
    from paper_2205_10027_gb300 import binding
    p = inputs.chain_n100()
    with binding.Handle(precision="fp64", max_iter=2) as h:
        theta, res = h.solve(p.S, p.lam, 1e-14)
    assert res["status"] == binding.MAX_ITER and res["iterations"] == 2
    ref = pista.pista(p.S, p.lam, tol=1e-14, max_iter=2)
    assert _rel(theta, ref["theta"]) <= 1e-12
    assert np.all(np.linalg.eigvalsh(theta) > 0)


def test_warm_start_at_the_solution(fp64):
    p = inputs.chain_n100()
    theta, _ = fp64.solve(p.S, p.lam, 1e-12)
    theta2, res = fp64.solve(p.S, p.lam, 1e-10, theta0=theta)
    assert res["iterations"] == 0
    assert np.array_equal(theta, theta2)


def test_device_memory_and_fp32(fp64):
    p = inputs.er_n2000(lam=0.1, n=200, seed=21)
    S32 = torch.from_numpy(p.S).cuda()
    theta_d, res = fp64.solve(S32, p.lam, 1e-9)
    theta_h, res_h = fp64.solve(p.S, p.lam, 1e-9)
    assert theta_d.is_cuda and theta_d.dtype == torch.float64
    assert np.array_equal(theta_d.cpu().numpy(), theta_h)   # same kernels, same inputs
    assert res["iterations"] == res_h["iterations"]


def test_input_errors(fp64, glasso):
    p = inputs.chain_n100()
    bad = p.S.copy()
    bad[3, 7] += 1e-6
    with pytest.raises(glasso.GlassoError) as e:
        fp64.solve(bad, 0.1, 1e-6)
    assert e.value.status == 2
    bad = p.S.copy()
    bad[5, 5] = np.nan
    with pytest.raises(glasso.GlassoError) as e:
        fp64.solve(bad, 0.1, 1e-6)
    assert e.value.status == 3
    with pytest.raises(glasso.GlassoError) as e:
        fp64.solve(p.S, -0.1, 1e-6)
    assert e.value.status == 1
    with pytest.raises(glasso.GlassoError) as e:
        fp64.solve(p.S, 0.1, 1e-6, theta0=-np.eye(100))
    assert e.value.status == 4
    # the handle still works after the errors
    _, res = fp64.solve(p.S, p.lam, 1e-6)
    assert res["status"] == 0


def test_monotone_pd_kkt_certificate_n600(fp64):
    """Properties that hold at any size: the returned Theta is PD and satisfies the KKT
    conditions of Sec. 5.1 to the stop tolerance (checked here with numpy's inverse)."""
    p = inputs.er_n2000(lam=0.08, n=600, seed=31)
    S = p.S.astype(np.float64)
    theta, res = fp64.solve(p.S, p.lam, 1e-9)
    assert res["status"] == 0
    assert np.all(np.linalg.eigvalsh(theta) > 0)
    W = np.linalg.inv(theta)
    g = S - W
    Z = np.where(theta != 0, g + p.lam * np.sign(theta), np.sign(g) * np.maximum(np.abs(g) - p.lam, 0))
    r = np.sum(np.abs(Z)) / np.sum(np.abs(theta))
    assert r <= 2e-9
    assert abs(res["rel_kkt_l1"] - r) <= 1e-3 * r + 1e-14


def test_stepwise_equals_solve(fp64, glasso):
    p = inputs.chain_n100()
    theta, res = fp64.solve(p.S, p.lam, p.tol)
    fp64.begin(p.S, p.lam)
    steps = 0
    while True:
        st, r = fp64.step(p.tol)
        assert r["kernel_launches"] > 0
        if st != glasso.PENDING:
            break
        steps += 1
    out = np.empty_like(p.S)
    fp64.end(out)
    assert st == glasso.OK and steps == res["iterations"]
    assert np.array_equal(out, theta)
    assert res["kernel_launches"] > 0


def test_profile_accounts_kernel_classes(glasso):
    p = inputs.grid_n10000(side=12, m=30)
    with glasso.Handle(precision="fp64") as h:   # fresh: no factorisation graph captured yet
        h.profile_start()
        h.solve(p.S, p.lam, 1e-6)
        prof = h.profile_stop()
    # the FP64 form takes the sparse sandwich on this (sparse) iterate
    for cls in ("spmm", "inverse", "gradient", "trial"):
        assert prof[cls]["launches"] > 0 and prof[cls]["ms"] > 0 and prof[cls]["work"] > 0
    assert "sandwich" not in prof
    # factorisations run launch by launch until their CUDA graph exists, then as one replay
    assert prof["trailing"]["launches"] > 0 and prof["factor"]["launches"] > 0


def test_profile_mixed_classes(glasso):
    """The split-precision form also accounts its FP64 residual and the symmetrising passes."""
    p = inputs.grid_n10000(side=12, m=30)
    with glasso.Handle(precision="tf32x3") as h:
        h.profile_start()
        h.solve(p.S, p.lam, 1e-6)
        prof = h.profile_stop()
    for cls in ("residual", "aux", "sandwich", "inverse"):
        assert prof[cls]["launches"] > 0 and prof[cls]["ms"] > 0 and prof[cls]["work"] > 0


def test_standardized_solve_follows_the_oracle_on_the_correlation_matrix(glasso):
    """glasso_config.standardize: the solve runs on D^{-1/2} S D^{-1/2} (entry (S_ij d_i) d_j
    on the lower triangle, mirrored), so it takes the oracle's path on that matrix."""
    p = inputs.chain_n100()
    S = p.S * np.linspace(0.5, 3.0, p.S.shape[0])[:, None] * np.linspace(0.5, 3.0, p.S.shape[0])[None, :]
    S = 0.5 * (S + S.T)
    d = 1.0 / np.sqrt(np.diag(S))
    C = (S * d[:, None]) * d[None, :]
    C = np.tril(C) + np.tril(C, -1).T
    with glasso.Handle(precision="fp64", standardize=True) as h:
        theta, res = h.solve(S, p.lam, 1e-8)
        with pytest.raises(glasso.GlassoError) as e:
            Z = S.copy()
            Z[3, 3] = 0.0
            h.solve(Z, p.lam, 1e-8)
        assert e.value.status == 1
    ref = pista.pista(C, p.lam, tol=1e-8)
    _same_path(res, theta, ref)
