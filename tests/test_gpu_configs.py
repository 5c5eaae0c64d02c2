"""Whole solves at the workloads' own sizes, every precision form against the FP64 oracle.

  * Erdos-Renyi n = 2,000 (average degree 5, m = 1,000, S stored in FP32), lambda in
    {0.05, 0.1}, tolerance 1e-6, in FP64, TF32x3 and BF16x3;
  * the 50 x 50 lattice (n = 2,500: several recursion levels on the tensor cores, 128 x 256
    tiles, the grouped tile order), tolerance 1e-6, all three forms;
  * the n = 10,000 lattice of the benchmark: the BF16x3 solve re-checked on the host (KKT from
    numpy's FP64 inverse of the returned Theta) and against the FP64 GPU form's result;
  * the paper's own protocol at n = 1,000 (Sec. 6.1.1, Table 1: chain, random U^T U, planar;
    m = 3% n, standardised samples, stop at eps = 1e-2), FP64 and BF16x3.

Stated per result.  FP64: objective gap <= 1e-10 always; where both sides take the same
path (the same iteration count) relative Frobenius <= 1e-9; where a free-set or accept test
lands within rounding of its threshold and the paths part (reading R17: Theta* is unique,
the path to it is not), both satisfy the stop test and lie within 1e3 tol of each other.
Split-precision forms: the stop test re-evaluated on the host in FP64 (<= 1.05 tol), the
iteration count within 15% (+3) of the oracle's, and within 1e3 tol (relative Frobenius) of
the oracle's result.  Each error is printed (pytest -rP shows it).
"""
import numpy as np
import pytest

from oracle import pista
from paper_2205_10027_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FORMS = ["fp64", "tf32x3", "bf16x3"]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _host_kkt(S, theta, lam):
    g = np.asarray(S, np.float64) - np.linalg.inv(theta)
    return float(np.sum(np.abs(pista.min_norm_subgradient(theta, g, lam))) / np.sum(np.abs(theta)))


def _check(prec, S, lam, tol, res, theta, ref, label, it_slack=3):
    assert res["status"] == 0 and ref["status"] == "converged", label
    err = _rel(theta, ref["theta"])
    gap = abs(res["objective"] - ref["F"]) / abs(ref["F"])
    r = _host_kkt(S, theta, lam)
    print(f"{label} {prec}: iterations {res['iterations']} (oracle {ref['iterations']}) "
          f"rel_frob {err:.2e} objective_gap {gap:.2e} host_kkt {r:.2e}")
    if prec == "fp64":
        assert gap <= 1e-10, label
        if res["iterations"] == ref["iterations"]:
            assert err <= 1e-9, label
        else:
            print(f"{label}: the FP64 paths parted at a rounding-level decision")
            assert r <= 1.05 * tol and err <= 1e3 * tol, label
    else:
        assert r <= 1.05 * tol, label
        assert abs(res["iterations"] - ref["iterations"]) <= max(it_slack, 0.15 * ref["iterations"] + 3), label
        assert err <= 1e3 * tol, label


@pytest.fixture(scope="module")
def er2000():
    out = {}
    for lam in (0.1, 0.05):
        p = inputs.er_n2000(lam=lam)
        out[lam] = (p, pista.pista(p.S.astype(np.float64), lam, tol=p.tol))
    return out


@pytest.mark.parametrize("lam", [0.1, 0.05])
@pytest.mark.parametrize("prec", FORMS)
def test_er_n2000(glasso, er2000, prec, lam):
    p, ref = er2000[lam]
    assert p.S.dtype == np.float32
    with glasso.Handle(precision=prec, max_iter=2000) as h:
        theta, res = h.solve(p.S, lam, p.tol)
    _check(prec, p.S, lam, p.tol, res, theta, ref, f"er_n2000 lam={lam}")


@pytest.fixture(scope="module")
def grid2500():
    p = inputs.grid_n10000(side=50, m=500, seed=2)
    return p, pista.pista(p.S, p.lam, tol=1e-6)


@pytest.mark.parametrize("prec", FORMS)
def test_grid_n2500(glasso, grid2500, prec):
    p, ref = grid2500
    with glasso.Handle(precision=prec, products="dense", max_iter=2000) as h:
        theta, res = h.solve(p.S, p.lam, 1e-6)
    _check(prec, p.S, p.lam, 1e-6, res, theta, ref, "grid50x50 dense products")


def test_grid_n10000_bf16x3_host_recheck(glasso):
    p = inputs.grid_n10000()
    S_dev = torch.from_numpy(np.ascontiguousarray(p.S)).cuda()
    with glasso.Handle(precision="bf16x3", max_iter=2000) as h:
        theta_m, res_m = h.solve(S_dev, p.lam, p.tol)
    with glasso.Handle(precision="fp64", max_iter=2000) as h:
        theta_f, res_f = h.solve(S_dev, p.lam, p.tol)
    theta_m, theta_f = theta_m.cpu().numpy(), theta_f.cpu().numpy()
    assert res_m["status"] == 0 and res_f["status"] == 0
    r = _host_kkt(p.S, theta_m, p.lam)
    err = _rel(theta_m, theta_f)
    print(f"grid100x100 bf16x3: iterations {res_m['iterations']} (fp64 form {res_f['iterations']}) "
          f"host_kkt {r:.2e} rel_frob_vs_fp64_form {err:.2e}")
    assert r <= 1.05 * p.tol
    assert err <= 1e3 * p.tol


PAPER = [("chain", 0.6), ("chain", 0.4), ("random", 0.6), ("random", 0.4), ("planar", 0.6), ("planar", 0.4)]


@pytest.mark.parametrize("kind,alpha", PAPER, ids=[f"{k}-{a}" for k, a in PAPER])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_paper_protocol_table1(glasso, prec, kind, alpha):
    eps = 1e-2
    S = inputs.paper_protocol(kind, 1000, seed=300)
    ref = pista.pista(S, alpha, tol=eps)
    with glasso.Handle(precision=prec) as h:
        theta, res = h.solve(S, alpha, eps)
    if prec == "fp64":
        _check(prec, S, alpha, eps, res, theta, ref, f"paper {kind} alpha={alpha}")
        return
    # at eps = 1e-2 the solve stops far from the optimum, so the split-precision form is held
    # to the oracle's path: the same iteration count (or one apart, when the loose stop test
    # lands within rounding of its threshold) and, on the same count, the iterate within the
    # direction's own accuracy (BF16x3 sandwich, relative error <= 1e-4 per step)
    assert res["status"] == 0 and ref["status"] == "converged"
    r = _host_kkt(S, theta, alpha)
    err = _rel(theta, ref["theta"])
    print(f"paper {kind} alpha={alpha} {prec}: iterations {res['iterations']} (oracle {ref['iterations']}) "
          f"rel_frob {err:.2e} host_kkt {r:.2e}")
    assert r <= 1.05 * eps
    assert abs(res["iterations"] - ref["iterations"]) <= 1
    if res["iterations"] == ref["iterations"]:
        assert err <= 1e-3
