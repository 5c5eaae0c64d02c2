"""The plain proximal-gradient method (glasso_method GISTA) on the GPU against the oracles:
the graphical-lasso optimum is unique, so G-ISTA must reach the point pISTA and the
independent proximal-gradient oracle reach, by its own route."""
import numpy as np
import pytest

from oracle import closed, gista, pista
from paper_2205_10027_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _host_kkt(S, theta, lam):
    g = S - np.linalg.inv(theta)
    return np.sum(np.abs(pista.min_norm_subgradient(theta, g, lam))) / np.sum(np.abs(theta))


def test_gista_two_by_two_closed_form(glasso):
    S = np.array([[1.3, 0.45], [0.45, 0.8]])
    lam = 0.2
    with glasso.Handle(precision="fp64", method="gista", max_iter=100000) as h:
        theta, res = h.solve(S, lam, 1e-12)
    assert res["status"] == 0
    assert _rel(theta, closed.two_by_two_solution(S, lam)) <= 1e-10


def test_gista_fp64_chain_matches_the_optimum(glasso):
    p = inputs.chain_n100()
    tol = 1e-8
    with glasso.Handle(precision="fp64", method="gista", max_iter=100000) as h:
        theta, res = h.solve(p.S, p.lam, tol)
    assert res["status"] == 0 and res["iterations"] > 0
    assert _host_kkt(p.S, theta, p.lam) <= 1.05 * tol
    ref = pista.pista(p.S, p.lam, tol=1e-11)
    assert _rel(theta, ref["theta"]) <= 1e-5
    # and the independent CPU proximal-gradient oracle lands on the same point
    g_theta, g_r, _ = gista.gista(p.S, p.lam, tol=tol)
    assert _rel(theta, g_theta) <= 1e-5


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_gista_split_precision_grid(glasso, precision):
    p = inputs.grid_n10000(side=12, m=60, seed=6)
    tol = 1e-6
    with glasso.Handle(precision=precision, method="gista", max_iter=100000) as h:
        theta, res = h.solve(p.S, p.lam, tol)
    assert res["status"] == 0
    assert _host_kkt(p.S, theta, p.lam) <= 1.05 * tol
    ref = pista.pista(p.S, p.lam, tol=1e-10)
    assert _rel(theta, ref["theta"]) <= 1e3 * tol
