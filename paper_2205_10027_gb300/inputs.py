"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds a ground-truth precision matrix Theta_true, draws m samples
y ~ N(0, Theta_true^{-1}) and forms the empirical covariance S of Sec. 3.1
(eq. empirical_cov: centred by the sample mean, divided by m).  It holds none of
pISTA's arithmetic, so both the CUDA path (through its tests and benchmark) and the
FP64 oracle take their inputs from here.

Generators (Sec. 6.1.1 describes the paper's own; the ones here follow the benchmark
configurations this library is measured on):
  chain  tridiagonal, diagonal 1.25, off-diagonals -0.5
  er     Erdos-Renyi graph of a given average degree, off-diagonal weights
         +-U[0.1, 0.5] (sign by a fair coin), diagonal shifted so lambda_min = 0.1
  grid   2-D lattice Laplacian-like precision, 4-neighbour weights -1, diagonal 4.1
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg


# ----------------------------------------------------------------------------------------
# ground-truth precision matrices
# ----------------------------------------------------------------------------------------
def theta_chain(n: int, diag: float = 1.25, off: float = -0.5) -> np.ndarray:
    T = np.zeros((n, n))
    idx = np.arange(n)
    T[idx, idx] = diag
    T[idx[:-1], idx[:-1] + 1] = off
    T[idx[:-1] + 1, idx[:-1]] = off
    return T


def theta_grid(side: int, diag: float = 4.1, off: float = -1.0, n: int | None = None) -> np.ndarray:
    """side x side lattice, nodes numbered row by row; the first n nodes are kept."""
    N = side * side
    n = N if n is None else n
    T = np.zeros((n, n))
    for v in range(n):
        T[v, v] = diag
        r, c = divmod(v, side)
        for rr, cc in ((r + 1, c), (r, c + 1)):
            if rr < side and cc < side:
                u = rr * side + cc
                if u < n:
                    T[v, u] = T[u, v] = off
    return T


def theta_er(n: int, avg_degree: float, rng: np.random.Generator, wlo: float = 0.1,
             whi: float = 0.5, min_eig: float = 0.1) -> np.ndarray:
    p = min(1.0, avg_degree / max(n - 1, 1))
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    iu, ju = iu[keep], ju[keep]
    w = rng.uniform(wlo, whi, iu.size) * np.where(rng.random(iu.size) < 0.5, -1.0, 1.0)
    T = np.zeros((n, n))
    T[iu, ju] = w
    T[ju, iu] = w
    shift = min_eig - float(np.linalg.eigvalsh(T)[0])
    T[np.arange(n), np.arange(n)] += shift
    return T


# ----------------------------------------------------------------------------------------
# samples and empirical covariance (eq. empirical_cov)
# ----------------------------------------------------------------------------------------
def sample_covariance(theta: np.ndarray, m: int, rng: np.random.Generator) -> np.ndarray:
    """y = L^{-T} z with Theta = L L^T and z ~ N(0, I), so cov(y) = Theta^{-1}."""
    n = theta.shape[0]
    L = np.linalg.cholesky(theta)
    Z = rng.standard_normal((n, m))
    Y = scipy.linalg.solve_triangular(L.T, Z, lower=False)
    Y -= Y.mean(axis=1, keepdims=True)
    S = (Y @ Y.T) / m
    return 0.5 * (S + S.T)


# ----------------------------------------------------------------------------------------
# benchmark workloads
# ----------------------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    S: np.ndarray            # float64, or float32 when the workload stores S in FP32
    lam: float
    tol: float
    meta: dict = field(default_factory=dict)


def chain_n100() -> Problem:
    """n = 100 chain, m = 50 samples, seed 0, lam = 0.1, tolerance 1e-8."""
    rng = np.random.default_rng(0)
    S = sample_covariance(theta_chain(100), 50, rng)
    return Problem("chain_n100_m50", S, 0.1, 1e-8, dict(n=100, m=50, seed=0))


def er_n2000(lam: float = 0.1, n: int = 2000, m: int | None = None, seed: int = 1) -> Problem:
    """Erdos-Renyi average degree 5, m = n/2 samples, S stored in FP32, tolerance 1e-6."""
    rng = np.random.default_rng(seed)
    m = n // 2 if m is None else m
    S = sample_covariance(theta_er(n, 5.0, rng), m, rng).astype(np.float32)
    return Problem(f"er_n{n}_m{m}", S, lam, 1e-6, dict(n=n, m=m, seed=seed, s_dtype="f32"))


def grid_n10000(side: int = 100, m: int = 2000, seed: int = 2, lam: float = 0.1) -> Problem:
    """side x side lattice (n = side^2), m samples, lam = 0.1, tolerance 1e-6."""
    rng = np.random.default_rng(seed)
    S = sample_covariance(theta_grid(side), m, rng)
    n = side * side
    return Problem(f"grid_n{n}_m{m}", S, lam, 1e-6, dict(n=n, m=m, seed=seed, side=side))


def batch_path_problems(count: int = 512, nmin: int = 32, nmax: int = 1024,
                        n_lambda: int = 8, seed: int = 3) -> list[dict]:
    """Independent problems with n log-uniform in [nmin, nmax], ER degree 3, m = n/2,
    S in FP32, and a descending lambda path logspace(0.5 -> 0.02)."""
    size_rng = np.random.default_rng(seed)
    ns = np.round(np.exp(size_rng.uniform(math.log(nmin), math.log(nmax), count))).astype(int)
    lams = list(np.logspace(math.log10(0.5), math.log10(0.02), n_lambda))
    probs = []
    for i, n in enumerate(ns):
        rng = np.random.default_rng(seed + i)
        S = sample_covariance(theta_er(int(n), 3.0, rng), max(int(n) // 2, 2), rng)
        probs.append(dict(n=int(n), S=S.astype(np.float32), lambdas=lams))
    return probs


def served_stream(count: int = 20000, rate_hz: float = 200.0, nmin: int = 64, nmax: int = 4096,
                  pool: int = 256, seed: int = 5):
    """Poisson arrivals; each request names a dataset id from a pool of seeded
    (structure, n, seed) triples, and a lambda ~ U[0.05, 0.3].  Returns (arrival times in s,
    dataset ids, lambdas, pool description); ``served_dataset`` builds S for an id."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, count)
    arrivals = np.cumsum(gaps)
    pool_desc = []
    for d in range(pool):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        structure = "chain" if rng.random() < 0.5 else "grid"
        pool_desc.append(dict(structure=structure, n=n, seed=1000 + d))
    ids = rng.integers(0, pool, count)
    lams = rng.uniform(0.05, 0.3, count)
    return arrivals, ids, lams, pool_desc


def served_dataset(desc: dict) -> np.ndarray:
    n, rng = desc["n"], np.random.default_rng(desc["seed"])
    if desc["structure"] == "chain":
        theta = theta_chain(n)
    else:
        theta = theta_grid(int(math.ceil(math.sqrt(n))), n=n)
    return sample_covariance(theta, n, rng)


# ----------------------------------------------------------------------------------------
# the paper's own synthetic protocol (Sec. 6.1.1): chain, random U^T U, planar Delaunay
# Laplacian, shifted by max(-1.2 lambda_min, 0.1) I; m = 3% n samples.  The samples are
# standardised to unit variance (diag(S) = I), the preprocessing the paper states for its
# real data, which is the reading under which these workloads reproduce Table 1.
# ----------------------------------------------------------------------------------------
def _shift_pd(T: np.ndarray) -> np.ndarray:
    n = T.shape[0]
    if n <= 2000:
        lmin = float(np.linalg.eigvalsh(T)[0])
    else:
        # the matrices are sparse: shift-invert Lanczos for the eigenvalue nearest below the
        # spectrum (a bound sigma below every eigenvalue by Gershgorin)
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        Ts = sp.csc_matrix(T)
        sigma = -float(np.max(np.abs(T).sum(axis=1))) - 1.0
        lmin = float(spla.eigsh(Ts, k=1, sigma=sigma, which="LM", return_eigenvectors=False)[0])
    return T + max(-1.2 * lmin, 0.1) * np.eye(n)


def paper_theta(kind: str, n: int, rng: np.random.Generator) -> np.ndarray:
    if kind == "chain":
        return _shift_pd(theta_chain(n, 1.0, -0.5))
    if kind == "random":
        # U sparse with +-1 entries; density chosen so that U^T U has about 0.5% nonzeros;
        # off-diagonal entries are kept in [-1, 1] as the paper describes
        p = math.sqrt(-math.log(1.0 - 0.005) / n)
        U = (rng.random((n, n)) < p) * np.where(rng.random((n, n)) < 0.5, -1.0, 1.0)
        T = U.T @ U
        off = T - np.diag(np.diag(T))
        T = np.diag(np.diag(T)) + np.clip(off, -1.0, 1.0)
        return _shift_pd(T)
    if kind == "planar":
        from scipy.spatial import Delaunay
        pts = rng.random((n, 2))
        tri = Delaunay(pts)
        T = np.zeros((n, n))
        for s in tri.simplices:
            for a in range(3):
                i, j = s[a], s[(a + 1) % 3]
                T[i, j] = T[j, i] = -1.0
        np.fill_diagonal(T, -T.sum(axis=1))
        return _shift_pd(T)
    raise ValueError(kind)


def paper_protocol(kind: str, n: int, seed: int, m_frac: float = 0.03, return_theta: bool = False):
    """S of the paper's synthetic protocol (standardised samples); with return_theta, also
    the ground-truth precision matrix it was sampled from."""
    rng = np.random.default_rng(seed)
    T = paper_theta(kind, n, rng)
    S = sample_covariance(T, max(2, int(round(m_frac * n))), rng)
    d = 1.0 / np.sqrt(np.diag(S))
    S = S * d[:, None] * d[None, :]
    S = 0.5 * (S + S.T)
    return (S, T) if return_theta else S
