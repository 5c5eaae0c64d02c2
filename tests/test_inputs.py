"""The seeded synthetic inputs have the structure the workloads call for (the input recipe:
generators, samples, the served stream), checked on the CPU."""
import math

import numpy as np

from paper_2205_10027_gb300 import inputs


def test_grid_precision_is_the_lattice_laplacian_shift():
    T = inputs.theta_grid(10)
    assert np.all(np.diag(T) == 4.1)
    off = T - np.diag(np.diag(T))
    assert set(np.unique(off)) == {-1.0, 0.0}
    deg = np.sum(off != 0, axis=1)
    assert deg.min() == 2 and deg.max() == 4           # corners and interior nodes
    assert np.sum(off != 0) == 2 * 2 * 10 * 9          # 180 lattice edges, both triangles
    # 4.1 minus the largest eigenvalue of the lattice adjacency (4 cos(pi / 11) for 10 x 10)
    assert math.isclose(np.linalg.eigvalsh(T)[0], 4.1 - 4 * math.cos(math.pi / 11), rel_tol=1e-12)


def test_chain_precision():
    T = inputs.theta_chain(6)
    assert np.all(np.diag(T) == 1.25)
    assert np.all(np.diag(T, 1) == -0.5) and np.count_nonzero(np.triu(T, 2)) == 0


def test_er_precision_degree_weights_and_shift():
    rng = np.random.default_rng(0)
    T = inputs.theta_er(400, 5.0, rng)
    off = T - np.diag(np.diag(T))
    w = np.abs(off[off != 0])
    assert w.min() >= 0.1 and w.max() <= 0.5
    assert abs(np.count_nonzero(off) / 400 - 5.0) < 0.5   # average degree
    assert math.isclose(np.linalg.eigvalsh(T)[0], 0.1, rel_tol=1e-9)
    assert np.allclose(T, T.T)


def test_sample_covariance_is_centred_and_divided_by_m():
    rng = np.random.default_rng(1)
    T = inputs.theta_chain(5)
    S = inputs.sample_covariance(T, 4000, rng)
    assert np.allclose(S, S.T)
    # converges to the true covariance
    assert np.max(np.abs(S - np.linalg.inv(T))) < 0.15
    # rank m - 1 when m <= n (centred samples)
    S_small = inputs.sample_covariance(inputs.theta_chain(20), 6, np.random.default_rng(2))
    assert np.linalg.matrix_rank(S_small) == 5


def test_served_stream_rate_and_ranges():
    arrivals, ids, lams, pool = inputs.served_stream(count=20000, rate_hz=200.0)
    assert np.all(np.diff(arrivals) > 0)
    assert abs(len(arrivals) / arrivals[-1] - 200.0) < 5.0
    assert lams.min() >= 0.05 and lams.max() <= 0.3
    ns = np.array([d["n"] for d in pool])
    assert ns.min() >= 64 and ns.max() <= 4096 and len(pool) == 256
    assert {d["structure"] for d in pool} == {"chain", "grid"}


def test_batch_problems_sizes_and_path():
    probs = inputs.batch_path_problems(count=40, seed=3)
    ns = np.array([p["n"] for p in probs])
    assert ns.min() >= 32 and ns.max() <= 1024
    lams = probs[0]["lambdas"]
    assert len(lams) == 8 and math.isclose(lams[0], 0.5) and math.isclose(lams[-1], 0.02)
    assert all(a > b for a, b in zip(lams, lams[1:]))
    assert probs[0]["S"].dtype == np.float32
