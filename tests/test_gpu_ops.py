"""Kernel-level parity: each single-step entry point of the C ABI against the FP64 oracle's
step on the same seeded inputs, at sizes that span one tile, several tiles and ragged tails."""
import numpy as np
import pytest

from oracle import pista

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [1, 2, 7, 64, 100, 129, 257, 700]


def _iterate_like(n, seed, density=0.05):
    """A symmetric positive-definite matrix with the sparsity of a pISTA iterate, and an S."""
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    if n > 1:
        mask = np.triu(rng.random((n, n)) < density, 1)
        vals = rng.uniform(-0.3, 0.3, (n, n)) * mask
        A = vals + vals.T
    A += np.diag(np.abs(A).sum(axis=1) + rng.uniform(0.2, 1.5, n))
    Y = rng.standard_normal((n, max(2, n // 2)))
    Y -= Y.mean(axis=1, keepdims=True)
    S = Y @ Y.T / Y.shape[1]
    return A, 0.5 * (S + S.T)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("n", SIZES)
def test_cholesky_logdet_pd(fp64, n):
    A, _ = _iterate_like(n, n)
    L, pd, ld = fp64.op_cholesky(_dev(A))
    Lref = np.linalg.cholesky(A)
    assert pd
    assert np.max(np.abs(_host(L) - Lref)) <= 1e-13 * np.max(np.abs(Lref)) * max(1, n) ** 0.5
    ok, ldref = pista.logdet(A)
    assert abs(ld - ldref) <= 1e-13 * max(1.0, abs(ldref)) * max(1, n) ** 0.5
    # an indefinite matrix is reported as not PD
    _, pd_bad, _ = fp64.op_cholesky(_dev(A - (np.max(np.linalg.eigvalsh(A)) * 0.5 + 1.0) * np.eye(n)))
    if n > 1:
        assert not pd_bad


@pytest.mark.parametrize("n", SIZES)
def test_inverse(fp64, n):
    A, _ = _iterate_like(n, 100 + n)
    W = _host(fp64.op_inverse(_dev(A)))
    Wref = pista.inverse(A)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(W - Wref) <= 1e-14 * cond * np.linalg.norm(Wref) * max(1, n) ** 0.5
    assert np.array_equal(W, W.T)


@pytest.mark.parametrize("n", SIZES)
def test_gradient_mask_sign_code(fp64, n):
    A, S = _iterate_like(n, 200 + n)
    lam = 0.05
    W = pista.inverse(A)
    X, code, sums = fp64.op_gradient(_dev(S), _dev(A), _dev(W), lam)
    ref = pista.step_gradient(S, A, W, lam)
    assert np.array_equal(_host(code), ref["code"])            # integer: bit-exact
    assert np.max(np.abs(_host(X) - ref["X"])) <= 1e-15 * (np.max(np.abs(ref["X"])) + 1e-300) * 4
    z_l1 = np.sum(np.abs(ref["X"]))
    assert sums[0] == pytest.approx(z_l1, rel=1e-12, abs=1e-300)
    assert sums[1] == pytest.approx(ref["a_l1"], rel=1e-12)
    assert sums[2] == pytest.approx(ref["z_fro"] ** 2, rel=1e-12, abs=1e-300)
    assert sums[3] == ref["nnz"]


@pytest.mark.parametrize("n", SIZES)
def test_sandwich(fp64, n):
    A, S = _iterate_like(n, 300 + n)
    X = pista.step_gradient(S, A, pista.inverse(A), 0.02)["X"]
    Y = _host(fp64.op_sandwich(_dev(A), _dev(X)))
    Yref = pista.step_sandwich(A, X)
    scale = np.linalg.norm(A) ** 2 * np.linalg.norm(X) + 1e-300
    assert np.linalg.norm(Y - Yref) <= 1e-14 * scale * max(1, n) ** 0.5
    assert np.array_equal(Y, Y.T)


@pytest.fixture(scope="module")
def fp64_dense(glasso):
    """An FP64 handle that forms the sandwich with dense products."""
    h = glasso.Handle(precision="fp64", products="dense")
    yield h
    h.close()


@pytest.mark.parametrize("n", SIZES)
def test_sandwich_dense_and_sparse_forms(fp64, fp64_dense, n):
    """The FP64 handle forms Theta X Theta from the CSR of Theta (auto); the dense form must give
    the same product to FP64 rounding, and both the oracle's."""
    A, S = _iterate_like(n, 350 + n)
    X = pista.step_gradient(S, A, pista.inverse(A), 0.02)["X"]
    Ys = _host(fp64.op_sandwich(_dev(A), _dev(X)))
    Yd = _host(fp64_dense.op_sandwich(_dev(A), _dev(X)))
    Yref = pista.step_sandwich(A, X)
    scale = np.linalg.norm(A) ** 2 * np.linalg.norm(X) + 1e-300
    for Y in (Ys, Yd):
        assert np.linalg.norm(Y - Yref) <= 1e-14 * scale * max(1, n) ** 0.5


@pytest.mark.parametrize("n", [64, 257])
def test_sparse_sandwich_is_exact_on_a_diagonal_theta(fp64, n):
    """Theta diagonal: the sparse form makes one rounded product per entry and step,
    Y_ij = fl(a_i fl(a_j X_ij)) on the lower triangle (mirrored), bit for bit."""
    rng = np.random.default_rng(n)
    a = rng.uniform(0.5, 2.0, n)
    X = rng.standard_normal((n, n))
    X = X + X.T
    Y = _host(fp64.op_sandwich(_dev(np.diag(a)), _dev(X)))
    E = a[:, None] * (a[None, :] * X)
    E = np.tril(E) + np.tril(E, -1).T
    assert np.array_equal(Y, E)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("t", [1.0, 0.25])
def test_trial_point(fp64, n, t):
    A, S = _iterate_like(n, 400 + n)
    lam = 0.05
    W = pista.inverse(A)
    g = pista.gradient(S, W)
    M = pista.free_set_mask(A, g, lam)
    G = pista.sign_guess(A, g)
    X = (g + lam * G) * M
    Y = pista.step_sandwich(A, X)
    code = (G * M).astype(np.int8)
    At = _host(fp64.op_trial(_dev(A), _dev(Y), _dev(code), lam, t))
    C = pista.coupling_C(A, lam)
    ref = pista.trial(A, Y - C * code, C, M, t)
    assert np.array_equal(At != 0.0, ref != 0.0)
    assert np.max(np.abs(At - ref)) <= 1e-14 * np.max(np.abs(ref))
    assert np.array_equal(At, At.T)
