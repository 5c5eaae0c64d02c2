"""The allocation-free gradient entry point, for callers that cannot allocate device memory
(a framework that owns every device allocation, a runtime that forbids cudaMalloc on its hot
path, an embedding with a fixed memory budget).  It is called through the C ABI on the
caller's own device buffers and must agree with glasso_op_gradient, the entry point that
stages through a handle's workspace, on two calls in a row (the shared scratch keeps the
previous call's contents).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from oracle import pista

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, seed):
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < 0.05, 1)
    vals = rng.uniform(-0.3, 0.3, (n, n)) * mask
    A = vals + vals.T
    A += np.diag(np.abs(A).sum(axis=1) + rng.uniform(0.2, 1.5, n))
    Y = rng.standard_normal((n, max(2, n // 2)))
    Y -= Y.mean(axis=1, keepdims=True)
    S = Y @ Y.T / Y.shape[1]
    S = 0.5 * (S + S.T)
    return S, A, pista.inverse(A)


def _device_problem(n, seed):
    """A large (S, A, W) triple generated on the device; the gradient pass needs no relation
    between A and W, only their shapes and values."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    S = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g) * 0.1
    S = 0.5 * (S + S.T)
    A = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    A = A * (torch.rand((n, n), device="cuda", generator=g) < 0.01)
    A = 0.5 * (A + A.T) + torch.eye(n, dtype=torch.float64, device="cuda")
    W = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g) * 0.1
    return [S.contiguous(), A.contiguous(), (0.5 * (W + W.T)).contiguous()]


def test_noalloc_matches_op_gradient_on_two_calls(glasso):
    lam = 0.05
    cases = [_problem(257, 1), _problem(100, 2)]   # second call smaller: stale scratch rows
    dev = [[torch.from_numpy(m).cuda() for m in c] for c in cases]
    dev.append(_device_problem(glasso.NOALLOC_MAX_N, 3))   # third call: the largest n allowed
    outs = []
    for (S, A, W) in dev:
        n = S.shape[0]
        outs.append((torch.empty((n, n), dtype=torch.float64, device="cuda"),
                     torch.empty((n, n), dtype=torch.int8, device="cuda"),
                     torch.empty(4, dtype=torch.float64, device="cuda")))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    free, held = [], []
    for (S, A, W), (X, code, sums) in zip(dev, outs):
        n = S.shape[0]
        st = glasso.glasso_gradient_noalloc(S.data_ptr(), A.data_ptr(), W.data_ptr(), n, lam,
                                            X.data_ptr(), code.data_ptr(), sums.data_ptr(), stream)
        assert st == 0
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        held.append(torch.cuda.memory_allocated())
    # nothing allocated through torch by any call, and no device memory taken by the calls
    # after the first (the first may load the library's module, which holds the scratch array)
    assert held[0] == held[1] == held[2]
    assert free[0] == free[1] == free[2]
    with glasso.Handle(precision="fp64") as h:
        for (S, A, W), (X, code, sums) in zip(dev, outs):
            Xr, coder, sumsr = h.op_gradient(S, A, W, lam)
            assert torch.equal(X, Xr)                    # same per-entry arithmetic
            assert torch.equal(code, coder)
            np.testing.assert_allclose(sums.cpu().numpy(), np.array(sumsr), rtol=1e-12, atol=0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch(glasso):
    big = glasso.NOALLOC_MAX_N + 1
    st = glasso.glasso_gradient_noalloc(C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), big, 0.1,
                                        C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), None)
    assert st == 6   # GLASSO_ERR_BUDGET, before any device work
    assert glasso.glasso_gradient_noalloc(None, None, None, 10, 0.1, None, None, None, None) == 1
