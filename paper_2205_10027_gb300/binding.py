"""ctypes binding of libglasso (include/glasso.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Importing this module loads the
in-tree ``libglasso.so`` and raises ImportError when it has not been built (there is no
CPU fallback).  Low-level functions keep the C names (``glasso_solve`` ...); ``Handle``
wraps them for numpy arrays (host memory) and torch CUDA tensors (device memory).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libglasso.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
lib = C.CDLL(LIB_PATH)

# ---- status, enums --------------------------------------------------------------------------
STATUS = {0: "GLASSO_OK", 1: "GLASSO_ERR_ARG", 2: "GLASSO_ERR_NOT_SYMMETRIC", 3: "GLASSO_ERR_NONFINITE",
          4: "GLASSO_ERR_NOT_PD", 5: "GLASSO_ERR_OOM", 6: "GLASSO_ERR_BUDGET", 7: "GLASSO_ERR_CUDA",
          8: "GLASSO_ERR_TIMEOUT", 9: "GLASSO_MAX_ITER", 10: "GLASSO_LINESEARCH_STALL",
          11: "GLASSO_PENDING", 12: "GLASSO_ERR_UNSUPPORTED"}
OK, PENDING, MAX_ITER, STALL = 0, 11, 9, 10
PRECISION = {"fp64": 0, "tf32x3": 1, "bf16x3": 2}
F64, F32 = 0, 1
HOST, DEVICE = 0, 1


class glasso_config(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("precision", C.c_int),
                ("max_iter", C.c_int), ("shrink", C.c_double), ("t_min", C.c_double),
                ("hbm_budget_bytes", C.c_size_t), ("serve_slots", C.c_int), ("products", C.c_int),
                ("method", C.c_int), ("standardize", C.c_int), ("fp32_panels", C.c_int),
                ("autotune", C.c_int)]


class glasso_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("trials", C.c_int32),
                ("nnz", C.c_int32), ("rel_kkt_l1", C.c_double), ("min_subgrad_fro", C.c_double),
                ("objective", C.c_double), ("logdet", C.c_double), ("seconds", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("kernel_launches", C.c_int64), ("step_t", C.c_double), ("step_dF", C.c_double),
                ("step_tier", C.c_int32), ("step_fallback", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PROF_CLASSES = ("sandwich", "trailing", "panel", "inverse", "refine", "gradient", "trial", "factor",
                "residual", "logdet2", "aux", "spmm")


class glasso_profile(C.Structure):
    _fields_ = [("ms", C.c_double * len(PROF_CLASSES)), ("work", C.c_double * len(PROF_CLASSES)),
                ("launches", C.c_int64 * len(PROF_CLASSES))]

    def as_dict(self):
        return {name: dict(ms=self.ms[i], work=self.work[i], launches=self.launches[i])
                for i, name in enumerate(PROF_CLASSES) if self.launches[i]}


class glasso_problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("S", C.c_void_p), ("dtype", C.c_int), ("n_lambda", C.c_int32),
                ("lambdas", C.POINTER(C.c_double)), ("tol", C.c_double),
                ("theta_out", C.POINTER(C.c_double))]


class glasso_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("S", C.c_void_p), ("dtype", C.c_int), ("lambda_", C.c_double),
                ("tol", C.c_double), ("dataset_id", C.c_int64)]


_h = C.c_void_p
_dp = C.c_void_p  # device or host pointer
_sig = {
    "glasso_config_default": (C.c_int, [C.POINTER(glasso_config)]),
    "glasso_create": (C.c_int, [C.POINTER(glasso_config), C.POINTER(C.c_void_p)]),
    "glasso_destroy": (C.c_int, [_h]),
    "glasso_last_error": (C.c_char_p, [_h]),
    "glasso_status_string": (C.c_char_p, [C.c_int]),
    "glasso_solve": (C.c_int, [_h, _dp, C.c_int, C.c_int, C.c_int64, C.c_double, C.c_double, _dp, _dp,
                               C.POINTER(glasso_result)]),
    "glasso_begin": (C.c_int, [_h, _dp, C.c_int, C.c_int, C.c_int64, C.c_double, _dp]),
    "glasso_step": (C.c_int, [_h, C.c_double, C.POINTER(glasso_result)]),
    "glasso_end": (C.c_int, [_h, _dp, C.POINTER(glasso_result)]),
    "glasso_profile_start": (C.c_int, [_h]),
    "glasso_profile_stop": (C.c_int, [_h, C.POINTER(glasso_profile)]),
    "glasso_probe_fp64_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "glasso_gradient_noalloc": (C.c_int, [_dp, _dp, _dp, C.c_int64, C.c_double, _dp, _dp, _dp, _dp]),
    "glasso_workspace_bytes": (C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    "glasso_solve_batch": (C.c_int, [_h, C.POINTER(glasso_problem), C.c_int32, C.POINTER(glasso_result)]),
    "glasso_submit": (C.c_int, [_h, C.POINTER(glasso_request), C.POINTER(C.c_uint64)]),
    "glasso_poll": (C.c_int, [_h, C.c_uint64, C.POINTER(glasso_result), _dp]),
    "glasso_op_cholesky": (C.c_int, [_h, _dp, C.c_int64, _dp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "glasso_op_inverse": (C.c_int, [_h, _dp, C.c_int64, _dp]),
    "glasso_op_gradient": (C.c_int, [_h, _dp, _dp, _dp, C.c_int64, C.c_double, _dp, _dp,
                                     C.POINTER(C.c_double)]),
    "glasso_op_sandwich": (C.c_int, [_h, _dp, _dp, C.c_int64, _dp]),
    "glasso_op_trial": (C.c_int, [_h, _dp, _dp, _dp, C.c_int64, C.c_double, C.c_double, _dp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype, _f.argtypes = _res, _args
    globals()[_name] = _f

EXPORTED = tuple(_sig)
NOALLOC_MAX_N = 16384  # GLASSO_NOALLOC_MAX_N


class GlassoError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    """Data pointer of a numpy array (host) or a torch tensor (its device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def probe_fp64_peak(device=0):
    """Measured FP64 FMA peak of the device, TFLOP/s."""
    v = C.c_double()
    st = glasso_probe_fp64_peak(device, C.byref(v))
    if st != OK:
        raise GlassoError(st, "glasso_probe_fp64_peak failed")
    return v.value


def workspace_bytes(n):
    """Device memory one solve of size n holds (glasso_workspace_bytes)."""
    v = C.c_size_t()
    st = glasso_workspace_bytes(n, C.byref(v))
    if st != OK:
        raise GlassoError(st, "glasso_workspace_bytes failed")
    return v.value


PRODUCTS = {"auto": 0, "dense": 1, "sparse": 2}
METHODS = {"pista": 0, "gista": 1}


class Handle:
    """A library handle.  precision: 'fp64', 'tf32x3' or 'bf16x3'; products: how the sandwich
    products are formed, 'auto', 'dense' or 'sparse' (glasso_products); method: 'pista'
    (Algorithm 1) or 'gista' (plain proximal gradient, glasso_method); standardize: solve on the
    correlation matrix of S (glasso_config.standardize); fp32_panels: factor the Cholesky panels
    of the split-precision forms in FP32 instead of FP64 (glasso_config.fp32_panels); autotune:
    measure the product kernels per shape (glasso_config.autotune)."""

    def __init__(self, precision="fp64", device=0, stream=None, max_iter=500, shrink=0.5, t_min=1e-4,
                 hbm_budget_bytes=0, serve_slots=8, products="auto", method="pista", standardize=False,
                 fp32_panels=False, autotune=True):
        cfg = glasso_config()
        glasso_config_default(C.byref(cfg))
        cfg.device = device
        cfg.stream = stream
        cfg.precision = PRECISION[precision]
        cfg.max_iter = max_iter
        cfg.shrink = shrink
        cfg.t_min = t_min
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.serve_slots = serve_slots
        cfg.products = PRODUCTS[products]
        cfg.method = METHODS[method]
        cfg.standardize = 1 if standardize else 0
        cfg.fp32_panels = 1 if fp32_panels else 0
        cfg.autotune = 1 if autotune else 0
        h = C.c_void_p()
        st = glasso_create(C.byref(cfg), C.byref(h))
        if st != OK:
            raise GlassoError(st, "glasso_create failed")
        self.h = h
        self.precision = precision

    def close(self):
        if self.h:
            glasso_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise GlassoError(st, glasso_last_error(self.h).decode())
        return st

    # ---- solve ---------------------------------------------------------------------------
    def solve(self, S, lam, tol, theta0=None, out=None, allow=(OK, MAX_ITER, STALL)):
        """Solve for a numpy S (host memory) or a torch CUDA tensor S (device memory).
        Returns (theta, result dict)."""
        res = glasso_result()
        if isinstance(S, np.ndarray):
            S = np.ascontiguousarray(S)
            if S.dtype not in (np.float32, np.float64):
                S = S.astype(np.float64)
            n = S.shape[0]
            out = np.empty((n, n), np.float64) if out is None else out
            t0 = None if theta0 is None else np.ascontiguousarray(theta0, dtype=np.float64)
            st = glasso_solve(self.h, _ptr(S), F32 if S.dtype == np.float32 else F64, HOST, n, lam, tol,
                              _ptr(t0), _ptr(out), C.byref(res))
        else:
            import torch
            n = S.shape[0]
            out = torch.empty((n, n), dtype=torch.float64, device=S.device) if out is None else out
            st = glasso_solve(self.h, _ptr(S), F32 if S.dtype == torch.float32 else F64, DEVICE, n, lam,
                              tol, _ptr(theta0), _ptr(out), C.byref(res))
        self._check(st, allow)
        return out, res.as_dict()

    # ---- step-wise solve -------------------------------------------------------------------
    def begin(self, S, lam, theta0=None):
        if isinstance(S, np.ndarray):
            S = np.ascontiguousarray(S)
            self._keep = S
            st = glasso_begin(self.h, _ptr(S), F32 if S.dtype == np.float32 else F64, HOST, S.shape[0], lam,
                              _ptr(None if theta0 is None else np.ascontiguousarray(theta0, np.float64)))
        else:
            import torch
            st = glasso_begin(self.h, _ptr(S), F32 if S.dtype == torch.float32 else F64, DEVICE, S.shape[0],
                              lam, _ptr(theta0))
        self._check(st)

    def step(self, tol=0.0):
        """One outer iteration; returns (status, result dict).  status PENDING = step taken."""
        res = glasso_result()
        st = glasso_step(self.h, tol, C.byref(res))
        self._check(st, (OK, PENDING, STALL))
        return st, res.as_dict()

    def end(self, out=None):
        res = glasso_result()
        self._check(glasso_end(self.h, _ptr(out), C.byref(res)))
        return out, res.as_dict()

    def profile_start(self):
        self._check(glasso_profile_start(self.h))

    def profile_stop(self):
        p = glasso_profile()
        self._check(glasso_profile_stop(self.h, C.byref(p)))
        return p.as_dict()

    def solve_batch(self, problems):
        """problems: list of dict(S=np.ndarray (f32/f64), lambdas=[...], tol=...).
        Returns (list of per-problem arrays [n_lambda, n, n], list of lists of result dicts)."""
        keep = []
        arr = (glasso_problem * len(problems))()
        outs = []
        for i, p in enumerate(problems):
            S = np.ascontiguousarray(p["S"])
            lams = np.ascontiguousarray(p["lambdas"], dtype=np.float64)
            out = np.empty((len(lams), S.shape[0], S.shape[0]), np.float64)
            keep += [S, lams, out]
            outs.append(out)
            arr[i].n = S.shape[0]
            arr[i].S = _ptr(S)
            arr[i].dtype = F32 if S.dtype == np.float32 else F64
            arr[i].n_lambda = len(lams)
            arr[i].lambdas = lams.ctypes.data_as(C.POINTER(C.c_double))
            arr[i].tol = p["tol"]
            arr[i].theta_out = out.ctypes.data_as(C.POINTER(C.c_double))
        total = sum(len(p["lambdas"]) for p in problems)
        res = (glasso_result * max(total, 1))()
        self._check(glasso_solve_batch(self.h, arr, len(problems), res))
        results, k = [], 0
        for p in problems:
            results.append([res[k + j].as_dict() for j in range(len(p["lambdas"]))])
            k += len(p["lambdas"])
        return outs, results

    # ---- serving ---------------------------------------------------------------------------
    def submit(self, S, lam, tol, dataset_id=-1):
        S = np.ascontiguousarray(S)
        if S.dtype not in (np.float32, np.float64):
            S = S.astype(np.float64)
        req = glasso_request(S.shape[0], _ptr(S), F32 if S.dtype == np.float32 else F64, lam, tol, dataset_id)
        ticket = C.c_uint64()
        self._check(glasso_submit(self.h, C.byref(req), C.byref(ticket)))
        return ticket.value

    def poll(self, ticket, n=None):
        """(status, result dict or None, theta or None); theta only if n is given."""
        res = glasso_result()
        out = None if n is None else np.empty((n, n), np.float64)
        st = glasso_poll(self.h, ticket, C.byref(res), _ptr(out))
        if st == PENDING:
            return st, None, None
        self._check(st, (OK, MAX_ITER, STALL))
        return st, res.as_dict(), out

    # ---- single steps on torch CUDA tensors (float64, n x n, contiguous) -----------------------
    def op_cholesky(self, A):
        import torch
        n = A.shape[0]
        L = torch.empty_like(A)
        pd, ld = C.c_int32(), C.c_double()
        self._check(glasso_op_cholesky(self.h, _ptr(A), n, _ptr(L), C.byref(pd), C.byref(ld)))
        return L, bool(pd.value), ld.value

    def op_inverse(self, A):
        W = A.new_empty(A.shape)
        self._check(glasso_op_inverse(self.h, _ptr(A), A.shape[0], _ptr(W)))
        return W

    def op_gradient(self, S, A, W, lam):
        import torch
        n = A.shape[0]
        X = torch.empty_like(A)
        code = torch.empty((n, n), dtype=torch.int8, device=A.device)
        sums = (C.c_double * 4)()
        self._check(glasso_op_gradient(self.h, _ptr(S), _ptr(A), _ptr(W), n, lam, _ptr(X), _ptr(code), sums))
        return X, code, list(sums)

    def op_sandwich(self, A, X):
        Y = A.new_empty(A.shape)
        self._check(glasso_op_sandwich(self.h, _ptr(A), _ptr(X), A.shape[0], _ptr(Y)))
        return Y

    def op_trial(self, A, Y, code, lam, t):
        At = A.new_empty(A.shape)
        self._check(glasso_op_trial(self.h, _ptr(A), _ptr(Y), _ptr(code), A.shape[0], lam, t, _ptr(At)))
        return At
