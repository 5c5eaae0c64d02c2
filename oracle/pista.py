"""pISTA (Algorithm 1, Sec. 4.4) restated step by step in plain numpy FP64.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs, never by the product package.  It shares no code with the
CUDA path.

Problem (Sec. 3.1, eq. sparse_obj):
    min_{A > 0}  F(A) = -log det A + tr(S A) + lam * ||A||_1,   ||A||_1 = sum_ij |A_ij|.

Readings of the paper taken here (the paper is silent or ambiguous on these):
  R1  ||A||_1 sums all n*n entries, the diagonal included (eq. sparse_obj).
  R2  The accepted update is masked, A_next = A + M (.) D (Sec. 4.1, eq. proximal_gen_free
      and conditions t_cond_pd / t_cond_min); Algorithm 1's unmasked "A + D" is read the same.
  R3  eq. d_sol is elementwise: D_ij = -A_ij + ST(A_ij - t B_ij, t C_ij)  (App. A.2).
  R4  Backtracking divides t by 2, and t restarts at 1 every outer iteration (Sec. 4.3.2).
  R5  Below t_min = 1e-4 the step is t_f = (0.9 / cond_2(A))^2 (Sec. 6, experimental setup);
      it is accepted when A_t is PD and passes the decrease test of R6, otherwise the solve
      stops with status "stall".
  R6  The decrease test of eq. t_cond_min, F(A_t) < F(A), is decided on the difference
      dF = F(A_t) - F(A) = -[log det A_t - log det A] + <S, dA> + lam sum(|A_t| - |A|),
      dA = A_t - A, with the linear terms summed entry by entry.  The log-det difference is
      first taken from the two Cholesky factors.  When that dF lies within 1000 delta of 0,
      delta = 16 u (|log det A| + |tr(SA)| + lam ||A||_1), u = 2^-53, rounding could decide
      the sign, so dF is re-evaluated with log det A_t - log det A = sum_i log1p(mu_i),
      mu the eigenvalues of E = L^{-1} dA L^{-T} (A = L L^T), which is accurate relative to
      dF itself.  Accept iff dF < 0.  Without this, FP64 pISTA stalls near r ~ 1e-7 on
      ill-conditioned problems, where the true decrease falls below the resolution of F.
  R7  Stop rule (Sec. 6): ||Z||_1 <= tol * ||A||_1 with Z the minimum-norm sub-gradient of F;
      it is checked before a direction is formed, so A0 itself may already satisfy it.
  R8  sign(0) = 0.   R9  The free set uses the strict test |g_ij| > lam (eq. free_set).
  R10 W and B are symmetrised by mirroring their lower triangle, so every iterate is
      exactly symmetric.
  R11 "A_ij != 0" is an exact comparison with 0.0 (soft-thresholding makes exact zeros).
  R12 eq. c with A_ji = A_ij: C_ii = lam A_ii^2, C_ij = lam (A_ii A_jj + A_ij^2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

T_MIN = 1e-4          # Sec. 6: the line search stops halving below this t
FALLBACK_FACTOR = 0.9  # Sec. 6: t <= (0.9 / cond(A))^2


# ----------------------------------------------------------------------------------------
# elementary pieces
# ----------------------------------------------------------------------------------------
def soft_threshold(v, c):
    """SoftThreshold(v, c) = sign(v) * max(|v| - c, 0)  (App. A.1, Lemma A.1)."""
    return np.sign(v) * np.maximum(np.abs(v) - c, 0.0)


def mirror_lower(M):
    """Symmetric matrix whose lower triangle is M's (reading R10)."""
    low = np.tril(M)
    return low + np.tril(M, -1).T


def cholesky(A):
    """Lower Cholesky factor of A, or None when A is not positive definite."""
    if not np.all(np.isfinite(A)):
        return None
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(L)) or np.any(np.diag(L) <= 0.0):
        return None
    return L


def logdet(A):
    """(is_pd, log det A) from the Cholesky factor: log det A = 2 sum_i log L_ii."""
    L = cholesky(A)
    if L is None:
        return False, np.nan
    return True, 2.0 * float(np.sum(np.log(np.diag(L))))


def objective(S, A, lam):
    """F(A) of eq. sparse_obj; +inf when A is not positive definite."""
    pd, ld = logdet(A)
    if not pd:
        return np.inf
    return -ld + float(np.sum(S * A)) + lam * float(np.sum(np.abs(A)))


UNIT_ROUNDOFF = 2.0 ** -53


def decrease_slack(S, A, lam):
    """delta of reading R6: the rounding allowance of the decrease test at the point A."""
    pd, ld = logdet(A)
    scale = abs(ld) + abs(float(np.sum(S * A))) + lam * float(np.sum(np.abs(A)))
    return 16.0 * UNIT_ROUNDOFF * scale


DIFF_BAND = 1000.0


def objective_difference(S, A, L, At, lam, delta):
    """(dF, tier): F(At) - F(A) as in reading R6, +inf when At is not PD.
    L is the Cholesky factor of A; tier is 1 (Cholesky log-dets) or 2 (eigenvalues of E)."""
    Lt = cholesky(At)
    if Lt is None:
        return np.inf, 1
    dA = At - A
    lin = float(np.sum(S * dA)) + lam * float(np.sum(np.abs(At) - np.abs(A)))
    dld = 2.0 * float(np.sum(np.log(np.diag(Lt)))) - 2.0 * float(np.sum(np.log(np.diag(L))))
    dF = -dld + lin
    if abs(dF) > DIFF_BAND * delta:
        return dF, 1
    X = scipy.linalg.solve_triangular(L, dA, lower=True)          # L^{-1} dA
    E = scipy.linalg.solve_triangular(L, X.T, lower=True)         # L^{-1} dA L^{-T}
    mu = np.linalg.eigvalsh(0.5 * (E + E.T))
    return -float(np.sum(np.log1p(mu))) + lin, 2


def inverse(A):
    """W = A^{-1} from the Cholesky factor, W = L^{-T} L^{-1}, mirrored (R10)."""
    L = cholesky(A)
    if L is None:
        raise np.linalg.LinAlgError("inverse of a matrix that is not positive definite")
    n = A.shape[0]
    Linv = scipy.linalg.solve_triangular(L, np.eye(n), lower=True)
    return mirror_lower(Linv.T @ Linv)


def gradient(S, W):
    """g = grad f(A) = S - A^{-1}  (eq. grad_hessian)."""
    return S - W


def free_set_mask(A, g, lam):
    """M_ij = 1 on the free set {A_ij != 0} U {|g_ij| > lam}  (eqs. free_set, M)."""
    return (A != 0.0) | (np.abs(g) > lam)


def sign_guess(A, g):
    """G_ij = sign(A_ij) where A_ij != 0, else -sign(g_ij)  (eq. G+)."""
    return np.where(A != 0.0, np.sign(A), -np.sign(g))


def min_norm_subgradient(A, g, lam):
    """Minimum-norm element Z of dF(A) (Sec. 5.1): entrywise
    g + lam sign(A) where A != 0, and the point of [g - lam, g + lam] nearest 0 where A = 0."""
    return np.where(A != 0.0, g + lam * np.sign(A), soft_threshold(g, lam))


def kkt_residual(A, g, lam):
    """(r, ||Z||_F): r = ||Z||_1 / ||A||_1 is the stop quantity of Sec. 6 (R7)."""
    Z = min_norm_subgradient(A, g, lam)
    return float(np.sum(np.abs(Z)) / np.sum(np.abs(A))), float(np.sqrt(np.sum(Z * Z)))


def coupling_C(A, lam):
    """C of eq. c (R12)."""
    d = np.diag(A)
    C = lam * (np.outer(d, d) + A * A)
    np.fill_diagonal(C, lam * d * d)
    return C


def direction_B(A, g, M, G, lam):
    """B of eq. b, as printed: A(g.M)A + lam A(G.M)A - C.(G.M); lower triangle mirrored."""
    GM = G * M
    B = A @ (g * M) @ A + lam * (A @ GM @ A) - coupling_C(A, lam) * GM
    return mirror_lower(B)


def trial(A, B, C, M, t):
    """A + M.D with D = -A + ST(A - tB, tC)  (eq. d_sol, R2, R3)."""
    D = -A + soft_threshold(A - t * B, t * C)
    return A + np.where(M, D, 0.0)


def initial_point(S, lam):
    """A0_ii = 1/(S_ii + lam), A0_ij = 0 (the G-ISTA start of Sec. 6)."""
    return np.diag(1.0 / (np.diag(S) + lam))


def cond2(A):
    """Spectral condition number lambda_max / lambda_min of a symmetric PD matrix."""
    ev = np.linalg.eigvalsh(A)
    return float(ev[-1] / ev[0])


def fallback_step(A):
    """t_f = (0.9 / cond_2(A))^2: the step of Sec. 6 once halving has gone below t_min
    (reading R5).  Lemma 4.1 bounds an acceptable step by (beta / gamma)^2 with beta, gamma
    bounds of the eigenvalues; Sec. 6 takes the current iterate's own, with the factor 0.9."""
    return (FALLBACK_FACTOR / cond2(A)) ** 2


# ----------------------------------------------------------------------------------------
# step functions (what one GPU kernel computes, for kernel-level parity)
# ----------------------------------------------------------------------------------------
def step_gradient(S, A, W, lam):
    """Everything the stop test and the direction need from (S, A, W):
    X = (g + lam G).M (this equals Z), code = G.M in {-1,0,1}, r, ||Z||_F, nnz(A), ||A||_1."""
    g = gradient(S, W)
    M = free_set_mask(A, g, lam)
    G = sign_guess(A, g)
    X = (g + lam * G) * M
    code = (G * M).astype(np.int8)
    r, zf = kkt_residual(A, g, lam)
    return dict(X=X, code=code, r=r, z_fro=zf, nnz=int(np.count_nonzero(A)),
                a_l1=float(np.sum(np.abs(A))))


def step_sandwich(A, X):
    """Y = A X A (both factors symmetric), lower triangle mirrored."""
    return mirror_lower(A @ X @ A)


# ----------------------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------------------
def pista(S, lam, tol, A0=None, max_iter=500, shrink=0.5, t_min=T_MIN, trace=False,
          fallback=None, trace_iterates=False):
    """pISTA(S, lam, A0) of Algorithm 1 with the readings R1-R12.

    fallback: optional callable (k, A) -> t replacing fallback_step(A) at outer iteration k
    (a test replays with it the step sizes another implementation took).
    trace_iterates: each trace record also keeps the iterate ("theta") and the last trial
    point ("trial") of its iteration.

    Returns a dict: theta, F, r (relative l1 KKT residual), z_fro, nnz, iterations,
    trials (line-search trials in total), status in {"converged", "max_iter", "stall"},
    and, if requested, a per-iteration trace.
    """
    S = np.asarray(S, dtype=np.float64)
    A = initial_point(S, lam) if A0 is None else np.array(A0, dtype=np.float64)
    F = objective(S, A, lam)
    if not np.isfinite(F):
        raise ValueError("the start point is not positive definite")
    hist = []
    total_trials = 0
    status = "max_iter"
    k = 0
    r = zf = np.nan
    while True:
        L = cholesky(A)
        W = inverse(A)
        g = gradient(S, W)
        r, zf = kkt_residual(A, g, lam)
        if r <= tol:
            status = "converged"
            break
        if k >= max_iter:
            status = "max_iter"
            break
        M = free_set_mask(A, g, lam)
        G = sign_guess(A, g)
        B = direction_B(A, g, M, G, lam)
        C = coupling_C(A, lam)
        delta = decrease_slack(S, A, lam)
        t = 1.0
        trials = 0
        accepted = False
        dF, tier = np.inf, 1
        while t >= t_min:
            At = trial(A, B, C, M, t)
            dF, tier = objective_difference(S, A, L, At, lam, delta)
            trials += 1
            if dF < 0.0:
                accepted = True
                break
            t *= shrink
        if not accepted:
            t = fallback_step(A) if fallback is None else float(fallback(k, A))
            At = trial(A, B, C, M, t)
            dF, tier = objective_difference(S, A, L, At, lam, delta)
            trials += 1
            accepted = bool(dF < 0.0)
        total_trials += trials
        if trace:
            hist.append(dict(k=k, F=F, r=r, z_fro=zf, nnz=int(np.count_nonzero(A)), t=t,
                             trials=trials, accepted=accepted, dF=dF, tier=tier,
                             delta=delta))
            if trace_iterates:
                hist[-1].update(theta=A, trial=At)
        if not accepted:
            status = "stall"
            break
        A = At
        F = objective(S, A, lam)
        k += 1
    out = dict(theta=A, F=F, r=r, z_fro=zf, nnz=int(np.count_nonzero(A)), iterations=k,
               trials=total_trials, status=status)
    if trace:
        out["trace"] = hist
    return out
