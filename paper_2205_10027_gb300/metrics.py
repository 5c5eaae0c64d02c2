"""Evaluation of an estimate against a known precision matrix (host side; no solver arithmetic).

support_mcc: the Matthews correlation coefficient of the estimated sparsity pattern, the
quality measure of the paper's sample-ratio study (Sec. 6.3, eq. MCC).  The paper does not
say which entries are counted; here every unordered off-diagonal pair (i < j) counts once,
since both matrices are symmetric and their diagonals are always nonzero.
"""
from __future__ import annotations

import math

import numpy as np


def support_counts(theta_true: np.ndarray, theta_hat: np.ndarray) -> tuple[int, int, int, int]:
    """(TP, TN, FP, FN) of the pattern theta_hat != 0 against theta_true != 0, pairs i < j."""
    iu = np.triu_indices(theta_true.shape[0], 1)
    t = np.asarray(theta_true)[iu] != 0.0
    h = np.asarray(theta_hat)[iu] != 0.0
    tp = int(np.sum(t & h))
    tn = int(np.sum(~t & ~h))
    fp = int(np.sum(~t & h))
    fn = int(np.sum(t & ~h))
    return tp, tn, fp, fn


def support_mcc(theta_true: np.ndarray, theta_hat: np.ndarray) -> float:
    """(TP TN - FP FN) / sqrt((TP + FP)(TP + FN)(TN + FP)(TN + FN)); 0 when a factor of the
    denominator is 0 (one of the patterns is all-zero or all-nonzero)."""
    tp, tn, fp, fn = support_counts(theta_true, theta_hat)
    den = (tp + fp) * (tp + fn) * (tn + fp) * (tn + fn)
    if den == 0:
        return 0.0
    return (tp * tn - fp * fn) / math.sqrt(den)
