"""Detection-quality metrics of Sec. IV-B, FP64 NumPy (test infrastructure only).

A detection map (one score per pixel) is judged against the anomaly labels:

* ROC: the true-positive rate TPR = TP / (TP + FN) against the false-positive
  rate FPR = FP / (FP + TN) over all thresholds; AUC is the area under it,
  which equals the Mann-Whitney probability that an anomaly scores above a
  background pixel (ties counting one half).
* AUC_TPR,tau and AUC_FPR,tau: the areas under TPR and FPR against the
  threshold tau, with the scores min-max normalised to [0, 1] (tau runs over
  [0, 1]).  For a pixel with normalised score v the indicator [v >= tau]
  integrates to v, so these areas are the mean normalised score of the
  anomalies and of the background.
* AUC_TD = (AUC + AUC_TPR,tau) / 2 and AUC_BS = (AUC - AUC_FPR,tau + 1) / 2.

The GPU computes the AUC from histograms of the normalised scores quantised
to `bins` levels, q = min(floor(v * bins), bins - 1) with v = (s - min) /
(max - min) in FP64; `auc_binned` is the same quantity (exact integer counts),
`auc_exact` the rank form on the unquantised scores.  A constant map has
AUC 1/2 and normalised scores 0.
"""
from __future__ import annotations

import numpy as np
import scipy.stats


def normalised(scores: np.ndarray) -> np.ndarray:
    s = np.asarray(scores, dtype=np.float64).ravel()
    lo, hi = s.min(), s.max()
    if hi == lo:
        return np.zeros_like(s)
    return (s - lo) / (hi - lo)


def quantised(scores: np.ndarray, bins: int) -> np.ndarray:
    return np.minimum(np.floor(normalised(scores) * bins), bins - 1).astype(np.int64)


def auc_exact(scores: np.ndarray, labels: np.ndarray) -> float:
    """Mann-Whitney form: (sum of the anomalies' ranks - n_p (n_p + 1) / 2) / (n_p n_n),
    ranks averaged over ties."""
    s = np.asarray(scores, dtype=np.float64).ravel()
    y = np.asarray(labels, dtype=bool).ravel()
    n_p, n_n = int(y.sum()), int((~y).sum())
    r = scipy.stats.rankdata(s)
    return float((r[y].sum() - n_p * (n_p + 1) / 2.0) / (n_p * n_n))


def auc_binned(scores: np.ndarray, labels: np.ndarray, bins: int):
    """AUC of the quantised map from the two histograms: 2 U = sum over levels of
    pos[q] (2 * background below q + background at q).  Returns (2U, n_p, n_n)."""
    q = quantised(scores, bins)
    y = np.asarray(labels, dtype=bool).ravel()
    pos = np.bincount(q[y], minlength=bins).astype(np.int64)
    neg = np.bincount(q[~y], minlength=bins).astype(np.int64)
    below = np.concatenate(([0], np.cumsum(neg)[:-1]))
    u2 = int(np.sum(pos * (2 * below + neg)))
    return u2, int(y.sum()), int((~y).sum())


def roc_metrics(scores: np.ndarray, labels: np.ndarray, bins: int = 1 << 16) -> dict:
    s = np.asarray(scores, dtype=np.float64).ravel()
    y = np.asarray(labels, dtype=bool).ravel()
    u2, n_p, n_n = auc_binned(s, y, bins)
    auc = u2 / (2.0 * n_p * n_n)
    lo, hi = s.min(), s.max()
    if hi == lo:
        tpr_tau = fpr_tau = 0.0
    else:
        tpr_tau = (s[y].sum() / n_p - lo) / (hi - lo)
        fpr_tau = (s[~y].sum() / n_n - lo) / (hi - lo)
    return {"auc": auc, "auc_tpr_tau": tpr_tau, "auc_fpr_tau": fpr_tau,
            "auc_td": (auc + tpr_tau) / 2.0, "auc_bs": (auc - fpr_tau + 1.0) / 2.0,
            "u2": u2, "positives": n_p, "negatives": n_n}
