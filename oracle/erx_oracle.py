"""FP64 NumPy oracle of the ERX per-line step (test infrastructure only).

Plain and slow on purpose: each function below is one step of Sec. III of the
paper, in the paper's order and notation, with library primitives (mean,
matrix product, Cholesky, triangular solve) as the only building blocks.  It
shares no code with the CUDA path; only tests, the smoke check and the
benchmark's CPU-baseline leg import it.

Readings taken where the paper is ambiguous (each is a decision, recorded here
so the code can be checked against it):

* Order: the line is scored against the statistics that already include it
  (Sec. III-D scores with mu_t and L_t, the state after the Sec. III-C update;
  Sec. IV-C calls alpha = 1 "only the current line").  Score-then-update is
  kept as an option.
* Factor: L_t is the Cholesky factor of K_t + 1e-5 I (the printed "lower
  triangle of K_t^-1 + 1e-5 I" cannot make L m = z - mu a Mahalanobis solve).
* Solve: column form L_t m_i = z_i - mu_t, delta_i = sqrt(m_i . m_i) (Sec. III-D).
* Ridge: absolute 1e-5, added at factorisation only, not stored in the state.
* Line covariance normaliser 1/(p-1) (Sec. III-C); normalisation uses the
  population standard deviation, and a line with zero spread gets delta_N = 0.
* Warm-up: the 99-line buffer of Sec. IV-B is a warm-up; those lines are
  scored like any other and flagged not-detecting.
* IMC (the ablation of Sec. IV-C that replaces the EMAs): a batch version of
  Welford's update (the paper cites Schubert and Gertz 2018), so the state is
  the mean and the 1/(n-1) covariance of all n pixels seen so far, every line
  weighed equally; the momentum is not used.
* "pooled": the other reading of the 99-line buffer (Sec. IV-B): the warm-up
  lines are pooled with equal weight (the IMC update) into the estimate the
  EMAs start from; from the first line after the warm-up on, the EMAs of
  Sec. III-C.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from .srp import srp_weights


def project(x: np.ndarray, w: np.ndarray | None) -> np.ndarray:
    """Sec. III-B: Z_t = X_t . W (identity when there is no projection)."""
    z = np.asarray(x, dtype=np.float64)
    if w is None:
        return z
    return z @ w


def line_stats(z: np.ndarray):
    """Sec. III-C: line mean mu_hat = (1/p) sum z_i and covariance
    K_hat = 1/(p-1) sum (z_i - mu_hat)(z_i - mu_hat)^T (two passes)."""
    p = z.shape[0]
    mu_hat = z.sum(axis=0) / p
    r = z - mu_hat
    k_hat = (r.T @ r) / (p - 1)
    return mu_hat, k_hat


def ema_update(mu, k, mu_hat, k_hat, alpha: float):
    """Sec. III-C: mu_t = (1-a) mu_{t-1} + a mu_hat_t, K_t = (1-a) K_{t-1} + a K_hat_t."""
    return (1.0 - alpha) * mu + alpha * mu_hat, (1.0 - alpha) * k + alpha * k_hat


def imc_update(mu, k, n_a: int, mu_hat, k_hat, n_b: int):
    """Sec. IV-C's IMC, batch Welford (Schubert and Gertz 2018): merge the n_a
    pixels summarised by (mu, k) with a line of n_b pixels (mu_hat, k_hat).
    With the scatter M = (n - 1) K of each part and delta = mu_hat - mu:
    mu' = mu + delta n_b / n,  M' = M_a + M_b + delta delta^T n_a n_b / n,
    n = n_a + n_b.  Returns (mu', K' = M' / (n - 1))."""
    n = n_a + n_b
    delta = mu_hat - mu
    mu_new = mu + delta * (n_b / n)
    m = k * (n_a - 1) + k_hat * (n_b - 1) + np.outer(delta, delta) * (n_a * n_b / n)
    return mu_new, m / (n - 1)


def cholesky_ridge(k: np.ndarray, ridge: float) -> np.ndarray:
    """Sec. III-D: lower L with L L^T = K_t + ridge * I."""
    d = k.shape[0]
    return np.linalg.cholesky(k + ridge * np.eye(d))


def mahalanobis(z: np.ndarray, mu: np.ndarray, lower: np.ndarray) -> np.ndarray:
    """Sec. III-D: forward substitution L m_i = z_i - mu, delta_i = sqrt(m_i . m_i)."""
    r = (z - mu).T                                    # d x p, one column per pixel
    m = scipy.linalg.solve_triangular(lower, r, lower=True)
    return np.sqrt(np.sum(m * m, axis=0))


def normalise(delta: np.ndarray) -> np.ndarray:
    """Sec. III-E: delta_N = (delta - mean) / std, population std; 0 when std = 0."""
    mean = delta.sum() / delta.size
    dev = delta - mean
    std = math.sqrt(float(np.sum(dev * dev)) / delta.size)
    if std == 0.0:
        return np.zeros_like(delta)
    return dev / std


class ERXOracle:
    """Line-by-line ERX detector state (Sec. III, Fig. 'ERX algorithm flowchart').

    Parameters follow the paper's symbols: ``bands`` = b, ``width`` = p,
    ``momentum`` = alpha (default 0.1, Sec. III-C), ``proj_dim`` = d (default 5,
    Sec. III-B), ``ridge`` = 1e-5 (Sec. III-D), ``warmup`` = 99 lines (Sec. IV-B),
    ``threshold`` = tau_N (Sec. III-E; None for no mask).
    ``proj`` is "none" (all bands), "srp" (matrix drawn from ``seed``) or an
    explicit b x d array.  ``averaging`` is "ema" (Sec. III-C), "imc" (the
    equal-weight ablation of Sec. IV-C) or "pooled" (IMC over the ``warmup``
    lines, the EMAs afterwards).
    """

    def __init__(self, bands: int, width: int, momentum: float = 0.1, proj="none",
                 proj_dim: int = 5, seed: int = 0, ridge: float = 1e-5,
                 warmup: int = 99, order: str = "update_then_score",
                 threshold: float | None = None, averaging: str = "ema"):
        if not (0.0 < momentum <= 1.0):
            raise ValueError("momentum must be in (0, 1]")
        if width < 2:
            raise ValueError("a line needs at least 2 pixels for its covariance")
        if order not in ("update_then_score", "score_then_update"):
            raise ValueError(order)
        if averaging not in ("ema", "imc", "pooled"):
            raise ValueError(averaging)
        self.averaging = averaging
        self.bands, self.width = bands, width
        self.alpha, self.ridge = float(momentum), float(ridge)
        self.warmup, self.order, self.threshold = warmup, order, threshold
        if isinstance(proj, np.ndarray):
            self.w = np.asarray(proj, dtype=np.float64)
        elif proj == "srp":
            self.w = srp_weights(bands, proj_dim, seed)
        elif proj == "none":
            self.w = None
        else:
            raise ValueError(proj)
        self.dim = bands if self.w is None else self.w.shape[1]
        self.t = 0
        self.mu = np.zeros(self.dim)
        self.k = np.zeros((self.dim, self.dim))

    def _update(self, mu_hat, k_hat):
        if self.t == 0:                       # Sec. III-C: start from the first line
            self.mu, self.k = mu_hat.copy(), k_hat.copy()
        elif self.averaging == "imc" or (self.averaging == "pooled" and self.t < self.warmup):
            # all lines so far have width pixels each
            self.mu, self.k = imc_update(self.mu, self.k, self.t * self.width, mu_hat, k_hat,
                                         self.width)
        else:
            self.mu, self.k = ema_update(self.mu, self.k, mu_hat, k_hat, self.alpha)

    def push(self, x: np.ndarray) -> dict:
        """Process one line x of shape (p, b); return its scores."""
        z = project(x, self.w)
        mu_hat, k_hat = line_stats(z)
        if self.order == "update_then_score":
            self._update(mu_hat, k_hat)
            mu, k = self.mu, self.k
        else:
            mu, k = (mu_hat, k_hat) if self.t == 0 else (self.mu, self.k)
        lower = cholesky_ridge(k, self.ridge)
        delta = mahalanobis(z, mu, lower)
        if self.order == "score_then_update":
            self._update(mu_hat, k_hat)
        dn = normalise(delta)
        out = {
            "delta": delta,
            "delta_n": dn,
            "detecting": self.t >= self.warmup,
        }
        if self.threshold is not None:
            out["mask"] = dn >= self.threshold
        self.t += 1
        return out

    def state(self):
        return self.t, self.mu.copy(), self.k.copy()

    def set_state(self, t, mu, k):
        self.t, self.mu, self.k = int(t), np.array(mu, np.float64), np.array(k, np.float64)


def run_cube(cube: np.ndarray, **kw) -> dict:
    """Run ERX over cube[line][pixel][band]; stacked per-line outputs."""
    n, p, b = cube.shape
    det = ERXOracle(b, p, **kw)
    outs = [det.push(cube[t]) for t in range(n)]
    res = {k: np.stack([o[k] for o in outs]) for k in ("delta", "delta_n")}
    res["detecting"] = np.array([o["detecting"] for o in outs])
    if "mask" in outs[0]:
        res["mask"] = np.stack([o["mask"] for o in outs])
    res["state"] = det.state()
    res["oracle"] = det
    return res
