"""FP64 oracle of the learned band encoder (test infrastructure only).

The paper lists learning-based extensions of ERX as future work (Sec. V,
conclusion) and uses sparse random projection (Sec. III-B) to shrink b bands
to d dimensions.  This learned counterpart replaces the random projection
with a small MLP, codes c = W2 relu(W1 xn + b1) + b2 with xn = (x - shift) *
scale, trained so that ERX run on the codes ranks pixels like ERX on all bands.

Training objective, per line t (processed in order, as the detector would):
  * codes C_t of the line's pixels;
  * code-space ERX statistics, update then score (Sec. III-C/D): the line's
    code mean and 1/(p-1) covariance update an EMA (mu_e, K_e) with momentum
    alpha (line 0 initialises it); P = (K_e + eps I)^-1;
  * delta_i = sqrt(r_i^T P r_i), r_i = c_i - mu_e;
  * L_t = mean_i (log(1 + delta_i) - log(1 + target_i))^2, target = full-band ERX delta.
The statistics (mu_e, K_e, P) are treated as constants when differentiating
(stop-gradient), so dL/dc_i = (2/p) (log1p(delta_i) - log1p(target_i)) /
(1 + delta_i) * P r_i / delta_i.  Parameters are updated with AdamW
(Loshchilov & Hutter): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
theta -= lr (m/(1-b1^k) / (sqrt(v/(1-b2^k)) + eps) + wd theta).
"""
from __future__ import annotations

import numpy as np


def init_params(bands: int, hidden: int, k: int, seed: int) -> dict:
    """He-style initial weights from a seeded generator (inputs, not method arithmetic)."""
    r = np.random.default_rng([seed, 0xE1C])
    return {
        "W1": r.standard_normal((hidden, bands)) * np.sqrt(2.0 / bands),
        "b1": np.zeros(hidden),
        "W2": r.standard_normal((k, hidden)) * np.sqrt(1.0 / hidden),
        "b2": np.zeros(k),
    }


def forward(params: dict, x: np.ndarray, shift: np.ndarray, scale: np.ndarray):
    """x: (p, b).  Returns codes (p, k) and the cache for backward."""
    xn = (np.asarray(x, np.float64) - shift) * scale
    a = xn @ params["W1"].T + params["b1"]
    h = np.maximum(a, 0.0)
    c = h @ params["W2"].T + params["b2"]
    return c, (xn, a, h)


def code_stats(c: np.ndarray):
    p = c.shape[0]
    mu = c.mean(axis=0)
    r = c - mu
    return mu, (r.T @ r) / (p - 1)


def loss_and_dcodes(c: np.ndarray, mu_e: np.ndarray, k_e: np.ndarray, ridge: float,
                    target: np.ndarray):
    """Loss of one line and dL/dc with the code statistics held constant."""
    p, k = c.shape
    P = np.linalg.inv(k_e + ridge * np.eye(k))
    r = c - mu_e
    u = r @ P                       # P symmetric: rows are (P r_i)^T
    delta = np.sqrt(np.maximum(np.sum(r * u, axis=1), 0.0))
    diff = np.log1p(delta) - np.log1p(target)
    loss = float(np.mean(diff * diff))
    coef = np.where(delta > 0, 2.0 * diff / ((1.0 + delta) * np.maximum(delta, 1e-300) * p), 0.0)
    return loss, coef[:, None] * u, delta


def backward(params: dict, cache, dc: np.ndarray) -> dict:
    xn, a, h = cache
    dh = (dc @ params["W2"]) * (a > 0)
    return {"W2": dc.T @ h, "b2": dc.sum(axis=0), "W1": dh.T @ xn, "b1": dh.sum(axis=0)}


class AdamW:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
        self.lr, self.b1, self.b2, self.eps, self.wd = lr, beta1, beta2, eps, wd
        self.m = {n: np.zeros_like(v) for n, v in params.items()}
        self.v = {n: np.zeros_like(v) for n, v in params.items()}
        self.k = 0

    def step(self, params, grads):
        self.k += 1
        c1 = 1.0 - self.b1 ** self.k
        c2 = 1.0 - self.b2 ** self.k
        for n in params:
            g = grads[n]
            self.m[n] = self.b1 * self.m[n] + (1 - self.b1) * g
            self.v[n] = self.b2 * self.v[n] + (1 - self.b2) * g * g
            upd = (self.m[n] / c1) / (np.sqrt(self.v[n] / c2) + self.eps)
            params[n] = params[n] - self.lr * (upd + self.wd * params[n])


class CodeEMA:
    """Code-space ERX statistics, update then score (Sec. III-C)."""

    def __init__(self, alpha: float):
        self.alpha, self.t, self.mu, self.k = alpha, 0, None, None

    def update(self, c):
        mu_h, k_h = code_stats(c)
        if self.t == 0:
            self.mu, self.k = mu_h, k_h
        else:
            a = self.alpha
            self.mu = (1 - a) * self.mu + a * mu_h
            self.k = (1 - a) * self.k + a * k_h
        self.t += 1
        return self.mu, self.k


def train_line(params, opt, ema: CodeEMA, x, target, shift, scale, ridge=1e-5):
    """One training step on one line; returns the line's loss."""
    c, cache = forward(params, x, shift, scale)
    mu_e, k_e = ema.update(c)
    loss, dc, _ = loss_and_dcodes(c, mu_e, k_e, ridge, target)
    opt.step(params, backward(params, cache, dc))
    return loss
