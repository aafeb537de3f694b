"""Plant plausible mistakes in the oracle (on the CPU) and require a pin to catch each.

This shows the pins in tests/oracle_checks.py are discriminating: a dropped
term, a wrong normaliser, swapped weights, a transposed factor or a wrong
statistic each make at least one of them fail.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import erx_oracle as eo
from tests import oracle_checks as oc


def _stats_over_p(z):
    p = z.shape[0]
    mu = z.sum(axis=0) / p
    r = z - mu
    return mu, (r.T @ r) / p


def _ema_swapped(mu, k, mu_hat, k_hat, alpha):
    return alpha * mu + (1 - alpha) * mu_hat, alpha * k + (1 - alpha) * k_hat


def _chol_no_ridge(k, ridge):
    return np.linalg.cholesky(k)


def _solve_transposed(z, mu, lower):
    m = scipy.linalg.solve_triangular(lower.T, (z - mu).T, lower=False)
    return np.sqrt(np.sum(m * m, axis=0))


def _normalise_ddof1(delta):
    return (delta - delta.mean()) / delta.std(ddof=1)


def _stats_uncentred(z):
    p = z.shape[0]
    mu = z.sum(axis=0) / p
    return mu, (z.T @ z) / (p - 1)


def _imc_no_between(mu, k, n_a, mu_hat, k_hat, n_b):
    n = n_a + n_b
    m = k * (n_a - 1) + k_hat * (n_b - 1)
    return mu + (mu_hat - mu) * (n_b / n), m / (n - 1)


def _imc_weights_by_line(mu, k, n_a, mu_hat, k_hat, n_b):
    # equal weight per line count instead of per pixel, and no between-line term
    t = n_a // n_b
    return (t * mu + mu_hat) / (t + 1), (t * k + k_hat) / (t + 1)


MUTATIONS = {
    "imc_between_term_dropped": ("imc_update", _imc_no_between),
    "imc_average_of_covariances": ("imc_update", _imc_weights_by_line),
    "cov_over_p": ("line_stats", _stats_over_p),
    "ema_weights_swapped": ("ema_update", _ema_swapped),
    "ridge_dropped": ("cholesky_ridge", _chol_no_ridge),
    "factor_transposed": ("mahalanobis", _solve_transposed),
    "normalise_ddof1": ("normalise", _normalise_ddof1),
    "cov_uncentred": ("line_stats", _stats_uncentred),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    attr, bad = MUTATIONS[name]
    monkeypatch.setattr(eo, attr, bad)
    failed = []
    for check, (fn, tol) in oc.ALL_CHECKS.items():
        try:
            err = fn()
        except (np.linalg.LinAlgError, ValueError, FloatingPointError):
            err = math.inf
        if not (err <= tol):
            failed.append(check)
    assert failed, f"mutation {name} passed every pin"


def test_init_from_zero_is_caught(monkeypatch):
    orig = eo.ERXOracle._update

    def bad(self, mu_hat, k_hat):
        if self.t == 0:
            self.mu, self.k = eo.ema_update(np.zeros_like(mu_hat), np.zeros_like(k_hat),
                                            mu_hat, k_hat, self.alpha)
        else:
            orig(self, mu_hat, k_hat)

    monkeypatch.setattr(eo.ERXOracle, "_update", bad)
    errs = {k: fn() for k, (fn, tol) in oc.ALL_CHECKS.items()}
    assert any(errs[k] > oc.ALL_CHECKS[k][1] for k in errs)


def test_order_swap_is_caught(monkeypatch):
    orig_init = eo.ERXOracle.__init__

    def swapped(self, *a, **kw):
        orig_init(self, *a, **kw)
        self.order = ("score_then_update" if self.order == "update_then_score"
                      else "update_then_score")

    monkeypatch.setattr(eo.ERXOracle, "__init__", swapped)
    errs = {k: fn() for k, (fn, tol) in oc.ALL_CHECKS.items()}
    assert any(errs[k] > oc.ALL_CHECKS[k][1] for k in errs)


def test_pooled_boundary_off_by_one_is_caught(monkeypatch):
    # the pooled reading switching to the EMAs one line late
    def late(self, mu_hat, k_hat):
        if self.t == 0:
            self.mu, self.k = mu_hat.copy(), k_hat.copy()
        elif self.averaging == "imc" or (self.averaging == "pooled" and self.t <= self.warmup):
            self.mu, self.k = eo.imc_update(self.mu, self.k, self.t * self.width, mu_hat, k_hat,
                                            self.width)
        else:
            self.mu, self.k = eo.ema_update(self.mu, self.k, mu_hat, k_hat, self.alpha)

    monkeypatch.setattr(eo.ERXOracle, "_update", late)
    errs = {k: fn() for k, (fn, tol) in oc.ALL_CHECKS.items()}
    assert any(errs[k] > oc.ALL_CHECKS[k][1] for k in errs)


# ---- the learned encoder's oracle ------------------------------------------

def _encoder_pins():
    from tests import test_oracle_encoder as te
    return [getattr(te, n) for n in dir(te) if n.startswith("test_")]


def _pins_fail():
    failed = []
    for pin in _encoder_pins():
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            failed.append(pin.__name__)
    return failed


def test_encoder_pins_pass_unmutated():
    assert _pins_fail() == []


def _code_ema_swapped(self, c):
    mu_h, k_h = self_stats = (c.mean(axis=0), np.cov(c, rowvar=False))
    if self.t == 0:
        self.mu, self.k = self_stats
    else:
        a = self.alpha
        self.mu = a * self.mu + (1 - a) * mu_h
        self.k = a * self.k + (1 - a) * k_h
    self.t += 1
    return self.mu, self.k


def _train_line_score_then_update(params, opt, ema, x, target, shift, scale, ridge=1e-5):
    from oracle import encoder as enc
    c, cache = enc.forward(params, x, shift, scale)
    if ema.t == 0:
        mu_e, k_e = enc.code_stats(c)
    else:
        mu_e, k_e = ema.mu, ema.k
    ema.update(c)
    loss, dc, _ = enc.loss_and_dcodes(c, mu_e, k_e, ridge, target)
    opt.step(params, enc.backward(params, cache, dc))
    return loss


def _backward_no_gate(params, cache, dc):
    xn, a, h = cache
    dh = dc @ params["W2"]
    return {"W2": dc.T @ h, "b2": dc.sum(axis=0), "W1": dh.T @ xn, "b1": dh.sum(axis=0)}


ENCODER_MUTATIONS = {
    "code_ema_weights_swapped": ("CodeEMA.update", _code_ema_swapped),
    "train_line_scores_before_update": ("train_line", _train_line_score_then_update),
    "backward_drops_relu_gate": ("backward", _backward_no_gate),
}


@pytest.mark.parametrize("name", sorted(ENCODER_MUTATIONS))
def test_encoder_mutation_is_caught(name, monkeypatch):
    from oracle import encoder as enc
    attr, bad = ENCODER_MUTATIONS[name]
    if attr == "CodeEMA.update":
        monkeypatch.setattr(enc.CodeEMA, "update", bad)
    else:
        monkeypatch.setattr(enc, attr, bad)
    assert _pins_fail(), f"mutation {name} passed every encoder pin"
