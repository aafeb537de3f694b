"""Pins of the learned-encoder oracle (CPU): finite differences of the loss
with the code statistics held constant, the AdamW update against its closed
form, and ReLU/bias conventions."""
import numpy as np

from oracle import encoder as enc


def _setup(p=40, b=12, h=9, k=4, seed=0):
    r = np.random.default_rng(seed)
    params = enc.init_params(b, h, k, seed)
    params["b1"] = r.standard_normal(h) * 0.1
    params["b2"] = r.standard_normal(k) * 0.1
    x = r.random((p, b))
    shift, scale = x.mean(axis=0), 1.0 / x.std(axis=0)
    target = np.abs(r.standard_normal(p)) * 2 + 0.5
    return params, x, shift, scale, target


def _loss_fixed_stats(params, x, shift, scale, mu_e, k_e, target, ridge=1e-3):
    c, _ = enc.forward(params, x, shift, scale)
    return enc.loss_and_dcodes(c, mu_e, k_e, ridge, target)[0]


def test_gradient_matches_finite_differences():
    params, x, shift, scale, target = _setup()
    c, cache = enc.forward(params, x, shift, scale)
    mu_e, k_e = enc.code_stats(c)
    loss, dc, _ = enc.loss_and_dcodes(c, mu_e, k_e, 1e-3, target)
    grads = enc.backward(params, cache, dc)
    r = np.random.default_rng(5)
    for name in ("W1", "b1", "W2", "b2"):
        for _ in range(6):
            idx = tuple(r.integers(0, s) for s in params[name].shape)
            h = 1e-6
            pp = {n: v.copy() for n, v in params.items()}
            pm = {n: v.copy() for n, v in params.items()}
            pp[name][idx] += h
            pm[name][idx] -= h
            fd = (_loss_fixed_stats(pp, x, shift, scale, mu_e, k_e, target)
                  - _loss_fixed_stats(pm, x, shift, scale, mu_e, k_e, target)) / (2 * h)
            assert abs(fd - grads[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd,
                                                                               grads[name][idx])


def test_code_delta_is_mahalanobis():
    params, x, shift, scale, target = _setup()
    c, _ = enc.forward(params, x, shift, scale)
    mu, kk = enc.code_stats(c)
    _, _, delta = enc.loss_and_dcodes(c, mu, kk, 1e-3, target)
    inv = np.linalg.inv(kk + 1e-3 * np.eye(kk.shape[0]))
    want = np.sqrt(np.einsum("ij,jk,ik->i", c - mu, inv, c - mu))
    assert np.allclose(delta, want, rtol=1e-12)


def test_adamw_first_step_closed_form():
    """After one step with gradient g: m_hat = g, v_hat = g^2, so each entry
    moves by -lr (g/(|g| + eps) + wd theta)."""
    theta = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -0.01, 2.0])}
    opt = enc.AdamW(theta, lr=0.01, eps=1e-8, wd=0.1)
    before = theta["w"].copy()
    opt.step(theta, g)
    want = before - 0.01 * (g["w"] / (np.abs(g["w"]) + 1e-8) + 0.1 * before)
    assert np.allclose(theta["w"], want, rtol=1e-12, atol=0)


def test_relu_blocks_gradient_of_inactive_units():
    params, x, shift, scale, target = _setup()
    params["b1"][:] = -100.0           # every hidden unit off
    c, cache = enc.forward(params, x, shift, scale)
    mu, kk = enc.code_stats(c + np.random.default_rng(0).standard_normal(c.shape))
    _, dc, _ = enc.loss_and_dcodes(c, mu, kk, 1e-3, target)
    g = enc.backward(params, cache, dc)
    assert np.all(g["W1"] == 0) and np.all(g["b1"] == 0) and np.all(g["W2"] == 0)


def test_training_reduces_loss():
    r = np.random.default_rng(1)
    b, p = 10, 60
    params = enc.init_params(b, 16, 3, 2)
    opt = enc.AdamW(params, lr=3e-3)
    xs = [r.random((p, b)) for _ in range(40)]
    shift, scale = np.mean(xs[0], 0), 1 / np.std(xs[0], 0)
    # targets: full-band RX of each line against its own statistics
    tg = []
    for x in xs:
        mu, kk = x.mean(0), np.cov(x.T)
        inv = np.linalg.inv(kk + 1e-5 * np.eye(b))
        tg.append(np.sqrt(np.einsum("ij,jk,ik->i", x - mu, inv, x - mu)))
    losses = []
    for epoch in range(6):
        ema = enc.CodeEMA(1.0)
        losses.append(np.mean([enc.train_line(params, opt, ema, x, t, shift, scale)
                               for x, t in zip(xs, tg)]))
    assert losses[-1] < 0.9 * losses[0]
