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


def test_code_ema_closed_form():
    """CodeEMA after T lines equals the solved Sec. III-C recursion: weights
    (1-a)^(T-1) for line 0 and a (1-a)^(T-1-j) for line j >= 1 on each line's
    code mean and 1/(p-1) covariance (numpy.cov), weights summing to 1."""
    r = np.random.default_rng(11)
    a, T, p, k = 0.3, 7, 25, 4
    codes = [r.standard_normal((p, k)) * (1 + j) + j for j in range(T)]
    ema = enc.CodeEMA(a)
    for c in codes:
        mu, kk = ema.update(c)
    w = [(1 - a) ** (T - 1)] + [a * (1 - a) ** (T - 1 - j) for j in range(1, T)]
    assert abs(sum(w) - 1.0) < 1e-15
    mu_want = sum(wj * c.mean(axis=0) for wj, c in zip(w, codes))
    k_want = sum(wj * np.cov(c, rowvar=False, ddof=1) for wj, c in zip(w, codes))
    assert ema.t == T
    assert np.allclose(mu, mu_want, rtol=1e-12, atol=1e-13)
    assert np.allclose(kk, k_want, rtol=1e-12, atol=1e-13)


def test_code_ema_first_line_initialises():
    c = np.random.default_rng(2).standard_normal((30, 5))
    mu, kk = enc.CodeEMA(0.1).update(c)
    assert np.allclose(mu, c.mean(axis=0), rtol=1e-14)
    assert np.allclose(kk, np.cov(c, rowvar=False), rtol=1e-12)


def _fd_grad(params, x, shift, scale, mu_e, k_e, target, ridge, h=1e-6):
    """Central differences of one line's loss, statistics held constant."""
    g = {}
    for name, v in params.items():
        g[name] = np.zeros_like(v)
        for idx in np.ndindex(v.shape):
            pp = {n: w.copy() for n, w in params.items()}
            pm = {n: w.copy() for n, w in params.items()}
            pp[name][idx] += h
            pm[name][idx] -= h
            g[name][idx] = (_loss_fixed_stats(pp, x, shift, scale, mu_e, k_e, target, ridge)
                            - _loss_fixed_stats(pm, x, shift, scale, mu_e, k_e, target, ridge)
                            ) / (2 * h)
    return g


def _loss_by_inverse(params, x, shift, scale, mu_e, k_e, target, ridge):
    """The line loss from its definition: explicit inverse, no Cholesky."""
    c, _ = enc.forward(params, x, shift, scale)
    inv = np.linalg.inv(k_e + ridge * np.eye(k_e.shape[0]))
    d = np.sqrt(np.einsum("ij,jk,ik->i", c - mu_e, inv, c - mu_e))
    return float(np.mean((np.log1p(d) - np.log1p(target)) ** 2))


def test_train_line_steps_follow_their_definition():
    """Two steps of train_line against the training objective written out:
    step 1 moves every parameter by AdamW's first-step closed form with the
    finite-difference gradient (statistics of line 1's own codes held
    constant); step 2's loss is the definition evaluated with the parameters
    after step 1 and the code EMA updated with line 2's codes (update then
    score, Sec. III-C/D)."""
    params, x1, shift, scale, t1 = _setup(p=30, b=5, h=6, k=3, seed=3)
    r = np.random.default_rng(9)
    x2 = x1 + 0.05 * r.standard_normal(x1.shape)
    t2 = t1[::-1].copy()
    ridge, lr, wd, alpha = 1e-3, 1e-2, 1e-3, 0.25
    p0 = {n: v.copy() for n, v in params.items()}
    opt = enc.AdamW(params, lr=lr, wd=wd)
    ema = enc.CodeEMA(alpha)
    l1 = enc.train_line(params, opt, ema, x1, t1, shift, scale, ridge)
    # step 1: statistics of line 1's codes under the initial parameters
    c1, _ = enc.forward(p0, x1, shift, scale)
    mu1, k1 = c1.mean(axis=0), np.cov(c1, rowvar=False)
    assert abs(l1 - _loss_by_inverse(p0, x1, shift, scale, mu1, k1, t1, ridge)) <= 1e-12 * l1
    g = _fd_grad(p0, x1, shift, scale, mu1, k1, t1, ridge)
    for n in p0:
        want = p0[n] - lr * (g[n] / (np.abs(g[n]) + opt.eps) + wd * p0[n])
        big = np.abs(g[n]) > 1e-6           # the sign of a vanishing gradient is noise
        assert np.allclose(params[n][big], want[big], rtol=0, atol=1e-9), n
    p1 = {n: v.copy() for n, v in params.items()}
    l2 = enc.train_line(params, opt, ema, x2, t2, shift, scale, ridge)
    c2, _ = enc.forward(p1, x2, shift, scale)
    mu2 = (1 - alpha) * mu1 + alpha * c2.mean(axis=0)
    k2 = (1 - alpha) * k1 + alpha * np.cov(c2, rowvar=False)
    assert abs(l2 - _loss_by_inverse(p1, x2, shift, scale, mu2, k2, t2, ridge)) <= 1e-10 * l2
