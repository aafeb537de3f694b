"""Learned band encoder on the GPU against its FP64 oracle, and the learned
form against full-band ERX (GPU)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import encoder as enc_or
from tests.gpu_util import need_gpu, rel_err, run_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to the nearest bf16 (ties to even), as float64."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _encoder(b, h, k, seed=3):
    from paper_2408_14947_gb300 import Encoder
    e = Encoder(b, h, k, seed=seed)
    p = enc_or.init_params(b, h, k, seed)
    r = np.random.default_rng(seed)
    p["b1"] = r.standard_normal(h) * 0.1
    p["b2"] = r.standard_normal(k) * 0.1
    theta = np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"]]).astype(np.float32)
    e.params(theta)
    # the oracle sees the weights the GPU multiplies with: bf16 W1, W2; float32 biases
    q = {"W1": bf16_round(p["W1"]), "b1": p["b1"].astype(np.float32).astype(np.float64),
         "W2": bf16_round(p["W2"]), "b2": p["b2"].astype(np.float32).astype(np.float64)}
    return e, q


def forward_parts(q, x, shift, scale):
    """The oracle forward at the tensor-core kernel's rounding points: xn =
    (x - shift) * scale in float32, then bf16; layer 1 by the oracle on those;
    the hidden activations relu(a) rounded to bf16; layer 2 on those.  Returns
    (xn_bf, a, h_bf, codes)."""
    xn = np.asarray(x, np.float32) - np.asarray(shift, np.float32)
    xn = bf16_round((xn * np.asarray(scale, np.float32)).astype(np.float32))
    b = xn.shape[1]
    _, (_, a, h) = enc_or.forward(q, xn, np.zeros(b), np.ones(b))
    h_bf = bf16_round(h.astype(np.float32))
    return xn, a, h_bf, h_bf @ q["W2"].T + q["b2"]


def forward_bf16(q, x, shift, scale):
    return forward_parts(q, x, shift, scale)[3]


U_BF16 = 2.0 ** -8     # unit roundoff of bf16 (8 significant bits)


def grad_bound(q, parts, dc, eps32=1e-4):
    """Componentwise bound on the GPU gradient's deviation from the oracle's
    gradient at the same rounding points: the backward rounds dL/dc to bf16
    (in dc W2 and in h^T dc) and dL/dh to bf16 (in dh^T xn), each a relative
    u = 2^-8, and accumulates in FP32; eps32 covers the FP32 forward and loss.
    Returns a vector in the parameter layout [W1 | b1 | W2 | b2]."""
    xn, a, h_bf, _ = parts
    gate = (a > 0).astype(np.float64)
    dabs = (np.abs(dc) @ np.abs(q["W2"])) * gate            # |dc| |W2| per pixel, unit
    bw1 = (2 * U_BF16 + eps32) * (dabs.T @ np.abs(xn))
    bb1 = (U_BF16 + eps32) * dabs.sum(axis=0)
    bw2 = (U_BF16 + eps32) * (np.abs(dc).T @ h_bf)
    bb2 = eps32 * np.abs(dc).sum(axis=0)
    return np.concatenate([bw1.ravel(), bb1, bw2.ravel(), bb2])


def _line(w, b, seed=0):
    cfg = synth.SceneConfig(bands=b, width=w, seed=seed, n_end=(3, 5), noise=0.02)
    return synth.gen_lines(cfg, 0, 1)[0]


def test_forward_matches_oracle():
    need_gpu()
    b, h, k = 40, 24, 8
    e, q = _encoder(b, h, k)
    x = _line(300, b)
    shift, scale = x.mean(0), 1.0 / (x.std(0) + 1e-3)
    e.set_norm(shift, scale)
    got = e.forward(to_dev(x)).cpu().numpy()
    # the inference forward runs on the tensor cores with bf16 activations
    want = forward_bf16(q, x, shift, scale)
    assert np.max(np.abs(got - want)) <= 1e-3 * np.max(np.abs(want))
    # and stays within bf16 rounding of the FP32-activation forward of the oracle
    full, _ = enc_or.forward(q, x, shift.astype(np.float32), scale.astype(np.float32))
    assert np.max(np.abs(got - full)) <= 2e-2 * np.max(np.abs(full))


def _oracle_line_grad(q, x, shift, scale, mu_e, k_e, target, ridge=1e-5):
    parts = forward_parts(q, x, shift, scale)
    loss, dc, _ = enc_or.loss_and_dcodes(parts[3], mu_e, k_e, ridge, target)
    gw = enc_or.backward(q, (parts[0], parts[1], parts[2]), dc)
    g = np.concatenate([gw["W1"].ravel(), gw["b1"], gw["W2"].ravel(), gw["b2"]])
    return g, loss, parts, dc


@pytest.mark.parametrize("b,h,k,w", [(32, 16, 8, 256), (224, 128, 32, 300), (40, 24, 5, 77)])
def test_line_gradient_matches_oracle(b, h, k, w):
    """Every entry of one line's gradient (tensor-core forward and backward)
    against the oracle's at the same rounding points (bf16 weights, inputs and
    hidden activations), within the componentwise bound of the rounding that
    only the GPU does (dL/dc and dL/dh to bf16, FP32 accumulation).  Widths
    that are not a multiple of the 128-pixel tile check the ragged tile."""
    need_gpu()
    e, q = _encoder(b, h, k, seed=4)
    x = _line(w, b, seed=1)
    shift = x.mean(0).astype(np.float32)
    scale = (1.0 / (x.std(0) + 1e-3)).astype(np.float32)
    e.set_norm(shift, scale)
    target = oracle.run_cube(x[None].astype(np.float64))["delta"][0] * 0.7 + 0.3
    e.reset_stats()
    g_gpu, loss_gpu = e.line_grad(to_dev(x), torch.from_numpy(target).cuda())
    codes = forward_bf16(q, x, shift, scale)
    mu, kk = enc_or.code_stats(codes)       # line 0: the EMA starts from the line's own stats
    g_or, loss, parts, dc = _oracle_line_grad(q, x, shift, scale, mu, kk, target)
    bound = grad_bound(q, parts, dc) + 1e-6 * np.max(np.abs(g_or))
    ratio = np.abs(g_gpu - g_or) / bound
    print(f"{b}x{h}x{k} w={w}: max |dg| / bound {ratio.max():.3f}, "
          f"max rel (|g| > 1e-2 max) {np.max((np.abs(g_gpu - g_or) / np.abs(g_or))[np.abs(g_or) > 1e-2 * np.abs(g_or).max()]):.2e}")
    assert np.all(ratio <= 1.0), (int(np.argmax(ratio)), ratio.max())
    assert abs(loss_gpu - loss) <= 1e-4 * loss
    # line_grad leaves the parameters as they were
    theta = e.params()
    assert np.array_equal(theta[:h * b].reshape(h, b).astype(np.float64) == 0, q["W1"] == 0)


def test_training_steps_match_oracle():
    """Eight training steps on the GPU, each checked against the oracle's step
    from the same parameters: after every GPU step the parameters are read
    back, the oracle computes that line's gradient at the GPU's rounding points
    (bf16 copies of the current weights, the code-space EMA continued line to
    line) and takes its own AdamW step from them.  With AdamW's eps = 1 an
    update is a smooth function of the moments (m / (sqrt(v) + 1), |g| << 1),
    so every parameter may differ from the oracle's prediction by at most lr
    times the bound on the first moment's deviation (the momentum-weighted sum
    of the steps' componentwise gradient bounds) plus the FP32 rounding of the
    master weight; every line's loss agrees to 1e-4."""
    need_gpu()
    from paper_2408_14947_gb300 import erx_train_opts_default
    b, h, k, w, steps = 48, 32, 8, 200, 8
    e, _ = _encoder(b, h, k, seed=6)
    cfg = synth.SceneConfig(bands=b, width=w, seed=3, n_end=(3, 5), noise=0.02)
    cube = synth.gen_lines(cfg, 0, steps)
    flat = cube.reshape(-1, b)
    shift = flat.mean(0).astype(np.float32)
    scale = (1.0 / (flat.std(0) + 1e-3)).astype(np.float32)
    e.set_norm(shift, scale)
    targets = oracle.run_cube(cube.astype(np.float64), warmup=0)["delta"]
    xd, td = to_dev(cube), torch.from_numpy(targets).cuda()
    o = erx_train_opts_default()
    o.lr, o.eps, o.weight_decay, o.momentum = 1e-2, 1.0, 1e-3, 0.2
    b1, b2 = float(np.float32(o.beta1)), float(np.float32(o.beta2))
    n1, n2 = h * b, k * h
    e.reset_stats()
    theta = e.params().astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    dm = np.zeros_like(theta)             # bound on |m_gpu - m_oracle|
    ema = enc_or.CodeEMA(o.momentum)
    worst = []
    for t in range(steps):
        q = {"W1": bf16_round(theta[:n1].reshape(h, b)),
             "b1": theta[n1:n1 + h].astype(np.float32).astype(np.float64),
             "W2": bf16_round(theta[n1 + h:n1 + h + n2].reshape(k, h)),
             "b2": theta[n1 + h + n2:].astype(np.float32).astype(np.float64)}
        codes = forward_bf16(q, cube[t], shift, scale)
        mu_e, k_e = ema.update(codes)
        g, loss, parts, dc = _oracle_line_grad(q, cube[t], shift, scale, mu_e, k_e, targets[t],
                                               o.ridge)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        dm = b1 * dm + (1 - b1) * (grad_bound(q, parts, dc) + 1e-6 * np.max(np.abs(g)))
        c1, c2 = 1 - b1 ** (t + 1), 1 - b2 ** (t + 1)
        pred = theta - o.lr * ((m / c1) / (np.sqrt(v / c2) + o.eps) + o.weight_decay * theta)
        lg = e.train(xd[t:t + 1], td[t:t + 1], o, want_loss=True)[0]
        new = e.params().astype(np.float64)
        tol = o.lr * dm / c1 + 2.0 ** -23 * np.abs(new) + 1e-6 * o.lr
        worst.append(float(np.max(np.abs(new - pred) / tol)))
        assert np.all(np.abs(new - pred) <= tol), (t, int(np.argmax(np.abs(new - pred) / tol)))
        assert abs(lg - loss) <= 1e-4 * loss, (t, lg, loss)
        theta = new
    print(f"{steps} steps: max |dtheta| / tol per step {np.round(worst, 3).tolist()}")


def test_first_training_step_is_adamw():
    """One step from the same weights: AdamW's first move is -lr (g/(|g|+eps) + wd theta),
    so the update's sign pattern follows the gradient's."""
    need_gpu()
    from paper_2408_14947_gb300 import erx_train_opts_default
    b, h, k, w = 32, 16, 8, 256
    e, q = _encoder(b, h, k, seed=5)
    x = _line(w, b, seed=2)
    e.set_norm(np.zeros(b, np.float32), np.ones(b, np.float32))
    target = oracle.run_cube(x[None].astype(np.float64))["delta"][0]
    xd, td = to_dev(x), torch.from_numpy(target).cuda()
    o = erx_train_opts_default()
    o.weight_decay = 0.0
    theta0 = e.params()
    e.reset_stats()
    g, _ = e.line_grad(xd, td, o)
    e.reset_stats()
    e.train(xd[None], td[None], o)
    step = e.params() - theta0
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    want = -o.lr * np.sign(g)
    assert np.allclose(step[big], want[big], rtol=1e-3, atol=1e-7)


def _c5(bands, width, lines, seed):
    """224-band reflectance lines with weak targets: 1 % of pixels in 3 x 3
    clusters are (1 - f) background + f target, f ~ U(0.05, 0.3) (the paper's
    synthetic cube mixes its targets 10 - 50 % with background, Sec. IV-A)."""
    cfg = synth.SceneConfig(bands=bands, width=width, seed=seed, n_end=(3, 5), noise=0.01,
                            scene_lines=2000, drift=0.05, anomaly_frac=0.01, cluster=3,
                            anomaly_mix=(0.05, 0.3))
    return cfg, synth.gen_lines(cfg, 0, lines)


def _spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(float)
    rb = np.argsort(np.argsort(b)).astype(float)
    return np.corrcoef(ra, rb)[0, 1]


def _auc(score, label):
    pos, neg = score[label], score[~label]
    if pos.size == 0:
        return np.nan
    allv = np.concatenate([pos, neg])
    ranks = np.argsort(np.argsort(allv)) + 1.0
    return (ranks[:pos.size].sum() - pos.size * (pos.size + 1) / 2) / (pos.size * neg.size)


@pytest.fixture(scope="module")
def trained():
    """An encoder 224 -> 64 -> 32 trained on 240 lines x 256 px of one stream,
    targets the full-band FP64 ERX scores of the same lines."""
    need_gpu()
    from paper_2408_14947_gb300 import Encoder, erx_train_opts_default
    cfg, cube = _c5(224, 256, 300, seed=7)
    full, _ = run_gpu(cube, form="fp64", warmup=0)
    e = Encoder(224, 64, 32, seed=1)
    flat = cube[:200].reshape(-1, 224)
    e.set_norm(flat.mean(0), 1.0 / (flat.std(0) + 1e-3))
    o = erx_train_opts_default()
    o.lr = 2e-3
    xs = to_dev(cube[:240])
    ts = torch.from_numpy(full["delta"][:240].astype(np.float64)).cuda()
    losses = []
    o.lr = 1e-3
    for epoch in range(5):
        e.reset_stats()
        losses.append(e.train(xs, ts, o, want_loss=True))
    return e, cfg, cube, full, losses


def test_training_reduces_loss(trained):
    e, cfg, cube, full, losses = trained
    first, last = float(np.mean(losses[0][:20])), float(np.mean(losses[-1][-20:]))
    assert last < 0.5 * first, (first, last)


def test_learned_form_matches_oracle_on_codes(trained):
    """The learned form's scores are ERX on the encoder's codes: the oracle run on
    the codes the encoder's forward gives for the same lines (the forward itself
    is checked against the oracle in test_forward_matches_oracle)."""
    e, cfg, cube, full, _ = trained
    from paper_2408_14947_gb300 import Detector
    test = cube[240:260]
    det = Detector(224, 256, in_dtype="f32", form="fp64", encoder=e, warmup=0)
    out = det.push(to_dev(test))
    det.sync()
    codes = e.forward(to_dev(test.reshape(-1, 224))).cpu().numpy().astype(np.float64)
    ref = oracle.run_cube(codes.reshape(len(test), 256, -1), warmup=0)
    assert rel_err(out[0].cpu().numpy(), ref["delta"]) < 1e-9


def test_learned_gains_over_srp_and_full_band(trained):
    """On held-out lines with weak (sub-pixel) targets, ERX on the 32 learned
    codes separates the targets better (per-line AUC) than ERX on a 32-dim
    sparse random projection (the paper's reduction) and than full-band ERX,
    whose 224 noisy bands dilute a weak target."""
    e, cfg, cube, full, _ = trained
    from paper_2408_14947_gb300 import Detector
    det_l = Detector(224, 256, in_dtype="f32", form="fp32", encoder=e, warmup=0)
    det_s = Detector(224, 256, in_dtype="f32", form="fp32", proj="srp", proj_dim=32, seed=5,
                     warmup=0)
    x = to_dev(cube)
    dl = det_l.push(x)[0].cpu().numpy()
    ds = det_s.push(x)[0].cpu().numpy()
    rl = np.mean([_spearman(dl[t], full["delta"][t]) for t in range(240, 300)])
    rs = np.mean([_spearman(ds[t], full["delta"][t]) for t in range(240, 300)])
    labels = synth.anomaly_mask(cfg, 0, 300)

    def line_auc(s):
        return np.nanmean([_auc(s[t], labels[t]) if labels[t].any() else np.nan
                           for t in range(240, 300)])
    auc_f, auc_l, auc_s = line_auc(full["delta"]), line_auc(dl), line_auc(ds)
    print(f"rank corr with full band: learned {rl:.3f} srp32 {rs:.3f}; per-line AUC: "
          f"full {auc_f:.3f} learned {auc_l:.3f} srp32 {auc_s:.3f}")
    assert auc_l > auc_s and auc_l > auc_f


def test_drift_monitor_and_fallback(trained):
    e, cfg, cube, full, _ = trained
    from paper_2408_14947_gb300 import Detector
    x = to_dev(cube[240:300])
    quiet = Detector(224, 256, in_dtype="f32", form="fp64", encoder=e, audit_every=5,
                     min_rank_corr=0.0, warmup=0)
    quiet.push(x)
    quiet.sync()
    last, low, n, fb = quiet.drift()
    assert n == 12 and not fb and -1.0 <= low <= last <= 1.0
    strict = Detector(224, 256, in_dtype="f32", form="fp64", encoder=e, audit_every=5,
                      min_rank_corr=0.9999, warmup=0)
    a = strict.push(x[:10])[0].cpu().numpy()
    b = strict.push(x[10:])[0].cpu().numpy()
    strict.sync()
    last, low, n, fb = strict.drift()
    assert fb
    # after the fallback, scores come from full-band ERX (statistics warmed on audited lines)
    corr = np.mean([_spearman(b[t], full["delta"][250 + t]) for t in range(40, 50)])
    assert corr > 0.99


def test_checkpoint_round_trip(tmp_path):
    """erx_encoder_save / erx_encoder_load: the restored encoder gives the same
    codes bit for bit, and one more training step on each (AdamW moments and
    the code-space EMA restored) gives the same parameters bit for bit."""
    need_gpu()
    from paper_2408_14947_gb300 import Encoder, erx_train_opts_default
    b, h, k, w = 40, 24, 8, 150
    cfg = synth.SceneConfig(bands=b, width=w, seed=8, n_end=(3, 5), noise=0.02)
    cube = synth.gen_lines(cfg, 0, 5)
    targets = torch.from_numpy(oracle.run_cube(cube.astype(np.float64), warmup=0)["delta"]).cuda()
    x = to_dev(cube)
    e = Encoder(b, h, k, seed=2)
    flat = cube.reshape(-1, b)
    e.set_norm(flat.mean(0), 1.0 / (flat.std(0) + 1e-3))
    o = erx_train_opts_default()
    e.train(x[:4], targets[:4], o)
    path = tmp_path / "enc.ckpt"
    e.save(path)
    r = Encoder.load(path)
    assert (r.bands, r.hidden, r.k) == (b, h, k)
    assert np.array_equal(r.params(), e.params())
    assert torch.equal(r.forward(x[4]), e.forward(x[4]))
    la = e.train(x[4:5], targets[4:5], o, want_loss=True)
    lb = r.train(x[4:5], targets[4:5], o, want_loss=True)
    assert np.array_equal(la, lb)
    assert np.array_equal(r.params(), e.params())
    e.close()
    r.close()
