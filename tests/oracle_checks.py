"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each check returns the largest discrepancy it sees, so the same checks can run
against the oracle as written (tests/test_oracle_pins.py) and against copies of
it with a planted mistake (tests/test_oracle_mutations.py), where at least one
check must then fail.
"""
import json
import math
import os
from fractions import Fraction as F

import numpy as np
import scipy.spatial.distance

import oracle
from oracle import erx_oracle as eo

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _cube(seed, t, w, b, scale=1.0):
    r = np.random.default_rng(seed)
    base = r.standard_normal((b, b)) / math.sqrt(b)
    return np.stack([(r.standard_normal((w, b)) @ base + 3.0) * scale for _ in range(t)])


def check_exact_golden():
    """Oracle delta^2 vs exact rationals (Sec. III-C/III-D) on tiny integer cubes."""
    with open(os.path.join(GOLDEN, "erx_exact_tiny.json")) as f:
        cases = json.load(f)["cases"]
    worst = 0.0
    for c in cases:
        cube = np.array(c["cube"], dtype=np.float64)
        proj = None if c["proj"] is None else np.array(
            [[float(F(v)) for v in row] for row in c["proj"]])
        res = eo.run_cube(cube, momentum=float(F(c["alpha"])), ridge=float(F(c["ridge"])),
                          proj="none" if proj is None else proj, order=c["order"])
        exact = np.array([[float(F(v)) for v in line] for line in c["delta2"]])
        worst = max(worst, rel(res["delta"] ** 2, exact))
        t, mu, k = res["state"]
        worst = max(worst, rel(mu, [float(F(v)) for v in c["final_mu"]]))
        worst = max(worst, rel(k, [[float(F(v)) for v in row] for row in c["final_K"]]))
    return worst


def check_hand_1d():
    """Worked by hand: one band, line (0, 1, 2): mean 1, covariance 1/(3-1)*(1+0+1) = 1,
    so delta = (1, 0, 1)/sqrt(1+eps) and delta_N = (1, -2, 1)/sqrt(2)."""
    eps = 1e-5
    out = eo.ERXOracle(1, 3, ridge=eps).push(np.array([[0.0], [1.0], [2.0]]))
    want = np.array([1.0, 0.0, 1.0]) / math.sqrt(1.0 + eps)
    want_n = np.array([1.0, -2.0, 1.0]) / math.sqrt(2.0)
    return max(float(np.max(np.abs(out["delta"] - want))),
               float(np.max(np.abs(out["delta_n"] - want_n))))


def check_closed_form_ema(alpha=0.1, t=12):
    """Sec. III-C recursion vs its solution: mu_T = (1-a)^(T-1) mu_hat_0 +
    sum_{j>=1} a (1-a)^(T-1-j) mu_hat_j, same weights for K (with np.mean / np.cov)."""
    cube = _cube(1, t, 9, 4)
    det = eo.ERXOracle(4, 9, momentum=alpha)
    for line in cube:
        det.push(line)
    wts = [(1 - alpha) ** (t - 1)] + [alpha * (1 - alpha) ** (t - 1 - j) for j in range(1, t)]
    mu = sum(w * line.mean(axis=0) for w, line in zip(wts, cube))
    k = sum(w * np.cov(line.T, ddof=1) for w, line in zip(wts, cube))
    return max(rel(det.mu, mu), rel(det.k, k), abs(sum(wts) - 1.0))


def check_alpha1_trace(order="update_then_score"):
    """alpha = 1 is RX on the current line (Sec. IV-C): sum_i delta_i^2 =
    (p-1) * sum_k lam_k / (lam_k + eps), lam = eig of the 1/(p-1) line covariance."""
    eps = 1e-3
    cube = _cube(2, 3, 11, 5)
    det = eo.ERXOracle(5, 11, momentum=1.0, ridge=eps, order=order)
    worst = 0.0
    for line in cube:
        out = det.push(line)
        lam = np.linalg.eigvalsh(np.cov(line.T, ddof=1))
        want = (11 - 1) * float(np.sum(lam / (lam + eps)))
        worst = max(worst, abs(float(np.sum(out["delta"] ** 2)) - want) / want)
    return worst


def check_textbook_rx():
    """alpha = 1, no ridge: delta equals the textbook Mahalanobis distance of each pixel
    to the line's own mean under the line's 1/(p-1) covariance (Sec. II-A form)."""
    cube = _cube(3, 2, 13, 4)
    det = eo.ERXOracle(4, 13, momentum=1.0, ridge=0.0)
    worst = 0.0
    for line in cube:
        out = det.push(line)
        vi = np.linalg.inv(np.cov(line.T, ddof=1))
        mu = line.mean(axis=0)
        want = np.array([scipy.spatial.distance.mahalanobis(x, mu, vi) for x in line])
        worst = max(worst, rel(out["delta"], want))
    return worst


def check_brute_inverse(order="update_then_score"):
    """delta_i^2 = r_i^T (K_t + eps I)^{-1} r_i with an explicit inverse (Sec. III-D)."""
    eps = 1e-5
    cube = _cube(4, 6, 10, 4, 0.01)
    det = eo.ERXOracle(4, 10, momentum=0.3, ridge=eps, order=order)
    worst = 0.0
    prev = None
    for t, line in enumerate(cube):
        mu_h = line.mean(axis=0)
        k_h = np.cov(line.T, ddof=1)
        if order == "update_then_score":
            cur = (mu_h, k_h) if prev is None else (0.7 * prev[0] + 0.3 * mu_h,
                                                    0.7 * prev[1] + 0.3 * k_h)
            use = cur
        else:
            use = (mu_h, k_h) if prev is None else prev
            cur = (mu_h, k_h) if prev is None else (0.7 * prev[0] + 0.3 * mu_h,
                                                    0.7 * prev[1] + 0.3 * k_h)
        out = det.push(line)
        inv = np.linalg.inv(use[1] + eps * np.eye(4))
        r = line - use[0]
        want = np.einsum("ij,jk,ik->i", r, inv, r)
        worst = max(worst, rel(out["delta"] ** 2, want))
        prev = cur
    return worst


def check_orthogonal_invariance():
    """x -> A x + c with A orthogonal leaves delta unchanged, ridge included."""
    b = 6
    cube = _cube(5, 5, 14, b)
    q, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((b, b)))
    c = np.arange(b, dtype=float)
    r1 = eo.run_cube(cube, momentum=0.2, ridge=1e-2)
    r2 = eo.run_cube(cube @ q.T + c, momentum=0.2, ridge=1e-2)
    return max(rel(r1["delta"], r2["delta"]), float(np.max(np.abs(r1["delta_n"] - r2["delta_n"]))))


def check_scale_invariance():
    """x -> g x with eps -> g^2 eps leaves delta unchanged."""
    cube = _cube(6, 4, 12, 5)
    g = 37.0
    r1 = eo.run_cube(cube, momentum=0.1, ridge=1e-3)
    r2 = eo.run_cube(cube * g, momentum=0.1, ridge=1e-3 * g * g)
    return rel(r1["delta"], r2["delta"])


def check_permutation():
    """Permuting the pixels of every line permutes delta the same way."""
    cube = _cube(7, 4, 15, 4)
    perm = np.random.default_rng(3).permutation(15)
    r1 = eo.run_cube(cube)
    r2 = eo.run_cube(cube[:, perm, :])
    return rel(r1["delta"][:, perm], r2["delta"])


def check_normalisation():
    """Sec. III-E: delta_N has mean 0 and population variance 1 per line."""
    cube = _cube(8, 5, 31, 3)
    r = eo.run_cube(cube)
    dn = r["delta_n"]
    return max(float(np.max(np.abs(dn.mean(axis=1)))),
               float(np.max(np.abs((dn ** 2).mean(axis=1) - 1.0))))


def check_stationary():
    """Identical lines: K_t = K_hat and mu_t = mu_hat for every t (weights sum to 1)."""
    line = _cube(9, 1, 10, 3)[0]
    det = eo.ERXOracle(3, 10, momentum=0.25)
    outs = [det.push(line)["delta"] for _ in range(6)]
    return max(rel(det.k, np.cov(line.T, ddof=1)), rel(det.mu, line.mean(axis=0)),
               max(rel(o, outs[0]) for o in outs))


def check_score_then_update_alpha1():
    """alpha = 1, score-then-update: line t (t >= 1) is scored against line t-1's
    statistics; line 0 against its own."""
    eps = 1e-4
    cube = _cube(10, 4, 9, 3)
    det = eo.ERXOracle(3, 9, momentum=1.0, ridge=eps, order="score_then_update")
    worst = 0.0
    for t, line in enumerate(cube):
        out = det.push(line)
        ref = cube[t - 1] if t else line
        vi = np.linalg.inv(np.cov(ref.T, ddof=1) + eps * np.eye(3))
        r = line - ref.mean(axis=0)
        worst = max(worst, rel(out["delta"] ** 2, np.einsum("ij,jk,ik->i", r, vi, r)))
    return worst


def check_srp_projection():
    """SRP makes Z = X W (Sec. III-B): run with the drawn W equals running on X @ W."""
    b, d, seed = 20, 4, 5
    w = oracle.srp_weights(b, d, seed)
    cube = _cube(11, 3, 16, b)
    r1 = eo.run_cube(cube, proj="srp", proj_dim=d, seed=seed, ridge=1e-3)
    r2 = eo.run_cube(cube @ w, ridge=1e-3)
    return rel(r1["delta"], r2["delta"])


def check_imc_pooled(order="update_then_score"):
    """IMC (Sec. IV-C) weighs every pixel seen so far equally: after line t the
    state is the mean and the 1/(n-1) covariance (numpy.cov) of all pixels of
    lines 0..t, and each line is scored (textbook RX, explicit inverse) against
    the pooled statistics of the lines its order prescribes."""
    p, b, T, ridge = 9, 4, 7, 1e-3
    r = np.random.default_rng(21)
    # lines with different means, so the between-line term of the pooled covariance matters
    cube = np.stack([r.standard_normal((p, b)) + 3.0 * r.standard_normal(b) for _ in range(T)])
    det = eo.ERXOracle(b, p, averaging="imc", ridge=ridge, order=order)
    worst = 0.0
    for t in range(T):
        out = det.push(cube[t])
        seen = cube[: t + 1].reshape(-1, b)
        worst = max(worst, rel(det.mu, seen.mean(axis=0)))
        worst = max(worst, rel(det.k, np.cov(seen.T, ddof=1)))
        ref = cube[: t + 1] if (order == "update_then_score" or t == 0) else cube[:t]
        ref = ref.reshape(-1, b)
        vi = np.linalg.inv(np.cov(ref.T, ddof=1) + ridge * np.eye(b))
        mu = ref.mean(axis=0)
        want = [scipy.spatial.distance.mahalanobis(x, mu, vi) for x in cube[t]]
        worst = max(worst, rel(out["delta"], want))
    return worst


def check_pooled_warmup(alpha=0.2, warmup=5, extra=4):
    """The pooled reading of the warm-up buffer: after the warm-up lines the
    state is their pooled mean and 1/(n-1) covariance (numpy.cov of all their
    pixels); after k more lines it is the closed form of the EMA started from
    there, mu = (1-a)^k mu_pool + sum_j a (1-a)^(k-1-j) mu_hat_j (same for K)."""
    p, b = 8, 3
    r = np.random.default_rng(33)
    cube = np.stack([r.standard_normal((p, b)) + 2.0 * r.standard_normal(b)
                     for _ in range(warmup + extra)])
    det = eo.ERXOracle(b, p, momentum=alpha, averaging="pooled", warmup=warmup, ridge=1e-3)
    for t in range(warmup):
        det.push(cube[t])
    pool = cube[:warmup].reshape(-1, b)
    worst = max(rel(det.mu, pool.mean(axis=0)), rel(det.k, np.cov(pool.T, ddof=1)))
    for t in range(warmup, warmup + extra):
        det.push(cube[t])
    k = extra
    mu = (1 - alpha) ** k * pool.mean(axis=0)
    kk = (1 - alpha) ** k * np.cov(pool.T, ddof=1)
    for j in range(k):
        z = cube[warmup + j]
        w = alpha * (1 - alpha) ** (k - 1 - j)
        mu = mu + w * z.mean(axis=0)
        kk = kk + w * np.cov(z.T, ddof=1)
    return max(worst, rel(det.mu, mu), rel(det.k, kk))


ALL_CHECKS = {
    "exact_golden": (check_exact_golden, 1e-11),
    "hand_1d": (check_hand_1d, 1e-14),
    "closed_form_ema": (check_closed_form_ema, 1e-12),
    "alpha1_trace": (check_alpha1_trace, 1e-10),
    "textbook_rx": (check_textbook_rx, 1e-9),
    "brute_inverse": (check_brute_inverse, 1e-9),
    "brute_inverse_stu": (lambda: check_brute_inverse("score_then_update"), 1e-9),
    "orthogonal_invariance": (check_orthogonal_invariance, 1e-9),
    "scale_invariance": (check_scale_invariance, 1e-9),
    "permutation": (check_permutation, 1e-12),
    "normalisation": (check_normalisation, 1e-12),
    "stationary": (check_stationary, 1e-12),
    "score_then_update_alpha1": (check_score_then_update_alpha1, 1e-9),
    "srp_projection": (check_srp_projection, 1e-9),
    "imc_pooled": (check_imc_pooled, 1e-9),
    "imc_pooled_stu": (lambda: check_imc_pooled("score_then_update"), 1e-9),
    "pooled_warmup": (check_pooled_warmup, 1e-11),
}
