"""Exact rational ERX on tiny inputs (test infrastructure only).

Same steps as the FP64 oracle (Sec. III-B..D of the paper) in
``fractions.Fraction`` arithmetic, so that squared Mahalanobis distances, which
are rational in the data, alpha and the ridge, come out exactly.  The squared
distance is obtained without a Cholesky factor (whose square roots are
irrational): delta_i^2 = r_i^T (K_t + eps I)^{-1} r_i with the linear system
solved by exact Gauss-Jordan elimination, which equals m_i . m_i for
L m_i = r_i since L L^T = K_t + eps I.
"""
from __future__ import annotations

from fractions import Fraction as F


def _mean(z):
    p, d = len(z), len(z[0])
    return [sum(z[i][j] for i in range(p)) / p for j in range(d)]


def _cov(z, mu):
    p, d = len(z), len(z[0])
    return [[sum((z[i][a] - mu[a]) * (z[i][b] - mu[b]) for i in range(p)) / (p - 1)
             for b in range(d)] for a in range(d)]


def _solve(a, b):
    """Exact solution x of a x = b (a nonsingular) by Gauss-Jordan elimination."""
    n = len(a)
    m = [list(a[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if m[r][c] != 0)
        m[c], m[piv] = m[piv], m[c]
        inv = 1 / m[c][c]
        m[c] = [v * inv for v in m[c]]
        for r in range(n):
            if r != c and m[r][c] != 0:
                f = m[r][c]
                m[r] = [vr - f * vc for vr, vc in zip(m[r], m[c])]
    return [m[i][n] for i in range(n)]


def erx_exact(cube, alpha=F(1, 10), ridge=F(1, 100000), w=None,
              order="update_then_score"):
    """Exact delta^2 for every pixel of every line of a tiny integer/rational cube.

    cube: nested lists [line][pixel][band] of ints or Fractions.
    w: optional projection matrix [band][dim] of Fractions (None: all bands).
    Returns ([line][pixel] delta^2 as Fraction, final (mu, K)).
    """
    alpha, ridge = F(alpha), F(ridge)
    mu = k = None
    out = []
    for t, line in enumerate(cube):
        z = [[F(v) for v in px] for px in line]
        if w is not None:
            z = [[sum(px[i] * w[i][j] for i in range(len(px))) for j in range(len(w[0]))]
                 for px in z]
        mu_h = _mean(z)
        k_h = _cov(z, mu_h)
        d = len(mu_h)
        if order == "update_then_score":
            if t == 0:
                mu, k = mu_h, k_h
            else:
                mu = [(1 - alpha) * a + alpha * b for a, b in zip(mu, mu_h)]
                k = [[(1 - alpha) * k[i][j] + alpha * k_h[i][j] for j in range(d)]
                     for i in range(d)]
            mu_s, k_s = mu, k
        else:
            mu_s, k_s = (mu_h, k_h) if t == 0 else (mu, k)
        a = [[k_s[i][j] + (ridge if i == j else 0) for j in range(d)] for i in range(d)]
        d2 = []
        for px in z:
            r = [px[j] - mu_s[j] for j in range(d)]
            x = _solve(a, r)
            d2.append(sum(ri * xi for ri, xi in zip(r, x)))
        out.append(d2)
        if order == "score_then_update":
            if t == 0:
                mu, k = mu_h, k_h
            else:
                mu = [(1 - alpha) * a_ + alpha * b_ for a_, b_ in zip(mu, mu_h)]
                k = [[(1 - alpha) * k[i][j] + alpha * k_h[i][j] for j in range(d)]
                     for i in range(d)]
    return out, (mu, k)
