"""The rank agreement a k-dimensional code can have with full-band RX (CPU).

For a Gaussian background in B bands, the full-band RX score is delta^2 =
||y||^2 with y the whitened residual, a sum of B independent squared unit
normals.  RX on any full-rank linear code c = A x (A: k x B) whitens the code
with its own covariance A K A^T, so delta_c^2 = ||P y||^2 with P the
orthogonal projector onto a k-dimensional subspace: k of the same B squared
components in a rotated basis.  Hence cov(delta_c^2, delta^2) = 2k,
var(delta^2) = 2B, var(delta_c^2) = 2k, and the correlation is sqrt(k / B)
for every such code -- a sparse random projection included.  At k = 32 of
B = 224 that is 0.378: where white noise dominates the background scores, no
linear 32-dimensional code can rank background pixels as full-band RX does,
and a nonlinear one has to reproduce the norm of the 192 dimensions it drops.
"""
import numpy as np
import pytest


@pytest.mark.parametrize("code", ["subspace", "srp"])
def test_linear_code_rank_agreement_is_sqrt_k_over_b(code):
    B, k, n = 224, 32, 200_000
    r = np.random.default_rng(7)
    q, _ = np.linalg.qr(r.standard_normal((B, B)))
    lam = np.logspace(0, 3, B)
    x = (r.standard_normal((n, B)) * np.sqrt(lam)) @ q.T          # covariance Q diag(lam) Q^T
    cov = (q * lam) @ q.T
    full = np.einsum("ij,ij->i", x @ np.linalg.inv(cov), x)        # delta^2, population stats
    if code == "subspace":
        a = r.standard_normal((k, B))
    else:                                                           # sparse random projection
        s = np.sqrt(B)
        u = r.random((k, B))
        a = np.where(u < 1 / (2 * s), 1.0, np.where(u < 1 / s, -1.0, 0.0)) * np.sqrt(s / k)
    c = x @ a.T
    cc = a @ cov @ a.T
    red = np.einsum("ij,ij->i", c @ np.linalg.inv(cc), c)
    pearson = np.corrcoef(red, full)[0, 1]
    assert abs(pearson - np.sqrt(k / B)) < 0.01, pearson
    rank = np.corrcoef(np.argsort(np.argsort(red)), np.argsort(np.argsort(full)))[0, 1]
    assert abs(rank - np.sqrt(k / B)) < 0.03, rank
