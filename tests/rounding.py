"""Rounding bounds of the tensor-core score forms (test infrastructure; CPU).

The TF32 and BF16 forms score a pixel as m = X r on the tensor cores, with
X = L^{-1} (formed in FP32 from the FP64 factor) and the residual r both
rounded to the operand type, and the products accumulated in FP32.  The first
-order effect of that rounding on delta = ||m|| is bounded per pixel by the
componentwise condition of the product, computed here from the oracle's own
state, so the tests can hold every pixel to a bound derived from the
arithmetic instead of to a tolerance picked by hand.
"""
import numpy as np


def score_condition(cube, **oracle_kw):
    """Componentwise condition of each score under rounding of the score's
    operands: c[t, i] = || |X_t| |r_ti| || / || X_t r_ti ||, with X_t = L_t^{-1}
    the inverse of the oracle's factor of line t and r_ti = z_ti - mu_t.

    A form that rounds both X and r to a unit roundoff u before an exactly
    accumulated product m = X r has |m_err| <= 2u |X||r| componentwise to first
    order, so its relative delta error is at most 2u c[t, i] (the FP32
    accumulation and the FP32 inverse add terms of order 2^-24 c)."""
    import scipy.linalg

    import oracle
    n, p, b = cube.shape
    det = oracle.ERXOracle(b, p, **oracle_kw)
    c = np.empty((n, p))
    for t in range(n):
        z = np.asarray(cube[t], np.float64)
        if det.order == "update_then_score":
            det.push(cube[t])
            mu, k = det.mu, det.k
        else:
            mu_hat = z.mean(axis=0)
            mu, k = (mu_hat, np.cov(z, rowvar=False)) if det.t == 0 else (det.mu, det.k)
            det.push(cube[t])
        low = np.linalg.cholesky(k + det.ridge * np.eye(b))
        x = scipy.linalg.solve_triangular(low, np.eye(b), lower=True)
        r = np.ascontiguousarray(z - mu)               # p x b
        c[t] = (np.linalg.norm(np.abs(r) @ np.abs(x).T, axis=1)
                / np.linalg.norm(r @ x.T, axis=1))
    return c
