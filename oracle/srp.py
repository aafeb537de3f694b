"""Sparse random projection matrix of ERX (test infrastructure; oracle side).

Sec. III-B of the paper: the projection W in R^{b x d} has entries
sqrt(s)/sqrt(d) * {+1 w.p. 1/(2s), 0 w.p. 1 - 1/s, -1 w.p. 1/(2s)} with the
sparsity s = sqrt(b), so about d*sqrt(b) entries are non-zero.

The paper draws W with scikit-learn's generator, which cannot be matched bit
for bit, so only the distribution is fixed by the paper.  Both this oracle and
the CUDA library draw W from one counter-based generator, each written from its
published definition: the k-th output (k = 0, 1, ...) of the SplitMix64
generator of Steele, Lea and Flood (OOPSLA 2014) started from ``seed``.  Entry
(i, j) (band i, output dimension j) uses output k = i*d + j, mapped to a
uniform u = (z >> 11) * 2^-53 in [0, 1); u < 1/(2s) gives +1, u < 1/s gives -1,
otherwise 0.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, n: int, start: int = 0) -> list[int]:
    """Outputs start .. start+n-1 of SplitMix64 seeded with ``seed``.

    Output k is mix(seed + (k+1) * gamma mod 2^64): the state advances by the
    golden-ratio increment before each output.
    """
    return [_mix((seed + (k + 1) * _GAMMA) & _MASK) for k in range(start, start + n)]


def srp_weights(bands: int, dim: int, seed: int) -> np.ndarray:
    """The b x d ERX projection matrix (float64), Sec. III-B."""
    s = math.sqrt(bands)
    p_half = 1.0 / (2.0 * s)
    p_nz = 1.0 / s
    mag = math.sqrt(s) / math.sqrt(dim)
    out = np.zeros((bands, dim), dtype=np.float64)
    z = splitmix64_stream(seed, bands * dim)
    for i in range(bands):
        for j in range(dim):
            u = (z[i * dim + j] >> 11) * 2.0 ** -53
            if u < p_half:
                out[i, j] = mag
            elif u < p_nz:
                out[i, j] = -mag
    return out
