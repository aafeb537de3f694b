"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import erx_oracle as eo
from tests import oracle_checks as oc


@pytest.mark.parametrize("name", sorted(oc.ALL_CHECKS))
def test_pin(name):
    fn, tol = oc.ALL_CHECKS[name]
    err = fn()
    assert err <= tol, f"{name}: {err} > {tol}"


def test_alpha1_trace_fails_under_score_then_update():
    # the identity is specific to scoring a line with its own statistics (Sec. IV-C)
    assert oc.check_alpha1_trace("score_then_update") > 1e-3


def test_splitmix64_published_vectors():
    with open(os.path.join(oc.GOLDEN, "splitmix64.json")) as f:
        g = json.load(f)
    for s in g["streams"]:
        got = oracle.splitmix64_stream(s["seed"], len(s["outputs"]))
        assert [str(v) for v in got] == s["outputs"]


def test_srp_distribution():
    """Sec. III-B: entries +-sqrt(s/d) with probability 1/(2s) each, s = sqrt(b);
    about d*sqrt(b) non-zeros."""
    b, d = 108, 5
    s = math.sqrt(b)
    mag = math.sqrt(s / d)
    nnz, pos, n_seeds = 0, 0, 400
    for seed in range(n_seeds):
        w = oracle.srp_weights(b, d, seed)
        nz = w[w != 0]
        assert np.allclose(np.abs(nz), mag, rtol=0, atol=1e-15)
        nnz += nz.size
        pos += int(np.sum(nz > 0))
    n = b * d * n_seeds
    p = 1 / s
    mean, sd = n * p, math.sqrt(n * p * (1 - p))
    assert abs(nnz - mean) < 4 * sd                       # ~ d sqrt(b) per matrix
    assert abs(nnz / n_seeds - d * math.sqrt(b)) < 1.0
    assert abs(pos - nnz / 2) < 4 * math.sqrt(nnz / 4)    # signs balanced


def test_srp_preserves_norm_in_expectation():
    """E ||W^T x||^2 = ||x||^2 for the Sec. III-B distribution."""
    b, d = 64, 8
    x = np.random.default_rng(0).standard_normal(b)
    vals = [np.sum((x @ oracle.srp_weights(b, d, seed)) ** 2) for seed in range(600)]
    m = float(np.mean(vals))
    se = float(np.std(vals)) / math.sqrt(len(vals))
    assert abs(m - x @ x) < 4 * se


def test_warmup_flag_and_mask():
    cube = oc._cube(12, 120, 6, 2)
    r = eo.run_cube(cube, warmup=99, threshold=1.0)
    assert not r["detecting"][:99].any() and r["detecting"][99:].all()
    assert np.array_equal(r["mask"], r["delta_n"] >= 1.0)


def test_normalise_zero_spread():
    assert np.array_equal(eo.normalise(np.full(7, 2.5)), np.zeros(7))


def test_invalid_configs():
    with pytest.raises(ValueError):
        eo.ERXOracle(3, 1)
    with pytest.raises(ValueError):
        eo.ERXOracle(3, 5, momentum=0.0)
    with pytest.raises(ValueError):
        eo.ERXOracle(3, 5, momentum=1.5)
