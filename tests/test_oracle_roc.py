"""Pins of the detection-quality oracle (Sec. IV-B metrics), CPU only."""
import numpy as np
import pytest

from oracle import roc


def _brute_auc(s, y):
    """P(anomaly scores above background) + 1/2 P(equal), by counting all pairs."""
    p, n = s[y], s[~y]
    gt = (p[:, None] > n[None, :]).sum()
    eq = (p[:, None] == n[None, :]).sum()
    return (gt + 0.5 * eq) / (len(p) * len(n))


def _case(seed, n=300, levels=None):
    r = np.random.default_rng(seed)
    y = r.random(n) < 0.2
    s = r.standard_normal(n) + 1.5 * y
    if levels:
        s = np.round((s - s.min()) / (s.max() - s.min()) * levels)   # integer scores, ties
    return s, y


@pytest.mark.parametrize("seed", range(4))
def test_exact_auc_is_pairwise_count(seed):
    s, y = _case(seed, levels=20)
    assert roc.auc_exact(s, y) == pytest.approx(_brute_auc(s, y), abs=1e-15)


@pytest.mark.parametrize("levels", [5, 37, 200])
def test_binned_auc_equals_pairwise_when_levels_are_distinct(levels):
    # integer scores 0..L with bins = L + 1: distinct scores never share a level
    s, y = _case(levels, n=500, levels=levels)
    u2, n_p, n_n = roc.auc_binned(s, y, int(s.max()) + 1)
    assert u2 / (2.0 * n_p * n_n) == pytest.approx(_brute_auc(s, y), abs=1e-15)


def test_binned_auc_converges_to_exact():
    s, y = _case(9, n=2000)
    ex = roc.auc_exact(s, y)
    for bins in (1 << 8, 1 << 12, 1 << 16):
        u2, n_p, n_n = roc.auc_binned(s, y, bins)
        assert abs(u2 / (2.0 * n_p * n_n) - ex) <= 2.0 / bins


def test_tau_areas_are_integrals_of_tpr_and_fpr():
    s, y = _case(3, n=400)
    m = roc.roc_metrics(s, y)
    v = roc.normalised(s)
    tau = np.linspace(0.0, 1.0, 200001)
    tpr = np.array([(v[y] >= t).mean() for t in tau[::100]])   # coarse curve for speed
    fpr = np.array([(v[~y] >= t).mean() for t in tau[::100]])
    grid = tau[::100]
    assert np.trapezoid(tpr, grid) == pytest.approx(m["auc_tpr_tau"], abs=2e-3)
    assert np.trapezoid(fpr, grid) == pytest.approx(m["auc_fpr_tau"], abs=2e-3)
    assert m["auc_td"] == pytest.approx((m["auc"] + m["auc_tpr_tau"]) / 2)
    assert m["auc_bs"] == pytest.approx((m["auc"] - m["auc_fpr_tau"] + 1) / 2)


def test_special_cases():
    y = np.array([0, 0, 1, 1, 0, 1], bool)
    sep = np.where(y, 2.0, 1.0) + np.arange(6) * 1e-3
    assert roc.roc_metrics(sep, y)["auc"] == 1.0
    assert roc.roc_metrics(-sep, y)["auc"] == 0.0
    const = roc.roc_metrics(np.ones(6), y)
    assert const["auc"] == 0.5 and const["auc_tpr_tau"] == 0.0 and const["auc_fpr_tau"] == 0.0


def test_matches_library_roc_auc():
    sk = pytest.importorskip("sklearn.metrics")
    s, y = _case(5, n=1000, levels=50)
    assert roc.auc_exact(s, y) == pytest.approx(sk.roc_auc_score(y, s), abs=1e-14)
