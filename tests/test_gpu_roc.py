"""Detection-quality metrics on the GPU (Sec. IV-B) against the oracle: the
quantised-map Mann-Whitney statistic bit for bit, the tau areas to rounding."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle import roc
from tests.gpu_util import need_gpu, run_gpu, torch

pytestmark = pytest.mark.gpu


def _map(seed, n, ties=False):
    r = np.random.default_rng(seed)
    y = r.random(n) < 0.01
    s = r.standard_normal(n) + 2.0 * y
    if ties:
        s = np.round(s * 4) / 4
    return s, y


@pytest.mark.parametrize("bins", [2, 100, 1 << 14, 1 << 16, 1 << 20])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_roc_metrics_match_oracle(bins, dtype):
    need_gpu()
    from paper_2408_14947_gb300 import roc_metrics
    for seed, n, ties in ((0, 100_003, False), (1, 40_000, True), (2, 7, False)):
        s, y = _map(seed, n, ties)
        y[0], y[1] = True, False                          # both classes present
        s = s.astype(dtype)
        got = roc_metrics(torch.from_numpy(s).cuda(), torch.from_numpy(y).cuda(), bins)
        ref = roc.roc_metrics(s.astype(np.float64), y, bins)
        assert got["u2"] == ref["u2"] and got["positives"] == ref["positives"]
        assert got["negatives"] == ref["negatives"] and got["auc"] == ref["auc"]
        for k in ("auc_tpr_tau", "auc_fpr_tau", "auc_td", "auc_bs"):
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-15), k
        if bins >= 1 << 16 and not ties:
            assert abs(got["auc"] - roc.auc_exact(s, y)) <= 2.0 / bins


def test_roc_metrics_rejects_single_class():
    need_gpu()
    from paper_2408_14947_gb300 import ErxError, roc_metrics
    s = torch.rand(100, device="cuda")
    with pytest.raises(ErxError):
        roc_metrics(s, torch.zeros(100, dtype=torch.uint8, device="cuda"))


def test_detection_map_of_erx_scores():
    """delta_N of the FP64 form on a cube with planted 3 x 3 targets: the GPU
    metrics of the map equal the oracle's metrics of the oracle's map to the
    rounding of the scores."""
    need_gpu()
    from paper_2408_14947_gb300 import roc_metrics
    cfg = dataclasses.replace(synth.dn_c2(width=128, bands=32, seed=3), anomaly_frac=0.01)
    cube = synth.gen_lines(cfg, 0, 60)
    lab = synth.anomaly_mask(cfg, 0, 60)
    got, _ = run_gpu(cube, in_bits=12, warmup=5)
    ref = oracle.run_cube(cube, warmup=5)
    g = roc_metrics(torch.from_numpy(got["delta_n"]).cuda(), torch.from_numpy(lab).cuda())
    r = roc.roc_metrics(ref["delta_n"], lab)
    assert g["auc"] == pytest.approx(r["auc"], abs=1e-4)
    assert g["auc_td"] == pytest.approx(r["auc_td"], abs=1e-4)
    assert g["auc_bs"] == pytest.approx(r["auc_bs"], abs=1e-4)
    assert r["auc"] > 0.9
