"""Synthetic cube generators: seeded, line-addressable, shaped like the workloads."""
import numpy as np

import synth


def test_line_addressable():
    for cfg in (synth.reflectance_c1(width=32, bands=8), synth.dn_c2(width=40, bands=12),
                synth.cov_c3(1e3, width=24, bands=10)):
        full = synth.gen_lines(cfg, 0, 9)
        part = synth.gen_lines(cfg, 4, 5)
        assert np.array_equal(full[4:], part)
        assert np.array_equal(synth.anomaly_mask(cfg, 0, 9)[4:], synth.anomaly_mask(cfg, 4, 5))


def test_dtypes_and_ranges():
    x = synth.gen_lines(synth.dn_c2(width=64, bands=16), 0, 4)
    assert x.dtype == np.uint16 and x.max() <= 4095
    y = synth.gen_lines(synth.reflectance_c1(width=64, bands=16), 0, 4)
    assert y.dtype == np.float32 and 0.0 <= y.min() and y.max() <= 1.0


def test_anomaly_fraction():
    cfg = synth.dn_c2(width=640, bands=8)
    m = synth.anomaly_mask(cfg, 0, 3000)
    assert 0.001 < m.mean() < 0.004


def test_c4_streams():
    cfgs = synth.stream_configs_c4(32)
    assert len(cfgs) == 32
    assert all(128 <= c.width <= 2048 and c.bands in (8, 16, 64, 108, 224) for c in cfgs)


def test_cov_condition():
    cfg = synth.cov_c3(1e4, width=2048, bands=6)
    x = synth.gen_lines(cfg, 0, 1)[0].astype(np.float64)
    lam = np.linalg.eigvalsh(np.cov(x.T))
    assert 2e3 < lam.max() / lam.min() < 5e4
