"""Synthetic hyperspectral line-scan cubes, addressable line by line.

Every line ``t`` of stream ``s`` is drawn from ``numpy.random.default_rng([seed,
s, tag, t])`` and every scene-level quantity from ``default_rng([seed, s, tag,
scene])``, so any line range can be regenerated without the lines before it.
Cubes are laid out ``[line][pixel][band]`` (band-interleaved-by-pixel), the
layout in which a line-scan camera delivers a line of ``p`` pixels by ``b``
bands (Sec. III-B of the paper: ``X_t`` in R^{p x b}).

The paper evaluates on three real cubes (Sec. IV-A: a 452 px x 3072 line x
108 band beach scene, a 600 x 2400 x 90 AVIRIS-derived scene and a 1116 x 2499
x 13 Sentinel-2 scene) that are not distributed with it; these generators stand
in for them with the same shapes and the same structure: a few material
spectra per scene, scene changes along track, sensor noise, and small anomalous
targets.  The speed tests of Sec. IV-C use uniformly random cubes
(``random_uniform_cube``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_TAG_SCENE = 11
_TAG_LINE = 12
_TAG_CLUSTER = 13
_TAG_STREAM = 14


def _smooth_spectra(rng: np.random.Generator, n: int, bands: int,
                    lo: float = 0.05, hi: float = 0.95) -> np.ndarray:
    """n smooth spectra over ``bands`` bands with values in [lo, hi]."""
    x = np.linspace(0.0, 1.0, bands)
    out = np.empty((n, bands))
    for k in range(n):
        s = rng.uniform(-0.3, 0.3) * x
        for _ in range(4):
            c, w, a = rng.uniform(0, 1), rng.uniform(0.05, 0.3), rng.uniform(-1, 1)
            s = s + a * np.exp(-0.5 * ((x - c) / w) ** 2)
        s = s - s.min()
        s = s / max(s.max(), 1e-12)
        base = rng.uniform(lo, hi)
        amp = rng.uniform(0.2, 0.6) * min(base - lo, hi - base) * 2
        out[k] = np.clip(base - amp / 2 + amp * s, lo, hi)
    return out


@dataclass(frozen=True)
class SceneConfig:
    """Mixture-of-materials background with scene switches and drift.

    Each pixel takes one of ``n_end`` material spectra of the current scene
    (weights from a Dirichlet draw, or ``weights`` when given) plus Gaussian
    noise of std ``noise`` per band.  Material spectra drift linearly by up to
    ``drift`` (reflectance units) per ``drift_lines`` lines.  Anomalies are
    ``cluster`` x ``cluster`` blocks (pixels x lines) carrying a scene-specific
    distinct spectrum, placed so that about ``anomaly_frac`` of all pixels are
    anomalous.  ``dn_max`` > 0 turns reflectance into integer digital numbers
    ``round(dn_max * r)`` stored as uint16; otherwise float32 reflectance.
    """
    bands: int
    width: int
    seed: int = 0
    stream: int = 0
    n_end: tuple = (3, 3)
    weights: tuple | None = None
    noise: float = 0.01
    scene_lines: int = 0          # 0: one scene for the whole cube
    drift: float = 0.05
    drift_lines: int = 1000
    anomaly_frac: float = 0.005
    cluster: int = 1
    dn_max: int = 0
    scale: float = 1.0            # multiplies reflectance before storage (f32 only)
    anomaly_mix: tuple | None = None  # (lo, hi): anomalies are (1-f) background + f target,
                                      # f ~ U(lo, hi) per pixel (weak, sub-pixel targets)

    @property
    def dtype(self):
        return np.uint16 if self.dn_max > 0 else np.float32

    def scene_of(self, t: int) -> int:
        return 0 if self.scene_lines <= 0 else t // self.scene_lines


@dataclass(frozen=True)
class CovSceneConfig:
    """Gaussian background with a prescribed covariance spectrum.

    Pixels are ``mu + Q diag(sqrt(lam)) g`` with ``g ~ N(0, I)``, ``Q`` a seeded
    random orthogonal matrix and ``lam`` log-spaced from ``lam_min`` to
    ``lam_min * kappa``; the background covariance has condition number
    ``kappa``.  Anomalies are 3 x 3 clusters offset by ``anomaly_sigma``
    standard deviations along a seeded direction.
    """
    bands: int
    width: int
    kappa: float = 1e2
    lam_min: float = 1e-3
    seed: int = 0
    stream: int = 0
    scene_lines: int = 0
    anomaly_frac: float = 0.002
    anomaly_sigma: float = 8.0
    cluster: int = 3

    dtype = np.float32

    def scene_of(self, t: int) -> int:
        return 0 if self.scene_lines <= 0 else t // self.scene_lines


# ---------------------------------------------------------------- presets

def reflectance_c1(seed: int = 0, width: int = 256, bands: int = 64) -> SceneConfig:
    """1000 x 256 x 64 float32 reflectance, 3 materials, 0.5 % single-pixel anomalies."""
    return SceneConfig(bands=bands, width=width, seed=seed, n_end=(3, 3),
                       weights=(0.5, 0.3, 0.2), noise=0.01, scene_lines=0,
                       drift=0.05, drift_lines=1000, anomaly_frac=0.005, cluster=1)


def dn_c2(seed: int = 0, width: int = 640, bands: int = 108) -> SceneConfig:
    """20000 x 640 x 108 uint16 12-bit DN, scenes of 3-5 materials switching every
    2000 lines, 0.2 % anomalies in 3 x 3 clusters."""
    return SceneConfig(bands=bands, width=width, seed=seed, n_end=(3, 5), noise=0.01,
                       scene_lines=2000, drift=0.02, drift_lines=1000,
                       anomaly_frac=0.002, cluster=3, dn_max=4095)


def cov_c3(kappa: float, seed: int = 0, width: int = 1024, bands: int = 224) -> CovSceneConfig:
    """1024 x 224 float32 Gaussian background with covariance condition number kappa."""
    return CovSceneConfig(bands=bands, width=width, kappa=kappa, seed=seed)


def stream_configs_c4(n_streams: int = 256, seed: int = 0,
                      widths=(128, 2048), band_choices=(8, 16, 64, 108, 224)):
    """Heterogeneous streams: widths uniform in [128, 2048], bands from the set,
    drift rate uniform in [0, 0.1] per 1000 lines, float32 reflectance."""
    out = []
    for s in range(n_streams):
        r = np.random.default_rng([seed, s, _TAG_STREAM])
        w = int(r.integers(widths[0], widths[1] + 1))
        b = int(r.choice(band_choices))
        drift = float(r.uniform(0.0, 0.1))
        out.append(SceneConfig(bands=b, width=w, seed=seed, stream=s, n_end=(3, 5),
                               noise=0.01, scene_lines=2000, drift=drift,
                               drift_lines=1000, anomaly_frac=0.002, cluster=3))
    return out


def random_uniform_cube(lines: int, width: int, bands: int, seed: int = 0) -> np.ndarray:
    """Uniform random float32 cube (the speed-test input of Sec. IV-C)."""
    out = np.empty((lines, width, bands), np.float32)
    for t in range(lines):
        out[t] = np.random.default_rng([seed, 0, _TAG_LINE, t]).random((width, bands), np.float32)
    return out


# ---------------------------------------------------------------- scenes

def _scene_mix(cfg: SceneConfig, scene: int):
    r = np.random.default_rng([cfg.seed, cfg.stream, _TAG_SCENE, scene])
    n = int(r.integers(cfg.n_end[0], cfg.n_end[1] + 1))
    ends = _smooth_spectra(r, n, cfg.bands)
    direction = _smooth_spectra(r, n, cfg.bands, 0.0, 1.0) * 2.0 - 1.0
    if cfg.weights is not None and len(cfg.weights) == n:
        w = np.asarray(cfg.weights, float)
    else:
        w = r.dirichlet(np.full(n, 2.0))
    anom = _smooth_spectra(r, 1, cfg.bands)[0]
    return ends, direction, w / w.sum(), anom


def _scene_cov(cfg: CovSceneConfig, scene: int):
    r = np.random.default_rng([cfg.seed, cfg.stream, _TAG_SCENE, scene])
    mu = _smooth_spectra(r, 1, cfg.bands)[0]
    q, rr = np.linalg.qr(r.standard_normal((cfg.bands, cfg.bands)))
    q = q * np.sign(np.diag(rr))
    lam = cfg.lam_min * np.logspace(0.0, np.log10(cfg.kappa), cfg.bands)
    v = r.standard_normal(cfg.bands)
    v /= np.linalg.norm(v)
    anom = mu + cfg.anomaly_sigma * np.sqrt(lam.mean()) * v
    return mu, q, lam, anom


def _cluster_mask(cfg, t: int) -> np.ndarray:
    """Anomalous pixels of line t: clusters of cfg.cluster pixels x lines."""
    c = max(int(cfg.cluster), 1)
    block = t // c
    r = np.random.default_rng([cfg.seed, cfg.stream, _TAG_CLUSTER, block])
    # expected clusters per block so that anomaly_frac of pixel-lines are anomalous
    lam = cfg.anomaly_frac * cfg.width / c
    k = int(r.poisson(lam))
    m = np.zeros(cfg.width, bool)
    if k:
        starts = r.integers(0, max(cfg.width - c, 0) + 1, size=k)
        for s0 in starts:
            m[s0:s0 + c] = True
    return m


def anomaly_mask(cfg, t0: int, n: int) -> np.ndarray:
    """Boolean [n][width] mask of planted anomalies for lines t0 .. t0+n-1."""
    return np.stack([_cluster_mask(cfg, t) for t in range(t0, t0 + n)])


def _line_mix(cfg: SceneConfig, t: int, cache: dict) -> np.ndarray:
    scene = cfg.scene_of(t)
    if scene not in cache:
        cache[scene] = _scene_mix(cfg, scene)
    ends, direction, w, anom = cache[scene]
    t_in = t - (scene * cfg.scene_lines if cfg.scene_lines > 0 else 0)
    e = ends + direction * (cfg.drift * t_in / cfg.drift_lines)
    r = np.random.default_rng([cfg.seed, cfg.stream, _TAG_LINE, t])
    pick = r.choice(len(w), size=cfg.width, p=w)
    x = e[pick].astype(np.float32)
    x += r.standard_normal((cfg.width, cfg.bands), dtype=np.float32) * np.float32(cfg.noise)
    m = _cluster_mask(cfg, t)
    if m.any():
        na = int(m.sum())
        target = anom.astype(np.float32) + r.standard_normal(
            (na, cfg.bands), dtype=np.float32) * np.float32(cfg.noise)
        if cfg.anomaly_mix is None:
            x[m] = target
        else:
            f = r.uniform(cfg.anomaly_mix[0], cfg.anomaly_mix[1], size=(na, 1)).astype(np.float32)
            x[m] = (1.0 - f) * x[m] + f * target
    np.clip(x, 0.0, 1.0, out=x)
    if cfg.dn_max > 0:
        return np.rint(x * np.float32(cfg.dn_max)).astype(np.uint16)
    if cfg.scale != 1.0:
        x *= np.float32(cfg.scale)
    return x


def _line_cov(cfg: CovSceneConfig, t: int, cache: dict) -> np.ndarray:
    scene = cfg.scene_of(t)
    if scene not in cache:
        cache[scene] = _scene_cov(cfg, scene)
    mu, q, lam, anom = cache[scene]
    r = np.random.default_rng([cfg.seed, cfg.stream, _TAG_LINE, t])
    g = r.standard_normal((cfg.width, cfg.bands))
    x = mu + (g * np.sqrt(lam)) @ q.T
    m = _cluster_mask(cfg, t)
    if m.any():
        x[m] = anom + (r.standard_normal((int(m.sum()), cfg.bands)) * np.sqrt(lam)) @ q.T
    return x.astype(np.float32)


def gen_lines(cfg, t0: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    """Lines t0 .. t0+n-1 of the cube described by cfg, as [n][width][bands]."""
    if out is None:
        out = np.empty((n, cfg.width, cfg.bands), cfg.dtype)
    cache: dict = {}
    f = _line_cov if isinstance(cfg, CovSceneConfig) else _line_mix
    for i in range(n):
        out[i] = f(cfg, t0 + i, cache)
    return out
