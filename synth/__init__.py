"""Seeded, line-addressable synthetic line-scan cubes.

This package holds input generators only: it draws pixels and anomaly masks and
contains none of the detector's arithmetic.  Both the CUDA path's tests and the
oracle's tests take their inputs from here.
"""
from .cubes import (  # noqa: F401
    SceneConfig,
    CovSceneConfig,
    reflectance_c1,
    dn_c2,
    cov_c3,
    gen_lines,
    anomaly_mask,
    stream_configs_c4,
    random_uniform_cube,
)
