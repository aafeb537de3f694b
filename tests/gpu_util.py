"""Helpers for the GPU tests: torch device plumbing around the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14947_gb300 import _build
    _build.build()


def to_dev(cube: np.ndarray):
    if cube.dtype == np.uint16:
        return torch.from_numpy(cube.view(np.int16)).cuda()
    return torch.from_numpy(np.ascontiguousarray(cube)).cuda()


def in_dtype(cube):
    return {np.dtype(np.uint16): "u16", np.dtype(np.float32): "f32",
            np.dtype(np.float64): "f64"}[cube.dtype]


def run_gpu(cube, push_sizes=None, profile=False, **kw):
    """Run the CUDA detector over cube; returns numpy outputs and the detector
    (with per-kernel launch counts and times when profile is set)."""
    from paper_2408_14947_gb300 import Detector
    n, p, b = cube.shape
    kw.setdefault("in_dtype", in_dtype(cube))
    det = Detector(b, p, **kw)
    if profile:
        det.profile(True)
    x = to_dev(cube)
    outs = []
    if push_sizes is None:
        push_sizes = [n]
    s = 0
    for m in push_sizes:
        outs.append(det.push(x[s:s + m]))
        s += m
    assert s == n
    det.sync()
    cat = [torch.cat([o[i] for o in outs]).cpu().numpy() for i in range(4)]
    return {"delta": cat[0], "delta_n": cat[1], "mask": cat[2].astype(bool),
            "detecting": cat[3].astype(bool)}, det


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def dn_err(got, ref_delta, ref_dn):
    """|delta_N error| / (mean/std + |delta_N|) per line: the delta_N bound that a
    relative delta error implies."""
    m = ref_delta.mean(axis=1, keepdims=True)
    s = ref_delta.std(axis=1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(s > 0, m / np.where(s > 0, s, 1.0), np.inf) + np.abs(ref_dn)
        e = np.abs(got - ref_dn) / scale
    # zero-spread lines have delta_N = 0 exactly on both sides
    e = np.where(np.isfinite(scale), e, np.abs(got - ref_dn))
    return float(np.max(e))

