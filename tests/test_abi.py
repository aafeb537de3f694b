"""The C-ABI library loads, exports what include/erx.h declares, and its
host-only logic behaves (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2408_14947_gb300 as erx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(erx_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2408_14947_gb300 import _build
    _build.build()
    return erx.load_library()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "erx_create" in names and "erx_push_lines" in names and len(names) >= 13
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_srp_weights_match_oracle(lib):
    for b, d, seed in ((108, 5, 0), (224, 32, 7), (13, 13, 99), (1, 1, 3)):
        assert np.array_equal(erx.erx_srp_weights(b, d, seed), oracle.srp_weights(b, d, seed))


def test_config_defaults(lib):
    c = erx.erx_config_default(108, 640)
    assert (c.bands, c.width, c.proj_dim, c.warmup_lines) == (108, 640, 5, 99)
    assert c.momentum == 0.1 and c.ridge == 1e-5 and c.order == erx.ERX_UPDATE_THEN_SCORE


@pytest.mark.parametrize("field,value", [("width", 1), ("bands", 0), ("momentum", 0.0),
                                         ("momentum", 1.5), ("ridge", -1.0), ("order", 7),
                                         ("in_dtype", 9), ("form", 99), ("proj", 4)])
def test_invalid_config_rejected_before_any_cuda_call(lib, field, value):
    c = erx.erx_config_default(8, 16)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert lib.erx_create(ctypes.byref(c), None, ctypes.byref(h)) == erx.ERX_EINVAL
    assert h.value is None


def test_beyond_limits_unsupported(lib):
    c = erx.erx_config_default(300, 16)
    h = ctypes.c_void_p()
    assert lib.erx_create(ctypes.byref(c), None, ctypes.byref(h)) == erx.ERX_EUNSUPPORTED


def test_null_handles(lib):
    assert lib.erx_destroy(None) == erx.ERX_OK
    assert lib.erx_push_lines(None, None, 0, 0, None, None, None, None) == erx.ERX_EINVAL
    assert lib.erx_sync(None, None) == erx.ERX_EINVAL
    assert lib.erx_dim(None) == -1
    for s in range(10):
        assert erx.erx_status_str(s).startswith("ERX_")


def test_host_side_argument_checks(lib):
    """Argument checks that return before any CUDA call."""
    assert lib.erx_selftest_bounded_wait(0, None) == erx.ERX_EINVAL
    assert lib.erx_selftest_bounded_wait((1 << 20) + 1, None) == erx.ERX_EINVAL
    assert lib.erx_batch_set_encoder(None, None) == erx.ERX_EINVAL
    assert lib.erx_batch_push(None, None) == erx.ERX_EINVAL
    assert lib.erx_batch_destroy(None) == erx.ERX_OK
    h = ctypes.c_void_p()
    assert lib.erx_batch_create(0, None, None, ctypes.byref(h)) == erx.ERX_EINVAL


def test_encoder_checkpoint_host_checks(lib, tmp_path):
    """Checkpoint files that are missing, truncated or of another kind are
    refused (ERX_EIO) before any device work."""
    h = ctypes.c_void_p()
    assert lib.erx_encoder_save(None, b"x") == erx.ERX_EINVAL
    assert lib.erx_encoder_load(None, None, ctypes.byref(h)) == erx.ERX_EINVAL
    missing = str(tmp_path / "missing.bin").encode()
    assert lib.erx_encoder_load(missing, None, ctypes.byref(h)) == erx.ERX_EIO
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTANENC" + bytes(32))
    assert lib.erx_encoder_load(str(bad).encode(), None, ctypes.byref(h)) == erx.ERX_EIO
    short = tmp_path / "short.bin"
    short.write_bytes(b"ERXENC01" + bytes(4))
    assert lib.erx_encoder_load(str(short).encode(), None, ctypes.byref(h)) == erx.ERX_EIO
    import struct
    big = tmp_path / "big.bin"          # sizes beyond the encoder's limits
    big.write_bytes(b"ERXENC01" + struct.pack("<4i2q", 224, 512, 32, 0, 0, 0))
    assert lib.erx_encoder_load(str(big).encode(), None, ctypes.byref(h)) == erx.ERX_EIO
    assert h.value is None
