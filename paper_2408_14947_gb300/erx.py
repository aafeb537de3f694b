"""ctypes binding of include/erx.h, function for function, plus a small
torch-tensor convenience wrapper (``Detector``).

Nothing here computes: every step of the ERX line step runs in liberx.so.  If
the library has not been built, loading fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_PKG, "_lib", "liberx.so")

ERX_OK, ERX_EINVAL, ERX_ENOMEM, ERX_ECUDA, ERX_ENOTPD, ERX_ERANGE, ERX_ESTATE, \
    ERX_EUNSUPPORTED, ERX_ETIMEOUT, ERX_EIO = range(10)
ERX_PROJ_NONE, ERX_PROJ_SRP, ERX_PROJ_LEARNED = 0, 1, 2
ERX_UPDATE_THEN_SCORE, ERX_SCORE_THEN_UPDATE = 0, 1
ERX_FLAG_SIMT_STATS, ERX_FLAG_PIPELINE = 1, 2
ERX_AVG_EMA, ERX_AVG_IMC, ERX_AVG_POOLED = 0, 1, 2
ERX_U16, ERX_F32, ERX_F64 = 0, 1, 2
ERX_FORM_FP64, ERX_FORM_FP32, ERX_FORM_TF32, ERX_FORM_BF16, ERX_FORM_TF32X3, ERX_FORM_FP64E = \
    0, 1, 2, 3, 4, 5
FORMS = {"fp64": ERX_FORM_FP64, "fp32": ERX_FORM_FP32, "tf32": ERX_FORM_TF32,
         "bf16": ERX_FORM_BF16, "tf32x3": ERX_FORM_TF32X3, "fp64e": ERX_FORM_FP64E}

_SAMPLE_BYTES = {ERX_U16: 2, ERX_F32: 4, ERX_F64: 8}


class ErxConfig(C.Structure):
    _fields_ = [
        ("bands", C.c_int32), ("width", C.c_int32), ("momentum", C.c_double),
        ("proj", C.c_int32), ("proj_dim", C.c_int32), ("seed", C.c_uint64),
        ("ridge", C.c_double), ("warmup_lines", C.c_int32), ("order", C.c_int32),
        ("in_dtype", C.c_int32), ("in_bits", C.c_int32), ("form", C.c_int32),
        ("threshold", C.c_double), ("block_lines", C.c_int32), ("flags", C.c_int32),
        ("srp_weights", C.POINTER(C.c_double)), ("averaging", C.c_int32),
    ]


class ErxRoc(C.Structure):
    _fields_ = [("auc", C.c_double), ("auc_tpr_tau", C.c_double), ("auc_fpr_tau", C.c_double),
                ("auc_td", C.c_double), ("auc_bs", C.c_double), ("positives", C.c_int64),
                ("negatives", C.c_int64), ("u2", C.c_uint64)]


class ErxTrainOpts(C.Structure):
    _fields_ = [("momentum", C.c_double), ("ridge", C.c_double), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float)]


class ErxError(RuntimeError):
    def __init__(self, status: int, where: str, bad_line: int = -1):
        self.status = status
        self.bad_line = bad_line
        super().__init__(f"{where}: {erx_status_str(status)}"
                         + (f" (line {bad_line})" if bad_line >= 0 else ""))


_lib = None


def load_library() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise ImportError(f"ERX CUDA library not built ({lib_path} missing); run "
                          "__graft_entry__.build() or python -m paper_2408_14947_gb300._build")
    lib = C.CDLL(lib_path)
    P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "erx_config_default": (None, [C.POINTER(ErxConfig), I32, I32]),
        "erx_create": (C.c_int, [C.POINTER(ErxConfig), P, C.POINTER(P)]),
        "erx_push_lines": (C.c_int, [P, P, I64, I64, P, P, P, P]),
        "erx_push_lines_host": (C.c_int, [P, P, I64, I64, P, P, P, P]),
        "erx_sync": (C.c_int, [P, C.POINTER(I64)]),
        "erx_reset": (C.c_int, [P]),
        "erx_get_state": (C.c_int, [P, C.POINTER(I64), P, P]),
        "erx_set_state": (C.c_int, [P, I64, P, P]),
        "erx_dim": (I32, [P]),
        "erx_get_projection": (C.c_int, [P, P]),
        "erx_srp_weights": (C.c_int, [I32, I32, U64, P]),
        "erx_destroy": (C.c_int, [P]),
        "erx_status_str": (C.c_char_p, [C.c_int]),
        "erx_profile_enable": (C.c_int, [P, I32]),
        "erx_profile_read": (C.c_int, [P, I32, I32, C.POINTER(D), C.POINTER(I64),
                                       C.POINTER(I64)]),
        "erx_kernel_name": (C.c_char_p, [I32]),
        "erx_roc_metrics": (C.c_int, [P, I32, P, I64, I32, P, C.POINTER(ErxRoc)]),
        "erx_selftest_bounded_wait": (C.c_int, [C.c_uint32, P]),
        "erx_train_opts_default": (None, [C.POINTER(ErxTrainOpts)]),
        "erx_encoder_create": (C.c_int, [I32, I32, I32, U64, P, C.POINTER(P)]),
        "erx_encoder_set_norm": (C.c_int, [P, P, P]),
        "erx_encoder_params": (C.c_int, [P, P, P]),
        "erx_encoder_nparams": (I64, [P]),
        "erx_encoder_dims": (I32, [P, C.POINTER(I32), C.POINTER(I32)]),
        "erx_encoder_reset_stats": (C.c_int, [P]),
        "erx_encoder_forward": (C.c_int, [P, P, I64, P]),
        "erx_encoder_train": (C.c_int, [P, P, I64, I32, P, C.POINTER(ErxTrainOpts), P]),
        "erx_encoder_line_grad": (C.c_int, [P, P, I32, P, C.POINTER(ErxTrainOpts), P, P]),
        "erx_encoder_destroy": (C.c_int, [P]),
        "erx_encoder_save": (C.c_int, [P, C.c_char_p]),
        "erx_encoder_load": (C.c_int, [C.c_char_p, P, C.POINTER(P)]),
        "erx_set_encoder": (C.c_int, [P, P, I32, D]),
        "erx_get_drift": (C.c_int, [P, C.POINTER(D), C.POINTER(D), C.POINTER(I64),
                                    C.POINTER(I32)]),
        "erx_batch_create": (C.c_int, [I32, C.POINTER(ErxConfig), P, C.POINTER(P)]),
        "erx_batch_buffers": (C.c_int, [P, I32, C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                        C.POINTER(P), C.POINTER(P)]),
        "erx_batch_push": (C.c_int, [P, P]),
        "erx_batch_sync": (C.c_int, [P, C.POINTER(I64)]),
        "erx_batch_get_state": (C.c_int, [P, I32, C.POINTER(I64), P, P]),
        "erx_batch_route": (C.c_int, [P, I32, C.POINTER(I32)]),
        "erx_batch_tune": (C.c_int, [P, I32, C.c_char_p]),
        "erx_batch_set_encoder": (C.c_int, [P, P]),
        "erx_batch_destroy": (C.c_int, [P]),
        "erx_push_lines_static": (C.c_int, [C.POINTER(ErxConfig), P, P, P, C.POINTER(I64), P,
                                            I64, I64, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != ERX_OK:
        raise ErxError(st, where)


def erx_status_str(status: int) -> str:
    return load_library().erx_status_str(status).decode()


def erx_config_default(bands: int, width: int) -> ErxConfig:
    cfg = ErxConfig()
    load_library().erx_config_default(C.byref(cfg), bands, width)
    return cfg


def erx_create(cfg: ErxConfig, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load_library().erx_create(C.byref(cfg), C.c_void_p(stream), C.byref(h)), "erx_create")
    return h.value


def erx_push_lines(ctx, lines_ptr, n_lines, stride_bytes, delta_ptr, dn_ptr=0, mask_ptr=0,
                   det_ptr=0):
    _check(load_library().erx_push_lines(ctx, lines_ptr, n_lines, stride_bytes, delta_ptr,
                                         dn_ptr or None, mask_ptr or None, det_ptr or None),
           "erx_push_lines")


def erx_push_lines_host(ctx, lines_ptr, n_lines, stride_bytes, delta_ptr, dn_ptr=0, mask_ptr=0,
                        det_ptr=0):
    _check(load_library().erx_push_lines_host(ctx, lines_ptr, n_lines, stride_bytes, delta_ptr,
                                              dn_ptr or None, mask_ptr or None, det_ptr or None),
           "erx_push_lines_host")


def erx_sync(ctx) -> None:
    bad = C.c_int64(-1)
    st = load_library().erx_sync(ctx, C.byref(bad))
    if st != ERX_OK:
        raise ErxError(st, "erx_sync", bad.value)


def erx_reset(ctx) -> None:
    _check(load_library().erx_reset(ctx), "erx_reset")


def erx_dim(ctx) -> int:
    return int(load_library().erx_dim(ctx))


def erx_get_state(ctx):
    import numpy as np
    d = erx_dim(ctx)
    t = C.c_int64()
    mu = np.zeros(d)
    k = np.zeros((d, d))
    _check(load_library().erx_get_state(ctx, C.byref(t), mu.ctypes.data, k.ctypes.data),
           "erx_get_state")
    return t.value, mu, k


def erx_set_state(ctx, t, mu, k) -> None:
    import numpy as np
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    k = np.ascontiguousarray(k, dtype=np.float64)
    _check(load_library().erx_set_state(ctx, int(t), mu.ctypes.data, k.ctypes.data),
           "erx_set_state")


def erx_get_projection(ctx, bands: int):
    import numpy as np
    w = np.zeros((bands, erx_dim(ctx)))
    _check(load_library().erx_get_projection(ctx, w.ctypes.data), "erx_get_projection")
    return w


def erx_srp_weights(bands: int, dim: int, seed: int):
    import numpy as np
    w = np.zeros((bands, dim))
    _check(load_library().erx_srp_weights(bands, dim, C.c_uint64(seed), w.ctypes.data),
           "erx_srp_weights")
    return w


ERX_K_COUNT = 15


def erx_push_lines_static(cfg, stream, mu_ptr, k_ptr, t, lines_ptr, n_lines, stride_bytes,
                          delta_ptr, dn_ptr=0, mask_ptr=0, det_ptr=0) -> int:
    """Context-free line step on caller-held state; returns the new line count.

    ERX_ENOTPD and ERX_ERANGE are raised after the lines have been processed
    (the state has advanced): the raised ErxError carries the new line count
    as ``t``, so a caller does not apply the same lines twice."""
    tt = C.c_int64(t)
    st = load_library().erx_push_lines_static(C.byref(cfg), C.c_void_p(stream), mu_ptr, k_ptr,
                                              C.byref(tt), lines_ptr, n_lines, stride_bytes,
                                              delta_ptr, dn_ptr or None, mask_ptr or None,
                                              det_ptr or None)
    if st != ERX_OK:
        err = ErxError(st, "erx_push_lines_static")
        err.t = tt.value
        raise err
    return tt.value


def roc_metrics(scores, labels, bins: int = 1 << 16, stream=None) -> dict:
    """Detection quality of a score map (Sec. IV-B) on the GPU: ROC AUC of the
    map quantised to `bins` levels, AUC_TPR,tau, AUC_FPR,tau, AUC_TD, AUC_BS.
    scores: CUDA float32/float64 tensor; labels: CUDA bool/uint8 tensor (same
    number of elements, nonzero = anomaly)."""
    import torch
    s = scores.contiguous()
    y = labels.contiguous().to(torch.uint8)
    assert s.is_cuda and y.is_cuda and s.numel() == y.numel()
    dt = {torch.float32: ERX_F32, torch.float64: ERX_F64}[s.dtype]
    st = stream if stream is not None else torch.cuda.current_stream()
    out = ErxRoc()
    _check(load_library().erx_roc_metrics(s.data_ptr(), dt, y.data_ptr(), s.numel(), bins,
                                          st.cuda_stream, C.byref(out)), "erx_roc_metrics")
    return {k: getattr(out, k) for k, _ in ErxRoc._fields_}


def erx_kernel_name(k: int) -> str:
    return load_library().erx_kernel_name(k).decode()


def selftest_bounded_wait(limit: int = 1000, stream=None) -> int:
    """Run the bounded-wait self-test (erx_selftest_bounded_wait) and return its
    status: ERX_ETIMEOUT when the wait ran out as designed."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return load_library().erx_selftest_bounded_wait(limit, C.c_void_p(st.cuda_stream))


def erx_profile_enable(ctx, on: bool) -> None:
    _check(load_library().erx_profile_enable(ctx, 1 if on else 0), "erx_profile_enable")


def erx_profile_read(ctx, kernel: int, reset: bool = False):
    """(total_ms, timed_launches, launches) for one kernel kind."""
    ms, timed, n = C.c_double(), C.c_int64(), C.c_int64()
    _check(load_library().erx_profile_read(ctx, kernel, 1 if reset else 0, C.byref(ms),
                                           C.byref(timed), C.byref(n)), "erx_profile_read")
    return ms.value, timed.value, n.value


def erx_destroy(ctx) -> None:
    _check(load_library().erx_destroy(ctx), "erx_destroy")


class Detector:
    """One ERX context driven with torch tensors (device memory and streams only).

    ``push(lines)`` takes a CUDA tensor [n][p][b] (uint16 viewed as int16,
    float32 or float64 samples) and returns (delta, delta_n, mask, detecting)
    CUDA tensors; every step runs in liberx.so on the tensor's stream.
    """

    def __init__(self, bands, width, momentum=0.1, proj="none", proj_dim=5, seed=0, ridge=1e-5,
                 warmup=99, order="update_then_score", in_dtype="f32", in_bits=16,
                 form="fp64", threshold=3.0, block_lines=0, srp_weights=None, stream=None,
                 simt_stats=False, encoder=None, audit_every=0, min_rank_corr=0.0,
                 averaging="ema", pipeline=False):
        import torch
        self.torch = torch
        cfg = erx_config_default(bands, width)
        cfg.momentum = momentum
        cfg.proj = {"none": ERX_PROJ_NONE, "srp": ERX_PROJ_SRP,
                    "learned": ERX_PROJ_LEARNED}[proj if encoder is None else "learned"]
        if encoder is not None:
            proj_dim = encoder.k
        cfg.proj_dim = proj_dim
        cfg.seed = seed
        cfg.ridge = ridge
        cfg.warmup_lines = warmup
        cfg.order = {"update_then_score": ERX_UPDATE_THEN_SCORE,
                     "score_then_update": ERX_SCORE_THEN_UPDATE}[order]
        cfg.in_dtype = {"u16": ERX_U16, "f32": ERX_F32, "f64": ERX_F64}[in_dtype]
        cfg.in_bits = in_bits
        cfg.form = FORMS[form]
        cfg.threshold = threshold if threshold is not None else math.inf
        cfg.block_lines = block_lines
        cfg.flags = (ERX_FLAG_SIMT_STATS if simt_stats else 0) | \
            (ERX_FLAG_PIPELINE if pipeline else 0)
        cfg.averaging = {"ema": ERX_AVG_EMA, "imc": ERX_AVG_IMC,
                         "pooled": ERX_AVG_POOLED}[averaging]
        self._w = None
        if srp_weights is not None:
            import numpy as np
            self._w = np.ascontiguousarray(srp_weights, dtype=np.float64)
            cfg.proj = ERX_PROJ_SRP
            cfg.proj_dim = self._w.shape[1]
            cfg.srp_weights = self._w.ctypes.data_as(C.POINTER(C.c_double))
        self.cfg = cfg
        self.bands, self.width = bands, width
        self.in_dtype = cfg.in_dtype
        self.score_dtype = torch.float64 if form in ("fp64", "fp64e") else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = erx_create(cfg, self.stream.cuda_stream)
        self.dim = erx_dim(self.ctx)
        self.encoder = encoder
        if encoder is not None:
            _check(load_library().erx_set_encoder(self.ctx, encoder.e, audit_every,
                                                  min_rank_corr), "erx_set_encoder")

    def push(self, lines, out=None):
        torch = self.torch
        assert lines.is_cuda and lines.dim() == 3 and lines.is_contiguous()
        n, p, b = lines.shape
        assert p == self.width and b == self.bands
        assert lines.element_size() == _SAMPLE_BYTES[self.in_dtype]
        dev = lines.device
        if out is None:
            out = (torch.empty((n, p), dtype=self.score_dtype, device=dev),
                   torch.empty((n, p), dtype=self.score_dtype, device=dev),
                   torch.empty((n, p), dtype=torch.uint8, device=dev),
                   torch.empty((n,), dtype=torch.uint8, device=dev))
        delta, dn, mask, det = out
        cur = torch.cuda.current_stream(dev)
        other = cur.cuda_stream != self.stream.cuda_stream
        if other:           # lines (and the outputs' memory) come from the caller's stream
            self.stream.wait_stream(cur)
        erx_push_lines(self.ctx, lines.data_ptr(), n, 0, delta.data_ptr(), dn.data_ptr(),
                       mask.data_ptr(), det.data_ptr())
        if other:           # outputs are written on the detector's stream
            cur.wait_stream(self.stream)
        return delta, dn, mask, det

    def push_host(self, lines, out):
        """lines and the four outputs are host (CPU) tensors; synchronous."""
        n = lines.shape[0]
        delta, dn, mask, det = out
        erx_push_lines_host(self.ctx, lines.data_ptr(), n, 0, delta.data_ptr(), dn.data_ptr(),
                            mask.data_ptr(), det.data_ptr())
        return out

    def sync(self):
        erx_sync(self.ctx)

    def reset(self):
        erx_reset(self.ctx)

    def state(self):
        return erx_get_state(self.ctx)

    def set_state(self, t, mu, k):
        erx_set_state(self.ctx, t, mu, k)

    def projection(self):
        return erx_get_projection(self.ctx, self.bands)

    def drift(self):
        """(last rank correlation, lowest, audits, fallback active)."""
        last, low, n, fb = C.c_double(), C.c_double(), C.c_int64(), C.c_int32()
        _check(load_library().erx_get_drift(self.ctx, C.byref(last), C.byref(low), C.byref(n),
                                            C.byref(fb)), "erx_get_drift")
        return last.value, low.value, n.value, bool(fb.value)

    def profile(self, on: bool = True):
        erx_profile_enable(self.ctx, on)

    def profile_read(self, reset: bool = False):
        """{kernel name: (total_ms, timed_launches, launches)}; reset clears after reading."""
        out = {erx_kernel_name(k): erx_profile_read(self.ctx, k) for k in range(ERX_K_COUNT)}
        if reset:
            erx_profile_read(self.ctx, 0, True)
        return out

    def close(self):
        if self.ctx:
            erx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batch of independent streams (erx_batch_*), one line each per step.

    ``streams`` is a list of dicts with ``bands`` and ``width`` (and optional
    momentum, ridge, warmup, order, threshold, and ``learned``: run ERX on the
    codes of ``encoder``, shared by all learned streams); ``form`` is shared.
    Inputs and outputs are batch-owned device buffers exposed as torch tensors.
    """

    def __init__(self, streams, form="fp64", stream=None, encoder=None):
        import torch
        self.torch = torch
        n = len(streams)
        cfgs = (ErxConfig * n)()
        for i, sd in enumerate(streams):
            load_library().erx_config_default(C.byref(cfgs[i]), sd["bands"], sd["width"])
            c = cfgs[i]
            c.in_dtype = ERX_F32
            c.form = FORMS[form]
            c.momentum = sd.get("momentum", 0.1)
            c.ridge = sd.get("ridge", 1e-5)
            c.warmup_lines = sd.get("warmup", 99)
            c.order = {"update_then_score": ERX_UPDATE_THEN_SCORE,
                       "score_then_update": ERX_SCORE_THEN_UPDATE}[sd.get("order",
                                                                      "update_then_score")]
            c.threshold = sd.get("threshold", 3.0)
            if sd.get("learned"):
                if encoder is None:
                    raise ValueError("learned streams need an encoder")
                c.proj = ERX_PROJ_LEARNED
                c.proj_dim = encoder.k
        self.n = n
        self.encoder = encoder
        self.streams = streams
        self.form = form
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(load_library().erx_batch_create(n, cfgs, C.c_void_p(self.stream.cuda_stream),
                                               C.byref(h)), "erx_batch_create")
        self.b = h.value
        self._ptrs = (C.c_void_p * n)()
        if any(sd.get("learned") for sd in streams):
            _check(load_library().erx_batch_set_encoder(self.b, C.c_void_p(encoder.e)),
                   "erx_batch_set_encoder")

    def dim(self, i):
        """ERX dimension of stream i: its bands, or the encoder's k if learned."""
        return self.encoder.k if self.streams[i].get("learned") else self.streams[i]["bands"]

    def buffers(self, i):
        """Raw device pointers (line, delta, delta_n, mask, detecting) of stream i."""
        p = [C.c_void_p() for _ in range(5)]
        _check(load_library().erx_batch_buffers(self.b, i, *[C.byref(q) for q in p]),
               "erx_batch_buffers")
        return [q.value for q in p]

    def push(self, lines=None):
        """lines: None (inputs already in place) or a list of n CUDA float32
        tensors (or None entries) holding one line each."""
        if lines is None:
            _check(load_library().erx_batch_push(self.b, None), "erx_batch_push")
            return
        for i, x in enumerate(lines):
            self._ptrs[i] = None if x is None else x.data_ptr()
        _check(load_library().erx_batch_push(self.b, self._ptrs), "erx_batch_push")

    def sync(self):
        bad = C.c_int64(-1)
        st = load_library().erx_batch_sync(self.b, C.byref(bad))
        if st != ERX_OK:
            raise ErxError(st, "erx_batch_sync", bad.value)

    def state(self, i):
        import numpy as np
        d = self.dim(i)
        t = C.c_int64()
        mu, k = np.zeros(d), np.zeros((d, d))
        _check(load_library().erx_batch_get_state(self.b, i, C.byref(t), mu.ctypes.data,
                                                  k.ctypes.data), "erx_batch_get_state")
        return t.value, mu, k

    def route(self, i):
        r = C.c_int32()
        _check(load_library().erx_batch_route(self.b, i, C.byref(r)), "erx_batch_route")
        return r.value

    def tune(self, reps=3, cache_path=None):
        _check(load_library().erx_batch_tune(self.b, reps,
                                             cache_path.encode() if cache_path else None),
               "erx_batch_tune")

    def views(self, i):
        """Torch views (no copy) of stream i's batch-owned device buffers:
        line [W][B] float32, delta and delta_n [W], mask [W], detecting [1]."""
        torch = self.torch
        line, dl, dn, mk, dt = self.buffers(i)
        w, bands = self.streams[i]["width"], self.streams[i]["bands"]
        st = "<f8" if self.form in ("fp64", "fp64e") else "<f4"
        return (_device_view(line, (w, bands), "<f4"), _device_view(dl, (w,), st),
                _device_view(dn, (w,), st), _device_view(mk, (w,), "|u1"),
                _device_view(dt, (1,), "|u1"))

    def close(self):
        if self.b:
            load_library().erx_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevBuf:
    """__cuda_array_interface__ over a library-owned device buffer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _device_view(ptr, shape, typestr):
    import torch
    return torch.as_tensor(_DevBuf(ptr, shape, typestr), device="cuda")


def erx_train_opts_default() -> ErxTrainOpts:
    o = ErxTrainOpts()
    load_library().erx_train_opts_default(C.byref(o))
    return o


class Encoder:
    """Learned band encoder (erx_encoder_*): bands -> hidden -> k, trained on the GPU."""

    def __init__(self, bands=224, hidden=128, k=32, seed=0, stream=None, _handle=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if _handle is None:
            h = C.c_void_p()
            _check(load_library().erx_encoder_create(bands, hidden, k, C.c_uint64(seed),
                                                     C.c_void_p(self.stream.cuda_stream),
                                                     C.byref(h)), "erx_encoder_create")
            _handle = h.value
        self.e = _handle
        b, hd = C.c_int32(), C.c_int32()
        self.k = int(load_library().erx_encoder_dims(self.e, C.byref(b), C.byref(hd)))
        self.bands, self.hidden = b.value, hd.value
        self.nparams = int(load_library().erx_encoder_nparams(self.e))

    def save(self, path):
        """Checkpoint: normalisation, weights, AdamW moments, code-space EMA."""
        _check(load_library().erx_encoder_save(self.e, os.fsencode(path)), "erx_encoder_save")

    @classmethod
    def load(cls, path, stream=None):
        import torch
        stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(load_library().erx_encoder_load(os.fsencode(path), C.c_void_p(stream.cuda_stream),
                                               C.byref(h)), "erx_encoder_load")
        return cls(stream=stream, _handle=h.value)

    def set_norm(self, shift, scale):
        import numpy as np
        s = np.ascontiguousarray(shift, np.float32)
        c = np.ascontiguousarray(scale, np.float32)
        _check(load_library().erx_encoder_set_norm(self.e, s.ctypes.data, c.ctypes.data),
               "erx_encoder_set_norm")

    def params(self, new=None):
        """Current parameter vector (numpy float32); `new` replaces it first."""
        import numpy as np
        out = np.zeros(self.nparams, np.float32)
        src = None
        if new is not None:
            src = np.ascontiguousarray(new, np.float32)
        _check(load_library().erx_encoder_params(self.e, out.ctypes.data,
                                                 None if src is None else src.ctypes.data),
               "erx_encoder_params")
        return out

    def split(self, theta):
        b, h, k = self.bands, self.hidden, self.k
        o1 = h * b
        return {"W1": theta[:o1].reshape(h, b), "b1": theta[o1:o1 + h],
                "W2": theta[o1 + h:o1 + h + k * h].reshape(k, h), "b2": theta[o1 + h + k * h:]}

    def reset_stats(self):
        _check(load_library().erx_encoder_reset_stats(self.e), "erx_encoder_reset_stats")

    def forward(self, x):
        """x: CUDA float32 [..., bands] -> codes [..., k]."""
        torch = self.torch
        xc = x.contiguous()
        n = xc.numel() // self.bands
        out = torch.empty(xc.shape[:-1] + (self.k,), dtype=torch.float32, device=x.device)
        cur = torch.cuda.current_stream(x.device)
        other = cur.cuda_stream != self.stream.cuda_stream
        if other:
            self.stream.wait_stream(cur)
        _check(load_library().erx_encoder_forward(self.e, xc.data_ptr(), n, out.data_ptr()),
               "erx_encoder_forward")
        if other:           # codes are written on the encoder's stream
            cur.wait_stream(self.stream)
        return out

    def train(self, lines, targets, opts=None, want_loss=False):
        """lines: CUDA float32 [n][p][bands]; targets: CUDA float64 [n][p]."""
        import numpy as np
        opts = opts or erx_train_opts_default()
        n, p, _ = lines.shape
        loss = np.zeros(n, np.float32) if want_loss else None
        _check(load_library().erx_encoder_train(
            self.e, lines.data_ptr(), n, p, targets.data_ptr(), C.byref(opts),
            None if loss is None else loss.ctypes.data), "erx_encoder_train")
        return loss

    def line_grad(self, line, target, opts=None):
        import numpy as np
        opts = opts or erx_train_opts_default()
        g = np.zeros(self.nparams, np.float32)
        loss = C.c_float()
        p = line.shape[0]
        _check(load_library().erx_encoder_line_grad(self.e, line.data_ptr(), p,
                                                    target.data_ptr(), C.byref(opts),
                                                    g.ctypes.data, C.byref(loss)),
               "erx_encoder_line_grad")
        return g, loss.value

    def close(self):
        if self.e:
            load_library().erx_encoder_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
