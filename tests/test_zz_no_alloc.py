"""erx_push_lines_static, the line step for callers that cannot allocate device
memory, against the context-based erx_push_lines (GPU).

Runs last (file name) so that a stop at the first failure has run every other
test; it must also pass alone in a fresh process, where its first call does
the per-device set-up.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import need_gpu, rel_err, run_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


CASES = [
    # form, input, order, tolerance against the context path
    ("fp64", "u16", "update_then_score", 1e-9),
    ("fp32", "u16", "update_then_score", 1e-4),
    ("fp64", "f32", "update_then_score", 1e-9),     # float lines: mean pass + FP64 scatter
    ("fp32", "f32", "update_then_score", 1e-4),     # float lines: FP32 scatter about a shift
    ("fp64", "u16", "score_then_update", 1e-9),
    ("fp32", "f32", "score_then_update", 1e-4),
]


def _static_cfg(erx, b, p, form, inp, order, warmup=5, threshold=2.0, ridge=1e-5):
    cfg = erx.erx_config_default(b, p)
    cfg.in_dtype = erx.ERX_U16 if inp == "u16" else erx.ERX_F32
    cfg.in_bits = 12
    cfg.form = erx.ERX_FORM_FP64 if form == "fp64" else erx.ERX_FORM_FP32
    cfg.order = (erx.ERX_UPDATE_THEN_SCORE if order == "update_then_score"
                 else erx.ERX_SCORE_THEN_UPDATE)
    cfg.warmup_lines = warmup
    cfg.threshold = threshold
    cfg.ridge = ridge
    return cfg


@pytest.mark.parametrize("form,inp,order,tol", CASES)
def test_static_matches_context_two_calls(form, inp, order, tol):
    need_gpu()
    import paper_2408_14947_gb300 as erx

    cfg_s = synth.dn_c2(width=160, bands=108, seed=4)
    cube = synth.gen_lines(cfg_s, 0, 15)
    if inp == "f32":
        cube = cube.astype(np.float32)
    n, p, b = cube.shape
    kw = {"in_bits": 12} if inp == "u16" else {}
    ref, det = run_gpu(cube, form=form, warmup=5, threshold=2.0, order=order, **kw)
    t_ref, mu_ref, k_ref = det.state()

    cfg = _static_cfg(erx, b, p, form, inp, order)
    sdt = torch.float64 if form == "fp64" else torch.float32
    x = to_dev(cube)
    mu = torch.full((b,), float("nan"), dtype=torch.float64, device="cuda")
    kp = torch.full((b * (b + 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
    delta = torch.empty((n, p), dtype=sdt, device="cuda")
    dn = torch.empty((n, p), dtype=sdt, device="cuda")
    mask = torch.empty((n, p), dtype=torch.uint8, device="cuda")
    flags = torch.empty((n,), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    t = 0
    for lo, hi in ((0, 7), (7, n)):               # two calls in a row, state carried over
        t = erx.erx_push_lines_static(
            cfg, stream, mu.data_ptr(), kp.data_ptr(), t, x[lo:hi].data_ptr(), hi - lo, 0,
            delta[lo:hi].data_ptr(), dn[lo:hi].data_ptr(), mask[lo:hi].data_ptr(),
            flags[lo:hi].data_ptr())
    assert t == n == t_ref
    torch.cuda.synchronize()
    assert rel_err(delta.cpu().numpy(), ref["delta"]) <= tol
    assert np.max(np.abs(dn.cpu().numpy() - ref["delta_n"])) <= 10 * tol
    assert np.array_equal(flags.cpu().numpy().astype(bool), ref["detecting"])
    assert rel_err(mu.cpu().numpy(), mu_ref) <= 1e-12
    kpn = kp.cpu().numpy()
    low = np.array([k_ref[a, c] for a in range(b) for c in range(a + 1)])
    assert rel_err(kpn, low) <= 1e-12


def test_static_not_pd_reports_advanced_line_count():
    """ridge 0 and constant lines: the first pivot is 0 (ERX_ENOTPD).  The call
    has still processed every line, and the error carries the new count."""
    need_gpu()
    import paper_2408_14947_gb300 as erx
    n, p, b = 3, 10, 4
    cfg = _static_cfg(erx, b, p, "fp64", "f32", "update_then_score", ridge=0.0)
    x = torch.ones((n, p, b), dtype=torch.float32, device="cuda")
    mu = torch.zeros((b,), dtype=torch.float64, device="cuda")
    kp = torch.zeros((b * (b + 1) // 2,), dtype=torch.float64, device="cuda")
    delta = torch.empty((n, p), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(erx.ErxError) as ei:
        erx.erx_push_lines_static(cfg, stream, mu.data_ptr(), kp.data_ptr(), 5, x.data_ptr(), n,
                                  0, delta.data_ptr())
    assert ei.value.status == erx.ERX_ENOTPD and ei.value.t == 5 + n
    # the state is usable afterwards: a valid line with a ridge goes through
    cfg.ridge = 1e-5
    xr = torch.rand((1, p, b), dtype=torch.float32, device="cuda")
    t = erx.erx_push_lines_static(cfg, stream, mu.data_ptr(), kp.data_ptr(), 0, xr.data_ptr(),
                                  1, 0, delta.data_ptr())
    assert t == 1 and torch.all(torch.isfinite(delta[0]))


def test_static_rejects_beyond_limits():
    need_gpu()
    import paper_2408_14947_gb300 as erx
    cfg = erx.erx_config_default(300, 64)
    t = 0
    with pytest.raises(erx.ErxError) as ei:
        erx.erx_push_lines_static(cfg, 0, 1, 1, t, 1, 1, 0, 1)
    assert ei.value.status == erx.ERX_EUNSUPPORTED
    cfg = erx.erx_config_default(16, 64)
    cfg.proj = erx.ERX_PROJ_SRP
    with pytest.raises(erx.ErxError) as ei:
        erx.erx_push_lines_static(cfg, 0, 1, 1, t, 1, 1, 0, 1)
    assert ei.value.status == erx.ERX_EUNSUPPORTED
    cfg = erx.erx_config_default(16, 64)
    cfg.averaging = erx.ERX_AVG_IMC
    with pytest.raises(erx.ErxError) as ei:
        erx.erx_push_lines_static(cfg, 0, 1, 1, t, 1, 1, 0, 1)
    assert ei.value.status == erx.ERX_EUNSUPPORTED
    cfg = erx.erx_config_default(16, 64)
    cfg.form = erx.ERX_FORM_TF32
    with pytest.raises(erx.ErxError) as ei:
        erx.erx_push_lines_static(cfg, 0, 1, 1, t, 1, 1, 0, 1)
    assert ei.value.status == erx.ERX_EINVAL
