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


@pytest.mark.parametrize("form,in_bits,tol", [("fp64", 12, 1e-9), ("fp32", 12, 1e-4)])
def test_static_matches_context_two_calls(form, in_bits, tol):
    need_gpu()
    import paper_2408_14947_gb300 as erx

    cfg_s = synth.dn_c2(width=160, bands=108, seed=4)
    cube = synth.gen_lines(cfg_s, 0, 15)
    n, p, b = cube.shape
    ref, det = run_gpu(cube, form=form, in_bits=in_bits, warmup=5, threshold=2.0)
    t_ref, mu_ref, k_ref = det.state()

    cfg = erx.erx_config_default(b, p)
    cfg.in_dtype = erx.ERX_U16
    cfg.in_bits = in_bits
    cfg.form = erx.ERX_FORM_FP64 if form == "fp64" else erx.ERX_FORM_FP32
    cfg.warmup_lines = 5
    cfg.threshold = 2.0
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
