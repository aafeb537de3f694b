"""Failure handling on the GPU without a fault: a bounded device wait that runs
out (ERX_ETIMEOUT, context still usable), an allocation that cannot succeed
(ERX_ENOMEM, nothing left allocated), and two contexts that do not disturb each
other."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, rel_err, run_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    need_gpu()
    from paper_2408_14947_gb300 import ERX_EINVAL, ERX_ETIMEOUT, selftest_bounded_wait
    assert selftest_bounded_wait(1000) == ERX_ETIMEOUT
    assert selftest_bounded_wait(0) == ERX_EINVAL
    # the device and the library keep working afterwards
    cube = synth.gen_lines(synth.dn_c2(width=96, bands=12, seed=2), 0, 6)
    got, _ = run_gpu(cube, in_bits=12, warmup=2)
    ref = oracle.run_cube(cube, warmup=2)
    assert rel_err(got["delta"], ref["delta"]) < 1e-9


def test_batch_allocation_failure_is_enomem():
    """400 streams of 2^20 px x 224 bands need 376 GB for their input lines
    alone, more than the device has: creation fails cleanly with ERX_ENOMEM
    (the request is refused outright, no memory is filled)."""
    need_gpu()
    from paper_2408_14947_gb300 import ERX_ENOMEM, ErxConfig
    from paper_2408_14947_gb300.erx import load_library
    lib = load_library()
    n = 400
    cfgs = (ErxConfig * n)()
    for i in range(n):
        lib.erx_config_default(C.byref(cfgs[i]), 224, 1 << 20)
        cfgs[i].in_dtype = 1   # float32
    free0 = torch.cuda.mem_get_info()[0]
    h = C.c_void_p()
    st = lib.erx_batch_create(n, cfgs, None, C.byref(h))
    assert st == ERX_ENOMEM and not h.value
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


def test_two_contexts_do_not_interfere():
    """Two detectors on different cubes and shapes, pushes interleaved line by
    line, give the same bits as each run alone."""
    need_gpu()
    from paper_2408_14947_gb300 import Detector
    a = synth.gen_lines(synth.dn_c2(width=130, bands=24, seed=3), 0, 8)
    b = synth.gen_lines(synth.dn_c2(width=77, bands=40, seed=4), 0, 8).astype(np.float32)
    ra, _ = run_gpu(a, in_bits=12, warmup=2, push_sizes=[1] * 8)
    rb, _ = run_gpu(b, form="fp32", warmup=2, push_sizes=[1] * 8)
    da = Detector(24, 130, in_dtype="u16", in_bits=12, warmup=2)
    db = Detector(40, 77, in_dtype="f32", form="fp32", warmup=2)
    xa, xb = to_dev(a), to_dev(b)
    oa, ob = [], []
    for t in range(8):
        oa.append(da.push(xa[t:t + 1])[0])
        ob.append(db.push(xb[t:t + 1])[0])
    da.sync()
    db.sync()
    assert np.array_equal(torch.cat(oa).cpu().numpy(), ra["delta"])
    assert np.array_equal(torch.cat(ob).cpu().numpy(), rb["delta"])
    da.close()
    db.close()


def test_nan_input_propagates_and_is_reported():
    """A NaN sample in line 3 makes that line's statistics, factor and scores
    NaN; the bad pivot is reported as ERX_ENOTPD with line 3 (the first one),
    and the lines before it are untouched."""
    need_gpu()
    from paper_2408_14947_gb300 import Detector, ErxError, ERX_ENOTPD
    cube = synth.gen_lines(synth.dn_c2(width=64, bands=8, seed=6), 0, 6).astype(np.float32)
    ref = oracle.run_cube(cube[:3].astype(np.float64), warmup=0)
    cube[3, 10, 2] = np.nan
    det = Detector(8, 64, in_dtype="f32", warmup=0)
    out = det.push(to_dev(cube))
    with pytest.raises(ErxError) as ei:
        det.sync()
    assert ei.value.status == ERX_ENOTPD and ei.value.bad_line == 3
    d = out[0].cpu().numpy()
    assert rel_err(d[:3], ref["delta"]) < 1e-9
    assert np.all(np.isnan(d[3]))
    det.close()
