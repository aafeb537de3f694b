"""CUDA path vs the FP64 CPU oracle, element by element (GPU).

Tolerances: the FP64 form must match to 1e-9 relative on delta (rounding
order only); the FP32 form to 1e-4 relative (float accumulation over p pixels
and d bands with FP64 state and factor).  delta_N is checked against the
bound that the delta tolerance implies, and the mask wherever the oracle's
delta_N is not within that bound of the threshold.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import dn_err, need_gpu, rel_err, run_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp64e": 1e-9, "fp32": 1e-4, "tf32": 5e-3, "bf16": 4e-2, "tf32x3": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _compare(got, ref, tol, thr=3.0):
    assert np.all(np.isfinite(got["delta"]))
    e = rel_err(got["delta"], ref["delta"])
    assert e <= tol, f"delta rel err {e} > {tol}"
    e_n = dn_err(got["delta_n"], ref["delta"], ref["delta_n"])
    assert e_n <= 4 * tol, f"delta_N err {e_n}"
    assert np.array_equal(got["detecting"], ref["detecting"])
    if "mask" in ref:
        m = ref["delta_n"]
        sure = np.abs(m - thr) > 4 * tol * (np.abs(m) + 10)
        assert np.array_equal(got["mask"][sure], ref["mask"][sure])


CASES = [
    # name, cube factory, detector kwargs
    ("c1_f32_full", lambda: synth.gen_lines(synth.reflectance_c1(width=150, bands=64), 0, 30), {}),
    ("c2_u16_int", lambda: synth.gen_lines(synth.dn_c2(width=200, bands=108), 0, 24),
     {"in_bits": 12}),
    ("c2_u16_16bit", lambda: synth.gen_lines(synth.dn_c2(width=77, bands=20), 0, 9),
     {"in_bits": 16}),
    ("c2_u16_srp5", lambda: synth.gen_lines(synth.dn_c2(width=130, bands=108), 0, 20),
     {"proj": "srp", "proj_dim": 5, "seed": 11}),
    ("c1_f32_srp7", lambda: synth.gen_lines(synth.reflectance_c1(width=99, bands=40), 0, 15),
     {"proj": "srp", "proj_dim": 7, "seed": 2}),
    ("c3_f64_k1e3", lambda: synth.gen_lines(synth.cov_c3(1e3, width=70, bands=33), 0, 6)
     .astype(np.float64), {}),
    ("stu_order", lambda: synth.gen_lines(synth.reflectance_c1(width=65, bands=12), 0, 11),
     {"order": "score_then_update"}),
    ("alpha1", lambda: synth.gen_lines(synth.reflectance_c1(width=64, bands=9), 0, 5),
     {"momentum": 1.0}),
    ("tiny_w2_b1", lambda: synth.gen_lines(synth.reflectance_c1(width=2, bands=1), 0, 7), {}),
]


def _oracle_kw(kw, cube):
    o = {k: v for k, v in kw.items() if k in ("momentum", "ridge", "warmup", "order",
                                              "proj", "proj_dim", "seed")}
    o["threshold"] = 3.0
    return o


@pytest.mark.parametrize("form", ["fp64", "fp32"])
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_parity(name, make, kw, form):
    cube = make()
    got, det = run_gpu(cube, form=form, warmup=3, threshold=3.0, **kw)
    ref = oracle.run_cube(cube, warmup=3, **_oracle_kw(kw, cube))
    tol = TOL[form]
    if form == "fp32" and name == "tiny_w2_b1":
        tol = 1e-5
    _compare(got, ref, tol)
    t, mu, k = det.state()
    assert t == cube.shape[0]
    st = ref["state"]
    assert rel_err(mu, st[1]) < (1e-12 if form == "fp64" else 1e-5)
    det.close()


def test_blocks_and_single_lines_agree():
    """Pushing line by line, in ragged blocks, or all at once gives identical
    bits: per-line arithmetic does not depend on the blocking."""
    cube = synth.gen_lines(synth.dn_c2(width=100, bands=30), 0, 23)
    a, _ = run_gpu(cube, in_bits=12)
    b, _ = run_gpu(cube, in_bits=12, push_sizes=[1] * 23)
    c, _ = run_gpu(cube, in_bits=12, block_lines=5, push_sizes=[7, 9, 7])
    for k in ("delta", "delta_n", "mask", "detecting"):
        assert np.array_equal(a[k], b[k]) and np.array_equal(a[k], c[k]), k


def test_state_roundtrip_and_resume():
    cube = synth.gen_lines(synth.reflectance_c1(width=80, bands=16), 0, 20)
    full, det = run_gpu(cube)
    from paper_2408_14947_gb300 import Detector
    from tests.gpu_util import to_dev
    d1 = Detector(16, 80)
    d1.push(to_dev(cube[:12]))
    t, mu, k = d1.state()
    d2 = Detector(16, 80)
    d2.set_state(t, mu, k)
    out = d2.push(to_dev(cube[12:]))
    d2.sync()
    assert np.array_equal(out[0].cpu().numpy(), full["delta"][12:])
    assert d2.state()[0] == 20


def test_exact_rational_golden_on_gpu():
    import json
    import os
    from fractions import Fraction as F
    path = os.path.join(os.path.dirname(__file__), "golden", "erx_exact_tiny.json")
    for c in json.load(open(path))["cases"]:
        if c["proj"] is not None or F(c["ridge"]) == 0:
            continue
        cube = np.array(c["cube"], dtype=np.float64)
        got, _ = run_gpu(cube, momentum=float(F(c["alpha"])), ridge=float(F(c["ridge"])),
                         order=c["order"])
        exact = np.array([[float(F(v)) for v in line] for line in c["delta2"]])
        assert rel_err(got["delta"] ** 2, exact) < 1e-9, c["name"]


def test_max_dim_224():
    cube = synth.gen_lines(synth.cov_c3(1e4, width=300, bands=224), 0, 3)
    got, _ = run_gpu(cube, warmup=0)
    ref = oracle.run_cube(cube, warmup=0, threshold=3.0)
    _compare(got, ref, 1e-9)


def test_empty_push_is_noop():
    from paper_2408_14947_gb300 import Detector
    det = Detector(4, 8)
    x = torch.zeros((0, 8, 4), dtype=torch.float32, device="cuda")
    det.push(x)
    det.sync()
    assert det.state()[0] == 0


def test_not_positive_definite_reports_line():
    """ridge 0 and a constant line: K_hat = 0, the first pivot is 0 (Sec. III-D
    motivates the ridge with exactly this failure)."""
    from paper_2408_14947_gb300 import Detector, ErxError, ERX_ENOTPD
    cube = np.ones((3, 10, 4), np.float32)
    det = Detector(4, 10, ridge=0.0)
    det.push(torch.from_numpy(cube).cuda())
    with pytest.raises(ErxError) as ei:
        det.sync()
    assert ei.value.status == ERX_ENOTPD and ei.value.bad_line == 0
    det.sync()  # cleared


def test_range_check_u16():
    from paper_2408_14947_gb300 import Detector, ErxError, ERX_ERANGE
    cube = synth.gen_lines(synth.dn_c2(width=20, bands=6), 0, 4)
    cube[2, 5, 3] = 5000
    det = Detector(6, 20, in_dtype="u16", in_bits=12)
    det.push(torch.from_numpy(cube.view(np.int16)).cuda())
    with pytest.raises(ErxError) as ei:
        det.sync()
    assert ei.value.status == ERX_ERANGE and ei.value.bad_line == 2


def test_projection_matches_oracle_draw():
    from paper_2408_14947_gb300 import Detector
    det = Detector(108, 16, proj="srp", proj_dim=5, seed=42)
    assert np.array_equal(det.projection(), oracle.srp_weights(108, 5, 42))


def test_host_buffers_match_device_path():
    cube = synth.gen_lines(synth.dn_c2(width=90, bands=20), 0, 17)
    dev, _ = run_gpu(cube, in_bits=12, block_lines=4)
    from paper_2408_14947_gb300 import Detector
    det = Detector(20, 90, in_dtype="u16", in_bits=12, block_lines=4)
    n = cube.shape[0]
    x = torch.from_numpy(cube.view(np.int16))
    outs = (torch.empty((n, 90), dtype=torch.float64), torch.empty((n, 90), dtype=torch.float64),
            torch.empty((n, 90), dtype=torch.uint8), torch.empty((n,), dtype=torch.uint8))
    det.push_host(x, outs)
    assert np.array_equal(outs[0].numpy(), dev["delta"])
    assert np.array_equal(outs[1].numpy(), dev["delta_n"])
    xp = x.pin_memory()
    det.reset()
    det.push_host(xp, outs)
    assert np.array_equal(outs[0].numpy(), dev["delta"])


def test_planted_anomaly_ranking_fp32_matches_fp64():
    """Ordered list of planted anomalies by delta_N is the same in both forms
    and in the oracle (ties within tolerance excepted)."""
    cfg = synth.dn_c2(width=256, bands=64, seed=5)
    cube = synth.gen_lines(cfg, 0, 60)
    m = synth.anomaly_mask(cfg, 0, 60)
    ref = oracle.run_cube(cube)
    for form in ("fp64", "fp32"):
        got, _ = run_gpu(cube, form=form, in_bits=12)
        o = np.argsort(-ref["delta_n"][m], kind="stable")
        g = np.argsort(-got["delta_n"][m], kind="stable")
        rv = ref["delta_n"][m][o]
        same = o == g
        close = np.abs(np.diff(rv, append=-np.inf)) < 1e-3
        assert np.all(same | close | np.roll(close, 1))


# relative gap below which two planted anomalies count as tied: a few times
# each form's stated error bar
RANK_TIES = [("fp64e", 1e-6), ("tf32x3", 1e-3), ("tf32", 2e-2), ("bf16", 0.15)]


@pytest.mark.parametrize("form,tie", RANK_TIES)
def test_planted_anomaly_ranking_every_form(form, tie):
    """For every pair of planted anomalies that the oracle orders clearly (delta_N
    apart by more than `tie` relative), the form orders them the same way: the
    ranking is the oracle's up to ties."""
    cfg = synth.dn_c2(width=256, bands=64, seed=5)
    cube = synth.gen_lines(cfg, 0, 60)
    m = synth.anomaly_mask(cfg, 0, 60)
    ref = oracle.run_cube(cube)["delta_n"][m]
    got = run_gpu(cube, form=form, in_bits=12)[0]["delta_n"][m].astype(np.float64)
    assert m.sum() >= 10
    gap = ref[:, None] - ref[None, :]
    scale = np.maximum(np.maximum(np.abs(ref[:, None]), np.abs(ref[None, :])), 1.0)
    clear = gap > tie * scale                       # oracle: i clearly above j
    agree = (got[:, None] - got[None, :]) > 0
    assert np.all(agree[clear]), (form, int((~agree[clear]).sum()))


@pytest.mark.parametrize("width,bands", [(640, 108), (2048, 127), (65, 1), (130, 16), (2, 5)])
def test_tensor_core_stats_match_integer_route_bitwise(width, bands):
    """The tcgen05 exact-integer SYRK (bf16 6-bit split, FP32 accumulation in
    TMEM) gives the same sums as the 32-bit integer route, hence identical
    scores, state and flags (from lines of two pixels, the fewest a line
    covariance needs, to 2048)."""
    cube = synth.gen_lines(synth.dn_c2(width=width, bands=bands, seed=9), 0, 9)
    a, da = run_gpu(cube, in_bits=12, warmup=2)
    b, db = run_gpu(cube, in_bits=12, warmup=2, simt_stats=True)
    for k in ("delta", "delta_n", "mask", "detecting"):
        assert np.array_equal(a[k], b[k]), k
    sa, sb = da.state(), db.state()
    assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])
    ka = da.profile_read()
    assert ka["stats_tc"][2] > 0 and ka["stats_int"][2] == 0
    kb = db.profile_read()
    assert kb["stats_tc"][2] == 0 and kb["stats_int"][2] > 0


def test_tensor_core_stats_range_check():
    from paper_2408_14947_gb300 import Detector, ErxError, ERX_ERANGE
    cube = synth.gen_lines(synth.dn_c2(width=100, bands=10), 0, 5)
    cube[3, 7, 2] = 4096
    det = Detector(10, 100, in_dtype="u16", in_bits=12)
    det.push(torch.from_numpy(cube.view(np.int16)).cuda())
    with pytest.raises(ErxError) as ei:
        det.sync()
    assert ei.value.status == ERX_ERANGE and ei.value.bad_line == 3
    assert det.profile_read()["stats_tc"][2] > 0


# name, cube factory, detector kwargs, whether S2 takes the tensor-core scatter
# (float lines, d > 16, p * d a multiple of 4)
TC_CASES = [
    ("c2_u16", lambda: synth.gen_lines(synth.dn_c2(width=300, bands=108), 0, 12), {"in_bits": 12},
     False),
    ("c1_f32", lambda: synth.gen_lines(synth.reflectance_c1(width=200, bands=64), 0, 10), {},
     True),
    ("c3_k1e3_d224", lambda: synth.gen_lines(synth.cov_c3(1e3, width=260, bands=224), 0, 3), {},
     True),
    ("c3_d130_w100", lambda: synth.gen_lines(synth.cov_c3(1e2, width=100, bands=130), 0, 4), {},
     True),
    ("c1_d40_w77", lambda: synth.gen_lines(synth.reflectance_c1(width=77, bands=40), 0, 6), {},
     True),
    ("ragged_d33", lambda: synth.gen_lines(synth.reflectance_c1(width=129, bands=33), 0, 6), {},
     False),
    ("srp5", lambda: synth.gen_lines(synth.dn_c2(width=140, bands=108), 0, 8),
     {"proj": "srp", "proj_dim": 5, "seed": 3}, False),
]


@pytest.mark.parametrize("form", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("name,make,kw,syrk", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_tensor_core_forms(name, make, kw, syrk, form):
    cube = make()
    got, det = run_gpu(cube, form=form, warmup=2, threshold=3.0, **kw)
    ref = oracle.run_cube(cube, warmup=2, **_oracle_kw(kw, cube))
    e = rel_err(got["delta"], ref["delta"])
    print(f"{name} {form}: max rel delta err {e:.3e}")
    assert e <= TOL[form], f"{name} {form}: {e}"
    prof = det.profile_read()
    assert prof["solve_tc"][2] > 0
    # the 3xTF32 form keeps S2 in FP32 SIMT
    assert (prof["syrk_tc"][2] > 0) == (syrk and form != "tf32x3")


@pytest.mark.parametrize("form,tol", [("tf32", 1.2e-3), ("bf16", 8e-3)])
@pytest.mark.parametrize("width,bands", [(200, 64), (260, 224), (77, 40), (64, 130)])
def test_tensor_core_scatter_matches_simt(form, tol, width, bands):
    """S2 on the tensor cores against the FP32 SIMT scatter, line by line
    (momentum 1: the state K is the last line's K_hat).  Each centred sample
    is rounded once (TF32: 2^-11, BF16: 2^-8 relative), so
    |dK_ab| <= 2 u sqrt(K_aa K_bb) plus FP32 accumulation."""
    cube = synth.gen_lines(synth.cov_c3(1e3, width=width, bands=bands, seed=5), 0, 3)
    for t in range(cube.shape[0]):
        _, d_tc = run_gpu(cube[t:t + 1], form=form, warmup=0, momentum=1.0)
        _, d_simt = run_gpu(cube[t:t + 1], form=form, warmup=0, momentum=1.0, simt_stats=True)
        assert d_tc.profile_read()["syrk_tc"][2] > 0
        assert d_simt.profile_read()["syrk_tc"][2] == 0
        k_tc, k_simt = d_tc.state()[2], d_simt.state()[2]
        dg = np.sqrt(np.diag(k_simt))
        e = np.max(np.abs(k_tc - k_simt) / np.outer(dg, dg))
        print(f"{form} {width}x{bands} line {t}: scatter err {e:.2e}")
        assert e <= tol, (form, width, bands, t, e)


def test_long_block_chunked_ema_matches_line_by_line():
    """Blocks longer than one EMA chunk (32 lines) chain chunk results in closed
    form; they agree with line-by-line pushes to rounding and with the oracle."""
    cube = synth.gen_lines(synth.reflectance_c1(width=70, bands=12), 0, 150)
    a, da = run_gpu(cube, block_lines=150)
    b, db = run_gpu(cube, push_sizes=[1] * 150)
    assert rel_err(a["delta"], b["delta"]) < 1e-12
    ref = oracle.run_cube(cube)
    assert rel_err(a["delta"], ref["delta"]) < 1e-9
    ta, ma, ka = da.state()
    tb, mb, kb = db.state()
    assert ta == tb == 150 and rel_err(ka, kb) < 1e-12
    for order in ("score_then_update",):
        c, _ = run_gpu(cube, block_lines=150, order=order)
        refc = oracle.run_cube(cube, order=order)
        assert rel_err(c["delta"], refc["delta"]) < 1e-9


# the cube's pooled covariance has kappa 1.1e4 .. 2e4; with the FP32 scatter
# compensated per 8-pixel run the FP32 scores sit near 1e-5 here (8e-5 to 1.05e-4
# with a plain running FP32 sum, which is what once needed a wider tolerance)
@pytest.mark.parametrize("form,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
@pytest.mark.parametrize("order", ["update_then_score", "score_then_update"])
def test_imc_matches_oracle(form, tol, order):
    """IMC averaging (Sec. IV-C ablation): a 70-line block (three chunks of the
    prefix sum), one single line and a 9-line block, against the oracle; the
    state is the pooled mean and covariance of every pixel seen."""
    cube = synth.gen_lines(synth.reflectance_c1(width=96, bands=24, seed=4), 0, 80)
    kw = {"averaging": "imc", "order": order}
    ref = oracle.run_cube(cube, warmup=3, threshold=3.0, **kw)
    got, det = run_gpu(cube, form=form, warmup=3, threshold=3.0, push_sizes=[70, 1, 9], **kw)
    _compare(got, ref, tol)
    t, mu, k = det.state()
    _, mu_o, k_o = ref["state"]
    assert t == 80
    # the FP32 form's line means sum runs of 8 samples in FP32 (relative 1e-7)
    tol_s = 1e-10 if form == "fp64" else 1e-6
    assert rel_err(mu, mu_o) < tol_s and rel_err(k, k_o) < tol_s


def test_imc_integer_statistics():
    """IMC on u16 lines through the exact integer statistics."""
    cube = synth.gen_lines(synth.dn_c2(width=64, bands=16, seed=2), 0, 40)
    ref = oracle.run_cube(cube, warmup=2, threshold=3.0, averaging="imc")
    got, det = run_gpu(cube, warmup=2, threshold=3.0, in_bits=12, averaging="imc",
                       push_sizes=[40])
    _compare(got, ref, 1e-9)
    assert det.profile_read()["stats_tc"][2] > 0


@pytest.mark.parametrize("form", ["fp64", "fp32", "tf32"])
def test_pipelined_score_then_update_is_bitwise_plain(form):
    """ERX_FLAG_PIPELINE: single-line pushes scored against the factor made at
    the end of the previous push, the update deferred to a second stream, give
    the same bits as score-then-update without it; interleaved block pushes and
    a set_state in mid-stream take the ordinary path and refactor."""
    cube = synth.gen_lines(synth.reflectance_c1(width=96, bands=24, seed=6), 0, 40)
    sizes = [1] * 12 + [5] + [1] * 23
    kw = dict(form=form, warmup=2, threshold=3.0, order="score_then_update")
    plain, dp = run_gpu(cube, push_sizes=sizes, **kw)
    piped, dq = run_gpu(cube, push_sizes=sizes, pipeline=True, **kw)
    for k in ("delta", "delta_n", "mask", "detecting"):
        assert np.array_equal(plain[k], piped[k]), k
    sp, sq = dp.state(), dq.state()
    assert sp[0] == sq[0] == 40 and np.array_equal(sp[1], sq[1]) and np.array_equal(sp[2], sq[2])
    ref = oracle.run_cube(cube, warmup=2, threshold=3.0, order="score_then_update")
    # the first lines are scored against one line's covariance, kappa 2.4e4 here:
    # inside the FP32 bar's range (1e-4 up to 1e6), above the TF32 bar's (5e-3 up
    # to 1e4; the kappa sweep gives TF32 5.0e-3 at 1e5)
    _compare(piped, ref, {"fp64": 1e-9, "fp32": 1e-4, "tf32": 2e-2}[form])
    # resume from a saved state: the next line takes the ordinary path
    x = to_dev(cube)
    dq.set_state(*sp)
    dp.set_state(*sp)
    for t in range(35, 40):
        a, b = dp.push(x[t:t + 1]), dq.push(x[t:t + 1])
        dp.sync(), dq.sync()
        assert torch.equal(a[0], b[0])


def test_pipeline_flag_needs_score_then_update():
    from paper_2408_14947_gb300 import Detector, ErxError
    with pytest.raises(ErxError):
        Detector(8, 16, order="update_then_score", pipeline=True)


@pytest.mark.parametrize("order", ["update_then_score", "score_then_update"])
def test_pooled_warmup_matches_oracle(order):
    """Pooled reading of the warm-up buffer: IMC over the 40 warm-up lines, the
    EMAs afterwards; the second push straddles the switch (its 20 lines are
    scanned in two parts), the first spans two 32-line chunks."""
    cube = synth.gen_lines(synth.reflectance_c1(width=80, bands=20, seed=8), 0, 80)
    kw = {"averaging": "pooled", "order": order}
    ref = oracle.run_cube(cube, warmup=40, threshold=3.0, momentum=0.2, **kw)
    got, det = run_gpu(cube, warmup=40, threshold=3.0, momentum=0.2, push_sizes=[33, 20, 1, 26],
                       **kw)
    _compare(got, ref, 1e-9)
    _, mu, k = det.state()
    _, mu_o, k_o = ref["state"]
    assert rel_err(mu, mu_o) < 1e-10 and rel_err(k, k_o) < 1e-10



FP64E_CASES = [
    ("c2_u16_108", lambda: synth.gen_lines(synth.dn_c2(width=200, bands=108), 0, 24),
     {"in_bits": 12}),
    ("c1_f32_ragged", lambda: synth.gen_lines(synth.reflectance_c1(width=77, bands=41), 0, 12), {}),
    ("c3_k1e4_d224", lambda: synth.gen_lines(synth.cov_c3(1e4, width=100, bands=224), 0, 3), {}),
    ("tiny_w2_b1", lambda: synth.gen_lines(synth.reflectance_c1(width=2, bands=1), 0, 7), {}),
    ("stu_order", lambda: synth.gen_lines(synth.reflectance_c1(width=65, bands=12), 0, 11),
     {"order": "score_then_update"}),
]


@pytest.mark.parametrize("name,make,kw", FP64E_CASES, ids=[c[0] for c in FP64E_CASES])
def test_fp64e_matches_oracle(name, make, kw):
    """FP64E: FP64 statistics, state and factor, the score in double-float on
    the FP32 pipe, held to the FP64 bar; blocks and single lines."""
    cube = make()
    ref = oracle.run_cube(cube, warmup=3, **_oracle_kw(kw, cube))
    for sizes in (None, [1] * cube.shape[0]):
        got, det = run_gpu(cube, form="fp64e", warmup=3, threshold=3.0, push_sizes=sizes, **kw)
        _compare(got, ref, TOL["fp64e"])
        assert det.profile_read()["solve_df"][2] > 0


def test_fp64e_pipelined():
    cube = synth.gen_lines(synth.dn_c2(width=96, bands=40, seed=4), 0, 20)
    kw = dict(form="fp64e", warmup=2, threshold=3.0, order="score_then_update", in_bits=12,
              push_sizes=[1] * 20)
    a, _ = run_gpu(cube, **kw)
    b, _ = run_gpu(cube, pipeline=True, **kw)
    assert np.array_equal(a["delta"], b["delta"])
    _compare(b, oracle.run_cube(cube, warmup=2, threshold=3.0, order="score_then_update"), 1e-9)


def test_fp64e_rejects_projection_and_f64():
    from paper_2408_14947_gb300 import Detector, ErxError
    with pytest.raises(ErxError):
        Detector(16, 32, form="fp64e", proj="srp", proj_dim=4)
    with pytest.raises(ErxError):
        Detector(16, 32, form="fp64e", in_dtype="f64")


@pytest.mark.parametrize("form,kw", [("fp64", {}), ("fp64e", {}), ("fp32", {}), ("tf32", {}),
                                     ("bf16", {}), ("tf32x3", {}),
                                     ("fp64", {"proj": "srp", "proj_dim": 6}),
                                     ("fp32", {"averaging": "imc"})])
def test_overlapped_blocks_are_bitwise_block_pushes(form, kw):
    """One push of 40 lines in 7-line blocks runs block b+1's statistics,
    update and factor on the context's stream while a second stream scores
    block b; it gives the same bits as pushing the same blocks one call at a
    time (one stream)."""
    cube = synth.gen_lines(synth.reflectance_c1(width=96, bands=40, seed=9), 0, 40)
    kw = dict(form=form, warmup=2, threshold=3.0, block_lines=7, **kw)
    one, d1 = run_gpu(cube, **kw)
    sep, d2 = run_gpu(cube, push_sizes=[7, 7, 7, 7, 7, 5], **kw)
    for k in ("delta", "delta_n", "mask", "detecting"):
        assert np.array_equal(one[k], sep[k]), k
    s1, s2 = d1.state(), d2.state()
    assert np.array_equal(s1[1], s2[1]) and np.array_equal(s1[2], s2[2])


@pytest.mark.parametrize("bands", [57, 108, 224])
@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_cluster_factor_is_bitwise_one_cta(bands, form):
    """Lines pushed one or three at a time at d >= 48 take the factor over a
    cluster of SMs (a master CTA for the pivot chain, helper CTAs for the
    trailing panels and the inverted diagonal blocks); the same 23 lines in
    one push take the one-CTA kernels.  Same K_t (momentum 1: each line's
    statistics alone), same factor bits, hence the same scores bit for bit.
    d = 57 ends on a one-column panel and a 25-row diagonal block; d = 224 is
    the largest d and the look-ahead kernel's range; FP32 takes the float copy
    of the factor without the FP64 block inversion."""
    cube = synth.gen_lines(synth.cov_c3(1e4, width=320, bands=bands), 0, 23)
    kw = dict(form=form, warmup=0, momentum=1.0)
    one, d1 = run_gpu(cube, profile=True, **kw)
    sep, d2 = run_gpu(cube, push_sizes=[1] * 14 + [3] * 3, profile=True, **kw)
    assert d1.profile_read()["chol"][2] == 1 and d2.profile_read()["chol"][2] == 17
    for k in ("delta", "delta_n", "mask", "detecting"):
        assert np.array_equal(one[k], sep[k]), k
    ref = oracle.run_cube(cube, warmup=0, threshold=3.0, momentum=1.0)
    assert rel_err(sep["delta"], ref["delta"]) <= TOL[form]


def test_cluster_factor_not_positive_definite_reports_line():
    """ridge 0 and constant lines at d = 64 (the cluster factor): the first
    pivot is 0, the line is reported and its scores poisoned, and the next
    push still runs."""
    from paper_2408_14947_gb300 import Detector, ErxError, ERX_ENOTPD
    det = Detector(64, 80, ridge=0.0)
    det.push(torch.ones((1, 80, 64), dtype=torch.float32, device="cuda"))
    with pytest.raises(ErxError) as ei:
        det.sync()
    assert ei.value.status == ERX_ENOTPD and ei.value.bad_line == 0
    det.sync()  # cleared
