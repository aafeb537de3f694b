"""Batched form: independent streams with uneven widths and band counts, one
line each per step, through one graph-replayed set of phase kernels (GPU).

Each stream of a batch must give the same bits as its own context pushed line
by line (the batch runs the same kernel bodies), and match the oracle."""
import json

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, rel_err, run_gpu, torch

pytestmark = pytest.mark.gpu

SHAPES = [(130, 8), (200, 16), (150, 64), (77, 108), (260, 224), (64, 33), (2, 5)]
STEPS = 6


def _cubes(seed=0):
    out = []
    for s, (w, b) in enumerate(SHAPES):
        cfg = synth.SceneConfig(bands=b, width=w, seed=seed, stream=s, n_end=(3, 5),
                                noise=0.01, scene_lines=3, drift=0.05)
        out.append(synth.gen_lines(cfg, 0, STEPS))
    return out


def _run_batch(form, cubes, warmup=2):
    from paper_2408_14947_gb300 import Batch
    b = Batch([{"bands": bb, "width": w, "warmup": warmup} for (w, bb) in SHAPES], form=form)
    dev = [torch.from_numpy(c).cuda() for c in cubes]
    outs = [[] for _ in SHAPES]
    for t in range(STEPS):
        b.push([x[t] for x in dev])
        b.sync()
        for i in range(len(SHAPES)):
            v = b.views(i)
            outs[i].append([v[1].cpu().numpy().copy(), v[2].cpu().numpy().copy(),
                            v[3].cpu().numpy().copy(), v[4].cpu().numpy().copy()])
    return b, outs


@pytest.mark.parametrize("form", ["fp64", "fp32", "tf32", "bf16", "tf32x3"])
def test_batch_matches_single_stream_contexts(form):
    need_gpu()
    cubes = _cubes()
    b, outs = _run_batch(form, cubes)
    for i, c in enumerate(cubes):
        # the batch takes line statistics with the FP32 SIMT scatter in every
        # non-FP64 form; the contexts are asked for the same
        ref, det = run_gpu(c, form=form, warmup=2, push_sizes=[1] * STEPS, simt_stats=True)
        got_d = np.stack([o[0] for o in outs[i]])
        got_n = np.stack([o[1] for o in outs[i]])
        assert np.array_equal(got_d, ref["delta"]), (form, SHAPES[i])
        assert np.array_equal(got_n, ref["delta_n"]), (form, SHAPES[i])
        assert np.array_equal(np.stack([o[3] for o in outs[i]])[:, 0].astype(bool),
                              ref["detecting"])
        tb, mub, kb = b.state(i)
        td, mud, kd = det.state()
        assert tb == td == STEPS and np.array_equal(kb, kd)
    b.close()


# These streams switch scene every 3 lines; K_t + ridge I reaches condition
# numbers of 1e5 .. 1e6 (few materials against 0.01 noise, and 224 bands over
# only 260 px).  FP32 and 3xTF32 hold the 1e-4 bar there (the kappa sweep gives
# 5e-5 at 1e6 with the compensated scatter).  TF32 and BF16 round the score's
# operands: each pixel is held to the first-order bound of that rounding, 2 u c
# with c the componentwise condition of L^{-1} r from the oracle's factor
# (tests/rounding.py), plus 10 % and 1e-4 for the FP32 scatter and inverse.  The
# bit-for-bit check against single-stream contexts above is the exact test of
# the batched path.
U_SCORE = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.mark.parametrize("form,tol", [("fp64", 1e-9), ("fp32", 1e-4), ("tf32", None),
                                      ("bf16", None), ("tf32x3", 1e-4)])
def test_batch_matches_oracle(form, tol):
    need_gpu()
    from tests.rounding import score_condition
    cubes = _cubes(seed=1)
    b, outs = _run_batch(form, cubes)
    for i, c in enumerate(cubes):
        ref = oracle.run_cube(c.astype(np.float64), warmup=2)
        got = np.stack([o[0] for o in outs[i]]).astype(np.float64)
        if tol is not None:
            assert rel_err(got, ref["delta"]) <= tol, (form, SHAPES[i])
        else:
            cond = score_condition(c.astype(np.float64), warmup=2)
            err = np.abs(got - ref["delta"]) / ref["delta"]
            bound = 2.2 * U_SCORE[form] * cond + 1e-4
            assert np.all(err <= bound), (form, SHAPES[i], float(np.max(err / bound)))
    b.close()


def test_batch_autotune_and_cache(tmp_path):
    need_gpu()
    from paper_2408_14947_gb300 import Batch, ErxError, ERX_ESTATE
    cubes = _cubes(seed=2)
    dev = [torch.from_numpy(c).cuda() for c in cubes]
    cache = str(tmp_path / "tune.json")
    b = Batch([{"bands": bb, "width": w} for (w, bb) in SHAPES], form="tf32")
    with pytest.raises(ErxError) as ei:
        b.tune(reps=2, cache_path=cache)          # needs one step first
    assert ei.value.status == ERX_ESTATE
    b.push([x[0] for x in dev])
    b.tune(reps=2, cache_path=cache)
    routes = [b.route(i) for i in range(len(SHAPES))]
    assert all(r in (1, 2) for r in routes)
    data = json.load(open(cache))
    assert len(data) >= len({bb for _, bb in SHAPES})
    for t in range(1, STEPS):
        b.push([x[t] for x in dev])
    b.sync()
    # tuning leaves the state alone: the last scores match the oracle over lines
    # 0 .. STEPS-1 (tolerance as in test_batch_matches_oracle for TF32)
    for i, c in enumerate(cubes):
        ref = oracle.run_cube(c.astype(np.float64))
        got = b.views(i)[1].cpu().numpy()
        assert rel_err(got, ref["delta"][-1]) <= 2e-2
    # a second batch with the same shapes reuses the cached choices
    b2 = Batch([{"bands": bb, "width": w} for (w, bb) in SHAPES], form="tf32")
    b2.push([x[0] for x in dev])
    b2.tune(reps=2, cache_path=cache)
    assert [b2.route(i) for i in range(len(SHAPES))] == routes
    b.close()
    b2.close()


# Learned streams (codes of one shared encoder) mixed with plain streams: the
# batch runs one encoder forward over all learned streams' pixels, then the
# same phase kernels on the codes.
LEARNED = [(130, 40, True), (96, 16, False), (77, 40, True), (256, 40, True), (50, 64, False)]


def _learned_setup(seed=3):
    from paper_2408_14947_gb300 import Encoder
    enc = Encoder(40, 24, 8, seed=seed)
    cubes = []
    for s, (w, bb, _) in enumerate(LEARNED):
        cfg = synth.SceneConfig(bands=bb, width=w, seed=seed, stream=s, n_end=(3, 5),
                                noise=0.01, scene_lines=3, drift=0.05)
        cubes.append(synth.gen_lines(cfg, 0, STEPS))
    flat = np.concatenate([c.reshape(-1, 40) for c, (_, bb, lr) in zip(cubes, LEARNED) if lr])
    enc.set_norm(flat.mean(0), 1.0 / (flat.std(0) + 1e-3))
    return enc, cubes


@pytest.mark.parametrize("form", ["fp64", "fp32", "bf16"])
def test_batch_learned_streams_match_contexts(form):
    need_gpu()
    from paper_2408_14947_gb300 import Batch
    enc, cubes = _learned_setup()
    b = Batch([{"bands": bb, "width": w, "warmup": 2, "learned": lr} for (w, bb, lr) in LEARNED],
              form=form, encoder=enc)
    assert [b.dim(i) for i in range(len(LEARNED))] == [8, 16, 8, 8, 64]
    dev = [torch.from_numpy(c).cuda() for c in cubes]
    got = [[] for _ in LEARNED]
    for t in range(STEPS):
        b.push([x[t] for x in dev])
        b.sync()
        for i in range(len(LEARNED)):
            v = b.views(i)
            got[i].append([v[1].cpu().numpy().copy(), v[2].cpu().numpy().copy()])
    for i, (c, (w, bb, lr)) in enumerate(zip(cubes, LEARNED)):
        kw = {"encoder": enc} if lr else {}
        ref, det = run_gpu(c, form=form, warmup=2, push_sizes=[1] * STEPS, simt_stats=True, **kw)
        assert np.array_equal(np.stack([g[0] for g in got[i]]), ref["delta"]), (form, i)
        assert np.array_equal(np.stack([g[1] for g in got[i]]), ref["delta_n"]), (form, i)
        tb, mub, kb = b.state(i)
        td, mud, kd = det.state()
        assert tb == td == STEPS and kb.shape == kd.shape and np.array_equal(kb, kd)
        det.close()
        if lr and form == "fp64":
            # and the oracle on the codes the encoder gives for these lines
            codes = enc.forward(torch.from_numpy(c.reshape(-1, bb)).cuda()).cpu().numpy()
            ref_o = oracle.run_cube(codes.astype(np.float64).reshape(STEPS, w, -1), warmup=2)
            assert rel_err(np.stack([g[0] for g in got[i]]), ref_o["delta"]) < 1e-9
    b.close()
    enc.close()


def test_batch_learned_needs_matching_encoder():
    need_gpu()
    import ctypes as C

    from paper_2408_14947_gb300 import Batch, Encoder, ERX_EINVAL
    from paper_2408_14947_gb300.erx import load_library
    enc, cubes = _learned_setup()
    lib = load_library()
    b = Batch([{"bands": 40, "width": 64, "learned": True}], form="fp32", encoder=enc)
    for other in (Encoder(40, 24, 6, seed=1), Encoder(32, 24, 8, seed=1)):
        # another code count or band count than the batch's learned streams
        assert lib.erx_batch_set_encoder(C.c_void_p(b.b), C.c_void_p(other.e)) == ERX_EINVAL
        other.close()
    b.close()
    # a batch without learned streams takes no encoder
    p = Batch([{"bands": 16, "width": 64}], form="fp32")
    assert lib.erx_batch_set_encoder(C.c_void_p(p.b), C.c_void_p(enc.e)) == ERX_EINVAL
    p.close()
    enc.close()


def test_tuned_fp64_batch_keeps_its_bits(tmp_path):
    """The FP64 autotuner picks factor schedules and score layouts that give the
    same bits: a tuned batch and its contexts agree exactly over the following
    steps, and the choices are cached per band count."""
    need_gpu()
    from paper_2408_14947_gb300 import Batch
    cubes = _cubes(seed=3)
    dev = [torch.from_numpy(c).cuda() for c in cubes]
    cache = str(tmp_path / "tune64.json")
    b = Batch([{"bands": bb, "width": w, "warmup": 2} for (w, bb) in SHAPES], form="fp64")
    b.push([x[0] for x in dev])
    b.tune(reps=2, cache_path=cache)
    outs = [[b.views(i)[1].cpu().numpy().copy()] for i in range(len(SHAPES))]
    for t in range(1, STEPS):
        b.push([x[t] for x in dev])
        b.sync()
        for i in range(len(SHAPES)):
            outs[i].append(b.views(i)[1].cpu().numpy().copy())
    for i, c in enumerate(cubes):
        ref, _ = run_gpu(c, form="fp64", warmup=2, push_sizes=[1] * STEPS)
        assert np.array_equal(np.stack(outs[i]), ref["delta"]), SHAPES[i]
    data = json.load(open(cache))
    for _, bb in SHAPES:
        assert any(k.endswith("|factor") and f"|d{bb}|" in k for k in data), bb
        assert any(k.endswith("|fp64layout") and f"|d{bb}|" in k for k in data), bb
    b.close()
