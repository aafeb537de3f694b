"""Benchmark of the ERX per-line step on one GB300 (or N replicas).

Workload (the paper's largest band count): 20000 lines x 640 px x 108 bands,
uint16 12-bit digital numbers, scenes switching every 2000 lines, 0.2 %
anomalies in 3 x 3 clusters (synthetic, seeded), FP64 form, all 108 bands
(no projection), alpha 0.1, ridge 1e-5, 99-line warm-up.  One step is one
pass of the whole line step over the whole cube from a fresh state; the cube
(2.76 GB) is resident in HBM and larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LINES, WIDTH, BANDS, BITS = 20000, 640, 108, 12
METRIC = "ERX lines/s, 640 px x 108 bands u16, FP64 form (p50/p99 line latency alongside)"
UNIT = "lines/s"
# FP64 pipe of GB300: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2070 MHz (the
# nominal 1.25 TFLOP/s FP64 rate over 152 SMs at the maximum SM clock).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# What the scalar DFMA pipe issues: 1.671 lanes per clock per SM, measured by
# pipe_probe.cu (python bench.py --pipe-probe), at the same clock.
DFMA_PIPE_GFLOPS = 152 * 1.671 * 2 * 2.070
IMAD_PEAK_GOPS = 152 * 64 * 2.070        # 32-bit integer multiply-add, per second (G)


def _gen_worker(args):
    name, shape, dtype, t0, n, kind, cfg_kw = args
    from multiprocessing import shared_memory

    import numpy as np

    import synth
    shm = shared_memory.SharedMemory(name=name)
    try:
        arr = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
        if kind == "c2":
            cfg = synth.dn_c2(**cfg_kw)
        elif kind == "c5":
            cfg = c5_config(**cfg_kw)
        else:
            cfg = synth.cov_c3(**cfg_kw)
        synth.gen_lines(cfg, t0, n, out=arr[t0:t0 + n])
    finally:
        shm.close()
    return n


def make_cube(n_lines: int, seed: int = 0, workers: int | None = None, kind: str = "c2",
              width: int = WIDTH, bands: int = BANDS, kappa: float = 1e3):
    """A seeded synthetic cube (C2-style u16 DN, or C3-style f32 with condition
    number kappa), generated in parallel by spawned processes."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np
    dtype = np.uint16 if kind == "c2" else np.float32
    shape = (n_lines, width, bands)
    nbytes = int(np.prod(shape)) * np.dtype(dtype).itemsize
    workers = workers or min(16, len(os.sched_getaffinity(0)))
    kw = {"seed": seed, "width": width, "bands": bands}
    if kind == "c3":
        kw["kappa"] = kappa
    shm = shared_memory.SharedMemory(create=True, size=nbytes)
    try:
        step = max(1, math.ceil(n_lines / (workers * 4)))
        jobs = [(shm.name, shape, dtype, t0, min(step, n_lines - t0), kind, kw)
                for t0 in range(0, n_lines, step)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            pool.map(_gen_worker, jobs)
        out = np.ndarray(shape, dtype=dtype, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return out


def c5_config(seed=0, width=1024, bands=224):
    """224-band reflectance stream with weak targets: 1 % of pixels in 3 x 3
    clusters mix a target spectrum into the background at 5-30 %."""
    import synth
    return synth.SceneConfig(bands=bands, width=width, seed=seed, n_end=(3, 5), noise=0.01,
                             scene_lines=2000, drift=0.05, anomaly_frac=0.01, cluster=3,
                             anomaly_mix=(0.05, 0.3))


def workload_config():
    """The workload every arm reports (reference and ours)."""
    return {"workload": f"C2: {LINES} lines x {WIDTH} px x {BANDS} bands u16 12-bit, "
                        f"scenes of 2000 lines, 0.2% 3x3 anomalies",
            "form": "fp64", "projection": "none (d = 108)", "alpha": 0.1,
            "l2": "inputs (2.76 GB) larger than L2; no flush"}


def max_over_ranks(value: float, device) -> float:
    """Largest value over all ranks (the slowest rank's time); identity at N = 1."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(lines_per_rank: int, world: int, ms_max: float) -> float:
    """Lines/s of the whole job: every rank's lines over the slowest rank's time."""
    return lines_per_rank * world / (ms_max / 1000.0)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(sample_lines: int, one_thread: bool = False):
    """Time the FP64 CPU oracle on the first `sample_lines` lines, in a fresh
    process with the BLAS thread count set to the usable cores."""
    cores = 1 if one_thread else len(os.sched_getaffinity(0))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import synth, oracle\n"
        "cube = synth.gen_lines(synth.dn_c2(width=%d, bands=%d), 0, %d)\n"
        "t = time.perf_counter(); oracle.run_cube(cube); dt = time.perf_counter() - t\n"
        "print(json.dumps({'lines': %d, 'seconds': dt}))\n"
    ) % (ROOT, WIDTH, BANDS, sample_lines, sample_lines)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": res["lines"] / res["seconds"], "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"first {sample_lines} lines of the {LINES}-line workload, "
                      f"{WIDTH} px x {BANDS} bands u16, FP64 NumPy oracle"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    sample = args.ref_lines
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(sample)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sample / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(workload_config(), sample_lines_per_step=sample),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_rel_err(got, ref):
    import numpy as np
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)))


def oracle_delta(cube, **kw):
    """FP64 oracle scores of cube (the parity reference for the accuracy columns)."""
    import oracle
    return oracle.run_cube(cube, **kw)["delta"]


def time_form(make, x, kw, dev, stream, reps: int = 2, ref=None):
    """lines/s of one detector configuration over the resident cube x (reset + push
    per step, one warm-up step), plus its per-kernel split.  ref: the FP64
    oracle's scores of the cube's first lines; the timed run's scores of those
    lines are compared with it (max relative delta error)."""
    import torch
    n, p, _ = x.shape
    det = make(**kw)
    sdt = torch.float64 if kw.get("form", "fp64") in ("fp64", "fp64e") else torch.float32
    out = (torch.empty((n, p), dtype=sdt, device=dev), torch.empty((n, p), dtype=sdt, device=dev),
           torch.empty((n, p), dtype=torch.uint8, device=dev),
           torch.empty((n,), dtype=torch.uint8, device=dev))
    det.reset()
    det.push(x, out)
    det.sync()
    det.profile(True)
    det.profile_read(reset=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        det.reset()
        det.push(x, out)
    b.record(stream)
    torch.cuda.synchronize()
    det.sync()
    prof = det.profile_read(reset=True)
    det.close()
    ms = a.elapsed_time(b) / reps
    # kernels_ms: event time on each kernel's own stream.  Every form but FP64
    # (and the learned one) overlaps a block's score (second stream) with the
    # next block's statistics and factor, so those times include each other's
    # share of the SMs and add up to more than ms_per_step.
    overlapped = kw.get("form", "fp64") != "fp64" and kw.get("encoder") is None
    res = {"lines_per_s": n / (ms / 1000.0), "ms_per_step": ms,
           "kernels_ms": {k: round(v[0] / reps, 3) for k, v in prof.items() if v[2]},
           "kernels_concurrent": overlapped}
    if ref is not None:
        res["max_rel_err"] = max_rel_err(out[0][:ref.shape[0]].cpu().numpy(), ref)
        res["err_lines"] = int(ref.shape[0])
    return res


def bench_batched(dev, stream, n_streams: int = 256, n_lines: int = 4, steps: int = 20):
    """One step = every stream takes one line (erx_batch_push: gather from
    resident lines + one graph launch).  lines/s counts all streams."""
    import numpy as np
    import torch

    import synth
    from paper_2408_14947_gb300 import Batch, Detector
    import oracle
    cfgs = synth.stream_configs_c4(n_streams)
    host = [synth.gen_lines(c, 0, n_lines) for c in cfgs]
    lines = [torch.from_numpy(h).to(dev) for h in host]
    shapes = [{"bands": c.bands, "width": c.width} for c in cfgs]
    out = {"workload": f"{n_streams} streams, widths U{{128..2048}}, bands from "
                       f"{{8,16,64,108,224}}, float32, {n_lines} resident lines cycled",
           "bytes_per_step": int(sum(c.width * c.bands * 4 for c in cfgs))}
    # the FP64 oracle on every stream's first lines, and the condition number of
    # each stream's ridged covariance after them
    na = ACC_LINES_BATCH
    refs, kappa = [], []
    for h in host:
        r = oracle.run_cube(h[:na], warmup=99, threshold=3.0)
        refs.append(r["delta"])
        k = r["state"][2]
        kappa.append(float(np.linalg.cond(k + 1e-5 * np.eye(k.shape[0]))))
    kappa = np.array(kappa)
    out["kappa"] = {"min": float(kappa.min()), "median": float(np.median(kappa)),
                    "max": float(kappa.max()), "streams_le_1e4": int((kappa <= 1e4).sum()),
                    "of": "K_t + ridge I after the checked lines, per stream"}
    for form in ("fp64", "fp32", "tf32", "bf16", "tf32x3"):
        b = Batch(shapes, form=form, stream=stream)
        # the first na steps are checked against the oracle (step 0 before the
        # autotuner runs, the others after it, as timed)
        errs = np.zeros(n_streams)
        for k in range(na):
            b.push([x[k] for x in lines])
            if k == 0:          # factor schedules, score kernels and FP64 layouts
                b.sync()
                b.tune(reps=3)
            b.sync()
            for i in range(n_streams):
                d_ = b.views(i)[1].cpu().numpy()
                errs[i] = max(errs[i], max_rel_err(d_, refs[i][k]))
        for k in range(na, na + 3):
            b.push([x[k % n_lines] for x in lines])
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            b.push([x[k % n_lines] for x in lines])
        e1.record(stream)
        torch.cuda.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1) / steps
        routes = sorted({b.route(i) for i in range(n_streams)})
        le = kappa <= 1e4
        out[form] = {"lines_per_s": n_streams / (ms / 1000.0), "ms_per_step": ms,
                     "routes": routes, "max_rel_err": float(errs.max()),
                     "max_rel_err_kappa_le_1e4": float(errs[le].max()) if le.any() else None,
                     "err_lines_per_stream": na}
        b.close()
    # the same lines through 256 separate single-stream contexts, one push each
    dets = [Detector(c.bands, c.width, in_dtype="f32", form="fp64", block_lines=1,
                     stream=stream) for c in cfgs]
    for k in range(2):
        for d_, x in zip(dets, lines):
            d_.push(x[k:k + 1])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(5):
        for d_, x in zip(dets, lines):
            d_.push(x[k % n_lines:k % n_lines + 1])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    out["fp64_separate_contexts"] = {"lines_per_s": n_streams / (ms / 1000.0), "ms_per_step": ms}
    for d_ in dets:
        d_.close()
    return out


def bench_learned(dev, stream, n_train: int = 2000, n_test: int = 200):
    """Train the 224 -> 128 -> 32 encoder on n_train lines x 1024 px (about 2e6
    spectra) against full-band FP64 ERX scores, then compare the learned form
    with full-band ERX and SRP-32 on held-out lines: lines/s, per-line AUC of
    the planted weak targets, rank correlation with full-band scores."""
    import numpy as np
    import torch

    import synth
    from paper_2408_14947_gb300 import Detector, Encoder, erx_train_opts_default
    W, B, K = 1024, 224, 32
    cube = make_cube(n_train + n_test, seed=11, kind="c5", width=W, bands=B)
    labels = synth.anomaly_mask(c5_config(seed=11, width=W, bands=B), n_train, n_test)
    flat = cube[:200].reshape(-1, B)
    shift, scale = flat.mean(0), 1.0 / (flat.std(0) + 1e-3)
    x = torch.from_numpy(cube).to(dev)
    held = cube[n_train:n_train + ACC_LINES_LEARNED].astype(np.float64)
    del cube, flat
    full = Detector(B, W, in_dtype="f32", form="fp64", warmup=0, stream=stream)
    fd = full.push(x)[0]
    full.sync()
    full.close()
    enc = Encoder(B, 128, K, seed=0, stream=stream)
    enc.set_norm(shift, scale)
    o = erx_train_opts_default()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    enc.train(x[:n_train], fd[:n_train], o)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    xt = x[n_train:]
    out = {"workload": f"{n_train} training lines + {n_test} held-out lines x {W} px x {B} "
                       "bands f32, weak 3x3 targets (5-30 % mixing)",
           "train_spectra": n_train * W, "train_seconds": train_s,
           "train_spectra_per_s": n_train * W / train_s}

    def auc(score, lab):
        pos, neg = score[lab], score[~lab]
        allv = np.concatenate([pos, neg])
        r = np.argsort(np.argsort(allv)) + 1.0
        return (r[:pos.size].sum() - pos.size * (pos.size + 1) / 2) / (pos.size * neg.size)

    def rank_corr(a, b):
        return np.corrcoef(np.argsort(np.argsort(a)), np.argsort(np.argsort(b)))[0, 1]

    ref = fd[n_train:].cpu().numpy()
    # FP64 oracle references for the first held-out lines: full band, SRP, and
    # ERX on the encoder's own codes (what the learned form computes)
    import oracle
    na = ACC_LINES_LEARNED
    codes = enc.forward(xt[:na].reshape(-1, B)).cpu().numpy().astype(np.float64)
    oref = {"learned": oracle.run_cube(codes.reshape(na, W, K), warmup=0)["delta"],
            "srp32": oracle.run_cube(held, warmup=0, proj="srp", proj_dim=32, seed=5)["delta"],
            "srp5": oracle.run_cube(held, warmup=0, proj="srp", proj_dim=5, seed=5)["delta"],
            "full": oracle.run_cube(held, warmup=0)["delta"]}
    rows = {}
    for name, kw in (("learned_fp32", {"form": "fp32", "encoder": enc}),
                     ("learned_fp64", {"form": "fp64", "encoder": enc}),
                     ("srp32_fp32", {"form": "fp32", "proj": "srp", "proj_dim": 32, "seed": 5}),
                     ("srp5_fp32", {"form": "fp32", "proj": "srp", "proj_dim": 5, "seed": 5}),
                     ("full_fp64", {"form": "fp64"}), ("full_fp32", {"form": "fp32"}),
                     ("full_bf16", {"form": "bf16"})):
        speed = time_form(lambda **k: Detector(B, W, in_dtype="f32", warmup=0, stream=stream, **k),
                          xt, kw, dev, stream)
        d_ = Detector(B, W, in_dtype="f32", warmup=0, stream=stream, **kw)
        s_ = d_.push(xt)[0].cpu().numpy()
        d_.close()
        aucs = [auc(s_[t], labels[t]) for t in range(n_test) if labels[t].any()]
        rows[name] = {"lines_per_s": speed["lines_per_s"], "auc": float(np.mean(aucs)),
                      "rank_corr_full": float(np.mean([rank_corr(s_[t], ref[t])
                                                       for t in range(n_test)])),
                      "max_rel_err": max_rel_err(s_[:na], oref[name.split("_")[0]]),
                      "err_vs": "FP64 oracle on the same " + (
                          "codes" if name.startswith("learned") else "lines") + f", {na} lines"}
    out["forms"] = rows
    out["rank_corr_linear_code_bound"] = {
        "value": math.sqrt(K / B),
        "meaning": "rank agreement of RX on any linear K-dim code with full-band RX on a "
                   "Gaussian background (tests/test_learned_bound.py)"}
    out["drift_monitor"] = learned_drift(enc, xt, stream)
    out["batched"] = bench_learned_batched(enc, xt, stream)
    enc.close()
    return out


DRIFT_MIN_RANK_CORR = 0.1   # the learned form falls back to full band below this
DRIFT_AUDIT_EVERY = 10


def learned_drift(enc, xt, stream):
    """The learned form's drift monitor: every DRIFT_AUDIT_EVERY-th line is also
    scored by full-band ERX; below DRIFT_MIN_RANK_CORR (Spearman of the two score
    vectors) the context falls back to full band.  Run on the held-out lines as
    they are, and with a per-band gain change (a sensor calibration drift: gains
    log-uniform in [1/4, 4], seeded), to which full-band RX is invariant (an
    invertible linear map of the bands) but the encoder, trained on the old
    gains, is not."""
    import numpy as np
    import torch

    from paper_2408_14947_gb300 import Detector
    n, W, B = xt.shape
    g = np.exp(np.random.default_rng(2408).uniform(np.log(0.25), np.log(4.0), B))
    gain = torch.from_numpy(g.astype(np.float32)).to(xt.device)
    res = {"min_rank_corr": DRIFT_MIN_RANK_CORR, "audit_every": DRIFT_AUDIT_EVERY}
    for name, xs in (("held_out", xt), ("band_gain_drift", (xt * gain).contiguous())):
        d_ = Detector(B, W, in_dtype="f32", warmup=0, stream=stream, form="fp32", encoder=enc,
                      audit_every=DRIFT_AUDIT_EVERY, min_rank_corr=DRIFT_MIN_RANK_CORR)
        first_fb = None
        for t0 in range(0, n, DRIFT_AUDIT_EVERY):
            d_.push(xs[t0:t0 + DRIFT_AUDIT_EVERY])
            d_.sync()
            if first_fb is None and d_.drift()[3]:
                first_fb = t0 + DRIFT_AUDIT_EVERY
        last, low, audits, fb = d_.drift()
        d_.close()
        res[name] = {"audits": audits, "lowest_rank_corr": low, "last_rank_corr": last,
                     "fell_back": fb, "fallback_by_line": first_fb,
                     "lines_on_learned_codes": first_fb if first_fb is not None else n,
                     "lines": n}
    return res


def bench_learned_batched(enc, xt, stream, n_streams: int = 64, steps: int = 30):
    """The learned form as a batch: 64 streams of 1024 px x 224 bands, one line
    each per step, ERX on the shared encoder's 32 codes (one encoder forward per
    step over all streams), against the same 64 streams on full-band ERX.
    Stream s takes held-out line (t + 3 s) mod n at step t; lines are resident."""
    import torch

    from paper_2408_14947_gb300 import Batch
    n, W, B = xt.shape
    lines = [[xt[(t + 3 * s) % n] for s in range(n_streams)] for t in range(steps + 3)]

    def run(learned, form):
        b = Batch([{"bands": B, "width": W, "warmup": 0, "learned": learned}] * n_streams,
                  form=form, stream=stream, encoder=enc if learned else None)
        for t in range(3):
            b.push(lines[t])
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(steps):
            b.push(lines[3 + t])
        e1.record(stream)
        b.sync()
        ms = e0.elapsed_time(e1)
        b.close()
        return {"lines_per_s": n_streams * steps / (ms * 1e-3), "ms_per_step": ms / steps}

    return {"workload": f"{n_streams} streams x {W} px x {B} bands f32, one line each per step, "
                        f"{steps} timed steps (line gather included)",
            "learned_fp32": run(True, "fp32"), "learned_fp64": run(True, "fp64"),
            "full_fp64": run(False, "fp64"), "full_bf16": run(False, "bf16")}


LATENCY_PERIOD_S = 1e-3   # lines arriving every millisecond (1000 lines/s)
ACC_LINES = 500           # lines of the 108-band cube checked against the oracle per form
ACC_LINES_224 = 150       # lines of the 224-band cube checked against the oracle per form
ACC_LINES_BATCH = 3       # lines of every batched stream checked against the oracle
ACC_LINES_LEARNED = 20    # held-out lines of the learned workload checked per form


def push_size_throughput(det, x, out, stream, sizes=(1, 64, 256), lines=(2000, 8192, 8192)):
    """lines/s of the FP64 form when the cube arrives n lines per push, pushes
    queued back to back (CUDA events on the detector's stream)."""
    import torch
    res = {}
    for n, m in zip(sizes, lines):
        m = min(m, x.shape[0]) // n * n
        det.reset()
        for j in range(0, min(m, 4 * n), n):      # warm-up pushes
            det.push(x[j:j + n], tuple(o[j:j + n] for o in out))
        det.sync()
        det.reset()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for j in range(0, m, n):
            det.push(x[j:j + n], tuple(o[j:j + n] for o in out))
        b.record(stream)
        det.sync()
        torch.cuda.synchronize()
        res[str(n)] = {"lines_per_s": m / (a.elapsed_time(b) * 1e-3), "lines": m}
    return res


def paced_latency(det, x, out, stream, n, period_s, offset=200):
    """p50/p99 of enqueue -> delta_N written for single-line pushes arriving every
    period_s (host-paced, so each push finds the GPU idle, as lines from a
    sensor would): CUDA events on the detector's stream around each push."""
    import torch
    lines = x.shape[0]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n)]
    t_next = time.perf_counter()
    for i, (a, b) in enumerate(ev):
        while time.perf_counter() < t_next:
            pass
        t_next += period_s
        j = offset + i % (lines - offset)
        a.record(stream)
        det.push(x[j:j + 1], out)
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    return {"p50": lat[len(lat) // 2], "p99": lat[int(0.99 * len(lat))], "lines": len(lat),
            "mode": f"one line per push, a line every {period_s * 1e3:g} ms"}


def bench_paper_speed(dev, stream, n_lines=3000, reps=2):
    """The paper's speed experiments (Sec. IV-C) on this GPU, ERX as the paper
    runs it (SRP d = 5, alpha 0.1, 99-line warm-up; FP64 form): uniform random
    cubes of 3000 lines, bands 10..200 at 500 px and pixels 100..1500 at 50
    bands; the SRP dimension sweep of the ablation (d = 1..50 and no SRP) and
    the three datasets' shapes (random data of the same size), with the
    paper's Jetson Xavier NX lines/s beside them (context only)."""
    import torch

    from paper_2408_14947_gb300 import Detector
    g = torch.Generator(device=dev)
    g.manual_seed(2408)

    def lps(width, bands, lines, **kw):
        x = torch.rand((lines, width, bands), generator=g, device=dev, dtype=torch.float32)
        det = Detector(bands, width, in_dtype="f32", stream=stream, form="fp64", momentum=0.1,
                       warmup=99, **kw)
        det.push(x)
        det.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            det.reset()
            det.push(x)
        e1.record(stream)
        torch.cuda.synchronize()
        det.sync()
        det.close()
        return lines * reps / (e0.elapsed_time(e1) / 1000.0)

    srp5 = {"proj": "srp", "proj_dim": 5}
    out = {"form": "fp64", "config": "SRP d = 5, alpha 0.1, warm-up 99 lines, uniform f32"}
    out["bands_sweep_500px"] = {b: lps(500, b, n_lines, **srp5) for b in range(10, 201, 10)}
    out["pixels_sweep_50b"] = {p: lps(p, 50, n_lines, **srp5) for p in range(100, 1501, 100)}
    paper_d = {1: 610, 3: 580, 5: 566, 10: 525, 20: 446, 30: 379, 50: 287, "none": 243}
    dsw = {}
    for d in (1, 3, 5, 10, 20, 30, 50, "none"):
        kw = {} if d == "none" else {"proj": "srp", "proj_dim": d}
        dsw[d] = {"lines_per_s": lps(600, 90, 2400, **kw), "paper_jetson": paper_d[d]}
    out["d_sweep_600px_90b"] = dsw
    shapes = {"beach_452x108": (452, 108, 3072, 561), "synthetic_600x90": (600, 90, 2400, 508),
              "snp_1116x13": (1116, 13, 2499, 561)}
    out["dataset_shapes"] = {k: {"lines_per_s": lps(w, b, n, **srp5), "paper_jetson": pj}
                             for k, (w, b, n, pj) in shapes.items()}
    return out


def bench_detection(dev, stream, n_lines=4000):
    """The ablation of Sec. IV-C as detection-quality curves, computed on the GPU
    (erx_roc_metrics): ROC AUC, AUC_TD and AUC_BS of the delta_N maps of lines
    99.. of a C2-style cube (640 px x 108 bands u16, scenes switching every 2000
    lines, 0.2 % anomalies in 3 x 3 clusters), over the momentum alpha (with
    IMC and the pooled warm-up) and the SRP dimension d (FP64 form)."""
    import numpy as np
    import torch

    import synth
    from paper_2408_14947_gb300 import Detector, roc_metrics
    cfg = synth.dn_c2(seed=7)
    cube = make_cube(n_lines, seed=7)
    lab = torch.from_numpy(synth.anomaly_mask(cfg, 0, n_lines)[99:]).to(dev)
    x = torch.from_numpy(cube.view(np.int16)).to(dev)

    def run(**kw):
        det = Detector(BANDS, WIDTH, in_dtype="u16", in_bits=BITS, stream=stream, **kw)
        out = det.push(x)
        det.sync()
        m = roc_metrics(out[1][99:], lab, stream=stream)
        det.close()
        return {k: round(m[k], 5) for k in ("auc", "auc_td", "auc_bs")}

    res = {"workload": f"{n_lines} lines x {WIDTH} px x {BANDS} bands u16, "
                       f"{int(lab.sum())} anomaly pixels scored (lines 99..)"}
    res["alpha_full_band"] = {a: run(momentum=a) for a in (1.0, 0.5, 0.1, 0.01, 1e-3, 1e-4)}
    res["alpha_full_band"]["imc"] = run(averaging="imc")
    res["alpha_full_band"]["pooled_warmup_0.1"] = run(averaging="pooled")
    res["d_sweep_alpha_0.1"] = {d: run(proj="srp", proj_dim=d) for d in (1, 3, 5, 10, 20, 50)}
    res["d_sweep_alpha_0.1"]["none"] = run()
    return res


def run_ours(args):
    import numpy as np
    import torch

    import paper_2408_14947_gb300 as erx
    from paper_2408_14947_gb300 import Detector, _build

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    _build.build()
    erx.load_library()
    dev = torch.device("cuda", local)

    t_gen = time.perf_counter()
    cube = make_cube(LINES, seed=rank)
    gen_s = time.perf_counter() - t_gen
    x = torch.from_numpy(cube.view(np.int16)).to(dev)
    stream = torch.cuda.Stream(device=dev)

    def detector(**kw):
        return Detector(BANDS, WIDTH, in_dtype="u16", in_bits=BITS, stream=stream, **kw)

    det = detector(form="fp64")
    out = (torch.empty((LINES, WIDTH), dtype=torch.float64, device=dev),
           torch.empty((LINES, WIDTH), dtype=torch.float64, device=dev),
           torch.empty((LINES, WIDTH), dtype=torch.uint8, device=dev),
           torch.empty((LINES,), dtype=torch.uint8, device=dev))

    def step(d, o):
        d.reset()
        d.push(x, o)

    for _ in range(args.warmup):
        step(det, out)
    det.sync()
    det.profile(True)
    det.profile_read(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step(det, out)
        e1.record(stream)
        torch.cuda.synchronize()
    det.sync()
    ms_total = e0.elapsed_time(e1)
    prof = det.profile_read(reset=True)
    # the timed run's scores of the first lines against the FP64 oracle
    ref_head = None
    if rank == 0 and not args.quick:
        ref_head = oracle_delta(cube[:ACC_LINES])
        head_err = max_rel_err(out[0][:ACC_LINES].cpu().numpy(), ref_head)
    det.profile(False)
    ms_total = max_over_ranks(ms_total, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_step = ms_total / args.steps
    value = whole_job_rate(LINES, world, ms_step)
    launches = sum(v[2] for v in prof.values())

    # roofline of the dominant kernel: the FP64 score kernel (d(d+1)/2 + d DFMA per pixel)
    d = BANDS
    dom = max(prof, key=lambda k: prof[k][0])
    ms_dom, n_dom, _ = prof[dom]
    blocks = max(1, n_dom // args.steps)
    lines_per_launch = LINES / blocks
    flops = {
        "solve_fp64": 2.0 * WIDTH * (d * (d + 1) / 2 + d),
        "chol": d ** 3 / 3.0 + d * 32 * 32 / 3.0,
        "stats_int": 2.0 * WIDTH * d * d,
    }
    per_line = flops.get(dom, 0.0)
    achieved = per_line * lines_per_launch / (ms_dom / n_dom / 1000.0) / 1e9 if n_dom else 0.0
    if dom == "stats_int":
        peak, unit, bound = IMAD_PEAK_GOPS * 2, "GOP/s", "alu"
    else:
        peak, unit, bound = FP64_PEAK_GFLOPS, "GFLOP/s", "alu"
    # DRAM bytes (read + write) of one solve_fp64 launch from the ncu capture in
    # profiles/solve_fp64_c2_2000x640x108.md: 383.9 MB for a 2000-line launch,
    # scaled to this run's average lines per launch (traffic grows with the lines).
    traffic = 383.88e6 * lines_per_launch / 2000.0 if dom == "solve_fp64" else None
    roof = {"bound": bound, "pipe": "fp64" if dom != "stats_int" else "int32", "kernel": dom,
            "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic, "algorithmic_bytes": (WIDTH * BANDS * 2 + WIDTH * 8 +
                                                      8 * BANDS * (BANDS + 1) / 2) * lines_per_launch,
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2070 MHz"}
    if roof["pipe"] == "fp64":
        roof["dfma_pipe_gflops"] = DFMA_PIPE_GFLOPS
        roof["frac_of_dfma_pipe"] = achieved / DFMA_PIPE_GFLOPS
        roof["dfma_pipe_note"] = ("scalar DFMA issue rate, 1.671 lanes/clk/SM at 2070 MHz "
                                  "(python bench.py --pipe-probe); the derived peak above is "
                                  "the nominal FP64 rate")
    if rank == 0 and not args.quick:
        pk = measure_pipe_peaks(dev)
        roof["fp64_dgemm_gflops"] = pk["dgemm_gflops"]
        roof["fp64_dgemm_note"] = ("cuBLAS DGEMM 4096^3 measured in this run: a library "
                                   "reference for the derived peak")
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[2] / args.steps,
                   "share": v[0] / max(1e-9, sum(w[0] for w in prof.values()))}
               for k, v in prof.items() if v[2]}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
              "data": "synthetic",
              "config": dict(workload_config(),
                             block_lines=det.cfg.block_lines or "auto",
                             parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                             gen_seconds=round(gen_s, 1)),
              "gpu_launches": launches, "roofline": roof, "kernels": kernels,
              "clocks": clk.summary()}
    if ref_head is not None:
        result["max_rel_err"] = {"value": head_err, "lines": ACC_LINES,
                                 "vs": "FP64 NumPy oracle, same lines", "bar": 1e-9}

    if rank == 0 and not args.quick:
        # p50 / p99 latency of one line pushed alone (stream mode), after warm-up
        lat = []
        det.reset()
        one = tuple(o[:1] for o in out)
        for i in range(200):
            det.push(x[i:i + 1], one)
        det.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.latency_lines)]
        for i, (a, b) in enumerate(ev):
            j = 200 + i % (LINES - 200)
            a.record(stream)
            det.push(x[j:j + 1], one)
            b.record(stream)
        torch.cuda.synchronize()
        lat = sorted(a.elapsed_time(b) for a, b in ev)
        result["latency_ms"] = {"p50": lat[len(lat) // 2], "p99": lat[int(0.99 * len(lat))],
                                "lines": len(lat), "mode": "one line per push, back to back"}
        result["latency_paced_ms"] = paced_latency(det, x, one, stream, args.latency_lines,
                                                   LATENCY_PERIOD_S)
        # throughput by push size: stream mode (one line per push, pushes queued
        # back to back) and block mode (64 and 256 lines per push)
        result["throughput_by_push_lines"] = push_size_throughput(det, x, out, stream)
        # score-then-update with the update deferred to a second stream (the
        # line is scored against the factor made at the end of the previous push)
        dpl = detector(form="fp64", order="score_then_update", pipeline=True)
        for i in range(200):
            dpl.push(x[i:i + 1], one)
        dpl.sync()
        result["latency_pipelined_ms"] = {
            "order": "score_then_update, ERX_FLAG_PIPELINE",
            "paced": paced_latency(dpl, x, one, stream, args.latency_lines, LATENCY_PERIOD_S)}
        dpl.sync()
        dpl.close()

        # other forms on the same cube, same step definition; each timed run's
        # scores of the first ACC_LINES lines against the FP64 oracle's
        refs = {"ema": ref_head,
                "imc": oracle_delta(cube[:ACC_LINES], averaging="imc"),
                "srp5": oracle_delta(cube[:ACC_LINES], proj="srp", proj_dim=5, seed=0)}
        forms = {"err_lines": ACC_LINES}
        for name, kw, rk in (("fp64e", {"form": "fp64e"}, "ema"), ("fp32", {"form": "fp32"}, "ema"),
                             ("tf32", {"form": "tf32"}, "ema"),
                             ("bf16", {"form": "bf16"}, "ema"),
                             ("tf32x3", {"form": "tf32x3"}, "ema"),
                             ("fp64_imc", {"form": "fp64", "averaging": "imc"}, "imc"),
                             ("fp64_srp5", {"form": "fp64", "proj": "srp", "proj_dim": 5}, "srp5"),
                             ("fp32_srp5", {"form": "fp32", "proj": "srp", "proj_dim": 5}, "srp5")):
            forms[name] = time_form(lambda **k: Detector(BANDS, WIDTH, in_dtype="u16",
                                                         in_bits=BITS, stream=stream, **k),
                                    x, kw, dev, stream, ref=refs[rk])
        result["forms_108"] = forms

        # 224 bands (AVIRIS raw band count): 2000 lines x 1024 px f32, kappa 1e3
        n224 = 2000
        cube224 = make_cube(n224, seed=1, kind="c3", width=1024, bands=224, kappa=1e3)
        x224 = torch.from_numpy(cube224).to(dev)
        ref224 = oracle_delta(cube224[:ACC_LINES_224])
        del cube224
        forms224 = {}
        for name in ("fp64", "fp64e", "fp32", "tf32", "bf16", "tf32x3"):
            forms224[name] = time_form(lambda **k: Detector(224, 1024, in_dtype="f32",
                                                            stream=stream, **k),
                                       x224, {"form": name}, dev, stream, ref=ref224)
        result["forms_224"] = {"workload": f"{n224} lines x 1024 px x 224 bands f32, "
                                           "Gaussian background, kappa 1e3",
                               "err_lines": ACC_LINES_224, **forms224}
        del x224

        # the paper's speed experiments and SRP dimension sweep at its shapes
        result["paper_speed_tests"] = bench_paper_speed(dev, stream)

        # the ablation of Sec. IV-C as detection-quality curves (GPU metrics)
        result["detection"] = bench_detection(dev, stream)

        # batched form: 256 streams, widths U{128..2048}, bands from {8,16,64,108,224}
        result["batched"] = bench_batched(dev, stream)

        # learned form: encoder trained on the method's own full-band scores
        result["learned"] = bench_learned(dev, stream)

        # end to end through the public host-buffer call: pinned input, results to host
        xh = torch.from_numpy(cube.view(np.int16)).pin_memory()
        oh = (torch.empty((LINES, WIDTH), dtype=torch.float64).pin_memory(),
              torch.empty((LINES, WIDTH), dtype=torch.float64).pin_memory(),
              torch.empty((LINES, WIDTH), dtype=torch.uint8).pin_memory(),
              torch.empty((LINES,), dtype=torch.uint8).pin_memory())
        det.reset()
        det.push_host(xh, oh)
        ts = []
        for _ in range(max(1, min(args.steps, 3))):
            det.reset()
            t0 = time.perf_counter()
            det.push_host(xh, oh)
            ts.append(time.perf_counter() - t0)
        h2d = cube.nbytes
        d2h = sum(o.numel() * o.element_size() for o in oh)
        result["e2e"] = {"value": LINES / statistics.median(ts), "unit": UNIT,
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        result["cpu_baseline"] = cpu_baseline(args.cpu_lines)
        one_t = cpu_baseline(args.cpu_lines // 10, one_thread=True)
        result["cpu_baseline"]["value_1thread"] = one_t["value"]
        result["cpu_baseline"]["sample_1thread"] = one_t["sample"] + ", 1 BLAS thread"
        result["pixel_spectra_per_s"] = value * WIDTH
    elif rank == 0:
        result["e2e"] = None
        result["cpu_baseline"] = None
    det.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def profile_batched(form, steps):
    """The C4 batch (256 streams) in one form: tuned, three warm-up steps, then
    `steps` timed steps (one graph launch each; capture the last steps'
    kernels)."""
    import torch

    import synth
    from paper_2408_14947_gb300 import Batch
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    cfgs = synth.stream_configs_c4(256)
    lines = [torch.from_numpy(synth.gen_lines(c, 0, 2)).to(dev) for c in cfgs]
    b = Batch([{"bands": c.bands, "width": c.width} for c in cfgs], form=form, stream=stream)
    b.push([x[0] for x in lines])
    b.sync()
    b.tune(reps=3)
    for k in range(3):
        b.push([x[k % 2] for x in lines])
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        b.push([x[k % 2] for x in lines])
    e1.record(stream)
    b.sync()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"c4_{form}", "steps": steps,
                      "ms_per_step": e0.elapsed_time(e1) / steps}))
    b.close()


def run_pipe_probe():
    """Compile pipe_probe.cu (beside this file) for sm_103a into _build/ and run
    it; it prints its own JSON object."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.abspath(__file__))
    out_dir = os.path.join(root, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "pipe_probe")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(root, "pipe_probe.cu")], check=True)
    subprocess.run([exe], check=True)


def measure_pipe_peaks(dev, n: int = 4096, reps: int = 5):
    """Library reference rates for the FP64 and FP32 pipes: cuBLAS DGEMM and
    SGEMM (TF32 off) on n x n x n, 2 n^3 flops, best of `reps` (CUDA events),
    with the clocks sampled meanwhile.  Context for the derived FP64 peak."""
    import torch
    local = dev.index or 0
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {"n": n, "how": "torch.matmul (cuBLAS), best of %d, CUDA events" % reps}
    try:
        with ClockSampler(local) as clk:
            for name, dt in (("dgemm", torch.float64), ("sgemm_no_tf32", torch.float32)):
                a = torch.randn((n, n), dtype=dt, device=dev)
                b_ = torch.randn((n, n), dtype=dt, device=dev)
                torch.matmul(a, b_)
                best = math.inf
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    torch.matmul(a, b_)
                    e1.record()
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                out[name + "_gflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e9
                del a, b_
        out["clocks"] = clk.summary()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["fp64_peak_derived_gflops"] = FP64_PEAK_GFLOPS
    return out


def profile_training(n_lines):
    """Encoder training (224 -> 128 -> 32) on C5 lines of 1024 px: one warm-up
    line, then `n_lines` timed lines (one AdamW step each)."""
    import torch

    from paper_2408_14947_gb300 import Detector, Encoder, erx_train_opts_default
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    W, B = 1024, 224
    cube = make_cube(n_lines + 1, seed=11, kind="c5", width=W, bands=B)
    x = torch.from_numpy(cube).to(dev)
    flat = cube.reshape(-1, B)
    full = Detector(B, W, in_dtype="f32", form="fp64", warmup=0, stream=stream)
    fd = full.push(x)[0]
    full.sync()
    full.close()
    enc = Encoder(B, 128, 32, seed=0, stream=stream)
    enc.set_norm(flat.mean(0), 1.0 / (flat.std(0) + 1e-3))
    o = erx_train_opts_default()
    enc.train(x[:1], fd[:1], o)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    enc.train(x[1:], fd[1:], o)
    e1.record(stream)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "c5_train", "lines": n_lines,
                      "ms_per_line": e0.elapsed_time(e1) / n_lines}))
    enc.close()


def run_profile_case(args):
    """One block of a named workload through one form, for profiler captures:
    a warm-up push, then one push of `--lines` lines (its kernels are the ones
    to capture: skip the warm-up push's launches)."""
    import numpy as np
    import torch

    from paper_2408_14947_gb300 import Detector, _build
    _build.build()
    kind, form = args.profile_case.split("_", 1)
    if kind == "c4":
        return profile_batched(form, args.lines)
    if args.profile_case == "c5_train":
        return profile_training(args.lines)
    avg = "ema"
    if form.endswith("_imc"):
        form, avg = form[: -len("_imc")], "imc"
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    if kind == "c2":
        cube = make_cube(args.lines, seed=0)
        x = torch.from_numpy(cube.view(np.int16)).to(dev)
        det = Detector(BANDS, WIDTH, in_dtype="u16", in_bits=BITS, form=form, stream=stream,
                       block_lines=args.lines, averaging=avg)
    elif kind == "c3":
        cube = make_cube(args.lines, seed=1, kind="c3", width=1024, bands=224, kappa=1e3)
        x = torch.from_numpy(cube).to(dev)
        det = Detector(224, 1024, in_dtype="f32", form=form, stream=stream,
                       block_lines=args.lines, averaging=avg)
    else:
        # learned codes 224 -> 128 -> 32 (untrained weights: the kernels' work is the same)
        from paper_2408_14947_gb300 import Encoder
        cube = make_cube(args.lines, seed=1, kind="c3", width=1024, bands=224, kappa=1e3)
        x = torch.from_numpy(cube).to(dev)
        enc = Encoder(224, 128, 32, seed=0, stream=stream)
        flat = cube[: min(len(cube), 64)].reshape(-1, 224)
        enc.set_norm(flat.mean(0), 1.0 / (flat.std(0) + 1e-3))
        det = Detector(224, 1024, in_dtype="f32", form=form, stream=stream,
                       block_lines=args.lines, encoder=enc)
    del cube
    det.push(x)
    det.sync()
    det.reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    det.push(x)
    e1.record(stream)
    det.sync()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "lines": args.lines,
                      "ms": e0.elapsed_time(e1)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-lines", type=int, default=3000)
    ap.add_argument("--ref-lines", type=int, default=1000)
    ap.add_argument("--latency-lines", type=int, default=10000)
    ap.add_argument("--quick", action="store_true", help="skip latency, forms, e2e, baseline")
    ap.add_argument("--lines", type=int, default=LINES,
                    help="lines of the workload cube (smaller cubes for profiler captures)")
    ap.add_argument("--peaks", action="store_true",
                    help="print cuBLAS DGEMM / SGEMM rates (FP64 and FP32 pipe references)")
    ap.add_argument("--pipe-probe", action="store_true",
                    help="build and run pipe_probe.cu: FP64 / FP32 / integer pipe rates per SM, "
                         "DFMA and double rsqrt latency, barrier and cluster costs (JSON)")
    ap.add_argument("--profile-case", default=None,
                    choices=["c2_fp64", "c2_fp64e", "c2_fp32", "c2_tf32", "c2_bf16", "c2_fp64_imc",
                             "c3_fp64", "c3_fp32", "c3_tf32", "c3_bf16", "c3_tf32x3", "c5_fp32",
                             "c5_fp64", "c4_fp64", "c4_fp32", "c4_tf32", "c4_bf16", "c4_tf32x3",
                             "c5_train"],
                    help="push one block of --lines lines of a workload (c2: 640 px x 108 "
                         "bands u16; c3: 1024 px x 224 bands f32, kappa 1e3; c5: c3 lines "
                         "through learned 32-dim codes) through one form (_imc: IMC "
                         "averaging), after one warm-up push; c4: the 256-stream batch, "
                         "--lines steps after three warm-up steps; c5_train: --lines encoder "
                         "training steps; for profiler captures, no bench line")
    args = ap.parse_args()
    globals()["LINES"] = args.lines
    if args.peaks:
        import torch
        print(json.dumps(measure_pipe_peaks(torch.device("cuda", 0))))
        return
    if args.pipe_probe:
        run_pipe_probe()
        return
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
