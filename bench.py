"""Benchmark: streaming exact DMD of HD-video-shaped uint8 frames on one GB300.

Workload (synthetic configuration 2): n = 1920*1080*3 uint8 pixels per frame,
window m = 100 snapshots, DMD rank r = 10. One step = one streamed frame
through the whole hot path: ingest into the ring slot, Gram row (m dot
products over n, exact int64), symmetric insert, FP64 eigensolvers
(sym-eig of G_X, A~, eig of A~), and Phi = X' V Sigma^-1 W (n x r complex64).

Printed JSON line (rank 0): snapshots/s over K timed steps in steady state
(CUDA events on the launch stream, barrier + synchronize around the timed
region, tracing off; the pipeline of depth frames is full when the region
opens and when it closes), then a traced pass of the same steps for the
per-kernel durations (the fused Phi + Gram-row pass against the measured
copy peak) and per-frame latency percentiles, an end-to-end figure through
the C ABI with pinned host buffers (starts with an empty pipeline and ends
with every frame's outputs delivered), the CPU oracle timed on a bounded
sample, and the SM clocks sampled during the timed region.

Secondary measurements in the same line: each kernel launched alone, the
full-window rebuild (tensor cores vs row passes), the 8-frame catch-up, the
Fourier-sparse Gram row, the BF16x3 tensor-core catch-up and rebuild of an
FP32 window (n = 2^22, m = 256), and batched serving of 64 mixed FP32/uint8 streams
with Poisson arrivals (aggregate snapshots/s, p50/p99 frame latency, and the
closed-loop capacity of one batched launch per tick against one push per
stream).

`--impl reference` times the CPU oracle alone (the reference arm).
Multi-GPU (torchrun): every rank streams its own independent video (weak
scaling, no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "streamed snapshots/s and Gram-update HBM GB/s vs ~8 TB/s; p99 frame latency"
UNIT = "snapshots/s"
H, W_, C_ = 1080, 1920, 3
M_WIN = 100
R_MODES = 10
DEPTH = 6          # frames in flight: the smallest depth whose pipeline hides the eigensolver
TRACED_STEPS = 40       # steps of the traced pass that follows the timed one


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--depth", type=int, default=DEPTH, help="DMD frames in flight (sdmd_step pipeline)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the rebuild and Fourier-sparse measurements")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--scpu-seconds", type=float, default=3.0,
                    help="seconds of the streaming CPU Gram update (host cores)")
    ap.add_argument("--case", choices=["bf16x3_catchup", "f32_catchup", "batched_rows", "fused_pass"], default=None,
                    help="run one small fixed workload (for a profiler capture of its kernel) and exit")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served Poisson-arrival run (0 skips the serving measurement)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(base, rank):
    """Seed of a rank's video: every rank streams its own independent video
    (the workload partitions into independent streams; no data exchange)."""
    return base + 1000 * rank


def max_over_ranks(ms, world, device):
    """The slowest rank's timed region (each rank times its own, between two
    barriers); on one rank, its own."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(world, steps, t_max_ms):
    """Whole-job throughput: the steps of every rank over the slowest rank's time."""
    return world * steps / (t_max_ms / 1e3)


def workload_config(n, extra=None):
    cfg = {"workload": "hd_video_u8: n=1920x1080x3 uint8, window m=100, DMD rank r=10, "
                       "one frame per step (push + modes)",
           "n": n, "m": M_WIN, "r": R_MODES, "frame": [H, W_, C_],
           "l2": "inputs larger than L2 (window ring = 100 x 6.2 MB = 622 MB > 129 MB L2)"}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------ CPU oracle --

def oracle_rate(band_frames, n_total, seconds):
    """Oracle (recompute-from-scratch exact-int64 Gram + FP64 dense DMD) on a
    band of each frame; band_frames is (T, band) uint8, generated before
    timing. Returns (snapshots/s scaled to full frames, info)."""
    import oracle
    from oracle import native
    T, band = band_frames.shape
    so = oracle.StreamOracle(band, M_WIN, "u8")
    for t in range(M_WIN):
        so.push(band_frames[t])
    steps = 0
    t0 = time.perf_counter()
    # the frames after the first window are streamed in a loop until the
    # sample's time is up (the oracle's cost does not depend on the values)
    while True:
        so.push(band_frames[M_WIN + steps % (T - M_WIN)])
        so.modes(R_MODES)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    rate_band = steps / el
    # the oracle's per-step cost is O(n m^2) + O(n m r): linear in the band
    rate_full = rate_band * band / n_total
    info = {"steps": steps, "seconds": el, "band_pixels": band,
            "threads": max(native.num_threads(), _blas_threads())}
    return rate_full, info


def streaming_cpu_rate(frames, seconds):
    """The streaming method on the host cores (Sec. 3.1, Eq. 12a-b; the
    paper's streaming CPU configuration): per push, the frame's copy into a
    100-slot host ring, its 100 exact int64 inner products and G's row and
    column, threaded over position blocks. Full HD frames; frames is (T, n)
    uint8, generated before timing (the cost does not depend on the values)."""
    from oracle import native
    T, n = frames.shape
    sc = native.StreamingCPU(n, M_WIN, "u8")
    sc.fill(frames)
    sc.push(frames[0])                                   # untimed warm-up push
    k = 0
    t0 = time.perf_counter()
    while True:
        sc.push(frames[k % T])
        k += 1
        if k >= 3 and time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    rate = k / el
    return {"value": rate, "unit": UNIT, "cores": native.scpu_threads(),
            "kind": "streaming CPU method: per push, ingest + %d exact int64 dot products + G row/column "
                    "(the Gram update only: no eigensolve, no Phi)" % M_WIN,
            "sample": "%d pushes of full %d-pixel frames into a %d-slot host ring, %.1f s" % (k, n, M_WIN, el),
            "GB/s": rate * M_WIN * n / 1e9,
            "gpu_counterpart": "kernels_isolated.gram_row (the same update on the GPU)"}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([p.get("num_threads", 1) for p in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1612_07875_gb300 import synth
    vs = synth.VideoStream(seed=synth.config_seed(2))
    n = vs.n
    band = n // 64
    total = M_WIN + max(args.warmup, 0) + args.steps
    bf = np.stack([vs.frame(t)[:band] for t in range(total)])     # generated before timing
    # warmup steps (untimed), then K timed steps, each on the band sample
    import oracle
    so = oracle.StreamOracle(band, M_WIN, "u8")
    for t in range(M_WIN):
        so.push(bf[t])
    t = M_WIN
    for _ in range(max(args.warmup, 0)):
        so.push(bf[t])
        so.modes(R_MODES)
        t += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        so.push(bf[t])
        so.modes(R_MODES)
        t += 1
    el = time.perf_counter() - t0
    value = args.steps / el * band / n
    from oracle import native
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            # the measured wall time of a timed step (on the band sample), so
            # that steps x ms_per_step is this run's timed region; `value` is
            # the rate scaled to full frames
            "ms_per_step": 1e3 * el / args.steps,
            "ms_per_step_full_frame_scaled": 1e3 * el / args.steps * n / band,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
            "data": "synthetic (seeded HD-video-shaped frames; no dataset)",
            "config": workload_config(n, {"parallelism": "1 GPU" if args.gpus <= 1 else
                                          "independent stream per GPU"}),
            "cpu_baseline": {"value": value, "unit": UNIT,
                             "cores": max(native.num_threads(), _blas_threads()), "kind": "oracle",
                             "sample": "each step: oracle recompute of G (exact int64) + dense FP64 DMD "
                                       "on a %d-pixel band (1/64 of each frame); rate scaled to full "
                                       "frames by n/band (the oracle's cost is linear in n)" % band},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- ours --

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measure_isolated(S, h, frames, t0, stream, phi, n, steps=8):
    """Serial push + modes steps (each kernel alone on the GPU), traced."""
    import torch
    sh = stream.cuda_stream
    lam = torch.empty(2 * R_MODES, dtype=torch.float64, device=frames.device)
    S.sdmd_sync(h, sh)
    stream.synchronize()
    chunk, tuned_us = S.sdmd_autotune(h, sh)          # the Gram-row schedule picked by measurement
    S.sdmd_trace(h, True)
    with torch.cuda.stream(stream):
        for i in range(steps):
            S.sdmd_push(h, frames[(t0 + i) % frames.shape[0]], sh)
            S.sdmd_modes(h, R_MODES, phi, lam, None, sh)
    stream.synchronize()
    out = {}
    for k, name in ((S.SDMD_K_GRAM_ROW, "gram_row"), (S.SDMD_K_PHI, "phi"), (S.SDMD_K_MODES, "modes_small_f64"),
                    (S.SDMD_K_INGEST, "ingest_copy")):
        cnt, ms = S.sdmd_trace_read(h, k)
        out[name] = {"launches": cnt, "us": 1e3 * ms / max(cnt, 1)}
    S.sdmd_trace(h, False)
    out["gram_row"]["GB/s"] = M_WIN * n / (out["gram_row"]["us"] * 1e-6) / 1e9
    out["gram_row"]["autotuned_chunk_bytes"] = chunk
    out["gram_row"]["autotune_us"] = tuned_us
    out["gram_row"]["note"] = "each launch after a sdmd_modes (serial push + modes steps)"
    out["phi"]["GB/s"] = ((M_WIN - 1) * n + n * R_MODES * 8) / (out["phi"]["us"] * 1e-6) / 1e9
    # the last eigensolver launch's phase clocks (SM cycles, in thousands)
    out["modes_small_f64"]["phase_kcycles"] = {k: v // 1000 for k, v in S.sdmd_modes_phase_cycles(h, sh).items()}
    out["serial_step_us"] = sum(out[k]["us"] for k in ("gram_row", "phi", "modes_small_f64", "ingest_copy"))
    # streaming background subtraction of the newest frame (Algorithm 3):
    # background column and foreground x_t - background, one pass over X'
    fg = torch.empty(n, dtype=torch.float32, device=frames.device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for what, name, extra in ((S.SDMD_RECON_BACKGROUND, "background", 0), (S.SDMD_RECON_FOREGROUND, "foreground", n)):
        with torch.cuda.stream(stream):
            S.sdmd_reconstruct(h, M_WIN - 1, what, fg, sh)      # warm-up
            ev0.record(stream)
            for _ in range(steps):
                S.sdmd_reconstruct(h, M_WIN - 1, what, fg, sh)
            ev1.record(stream)
        stream.synchronize()
        us = 1e3 * ev0.elapsed_time(ev1) / steps
        out[name] = {"launches": 2 * steps, "us": us,
                     "GB/s": ((M_WIN - 1) * n + 4 * n + extra) / (us * 1e-6) / 1e9}
    # POD modes U = X V Sigma^-1 (SVD-only output), n x r FP32, one pass over X
    U = torch.empty(R_MODES, n, dtype=torch.float32, device=frames.device)
    with torch.cuda.stream(stream):
        S.sdmd_pod_modes(h, R_MODES, U, sh)
        ev0.record(stream)
        for _ in range(steps):
            S.sdmd_pod_modes(h, R_MODES, U, sh)
        ev1.record(stream)
    stream.synchronize()
    us = 1e3 * ev0.elapsed_time(ev1) / steps
    out["pod_modes"] = {"launches": 2 * steps, "us": us,
                        "GB/s": ((M_WIN - 1) * n + 4 * n * R_MODES) / (us * 1e-6) / 1e9}
    del U
    # the Gram-row update sustained: sdmd_push back to back, nothing else queued
    S.sdmd_trace(h, True)
    with torch.cuda.stream(stream):
        for i in range(20):
            S.sdmd_push(h, frames[(t0 + steps + i) % frames.shape[0]], sh)
    stream.synchronize()
    cnt, ms = S.sdmd_trace_read(h, S.SDMD_K_GRAM_ROW)
    S.sdmd_trace(h, False)
    us = 1e3 * ms / max(cnt, 1)
    out["gram_row_sustained"] = {"launches": cnt, "us": us, "GB/s": M_WIN * n / (us * 1e-6) / 1e9,
                                 "note": "sdmd_push back to back (the streaming Gram update alone)"}
    return out


def measure_rebuild(S, h, stream, n, reps=3):
    """Full-window rebuild of G on the benchmark handle: the tensor-core pass
    (one read of the window, exact int64) and the row-kernel pass (one Gram-row
    pass per snapshot, bit-identical to streaming), mean of `reps` each."""
    import torch
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for opt, name in ((1, "tensor_core"), (0, "row_passes")):
        S.sdmd_set_option(h, S.SDMD_OPT_REBUILD_TENSOR, opt)
        S.sdmd_rebuild(h, stream.cuda_stream)      # warm-up (and first-use allocation)
        torch.cuda.synchronize()
        r0.record(stream)
        for _ in range(reps):
            S.sdmd_rebuild(h, stream.cuda_stream)
        r1.record(stream)
        stream.synchronize()
        ms = r0.elapsed_time(r1) / reps
        passes = 1 if opt else M_WIN
        flops = 2.0 * 128 * ((M_WIN + 1 + 15) // 16 * 16) * n      # MMA work incl. padding rows
        out[name] = {"ms": ms, "window_passes": passes,
                     "GB/s": passes * M_WIN * n / (ms * 1e-3) / 1e9}
        if opt:
            out[name]["TFLOP/s"] = flops / (ms * 1e-3) / 1e12
    S.sdmd_set_option(h, S.SDMD_OPT_REBUILD_TENSOR, 1)
    out["note"] = "tensor_core: centred fp16 pixels, FP32 TMEM accumulators drained to int64 (exact); " \
                  "row_passes: bit-identical to the streamed G"
    return out


def measure_catchup(S, h, frames, t0, stream, n, k=8, reps=3):
    """Multi-column catch-up: k frames appended with one sdmd_push_batch (one
    tensor-core pass over the window) vs k sdmd_push calls (k Gram-row passes)."""
    import torch
    sh = stream.cuda_stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    S.sdmd_sync(h, sh)
    out = {}
    for name in ("push_batch", "single_pushes"):
        times = []
        for r in range(reps + 1):
            i0 = (t0 + r * k) % (frames.shape[0] - k)
            block = frames[i0:i0 + k]
            with torch.cuda.stream(stream):
                e0.record(stream)
                if name == "push_batch":
                    S.sdmd_push_batch(h, k, block, n, sh)
                else:
                    for j in range(k):
                        S.sdmd_push(h, block[j], sh)
                e1.record(stream)
            stream.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
        ms = sum(times) / len(times)
        out[name] = {"ms": ms, "frames_per_s": k / (ms * 1e-3)}
    out["k"] = k
    out["note"] = "push_batch: ingest + one exact tensor-core pass for the k new rows/columns"
    return out


def measure_bf16x3(S, dev, stream, n=1 << 22, m=256, ks=(8, 64), reps=3):
    """FP32 window shaped like the precision-sweep workload (n = 2^22, m = 256):
    k frames appended with one sdmd_push_batch under SDMD_OPT_F32_BF16X3 (k <= 16:
    one CUDA-core pass with FP32 products; larger k: BF16x3 on the tensor cores)
    against k FP32 sdmd_push calls, the BF16x3 rebuild against the FP32 row passes, and
    the BF16x3 error of the k new rows on sampled entries against FP64 dot
    products of the same FP32 frames."""
    import torch
    sh = stream.cuda_stream
    g = torch.Generator(device=dev)
    g.manual_seed(1612)
    kmax = max(ks)
    frames = torch.randn(m + kmax * (reps + 1), n, device=dev, generator=g)
    h = S.sdmd_create(n, m, S.SDMD_F32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"n": n, "m": m}
    try:
        with torch.cuda.stream(stream):
            for t in range(m):
                S.sdmd_push(h, frames[t], sh)
        nxt = m

        def timed(fn, r=reps):
            ts = []
            for i in range(r + 1):
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                stream.synchronize()
                if i:
                    ts.append(e0.elapsed_time(e1))
            return sum(ts) / len(ts)

        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 0)
        src = [0]

        def one_push():
            j = m + src[0] % (kmax * reps)
            src[0] += 1
            S.sdmd_push(h, frames[j], sh)
        ms1 = timed(one_push, r=8)
        out["fp32_push"] = {"ms": ms1, "snapshots_per_s": 1e3 / ms1, "GB/s": m * n * 4 / (ms1 * 1e-3) / 1e9}
        S.sdmd_set_option(h, S.SDMD_OPT_F32_FP64, 1)
        ms64 = timed(one_push, r=3)
        S.sdmd_set_option(h, S.SDMD_OPT_F32_FP64, 0)
        out["fp64_push"] = {"ms": ms64, "snapshots_per_s": 1e3 / ms64,
                            "note": "FP64 products and sums (reference precision)"}
        G = torch.empty(m, m, dtype=torch.float64, device=dev)
        for split, name, bound in ((1, "bf16x3", 1e-6), (2, "bf16x2", 3e-5)):
            S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, split)
            for k in ks:
                def batch():
                    j = m + (src[0] * k) % (kmax * reps)
                    src[0] += 1
                    S.sdmd_push_batch(h, k, frames[j:j + k], n, sh)
                msb = timed(batch)
                ent = {"ms": msb, "snapshots_per_s": k / (msb * 1e-3),
                       "window_GB/s": m * n * 4 / (msb * 1e-3) / 1e9, "vs_fp32_push": (k / msb) / (1.0 / ms1),
                       "path": ("CUDA cores, FP32 products (k <= 16)" if k <= 16 else
                                "tensor cores, %s split" % name)}
                ent["frac_of_copy_peak"] = ent["window_GB/s"] / measured_peaks()[0]
                # error of the k newest rows (the last batch) on sampled entries
                stream.synchronize()
                S.sdmd_gram(h, G, sh)
                stream.synchronize()
                j = m + ((src[0] - 1) * k) % (kmax * reps)
                step = 4 if k > 16 else 1
                Wh = frames[j:j + k][::step].cpu().numpy().astype(np.float64)   # exact FP32 values
                ref = Wh @ Wh.T
                bnd = np.abs(Wh) @ np.abs(Wh).T
                sel = np.arange(m - k, m, step)
                got = G.cpu().numpy()[np.ix_(sel, sel)]
                ent["sampled_error"] = {
                    "max_abs_err_over_sum_abs_products": float((np.abs(got - ref) / bnd).max()),
                    "rel_frobenius": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                    "entries": int(sel.size ** 2), "bound": bound,
                    "reference": "FP64 dot products of the same FP32 frames on the host (numpy)"}
                out["%s_push_batch_k%d" % (name, k)] = ent
        out["per_kappa"] = bf16x3_kappa_sweep(S, h, dev, stream, n, m)
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 1)
        msr = timed(lambda: S.sdmd_rebuild(h, sh), r=2)
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 0)
        msr_rows = timed(lambda: S.sdmd_rebuild(h, sh), r=1)
        flops = 6 * 2.0 * n * m * m / 2
        out["rebuild"] = {"bf16x3_ms": msr, "fp32_rows_ms": msr_rows, "speedup": msr_rows / msr,
                          "bf16x3_TFLOP/s_useful": flops / (msr * 1e-3) / 1e12}
        if S.sdmd_status(h, sh) != S.SDMD_OK:
            raise RuntimeError("BF16x3 measurement status: " + S.sdmd_last_error())
        out["note"] = ("random N(0,1) FP32 frames; window_GB/s = window bytes / batch time; the rebuild's "
                       "useful flops count the six bf16 products of the lower triangle")
        return out
    finally:
        S.sdmd_destroy(h)
        del frames
        torch.cuda.empty_cache()


def measure_config1(S, synth, dev, stream, n_snap=200, m=32, r=10, depths=(1, 4)):
    """The planted-mode FP32 stream (n = 64 x 64, window m = 32, 200
    snapshots, rank r = 10): every snapshot through sdmd_step (push + exact
    DMD with Phi), device-resident snapshots, timed over the whole stream
    (window ramp-up included, outputs complete at the end) at depth 1 (one
    frame at a time) and with frames in flight; per-frame latency from the
    frame trace of a second, traced run."""
    import torch
    ps = synth.PlantedStream(side=64, noise_var=1e-3, seed=synth.config_seed(1))
    n = ps.n
    X = torch.from_numpy(np.stack([ps.snapshot(t) for t in range(n_snap)])).to(dev)
    sh = stream.cuda_stream
    out = {"n": n, "m": m, "r": r, "snapshots": n_snap}
    for D in depths:
        res = {}
        for traced in (False, True):
            h = S.sdmd_create_ex(n, m, S.SDMD_F32, D)
            phis = [torch.empty(r, n, 2, dtype=torch.float32, device=dev) for _ in range(max(D, 1))]
            lam = torch.empty(n_snap, 2 * r, dtype=torch.float64, device=dev)
            rk = torch.empty(n_snap, dtype=torch.int32, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            try:
                S.sdmd_trace(h, traced)
                torch.cuda.synchronize()
                e0.record(stream)
                with torch.cuda.stream(stream):
                    for t in range(n_snap):
                        S.sdmd_step(h, X[t], r, phis[t % len(phis)], lam[t], rk[t:t + 1], sh)
                    S.sdmd_sync(h, sh)
                e1.record(stream)
                stream.synchronize()
                if S.sdmd_status(h, sh) != S.SDMD_OK:
                    raise RuntimeError("config-1 status: " + S.sdmd_last_error())
                if traced:
                    fm = np.array(S.sdmd_trace_times(h, S.SDMD_K_FRAME))
                    if D == 1:
                        fm = np.array([])
                    ml, mms = S.sdmd_trace_read(h, S.SDMD_K_MODES)
                    res["modes_us"] = 1e3 * mms / max(ml, 1)
                    if fm.size:
                        res["latency_ms"] = {"p50": float(np.percentile(fm, 50)),
                                             "p99": float(np.percentile(fm, 99))}
                else:
                    ms = e0.elapsed_time(e1)
                    res["snapshots_per_s"] = n_snap / (ms * 1e-3)
                    res["ms_per_snapshot"] = ms / n_snap
                    if D == 1:
                        res["latency_ms"] = {"mean": ms / n_snap,
                                             "note": "one frame at a time: the step time is the latency"}
                S.sdmd_trace(h, False)
            finally:
                S.sdmd_destroy(h)
        out["depth%d" % D] = res
    out["note"] = ("FP32 rows (FP32 products, FP64 sums), df64 eigensolvers, CUDA-core Phi; the window "
                   "(512 KiB) stays in L2, so the step is latency-bound, not HBM-bound")
    return out


def conditioned_window(cs, ts, dev):
    """The conditioned-spectrum snapshots of synth.ConditionedStream for the
    times ts (len(ts) x n FP32), built on the device from the stream's own
    parameters (frequencies, cos/sin kind, geometric spectrum, seeded
    temporal coefficients): the same recipe as ConditionedStream.snapshots,
    evaluated in FP32 on the GPU because the host takes seconds per window at
    n = 2^22 (both arms of every comparison below read these FP32 values)."""
    import torch
    n = cs.n
    i = torch.arange(n, device=dev, dtype=torch.float64)
    A = torch.from_numpy(np.stack([cs.coeffs(t) * cs.s for t in ts])).to(dev)            # T x K
    X = torch.zeros(len(ts), n, device=dev, dtype=torch.float32)
    for k in range(cs.K):
        arg = (2.0 * np.pi * float(cs.freq[k]) / n) * i
        b = (torch.cos(arg) if cs.phase_kind[k] == 0 else torch.sin(arg)).float()
        X.add_(A[:, k:k + 1].float() * b[None, :])
    X.mul_(float(np.sqrt(2.0)))          # sqrt(2 / n) of the basis times sqrt(n)
    return X


def bf16x3_kappa_sweep(S, h, dev, stream, n, m, kappas=(1e2, 1e4, 1e6, 1e8), k=8, ns=16):
    """Gram error against host FP64 per condition number, at the precision
    sweep's size: per kappa a planted-spectrum window of m snapshots is
    pushed with FP32 rows, rebuilt with BF16x3, then moved by k snapshots
    with one BF16x3 catch-up; each Gram's sampled ns x ns block (ns window
    positions, including the k newest) is compared with FP64 dot products of
    the same FP32 snapshots computed on the host with numpy (the oracle's
    definition G = W^T W in FP64)."""
    import torch
    from paper_1612_07875_gb300 import synth
    sh = stream.cuda_stream
    G = torch.empty(m, m, dtype=torch.float64, device=dev)
    rows = []
    for kappa in kappas:
        cs = synth.ConditionedStream(n=n, K=m, kappa=kappa, seed=synth.config_seed(4))
        X = conditioned_window(cs, range(m + k), dev)
        torch.cuda.synchronize()             # built on torch's stream; the pushes run on `stream`
        sel = np.unique(np.concatenate([np.linspace(0, m - k - 1, ns - k).round().astype(int),
                                        np.arange(m - k, m)]))
        entry = {"kappa_target": kappa}
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 0)
        with torch.cuda.stream(stream):
            for t in range(m):
                S.sdmd_push(h, X[t], sh)
        for name, w0 in (("fp32_rows", 0), ("bf16x3_rebuild", 0), ("bf16x3_catch_up_k%d" % k, k)):
            with torch.cuda.stream(stream):
                if name == "bf16x3_rebuild":
                    S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 1)
                    S.sdmd_rebuild(h, sh)
                elif name.startswith("bf16x3_catch"):
                    S.sdmd_push_batch(h, k, X[m:m + k], n, sh)
                S.sdmd_gram(h, G, sh)
            stream.synchronize()
            Wh = X[w0 + sel].cpu().numpy().astype(np.float64)        # ns x n, exact FP32 values
            ref = Wh @ Wh.T
            bnd = np.abs(Wh) @ np.abs(Wh).T
            got = G.cpu().numpy()[np.ix_(sel, sel)]
            entry[name] = {"rel_frobenius": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                           "max_abs_err_over_sum_abs_products": float((np.abs(got - ref) / bnd).max())}
        Gf = G.cpu().numpy()
        lam = np.linalg.eigvalsh(Gf)
        # lambda_min below the Gram's rounding comes out <= 0: no finite condition number
        entry["cond_G_measured"] = float(lam.max() / lam.min()) if lam.min() > 0 else None
        entry["lambda_min_over_max"] = float(lam.min() / lam.max())
        rows.append(entry)
        del X
        torch.cuda.empty_cache()
    S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 0)
    return {"n": n, "m": m, "sampled_entries": ns * ns, "kappas": rows,
            "reference": "host FP64 (numpy) dot products of the same FP32 snapshots on a sampled "
                         "block; the full-window comparison with the oracle is the test "
                         "test_conditioned_full_size_kappa_1e8"}


def measure_sparse(S, synth, dev, stream, m=64, pushes=40):
    """Per-push time of the Fourier-sparse Gram row (scatter + row kernels)."""
    import torch
    fs = synth.FourierSparseStream(seed=synth.config_seed(3))
    snaps = [fs.snapshot(t) for t in range(m + 3 + pushes)]
    dev_snaps = [(torch.from_numpy(i).to(dev), torch.from_numpy(v.view(np.float32)).to(dev)) for i, v in snaps]
    sh = stream.cuda_stream
    h = S.sdmd_create_sparse(fs.N, m, fs.nnz + 16)
    try:
        for t in range(m + 3):
            i, v = dev_snaps[t]
            S.sdmd_push_sparse(h, i.numel(), i, v, sh)
        stream.synchronize()
        S.sdmd_trace(h, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(m + 3, m + 3 + pushes):
            i, v = dev_snaps[t]
            S.sdmd_push_sparse(h, i.numel(), i, v, sh)
        e1.record(stream)
        stream.synchronize()
        tot = e0.elapsed_time(e1)
        rl, rms = S.sdmd_trace_read(h, S.SDMD_K_GRAM_ROW)
        S.sdmd_trace(h, False)
        # f3: DMD in coefficient space -- complex small-matrix DMD, then the
        # compressed modes on the union support of X'
        r = 10
        fm = {}
        for rep in range(4):
            e0.record(stream)
            S.sdmd_modes(h, r, None, None, None, sh)
            e1.record(stream)
            stream.synchronize()
            t_modes = e0.elapsed_time(e1)
            cnt = S.sdmd_fourier_modes(h, r, stream=sh)
            if rep == 0:
                idx = torch.empty(cnt, dtype=torch.int32, device=dev)
                phi = torch.empty(r, cnt, 2, dtype=torch.float32, device=dev)
            e0.record(stream)
            S.sdmd_fourier_modes(h, r, idx, phi, cnt, sh)
            e1.record(stream)
            stream.synchronize()
            if rep:
                fm.setdefault("modes_ms", []).append(t_modes)
                fm.setdefault("fourier_modes_ms", []).append(e0.elapsed_time(e1))
        ok = S.sdmd_status(h, sh) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)
    nnz = fs.nnz
    return {"config": "1024x1024 complex64 field, nnz=%d (1%%), window m=%d" % (nnz, m),
            "snapshots/s": pushes / (tot * 1e-3), "push_us": 1e3 * tot / pushes,
            "row_kernels_us": 1e3 * rms / max(rl, 1),
            "algorithmic_bytes_per_push": m * nnz * 12 + nnz * 12, "status_ok": ok,
            "bound": "latency / L2 (lookup table 12 MB and window 8 MB are L2-resident)",
            "fourier_dmd": {"r": r, "modes_complex_ms": float(np.mean(fm["modes_ms"])),
                            "fourier_modes_ms": float(np.mean(fm["fourier_modes_ms"])),
                            "support": cnt, "compressed_output_bytes": cnt * (4 + 8 * r),
                            "dense_output_bytes": fs.N * 8 * r,
                            "note": "sdmd_modes (FP64 Jacobi + complex A~) and sdmd_fourier_modes "
                                    "(support bitmap, prefix, compaction, gathers) on the same window"}}


def measure_dense_complex(S, synth, dev, stream, m=64, pushes=20):
    """The same 1024 x 1024 field pushed dense: the physical complex64 field
    (the inverse transform of its coefficients) through the dense complex
    Gram row, m = 64 -- the HBM-bound alternative to the sparse row (Sec. 3.5:
    both give the same Gram by Parseval). Frames cycle through 8 fields
    generated before timing (the row's cost does not depend on the values)."""
    import torch
    fs = synth.FourierSparseStream(seed=synth.config_seed(3))
    n = fs.N
    X = torch.stack([torch.from_numpy(fs.physical(t).astype(np.complex64).view(np.float32)) for t in range(8)])
    X = X.to(dev)
    sh = stream.cuda_stream
    h = S.sdmd_create(n, m, S.SDMD_C64)
    try:
        for t in range(m + 2):
            S.sdmd_push(h, X[t % 8], sh)
        stream.synchronize()
        chunk, _ = S.sdmd_autotune(h, sh)            # the Gram row's schedule for this shape
        S.sdmd_trace(h, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(pushes):
            S.sdmd_push(h, X[t % 8], sh)
        e1.record(stream)
        stream.synchronize()
        tot = e0.elapsed_time(e1)
        rl, rms = S.sdmd_trace_read(h, S.SDMD_K_GRAM_ROW)
        S.sdmd_trace(h, False)
        ok = S.sdmd_status(h, sh) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)
    peak, peak_kind = measured_peaks()
    row_us = 1e3 * rms / max(rl, 1)
    nbytes = m * n * 8
    return {"config": "1024x1024 complex64 physical field, window m=%d" % m,
            "snapshots/s": pushes / (tot * 1e-3), "push_us": 1e3 * tot / pushes, "row_kernel_us": row_us,
            "algorithmic_bytes_per_push": nbytes, "GB/s": nbytes / (row_us * 1e-6) / 1e9,
            "frac_of_copy_peak": nbytes / (row_us * 1e-6) / 1e9 / peak if peak else None,
            "autotuned_chunk_bytes": chunk, "status_ok": ok, "bound": "hbm"}


def measure_serving(S, synth, dev, seconds, capacity_ticks=12):
    """Batched serving of 64 concurrent streams (FP32 and uint8 mixed, n
    log-uniform in [2^16, 2^22], m in {16..256}, Poisson arrivals at 10-120 Hz
    each): windows filled first (untimed), then `seconds` of real-time
    arrivals submitted from pinned host memory as they fall due; each tick
    pushes every stream's oldest queued frame in one batched launch. Latency
    of a frame = its tick's completion minus its scheduled arrival. Then the
    closed-loop capacity: every stream pushes one device-resident frame per
    tick, batched (sdmd_push_many) against the same frames pushed one handle
    at a time (sdmd_push), both timed with CUDA events."""
    import torch
    from collections import deque
    mix = synth.ServingMix()
    specs = mix.specs
    DT = {"u8": S.SDMD_U8, "f32": S.SDMD_F32}
    EL = {"u8": 1, "f32": 4}
    pu8, pf32 = mix.pools()
    host = {"u8": torch.from_numpy(pu8).pin_memory(), "f32": torch.from_numpy(pf32).pin_memory()}
    devp = {k: v.to(dev) for k, v in host.items()}
    hbase = {k: v.data_ptr() for k, v in host.items()}
    dbase = {k: v.data_ptr() for k, v in devp.items()}
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.8)
    srv = S.sdmd_server_create(budget)
    st = S.sdmd_server_stream(srv)
    ns = len(specs)
    try:
        sids = [S.sdmd_server_open(srv, n, m, DT[k]) for k, n, m, _ in specs]
        active = sum(S.sdmd_server_state(srv, s) == S.SDMD_STREAM_ACTIVE for s in sids)
        fcount = [0] * ns

        def haddr(i):
            k, n, _, _ = specs[i]
            a = hbase[k] + EL[k] * mix.offset(i, fcount[i])
            fcount[i] += 1
            return a

        # warm-up: every window filled, then the Gram-row schedules autotuned
        for j in range(max(s[2] for s in specs)):
            for i in range(ns):
                if j < specs[i][2]:
                    S.sdmd_server_submit(srv, sids[i], haddr(i))
            S.sdmd_server_tick(srv)
        t_at = time.perf_counter()
        S.sdmd_server_autotune(srv)
        autotune_s = time.perf_counter() - t_at
        arr = mix.arrivals(seconds)
        ev_t = np.concatenate(arr) * 1e3
        ev_s = np.concatenate([np.full(len(a), i) for i, a in enumerate(arr)])
        order = np.argsort(ev_t, kind="stable")
        ev_t, ev_s = ev_t[order].tolist(), ev_s[order].tolist()
        backlog = [deque() for _ in range(ns)]
        qlen = [0] * ns
        gram_bytes = 0
        ticks = 0
        nxt, nev = 0, len(ev_t)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.2)
        S.sdmd_server_reset_stats(srv)
        T0 = S.sdmd_server_clock_ms()
        while True:
            now = S.sdmd_server_clock_ms() - T0
            while nxt < nev and ev_t[nxt] <= now:
                backlog[ev_s[nxt]].append(ev_t[nxt] + T0)
                nxt += 1
            queued = False
            for i in range(ns):
                b = backlog[i]
                while b and qlen[i] < 4:
                    S.sdmd_server_submit(srv, sids[i], haddr(i), b.popleft())
                    qlen[i] += 1
                if qlen[i]:
                    queued = True
            if queued:
                S.sdmd_server_tick(srv)
                ticks += 1
                for i in range(ns):
                    if qlen[i]:
                        qlen[i] -= 1
                        k, n, m, _ = specs[i]
                        gram_bytes += m * n * EL[k]
            elif nxt >= nev:
                break
            else:
                wait = (ev_t[nxt] - now) * 1e-3
                if wait > 0.0005:
                    time.sleep(wait - 0.0003)
        wall = (S.sdmd_server_clock_ms() - T0) * 1e-3
        clk = clocks.stop()
        p50, p99, frames = S.sdmd_server_stats(srv)
        served = {"streams": ns, "active": active, "seconds": seconds, "offered_hz": sum(s[3] for s in specs),
                  "frames": frames, "snapshots_per_s": frames / wall, "ticks": ticks,
                  "frames_per_tick": frames / max(ticks, 1),
                  "gram_GB/s": gram_bytes / wall / 1e9,
                  "latency_ms": {"p50": p50, "p99": p99,
                                 "definition": "tick completion (host) minus the frame's scheduled arrival"},
                  "hbm_footprint_GB": S.sdmd_server_used_bytes(srv) / 1e9, "budget_GB": budget / 1e9,
                  "clocks": clk}

        # tick cost, every stream one queued frame (device sources), graph
        # ticks against copies + kernel launched on the stream
        def daddr0(i):
            k, n, _, _ = specs[i]
            a = dbase[k] + EL[k] * mix.offset(i, fcount[i])
            fcount[i] += 1
            return a
        ticks = {}
        for graphs in (True, False, True, False):
            S.sdmd_server_set_graphs(srv, graphs)
            for rep in range(2):
                t0 = time.perf_counter()
                for _ in range(capacity_ticks):
                    for i in range(ns):
                        S.sdmd_server_submit(srv, sids[i], daddr0(i))
                    S.sdmd_server_tick(srv)
                el = (time.perf_counter() - t0) / capacity_ticks
                if rep:
                    key = "graph" if graphs else "direct"
                    ticks[key] = min(ticks.get(key, 1e9), el)
        S.sdmd_server_set_graphs(srv, True)
        served["tick_ms"] = {"graph": 1e3 * ticks["graph"], "direct": 1e3 * ticks["direct"],
                             "note": "host clock per closed-loop tick (64 submits of device-resident frames, "
                                     "the batched push, synchronisation)"}
        served["autotune_s"] = autotune_s
        served["graph_stats"] = dict(zip(("builds", "updates"), S.sdmd_server_graph_stats(srv)))

        # closed-loop capacity, device-resident frames
        hs = [S.sdmd_server_handle(srv, s) for s in sids]

        def daddr(i):
            k, n, _, _ = specs[i]
            a = dbase[k] + EL[k] * mix.offset(i, fcount[i])
            fcount[i] += 1
            return a
        tick_bytes = sum(m * n * EL[k] for k, n, m, _ in specs)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sobj = torch.cuda.ExternalStream(st)
        out = {}
        for mode in ("single", "batched", "single", "batched"):
            for rep in range(2):                      # untimed pass, then timed
                xs = [[daddr(i) for i in range(ns)] for _ in range(capacity_ticks)]
                torch.cuda.synchronize()
                e0.record(sobj)
                for t in range(capacity_ticks):
                    if mode == "batched":
                        S.sdmd_push_many(hs, xs[t], st)
                    else:
                        for i in range(ns):
                            S.sdmd_push(hs[i], xs[t][i], st)
                e1.record(sobj)
                torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[mode] = max(out.get(mode, 0.0), ns * capacity_ticks / (ms * 1e-3))
        for h in hs:
            if S.sdmd_status(h, st) != S.SDMD_OK:
                raise RuntimeError("served stream status: " + S.sdmd_last_error())
        served["capacity"] = {"batched_snapshots_per_s": out["batched"], "single_snapshots_per_s": out["single"],
                              "batched_gram_GB/s": out["batched"] / ns * tick_bytes / 1e9,
                              "ticks": capacity_ticks,
                              "note": "every stream pushes one frame per tick, windows full; batched = one "
                                      "sdmd_push_many launch per tick, single = one sdmd_push per stream"}
        # the served streams' DMD eigensolvers (r = min(10, m - 1)): one
        # sdmd_modes_many launch (a CTA per stream) against one sdmd_modes
        # launch per stream, in stream order
        rs = [min(R_MODES, m - 1) for _, _, m, _ in specs]
        lam_bufs = [torch.empty(2 * r, dtype=torch.float64, device="cuda") for r in rs]
        mt = {}
        for mode in ("per_stream", "batched", "per_stream", "batched"):
            for rep in range(2):
                torch.cuda.synchronize()
                e0.record(sobj)
                if mode == "batched":
                    S.sdmd_modes_many(hs, rs, lam_bufs, None, st)
                else:
                    for i in range(ns):
                        S.sdmd_modes(hs[i], rs[i], None, lam_bufs[i], None, st)
                e1.record(sobj)
                torch.cuda.synchronize()
            mt[mode] = min(mt.get(mode, 1e30), e0.elapsed_time(e1))
        served["modes"] = {"batched_ms": mt["batched"], "per_stream_ms": mt["per_stream"],
                           "streams": ns, "speedup": mt["per_stream"] / mt["batched"],
                           "note": "eigensolvers of every served stream (r = min(10, m - 1)); batched = one "
                                   "sdmd_modes_many launch, per_stream = one sdmd_modes per stream"}
        return served
    finally:
        S.sdmd_server_destroy(srv)
        del devp
        torch.cuda.empty_cache()


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1612_07875_gb300 import sdmd as S
    from paper_1612_07875_gb300 import synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, Wm = args.steps, max(args.warmup, 3)
    Kt = TRACED_STEPS
    vs = synth.VideoStream(seed=rank_seed(synth.config_seed(2), rank))
    n = vs.n
    nframes = M_WIN + Wm + K + Kt
    # every frame of the run resident in HBM before timing
    frames = torch.empty(nframes, n, dtype=torch.uint8, device=dev)
    for t in range(nframes):
        frames[t].copy_(torch.from_numpy(vs.frame(t)))
    torch.cuda.synchronize()

    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    D = max(1, args.depth)
    h = S.sdmd_create_ex(n, M_WIN, S.SDMD_U8, D)
    phis = [torch.empty(R_MODES, n, 2, dtype=torch.float32, device=dev) for _ in range(D)]
    lam = torch.empty(Wm + K + Kt, 2 * R_MODES, dtype=torch.float64, device=dev)
    rdev = torch.empty(Wm + K + Kt, dtype=torch.int32, device=dev)

    def steps(i0, count):
        with torch.cuda.stream(stream):
            for i in range(i0, i0 + count):
                S.sdmd_step(h, frames[M_WIN + i], R_MODES, phis[i % D], lam[i], rdev[i:i + 1], sh)

    # warm-up: fill the window, then Wm pipelined steps; the pipeline stays
    # full (depth - 1 frames' Phi still deferred) so the timed steps run in
    # steady state. The clock sampler starts first, so that the GPU is busy
    # with the warm-up steps right up to the timed region (no idle gap)
    with torch.cuda.stream(stream):
        for t in range(M_WIN):
            S.sdmd_push(h, frames[t], sh)
    stream.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    steps(0, Wm)
    stream.synchronize()             # (no status read here: it would drain the pipeline)

    # ---- timed region: K pipelined steps (push + DMD per frame), no tracing.
    #      Steady state: the pipeline is full when the region opens and when
    #      it closes, so each timed step runs one frame's Gram row and
    #      eigensolver launch and one earlier frame's Phi; the drain of the
    #      last depth - 1 frames' Phi is not part of a step (it runs in the
    #      traced pass below)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    steps(Wm, K)
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(total_ms, world, dev)
    value = job_rate(world, K, t_max)

    # ---- traced pass (after the timed one, same steady state): per-kernel
    #      CUDA-event durations for the roofline and per-frame latency
    S.sdmd_trace(h, True)
    tt0 = torch.cuda.Event(enable_timing=True)
    tt1 = torch.cuda.Event(enable_timing=True)
    tt0.record(stream)
    steps(Wm + K, Kt)
    tt1.record(stream)
    S.sdmd_sync(h, sh)               # drain (traced: the last frames' latency includes it)
    stream.synchronize()
    traced_ms = tt0.elapsed_time(tt1)
    frame_ms = np.array(S.sdmd_trace_times(h, S.SDMD_K_FRAME))
    traces = {k: S.sdmd_trace_read(h, k) for k in range(S.SDMD_K_COUNT) if k != S.SDMD_K_FRAME}
    S.sdmd_trace(h, False)
    if S.sdmd_status(h, sh) != S.SDMD_OK:     # the device status word covers warm-up, timed and traced steps
        raise RuntimeError("device status after the timed and traced steps: " + S.sdmd_last_error())
    per_step = frame_ms if frame_ms.size else np.array([traced_ms / Kt])

    # ---- the same kernels launched one at a time (no overlap): per-kernel
    #      durations without contention, for the kernel rooflines
    iso = measure_isolated(S, h, frames, 0, stream, phis[0], n)

    # ---- roofline of the dominant kernel: Phi of frame f fused with the Gram
    #      row of frame f + depth - 1 (one pass over the union of the windows)
    peak, peak_kind = measured_peaks()
    ktot = (M_WIN - 1) + (D - 1)
    fl, fms = traces[S.SDMD_K_FUSED]
    fused_us = 1e3 * fms / max(fl, 1)
    fused_bytes = ktot * n + n * R_MODES * 8      # union slots read once + Phi (n x r complex64) written
    fused_gbs = fused_bytes / (fused_us * 1e-6) / 1e9 if fl else 0.0
    gl, gms = traces[S.SDMD_K_GRAM_ROW]
    gram_us = 1e3 * gms / max(gl, 1)
    gram_bytes = M_WIN * n            # m slots x n bytes read (x_new is one of them)
    pl, pms = traces[S.SDMD_K_PHI]
    phi_us = 1e3 * pms / max(pl, 1)
    phi_bytes = (M_WIN - 1) * n + n * R_MODES * 8
    ml, mms = traces[S.SDMD_K_MODES]
    il, ims = traces[S.SDMD_K_INGEST]
    # this library's kernels launched in the timed region: the traced pass
    # runs the same steady-state steps, so its per-step count (a fused pass
    # is two kernels, the pass and its finish kernel; a frame's eigensolver
    # one (it reads G in place); an unfused Gram row one; the ingest one
    # (device frames with 16-byte aligned rows take the library's copy
    # kernel); the drain's Phi launches after the last traced step are not
    # counted) times the timed steps
    n_launch = int(round((2 * fl + gl + ml + il) * K / Kt))
    kernels = {"fused_phi_gram_row": {"launches": fl, "us": fused_us, "GB/s": fused_gbs,
                                      "algorithmic_bytes": fused_bytes, "union_slots": ktot},
               "gram_row": {"launches": gl, "us": gram_us,
                            "GB/s": gram_bytes / (gram_us * 1e-6) / 1e9 if gl else 0.0,
                            "note": "unfused launches only (window ramp-up)"},
               "phi": {"launches": pl, "us": phi_us, "GB/s": phi_bytes / (phi_us * 1e-6) / 1e9 if pl else 0.0,
                       "note": "unfused launches only (ramp-up, final sync)"},
               "modes_small_f64": {"launches": ml, "us": 1e3 * mms / max(ml, 1)},
               "ingest_copy": {"launches": il, "us": 1e3 * ims / max(il, 1)}}
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get("fused_phi_gram_row_u8_hd_m100_d%d" % (D - 1))
        except (OSError, ValueError):
            traffic = None

    # ---- end to end through the C ABI with pinned host frames: Wm warm-up
    #      steps fill the pipeline, then K timed steps; the region closes when
    #      every timed frame's eigenvalues and rank have landed in host memory
    #      (host clock between two device-wide synchronisations), with the
    #      pipeline full again (the last frames' Phi, device outputs, run in
    #      the next steps as in steady state)
    e2e = None
    if not args.no_e2e:
        Ke = K
        # pinned host frames copied as soon as each call is made (on the
        # handle's copy stream), overlapping the kernels queued before it
        S.sdmd_set_option(h, S.SDMD_OPT_HOST_EARLY_READ, 1)
        host = torch.empty(Wm + Ke, n, dtype=torch.uint8).pin_memory()
        host.copy_(frames[M_WIN:M_WIN + Wm + Ke].cpu())
        lam_h = torch.empty(Wm + Ke, 2 * R_MODES, dtype=torch.float64).pin_memory()
        r_h = torch.empty(Wm + Ke, dtype=torch.int32).pin_memory()
        with torch.cuda.stream(stream):
            for i in range(Wm):
                S.sdmd_step(h, host[i], R_MODES, phis[i % D], lam_h[i], r_h[i:i + 1], sh)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(Wm, Wm + Ke):
                S.sdmd_step(h, host[i], R_MODES, phis[i % D], lam_h[i], r_h[i:i + 1], sh)
        torch.cuda.synchronize()
        ems = max_over_ranks(1e3 * (time.perf_counter() - t0), world, dev)
        S.sdmd_sync(h, sh)
        stream.synchronize()
        got_k = r_h[Wm:].numpy()
        e2e = {"value": job_rate(world, Ke, ems), "unit": UNIT, "h2d_bytes_per_step": n,
               "d2h_bytes_per_step": 2 * R_MODES * 8 + 4, "steps": Ke,
               "ranks_read_back": [int(got_k.min()), int(got_k.max())],
               "note": "sdmd_step on pinned host frames with SDMD_OPT_HOST_EARLY_READ after a warm-up that "
                       "fills the pipeline; host clock from a device-wide synchronize before the first timed "
                       "call to one after the last, when every timed frame's lambda and rank are in pinned "
                       "host memory"}
    # ---- a9: full-window rebuild of G; f2: multi-column catch-up of 8 frames
    rebuild = sparse = catchup = None
    if not args.no_secondary:
        rebuild = measure_rebuild(S, h, stream, n)
        catchup = measure_catchup(S, h, frames, 0, stream, n)
    S.sdmd_destroy(h)
    band_frames = frames[:, :n // 64].cpu().numpy()     # CPU oracle sample (generated above)
    scpu_frames = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        scpu_frames = frames[:4].cpu().numpy()          # streaming CPU sample
    del frames
    torch.cuda.empty_cache()
    # ---- a10: Fourier-sparse Gram row, 1024x1024 field, nnz 10,486, m = 64
    if not args.no_secondary:
        sparse = measure_sparse(S, synth, dev, stream)
        sparse["dense_physical"] = measure_dense_complex(S, synth, dev, stream)

    # ---- the planted-mode FP32 stream (n = 4096, m = 32, 200 snapshots)
    config1 = None
    if not args.no_secondary:
        config1 = measure_config1(S, synth, dev, stream)

    # ---- FP32 window n = 2^22, m = 256: BF16x3 tensor-core catch-up / rebuild
    bf16x3 = None
    if not args.no_secondary:
        bf16x3 = measure_bf16x3(S, dev, stream)

    # ---- batched serving of 64 mixed streams (Poisson arrivals)
    serving = None
    if not args.no_secondary and args.serve_seconds > 0:
        serving = measure_serving(S, synth, dev, args.serve_seconds)

    cpu = scpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        scpu = streaming_cpu_rate(scpu_frames, args.scpu_seconds)
        rate, info = oracle_rate(band_frames, n, args.cpu_sample_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": info["threads"], "kind": "oracle",
               "sample": "%d oracle steps (exact int64 Gram recompute + dense FP64 DMD r=10) on a "
                         "%d-pixel band (1/64 of each frame), %.1f s; rate scaled to full frames by "
                         "n/band" % (info["steps"], info["band_pixels"], info["seconds"])}

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic (seeded HD-video-shaped frames; no dataset)",
        "config": workload_config(n, {"parallelism": "independent stream per GPU" if world > 1 else "1 GPU"}),
        "roofline": {"bound": "hbm", "kernel": "fused_phi_gram_row_u8", "achieved": fused_gbs, "peak": peak,
                     "unit": "GB/s", "frac": fused_gbs / peak, "traffic": traffic,
                     "peak_kind": "%s hbm_gbs (copy)" % peak_kind,
                     "algorithmic_bytes_per_launch": fused_bytes,
                     "gram_row_isolated": {"achieved": iso["gram_row_sustained"]["GB/s"],
                                           "frac": iso["gram_row_sustained"]["GB/s"] / peak,
                                           "us": iso["gram_row_sustained"]["us"],
                                           "single_after_modes_us": iso["gram_row"]["us"]},
                     "note": "Phi of frame f (tensor cores) and the exact Gram row of frame f + %d in one "
                             "pass over %d window slots; launch durations (CUDA events on the push stream) "
                             "from the traced pass of %d steady-state steps that follows the untraced timed "
                             "region, beside other frames' eigensolvers; gram_row_isolated: the stand-alone "
                             "Gram-row kernel (sdmd_push) alone on the GPU" % (D - 1, ktot, Kt)},
        "roofline_isolated": {"bound": "hbm", "kernel": "gram_row_u8",
                              "achieved": iso["gram_row_sustained"]["GB/s"], "peak": peak, "unit": "GB/s",
                              "frac": iso["gram_row_sustained"]["GB/s"] / peak,
                              "algorithmic_bytes_per_launch": gram_bytes,
                              "note": "the stand-alone Gram-row kernel of sdmd_push, 20 pushes back to back with "
                                      "nothing else on the GPU (kernels_isolated.gram_row: one launch after each "
                                      "sdmd_modes)"},
        "kernels_isolated": iso,
        "gram_update": {"GB/s_isolated": iso["gram_row_sustained"]["GB/s"],
                        "us_isolated": iso["gram_row_sustained"]["us"],
                        "frac_of_peak_isolated": iso["gram_row_sustained"]["GB/s"] / peak,
                        "in_pipeline": "fused into fused_phi_gram_row (the window is read once per frame for "
                                       "both the Gram row and Phi)"},
        "kernels": kernels,
        "latency_ms": {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99)),
                       "max": float(per_step.max()),
                       "definition": "per frame: sdmd_step call on the stream to its DMD outputs complete"},
        "pipeline_depth": D,
        "timing": {"rule": "steady state: warm-up steps leave depth - 1 frames' Phi deferred, the timed "
                           "region (tracing off) runs K steps and closes with the pipeline full again; "
                           "each timed step = one frame's ingest, fused Gram row, eigensolver launch and "
                           "an earlier frame's Phi; the drain runs after the traced pass, outside it",
                   "traced_steps": Kt, "traced_ms_per_step": traced_ms / Kt},
        "gpu_launches": n_launch,
        "rebuild": rebuild,
        "catch_up": catchup,
        "sparse_row": sparse,
        "serving": serving,
        "fp32_bf16x3": bf16x3,
        "config1_planted_f32": config1,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "cpu_streaming": scpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_case(name):
    """Small fixed workloads for profiler captures of one kernel each:
    bf16x3_catchup: 128 random FP32 frames of n = 2^20 fill a window of 128,
      then three sdmd_push_batch calls of k = 32 under SDMD_OPT_F32_BF16X3 = 1
      (gram_f32_tc launches: BF16x3 on the tensor cores, stacked B);
    f32_catchup: 256 random FP32 frames of n = 2^20 fill a window of 256, then
      three sdmd_push_batch calls of k = 8 under the same option (gram_f32_simt
      launches: FP32 products on the CUDA cores, two window rows per thread);
    batched_rows: 24 streams of the serving mix (each window at most 200 MB)
      take 260 frames each through sdmd_push_many (gram_rows_batched launches);
    fused_pass: the HD video stream (n = 1920 x 1080 x 3 uint8, m = 100,
      r = 10) fills its window, then 24 sdmd_step calls at the bench's default depth: the fused
      Phi + Gram-row launches of the bench's pipeline (phi_tc_u8 launches;
      the first ones are the steady-state fused passes)."""
    import torch

    from paper_1612_07875_gb300 import sdmd as S
    from paper_1612_07875_gb300 import synth
    dev = torch.device("cuda", 0)
    if name in ("bf16x3_catchup", "f32_catchup"):
        n, m, k = (1 << 20, 128, 32) if name == "bf16x3_catchup" else (1 << 20, 256, 8)
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        frames = torch.randn(m + k, n, device=dev, generator=g)
        h = S.sdmd_create(n, m, S.SDMD_F32)
        for t in range(m):
            S.sdmd_push(h, frames[t])
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 1)
        for _ in range(3):
            S.sdmd_push_batch(h, k, frames[m:m + k], n)
        torch.cuda.synchronize()
        ok = S.sdmd_status(h) == S.SDMD_OK
        S.sdmd_destroy(h)
        info = {"n": n, "m": m, "k": k, "launches": 3}
    elif name == "fused_pass":
        vs = synth.VideoStream(seed=synth.config_seed(2))
        n, D, T = vs.n, DEPTH, M_WIN + 24
        frames = torch.empty(T, n, dtype=torch.uint8, device=dev)
        for t in range(T):
            frames[t].copy_(torch.from_numpy(vs.frame(t)))
        h = S.sdmd_create_ex(n, M_WIN, S.SDMD_U8, D)
        phis = [torch.empty(R_MODES, n, 2, dtype=torch.float32, device=dev) for _ in range(D)]
        lam = torch.empty(T, 2 * R_MODES, dtype=torch.float64, device=dev)
        rk = torch.empty(T, dtype=torch.int32, device=dev)
        for t in range(M_WIN):
            S.sdmd_push(h, frames[t])
        for t in range(M_WIN, T):
            S.sdmd_step(h, frames[t], R_MODES, phis[t % D], lam[t], rk[t:t + 1])
        S.sdmd_sync(h)
        torch.cuda.synchronize()
        ok = S.sdmd_status(h) == S.SDMD_OK
        S.sdmd_destroy(h)
        info = {"n": n, "m": M_WIN, "r": R_MODES, "depth": D, "steps": T - M_WIN}
    else:
        mix = synth.ServingMix()
        specs = [sp for sp in mix.specs if sp[2] * sp[1] * (1 if sp[0] == "u8" else 4) <= 200e6][:24]
        dts = {"u8": S.SDMD_U8, "f32": S.SDMD_F32}
        hs = [S.sdmd_create(n, m, dts[kind]) for kind, n, m, _ in specs]
        g = torch.Generator(device=dev)
        g.manual_seed(3)
        pool = {"u8": torch.randint(0, 256, (mix.pool_len,), dtype=torch.uint8, device=dev, generator=g),
                "f32": torch.randn(mix.pool_len, device=dev, generator=g)}
        for j in range(260):
            S.sdmd_push_many(hs, [pool[kind][mix.offset(i, j):mix.offset(i, j) + n]
                                  for i, (kind, n, m, _) in enumerate(specs)])
        torch.cuda.synchronize()
        ok = all(S.sdmd_status(h) == S.SDMD_OK for h in hs)
        for h in hs:
            S.sdmd_destroy(h)
        info = {"streams": len(specs), "launches": 260,
                "GB_per_launch": sum(m * n * (1 if kind == "u8" else 4) for kind, n, m, _ in specs) / 1e9}
    if not ok:
        raise RuntimeError("device status after the %s case: %s" % (name, S.sdmd_last_error()))
    print(json.dumps({"case": name, "ok": True, **info}), flush=True)


def main():
    args = parse()
    if args.case:
        run_case(args.case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
