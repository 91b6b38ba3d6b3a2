#!/usr/bin/env python
"""Benchmark of the SRT3D hot path on GB300.

One step = the whole hot path on one synthetic lidar frame already resident
in HBM: photon sketch of the pixel-sorted stamp stream (Eq. 3), normalisation,
and SRT3D reconstruction from the sketch (matched-filter init + iterations of
gradient step, APSS depth projection and intensity smoothing, Eq. 8).

Workload: 256x256 pixels, T=4096, sigma=6 bins, 1000 photons/pixel (~65.5M
photons), SBR=0.5, 10% two-surface pixels, m=10, K=2, 30 iterations.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
on the host cores on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(rows=256, cols=256, T=4096, sigma=6.0, mean_photons=1000.0, sbr=0.5, two_surface_frac=0.10, m=10,
                iters=30, k_max=2)
WORKLOAD_NAME = "srt3d_256x256_T4096_m10_K2_it30"
METRIC = "photons/s sketched + SRT3D-reconstructed (frames/s, p50/p99 frame latency alongside)"
UNIT = "photons/s"
E2E_DEPTH = 3  # frames in flight in the end-to-end throughput run
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernels on this workload, from the committed ncu captures named
# beside them; a kernel changed since its capture must be taken out of here
NCU_TRAFFIC = {
    "iter_all": (7.777536e6, "profiles/k_iter_persistent_256x256_T4096_m10_K2_it30.md"),
    "sketch_stream": (136.272896e6, "profiles/k_sketch_stream_256x256_T4096_m10.md"),
}
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hist-steps", type=int, default=10)
    ap.add_argument("--hist-rows", type=int, default=512,
                    help="side of the square histogram frame of the histogram section (512 = the workload)")
    ap.add_argument("--only", choices=["all", "step", "hist", "serving", "batch", "surfaces", "pixelwise",
                                       "streamtc", "table1", "births"],
                    default="all")
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--cpu-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--ref-sample-seconds", type=float, default=None,
                    help="CPU seconds per worker and step of the reference arm (default: the run fits in minutes)")
    return ap.parse_args()


def spec_and_params():
    from paper_2203_00952_gb300 import synth

    w = WORKLOAD
    spec = synth.FrameSpec(rows=w["rows"], cols=w["cols"], T=w["T"], sigma=w["sigma"], mean_photons=w["mean_photons"],
                           sbr=w["sbr"], two_surface_frac=w["two_surface_frac"])
    prm = dict(iters=w["iters"], k_max=w["k_max"], radius=1, apss_h=2.5, d_max=6 * w["sigma"], depth_scale=0.125,
               prune_alpha=0.02, smooth_lambda=0.5, min_sep=3 * w["sigma"])
    return spec, prm


# ----------------------------------------------------------------- CPU oracle

def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_block(task):
    """One bounded sample of the FP64 oracle on a block of rows of the frame:
    the sketch of the block, the matched-filter init of its first p_in pixels,
    and the iterations on the block from its (untimed) init. Returns the stage
    times and the depth error of the result's first surface."""
    import numpy as np

    import oracle
    from oracle.reconstruct import Params
    from paper_2203_00952_gb300 import synth

    stamps, offsets, truth, rows_sk, cols, p_in, prm, T, m, sigma, n_max = task
    p = Params(**prm)
    t0 = time.perf_counter()
    hh = oracle.h_hat(synth.impulse_response(T, sigma), m)
    S, n = oracle.sketch_stream(stamps, offsets, T, m)
    z_blk = oracle.finalize(S, n)
    t_sk = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.init_matched_filter(z_blk[:p_in], n[:p_in], hh, T, p)
    t_init = time.perf_counter() - t0
    st = oracle.init_matched_filter(z_blk, n, hh, T, p)[:3]
    eta = oracle.step_sizes(hh, n_max, p.k_max, T)
    t0 = time.perf_counter()
    for _ in range(p.iters):
        st = oracle.iterate(z_blk, n, st[0], st[1], st[2], hh, T, rows_sk, cols, p, *eta)[:3]
    t_it = time.perf_counter() - t0
    err = np.abs(st[0][:, 0] - truth)
    det = st[2][:, 0].astype(bool) & (err <= 3 * sigma)
    return dict(t_sk=t_sk, t_init=t_init, t_it=t_it, photons=int(offsets[-1]),
                dae_bins=float(err[det].mean()) if det.any() else None, detections=float(det.mean()))


def cpu_oracle_samples(frame_index: int, budget_s: float, count: int, workers: int = 1):
    """Time the FP64 oracle on `count` bounded samples of the workload. A
    sample runs `workers` processes at once (the host's cores), each on its own
    block of rows with about `budget_s` seconds of CPU work; a worker's stage
    times scale to the whole frame, and the frame time with all workers is the
    slowest worker's estimate divided by their number. Each sample returns that
    full-frame throughput (photons/s), the one-core figure, a description and
    the oracle's depth error on the first block."""
    import numpy as np

    from paper_2203_00952_gb300 import synth

    spec, prm = spec_and_params()
    fr = synth.make_stream_frame(spec, synth.SEED_256x256, frame_index)
    P, T, m = spec.num_pixels, spec.T, WORKLOAD["m"]
    N = int(fr.offsets[-1])
    n_max = float(np.diff(fr.offsets.astype(np.int64)).max())
    scale = max(budget_s / 12.0, 1e-3)
    rows_sk = int(min(spec.rows, max(1, round(16 * scale))))
    p_sk = rows_sk * spec.cols
    p_in = int(min(p_sk, max(32, round(2048 * scale))))
    oprm = {k: prm[k] for k in ("iters", "k_max", "radius", "apss_h", "d_max", "depth_scale", "prune_alpha",
                                "smooth_lambda", "min_sep")}

    def task(j):
        r0 = (j * rows_sk) % (spec.rows - rows_sk + 1)
        a, b = r0 * spec.cols, r0 * spec.cols + p_sk
        lo, hi = int(fr.offsets[a]), int(fr.offsets[b])
        return (fr.stamps[lo:hi].copy(), (fr.offsets[a:b + 1] - fr.offsets[a]).astype(np.uint32),
                fr.truth.depth[a:b, 0].copy(), rows_sk, spec.cols, p_in, oprm, T, m, spec.sigma, n_max), (a, b)

    pool = None
    if workers > 1:
        import multiprocessing as mp

        pool = mp.get_context("spawn").Pool(workers)
    out = []
    try:
        for i in range(count):
            tasks = [task(i * workers + j) for j in range(workers)]
            args = [t for t, _ in tasks]
            res = pool.map(_oracle_block, args) if pool else [_oracle_block(args[0])]
            t_frames = [r["t_sk"] * P / p_sk + r["t_init"] * P / p_in + r["t_it"] * P / p_sk for r in res]
            t_frame = max(t_frames) / workers
            desc = (f"FP64 numpy oracle, {workers} process(es) x 1 thread, each on its own block: sketch of "
                    f"{p_sk} px (~{res[0]['photons']} photons), matched-filter init of {p_in} px, {WORKLOAD['iters']} "
                    f"iterations on a {rows_sk}x{spec.cols} block; each worker's stage times scaled to the "
                    f"{P}-pixel frame ({N} photons), frame time = slowest worker / {workers}")
            a, b = tasks[0][1]
            out.append(dict(value=N / t_frame, value_one_core=N / float(np.median(t_frames)), t_frame_s=t_frame,
                            cores=workers, sample=desc,
                            stages=dict(sketch_s=res[0]["t_sk"], init_s=res[0]["t_init"], iters_s=res[0]["t_it"]),
                            block=dict(first_pixel=a, last_pixel=b, dae_bins=res[0]["dae_bins"],
                                       detections=res[0]["detections"])))
    finally:
        if pool:
            pool.close()
            pool.join()
    return out


def run_cpu_child(budget_s: float, count: int = 1, frame_index: int = 0, workers: int = 1):
    """Run the oracle timing in a fresh process (a new interpreter, not a fork
    of one that touched the GPU; its workers are spawned), one thread per
    worker process."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-child", f"{budget_s}:{count}:{frame_index}:{workers}"]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError("cpu baseline failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid=None):
        self.samples = []
        self.proc = None
        self.t_on = self.t_off = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_uuid:
            cmd += ["-i", gpu_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark_on(self):
        self.t_on = time.time()

    def mark_off(self):
        self.t_off = time.time()

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        import statistics

        rows = [s for t, s in self.samples if self.t_on and self.t_off and self.t_on - 0.2 <= t <= self.t_off + 0.2]
        if not rows:
            rows = [s for _, s in self.samples[-3:]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        smx = [float(r[2]) for r in rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smx) if smx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- histogram path

HIST_M = 32


def hist_section(B, ctx, dev, steps, flush, rows=512):
    """Histogram sketch of the 512x512 x 4096-bin workload (10 000 counts/px,
    SBR 0.2, m = 32) in every precision: device time per launch (CUDA events,
    L2 evicted between launches), HBM roofline, tensor throughput, and the
    error against the FP64 oracle on sampled pixels. `rows` < 512 runs the
    same recipe on a rows x rows frame (a smaller case for profiling)."""
    import dataclasses

    import numpy as np
    import torch

    import oracle
    from paper_2203_00952_gb300 import synth

    spec = dataclasses.replace(synth.frame_512x512_hist(), rows=rows, cols=rows)
    hist, _ = synth.make_hist_frame_torch(spec, synth.SEED_512x512, device=dev)
    P, T, m = spec.num_pixels, spec.T, HIST_M
    S = torch.empty(P, m, 2, device=dev)
    n = torch.empty(P, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(5)
    pix = np.sort(rng.choice(P, 32, replace=False))
    y_s = hist[torch.from_numpy(pix).to(dev)].cpu().numpy().view(np.uint16)
    S_ref, n_ref = oracle.sketch_hist(y_s, m)
    hbm_peak, peak_kind = load_peaks()
    out = {"workload": f"hist_{rows}x{rows}_T4096_m32", "photon_equivalents_per_frame": int(n_ref.mean() * P)}
    names = {B.SRT3D_FP32: "fp32", B.SRT3D_FP16_SPLIT: "fp16_split", B.SRT3D_BF16: "bf16"}
    for prec in (B.SRT3D_FP16_SPLIT, B.SRT3D_BF16, B.SRT3D_FP32):
        for _ in range(2):
            B.srt3d_sketch_hist(ctx, hist, T, m, prec, S, n, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            B.srt3d_sketch_hist(ctx, hist, T, m, prec, S, n, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        B.srt3d_sync(ctx, stream)
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        alg_bytes = P * T * 2 + P * m * 8 + P * 4
        nn = 2 * ((2 * m + 15) // 16) * 16 if prec == B.SRT3D_FP16_SPLIT else ((2 * m + 15) // 16) * 16
        err = float(np.max(np.abs(np.asarray(S.cpu()).view(np.complex64)[pix, :, 0] - S_ref) / n_ref[:, None]))
        ach = alg_bytes / (ms / 1e3) / 1e9
        out[names[prec]] = {"ms": ms, "GB_per_s": ach, "hbm_frac": ach / hbm_peak,
                            "tensor_tflops": (2.0 * P * T * nn / (ms / 1e3) / 1e12) if prec else None,
                            "photons_per_s": float(n_ref.mean() * P / (ms / 1e3)),
                            "max_err_normalised": err}
    out["hbm_peak_gbs"] = hbm_peak
    out["peak_source"] = f"MEASURED_PEAKS.json ({peak_kind})"
    del hist, S, n
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------- stream via tensor cores
def stream_tc_section(B, ctx, dev, stamps, offsets, fr, spec, steps, flush):
    """Sketch of the 256x256 stamp stream three ways, at m = 10 and m = 32:
    the CUDA-core stream kernel (srt3d_sketch_stream), the composed
    tensor-core route (device histogram, then the split-FP16 tcgen05 sketch;
    srt3d_sketch_stream_tc) and the fused one (stamps sorted by stage, each
    stage's histogram built in shared memory; srt3d_sketch_stream_tc_fused).
    Device time per call (CUDA events, L2 evicted between calls), the error of
    the second against the first and whether the third equals the second bit
    for bit. Also the CUDA-core kernel at m = 1 and 4 against the HBM
    roofline."""
    import numpy as np
    import torch

    P, T = spec.num_pixels, spec.T
    N = int(fr.offsets[-1])
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "stream_256x256_T4096", "photons": N}

    def timed(fn):
        for _ in range(2):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        B.srt3d_sync(ctx, stream)
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    for m in (10, 32):
        S1 = torch.empty(P, m, 2, device=dev)
        S2 = torch.empty(P, m, 2, device=dev)
        n1 = torch.empty(P, dtype=torch.int32, device=dev)
        n2 = torch.empty(P, dtype=torch.int32, device=dev)
        ms_cc = timed(lambda: B.srt3d_sketch_stream(ctx, stamps, offsets, T, m, 0, S1, n1, stream))
        ms_tc = timed(lambda: B.srt3d_sketch_stream_tc(ctx, stamps, offsets, T, m, B.SRT3D_FP16_SPLIT, S2, n2,
                                                       stream))
        nn = torch.clamp(n1.to(torch.float32), min=1.0)[:, None]
        err = float(((S2 - S1).norm(dim=-1) / nn).max().item())
        out[f"m{m}"] = {"cuda_cores_ms": ms_cc, "tensor_cores_ms": ms_tc,
                        "cuda_cores_photons_per_s": N / (ms_cc / 1e3), "tensor_cores_photons_per_s": N / (ms_tc / 1e3),
                        "counts_equal": bool(torch.equal(n1, n2)), "max_diff_normalised": err}
        try:
            S3 = torch.empty(P, m, 2, device=dev)
            n3 = torch.empty(P, dtype=torch.int32, device=dev)
            ms_fu = timed(lambda: B.srt3d_sketch_stream_tc_fused(ctx, stamps, offsets, T, m, B.SRT3D_FP16_SPLIT,
                                                                 S3, n3, stream))
            # the fused route's two kernels, timed apart (profiler events)
            B.srt3d_profile_enable(ctx, True)
            for i in range(3):
                flush.fill_(float(i))
                B.srt3d_sketch_stream_tc_fused(ctx, stamps, offsets, T, m, B.SRT3D_FP16_SPLIT, S3, n3, stream)
            torch.cuda.synchronize(dev)
            prof = B.profile_totals(ctx)
            B.srt3d_profile_enable(ctx, False)
            out[f"m{m}"].update({
                "fused_tensor_cores_ms": ms_fu, "fused_tensor_cores_photons_per_s": N / (ms_fu / 1e3),
                "fused_kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items()
                                     if k in ("bucket_stream", "sketch_stream_tc")},
                "fused_equals_composed": bool(torch.equal(S2, S3) and torch.equal(n2, n3))})
            del S3, n3
        except Exception as exc:  # the main line must still print
            out[f"m{m}"]["fused_error"] = repr(exc)[:200]
            try:
                B.srt3d_profile_enable(ctx, False)
            except Exception:
                pass
        del S1, S2, n1, n2
    # few harmonics: where the CUDA-core kernel's arithmetic falls below its
    # 2 bytes per photon, it is bound by HBM (algorithmic bytes: the stamps,
    # the offsets, the sums and the counts)
    hbm_peak, peak_kind = load_peaks()
    for m in (1, 4):
        try:
            S1 = torch.empty(P, m, 2, device=dev)
            n1 = torch.empty(P, dtype=torch.int32, device=dev)
            ms = timed(lambda: B.srt3d_sketch_stream(ctx, stamps, offsets, T, m, 0, S1, n1, stream))
            gbs = (2 * N + 4 * (P + 1) + 8 * m * P + 4 * P) / (ms / 1e3) / 1e9
            out[f"m{m}"] = {"cuda_cores_ms": ms, "cuda_cores_photons_per_s": N / (ms / 1e3), "GB_per_s": gbs,
                            "hbm_frac": gbs / hbm_peak, "peak_source": f"MEASURED_PEAKS.json ({peak_kind})"}
            del S1, n1
        except Exception as exc:  # the main line must still print
            out[f"m{m}"] = {"error": repr(exc)[:200]}
    return out


# ----------------------------------------------------------------- array sizes of Table 1
TABLE1_SIZES = (141, 282, 423, 564, 705)


def table1_section(B, ctx, dev, steps, flush):
    """SRT3D on the array sizes of the paper's timing table (Table 1: 141^2 to
    705^2 pixels, m = 5 and 10; head-like frames, T = 4613, one surface per
    pixel, SBR 1, 100 photons per pixel; 30 iterations, since the table states
    no count). Device time per frame (CUDA events, L2 evicted between frames)
    of the reconstruction alone (init + iterations) and of the whole step
    (sketch, finalize, reconstruct). The paper's numbers are from a laptop
    RTX 3070: context, not a target."""
    import numpy as np
    import torch

    from paper_2203_00952_gb300 import synth

    T, sigma = 4613, 6.0
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "srt3d_table1_sizes_T4613_K1_it30_100ph_sbr1", "iters": 30, "k_max": 1,
           "paper_ms_rtx3070_laptop": {"m5": [6, 12, 28, 55, 68], "m10": [7, 18, 35, 60, 88]}}
    for side in TABLE1_SIZES:
        try:
            spec = synth.FrameSpec(rows=side, cols=side, T=T, sigma=sigma, mean_photons=100.0, sbr=1.0)
            stamps, offsets, _ = synth.make_stream_frame_torch(spec, synth.SEED_256x256 + 11, 0, device=dev)
            P = spec.num_pixels
            N = int(offsets[-1].item())
            h = torch.from_numpy(synth.impulse_response(T, sigma).astype(np.float32)).to(dev)
            depth = torch.empty(P, 1, device=dev)
            alpha = torch.empty(P, 1, device=dev)
            active = torch.empty(P, 1, dtype=torch.uint8, device=dev)
            alpha0 = torch.empty(P, device=dev)
            prm = B.make_params(iters=30, k_max=1, d_max=6 * sigma, min_sep=3 * sigma)
            row = {"pixels": P, "photons": N}
            for m in (5, 10):
                S = torch.empty(P, m, 2, device=dev)
                n = torch.empty(P, dtype=torch.int32, device=dev)

                def sketch():
                    B.srt3d_sketch_stream(ctx, stamps, offsets, T, m, 0, S, n, stream)
                    B.srt3d_finalize(ctx, S, n, m, S, stream)

                def recon():
                    B.srt3d_reconstruct(ctx, S, n, side, side, T, m, h, prm, depth, alpha, active, alpha0,
                                        stream)

                sketch()
                recon()
                ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
                for i in range(steps):
                    flush.fill_(float(i))
                    ev[i][0].record(stream)
                    sketch()
                    ev[i][1].record(stream)
                    recon()
                    ev[i][2].record(stream)
                torch.cuda.synchronize(dev)
                B.srt3d_sync(ctx, stream)
                rec = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
                full = float(np.mean([e[0].elapsed_time(e[2]) for e in ev]))
                row[f"m{m}"] = {"reconstruct_ms": rec, "step_ms": full, "frames_per_s": 1e3 / full}
                del S, n
            out[f"{side}x{side}"] = row
            del stamps, offsets, depth, alpha, active, alpha0
            torch.cuda.empty_cache()
        except Exception as exc:  # the main line must still print
            out[f"{side}x{side}"] = {"error": repr(exc)[:200]}
    return out


def births_section(B, ctx, dev, stamps, offsets, fr, spec, prm_main, steps, flush):
    """The benchmark frame reconstructed with RT3D's birth move after
    iterations 10 and 20 (birth_every = 10) beside the same reconstruction
    without births, from an init whose second surfaces were dropped (the case
    births exist for): device time of the reconstruction and the share of
    true second surfaces found within 3 sigma."""
    import numpy as np
    import torch

    from paper_2203_00952_gb300 import synth

    P, T, m, K = spec.num_pixels, spec.T, WORKLOAD["m"], WORKLOAD["k_max"]
    stream = torch.cuda.current_stream(dev)
    S = torch.empty(P, m, 2, device=dev)
    n = torch.empty(P, dtype=torch.int32, device=dev)
    B.srt3d_sketch_stream(ctx, stamps, offsets, T, m, 0, S, n, stream)
    B.srt3d_finalize(ctx, S, n, m, S, stream)
    h = torch.from_numpy(synth.impulse_response(T, spec.sigma).astype(np.float32)).to(dev)
    bufs = [torch.empty(P, K, device=dev), torch.empty(P, K, device=dev),
            torch.empty(P, K, dtype=torch.uint8, device=dev), torch.empty(P, device=dev)]
    p_init = B.make_params(init_mode=B.SRT3D_INIT_MATCHED, **{**prm_main, "iters": 0})
    B.srt3d_reconstruct(ctx, S, n, spec.rows, spec.cols, T, m, h, p_init, *bufs, stream)
    init = [b.clone() for b in bufs]
    init[1][:, 1:] = 0.0
    init[2][:, 1:] = 0
    has2 = fr.truth.nsurf == 2
    out = {"workload": WORKLOAD_NAME + "_second_surfaces_dropped_at_init", "birth_every": 10}
    for name, be in (("without_births", 0), ("with_births", 10)):
        prm = B.make_params(init_mode=B.SRT3D_INIT_GIVEN, birth_every=be, **prm_main)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps + 1):
            for b, b0 in zip(bufs, init):
                b.copy_(b0)
            flush.fill_(float(i))
            if i:
                ev[i - 1][0].record(stream)
            B.srt3d_reconstruct(ctx, S, n, spec.rows, spec.cols, T, m, h, prm, *bufs, stream)
            if i:
                ev[i - 1][1].record(stream)
        torch.cuda.synchronize(dev)
        B.srt3d_sync(ctx, stream)
        d = bufs[0].cpu().numpy()
        act = bufs[2].cpu().numpy().astype(bool)
        err = np.abs(d[:, :, None] - np.nan_to_num(fr.truth.depth, nan=-1e9)[:, None, :])
        err = np.minimum(err, T - err)
        found2 = (np.where(act[:, :, None], err, np.inf)[:, :, 1].min(axis=1) <= 3 * spec.sigma)
        out[name] = {"reconstruct_ms": float(np.mean([a.elapsed_time(b) for a, b in ev])),
                     "second_surfaces_found": float(found2[has2].mean())}
    return out


# ----------------------------------------------------------------- pixelwise
def pixelwise_section(B, ctx, dev, stamps, offsets, fr, spec, prm_main, steps, flush):
    """Pixelwise sketched estimates on the 256x256 frame (regularize = 0,
    K = 2, 30 steps): W = I (the SMLE comparison of Sec. 4) and W =
    (Sigma_theta + ridge I)^-1 (Eq. 6); step time (sketch, finalize,
    reconstruct; CUDA events, L2 evicted between steps) and the depth error
    of the first surface against the synthetic truth."""
    import numpy as np
    import torch

    from paper_2203_00952_gb300 import synth

    P, T, m, K = spec.num_pixels, spec.T, WORKLOAD["m"], WORKLOAD["k_max"]
    N = int(fr.offsets[-1])
    S = torch.empty(P, m, 2, device=dev)
    n = torch.empty(P, dtype=torch.int32, device=dev)
    depth = torch.empty(P, K, device=dev)
    alpha = torch.empty(P, K, device=dev)
    active = torch.empty(P, K, dtype=torch.uint8, device=dev)
    alpha0 = torch.empty(P, device=dev)
    h = torch.from_numpy(synth.impulse_response(T, spec.sigma).astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "pixelwise_256x256_T4096_m10_K2_it30"}
    for name, wgt in (("W_identity", 0), ("W_precision", 1)):
        prm = B.make_params(iters=prm_main.iters, k_max=K, regularize=0, weighting=wgt, d_max=prm_main.d_max,
                            min_sep=prm_main.min_sep)

        def step():
            B.srt3d_sketch_stream(ctx, stamps, offsets, T, m, 0, S, n, stream)
            B.srt3d_finalize(ctx, S, n, m, S, stream)
            B.srt3d_reconstruct(ctx, S, n, spec.rows, spec.cols, T, m, h, prm, depth, alpha, active, alpha0, stream)

        for _ in range(3):
            step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        d = depth.cpu().numpy()
        act = active.cpu().numpy().astype(bool)
        err = np.abs(d[:, 0] - fr.truth.depth[:, 0])
        err = np.minimum(err, T - err)
        det = act[:, 0] & (err <= 3 * spec.sigma)
        out[name] = {"ms_per_step": ms, "photons_per_s": N / (ms / 1e3), "dae_bins": float(err[det].mean()),
                     "detections": float(det.mean())}
    del S, n, depth, alpha, active, alpha0
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------- K = 3
SURF = dict(rows=256, cols=256, T=4096, sigma=6.0, mean_photons=1500.0, sbr=1.0, sep_lo=300.0, sep_hi=700.0,
            n_surf=3, m=20, iters=30)


def surfaces_section(B, ctx, dev, steps, flush):
    """Three surfaces per pixel (k_max = 3): a 256x256 frame with three
    surfaces 300-700 bins apart in every pixel, m = 20, 30 iterations; the
    whole step (sketch, finalize, reconstruct) timed with CUDA events, L2
    evicted between steps, and the recovery of the true surfaces."""
    import numpy as np
    import torch

    from paper_2203_00952_gb300 import synth

    w = SURF
    spec = synth.FrameSpec(rows=w["rows"], cols=w["cols"], T=w["T"], sigma=w["sigma"],
                           mean_photons=w["mean_photons"], sbr=w["sbr"], sep_lo=w["sep_lo"], sep_hi=w["sep_hi"])
    fr = synth.make_multi_surface_frame(spec, w["n_surf"], synth.SEED_256x256 + 7)
    P, T, m, K = spec.num_pixels, spec.T, w["m"], w["n_surf"]
    N = int(fr.offsets[-1])
    stamps = torch.from_numpy(fr.stamps.view(np.int16)).to(dev)
    offsets = torch.from_numpy(fr.offsets.view(np.int32)).to(dev)
    S = torch.empty(P, m, 2, device=dev)
    n = torch.empty(P, dtype=torch.int32, device=dev)
    depth = torch.empty(P, K, device=dev)
    alpha = torch.empty(P, K, device=dev)
    active = torch.empty(P, K, dtype=torch.uint8, device=dev)
    alpha0 = torch.empty(P, device=dev)
    h = torch.from_numpy(synth.impulse_response(T, spec.sigma).astype(np.float32)).to(dev)
    prm = B.make_params(iters=w["iters"], k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    stream = torch.cuda.current_stream(dev)

    def step():
        B.srt3d_sketch_stream(ctx, stamps, offsets, T, m, 0, S, n, stream)
        B.srt3d_finalize(ctx, S, n, m, S, stream)
        B.srt3d_reconstruct(ctx, S, n, spec.rows, spec.cols, T, m, h, prm, depth, alpha, active, alpha0, stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    B.srt3d_profile_enable(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    st = B.srt3d_sync(ctx, stream, check=False)
    prof = B.profile_totals(ctx)
    B.srt3d_profile_enable(ctx, False)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    d = depth.cpu().numpy()
    act = active.cpu().numpy().astype(bool)
    err = np.abs(d[:, :, None] - fr.truth.depth[:, None, :])
    err = np.minimum(err, T - err)
    found = float(np.mean(np.where(act[:, :, None], err, np.inf).min(axis=1) <= 3 * spec.sigma))
    del stamps, offsets, S, n, depth, alpha, active, alpha0
    torch.cuda.empty_cache()
    return {"workload": f"srt3d_256x256_T4096_m20_K3_it30_three_surfaces", "photons_per_frame": N,
            "ms_per_step": ms, "photons_per_s": N / (ms / 1e3), "frames_per_s": 1e3 / ms,
            "kernel_ms": {k: v[0] / v[1] for k, v in prof.items()}, "surfaces_found_within_3sigma": found,
            "device_status": int(st)}


# ----------------------------------------------------------------- serving

SERVE = dict(sizes=(128, 256, 512), T=2048, m=16, sigma=4.0, nbar=(50.0, 2000.0), sbr=1.0, chunks=8, iters=25,
             rate=300.0)


def chunk_split(stamps, offsets, nchunks):
    """Split every pixel's photons into `nchunks` consecutive runs (arrival
    order); returns a list of (stamps, offsets) numpy arrays."""
    import numpy as np

    off = offsets.astype(np.int64)
    cnt = np.diff(off)
    out = []
    for k in range(nchunks):
        a = off[:-1] + (k * cnt) // nchunks
        b = off[:-1] + ((k + 1) * cnt) // nchunks
        ln = b - a
        o = np.zeros(len(cnt) + 1, np.uint32)
        np.cumsum(ln, out=o[1:])
        idx = np.repeat(a - o[:-1].astype(np.int64), ln) + np.arange(int(o[-1]))
        out.append((stamps[idx], o))
    return out


def serving_section(B, dev, seconds):
    """Frames arrive as a Poisson process; each frame's photons come in 8
    chunks spread over 1/300 s (host pinned buffers) and are sketched online
    on the device; the last chunk starts the reconstruction; results are
    polled back to host memory. Reports latency from the last chunk to the
    result (and from the first chunk), and the sustained photon rate."""
    import heapq

    import numpy as np
    import torch

    from paper_2203_00952_gb300 import synth

    cfg = SERVE
    rng = np.random.default_rng(synth.SEED_SERVE)
    pool = []
    for i, n in enumerate(cfg["sizes"]):
        for nbar in (150.0, 800.0):  # two photon levels per size inside the log-uniform range
            spec = synth.FrameSpec(rows=n, cols=n, T=cfg["T"], sigma=cfg["sigma"], mean_photons=nbar,
                                   sbr=cfg["sbr"], two_surface_frac=0.1)
            fr = synth.make_stream_frame(spec, synth.SEED_SERVE, len(pool))
            ch = []
            for st, off in chunk_split(fr.stamps, fr.offsets, cfg["chunks"]):
                st_p = torch.from_numpy(st.view(np.int16)).pin_memory().numpy().view(np.uint16)
                off_p = torch.from_numpy(off.view(np.int32)).pin_memory().numpy().view(np.uint32)
                ch.append((st_p, off_p))
            pool.append((spec, ch, int(fr.offsets[-1])))
    h = {cfg["sigma"]: synth.impulse_response(cfg["T"], cfg["sigma"]).astype(np.float32)}
    prm = B.make_params(iters=cfg["iters"], k_max=2, d_max=6 * cfg["sigma"], min_sep=3 * cfg["sigma"])
    ctx = B.srt3d_create(int(dev.index or 0))
    outbuf = {}

    def out_for(spec):
        key = (spec.rows, spec.cols)
        if key not in outbuf:
            P = spec.num_pixels
            outbuf[key] = (np.zeros((P, 2), np.float32), np.zeros((P, 2), np.float32), np.zeros((P, 2), np.uint8),
                           np.zeros(P, np.float32), None)
        return outbuf[key]

    # warm-up: one frame of each pool entry
    for j, (spec, ch, _) in enumerate(pool):
        for k, (st, off) in enumerate(ch):
            B.srt3d_submit(ctx, 10**9 + j, spec.rows, spec.cols, spec.T, cfg["m"], h[cfg["sigma"]], prm, st, off,
                           int(k == len(ch) - 1))
        B.srt3d_poll(ctx, 10**9 + j, 60_000_000, *out_for(spec))
    arrivals = np.cumsum(rng.exponential(1.0 / cfg["rate"], size=int(seconds * cfg["rate"] * 1.5) + 8))
    arrivals = arrivals[arrivals < seconds]
    choice = rng.integers(0, len(pool), size=len(arrivals))
    # chunk k of frame i is due at arrival_i + k / (rate * chunks); chunk k+1
    # is scheduled only once chunk k has been accepted
    events = [(float(t), i, 0) for i, t in enumerate(arrivals)]
    heapq.heapify(events)
    t0 = time.perf_counter()
    deadline = seconds + 120.0
    first_at, last_at, lat_last, lat_first, photons = {}, {}, [], [], 0
    inflight = []
    busy_retries = 0
    while events or inflight:
        now = time.perf_counter() - t0
        if now > deadline:
            raise RuntimeError(f"serving run exceeded {deadline:.0f} s ({len(inflight)} frames in flight)")
        if events and events[0][0] <= now:
            t, i, k = heapq.heappop(events)
            spec, ch, nph = pool[choice[i]]
            st, off = ch[k]
            rc = B.srt3d_submit(ctx, i, spec.rows, spec.cols, spec.T, cfg["m"], h[cfg["sigma"]], prm, st, off,
                                int(k == cfg["chunks"] - 1), check=False)
            if rc == B.SRT3D_EBUSY:
                busy_retries += 1
                heapq.heappush(events, (now + 2e-4, i, k))
            elif rc != B.SRT3D_OK:
                raise RuntimeError(f"srt3d_submit failed: {rc}")
            else:
                if k == 0:
                    first_at[i] = time.perf_counter()
                if k == cfg["chunks"] - 1:
                    last_at[i] = time.perf_counter()
                    inflight.append(i)
                else:
                    due = float(arrivals[i]) + (k + 1) / (cfg["rate"] * cfg["chunks"])
                    heapq.heappush(events, (max(due, now), i, k + 1))
        # poll every frame in flight without waiting
        progressed = False
        for i in list(inflight):
            spec, ch, nph = pool[choice[i]]
            rc = B.srt3d_poll(ctx, i, 0, *out_for(spec), check=False)
            if rc == B.SRT3D_OK:
                tnow = time.perf_counter()
                lat_last.append(tnow - last_at[i])
                lat_first.append(tnow - first_at[i])
                photons += nph
                inflight.remove(i)
                progressed = True
            elif rc != B.SRT3D_ETIMEDOUT:
                raise RuntimeError(f"srt3d_poll failed: {rc}")
        if not progressed and events:
            wait = events[0][0] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 2e-4))
    wall = time.perf_counter() - t0
    B.srt3d_destroy(ctx)
    lat_last = np.array(lat_last) * 1e3
    lat_first = np.array(lat_first) * 1e3
    return {"workload": "serving_poisson300_T2048_m16_K2_it25_8chunks", "seconds_offered": seconds,
            "frames": int(len(lat_last)), "photons_per_s": photons / wall, "frames_per_s": len(lat_last) / wall,
            "latency_last_chunk_ms": {"p50": float(np.percentile(lat_last, 50)),
                                      "p99": float(np.percentile(lat_last, 99))},
            "latency_first_chunk_ms": {"p50": float(np.percentile(lat_first, 50)),
                                       "p99": float(np.percentile(lat_first, 99))},
            "admission_retries": busy_retries,
            "pool": "6 frames: {128,256,512}^2 x {150, 800} photons/px, SBR 1, 10% two-surface; chunks from pinned "
                    "host memory"}


# ----------------------------------------------------------------- batched uneven frames

def batch_section(B, ctx, dev, steps, flush):
    """64 uneven frames (sizes {64,128,256,512}^2, T in {1024,4096}, m in
    {4,16}, photons/px log-uniform [10,5000], SBR log-uniform [0.05,5]) through
    srt3d_process_batch: one launch per stage over all frames, the 20
    iterations of all frames in one cooperative launch, one CUDA graph per
    batch. The first call tunes (sketch lanes, iteration tile height) and
    captures; the timed calls replay."""
    import numpy as np
    import torch

    from paper_2203_00952_gb300 import synth

    specs = synth.batch_specs(64)
    frames, keep = [], []
    photons = 0
    for i, (spec, m) in enumerate(specs):
        st, off, _ = synth.make_stream_frame_torch(spec, synth.SEED_BATCH, i, device=dev)
        P = spec.num_pixels
        h = torch.from_numpy(synth.impulse_response(spec.T, spec.sigma).astype(np.float32)).to(dev)
        bufs = (torch.empty(P, m, 2, device=dev), torch.empty(P, dtype=torch.int32, device=dev),
                torch.empty(P, 2, device=dev), torch.empty(P, 2, device=dev),
                torch.empty(P, 2, dtype=torch.uint8, device=dev), torch.empty(P, device=dev))
        frames.append(B.make_frame(st, off, spec.rows, spec.cols, spec.T, m, h, *bufs))
        keep.append((st, off, h, bufs))
        photons += st.numel()
    prm = B.make_params(iters=20, k_max=2, d_max=36.0, min_sep=18.0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    B.srt3d_process_batch(ctx, frames, prm, stream)
    B.srt3d_sync(ctx, stream)
    setup_s = time.perf_counter() - t0
    for _ in range(2):
        B.srt3d_process_batch(ctx, frames, prm, stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        B.srt3d_process_batch(ctx, frames, prm, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    B.srt3d_sync(ctx, stream)
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    del keep, frames
    torch.cuda.empty_cache()
    return {"workload": "batch64_uneven_T1024-4096_m4-16_K2_it20", "frames": len(specs), "photons": photons,
            "ms_per_batch": ms, "photons_per_s": photons / (ms / 1e3), "frames_per_s": len(specs) / (ms / 1e3),
            "first_call_s": setup_s,
            "launch": "one CUDA graph per batch: one sketch launch per m class (writing z = S/n), one prep "
                      "launch, one init launch per instantiated m, and one cooperative launch running the 20 "
                      "iterations of all frames"}


# ----------------------------------------------------------------- GPU arm

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def fp32_peak_tflops():
    """FP32 FMA peak in flops: SMs x 128 lanes x 2 flops x max SM clock
    (80.5 TFLOP/s on a GB300; there is no measured FP32 figure)."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def mf_grid_spacing(T, m):
    """Grid spacing D of the matched-filter branch and bound (largest power
    of two <= 64 with w_m^2 D^2 / 8 <= 0.08, w_m = 2 pi m / T)."""
    w = 2.0 * math.pi * m / T
    D = 64
    while D > 1 and w * w * D * D / 8.0 > 0.08:
        D //= 2
    return D


# ----------------------------------------------------------------- multi-rank
# Frames are independent, so N ranks are N replicas: each rank sketches and
# reconstructs its own frame (seeded by its rank), the step time is the
# maximum over ranks, and the value counts the photons of all ranks.

def rank_frame(spec, rank):
    """The frame of rank `rank` (independent seeded frames, no data exchange)."""
    from paper_2203_00952_gb300 import synth

    return synth.make_stream_frame(spec, synth.SEED_256x256, rank)


def max_over_ranks(total_ms, world, device):
    """Largest timed-region duration over the ranks (all ranks get it)."""
    if world <= 1:
        return float(total_ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, photons_per_frame, steps, total_ms):
    """Whole-job photons per second: every rank processes one frame per step."""
    return world * photons_per_frame * steps / (total_ms / 1e3)


def kernel_work(name, N, P, m, T, K, iters, act_pts):
    """Algorithmic work of one launch of kernel `name` in FP32 flops (an FMA
    counts two). act_pts = active points (pixel, surface) per iteration
    (the mean of the counts after init and after the last iteration).
    Returns (bound, amount, unit)."""
    if name == "sketch_stream":
        # per photon: the first harmonic a table value accumulated (2 flops),
        # each further harmonic one packed Chebyshev FMA on (re, im) (4 flops)
        # and its accumulation (2 flops)
        return "alu", N * (6 * m - 4) / 1e12, "TFLOP"
    if name == "init":
        # the scores every pixel needs, per pixel and pass: every grid point
        # t = g D by complex Horner, 4 FMA per harmonic after the first and 2
        # for the last step; surviving intervals are not counted
        G = -(-T // mf_grid_spacing(T, m))
        return "alu", P * K * G * 2 * (4 * m - 2) / 1e12, "TFLOP"
    # the iteration (per point and iteration, active points only): m complex
    # multiply-accumulates of the gradient (8 flops each) and (2r+1)^2 K
    # neighbour terms of the APSS normal, sphere and smoothing sums (~60 flops
    # each, r = 1)
    per_iter = act_pts * (8 * m + 9 * K * 60)
    if name == "iter":
        return "alu", per_iter / 1e12, "TFLOP"
    if name == "iter_all":
        return "alu", iters * per_iter / 1e12, "TFLOP"
    if name == "finalize":
        return "hbm", (P * m * 16 + P * 4) / 1e9, "GB"
    return None, None, None


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2203_00952_gb300 import binding as B
    from paper_2203_00952_gb300 import build as builder
    from paper_2203_00952_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    builder.build()
    if args.only == "serving":
        res = serving_section(B, dev, args.serving_seconds)
        if rank == 0:
            print(json.dumps({"serving": res}), flush=True)
        return
    if args.only == "batch":
        ctx = B.srt3d_create(local)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        res = batch_section(B, ctx, dev, args.batch_steps, flush)
        B.srt3d_destroy(ctx)
        if rank == 0:
            print(json.dumps({"batch": res}), flush=True)
        return
    if args.only == "surfaces":
        ctx = B.srt3d_create(local)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        res = surfaces_section(B, ctx, dev, args.batch_steps, flush)
        B.srt3d_destroy(ctx)
        if rank == 0:
            print(json.dumps({"surfaces": res}), flush=True)
        return
    if args.only == "hist":
        # histogram path alone (for profiling): no step timing, no baseline
        ctx = B.srt3d_create(local)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        res = hist_section(B, ctx, dev, args.hist_steps, flush, args.hist_rows)
        B.srt3d_destroy(ctx)
        if rank == 0:
            print(json.dumps({"hist_sketch": res}), flush=True)
        return
    spec, prm = spec_and_params()
    m, K = WORKLOAD["m"], WORKLOAD["k_max"]

    # CPU baseline first (own single-threaded process), rank 0 at N=1 only
    cpu = oracle_block = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c = run_cpu_child(12.0, workers=host_cores())[0]
        cpu = {"value": c["value"], "unit": UNIT, "cores": c["cores"], "kind": "oracle", "sample": c["sample"],
               "value_one_core": c["value_one_core"]}
        oracle_block = c.get("block")

    fr = rank_frame(spec, rank)
    P, T = spec.num_pixels, spec.T
    N = int(fr.offsets[-1])
    stamps = torch.from_numpy(fr.stamps.view(np.int16)).to(dev)
    offsets = torch.from_numpy(fr.offsets.view(np.int32)).to(dev)
    S = torch.empty(P, m, 2, device=dev)
    n = torch.empty(P, dtype=torch.int32, device=dev)
    z = torch.empty(P, m, 2, device=dev)
    depth = torch.empty(P, K, device=dev)
    alpha = torch.empty(P, K, device=dev)
    active = torch.empty(P, K, dtype=torch.uint8, device=dev)
    alpha0 = torch.empty(P, device=dev)
    h = torch.from_numpy(synth.impulse_response(T, spec.sigma).astype(np.float32)).to(dev)
    params = B.make_params(init_mode=B.SRT3D_INIT_MATCHED, **prm)
    ctx = B.srt3d_create(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(st, sd, od, zz):
        # a frame sketched in one call: the sketch stores z = S / n itself
        # (accumulate = 2), the values srt3d_finalize would give
        B.srt3d_sketch_stream(ctx, sd, od, T, m, 2, zz, n, st)
        B.srt3d_reconstruct(ctx, zz, n, spec.rows, spec.cols, T, m, h, params, depth, alpha, active, alpha0, st)

    for _ in range(max(args.warmup, 3)):
        step(stream, stamps, offsets, z)
    B.srt3d_sync(ctx, stream)
    # active points after init (a reconstruction with no iterations), for the
    # iteration kernel's algorithmic work
    p0 = B.make_params(init_mode=B.SRT3D_INIT_MATCHED, **{**prm, "iters": 0})
    B.srt3d_reconstruct(ctx, z, n, spec.rows, spec.cols, T, m, h, p0, depth, alpha, active, alpha0, stream)
    B.srt3d_sync(ctx, stream)
    act_init = int(active.sum().item())

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    time.sleep(0.6)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    B.srt3d_profile_enable(ctx, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.mark_on()
    w0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # evict L2 between steps (outside the step events)
        ev[i][0].record(stream)
        step(stream, stamps, offsets, z)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - w0
    clocks.mark_off()
    st = B.srt3d_sync(ctx, stream, check=False)
    if st != B.SRT3D_OK:
        raise RuntimeError(f"device error during the timed region: {st}")
    per_step = np.array([a.elapsed_time(b) for a, b in ev])
    prof = B.profile_totals(ctx)
    B.srt3d_profile_enable(ctx, False)
    clocks.stop()
    total_ms = max_over_ranks(float(per_step.sum()), world, dev)

    # quality of the last step's result against the synthetic truth
    d = depth.cpu().numpy()
    act = active.cpu().numpy().astype(bool)
    act_final = int(act.sum())
    act_pts = 0.5 * (act_init + act_final)
    err = np.abs(d[:, 0] - fr.truth.depth[:, 0])
    det = act[:, 0] & (err <= 3 * spec.sigma)
    dae = float(err[det].mean())
    # the same measure on the oracle's block: "at fixed depth error" holds when
    # the GPU's DAE on those pixels is within 5 % of the FP64 oracle's
    fixed_error = None
    if oracle_block and oracle_block.get("dae_bins"):
        a, b = oracle_block["first_pixel"], oracle_block["last_pixel"]
        dg = float(err[a:b][det[a:b]].mean())
        fixed_error = {"pixels": [a, b], "gpu_dae_bins": dg, "oracle_dae_bins": oracle_block["dae_bins"],
                       "gpu_detections": float(det[a:b].mean()), "oracle_detections": oracle_block["detections"],
                       "within_5pct": dg <= 1.05 * oracle_block["dae_bins"],
                       "note": "oracle run on the block alone (its rows at the block edge lack the neighbours "
                               "the frame gives the GPU)"}

    # end to end through the public host-buffer API: srt3d_submit (pinned
    # stamps and offsets, copied to the device inside) + srt3d_poll (results
    # copied back to host memory)
    host_stamps = torch.from_numpy(fr.stamps.view(np.int16)).pin_memory().numpy().view(np.uint16)
    host_offsets = torch.from_numpy(fr.offsets.view(np.int32)).pin_memory().numpy().view(np.uint32)
    h_host = synth.impulse_response(T, spec.sigma).astype(np.float32)
    outs = (np.zeros((P, K), np.float32), np.zeros((P, K), np.float32), np.zeros((P, K), np.uint8),
            np.zeros(P, np.float32), None)
    # latency: one frame at a time (submit, then poll)
    lat = []
    for i in range(4):
        t0 = time.perf_counter()
        B.srt3d_submit(ctx, 1 + i, spec.rows, spec.cols, T, m, h_host, params, host_stamps, host_offsets, 1)
        B.srt3d_poll(ctx, 1 + i, 60_000_000, *outs)
        if i >= 1:
            lat.append((time.perf_counter() - t0) * 1e3)
    e2e_latency_ms = float(np.median(lat))
    # throughput: a window of E2E_DEPTH frames in flight, as a streaming client
    # runs it; every frame uploads its stamps and offsets from pinned host
    # memory and reads its results back inside the timed region (the pinned
    # arrays are kept until each poll, so submit does not wait for the upload)
    fid0, nfr, done = 100, args.e2e_steps, 0
    t0 = time.perf_counter()
    for i in range(nfr):
        while True:
            try:
                B.srt3d_submit(ctx, fid0 + i, spec.rows, spec.cols, T, m, h_host, params, host_stamps,
                               host_offsets, B.SRT3D_LAST_CHUNK | B.SRT3D_CHUNK_KEEP)
                break
            except B.SRT3DError as e:  # admission full: retire the oldest frame first
                if e.status != B.SRT3D_EBUSY or done >= i:
                    raise
                B.srt3d_poll(ctx, fid0 + done, 60_000_000, *outs)
                done += 1
        if i - done + 1 >= E2E_DEPTH:
            B.srt3d_poll(ctx, fid0 + done, 60_000_000, *outs)
            done += 1
    while done < nfr:
        B.srt3d_poll(ctx, fid0 + done, 60_000_000, *outs)
        done += 1
    e2e_ms = (time.perf_counter() - t0) * 1e3 / nfr
    h2d = fr.stamps.nbytes + fr.offsets.nbytes + h_host.nbytes
    d2h = sum(o.nbytes for o in outs if o is not None)

    hist = batch = surfaces = pixelwise = stream_tc = table1 = births = None
    if args.only in ("all", "streamtc") and rank == 0:
        stream_tc = stream_tc_section(B, ctx, dev, stamps, offsets, fr, spec, args.hist_steps, flush)
    if args.only in ("all", "hist") and rank == 0:
        hist = hist_section(B, ctx, dev, args.hist_steps, flush)
    if args.only in ("all", "pixelwise") and rank == 0:
        pixelwise = pixelwise_section(B, ctx, dev, stamps, offsets, fr, spec, params, args.batch_steps, flush)
    if args.only in ("all", "births") and rank == 0:
        try:
            births = births_section(B, ctx, dev, stamps, offsets, fr, spec, prm, args.batch_steps, flush)
        except Exception as exc:  # the main line must still print
            births = {"error": repr(exc)[:300]}
    if args.only == "all" and rank == 0:
        del stamps, offsets, S, z
        torch.cuda.empty_cache()
        batch = batch_section(B, ctx, dev, args.batch_steps, flush)
        surfaces = surfaces_section(B, ctx, dev, args.batch_steps, flush)
    B.srt3d_destroy(ctx)
    serving = None
    if args.only == "all" and rank == 0 and world == 1:
        try:
            serving = serving_section(B, dev, args.serving_seconds)
        except Exception as exc:  # the main line must still print
            serving = {"error": repr(exc)[:300]}
    if args.only in ("all", "table1") and rank == 0:
        # last, on its own context: nothing after it needs the device
        try:
            tctx = B.srt3d_create(local)
            try:
                table1 = table1_section(B, tctx, dev, 3, flush)
            finally:
                B.srt3d_destroy(tctx)
        except Exception as exc:  # the main line must still print
            table1 = {"error": repr(exc)[:300]}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    ms_per_step = total_ms / args.steps
    value = job_value(world, N, args.steps, total_ms)
    hbm_peak, peak_kind = load_peaks()
    rooflines = {}
    for name, (ms, cnt) in prof.items():
        bound, amount, unit = kernel_work(name, N, P, m, T, K, WORKLOAD["iters"], act_pts)
        avg_ms = ms / cnt
        entry = {"avg_ms": avg_ms, "launches": cnt, "share": ms / sum(v[0] for v in prof.values())}
        if bound == "alu":
            ach = amount / (avg_ms / 1e3)
            entry.update(bound="alu", achieved=ach, peak=fp32_peak_tflops(), unit="TFLOP/s",
                         frac=ach / fp32_peak_tflops())
        elif bound == "hbm":
            ach = amount / (avg_ms / 1e3)
            entry.update(bound="hbm", achieved=ach, peak=hbm_peak, unit="GB/s", frac=ach / hbm_peak)
        rooflines[name] = entry
    dominant = max(prof.items(), key=lambda kv: kv[1][0])[0]
    dom = rooflines[dominant]
    traffic = NCU_TRAFFIC.get(dominant, (None, None))[0]
    for name, entry in rooflines.items():
        if name in NCU_TRAFFIC:
            entry["traffic"], entry["traffic_source"] = NCU_TRAFFIC[name]
    roofline = {"kernel": dominant, "bound": dom.get("bound"), "achieved": dom.get("achieved"),
                "peak": dom.get("peak"), "unit": dom.get("unit"), "frac": dom.get("frac"), "traffic": traffic,
                "peak_source": "FP32 FMA peak: 152 SMs x 128 lanes x 2 flops x 2070 MHz (no measured FP32 figure)"
                if dom.get("bound") == "alu" else f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "work": "FP32 flops on active points: per iteration act_pts x (8 m + 9 K 60)"
                if dominant in ("iter_all", "iter") else None,
                "avg_ms": dom["avg_ms"],
                "traffic_unit": "DRAM bytes per launch (ncu)",
                "traffic_source": NCU_TRAFFIC.get(dominant, (None, None))[1]}
    sk = rooflines.get("sketch_stream", {})
    sk_hbm = (2 * N + 4 * (P + 1) + 8 * m * P + 4 * P) / 1e9 / (sk["avg_ms"] / 1e3) if sk else None
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generator of the Eq. 1 observation model: smooth depth map, Poisson counts, SBR, Gaussian pulse)",
        "config": workload_config(N),
        "frames_per_s": world * args.steps / (total_ms / 1e3),
        "latency_ms": {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99))},
        "sketch_photons_per_s": N / (sk["avg_ms"] / 1e3) if sk else None,
        "sketch_hbm_gbs": sk_hbm,
        "active_points": {"after_init": act_init, "after_last_iteration": act_final, "mean": act_pts,
                          "of": P * K},
        "dae_bins": dae,
        "detections": float(det.mean()),
        "fixed_depth_error": fixed_error,
        "wall_s": wall,
        "clocks": clocks.summary(),
        "e2e": {"value": world * N / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "frames_in_flight": E2E_DEPTH,
                "latency_ms": e2e_latency_ms,
                "api": "srt3d_submit (pinned host stamps/offsets) + srt3d_poll (host results), host wall clock; "
                       "value over a window of frames in flight, latency_ms one frame at a time"},
        "gpu_launches": int(sum(v[1] for v in prof.values())),
        "roofline": roofline,
        "rooflines": rooflines,
        "cpu_baseline": cpu,
        "hist_sketch": hist,
        "batch": batch,
        "surfaces": surfaces,
        "pixelwise": pixelwise,
        "births": births,
        "stream_tc": stream_tc,
        "table1_sizes": table1,
        "serving": serving,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------- reference arm

def workload_config(photons_per_frame):
    """The `config` of both arms' JSON lines (the same workload)."""
    return {"workload": WORKLOAD_NAME, **{k: WORKLOAD[k] for k in ("rows", "cols", "T", "m", "iters", "k_max")},
            "photons_per_frame": int(photons_per_frame), "frames_per_step_per_gpu": 1,
            "l2": "256 MiB buffer written between steps, outside the per-step events; stamps 131 MB"}


_REF_FRAME = None


def _ref_worker_init(frame_index):
    """Pool initialiser: each worker builds the benchmark frame from its seed
    (the same bytes the GPU arm uses) once."""
    global _REF_FRAME
    from paper_2203_00952_gb300 import synth

    spec, _ = spec_and_params()
    _REF_FRAME = (spec, synth.make_stream_frame(spec, synth.SEED_256x256, frame_index))


def _ref_band(task):
    """The whole oracle step on one band of rows of the frame: sketch, matched
    -filter init and the iterations, with two extra rows on each side (the
    APSS stencil's reach) whose results are dropped. Returns seconds and the
    band's result rows."""
    import numpy as np

    import oracle
    from oracle.reconstruct import Params
    from paper_2203_00952_gb300 import synth

    r0, r1, prm, m, n_max = task
    spec, fr = _REF_FRAME
    t0 = time.perf_counter()
    ha, hb = max(0, r0 - 2), min(spec.rows, r1 + 2)
    a, b = ha * spec.cols, hb * spec.cols
    lo, hi = int(fr.offsets[a]), int(fr.offsets[b])
    S, n = oracle.sketch_stream(fr.stamps[lo:hi], (fr.offsets[a:b + 1] - fr.offsets[a]).astype(np.uint32),
                                spec.T, m)
    z = oracle.finalize(S, n)
    hh = oracle.h_hat(synth.impulse_response(spec.T, spec.sigma), m)
    p = Params(**prm)
    st = oracle.init_matched_filter(z, n, hh, spec.T, p)[:3]
    eta = oracle.step_sizes(hh, n_max, p.k_max, spec.T)
    for _ in range(p.iters):
        st = oracle.iterate(z, n, st[0], st[1], st[2], hh, spec.T, hb - ha, spec.cols, p, *eta)[:3]
    keep = slice((r0 - ha) * spec.cols, (r1 - ha) * spec.cols)
    return time.perf_counter() - t0, st[0][keep], st[2][keep]


def reference_arm(args):
    """The FP64 oracle, as it stands, on the benchmark workload: each step is
    one whole 256x256 frame (sketch, init, 30 iterations) split into row bands
    over one single-threaded process per host core, timed by the wall clock
    around the step. Rank 0 only."""
    import multiprocessing as mp
    import statistics

    import numpy as np

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        os.environ[k] = "1"
    from paper_2203_00952_gb300 import synth

    spec, prm = spec_and_params()
    workers = host_cores()
    fr = synth.make_stream_frame(spec, synth.SEED_256x256, 0)
    N = int(fr.offsets[-1])
    n_max = float(np.diff(fr.offsets.astype(np.int64)).max())
    oprm = {k: prm[k] for k in ("iters", "k_max", "radius", "apss_h", "d_max", "depth_scale", "prune_alpha",
                                "smooth_lambda", "min_sep")}
    bounds = np.linspace(0, spec.rows, workers + 1).round().astype(int)
    tasks = [(int(bounds[i]), int(bounds[i + 1]), oprm, WORKLOAD["m"], n_max) for i in range(workers)
             if bounds[i + 1] > bounds[i]]
    secs, dae = [], None
    with mp.get_context("spawn").Pool(len(tasks), initializer=_ref_worker_init, initargs=(0,)) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.map(_ref_band, tasks, chunksize=1)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                secs.append(dt)
    t = np.concatenate([r[1] for r in res])
    act = np.concatenate([r[2] for r in res])
    err = np.abs(t[:, 0] - fr.truth.depth[:, 0])
    det = act[:, 0] & (err <= 3 * spec.sigma)
    dae = float(err[det].mean()) if det.any() else None
    value = N * len(secs) / sum(secs)
    sample = (f"FP64 numpy oracle on the whole {spec.rows}x{spec.cols} frame ({N} photons) every step: "
              f"{len(tasks)} single-threaded processes, each one band of rows (+2 rows each side, dropped) "
              f"through sketch, matched-filter init and {WORKLOAD['iters']} iterations; wall clock per step")
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded generator of the Eq. 1 observation model: smooth depth map, Poisson counts, SBR, Gaussian pulse)",
        "config": workload_config(N),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(tasks), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "dae_bins": dae,
        "detections": float(det.mean()),
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.cpu_child is not None:
        budget, count, frame, workers = args.cpu_child.split(":")
        print(json.dumps(cpu_oracle_samples(int(frame), float(budget), int(count), int(workers))), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
