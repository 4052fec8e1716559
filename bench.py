#!/usr/bin/env python3
"""Benchmark of the GB300 JPEG decode back-end (one JSON line on stdout).

Workload (one "step"): the three 8192 x 8192 synthetic images of the
full-size configuration -- 4:4:4, 4:2:2 (H2V1) and 4:2:0 (H2V2), quality 90,
textured content, triangular upsampling -- each decoded by one launch of the
fused kernel through the C ABI (dequant + IDCT + upsample + YCbCr->RGB).
Inputs are int16 coefficient planes already resident in HBM; 1.48 GB move per
step, far larger than L2, so no flush is needed between steps.

  value       MPix/s over the timed steps (device-timed, CUDA events), summed
              over ranks (each rank decodes its own replica: weak scaling)
  e2e         the same metric through jdec_decode_host_batch: pinned host planes in,
              pinned host RGB out, copies inside the timed region
  roofline    algorithmic bytes (128 B per coefficient block + 3 B per pixel)
              per launch / mean launch time, against the measured HBM peak
  cpu_baseline  the CPU oracle on the host cores, on a bounded sample

``--impl reference`` times the CPU oracle (the reference arm of this
comparison) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPix/s for dequant+IDCT+upsample+YCC→RGB, % HBM peak, batched vs plain, p99 ms"
SIDE = 8192
QUALITY = 90
VARIANTS = ["444", "422", "420"]
L2_BYTES = 129 * 1024 * 1024   # GB300 L2 capacity
SEED = 13115304 + 2000
WORKLOAD = "8192x8192 q90 texture, 4:4:4 + 4:2:2 + 4:2:0, triangular upsampling (3 images per step)"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device=None) -> float:
    """The slowest rank's time (all ranks call this together)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(px_per_rank_step: float, steps: int, ws: int, ms: float) -> float:
    """Pixels decoded by all ranks over the slowest rank's time (replicas:
    every rank decodes its own copy of the step's images)."""
    return px_per_rank_step * steps * ws / (ms / 1e3) / 1e6


def make_workload(size=(SIDE, SIDE), variants=VARIANTS):
    from paper_1311_5304_gb300 import synth
    return [synth.make_image(size[0], size[1], s, QUALITY, seed=SEED, kind="texture", sigma=4.0, cover=0.85,
                             fancy=True) for s in variants]


def alg_bytes(img) -> int:
    return img.coef_bytes() + img.rgb_bytes()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# Sources that decide the single-image launches' DRAM traffic: the device code
# and the host code that plans those launches (strip widths, grids).
TRAFFIC_SOURCES = ("jdec_api.cu", "jdec_common.h", "jdec_device.cuh", "jdec_kernels.cu", "jdec_kernels.cuh", "jdec_launch.h",
                   "jdec_work.cuh")


def _code_only(text: str) -> str:
    """Source text without comments and with whitespace collapsed (comment
    edits do not change the kernels)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1311_5304_gb300", "csrc")
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes (read + write) of one step's three launches from the
    committed ncu summary, if it was taken on the current kernel sources
    (else None)."""
    path = os.path.join(ROOT, "profiles", "fused_kernel_8192_ncu.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"dram_bytes_per_step:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_tr or m_sha.group(1) != kernel_source_sha():
        return None
    return float(m_tr.group(1))


def profiled_inst_per_px():
    """Warp instructions per pixel of each variant (4:4:4, 4:2:2, 4:2:0) from
    the committed ncu summary, if it was taken on the current kernel sources
    (else None): the ops-per-pixel figure beside the bytes."""
    path = os.path.join(ROOT, "profiles", "fused_kernel_8192_ncu.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    m_row = re.search(r"\|\s*warp instructions per pixel\s*\|\s*([0-9.]+)\s*\|\s*([0-9.]+)\s*\|\s*([0-9.]+)\s*\|", txt)
    if not m_sha or not m_row or m_sha.group(1) != kernel_source_sha():
        return None
    return dict(zip(("444", "422", "420"), (float(m_row.group(i)) for i in (1, 2, 3))))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def variant_stats(variants, imgs, bytes_v, per_var_ms, launch_ms, peak, inst_px=None):
    """Per-variant line of the roofline object: bytes, mean / p50 / p99 launch
    time, GB/s and fraction of the peak, GPix/s, the workload's nonzero-AC
    fraction and (when known for these sources) warp instructions per pixel."""
    from paper_1311_5304_gb300 import synth
    out = {}
    for i, v in enumerate(variants):
        ms = per_var_ms[i]
        srt = sorted(launch_ms[i])
        out[v] = {"bytes": bytes_v[i], "ms": round(ms, 4),
                  "ms_p50": round(srt[len(srt) // 2], 4),
                  "ms_p99": round(srt[min(len(srt) - 1, (99 * len(srt)) // 100)], 4),
                  "gbs": round(bytes_v[i] / (ms / 1e3) / 1e9, 1),
                  "frac": round(bytes_v[i] / (ms / 1e3) / 1e9 / peak, 4),
                  "gpix_s": round(imgs[i].width * imgs[i].height / (ms / 1e3) / 1e9, 1),
                  "nonzero_ac": round(synth.nonzero_ac_fraction(imgs[i]), 4),
                  "warp_inst_per_px": (inst_px or {}).get(v)}
    return out


def run_ours(args, ws, rank, local):
    import torch
    from paper_1311_5304_gb300 import jdec

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    t_gen = time.time()
    imgs = make_workload(args.size, args.variants)
    log(f"[bench] workload generated in {time.time() - t_gen:.1f}s")
    planes = [[torch.from_numpy(np.ascontiguousarray(p)).to(dev) for p in im.planes] for im in imgs]
    rgbs = [torch.empty((im.height, im.width, 3), dtype=torch.uint8, device=dev) for im in imgs]
    ctx = jdec.Context(device=local)
    keep = []
    descs = [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), planes[i], im.qtabs, rgbs[i],
                             fancy=True, keep=keep) for i, im in enumerate(imgs)]
    stream = torch.cuda.current_stream(dev)
    px_step = sum(im.width * im.height for im in imgs)
    bytes_v = [alg_bytes(im) for im in imgs]

    def step(evs=None):
        for i, d in enumerate(descs):
            if evs is not None:
                evs[i][0].record(stream)
            ctx.decode_coeffs(d, stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    ctx.sync(stream)

    K = args.steps
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in descs]
           for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    for k in range(K):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ctx.sync(stream)
    elapsed_ms = t_start.elapsed_time(t_end)
    launch_ms = [sorted(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(K)) for i in range(len(descs))]
    per_var_ms = [statistics.mean(v) for v in launch_ms]
    elapsed_ms = max_over_ranks(elapsed_ms, ws, dev)
    value = whole_job_mpix_s(px_step, K, ws, elapsed_ms)

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        host_planes = [[torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in im.planes] for im in imgs]
        host_rgb = [torch.empty((im.height, im.width, 3), dtype=torch.uint8).pin_memory() for im in imgs]
        hdescs = [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp),
                                  [hp.numpy() for hp in host_planes[i]], im.qtabs, host_rgb[i].numpy(),
                                  fancy=True, keep=keep, host=True) for i, im in enumerate(imgs)]
        ctx.decode_host_batch(hdescs, stream)
        ctx.sync(stream)
        Ke = max(1, min(args.e2e_steps, K))
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(Ke):
            ctx.decode_host_batch(hdescs, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        e_ms = max_over_ranks(a.elapsed_time(b), ws, dev)
        ctx.sync(stream)
        e2e = {"value": round(whole_job_mpix_s(px_step, Ke, ws, e_ms), 1), "unit": "MPix/s",
               "h2d_bytes_per_step": int(sum(im.coef_bytes() for im in imgs)),
               "d2h_bytes_per_step": int(sum(im.rgb_bytes() for im in imgs)),
               "steps": Ke, "ms_per_step": round(e_ms / Ke, 3),
               "api": "jdec_decode_host_batch (the step's images from pinned host buffers; banded "
                      "H2D/decode/D2H overlapping across images)"}

    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    tot_bytes = sum(bytes_v)
    tot_ms = sum(per_var_ms)
    achieved = tot_bytes / (tot_ms / 1e3) / 1e9
    default_workload = args.size == (SIDE, SIDE) and args.variants == VARIANTS
    # the committed counters were taken on the default workload only
    traffic = profiled_traffic() if default_workload else None
    inst_px = profiled_inst_per_px()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                "kernel": "jdec_fused_kernel (3 variants per step)",
                "algorithmic_bytes_per_step": tot_bytes,
                "by_variant": variant_stats(args.variants, imgs, bytes_v, per_var_ms, launch_ms, peak,
                                            inst_px if default_workload else None)}

    workload = WORKLOAD if default_workload else \
        f"{args.size[0]}x{args.size[1]} q90 texture, {'+'.join(args.variants)}, triangular upsampling"
    out = {"metric": METRIC, "value": round(value, 1), "unit": "MPix/s", "n_gpus": ws, "steps": K,
           "warmup": args.warmup, "ms_per_step": round(elapsed_ms / K, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded)",
           "config": {"workload": workload, "images_per_step": len(imgs), "mpix_per_step": px_step / 1e6,
                      "seed": SEED, "kernel_source_sha": kernel_source_sha(),
                      "sms": torch.cuda.get_device_properties(dev).multi_processor_count, "l2": (f"inputs larger than L2 ({tot_bytes / 1e9:.2f} GB moved per step)" if tot_bytes > L2_BYTES
                                 else f"inputs fit in L2 ({tot_bytes / 1e9:.3f} GB per step): not a roofline measurement"),
                      "parallelism": f"replicas x{ws}"},
           "e2e": e2e, "roofline": roofline, "clocks": clocks, "gpu_launches": len(descs) * K}

    if not args.no_batch:
        out["batch"] = bench_batched(ctx, dev, stream, args.batch_steps, 2, args.batch_images)
    if not args.no_serve:
        out["serving"] = bench_serving(ctx, dev, [2000, 5000, 10000, 20000, 50000], args.serve_requests, 8.0)
    if not args.no_jpeg:
        out["jpeg"] = bench_jpeg(ctx, dev, stream)
    if not args.no_sparsity:
        out["sparsity"] = bench_sparsity(ctx, dev, stream)
        for r in out["sparsity"]["by_quality"]:
            r["frac"] = round(r["gbs"] / float(measured_peaks()[0]["hbm_gbs"]), 4)
    if not args.no_aan:
        out["idct_aan"] = bench_aan(ctx, stream, imgs, planes, rgbs, args.variants, per_var_ms,
                                    min(K, args.aan_steps), keep)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(imgs, args.cpu_seconds)
        out["partition_sps"] = sps_estimate(out, imgs)
    if ws > 1:
        torch.distributed.destroy_process_group()
    ctx.close()
    return out


CONFIG3 = [(30, 2), (50, 4), (75, 8), (90, 16), (98, 32)]   # (quality, grain sigma)


def bench_sparsity(ctx, dev, stream, reps=20):
    """4000x3000 4:2:0 images across the quality / detail sweep (triangular
    upsampling).  One image is 72 MB of traffic, below L2's 129 MB, so each
    quality is timed over rotating copies in separate buffers totalling at
    least 4 x L2."""
    import torch
    from paper_1311_5304_gb300 import jdec, synth
    out = []
    for q, sigma in CONFIG3:
        img = synth.make_image(4000, 3000, "420", q, seed=13115304 + 3000 + q, kind="gradient", sigma=sigma,
                               fancy=True)
        nbytes = alg_bytes(img)
        nsets = -(-4 * L2_BYTES // nbytes)
        keep = []
        descs = []
        for _ in range(nsets):
            pl = [torch.from_numpy(np.ascontiguousarray(p)).to(dev) for p in img.planes]
            rgb = torch.empty((img.height, img.width, 3), dtype=torch.uint8, device=dev)
            descs.append(jdec.make_image(img.width, img.height, "420", pl, img.qtabs, rgb, fancy=True, keep=keep))
        for d in descs:
            ctx.decode_coeffs(d, stream)
        ctx.sync(stream)
        evs = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(reps * nsets)]
        torch.cuda.synchronize(dev)
        for r in range(reps):
            for i, d in enumerate(descs):
                e = evs[r * nsets + i]
                e[0].record(stream)
                ctx.decode_coeffs(d, stream)
                e[1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.sync(stream)
        t = sorted(a.elapsed_time(b) for a, b in evs)
        ms = statistics.mean(t)
        bits = 8.0 * len(synth.encode_jfif(img)) / (img.width * img.height)
        out.append({"quality": q, "sigma": sigma, "nonzero_ac": round(synth.nonzero_ac_fraction(img), 4),
                    "bits_per_px": round(bits, 3), "us": round(ms * 1e3, 2), "us_p99": round(t[(99 * len(t)) // 100] * 1e3, 2),
                    "gpix_s": round(img.width * img.height / (ms / 1e3) / 1e9, 1),
                    "gbs": round(nbytes / (ms / 1e3) / 1e9, 1)})
        del descs, keep
    return {"workload": "4000x3000 4:2:0, gradient + grain, q30..98, triangular upsampling",
            "l2": "rotating copies in separate buffers, >= 4 x L2 per quality", "launches_per_quality": "reps x copies",
            "by_quality": out}


def bench_aan(ctx, stream, imgs, planes, rgbs, variants, llm_ms, steps, keep):
    """The same step with the AAN scaled IDCT (JDEC_IDCT_AAN): per-variant
    CUDA-event launch times beside the default LLM form's."""
    import torch
    from paper_1311_5304_gb300 import jdec
    descs = [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), planes[i], im.qtabs, rgbs[i],
                             fancy=True, keep=keep, aan=True) for i, im in enumerate(imgs)]
    for _ in range(5):
        for d in descs:
            ctx.decode_coeffs(d, stream)
    ctx.sync(stream)
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in descs]
           for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        for i, d in enumerate(descs):
            evs[k][i][0].record(stream)
            ctx.decode_coeffs(d, stream)
            evs[k][i][1].record(stream)
    torch.cuda.synchronize()
    ctx.sync(stream)
    ms = [statistics.mean(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(steps)) for i in range(len(descs))]
    px = sum(im.width * im.height for im in imgs)
    return {"flag": "JDEC_IDCT_AAN", "steps": steps, "mpix_s": round(px / (sum(ms) / 1e3) / 1e6, 1),
            "vs_llm": round(sum(llm_ms) / sum(ms), 4),
            "by_variant": {v: {"ms": round(ms[i], 4), "llm_ms": round(llm_ms[i], 4),
                               "gpix_s": round(imgs[i].width * imgs[i].height / (ms[i] / 1e3) / 1e9, 1)}
                           for i, v in enumerate(variants)}}


def sps_estimate(out, imgs, dispatch_s=20e-6):
    """Sec. 5's simple partitioning scheme applied to this step as a planning
    calculation: the rows the host cores (at the oracle's measured rate)
    would take so that they finish with the GPU (at the device-resident and
    at the end-to-end rate), the Newton root of the balance equation.  Not
    executed: the library has no CPU back-end."""
    from paper_1311_5304_gb300 import partition
    w = imgs[0].width
    h = sum(im.height for im in imgs)           # the step's images stacked
    cpu_px_s = out["cpu_baseline"]["value"] * 1e6
    res = {"cpu_px_s": cpu_px_s, "dispatch_s": dispatch_s, "mcu_rows": 16, "executed": False}
    for name, rate in (("device_resident", out["value"]), ("end_to_end", (out.get("e2e") or {}).get("value"))):
        if not rate:
            continue
        gpu_px_s = rate * 1e6
        p_cpu = lambda x: x * w / cpu_px_s      # noqa: E731
        p_gpu = lambda y: y * w / gpu_px_s      # noqa: E731
        t_disp = lambda y: dispatch_s           # noqa: E731
        x = partition.sps_split(h, 16, p_cpu, p_gpu, t_disp)
        t0 = partition.balanced_time(h, 0, p_cpu, p_gpu, t_disp)
        t1 = partition.balanced_time(h, x, p_cpu, p_gpu, t_disp)
        res[name] = {"cpu_rows": x, "rows": h, "cpu_share": round(x / h, 5),
                     "predicted_speedup": round(t0 / t1, 4)}
    return res


def bench_batched(ctx, dev, stream, steps, warmup, nimages=1024):
    """Config-4 workload: 1024 images (W ~ U[160, 4096], H ~ U[120, 3072],
    40/30/30 % 4:2:0 / 4:2:2 / 4:4:4, quality ~ U{50..95}) decoded by one
    batched call (one persistent launch per variant class, replayed from a
    CUDA graph) versus one plain call per image, both device-timed with CUDA
    events."""
    import torch
    from paper_1311_5304_gb300 import jdec, synth
    seed = 13115304 + 4000
    specs = synth.batch_specs(nimages, seed)
    atl = {sm: synth.atlas(sm, seed=seed + k) for k, sm in enumerate(("420", "422", "444"))}
    offs = synth.crop_offsets(specs, atl, seed)
    dev_atl = {sm: [torch.from_numpy(pl).to(dev) for pl in a.planes] for sm, a in atl.items()}
    keep, descs, px, nbytes = [], [], 0, 0
    for i, (w, h, sm, q) in enumerate(specs):
        pl = [t.contiguous() for t in synth.crop_planes(dev_atl[sm], sm, w, h, offs[i])]
        rgb = torch.empty((h, w, 3), dtype=torch.uint8, device=dev)
        qt = [synth.quality_table(q, False), synth.quality_table(q, True), synth.quality_table(q, True)]
        descs.append(jdec.make_image(w, h, sm, pl, qt, rgb, keep=keep))
        px += w * h
        nbytes += sum(t.numel() * 2 for t in pl) + 3 * w * h
    del dev_atl

    def timed(fn, k):
        for _ in range(warmup):
            fn()
        ctx.sync(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ctx.sync(stream)
        return a.elapsed_time(b) / k

    def plain():
        for d in descs:
            ctx.decode_coeffs(d, stream)

    t_batch = timed(lambda: ctx.decode_batch(descs, stream), steps)
    t_plain = timed(plain, max(1, steps // 2))
    # autotuned: a context with the batch tuner on; its first call (in the
    # untimed warm-up) times the candidate shapes per class and keeps the
    # fastest, later calls replay the tuned graph
    tune_path = os.path.join(tempfile.mkdtemp(), "batch_tune.json")
    with jdec.Context(device=dev.index or 0, autotune=True, tune_file=tune_path) as tctx:
        t0 = time.perf_counter()
        tctx.decode_batch(descs, stream)
        tctx.sync(stream)
        tune_s = time.perf_counter() - t0
        for _ in range(warmup):
            tctx.decode_batch(descs, stream)
        tctx.sync(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            tctx.decode_batch(descs, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        tctx.sync(stream)
        t_tuned = a.elapsed_time(b) / steps
    with open(tune_path) as f:
        picks = [e for e in json.load(f)["entries"] if len(e) >= 5 and e[4] == 1]
    peak = float(measured_peaks()[0]["hbm_gbs"])
    return {"workload": f"{nimages} images, W~U[160,4096], H~U[120,3072], 40/30/30% 4:2:0/4:2:2/4:4:4, q~U{{50..95}}",
            "mpix": round(px / 1e6, 1), "gbytes": round(nbytes / 1e9, 2),
            "batched": {"ms": round(t_batch, 3), "mpix_s": round(px / t_batch / 1e3, 1),
                        "gbs": round(nbytes / t_batch / 1e6, 1), "frac": round(nbytes / t_batch / 1e6 / peak, 4),
                        # one launch per variant class present (all tables here fit 8 bits)
                        "launches": len({sm for (_, _, sm, _) in specs}),
                        "api": "jdec_decode_batch (one persistent launch per variant class, CUDA graph replay)"},
            "autotuned": {"ms": round(t_tuned, 3), "mpix_s": round(px / t_tuned / 1e3, 1),
                          "gbs": round(nbytes / t_tuned / 1e6, 1), "frac": round(nbytes / t_tuned / 1e6 / peak, 4),
                          "tuning_s": round(tune_s, 2),
                          "picks": [{"class": e[0], "size_class": e[1], "strip_mcus": e[2], "idct_threads": e[3]}
                                    for e in picks],
                          "api": "jdec_decode_batch with jdec_options.autotune = 1 (tuned per class and size class)"},
            "plain": {"ms": round(t_plain, 3), "mpix_s": round(px / t_plain / 1e3, 1), "launches": len(descs),
                      "api": "jdec_decode_coeffs per image"},
            "speedup_batched_vs_plain": round(t_plain / t_batch, 3),
            "speedup_autotuned_vs_plain": round(t_plain / t_tuned, 3)}


def bench_jpeg(ctx, dev, stream, reps=3):
    """Whole-stream decode of one 8192x8192 4:2:0 q90 JPEG (restart marker at
    every MCU row) from host bytes to device RGB: host entropy decoding then
    one back-end launch, against jdec_decode_jpeg, which overlaps chunked
    host decoding with the back-end (1 thread) and decodes restart-aligned
    chunks on all host cores.  Wall-clock times (host decoding is the
    dominant stage)."""
    import torch
    from paper_1311_5304_gb300 import jdec, synth
    img = synth.make_image(SIDE, SIDE, "420", QUALITY, seed=SEED, kind="texture", sigma=4.0, cover=0.85, fancy=True)
    mx = img.planes[0].shape[1] // 2
    data = synth.encode_jfif(img, mx)
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    rgb = torch.empty((SIDE, SIDE, 3), dtype=torch.uint8, device=dev)
    info = jdec.jpeg_parse(data)
    hplanes = [torch.empty((info.blocks_h[c], info.blocks_w[c], 64), dtype=torch.int16).pin_memory() for c in range(3)]
    dplanes = [torch.empty_like(p, device=dev) for p in hplanes]
    keep = []
    desc = jdec.make_image(SIDE, SIDE, "420", dplanes, [np.array(info.qtab[c][:], np.uint16) for c in range(3)],
                           rgb, keep=keep)

    def serial():
        jdec.entropy_decode(data, hplanes)
        for h, d in zip(hplanes, dplanes):
            d.copy_(h, non_blocking=True)
        ctx.decode_coeffs(desc, stream)

    def timed(fn):
        fn()
        ctx.sync(stream)
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            ctx.sync(stream)
            ts.append(time.perf_counter() - t)
        return min(ts) * 1e3

    t_serial = timed(serial)
    t_huff = timed(lambda: jdec.entropy_decode(data, hplanes))
    t_pipe1 = timed(lambda: ctx.decode_jpeg(data, rgb, threads=1, stream=stream))
    t_pipen = timed(lambda: ctx.decode_jpeg(data, rgb, threads=ncores, stream=stream))
    # chunk-size profile of the 1-thread pipeline (Sec. 4.5 picks the largest
    # chunk among the fastest)
    my = info.blocks_h[0] // 2
    prof = {}
    for rows in (my, my // 4, my // 16, my // 64, 1):
        with jdec.Context(device=dev.index, jpeg_chunk_rows=rows) as c2:
            prof[rows] = timed(lambda: c2.decode_jpeg(data, rgb, threads=1, stream=stream))
    best = min(prof.values())
    pick = max(r for r, t in prof.items() if t <= 1.02 * best)
    mpix = SIDE * SIDE / 1e6
    # Sec. 5's pipelined partitioning (PPS) for this stream, as a planning
    # calculation from the measured stages: host Huffman per pixel row (one
    # thread), the device back-end, and the oracle's one-core rate for the
    # host's share of the back-end
    from paper_1311_5304_gb300 import partition
    huff_row = t_huff / 1e3 / SIDE
    gpu_row = (t_serial - t_huff) / 1e3 / SIDE
    cpu_row = SIDE / 64e6                  # ~64 MPix/s: the oracle on one host core
    pps_rows = partition.pps_split(SIDE, 16, pick * 16, lambda r: r * huff_row, lambda x: x * cpu_row,
                                   lambda y: y * gpu_row)
    return {"workload": "8192x8192 4:2:0 q90 texture JPEG, restart interval = 1 MCU row",
            "jpeg_mbytes": round(len(data) / 1e6, 1), "host_cores": ncores,
            "serial": {"ms": round(t_serial, 1), "mpix_s": round(mpix / t_serial * 1e3, 1),
                       "api": "jdec_entropy_decode (1 thread) + copy + jdec_decode_coeffs"},
            "pipelined_1_thread": {"ms": round(t_pipe1, 1), "mpix_s": round(mpix / t_pipe1 * 1e3, 1),
                                   "api": "jdec_decode_jpeg threads=1"},
            "pipelined_all_cores": {"ms": round(t_pipen, 1), "mpix_s": round(mpix / t_pipen * 1e3, 1),
                                    "api": f"jdec_decode_jpeg threads={ncores}"},
            "huffman_1_thread_ms": round(t_huff, 1),
            "amdahl_max_speedup_1_thread": round(t_serial / t_huff, 4),
            "chunk_profile_1_thread": {"ms_by_chunk_mcu_rows": {str(r): round(t, 1) for r, t in prof.items()},
                                       "picked_mcu_rows": pick},
            "partition_pps": {"cpu_rows": pps_rows, "rows": SIDE, "chunk_rows": pick * 16, "executed": False,
                              "note": ("host rows after the first chunk outlast the device's whole share"
                                       if huff_row * (SIDE - pick * 16) >= gpu_row * SIDE else
                                       "one MCU row of host back-end work outlasts the whole device share"
                                       if pps_rows == 0 else "the host takes rows")}}


def bench_serving(ctx, dev, rates, max_requests, budget_gb):
    """Config-5 workload: Poisson arrivals, 70% 160x160 / 25% 1920x1080 / 5%
    4000x3000, all 4:2:0 at quality ~ U{80..92}; HBM budget 8 GB.  Full mode
    entropy-decodes each JPEG on the host; coefficient mode starts from
    page-locked coefficient planes.  Latency: arrival -> RGB ready on device.
    The budget is in GiB (2^30 bytes)."""
    from paper_1311_5304_gb300 import serve
    out = {"mix": "70% 160x160, 25% 1920x1080, 5% 4000x3000; 4:2:0 q~U{80..92}", "hbm_budget_gib": budget_gb}
    for mode in ("full", "coef"):
        pool = serve.request_pool(13115304 + 5000, mode=mode)
        # batched (continuous batching, jdec_decode_batch) and plain (one
        # jdec_decode_coeffs per request as it is admitted) on the same arrivals
        for plain in (False, True):
            srv = serve.Server(ctx, device=dev.index or 0, hbm_budget_bytes=int(budget_gb * (1 << 30)), plain=plain)
            rows = []
            try:
                for rate in rates:
                    n = int(min(max_requests, max(200, rate * 0.5)))
                    rows.append(serve.run_load(srv, pool, rate, n, seed=int(rate), mode=mode, timeout=60))
            finally:
                srv.close()
            out[mode + ("_plain" if plain else "")] = rows
        out["host_threads"] = srv.workers
    out["api"] = {"batched": "serve.Server: jdec_decode_batch over the admitted requests",
                  "plain": "serve.Server(plain=True): one jdec_decode_coeffs per request"}
    return out


ARM_PARTS = {"0xd4f": "Arm Neoverse V2 (Grace)", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    v = line.split(":", 1)[1].strip()
                    return ARM_PARTS.get(v.lower(), v)
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(imgs, seconds):
    """The oracle (as it stands) on the host cores: whole 8192^2 images of the
    step, decoded until `seconds` of wall time have passed; plus one
    single-threaded band for the per-core rate."""
    import oracle
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    from paper_1311_5304_gb300 import synth
    im = imgs[-1]
    hs, vs, mx, my = synth.geometry(im.width, 256, im.sampling)
    band = [p[:my * vs[c]] for c, p in enumerate(im.planes)]
    t1 = time.time()
    oracle.backend_decode(im.width, 256, im.h_samp, im.v_samp, band, im.qtabs, True, threads=1)
    single = im.width * 256 / (time.time() - t1) / 1e6
    done_px, t0, n = 0, time.time(), 0
    while True:
        im = imgs[n % len(imgs)]
        oracle.backend_decode(im.width, im.height, im.h_samp, im.v_samp, im.planes, im.qtabs, True, threads=threads)
        done_px += im.width * im.height
        n += 1
        if time.time() - t0 >= seconds and n >= len(imgs):
            break
    dt = time.time() - t0
    return {"value": round(done_px / dt / 1e6, 2), "unit": "MPix/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} whole {imgs[0].width}x{imgs[0].height} images of the step (cycling the samplings), {dt:.1f}s wall",
            "single_thread_mpix_s": round(single, 2), "single_thread_sample": "one 8192x256 4:2:0 band",
            "cpu_model": cpu_model()}


def run_reference(args, ws, rank):
    """The CPU oracle timed as the reference arm (rank 0 only).  A step is the
    step of the GPU arm -- the three whole 8192 x 8192 images -- whenever
    warm-up plus timed steps fit about two minutes of wall time on the host
    cores; otherwise each step is one band of rows of each image, sized to fit,
    and the workload label says so."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    imgs = make_workload()
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    from paper_1311_5304_gb300 import synth

    def band_img(im, band):
        if band >= im.height:
            return im.width, im.height, im.h_samp, im.v_samp, im.planes, im.qtabs
        hs, vs, mx, my = synth.geometry(im.width, band, im.sampling)
        planes = [p[:my * vs[c]] for c, p in enumerate(im.planes)]
        return im.width, band, im.h_samp, im.v_samp, planes, im.qtabs

    def run(bands):
        for (w, h, hs, vs, planes, qt) in bands:
            oracle.backend_decode(w, h, hs, vs, planes, qt, True, threads=threads)

    whole = [band_img(im, im.height) for im in imgs]
    t0 = time.time()
    run(whole)
    t_whole = time.time() - t0
    budget_s = 120.0
    nsteps = args.steps + args.warmup
    if nsteps * t_whole <= budget_s:
        bands, band = whole, SIDE
        workload = WORKLOAD
        sample = f"{args.steps} steps of the three whole {SIDE}x{SIDE} images"
    else:
        band = int(max(16, min(SIDE, SIDE * budget_s / nsteps / max(t_whole, 1e-6))) // 16 * 16)
        bands = [band_img(im, band) for im in imgs]
        workload = (f"rows 0..{band - 1} of the three {SIDE}x{SIDE} q90 texture images (4:4:4 + 4:2:2 + 4:2:0, "
                    f"triangular upsampling) per step")
        sample = f"{args.steps} steps of 3 x {SIDE}x{band} bands"
    px = sum(b[0] * b[1] for b in bands)
    for _ in range(args.warmup):
        run(bands)
    t0 = time.time()
    for _ in range(args.steps):
        run(bands)
    dt = time.time() - t0
    value = px * args.steps / dt / 1e6
    return {"metric": METRIC, "value": round(value, 2), "unit": "MPix/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded)",
            "impl": "reference",
            "config": {"workload": workload, "images_per_step": len(imgs), "mpix_per_step": px / 1e6,
                       "rows_per_image": band},
            "cpu_baseline": {"value": round(value, 2), "unit": "MPix/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 2), "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-jpeg", action="store_true", help="skip the whole-stream JPEG decode timing")
    ap.add_argument("--no-aan", action="store_true", help="skip the AAN-IDCT timing of the step")
    ap.add_argument("--no-sparsity", action="store_true", help="skip the 4000x3000 quality sweep")
    ap.add_argument("--aan-steps", type=int, default=300)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--batch-steps", type=int, default=6)
    ap.add_argument("--batch-images", type=int, default=1024)
    ap.add_argument("--size", default=f"{SIDE}x{SIDE}", help="WxH of every image of the step")
    ap.add_argument("--variants", default=",".join(VARIANTS), help="samplings decoded per step")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.size = tuple(int(v) for v in args.size.lower().split("x"))
    args.variants = [v for v in args.variants.split(",") if v]
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        from paper_1311_5304_gb300 import build as jbuild
        jbuild.build()
        out = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
