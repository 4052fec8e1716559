"""Continuous-batching decode server on one GPU.

A request is a baseline JPEG stream (or, in coefficient mode, entropy-decoded
coefficient planes).  The server

* entropy-decodes arriving requests on a pool of host threads (the library's
  native decoder; the sequential stage of Sec. 2 stays on the CPU) into
  page-locked host planes;
* admits decoded requests in arrival order while their device footprint
  (coefficient planes + RGB output) fits the HBM budget; admission copies the
  planes to the device on a copy stream;
* whenever fewer than ``max_inflight`` batches are on the GPU, launches one
  batched decode (``jdec_decode_batch``: one persistent launch, CUDA graph)
  over every admitted request not yet launched, on the compute stream, after
  their copies;
* retires finished batches: records each request's latency from arrival to
  the batch's completion event (RGB ready in device memory) and releases its
  budget.

Host decoding of new requests overlaps GPU work on earlier ones, and requests
that arrive while others are on the GPU join the next batch as slots and
memory free up (Sec. 4.5's CPU/GPU overlap, applied across requests).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import jdec


@dataclass
class Request:
    rid: int
    arrival: float                       # host clock (time.perf_counter) seconds
    data: bytes | None = None            # JPEG stream (full mode)
    coefs: object = None                 # synth.CoefImage (coefficient mode)
    fancy: bool = True
    # filled by the server
    width: int = 0
    height: int = 0
    sampling: tuple = ()
    qtabs: list = field(default_factory=list)
    host_planes: list = field(default_factory=list)
    host_buf: object = None              # the planes' single page-locked buffer (planes are views)
    dev_buf: object = None               # its device copy
    dev_planes: list = field(default_factory=list)
    rgb: object = None                   # device RGB (H, W, 3) uint8
    dev_bytes: int = 0
    copy_event: object = None
    done_time: float = 0.0
    error: str | None = None


class Server:
    def __init__(self, ctx: jdec.Context, device: int = 0, hbm_budget_bytes: int = 8 << 30,
                 workers: int | None = None, max_inflight: int = 2, max_batch: int = 1024,
                 keep_results: bool = False):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.dev = torch.device("cuda", device)
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.keep = keep_results
        nthr = workers or max(1, (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                                  else (os.cpu_count() or 2)) - 1)
        self.pool = cf.ThreadPoolExecutor(max_workers=nthr)
        self.workers = nthr
        self.copy_stream = torch.cuda.Stream(device=self.dev)
        self.comp_stream = torch.cuda.Stream(device=self.dev)
        self.decoding = collections.deque()      # (req, future) in arrival order
        self.ready = collections.deque()         # host-decoded, waiting for admission
        self.admitted = []                       # on device (copy issued), not launched
        self.inflight = collections.deque()      # (event, [req])
        self.finished = []
        self.peak_used = 0
        # device clock reference for completion times
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_event.record(self.comp_stream)
        self.comp_stream.synchronize()
        self.t0_host = time.perf_counter()

    # ---- host side ------------------------------------------------------------
    @staticmethod
    def _plane_views(buf, shapes):
        """Consecutive views of one flat buffer with the given plane shapes."""
        views, off = [], 0
        for (bh, bw) in shapes:
            n = bh * bw * 64
            views.append(buf[off:off + n].view(bh, bw, 64))
            off += n
        return views

    def _host_decode(self, req: Request) -> Request:
        torch = self.torch
        if req.coefs is not None:
            im = req.coefs
            req.width, req.height = im.width, im.height
            req.sampling = (im.h_samp, im.v_samp)
            req.qtabs = im.qtabs
            req.host_planes = im.planes          # already page-locked (torch) or numpy
            req.host_buf = getattr(im, "host_buf", None)
            return req
        info = jdec.jpeg_parse(req.data)
        req.width, req.height = info.width, info.height
        req.sampling = (tuple(info.h_samp), tuple(info.v_samp)) if info.ncomp == 3 else "gray"
        req.qtabs = [np.array(info.qtab[c][:], np.uint16) for c in range(info.ncomp)]
        shapes = [(info.blocks_h[c], info.blocks_w[c]) for c in range(info.ncomp)]
        req.host_buf = torch.empty(sum(h * w * 64 for h, w in shapes), dtype=torch.int16, pin_memory=True)
        planes = self._plane_views(req.host_buf, shapes)
        jdec.entropy_decode(req.data, planes)
        req.host_planes = planes
        return req

    def submit(self, req: Request) -> None:
        if req.coefs is not None and not self.decoding:
            # nothing to decode on the host: ready at once, in arrival order
            self._host_decode(req)
            self._ready_or_reject(req)
            return
        self.decoding.append((req, self.pool.submit(self._host_decode, req)))

    @staticmethod
    def footprint(req: Request) -> int:
        return sum(p.shape[0] * p.shape[1] * 128 for p in req.host_planes) + 3 * req.width * req.height

    # ---- scheduler steps ------------------------------------------------------
    def _ready_or_reject(self, req: Request):
        req.dev_bytes = self.footprint(req)
        if req.dev_bytes > self.budget:
            req.error = "request larger than the HBM budget"
            self.finished.append(req)
        else:
            self.ready.append(req)

    def _collect_decoded(self):
        while self.decoding and self.decoding[0][1].done():
            req, fut = self.decoding.popleft()
            try:
                fut.result()
                self._ready_or_reject(req)
            except Exception as e:   # a malformed stream fails only its own request
                req.error = str(e)
                self.finished.append(req)

    def _admit(self):
        torch = self.torch
        with torch.cuda.stream(self.copy_stream):
            while self.ready and self.used + self.ready[0].dev_bytes <= self.budget:
                req = self.ready.popleft()
                self.used += req.dev_bytes
                self.peak_used = max(self.peak_used, self.used)
                if req.host_buf is not None:
                    # one copy for all planes (descriptors point into it)
                    req.dev_buf = req.host_buf.to(self.dev, non_blocking=True)
                else:
                    req.dev_planes = [p.to(self.dev, non_blocking=True) if isinstance(p, torch.Tensor)
                                      else torch.from_numpy(np.ascontiguousarray(p)).to(self.dev, non_blocking=True)
                                      for p in req.host_planes]
                req.rgb = torch.empty((req.height, req.width, 3), dtype=torch.uint8, device=self.dev)
                req.copy_event = torch.cuda.Event()
                req.copy_event.record(self.copy_stream)
                self.admitted.append(req)

    def _launch(self):
        if not self.admitted or len(self.inflight) >= self.max_inflight:
            return
        torch = self.torch
        batch, self.admitted = self.admitted[:self.max_batch], self.admitted[self.max_batch:]
        keep = []
        descs = [jdec.make_image_flat(r.width, r.height, r.sampling, r.dev_buf.data_ptr(),
                                      [p.shape[:2] for p in r.host_planes], r.qtabs, r.rgb.data_ptr(),
                                      3 * r.width, fancy=r.fancy, keep=keep) if r.dev_buf is not None else
                 jdec.make_image(r.width, r.height, r.sampling, r.dev_planes, r.qtabs, r.rgb, fancy=r.fancy,
                                 keep=keep) for r in batch]
        for r in batch:
            self.comp_stream.wait_event(r.copy_event)
            if r.dev_buf is not None:
                r.dev_buf.record_stream(self.comp_stream)
            else:
                for p in r.dev_planes:
                    p.record_stream(self.comp_stream)
            r.rgb.record_stream(self.comp_stream)
        self.ctx.decode_batch(descs, self.comp_stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.comp_stream)
        self.inflight.append((ev, batch, keep))

    def _retire(self):
        while self.inflight and self.inflight[0][0].query():
            ev, batch, _ = self.inflight.popleft()
            done = self.t0_host + self.t0_event.elapsed_time(ev) / 1e3
            for r in batch:
                r.done_time = done
                self.used -= r.dev_bytes
                r.dev_planes = []
                r.dev_buf = None
                r.host_planes = []
                r.host_buf = None
                if not self.keep:
                    r.rgb = None
                self.finished.append(r)

    def step(self):
        self._collect_decoded()
        self._retire()
        self._admit()
        self._launch()

    def idle(self) -> bool:
        return not (self.decoding or self.ready or self.admitted or self.inflight)

    def drain(self, timeout: float = 60.0) -> bool:
        t = time.perf_counter()
        while not self.idle():
            self.step()
            if time.perf_counter() - t > timeout:
                return False
            time.sleep(0.0002)
        return True

    def close(self):
        self.pool.shutdown(wait=True)
        self.ctx.sync(self.comp_stream, check=False)


# ---- load generation -------------------------------------------------------------

SERVE_MIX = ((160, 160, 0.70), (1920, 1080, 0.25), (4000, 3000, 0.05))


def request_pool(seed: int, per_class=(16, 8, 4), mode: str = "full", mix=SERVE_MIX):
    """Distinct synthetic requests per size class (all 4:2:0, quality ~ U{80..92}).
    Full mode: JPEG streams; coefficient mode: CoefImages with page-locked planes."""
    from . import synth
    import torch
    rng = np.random.default_rng([seed, 0x5E7E])
    pool = []
    for (w, h, _), k in zip(mix, per_class):
        items = []
        for i in range(k):
            q = int(rng.integers(80, 93))
            img = synth.make_image(w, h, "420", q, seed=seed + 7919 * len(pool) + i, kind="texture", sigma=3.0,
                                   cover=0.7, fancy=True)
            if mode == "full":
                items.append(synth.encode_jfif(img))
            else:
                # page-locked planes in one buffer (one copy per request)
                buf = torch.empty(sum(p.size for p in img.planes), dtype=torch.int16).pin_memory()
                views = Server._plane_views(buf, [p.shape[:2] for p in img.planes])
                for v, p in zip(views, img.planes):
                    v.copy_(torch.from_numpy(p))
                img.planes = views
                img.host_buf = buf
                items.append(img)
        pool.append(items)
    return pool


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, int(rate)])
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_load(server: Server, pool, rate: float, n: int, seed: int, mode: str = "full", timeout: float = 60.0,
             mix=SERVE_MIX):
    """Offers n requests with Poisson arrivals at `rate` req/s; returns stats."""
    rng = np.random.default_rng([seed, 0xA11])
    probs = np.array([m[2] for m in mix])
    cls = rng.choice(len(mix), size=n, p=probs / probs.sum())
    pick = [int(rng.integers(0, len(pool[c]))) for c in cls]
    times = poisson_arrivals(rate, n, seed)
    server.finished = []
    t_start = time.perf_counter()
    i = 0
    while i < n:
        now = time.perf_counter() - t_start
        while i < n and times[i] <= now:
            item = pool[cls[i]][pick[i]]
            arrival = t_start + times[i]
            req = Request(i, arrival, data=item if mode == "full" else None, coefs=item if mode != "full" else None)
            server.submit(req)
            i += 1
        server.step()
        if time.perf_counter() - t_start > timeout:
            break
    ok = server.drain(timeout)
    done = [r for r in server.finished if r.error is None]
    lat = np.array([r.done_time - r.arrival for r in done]) * 1e3
    px = sum(r.width * r.height for r in done)
    span = (max(r.done_time for r in done) - t_start) if done else 1.0
    offered_px = sum(mix[c][0] * mix[c][1] for c in cls)
    return {"rate_req_s": rate, "requests": n, "completed": len(done), "errors": sum(r.error is not None for r in server.finished),
            "drained": ok, "offered_mpix_s": round(offered_px / times[-1] / 1e6, 1),
            "mpix_s": round(px / span / 1e6, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3) if len(lat) else None,
            "p99_ms": round(float(np.percentile(lat, 99)), 3) if len(lat) else None,
            "peak_hbm_gb": round(server.peak_used / 1e9, 3)}
