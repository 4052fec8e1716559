"""Continuous-batching decode server on one GPU.

A request is a baseline JPEG stream (or, in coefficient mode, entropy-decoded
coefficient planes).  The server

* entropy-decodes arriving requests on a pool of host threads (the library's
  native decoder; the sequential stage of Sec. 2 stays on the CPU) into
  page-locked host planes;
* admits decoded requests in arrival order while their device footprint
  (coefficient planes + RGB output) fits the HBM budget: the budget is one
  device arena, reserved when the server starts and handed out as a ring in
  admission order (requests retire in that order too), so admission allocates
  nothing; it copies the planes into the request's arena region on a copy
  stream;
* whenever fewer than ``max_inflight`` batches are on the GPU, launches one
  batched decode (``jdec_decode_batch``: one persistent launch, CUDA graph)
  over every admitted request not yet launched, on the compute stream, after
  their copies;
* retires finished batches: records each request's latency from arrival to
  the batch's completion event (RGB ready in device memory) and releases its
  budget.

With ``plain=True`` the same server decodes each admitted request with its
own ``jdec_decode_coeffs`` launch as soon as its copy is issued (no batching,
no cap on launches in flight): the per-image mode that batching is compared
with.

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
    desc: object = None                  # jdec_image template (pointers filled at launch)
    keep: list = field(default_factory=list)
    coef_bytes: int = 0
    plane_offs: tuple = ()               # byte offset of each plane in the request's region
    offset: int = -1                     # the request's region in the arena (-1: none)
    rgb: object = None                   # device RGB (H, W, 3) uint8 (kept results only)
    dev_bytes: int = 0
    copy_event: object = None
    done_time: float = 0.0
    error: str | None = None


def _align(n: int, a: int = 256) -> int:
    return (n + a - 1) // a * a


class ArenaRing:
    """Regions of one device arena handed out in FIFO order: allocations are
    released in the order they were made, so the free space is at most two
    runs (after the newest region, and before the oldest one)."""

    def __init__(self, size: int):
        self.size = int(size)
        self.live = collections.deque()   # (start, end) in allocation order
        self.used = 0

    def alloc(self, n: int) -> int:
        """Start offset of a region of n bytes (256-byte aligned), or -1."""
        n = _align(n)
        if n > self.size:
            return -1
        if not self.live:
            start = 0
        else:
            first, head = self.live[0][0], self.live[-1][1]
            if self.live[-1][0] >= first:          # not wrapped: free = [head, size) + [0, first)
                if head + n <= self.size:
                    start = head
                elif n <= first:
                    start = 0
                else:
                    return -1
            elif head + n <= first:                # wrapped: free = [head, first)
                start = head
            else:
                return -1
        self.live.append((start, start + n))
        self.used += n
        return start

    def release_oldest(self) -> None:
        a, b = self.live.popleft()
        self.used -= b - a


class Server:
    def __init__(self, ctx: jdec.Context, device: int = 0, hbm_budget_bytes: int = 8 << 30,
                 workers: int | None = None, max_inflight: int = 2, max_batch: int = 1024,
                 keep_results: bool = False, plain: bool = False):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.dev = torch.device("cuda", device)
        self.budget = int(hbm_budget_bytes)
        # the budget, reserved once: every admitted request's planes and RGB
        # live in it (no device allocation per request)
        self.arena = torch.empty(self.budget, dtype=torch.uint8, device=self.dev)
        self.arena_ptr = self.arena.data_ptr()
        self.ring = ArenaRing(self.budget)
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.keep = keep_results
        self.plain = plain
        nthr = workers or max(1, (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                                  else (os.cpu_count() or 2)) - 1)
        self.pool = cf.ThreadPoolExecutor(max_workers=nthr)
        self.workers = nthr
        self.copy_stream = torch.cuda.Stream(device=self.dev)
        self.comp_stream = torch.cuda.Stream(device=self.dev)
        self.decoding = collections.deque()      # (req, future) in arrival order
        self.ready = collections.deque()         # host-decoded, waiting for admission
        self.admitted = []                       # on device (copy issued), not launched
        self.inflight = collections.deque()      # (event, [req], keep)
        self.finished = []
        self.peak_used = 0
        self._templates = {}                     # descriptor templates (see _describe)
        # device clock reference for completion times
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_event.record(self.comp_stream)
        self.comp_stream.synchronize()
        self.t0_host = time.perf_counter()

    @property
    def used(self) -> int:
        return self.ring.used

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

    def _describe(self, req: Request) -> None:
        """Request geometry, its arena footprint and a descriptor whose
        pointers are filled in at launch.  Descriptors are copied from
        templates cached by geometry and quantisation tables (requests of one
        size class and quality share one)."""
        shapes = tuple((int(p.shape[0]), int(p.shape[1])) for p in req.host_planes)
        key = (req.width, req.height, str(req.sampling), req.fancy, shapes,
               b"".join(np.ascontiguousarray(q, np.uint16).tobytes() for q in req.qtabs))
        hit = self._templates.get(key)
        if hit is None:
            offs, off = [], 0
            for bh, bw in shapes:
                offs.append(off)
                off += bh * bw * 128
            keep = []
            tmpl = jdec.make_image_flat(req.width, req.height, req.sampling, 0, shapes, req.qtabs, 0,
                                        3 * req.width, fancy=req.fancy, keep=keep)
            coef_bytes = _align(off)
            hit = (tmpl, keep, tuple(offs), coef_bytes, _align(coef_bytes + 3 * req.width * req.height))
            if len(self._templates) >= 4096:
                self._templates.clear()
            self._templates[key] = hit
        tmpl, keep, req.plane_offs, req.coef_bytes, req.dev_bytes = hit
        req.keep = keep                    # the template's quantisation tables
        req.desc = type(tmpl).from_buffer_copy(tmpl)

    def _host_decode(self, req: Request) -> Request:
        torch = self.torch
        if req.coefs is not None:
            im = req.coefs
            req.width, req.height = im.width, im.height
            req.sampling = (im.h_samp, im.v_samp)
            req.qtabs = im.qtabs
            buf = getattr(im, "host_buf", None)
            if buf is None:
                # stage numpy planes in one page-locked buffer
                buf = torch.empty(sum(p.size for p in im.planes), dtype=torch.int16, pin_memory=True)
                for v, p in zip(self._plane_views(buf, [p.shape[:2] for p in im.planes]), im.planes):
                    v.copy_(torch.from_numpy(np.ascontiguousarray(p)))
                req.host_planes = self._plane_views(buf, [p.shape[:2] for p in im.planes])
            else:
                req.host_planes = im.planes          # views of host_buf already
            req.host_buf = buf
            self._describe(req)
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
        self._describe(req)
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
        """Device bytes of a described request: planes + RGB, 256-byte aligned."""
        return req.dev_bytes

    # ---- scheduler steps ------------------------------------------------------
    def _ready_or_reject(self, req: Request):
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
        """Admits ready requests in arrival order while the arena has room;
        one copy per request into its region, one event per call."""
        torch = self.torch
        admitted = []
        with torch.cuda.stream(self.copy_stream):
            while self.ready:
                req = self.ready[0]
                off = self.ring.alloc(req.dev_bytes)
                if off < 0:
                    break
                self.ready.popleft()
                req.offset = off
                src = req.host_buf.view(torch.uint8)
                self.arena[off:off + src.numel()].copy_(src, non_blocking=True)
                admitted.append(req)
        if admitted:
            self.peak_used = max(self.peak_used, self.ring.used)
            ev = torch.cuda.Event()
            ev.record(self.copy_stream)
            for req in admitted:
                req.copy_event = ev
            self.admitted.extend(admitted)

    def _fill(self, req: Request):
        """The request's descriptor with its arena addresses."""
        d = req.desc
        base = self.arena_ptr + req.offset
        for c, o in enumerate(req.plane_offs):
            d.coef[c] = base + o
        d.rgb = base + req.coef_bytes
        return d

    def _launch_plain(self):
        # one launch per request, in admission order, each after its own copy
        torch = self.torch
        batch, self.admitted = self.admitted, []
        last = None
        for r in batch:
            if r.copy_event is not last:
                self.comp_stream.wait_event(r.copy_event)
                last = r.copy_event
            self.ctx.decode_coeffs(self._fill(r), self.comp_stream)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.comp_stream)
            self.inflight.append((ev, [r]))

    def _launch(self):
        if not self.admitted:
            return
        if self.plain:
            self._launch_plain()
            return
        if len(self.inflight) >= self.max_inflight:
            return
        torch = self.torch
        batch, self.admitted = self.admitted[:self.max_batch], self.admitted[self.max_batch:]
        # copies run in order on one stream: the newest event covers them all
        self.comp_stream.wait_event(batch[-1].copy_event)
        self.ctx.decode_batch([self._fill(r) for r in batch], self.comp_stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.comp_stream)
        self.inflight.append((ev, batch))

    def _retire(self):
        while self.inflight and self.inflight[0][0].query():
            ev, batch = self.inflight.popleft()
            done = self.t0_host + self.t0_event.elapsed_time(ev) / 1e3
            for r in batch:
                r.done_time = done
                if self.keep:
                    # copied out on the copy stream, so that later copies into
                    # the released region are ordered after it
                    n = 3 * r.width * r.height
                    o = r.offset + r.coef_bytes
                    with self.torch.cuda.stream(self.copy_stream):
                        r.rgb = self.arena[o:o + n].view(r.height, r.width, 3).clone()
                self.ring.release_oldest()
                r.offset = -1
                r.host_planes = []
                r.host_buf = None
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
        self.comp_stream.synchronize()
        self.copy_stream.synchronize()
        self.arena = None


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
