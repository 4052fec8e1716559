"""Seeded synthetic workloads for the JPEG decode back-end.

The paper's image corpora are not available, so every input here is made from
a seed: a synthetic RGB image is generated, converted to YCbCr, its chroma is
box-filtered down to the sampling's resolution, each 8x8 block is forward-DCT'd
in floating point (T.81 A.3.3 normalisation) and quantised with the T.81
Annex K example tables scaled by the usual quality rule.  The result is a set
of entropy-decoded int16 coefficient planes in natural order, which is what
the back-end takes (Sec. 4: "an array of short").

This module holds no decode arithmetic: it is the input side only, shared by
the tests and the benchmark.  Content recipes:

* ``gradient``: smooth 2-D colour gradients plus i.i.d. Gaussian noise of a
  given sigma (the 512x512 check image; the 4000x3000 sparsity sweep).
* ``texture``: smooth regions plus patches of multi-octave gradient
  ("Perlin") noise covering a chosen fraction of the area; at quality 90,
  coverage 0.85 and grain sigma 4 about 41% of the luma AC coefficients are
  nonzero (17-27% of the smoother chroma), with magnitudes falling off along
  the zig-zag order.

Every pixel is a pure function of (seed, x, y) -- the Gaussian grain comes from
a counter-based generator keyed by the pixel index -- so results do not depend
on the thread count.  The generator and the JFIF writer are C
(``synth_gen.c``, ``synth_jfif.c``) for speed.
"""
from __future__ import annotations

import ctypes as _ct
import os
from dataclasses import dataclass, field

import numpy as np

# ITU-T T.81 Annex K, Table K.1 (luminance) and Table K.2 (chrominance),
# natural (row-major) order.
ANNEX_K_LUMA = np.array([
    16, 11, 10, 16, 24, 40, 51, 61,
    12, 12, 14, 19, 26, 58, 60, 55,
    14, 13, 16, 24, 40, 57, 69, 56,
    14, 17, 22, 29, 51, 87, 80, 62,
    18, 22, 37, 56, 68, 109, 103, 77,
    24, 35, 55, 64, 81, 104, 113, 92,
    49, 64, 78, 87, 103, 121, 120, 101,
    72, 92, 95, 98, 112, 100, 103, 99], np.int64)
ANNEX_K_CHROMA = np.array([
    17, 18, 24, 47, 99, 99, 99, 99,
    18, 21, 26, 66, 99, 99, 99, 99,
    24, 26, 56, 99, 99, 99, 99, 99,
    47, 66, 99, 99, 99, 99, 99, 99] + [99] * 32, np.int64)

SAMPLINGS = {
    "444": ((1, 1, 1), (1, 1, 1)),
    "422": ((2, 1, 1), (1, 1, 1)),
    "420": ((2, 1, 1), (2, 1, 1)),
    "440": ((1, 1, 1), (2, 1, 1)),
}


def quality_table(quality: int, chroma: bool) -> np.ndarray:
    """Annex K table scaled by the quality rule s = 5000/q (q < 50) or
    200 - 2q, Q = clamp((t*s + 50) // 100, 1, 255)."""
    q = min(max(int(quality), 1), 100)
    s = 5000 // q if q < 50 else 200 - 2 * q
    t = ANNEX_K_CHROMA if chroma else ANNEX_K_LUMA
    return np.clip((t * s + 50) // 100, 1, 255).astype(np.uint16)


@dataclass
class CoefImage:
    """One image as the back-end sees it."""
    width: int
    height: int
    sampling: str
    h_samp: tuple
    v_samp: tuple
    planes: list            # 3 x (blocks_h, blocks_w, 64) int16, natural order
    qtabs: list             # 3 x (64,) uint16, natural order
    fancy: bool = True
    meta: dict = field(default_factory=dict)

    @property
    def blocks(self):
        return [(p.shape[0], p.shape[1]) for p in self.planes]

    def coef_bytes(self) -> int:
        return sum(p.nbytes for p in self.planes)

    def rgb_bytes(self) -> int:
        return 3 * self.width * self.height


def geometry(width: int, height: int, sampling: str):
    hs, vs = SAMPLINGS[sampling]
    hmax, vmax = max(hs), max(vs)
    mx = -(-width // (8 * hmax))
    my = -(-height // (8 * vmax))
    return hs, vs, mx, my


# ---- content and encoder side (C, multithreaded: synth_gen.c) ----------------

def make_image(width: int, height: int, sampling: str = "420", quality: int = 75,
               seed: int = 13115304, kind: str = "gradient", sigma: float = 8.0,
               fancy: bool = True, cover: float = 0.45, threads: int = 0) -> CoefImage:
    """Seeded synthetic image -> quantised coefficient planes (natural order)."""
    hs, vs, mx, my = geometry(width, height, sampling)
    qtabs = [quality_table(quality, False), quality_table(quality, True), quality_table(quality, True)]
    planes = [np.zeros((my * vs[c], mx * hs[c], 64), np.int16) for c in range(3)]
    lib = _enc()
    h = np.array(hs, np.int32)
    v = np.array(vs, np.int32)
    qp = np.array([q.ctypes.data for q in qtabs], np.uint64)
    pp = np.array([p.ctypes.data for p in planes], np.uint64)
    nthr = threads if threads > 0 else max(1, min(32, os.cpu_count() or 1))
    lib.synth_make_coefs(int(width), int(height), h.ctypes.data, v.ctypes.data, _ct.c_uint64(int(seed)),
                         1 if kind == "texture" else 0, float(sigma), float(cover), qp.ctypes.data,
                         pp.ctypes.data, int(nthr))
    return CoefImage(width, height, sampling, hs, vs, planes, qtabs, fancy,
                     dict(seed=seed, kind=kind, sigma=sigma, quality=quality, cover=cover))


def render_rgb(width: int, height: int, seed: int = 13115304, kind: str = "gradient", sigma: float = 8.0,
               cover: float = 0.45, y0: int = 0, y1: int | None = None) -> np.ndarray:
    """The synthetic source image (float32 RGB rows [y0, y1)) before encoding."""
    y1 = height if y1 is None else y1
    out = np.zeros((y1 - y0, width, 3), np.float32)
    _enc().synth_render_rgb(int(width), int(height), _ct.c_uint64(int(seed)), 1 if kind == "texture" else 0,
                            float(sigma), float(cover), int(y0), int(y1), out.ctypes.data)
    return out


def nonzero_ac_fraction(img: CoefImage) -> float:
    nz = tot = 0
    for p in img.planes:
        ac = p[..., 1:]
        nz += int(np.count_nonzero(ac))
        tot += ac.size
    return nz / max(tot, 1)


def random_coefs(rng, blocks_h: int, blocks_w: int, dense: bool = False, lo=-1024, hi=1023):
    """Unstructured coefficient planes (edge cases: arbitrary int16 content)."""
    if dense:
        return rng.integers(lo, hi + 1, size=(blocks_h, blocks_w, 64), dtype=np.int64).astype(np.int16)
    scale = np.exp(-np.arange(64) / 10.0) * 200.0
    z = rng.laplace(0.0, 1.0, size=(blocks_h, blocks_w, 64)) * scale
    z *= rng.random(size=z.shape) < 0.35 + 0.65 * np.exp(-np.arange(64) / 6.0)
    return np.clip(np.rint(z), -2047, 2047).astype(np.int16)


def random_image(rng, width: int, height: int, sampling: str, fancy: bool = True,
                 dense: bool = False, qmax: int = 255) -> CoefImage:
    hs, vs, mx, my = geometry(width, height, sampling)
    planes = [random_coefs(rng, my * vs[c], mx * hs[c], dense) for c in range(3)]
    qtabs = [rng.integers(1, qmax + 1, size=64).astype(np.uint16) for _ in range(3)]
    return CoefImage(width, height, sampling, hs, vs, planes, qtabs, fancy, dict(kind="random"))


# ---- JFIF byte streams (input side of the serving loop) ----------------------

import os as _os
import subprocess as _sp
import threading as _th

_SYN_DIR = _os.path.dirname(_os.path.abspath(__file__))
_SYN_LIB = _os.path.join(_SYN_DIR, "_build", "libsynth.so")
_SYN_SRC = ["synth_gen.c", "synth_jfif.c"]
_syn_lock = _th.Lock()
_syn = None


def build_encoder(force: bool = False) -> str:
    """Compiles the input-side C helpers (generator + JFIF writer) with gcc."""
    srcs = [_os.path.join(_SYN_DIR, f) for f in _SYN_SRC]
    if not force and _os.path.exists(_SYN_LIB) and all(
            _os.path.getmtime(_SYN_LIB) >= _os.path.getmtime(f) for f in srcs):
        return _SYN_LIB
    _os.makedirs(_os.path.dirname(_SYN_LIB), exist_ok=True)
    tmp = _SYN_LIB + f".tmp{_os.getpid()}"
    _sp.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm", "-lpthread"], check=True)
    _os.replace(tmp, _SYN_LIB)
    return _SYN_LIB


def _enc():
    global _syn
    with _syn_lock:
        if _syn is None:
            _syn = _ct.CDLL(build_encoder())
            P = _ct.c_void_p
            _syn.synth_jfif_encode.argtypes = [_ct.c_int, _ct.c_int, P, P, P, P, P, P, _ct.c_int, P, _ct.c_int64]
            _syn.synth_jfif_encode.restype = _ct.c_int64
            _syn.synth_jfif_encode_n.argtypes = [_ct.c_int, _ct.c_int, _ct.c_int, P, P, P, P, P, P, _ct.c_int, P,
                                                 _ct.c_int64]
            _syn.synth_jfif_encode_n.restype = _ct.c_int64
            _syn.synth_make_coefs.argtypes = [_ct.c_int, _ct.c_int, P, P, _ct.c_uint64, _ct.c_int, _ct.c_double,
                                              _ct.c_double, P, P, _ct.c_int]
            _syn.synth_make_coefs.restype = _ct.c_int
            _syn.synth_render_rgb.argtypes = [_ct.c_int, _ct.c_int, _ct.c_uint64, _ct.c_int, _ct.c_double,
                                              _ct.c_double, _ct.c_int, _ct.c_int, P]
            _syn.synth_render_rgb.restype = _ct.c_int
        return _syn


def encode_jfif(img: CoefImage, restart_interval: int = 0) -> bytes:
    """Baseline JFIF stream of ``img`` (optimal Huffman tables per image)."""
    for p in img.planes:
        if p.size and (np.abs(p[..., 1:]).max(initial=0) > 1023 or np.abs(p[..., 0]).max(initial=0) > 2047):
            raise ValueError("coefficients outside the 8-bit baseline range")
    planes = [np.ascontiguousarray(p, np.int16) for p in img.planes]
    qt = [np.ascontiguousarray(q, np.uint16) for q in img.qtabs]
    ncomp = len(planes)   # 3, or 1 for a grayscale image
    hs = np.array(list(img.h_samp)[:3] + [1] * (3 - len(img.h_samp)), np.int32)
    vs = np.array(list(img.v_samp)[:3] + [1] * (3 - len(img.v_samp)), np.int32)
    bw = np.array([p.shape[1] for p in planes] + [0] * (3 - ncomp), np.int32)
    bh = np.array([p.shape[0] for p in planes] + [0] * (3 - ncomp), np.int32)
    pp = np.array([p.ctypes.data for p in planes] + [0] * (3 - ncomp), np.uint64)
    qp = np.array([q.ctypes.data for q in qt] + [0] * (3 - ncomp), np.uint64)
    cap = max(4096, sum(p.size for p in planes) * 2)
    while True:
        out = np.empty(cap, np.uint8)
        n = _enc().synth_jfif_encode_n(img.width, img.height, ncomp, hs.ctypes.data, vs.ctypes.data,
                                       pp.ctypes.data, bw.ctypes.data, bh.ctypes.data, qp.ctypes.data,
                                       int(restart_interval), out.ctypes.data, cap)
        if n < 0:
            raise ValueError("encoder: inconsistent image description")
        if n <= cap:
            return out[:n].tobytes()
        cap = int(n)


def gray_image(img: CoefImage) -> CoefImage:
    """The luma plane of a 4:4:4 image as a single-component (grayscale) image."""
    if img.sampling != "444":
        raise ValueError("grayscale images are taken from 4:4:4 images")
    return CoefImage(img.width, img.height, "gray", (1, 1, 1), (1, 1, 1), [img.planes[0]], [img.qtabs[0]],
                     False, dict(img.meta))


# ---- batched workload: many images of mixed size and sampling ----------------

def batch_specs(n: int, seed: int, wmin=160, wmax=4096, hmin=120, hmax=3072,
                mix=(("420", 0.4), ("422", 0.3), ("444", 0.3)), qrange=(50, 95)):
    """Sizes, samplings and qualities of an n-image batch: W ~ U[wmin, wmax],
    H ~ U[hmin, hmax], sampling drawn from `mix`, quality ~ U{qrange}."""
    rng = np.random.default_rng([seed, 0xBA7C])
    names = [m[0] for m in mix]
    probs = np.array([m[1] for m in mix], np.float64)
    probs /= probs.sum()
    out = []
    for _ in range(n):
        w = int(rng.integers(wmin, wmax + 1))
        h = int(rng.integers(hmin, hmax + 1))
        s = str(rng.choice(names, p=probs))
        q = int(rng.integers(qrange[0], qrange[1] + 1))
        out.append((w, h, s, q))
    return out


def atlas(sampling: str, width: int = 4096, height: int = 3072, seed: int = 13115304, quality: int = 85) -> CoefImage:
    """A large textured image whose coefficient planes are cropped into the
    images of a batch (each crop then gets its own quantisation tables)."""
    return make_image(width, height, sampling, quality, seed=seed, kind="texture", sigma=4.0, cover=0.85)


def crop_offsets(specs, atlases, seed: int):
    """MCU-aligned crop origin (ox, oy) of every image inside its atlas."""
    rng = np.random.default_rng([seed, 0xC409])
    offs = []
    for (w, h, s, q) in specs:
        a = atlases[s]
        hs, vs, mx, my = geometry(w, h, s)
        _, _, amx, amy = geometry(a.width, a.height, s)
        offs.append((int(rng.integers(0, amx - mx + 1)), int(rng.integers(0, amy - my + 1))))
    return offs


def crop_planes(planes, sampling, w, h, off):
    """Crop of atlas coefficient planes (numpy or torch) for a w x h image."""
    hs, vs, mx, my = geometry(w, h, sampling)
    ox, oy = off
    return [planes[c][oy * vs[c]:(oy + my) * vs[c], ox * hs[c]:(ox + mx) * hs[c]] for c in range(3)]


def batch_image(specs, atlases, offs, i, fancy=True) -> CoefImage:
    """Host copy of batch image i (for the oracle)."""
    w, h, s, q = specs[i]
    planes = [np.ascontiguousarray(p) for p in crop_planes(atlases[s].planes, s, w, h, offs[i])]
    hs, vs, _, _ = geometry(w, h, s)
    qt = [quality_table(q, False), quality_table(q, True), quality_table(q, True)]
    return CoefImage(w, h, s, hs, vs, planes, qt, fancy, dict(quality=q))
