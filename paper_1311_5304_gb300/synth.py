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
* ``texture``: smooth regions plus elliptical patches of multi-octave
  gradient ("Perlin") noise, giving 30-60% nonzero AC coefficients at
  quality 90 with magnitudes falling off along the zig-zag order.

Noise is drawn per band of 64 pixel rows from ``numpy.random.default_rng``
seeded with ``(seed, band)``, so results do not depend on anything but the
arguments.
"""
from __future__ import annotations

import math
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
}

BAND = 64  # pixel rows per noise band (a multiple of every MCU height)


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


# ---- content ------------------------------------------------------------------

def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


class _Gradient2D:
    """Gradient noise on a square lattice: random unit gradients at lattice
    points, quintic fade, bilinear blend of the four corner dot products."""

    def __init__(self, rng, width, height, cell):
        self.cell = float(cell)
        gw = int(math.ceil(width / cell)) + 2
        gh = int(math.ceil(height / cell)) + 2
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(gh, gw))
        self.gx = np.cos(ang).astype(np.float32)
        self.gy = np.sin(ang).astype(np.float32)

    def __call__(self, xs, ys):
        fx = xs / self.cell
        fy = ys / self.cell
        x0 = np.floor(fx).astype(np.int64)
        y0 = np.floor(fy).astype(np.int64)
        tx = (fx - x0).astype(np.float32)
        ty = (fy - y0).astype(np.float32)

        def corner(dx, dy):
            gx = self.gx[y0 + dy, x0 + dx]
            gy = self.gy[y0 + dy, x0 + dx]
            return gx * (tx - dx) + gy * (ty - dy)

        u, v = _fade(tx), _fade(ty)
        a = corner(0, 0) + u * (corner(1, 0) - corner(0, 0))
        b = corner(0, 1) + u * (corner(1, 1) - corner(0, 1))
        return a + v * (b - a)


class _Content:
    def __init__(self, width, height, seed, kind, sigma, texture_cover=0.45):
        self.w, self.h, self.kind, self.sigma, self.seed = width, height, kind, float(sigma), seed
        rng = np.random.default_rng([seed, 0x5EED])
        # smooth part: per channel a + b x + c y + d sin(...)
        self.coef = rng.uniform(-1.0, 1.0, size=(3, 6)).astype(np.float32)
        self.base = rng.uniform(70.0, 180.0, size=3).astype(np.float32)
        self.freq = rng.uniform(0.5, 3.0, size=(3, 2)).astype(np.float32)
        if kind == "texture":
            self.octaves = [_Gradient2D(rng, width, height, cell) for cell in (24, 10, 4)]
            # elliptical patches covering roughly texture_cover of the area
            npatch = max(1, int(texture_cover * width * height / (np.pi * (0.08 * max(width, height)) ** 2 * 0.6)))
            npatch = min(npatch, 400)
            self.pc = rng.uniform(0, 1, size=(npatch, 2)) * np.array([width, height])
            self.pr = rng.uniform(0.04, 0.12, size=(npatch, 2)) * max(width, height)
            self.pa = rng.uniform(18.0, 55.0, size=npatch).astype(np.float32)
            self.tint = rng.uniform(0.4, 1.0, size=(npatch, 3)).astype(np.float32)

    def rgb(self, y0, y1, band_index):
        """Float32 RGB rows [y0, y1) for x in [0, W) (true image only)."""
        w, h = self.w, self.h
        ys = np.arange(y0, y1, dtype=np.float32)[:, None]
        xs = np.arange(0, w, dtype=np.float32)[None, :]
        nx, ny = xs / max(w, 1), ys / max(h, 1)
        out = np.empty((y1 - y0, w, 3), np.float32)
        for c in range(3):
            a = self.coef[c]
            f = self.freq[c]
            out[..., c] = (self.base[c] + 50.0 * a[0] * nx + 50.0 * a[1] * ny
                           + 25.0 * a[2] * np.sin(2 * np.pi * (f[0] * nx + a[3]))
                           * np.cos(2 * np.pi * (f[1] * ny + a[4])) + 10.0 * a[5] * nx * ny)
        if self.kind == "texture":
            X = np.broadcast_to(xs, (y1 - y0, w))
            Y = np.broadcast_to(ys, (y1 - y0, w))
            tex = 0.0
            for amp, octv in zip((1.0, 0.6, 0.45), self.octaves):
                tex = tex + amp * octv(X, Y)
            # mask: union of ellipses with soft edges, strongest patch wins
            amp_map = np.zeros((y1 - y0, w), np.float32)
            tint = np.ones((y1 - y0, w, 3), np.float32)
            for (cx, cy), (rx, ry), pa, tn in zip(self.pc, self.pr, self.pa, self.tint):
                if cy + ry < y0 or cy - ry > y1:
                    continue
                d = ((X - cx) / rx) ** 2 + ((Y - cy) / ry) ** 2
                m = np.clip((1.2 - d) * 2.0, 0.0, 1.0) * pa
                sel = m > amp_map
                amp_map = np.where(sel, m, amp_map)
                tint = np.where(sel[..., None], tn, tint)
            out += (tex * amp_map)[..., None] * tint
        if self.sigma > 0:
            rng = np.random.default_rng([self.seed, 0xB0D, band_index])
            out += rng.standard_normal(out.shape, dtype=np.float32) * np.float32(self.sigma)
        return out


# ---- encoder side: colour transform, downsampling, FDCT, quantisation --------

def _rgb_to_ycc(rgb):
    r, g, b = rgb[..., 0], rgb[..., 1], rgb[..., 2]
    y = 0.299 * r + 0.587 * g + 0.114 * b
    cb = -0.168736 * r - 0.331264 * g + 0.5 * b + 128.0
    cr = 0.5 * r - 0.418688 * g - 0.081312 * b + 128.0
    return [np.clip(np.rint(p), 0, 255).astype(np.float32) for p in (y, cb, cr)]


def _dct_matrix():
    d = np.zeros((8, 8), np.float64)
    for u in range(8):
        cu = math.sqrt(0.5) if u == 0 else 1.0
        for x in range(8):
            d[u, x] = 0.5 * cu * math.cos((2 * x + 1) * u * math.pi / 16.0)
    return d


_D = _dct_matrix()


def _fdct_quant(plane, q):
    """plane: (8*bh, 8*bw) float samples; returns (bh, bw, 64) int16."""
    hh, ww = plane.shape
    bh, bw = hh // 8, ww // 8
    blk = plane.reshape(bh, 8, bw, 8).transpose(0, 2, 1, 3).astype(np.float64) - 128.0
    # blk[a, b, i, j]: i = sample row, j = sample column.  F = D blk D^T puts
    # the vertical frequency on the row and the horizontal one on the column,
    # which is the natural coefficient order.
    F = np.einsum("vi,abij,uj->abvu", _D, blk, _D, optimize=True)
    qf = q.reshape(8, 8).astype(np.float64)
    z = F / qf
    zq = np.sign(z) * np.floor(np.abs(z) + 0.5)
    return np.clip(zq, -2047, 2047).astype(np.int16).reshape(bh, bw, 64)


def make_image(width: int, height: int, sampling: str = "420", quality: int = 75,
               seed: int = 13115304, kind: str = "gradient", sigma: float = 8.0,
               fancy: bool = True, texture_cover: float = 0.45) -> CoefImage:
    """Seeded synthetic image -> quantised coefficient planes."""
    hs, vs, mx, my = geometry(width, height, sampling)
    hmax, vmax = max(hs), max(vs)
    pw, ph = mx * 8 * hmax, my * 8 * vmax
    content = _Content(width, height, seed, kind, sigma, texture_cover)
    qtabs = [quality_table(quality, False), quality_table(quality, True), quality_table(quality, True)]
    planes = [np.zeros((my * vs[c], mx * hs[c], 64), np.int16) for c in range(3)]
    for band, y0 in enumerate(range(0, ph, BAND)):
        y1 = min(y0 + BAND, ph)
        ty1 = min(y1, height)
        if y0 < height:
            rgb = content.rgb(y0, ty1, band)
        else:
            rgb = content.rgb(height - 1, height, band)
        # replicate the true image into the padding (right and bottom edges)
        rows = np.clip(np.arange(y0, y1), 0, height - 1) - (y0 if y0 < height else height - 1)
        rgb = rgb[rows]
        if pw > width:
            rgb = np.concatenate([rgb, np.repeat(rgb[:, -1:], pw - width, axis=1)], axis=1)
        comps = _rgb_to_ycc(rgb)
        for c in range(3):
            sx, sy = hmax // hs[c], vmax // vs[c]
            p = comps[c]
            if sx > 1 or sy > 1:
                p = p.reshape(p.shape[0] // sy, sy, p.shape[1] // sx, sx).mean(axis=(1, 3))
                p = np.rint(p)
            by0 = (y0 // sy) // 8
            planes[c][by0:by0 + p.shape[0] // 8] = _fdct_quant(p, qtabs[c])
    return CoefImage(width, height, sampling, hs, vs, planes, qtabs, fancy,
                     dict(seed=seed, kind=kind, sigma=sigma, quality=quality))


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

import ctypes as _ct
import os as _os
import subprocess as _sp
import threading as _th

_SYN_DIR = _os.path.dirname(_os.path.abspath(__file__))
_SYN_LIB = _os.path.join(_SYN_DIR, "_build", "libsynth_jfif.so")
_syn_lock = _th.Lock()
_syn = None


def build_encoder(force: bool = False) -> str:
    src = _os.path.join(_SYN_DIR, "synth_jfif.c")
    if not force and _os.path.exists(_SYN_LIB) and _os.path.getmtime(_SYN_LIB) >= _os.path.getmtime(src):
        return _SYN_LIB
    _os.makedirs(_os.path.dirname(_SYN_LIB), exist_ok=True)
    tmp = _SYN_LIB + f".tmp{_os.getpid()}"
    _sp.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, src], check=True)
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
        return _syn


def encode_jfif(img: CoefImage, restart_interval: int = 0) -> bytes:
    """Baseline JFIF stream of ``img`` (optimal Huffman tables per image)."""
    for p in img.planes:
        if p.size and (np.abs(p[..., 1:]).max(initial=0) > 1023 or np.abs(p[..., 0]).max(initial=0) > 2047):
            raise ValueError("coefficients outside the 8-bit baseline range")
    planes = [np.ascontiguousarray(p, np.int16) for p in img.planes]
    qt = [np.ascontiguousarray(q, np.uint16) for q in img.qtabs]
    hs = np.array(img.h_samp, np.int32)
    vs = np.array(img.v_samp, np.int32)
    bw = np.array([p.shape[1] for p in planes], np.int32)
    bh = np.array([p.shape[0] for p in planes], np.int32)
    pp = np.array([p.ctypes.data for p in planes], np.uint64)
    qp = np.array([q.ctypes.data for q in qt], np.uint64)
    cap = max(4096, sum(p.size for p in planes) * 2)
    while True:
        out = np.empty(cap, np.uint8)
        n = _enc().synth_jfif_encode(img.width, img.height, hs.ctypes.data, vs.ctypes.data,
                                     pp.ctypes.data, bw.ctypes.data, bh.ctypes.data, qp.ctypes.data,
                                     int(restart_interval), out.ctypes.data, cap)
        if n < 0:
            raise ValueError("encoder: inconsistent image description")
        if n <= cap:
            return out[:n].tobytes()
        cap = int(n)
