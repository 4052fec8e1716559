"""Helpers shared by the GPU tests: decode through the C ABI and through the
oracle, compare bit for bit."""
import os

import numpy as np

from paper_1311_5304_gb300 import jdec, synth

POISON = 0xCD


def oracle_rgb(orc, img, threads=None, aan=False):
    threads = threads or max(1, min(32, os.cpu_count() or 1))
    return orc.backend_decode(img.width, img.height, img.h_samp, img.v_samp, img.planes, img.qtabs,
                              img.fancy, threads=threads, aan=aan)


def upload(img):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in img.planes]


def gpu_rgb(ctx, img, pitch=None, offset=0, planes=None, check=True, aan=False):
    """Decodes on the GPU into a poisoned buffer; returns (rgb HxWx3, raw
    buffer as numpy) so callers can check the untouched bytes too."""
    import torch
    planes = planes if planes is not None else upload(img)
    pitch = pitch if pitch is not None else 3 * img.width
    raw = torch.full((offset + pitch * img.height + 64,), POISON, dtype=torch.uint8, device="cuda")
    view = raw[offset:]
    keep = []
    im = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), planes, img.qtabs, view,
                         rgb_pitch=pitch, fancy=img.fancy, keep=keep, aan=aan)
    st = ctx.decode_coeffs(im, check=check)
    torch.cuda.synchronize()
    if check:
        ctx.sync()
    host = raw.cpu().numpy()
    rows = host[offset:offset + pitch * img.height].reshape(img.height, pitch)
    rgb = rows[:, :3 * img.width].reshape(img.height, img.width, 3)
    return rgb, host, st


def assert_same(got, want, what=""):
    if np.array_equal(got, want):
        return
    d = np.argwhere(got != want)
    y, x = d[0][0], d[0][1]
    raise AssertionError(f"{what}: {len(d)} mismatching values; first at y={y} x={x}: "
                         f"gpu={got[y, x].tolist()} oracle={want[y, x].tolist()}")


def assert_padding_untouched(host, img, pitch, offset):
    assert np.all(host[:offset] == POISON)
    rows = host[offset:offset + pitch * img.height].reshape(img.height, pitch)
    assert np.all(rows[:, 3 * img.width:] == POISON)
    assert np.all(host[offset + pitch * img.height:] == POISON)
