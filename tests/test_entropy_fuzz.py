"""Robustness of the host JPEG parser and Huffman decoder (outside the hot
path, but it reads untrusted bytes): seeded random mutations of valid
baseline streams -- byte overwrites, bit flips, deletions, insertions,
truncation -- of every sampling, with and without restart intervals, and a
grayscale stream.  Every call either succeeds or returns an error status;
the one-thread and threaded decoders agree on which, and on the planes when
both succeed.  (The same mutants were
run against an AddressSanitizer build of the decoder without findings.)"""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth


def _streams():
    out = []
    for s, ri in (("420", 0), ("420", 2), ("444", 3), ("422", 0), ("440", 1)):
        img = synth.make_image(48, 40, s, 80, seed=3, kind="texture", sigma=4)
        mx = img.planes[0].shape[1] // img.h_samp[0]
        out.append(synth.encode_jfif(img, ri * mx))
    gray = synth.gray_image(synth.make_image(40, 24, "444", 80, seed=4, kind="texture", sigma=4))
    out.append(synth.encode_jfif(gray, 5))
    return out


def _mutate(rng, d):
    d = bytearray(d)
    kind = rng.integers(0, 4)
    for _ in range(int(rng.integers(1, 6))):
        pos = int(rng.integers(0, len(d)))
        if kind == 0:
            d[pos] = int(rng.integers(0, 256))
        elif kind == 1:
            d[pos] ^= 1 << int(rng.integers(0, 8))
        elif kind == 2:
            del d[pos:pos + int(rng.integers(1, 16))]
        else:
            d[pos:pos] = bytes(rng.integers(0, 256, size=int(rng.integers(1, 8))).astype(np.uint8))
    if rng.integers(0, 8) == 0:
        d = d[:int(rng.integers(0, len(d)))]
    return bytes(d)


@pytest.mark.parametrize("seed", [1, 2])
def test_mutated_streams_fail_cleanly(seed):
    base = _streams()
    rng = np.random.default_rng(seed)
    decoded = rejected = 0
    for it in range(1200):
        data = _mutate(rng, base[it % len(base)])
        try:
            info = jdec.jpeg_parse(data)
        except jdec.JdecError as e:
            assert e.status in (jdec.EINVAL, jdec.EUNSUPPORTED)
            rejected += 1
            continue
        nc = info.ncomp
        if sum(info.blocks_w[c] * info.blocks_h[c] for c in range(nc)) > 200000:
            continue   # a mutated frame size: valid, but not worth the memory here
        outcome, results = [], []
        for threads in (1, 3):
            planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(nc)]
            try:
                jdec.entropy_decode(data, planes, threads=threads)
                outcome.append(True)
            except jdec.JdecError as e:
                assert e.status in (jdec.EINVAL, jdec.EUNSUPPORTED)
                outcome.append(False)
            results.append(planes)
        assert outcome[0] == outcome[1], it
        if outcome[0]:
            assert all(np.array_equal(a, b) for a, b in zip(*results)), it
        decoded += outcome[0]
    # the mutants exercise both outcomes
    assert decoded > 50 and rejected > 50
