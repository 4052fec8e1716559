"""The serving arena's ring allocator (host logic, no GPU): regions come out
in FIFO order, never overlap, stay within the arena, and free space is
reused after the oldest regions are released, including across the wrap."""
import numpy as np

from paper_1311_5304_gb300.serve import ArenaRing


def _overlaps(live):
    iv = sorted(live)
    return any(a[1] > b[0] for a, b in zip(iv, iv[1:]))


def test_ring_fifo_regions_never_overlap():
    rng = np.random.default_rng(5)
    ring = ArenaRing(1 << 20)
    pending = []
    wraps = 0
    for step in range(20000):
        if pending and rng.random() < 0.4:
            ring.release_oldest()
            pending.pop(0)
        n = int(rng.integers(1, 200000))
        off = ring.alloc(n)
        while off < 0 and pending:
            ring.release_oldest()       # retire the oldest until the request fits
            pending.pop(0)
            off = ring.alloc(n)
        assert off >= 0                  # an empty ring always takes a region <= its size
        assert off % 256 == 0 and off + n <= ring.size
        wraps += bool(pending) and off < pending[-1][0]
        pending.append((off, off + n))
        assert not _overlaps(pending)
        assert [r[0] for r in ring.live] == [p[0] for p in pending]
        assert ring.used == sum(b - a for a, b in ring.live)
        assert ring.used <= ring.size
    assert wraps > 100


def test_ring_wraps_and_refuses_when_full():
    ring = ArenaRing(1000 * 256)
    a = ring.alloc(600 * 256)
    b = ring.alloc(300 * 256)
    assert (a, b) == (0, 600 * 256)
    assert ring.alloc(200 * 256) == -1          # only 100 blocks left at the end
    ring.release_oldest()                        # frees [0, 600)
    c = ring.alloc(200 * 256)                    # does not fit after b: wraps to 0
    assert c == 0
    assert ring.alloc(500 * 256) == -1           # [200, 600) is free, 400 blocks
    assert ring.alloc(400 * 256) == 200 * 256
    assert ring.alloc(1) == -1
    assert ring.alloc(2000 * 256) == -1          # larger than the arena


def test_empty_ring_starts_at_zero():
    ring = ArenaRing(4096)
    assert ring.alloc(4096) == 0
    ring.release_oldest()
    assert ring.alloc(100) == 0 and ring.used == 256
