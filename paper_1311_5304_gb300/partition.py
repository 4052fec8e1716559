"""The simple partitioning scheme of Sec. 5 (SPS, Eq. 7-9) as a planning
calculation.

After host Huffman decoding, SPS gives ``x`` image rows to the CPU and the
other ``h - x`` to the GPU, choosing ``x`` so that both finish together: the
root of

    f(x) = T_dispatch(h - x) + P_CPU(x) - P_GPU(h - x)

found by Newton's method and rounded to whole MCU rows (libjpeg-turbo decodes
in MCU units; so does this library).  Of the two neighbouring MCU multiples,
and no split at all, the one with the shorter parallel phase is taken: when
one MCU row costs the CPU more than the whole imbalance, rounding the root to
the nearest multiple, as the paper does, can be slower than not splitting.  The cost functions are whatever model
the caller has -- the paper fits polynomials per platform; ``bench.py`` uses
linear models from its own measurements.

This module only computes the split.  The library has no CPU back-end to give
rows to (its only CPU implementation of the back-end is the test oracle), so
the split is reported as an estimate of what co-processing would gain, not
executed.
"""
from __future__ import annotations

from typing import Callable

Cost = Callable[[float], float]


def sps_split(h: int, mcu_rows: int, p_cpu: Cost, p_gpu: Cost, t_dispatch: Cost | None = None,
              x0: float | None = None, max_iter: int = 60) -> int:
    """Rows for the CPU (a multiple of ``mcu_rows`` in [0, h], or h) that
    balance the CPU's and the GPU's parallel phase.  ``p_cpu(x)``: CPU time for x
    rows; ``p_gpu(y)``: GPU time (kernels and transfers) for y rows;
    ``t_dispatch(y)``: CPU time spent launching the GPU's y rows."""
    if h <= 0:
        return 0
    td = t_dispatch or (lambda y: 0.0)

    def f(x: float) -> float:
        return td(h - x) + p_cpu(x) - p_gpu(h - x)

    # no rows for the CPU when, with none, its dispatch work already lasts as
    # long as the GPU's whole share; all rows when the CPU finishes the whole
    # image before the GPU would finish nothing
    if f(0.0) >= 0.0:
        return 0
    if f(float(h)) <= 0.0:
        return h
    x = float(h) / 2 if x0 is None else min(max(float(x0), 0.0), float(h))
    step = max(1e-3, h * 1e-6)
    for _ in range(max_iter):
        fx = f(x)
        d = (f(min(x + step, h)) - f(max(x - step, 0.0))) / (min(x + step, h) - max(x - step, 0.0))
        if d == 0.0:
            break
        nx = min(max(x - fx / d, 0.0), float(h))
        if abs(nx - x) < 1e-6:
            x = nx
            break
        x = nx
    lo = min(h, int(x // mcu_rows) * mcu_rows)
    cands = {0, lo, min(h, lo + mcu_rows)}
    return min(sorted(cands), key=lambda r: balanced_time(h, r, p_cpu, p_gpu, t_dispatch))


def balanced_time(h: int, x: int, p_cpu: Cost, p_gpu: Cost, t_dispatch: Cost | None = None) -> float:
    """Parallel-phase time of a split: the later of the two sides (Sec. 5,
    T_total = max(T_CPU, T_GPU) without the shared Huffman term)."""
    td = t_dispatch or (lambda y: 0.0)
    return max(td(h - x) + p_cpu(x), p_gpu(h - x))


def pps_split(h: int, mcu_rows: int, chunk_rows: int, t_huffman: Cost, p_cpu: Cost, p_gpu: Cost,
              t_dispatch: Cost | None = None) -> int:
    """The pipelined scheme of Sec. 5 (PPS): the CPU entropy-decodes the whole
    image -- all but the first GPU chunk of it while the GPU already works --
    and then transforms its own x rows, so its side of the balance is
    T_Huffman(h - c) + P_CPU(x) (+ dispatch), the GPU's P_GPU(h - x).
    ``t_huffman(rows)``: host decoding time for that many rows."""
    rest = t_huffman(max(0, h - chunk_rows))
    return sps_split(h, mcu_rows, lambda x: rest + p_cpu(x), p_gpu, t_dispatch)
