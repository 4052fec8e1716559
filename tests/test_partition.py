"""Sec. 5's simple partitioning scheme (Eq. 7-9) as computed by
partition.sps_split: the Newton root of the balance equation, pinned against
the closed-form root of linear cost models, the clamps at both ends and the
rounding to whole MCU rows."""
import pytest

from paper_1311_5304_gb300 import partition


@pytest.mark.parametrize("a,b,c,d", [(1.0, 1.0, 0.0, 0.0), (50.0, 1.0, 30.0, 5.0), (0.2, 3.0, 100.0, 1.0)])
def test_linear_models_give_the_closed_form_root(a, b, c, d):
    # f(x) = d + a x - (b (h - x) + c)  =>  x* = (b h + c - d) / (a + b)
    h = 4096
    x = partition.sps_split(h, 1, lambda x: a * x, lambda y: b * y + c, lambda y: d)
    want = (b * h + c - d) / (a + b)
    assert abs(x - want) <= 1.0 + 1e-9
    # balanced: neither side is more than one row's cost slower
    t_cpu, t_gpu = d + a * x, b * (h - x) + c
    assert abs(t_cpu - t_gpu) <= max(a, b)


def test_rounding_to_mcu_rows_and_clamps():
    h = 1000
    x = partition.sps_split(h, 16, lambda x: 1.0 * x, lambda y: 1.0 * y)
    assert x % 16 == 0 and abs(x - 500) <= 16
    # one MCU row of CPU work costs more than the whole imbalance: no split
    assert partition.sps_split(h, 16, lambda x: 5.0 * x, lambda y: 0.01 * y + 1.0, lambda y: 0.5) == 0
    # a GPU far faster than the dispatch cost: nothing for the CPU
    assert partition.sps_split(h, 8, lambda x: 10.0 * x, lambda y: 0.001 * y, lambda y: 5.0) == 0
    # a GPU with a fixed cost above the CPU's whole-image time: everything for the CPU
    assert partition.sps_split(h, 8, lambda x: 0.01 * x, lambda y: 100.0 + y) == h


def test_split_never_loses_to_either_side_alone():
    h = 8192
    p_cpu = lambda x: x / 30.0          # noqa: E731
    p_gpu = lambda y: 2.0 + y / 900.0   # noqa: E731
    x = partition.sps_split(h, 16, p_cpu, p_gpu)
    t = partition.balanced_time(h, x, p_cpu, p_gpu)
    assert t <= partition.balanced_time(h, 0, p_cpu, p_gpu) + 1e-12
    assert t <= partition.balanced_time(h, h, p_cpu, p_gpu) + 1e-12


def test_pps_counts_the_overlapped_huffman_on_the_cpu_side():
    h, c = 4096, 256
    p_cpu = lambda x: 1.0 * x          # noqa: E731
    p_gpu = lambda y: 1.0 * y          # noqa: E731
    huff = lambda rows: 0.25 * rows    # noqa: E731
    x = partition.pps_split(h, 1, c, huff, p_cpu, p_gpu)
    # 0.25 (h - c) + x = h - x
    want = (h - 0.25 * (h - c)) / 2
    assert abs(x - want) <= 1.0
    # host decoding slower than the GPU's whole share: the CPU takes no rows
    assert partition.pps_split(h, 16, c, lambda r: 10.0 * r, p_cpu, lambda y: 0.001 * y) == 0
