"""The benchmark's roofline numerator (algorithmic HBM bytes of a solve) on
the CPU: per-cell bytes of one PCG iteration of the fused schedule, which
levels the single-CTA solver keeps in shared memory, and the total for the
1024^2 workload at its measured iteration counts."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

DIMS_1024 = [(1024, 1024, 1), (256, 256, 1), (64, 64, 1), (16, 16, 1), (4, 4, 1)]


@pytest.mark.parametrize("prec,k,per_cell", [(0, 0, 169.0), (0, 2, 169.0), (1, 1, 84.5), (1, 0, 140.0)])
def test_bytes_per_cell_2d(prec, k, per_cell):
    # (3d + 15 + 2/s^d) words per cell: 21.125 words in 2D with s = 4
    assert bench.level_bytes_per_iter(k, (10, 7, 1), prec) == pytest.approx(per_cell * 70)


def test_bytes_per_cell_3d():
    words = 9 + 15 + 2 / 64
    assert bench.level_bytes_per_iter(1, (8, 8, 8), 0, dim=3) == pytest.approx(8 * words * 512)


def test_shared_memory_levels_at_1024():
    assert bench.smem_resident_levels(DIMS_1024, 1) == {2, 3, 4}
    assert 1 not in bench.smem_resident_levels(DIMS_1024, 0)


def test_algorithmic_bytes_of_a_1024_solve():
    stats = {"dims": DIMS_1024, "iters": [9, 101, 1227, 4635, 4635]}
    expect = 9 * 140.0 * 1024 ** 2 + 101 * 84.5 * 256 ** 2
    assert bench.hbm_bytes_of_solve(stats, 1) == pytest.approx(expect)
    assert expect == pytest.approx(1.881e9, rel=1e-3)
