"""The work and byte model bench.py reports against, checked on the CPU.

Sec. 3's cost discussion after Alg. 2 counts step 3's tall products; the model
adds the triangular solve with R_ii and the two sketches per column (W_i in
step 1, Q_i in step 5).  These tests fix the model
at the n = 1e6, m = 1000, m_p = 50, SRHT k = 2000 workload with the terms
written out by hand, and tie the two-pass bytes to the sum of the tall
kernel's per-launch bytes, which is what the live roofline divides by."""
import math
import sys
from pathlib import Path

import pytest

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402

N, M, MB, K = 1_000_000, 1000, 50, 2000


def test_algorithmic_flops_at_the_qr_workload():
    npad = 1 << 20  # 2^ceil(log2 1e6)
    tall = N * M * (M - MB)          # sum over blocks of 2 n c_i m_p, c_i = (i - 1) m_p
    trsm = N * M * MB                 # n m_p^2 per block, p blocks
    srht = 2 * M * npad * 20          # n' log2 n' additions per column, W and Q
    assert tall == 9.5e11 and trsm == 5.0e10
    assert bench.algorithmic_flops(N, M, MB, K, "srht") == pytest.approx(tall + trsm + srht, rel=1e-15)
    assert bench.algorithmic_flops(N, M, MB, K, "srht") == pytest.approx(1.04194304e12, rel=1e-12)


def test_tall_products_are_the_sum_over_blocks():
    p = M // MB
    by_block = sum(2 * N * (i * MB) * MB for i in range(p))
    assert by_block == N * M * (M - MB)


def test_dense_sketch_flops_are_two_k_n_per_column():
    assert bench.sketch_flops_per_col(10_000, 200, "gauss") == 2 * 200 * 10_000
    assert bench.sketch_flops_per_col(10_000, 200, "rademacher") == 2 * 200 * 10_000
    # SRHT pads to the next power of two
    assert bench.sketch_flops_per_col(16_385, 300, "srht") == (1 << 15) * 15


def test_minimum_bytes_single_pass():
    p = M // MB
    basis_reads = 4 * N * MB * sum(range(p))   # block i reads Q_{1:i-1}
    w_and_q = 4 * 2 * N * M                    # W read once, Q written once
    assert basis_reads + w_and_q == 4.6e10
    assert bench.algorithmic_bytes(N, M, MB, 4) == pytest.approx(4.6e10, rel=1e-15)
    assert bench.algorithmic_bytes(N, M, MB, 8) == pytest.approx(9.2e10, rel=1e-15)


def test_two_pass_bytes_equal_the_tall_launch_bytes():
    """Every block's first pass and every block but the first one's second
    pass: launches of 4 n (c + 2 m_p) bytes each, c the basis columns read."""
    p = M // MB
    first = [4 * N * (i * MB + 2 * MB) for i in range(p)]
    second = [4 * N * (i * MB + 2 * MB) for i in range(1, p)]
    assert bench.two_pass_bytes(N, M, MB, 4, p - 1) == pytest.approx(sum(first) + sum(second), rel=1e-12)
    assert bench.two_pass_bytes(N, M, MB, 4, p - 1) == pytest.approx(9.16e10, rel=1e-12)


def test_overhead_is_zero_without_richardson_and_second_pass():
    assert bench.overhead_flops(N, M, MB, K, "srht", 0, 0) == 0.0
    one = bench.overhead_flops(N, M, MB, K, "srht", 1, 0)
    assert one == pytest.approx(2.0 * K * M * (M - MB))
    assert math.isfinite(bench.overhead_flops(N, M, MB, K, "srht", 1, 19))
