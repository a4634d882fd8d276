"""Host-side accounting of bench.py (no GPU): the mulmods the roofline
attributes to the row kernel plus those of the column kernels make up the
whole product of Eq. 2, for both row lengths."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_split_mulmods_add_up():
    import bench
    for log2n in range(12, 18):
        n = 1 << log2n
        for row_log in (10, 12):
            cl = log2n - row_log
            cols = 2 * cl * (n // 2) + cl * (n // 2)  # forward a, b; inverse c
            assert bench.rows_kernel_mulmods(log2n, row_log) + cols == bench.mulmods_per_polymul(log2n)


def test_mulmods_closed_form():
    import bench
    # 3 transforms of N/2 log2 N butterflies plus N products: 25 N at N = 2^16
    assert bench.mulmods_per_polymul(16) == 25 * (1 << 16)
    assert bench.rows_kernel_mulmods(16, 10) == 16 * (1 << 16)
    assert bench.rows_kernel_mulmods(16, 12) == 19 * (1 << 16)
