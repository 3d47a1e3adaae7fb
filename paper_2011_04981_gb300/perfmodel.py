"""Operation and byte counts of the AX operator, used to turn times into rates.

Flops per grid point (Section III of arXiv 2011.04981 quotes 203 for n = 16):
six n-term contractions at 2n-1 operations each (n products, n-1 sums), the
symmetric 3x3 geometric product at 9 products + 6 sums, and 2 sums that add the
three transposed contractions: 6(2n-1) + 15 + 2 = 12n + 11.

Bytes per grid point (algorithmic, FP64): u read (8), six geometric factors
read (48) and w written (8) = 64; D is n^2 values per launch and is ignored.
"""


def ax_flops_per_point(nx: int) -> int:
    return 6 * (2 * nx - 1) + 15 + 2


def ax_flops_per_element(nx: int) -> int:
    return ax_flops_per_point(nx) * nx ** 3


def ax_bytes_per_point(value_bytes: int = 8) -> int:
    """u + 6 geometric factors + w, each ``value_bytes`` wide."""
    return 8 * value_bytes


def matmul_flops_per_cycle(nx: int) -> int:
    """One n-term contraction result per cycle: n products and n-1 sums."""
    return 2 * nx - 1
