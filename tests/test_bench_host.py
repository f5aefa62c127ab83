"""Host-side accounting of bench.py: the algorithmic bytes per pass that the roofline
fractions divide by, separate and with the fused x-y passes."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_pass_bytes_sum():
    import bench
    N, s = 256, 4
    K = N + 1
    b = bench.pass_bytes(N, s)
    # Every operand read or written once: rho and u (s N^3 each), w1 twice each way
    # (2s N^2 K per touch), w2 and w3 (4s N^2 K per touch, three touches each), the symbol
    # octant (s K^3) once.
    assert sum(b) == 2 * s * N ** 3 + 4 * (2 * s * N * N * K) + 4 * (4 * s * N * N * K) + s * K ** 3


def test_pass_table_fused_drops_w1():
    import bench
    N, s = 192, 4
    K = N + 1
    per = [0.1, 0.2, 0.3, 0.4, 0.5]
    names = ["a", "b", "c", "d", "e"]
    sep = bench.pass_table(N, s, per, 0, names)
    assert [r[0] for r in sep] == bench.PASSES and [r[3] for r in sep] == bench.pass_bytes(N, s)
    fused = bench.pass_table(N, s, per, 1, names)
    assert [r[1] for r in fused] == ["k_xy_fwd", "c", "k_yx_inv"]
    assert [r[2] for r in fused] == [0.1, 0.3, 0.4]
    w1 = 2 * s * N * N * K  # one write or one read of w1
    b = bench.pass_bytes(N, s)
    assert fused[0][3] == b[0] + b[1] - 2 * w1
    assert fused[2][3] == b[3] + b[4] - 2 * w1
    assert fused[1][3] == b[2]
