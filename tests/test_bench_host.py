"""Host-side accounting of bench.py: the algorithmic bytes per pass that the roofline
fractions divide by, separate and with the fused x-y passes."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_pass_bytes_sum():
    import bench
    N = 256
    # Per grid point in FP32: rho and u (4 B each), the x spectrum written and read twice
    # each way (8 B per touch), the y-padded spectrum written and read twice each way
    # (16 B per touch): 104 B; FP64 doubles it.  The symbol octant is not algorithmic.
    assert sum(bench.pass_bytes(N, 4)) == 104 * N ** 3
    assert sum(bench.pass_bytes(N, 8)) == 208 * N ** 3
    assert bench.pass_bytes(N, 4)[2] == 32 * N ** 3
    assert bench.symbol_bytes(N, 4) == 4 * (N + 1) ** 3


def test_errors_are_relative_l2_and_linf():
    import numpy as np
    import bench
    ref = np.array([3.0, -4.0, 0.0])
    e = bench.errors(ref + np.array([0.0, 0.0, 0.5]), ref)
    assert abs(e["rel_l2"] - 0.1) < 1e-15 and abs(e["rel_linf"] - 0.125) < 1e-15


def test_pass_table_fused_drops_w1():
    import bench
    N, s = 192, 4
    per = [0.1, 0.2, 0.3, 0.4, 0.5]
    names = ["a", "b", "c", "d", "e"]
    sep = bench.pass_table(N, s, per, 0, names)
    assert [r[0] for r in sep] == bench.PASSES and [r[3] for r in sep] == bench.pass_bytes(N, s)
    fused = bench.pass_table(N, s, per, 1, names)
    assert [r[1] for r in fused] == ["k_xy_fwd", "c", "k_yx_inv"]
    assert [r[2] for r in fused] == [0.1, 0.3, 0.4]
    w1 = 2 * s * N ** 3     # one write or one read of the x spectrum (N^3 complex)
    b = bench.pass_bytes(N, s)
    assert fused[0][3] == b[0] + b[1] - 2 * w1
    assert fused[2][3] == b[3] + b[4] - 2 * w1
    assert fused[1][3] == b[2]


def test_traffic_table_is_plausible_and_keyed_by_source():
    """Each DRAM traffic figure bench.py can report lies between the z pass's algorithmic
    bytes and those plus the symbol octant read twice (the excess ncu showed at N = 512),
    and is looked up by the hash of the kernel sources it was taken on, so a figure taken on
    other sources is reported as null."""
    import bench
    assert bench.NCU_TRAFFIC, "no traffic figure"
    for (key_hash, kernel, N), traffic in bench.NCU_TRAFFIC.items():
        assert len(key_hash) == 16 and int(key_hash, 16) >= 0
        alg = bench.pass_bytes(N, 4)[2]
        assert alg <= traffic <= alg + 2 * bench.symbol_bytes(N, 4), (kernel, N, traffic)
        assert bench.NCU_TRAFFIC.get(("0" * 16, kernel, N)) is None
