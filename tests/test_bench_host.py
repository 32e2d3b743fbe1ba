"""Host-side arithmetic of the measurement: the algorithmic bytes the roofline
divides by, pinned to figures derived by hand from the array sizes (no GPU).

cube64_a8: 64^3 voxels, alpha 8, one plane wave.  The present-time grid is
M0 = 72^3 (half spectrum H0 = 37), the history grid Mh = 128^3 (Hh = 65), 26
history lags.  cube64_b16: the same cube with 16 plane waves.
"""
import types

import bench
from paper_2607_28309_b300 import mvp_bench

INFO = types.SimpleNamespace(M0=(72, 72, 72), Mh=(128, 128, 128), ell=26)
N = (64, 64, 64)


def test_z_pass_and_history_bytes_cube64_a8():
    kb = bench.kernel_bytes(INFO, N, 1, 1, [40])
    planes = 3 * 64 * 72 * 37 * 8          # (component, z, ky, kx) complex FP32
    lam0 = 6 * 37 * 37 * 37 * 4            # Lambda0 octant, six components, FP32
    assert kb["z_green"] == 2 * planes + lam0 == 9_399_480
    slot = 3 * 128 * 128 * 65 * 8          # one history-ring slot
    lam_h = 6 * 65 ** 3 * 4                # one Lambda_k octant
    out = 3 * 64 * 128 * 65 * 8            # the Nz kept planes of the inverse z pass
    # critical path: the step's partial sum + the lag-1 slot + Lambda_1 in, the kept planes out
    assert kb["z_history"] == 2 * slot + lam_h + out
    # step 40 is the first of a time block (40 mod 8 = 0): the block pass reads the
    # 25 ring slots within ell of it and Lambda_2..Lambda_26 once, writes 8 partial sums
    assert kb["hist_side"] == 25 * slot + 25 * lam_h + 8 * slot
    # step 43 (t = 3): near lags 2..4 onto its partial sum
    assert bench.kernel_bytes(INFO, N, 1, 1, [43])["hist_side"] == 3 * (slot + lam_h) + 2 * slot
    # averaged over a whole block (steps 40..47): one block pass, near lags 1+2+...+7 = 28,
    # seven near read-modify-writes of a partial sum; less than half the direct sum's
    # 26 (slot + Lambda) per step
    kb8 = bench.kernel_bytes(INFO, N, 1, 1, list(range(40, 48)))
    assert kb8["hist_side"] * 8 == 25 * slot + 25 * lam_h + 8 * slot + 28 * (slot + lam_h) + 7 * 2 * slot
    assert kb8["hist_side"] + kb8["z_history"] - out < 26 * (slot + lam_h) / 2


def test_spread_history_schedule_bytes_cube64_a8():
    slot = 3 * 128 * 128 * 65 * 8
    lam_h = 6 * 65 ** 3 * 4
    out = 3 * 64 * 128 * 65 * 8
    kb = bench.kernel_bytes(INFO, N, 1, 1, [40], spread=True)
    # step 40 is the first of a time block (40 mod 8 = 0): the recent part of the block
    # reads the 8 newest of the 25 ring slots within ell of it (ages 0..7) and
    # Lambda_2..Lambda_16, and reads and writes the block's 8 partial sums; and one
    # eighth of the next block's old part (block 48: the 17 slots of ages 8..24, its
    # Lambda_10..Lambda_26, 8 partial sums written)
    old48 = (17 * slot + 17 * lam_h + 8 * slot) / 8
    assert kb["hist_side"] == 8 * slot + 15 * lam_h + 16 * slot + old48
    # step 43 (t = 3): near lags 2..4 onto its partial sum, and its chunk of block 48's old part
    assert bench.kernel_bytes(INFO, N, 1, 1, [43], spread=True)["hist_side"] == 3 * (slot + lam_h) + 2 * slot + old48
    # averaged over a whole block (steps 40..47): the recent part once, the next block's
    # old part once, near lags 1+2+...+7 = 28, seven near read-modify-writes of a
    # partial sum; less than half the direct sum's 26 (slot + Lambda) per step
    kb8 = bench.kernel_bytes(INFO, N, 1, 1, list(range(40, 48)), spread=True)
    assert abs(kb8["hist_side"] * 8 - (8 * slot + 15 * lam_h + 16 * slot + 8 * old48 + 28 * (slot + lam_h)
                                       + 7 * 2 * slot)) < 1e-6 * kb8["hist_side"]
    assert kb8["hist_side"] + kb8["z_history"] - out < 26 * (slot + lam_h) / 2


def test_fused_solver_pass_bytes_cube64_a8():
    kb = bench.kernel_bytes(INFO, N, 1, 1, [26])
    vec = 3 * 64 ** 3 * 4                  # one FP32 solver vector
    planes = 3 * 64 * 72 * 37 * 8
    eps = 64 ** 3 * 4
    assert kb["fwd_half"] == 10 * vec + planes == 35_549_184
    assert kb["fwd_y1"] == 3 * vec + planes
    assert kb["inv_half"] == planes + eps + 9 * vec == 33_452_032
    assert kb["inv_v"] == planes + eps + 6 * vec == 24_014_848


def test_fp64_doubles_the_real_element():
    k32 = bench.kernel_bytes(INFO, N, 1, 1, [41], TB=8)
    k64 = bench.kernel_bytes(INFO, N, 1, 0, [41], TB=8)
    assert k64["z_green"] == 2 * k32["z_green"]
    assert k64["z_history"] == 2 * k32["z_history"]


def test_product_pass_bytes_cube64_b16():
    vec = 16 * 3 * 64 ** 3 * 4
    planes = 16 * 3 * 64 * 72 * 37 * 8
    lam = 6 * 37 ** 3 * 4
    eps = 64 ** 3 * 4
    assert mvp_bench.info_plane_fits(INFO, N, 4)
    expect = (vec + planes) + (2 * planes + lam) + (planes + eps + 2 * vec)
    assert mvp_bench.pass_bytes(INFO, N, 16, 4) == expect == 415_141_048


def test_profiled_traffic_is_a_number_or_none():
    assert bench.profiled_traffic("no_such_kernel_class") is None
    t = bench.profiled_traffic("z_green")
    assert t is None or t > 0
