"""CPU tests of the library's host-side launch planning (srt3d_plan): no GPU
and no context are needed. Each planned quantity is checked against the
definition it follows, not against a copy of the library's arithmetic."""
import math

import numpy as np
import pytest

from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import build as builder

TILE_W = 16  # columns per tile of the iteration kernel


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()


def _plan(rows=256, cols=256, T=4096, m=10, k_max=2, radius=1, mean=1000.0, sms=152, bps=2):
    return B.srt3d_plan(rows, cols, T, m, k_max, radius, mean, sms, bps)


def test_frame_of_the_main_workload():
    # 256 x 256 pixels, T = 4096, m = 10, two points per pixel, radius 1, on
    # 152 SMs with two iteration CTAs each
    p = _plan()
    assert p["sketch_m"] == 10 and p["init_m"] == 10
    assert p["init_grid_spacing"] == 32 and p["init_grid_points"] == 128
    assert p["sketch_lanes"] == 16
    assert p["tile_height"] == 14 and p["tiles"] == 16 * 19 == 304


@pytest.mark.parametrize("T", [2, 3, 64, 1000, 1024, 4096, 4613, 8192, 65536])
@pytest.mark.parametrize("m", [1, 2, 3, 7, 10, 16, 20, 32])
def test_grid_spacing_is_the_largest_power_of_two_within_the_curvature_bound(T, m):
    # the score s(t) = Re sum_l c_l e^{i w_l t} has |s''| <= sum |c_l| w_l^2
    # <= sum |c_l| w_m^2, so between grid points D apart it rises at most
    # (sum |c_l|) w_m^2 D^2 / 8 above the chord; the plan keeps w_m^2 D^2 / 8
    # <= 0.08 with D a power of two <= 64, as large as allowed
    p = _plan(T=T, m=m)
    D = p["init_grid_spacing"]
    assert D >= 1 and D <= 64 and D & (D - 1) == 0
    w = 2 * math.pi * m / T
    bound = lambda d: w * w * d * d / 8.0  # noqa: E731
    assert D == 1 or bound(D) <= 0.08
    assert D == 64 or bound(2 * D) > 0.08
    assert p["init_grid_points"] == -(-T // D)


def test_instantiations_cover_m_and_grow_with_it():
    prev_s = prev_i = 0
    for m in range(1, 33):
        p = _plan(m=m)
        assert p["sketch_m"] >= m and p["init_m"] >= m
        assert p["sketch_m"] >= prev_s and p["init_m"] >= prev_i
        prev_s, prev_i = p["sketch_m"], p["init_m"]
    assert _plan(m=32)["sketch_m"] == 32 and _plan(m=32)["init_m"] == 32


def test_sketch_lanes_follow_the_photon_density():
    lanes = [_plan(mean=x)["sketch_lanes"] for x in (0.0, 1.0, 10.0, 50.0, 100.0, 200.0, 1000.0, 1e6)]
    assert all(v in (4, 8, 16, 32) for v in lanes)
    assert lanes == sorted(lanes)
    assert lanes[0] == 4 and lanes[-1] == 16


def test_tile_plan_fits_the_device_at_once():
    rng = np.random.default_rng(3)
    for _ in range(300):
        rows, cols = int(rng.integers(1, 700)), int(rng.integers(1, 700))
        sms, bps = int(rng.integers(1, 200)), int(rng.integers(1, 4))
        k, r = int(rng.integers(1, 5)), int(rng.integers(1, 4))
        p = _plan(rows=rows, cols=cols, k_max=k, radius=r, sms=sms, bps=bps)
        tiles_x = -(-cols // TILE_W)
        th = p["tile_height"]
        if th:
            assert 4 <= th <= 16
            assert p["tiles"] == tiles_x * -(-rows // th)
            assert p["tiles"] <= sms * bps
            assert not (k > 2 and r > 1)
        else:
            assert p["tiles"] == 0
            # either the frame runs per iteration by rule, or even the
            # shortest tiles (4 rows) would not all fit at once
            assert (k > 2 and r > 1) or tiles_x * -(-rows // 4) > sms * bps


def test_larger_frames_fall_back_to_one_launch_per_iteration():
    assert _plan(rows=512, cols=512)["tile_height"] == 0
    assert _plan(k_max=3, radius=2, bps=4)["tile_height"] == 0
    assert _plan(k_max=3, radius=1)["tile_height"] > 0


@pytest.mark.parametrize("kw", [dict(rows=0), dict(cols=0), dict(T=1), dict(T=65537), dict(m=0), dict(m=33),
                                dict(k_max=0), dict(k_max=5), dict(radius=0), dict(radius=4), dict(sms=0),
                                dict(bps=0), dict(mean=-1.0), dict(mean=float("nan"))])
def test_invalid_arguments_are_refused(kw):
    with pytest.raises(B.SRT3DError) as ei:
        _plan(**kw)
    assert ei.value.status == B.SRT3D_EINVAL


def test_bench_counts_the_grid_the_library_plans():
    # bench.py's roofline counts the init's grid points with its own copy of
    # the spacing rule; it must match what the library launches
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    for T in (64, 1024, 2048, 4096, 4613, 65536):
        for m in (1, 4, 10, 16, 20, 32):
            assert bench.mf_grid_spacing(T, m) == _plan(T=T, m=m)["init_grid_spacing"]


def test_serving_frame_bytes_hold_the_frame_state():
    # an admitted frame keeps on the device its sketch state S (P x m complex
    # FP32), counts n, impulse response h (T FP32) and results (depth, alpha
    # as FP32 and active as bytes per point, alpha_0 per pixel), plus the
    # reconstruction's scratch (including a fixed 16 KiB of progress flags
    # for the tiles of the one-launch iteration kernel and 4 KiB of partial
    # sums of hhat); each array starts on a 256-byte boundary
    for rows, cols, T, m, k in [(1, 1, 2, 1, 1), (32, 32, 1024, 4, 1), (256, 256, 4096, 10, 2),
                                (141, 141, 4613, 16, 2), (512, 512, 2048, 32, 4)]:
        P = rows * cols
        b = _plan(rows=rows, cols=cols, T=T, m=m, k_max=k)["serving_frame_bytes"]
        own = P * m * 8 + P * 4 + T * 4 + P * k * (4 + 4 + 1) + P * 4
        assert b >= own and b % 256 == 0
        assert b < own * 3 + 256 * 16 + 4096 * 4 + 4096
    base = _plan()["serving_frame_bytes"]
    for kw in (dict(rows=257), dict(cols=300), dict(m=11), dict(k_max=3), dict(T=8192)):
        assert _plan(**kw)["serving_frame_bytes"] > base
