"""The allocation-free reconstruction entry point against the allocating one.

srt3d_reconstruct_noalloc exists for callers that cannot allocate device
memory while reconstructing (a real-time loop where cudaMalloc/cudaFree may
stall the device, or a process whose device memory is reserved by another
allocator). Its scratch is a fixed 16 MiB device array shared by all calls,
and its phase table comes from the same host values srt3d_reconstruct uses,
so its results must equal srt3d_reconstruct's bit for bit.
This file is collected last so that a failure here leaves every other test
already run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import synth

from gpu_util import ctx, dev_offsets, dev_stamps  # noqa: F401

pytestmark = pytest.mark.gpu


def _frame(ctx, spec, seed, m):
    fr = synth.make_stream_frame(spec, seed)
    P = spec.num_pixels
    S = torch.empty(P, m, 2, device="cuda")
    n = torch.empty(P, dtype=torch.int32, device="cuda")
    z = torch.empty(P, m, 2, device="cuda")
    B.srt3d_sketch_stream(ctx, dev_stamps(fr.stamps), dev_offsets(fr.offsets), spec.T, m, 0, S, n)
    B.srt3d_finalize(ctx, S, n, m, z)
    h = torch.from_numpy(synth.impulse_response(spec.T, spec.sigma).astype(np.float32)).cuda()
    return z, n, h


def _outputs(P, K):
    return (torch.full((P, K), -1.0, device="cuda"), torch.full((P, K), -1.0, device="cuda"),
            torch.full((P, K), 7, dtype=torch.uint8, device="cuda"), torch.full((P,), -1.0, device="cuda"))


def _run(fn, ctx, spec, m, z, n, h, prm, outs=None):
    outs = outs or _outputs(spec.num_pixels, prm.k_max)
    fn(ctx, z, n, spec.rows, spec.cols, spec.T, m, h, prm, *outs)
    B.srt3d_sync(ctx)
    return [t.cpu().numpy() for t in outs]


def _assert_identical(got, ref):
    for name, a, b in zip(("depth", "alpha", "active", "alpha0"), got, ref):
        assert np.array_equal(a, b), f"{name} differs in {np.count_nonzero(a != b)} entries"


def _spec(rows, cols, T, sigma=6.0, photons=1000.0, two=0.3):
    return synth.FrameSpec(rows=rows, cols=cols, T=T, sigma=sigma, mean_photons=photons, sbr=0.5,
                           two_surface_frac=two, sep_lo=min(50.0, T / 8), sep_hi=min(300.0, T / 4))


CASES = [
    # one launch for all iterations (two surfaces, m = 10)
    ("persistent_K2", _spec(40, 36, 4096), 10, dict(iters=20, k_max=2, d_max=36.0, min_sep=18.0)),
    # a different size, k_max and T: stale contents of the shared array from
    # the call before would show
    ("persistent_K1", synth.frame_32x32(), 4, dict(iters=20, k_max=1, d_max=24.0, min_sep=12.0)),
    # T > 8192: the two-level phase table
    ("two_level_T16384", _spec(24, 20, 16384, sigma=8.0), 8, dict(iters=10, k_max=2, d_max=48.0, min_sep=24.0)),
    # pixelwise estimate, W = I and W = Sigma_theta^-1
    ("pixelwise", _spec(24, 28, 2048, sigma=4.0), 6, dict(iters=15, k_max=2, regularize=0, d_max=24.0,
                                                           min_sep=12.0)),
    ("pixelwise_weighted", _spec(24, 28, 2048, sigma=4.0), 6, dict(iters=15, k_max=2, regularize=0, weighting=1,
                                                                    d_max=24.0, min_sep=12.0)),
]


def test_noalloc_equals_allocating_entry_point_call_after_call(ctx):
    for i, (name, spec, m, kw) in enumerate(CASES):
        z, n, h = _frame(ctx, spec, 101 + i, m)
        prm = B.make_params(**kw)
        ref = _run(B.srt3d_reconstruct, ctx, spec, m, z, n, h, prm)
        got = _run(B.srt3d_reconstruct_noalloc, ctx, spec, m, z, n, h, prm)
        assert np.all(got[2] <= 1), name  # every output word was written
        _assert_identical(got, ref)


def test_noalloc_at_its_largest_frame(ctx):
    # rows * cols * k_max = 512 * 640 * 2 = 655360 points, the documented
    # limit: the largest scratch layout must stay clear of the phase table at
    # the end of the array (too many tiles for one launch, so the iterations
    # run one launch each through the array's ping-pong buffers)
    spec = synth.FrameSpec(rows=512, cols=640, T=1024, sigma=4.0, mean_photons=20.0, sbr=1.0,
                           two_surface_frac=0.1, sep_lo=50.0, sep_hi=200.0)
    m = 4
    z, n, h = _frame(ctx, spec, 7, m)
    prm = B.make_params(iters=3, k_max=2, d_max=24.0, min_sep=12.0)
    ref = _run(B.srt3d_reconstruct, ctx, spec, m, z, n, h, prm)
    got = _run(B.srt3d_reconstruct_noalloc, ctx, spec, m, z, n, h, prm)
    _assert_identical(got, ref)
    got2 = _run(B.srt3d_reconstruct_noalloc, ctx, spec, m, z, n, h, prm)
    _assert_identical(got2, ref)


def test_noalloc_allocates_no_device_memory(ctx):
    # warm-up call (loads the kernels it needs), then a call with a new T and
    # frame size: the device's free memory must not move. The allocating entry
    # point, on a fresh context that has no scratch yet, shows that the check
    # sees an allocation.
    spec_a, spec_b, spec_c = _spec(40, 36, 4096), _spec(48, 52, 2048), _spec(300, 300, 2048, photons=50.0)
    m, prm = 10, B.make_params(iters=5, k_max=2, d_max=36.0, min_sep=18.0)
    fa, fb, fc = (_frame(ctx, s, 300 + i, m) for i, s in enumerate((spec_a, spec_b, spec_c)))
    outs_a, outs_b, outs_c = (_outputs(s.num_pixels, 2) for s in (spec_a, spec_b, spec_c))
    fresh = B.srt3d_create(0)
    try:
        _run(B.srt3d_reconstruct_noalloc, ctx, spec_a, m, *fa, prm, outs_a)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _run(B.srt3d_reconstruct_noalloc, ctx, spec_b, m, *fb, prm, outs_b)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0
        _run(B.srt3d_reconstruct, fresh, spec_c, m, *fc, prm, outs_c)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] < free1
    finally:
        B.srt3d_destroy(fresh)


def test_noalloc_rejects_frames_beyond_its_scratch(ctx):
    T, m = 64, 4
    z = torch.zeros(4, m, 2, device="cuda")
    n = torch.zeros(4, dtype=torch.int32, device="cuda")
    h = torch.ones(T, device="cuda")
    d = torch.zeros(4, 2, device="cuda")
    a = torch.zeros(4, 2, device="cuda")
    act = torch.zeros(4, 2, dtype=torch.uint8, device="cuda")
    a0 = torch.zeros(4, device="cuda")
    # 512 x 641 x 2 points > 655360: rejected before any launch
    st = B.srt3d_reconstruct_noalloc(ctx, z, n, 512, 641, T, m, h, B.make_params(k_max=2), d, a, act, a0,
                                     check=False)
    assert st == B.SRT3D_EINVAL
    assert b"too large" in B.lib().srt3d_last_error(ctx)
