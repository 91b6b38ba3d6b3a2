"""The allocation-free reconstruction entry point against the allocating one.

srt3d_reconstruct_noalloc exists for callers that cannot allocate device
memory while reconstructing (a real-time loop where cudaMalloc/cudaFree may
stall the device, or a process whose device memory is reserved by another
allocator). Its scratch is a fixed 16 MiB device array shared by all calls.
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

DEPTH_TOL = 0.05
INTENSITY_RTOL = 1e-3


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


def _run(fn, ctx, spec, m, z, n, h, prm):
    P, K = spec.num_pixels, prm.k_max
    depth = torch.full((P, K), -1.0, device="cuda")
    alpha = torch.full((P, K), -1.0, device="cuda")
    active = torch.full((P, K), 7, dtype=torch.uint8, device="cuda")
    alpha0 = torch.full((P,), -1.0, device="cuda")
    fn(ctx, z, n, spec.rows, spec.cols, spec.T, m, h, prm, depth, alpha, active, alpha0)
    B.srt3d_sync(ctx)
    return [t.cpu().numpy() for t in (depth, alpha, active, alpha0)]


def _compare(a, b, n):
    da, aa, acta, a0a = a
    db, ab, actb, a0b = b
    flips = np.count_nonzero(acta != actb)
    assert flips <= max(1, int(1e-3 * acta.size))
    both = (acta == 1) & (actb == 1)
    assert np.max(np.abs(da - db)[both], initial=0.0) <= DEPTH_TOL
    nn = n.astype(np.float64)[:, None]
    rel = np.abs(nn * aa - nn * ab)[both] / np.maximum(nn * ab, 1e-12)[both]
    assert np.max(rel, initial=0.0) <= INTENSITY_RTOL
    same = np.all(acta == actb, axis=1)
    np.testing.assert_allclose(a0a[same], a0b[same], atol=1e-5)


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row(ctx):
    # call 1: a two-surface frame; call 2: a different size and k_max, so any
    # stale contents of the shared array from call 1 would show up
    cases = [
        (synth.FrameSpec(rows=40, cols=36, T=4096, sigma=6.0, mean_photons=1000.0, sbr=0.5, two_surface_frac=0.3),
         10, dict(iters=20, k_max=2, d_max=36.0, min_sep=18.0)),
        (synth.frame_32x32(), 4, dict(iters=20, k_max=1, d_max=24.0, min_sep=12.0)),
    ]
    for i, (spec, m, kw) in enumerate(cases):
        z, n, h = _frame(ctx, spec, 101 + i, m)
        prm = B.make_params(**kw)
        ref = _run(B.srt3d_reconstruct, ctx, spec, m, z, n, h, prm)
        got = _run(B.srt3d_reconstruct_noalloc, ctx, spec, m, z, n, h, prm)
        _compare(got, ref, n.cpu().numpy().view(np.uint32))


def test_noalloc_rejects_frames_beyond_its_scratch(ctx):
    T, m = 64, 4
    z = torch.zeros(4, m, 2, device="cuda")
    n = torch.zeros(4, dtype=torch.int32, device="cuda")
    h = torch.ones(T, device="cuda")
    d = torch.zeros(4, 2, device="cuda")
    a = torch.zeros(4, 2, device="cuda")
    act = torch.zeros(4, 2, dtype=torch.uint8, device="cuda")
    a0 = torch.zeros(4, device="cuda")
    # 573 x 573 x 2 points > 655360: rejected before any launch
    st = B.srt3d_reconstruct_noalloc(ctx, z, n, 573, 573, T, m, h, B.make_params(k_max=2), d, a, act, a0, check=False)
    assert st == B.SRT3D_EINVAL
    assert b"too large" in B.lib().srt3d_last_error(ctx)
