"""Serving runtime (continuous batching): frames arrive in chunks, are sketched
online into device state (the online update of Sec. 2) and reconstructed
(Sec. 3). Each frame's result must be the same alone and in a mix of
concurrently running frames, chunked sketches must match one-shot ones, and
admission / errors must behave as documented in include/srt3d.h."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import synth

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture()
def sctx():
    require_gpu()
    from paper_2203_00952_gb300 import build as builder

    builder.build()
    c = B.srt3d_create(0)
    yield c
    B.srt3d_destroy(c)


def frames(num=6):
    specs = [(16, 16, 256, 4), (24, 20, 1024, 8), (32, 32, 1024, 4), (8, 40, 512, 6), (20, 20, 256, 10),
             (33, 17, 1024, 16)][:num]
    out = []
    for i, (r, c, T, m) in enumerate(specs):
        spec = synth.FrameSpec(rows=r, cols=c, T=T, sigma=3.0, mean_photons=150.0, sbr=1.0, two_surface_frac=0.2,
                               sep_lo=min(50.0, T / 8), sep_hi=min(300.0, T / 4))
        fr = synth.make_stream_frame(spec, 900 + i)
        prm = B.make_params(iters=10, k_max=2, d_max=18.0, min_sep=9.0)
        out.append((fr, m, prm))
    return out


def chunks_of(fr, nchunks, rng):
    """Split each pixel's photons into `nchunks` contiguous pieces (arrival order)."""
    P = fr.spec.num_pixels
    off = fr.offsets.astype(np.int64)
    cuts = []
    for p in range(P):
        c = np.sort(rng.integers(off[p], off[p + 1] + 1, size=nchunks - 1))
        cuts.append(np.concatenate([[off[p]], c, [off[p + 1]]]))
    out = []
    for k in range(nchunks):
        per = [fr.stamps[cuts[p][k]:cuts[p][k + 1]] for p in range(P)]
        st = np.concatenate(per).astype(np.uint16) if per else np.zeros(0, np.uint16)
        o = np.zeros(P + 1, np.uint32)
        o[1:] = np.cumsum([len(x) for x in per])
        out.append((np.ascontiguousarray(st), o))
    return out


def outputs(fr, prm):
    P, K = fr.spec.num_pixels, prm.k_max
    return (np.zeros((P, K), np.float32), np.zeros((P, K), np.float32), np.zeros((P, K), np.uint8),
            np.zeros(P, np.float32), np.zeros(P, np.uint32))


def poll(ctx, fid, fr, prm, timeout_us=20_000_000):
    o = outputs(fr, prm)
    B.srt3d_poll(ctx, fid, timeout_us, *o)
    return o


def submit_all(ctx, fid, fr, m, prm, chunk_list):
    h = synth.impulse_response(fr.spec.T, fr.spec.sigma).astype(np.float32)
    for k, (st, off) in enumerate(chunk_list):
        B.srt3d_submit(ctx, fid, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, st, off, int(k == len(chunk_list) - 1))


def test_alone_equals_mix(sctx):
    fs = frames()
    rng = np.random.default_rng(1)
    chunked = [chunks_of(fr, 8, rng) for fr, _, _ in fs]
    alone = []
    for i, (fr, m, prm) in enumerate(fs):
        submit_all(sctx, 100 + i, fr, m, prm, chunked[i])
        alone.append(poll(sctx, 100 + i, fr, prm))
    # mix: chunks of all frames interleaved, frames overlapping on the device
    for k in range(8):
        for i, (fr, m, prm) in enumerate(fs):
            h = synth.impulse_response(fr.spec.T, fr.spec.sigma).astype(np.float32)
            st, off = chunked[i][k]
            B.srt3d_submit(sctx, 200 + i, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, st, off, int(k == 7))
    mixed = [poll(sctx, 200 + i, fr, prm) for i, (fr, m, prm) in enumerate(fs)]
    for a, b in zip(alone, mixed):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_kept_pinned_chunks_upload_asynchronously_with_identical_results(sctx):
    fs = frames(3)
    rng = np.random.default_rng(4)
    ref, kept, pinned = [], [], []
    for i, (fr, m, prm) in enumerate(fs):
        ch = chunks_of(fr, 3, rng)
        submit_all(sctx, 300 + i, fr, m, prm, ch)
        ref.append(poll(sctx, 300 + i, fr, prm))
        pinned.append([(torch.from_numpy(st.view(np.int16)).pin_memory().numpy().view(np.uint16),
                        torch.from_numpy(off.view(np.int32)).pin_memory().numpy().view(np.uint32)) for st, off in ch])
    # all frames in flight, submit returning before the uploads finish
    for i, (fr, m, prm) in enumerate(fs):
        h = synth.impulse_response(fr.spec.T, fr.spec.sigma).astype(np.float32)
        for k, (st, off) in enumerate(pinned[i]):
            flags = B.SRT3D_CHUNK_KEEP | (B.SRT3D_LAST_CHUNK if k == 2 else 0)
            B.srt3d_submit(sctx, 400 + i, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, st, off, flags)
    for i, (fr, m, prm) in enumerate(fs):
        kept.append(poll(sctx, 400 + i, fr, prm))
    for a, b in zip(ref, kept):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_chunked_matches_one_shot_and_oracle_counts(sctx):
    fr, m, prm = frames(2)[1]
    rng = np.random.default_rng(2)
    submit_all(sctx, 1, fr, m, prm, chunks_of(fr, 8, rng))
    a = poll(sctx, 1, fr, prm)
    submit_all(sctx, 2, fr, m, prm, [(fr.stamps, fr.offsets)])
    b = poll(sctx, 2, fr, prm)
    assert np.array_equal(a[4], np.diff(fr.offsets.astype(np.int64)))
    assert np.array_equal(a[4], b[4])
    flips = np.count_nonzero(a[2] != b[2])
    assert flips <= max(1, int(1e-3 * a[2].size))
    both = (a[2] == 1) & (b[2] == 1)
    assert np.max(np.abs(a[0] - b[0])[both], initial=0.0) <= 0.05
    # the sketch state itself: chunked FP32 accumulation vs the oracle
    S_ref, n_ref = oracle.sketch_stream(fr.stamps, fr.offsets, fr.spec.T, m)
    assert np.array_equal(n_ref, a[4].astype(np.int64))


def test_admission_by_budget(sctx):
    require_gpu()
    fs = frames(3)
    fr0, m0, prm0 = fs[2]  # 32x32
    # a context whose budget holds one such frame (its device state as the
    # host plan charges it) and half of a second
    need = B.srt3d_plan(32, 32, fr0.spec.T, m0, 2, 1, 150.0, 152, 2)["serving_frame_bytes"]
    c2 = B.srt3d_create(0, int(1.5 * need))
    try:
        h = synth.impulse_response(fr0.spec.T, fr0.spec.sigma).astype(np.float32)
        B.srt3d_submit(c2, 1, 32, 32, fr0.spec.T, m0, h, prm0, fr0.stamps, fr0.offsets, 1)
        st = B.srt3d_submit(c2, 2, 32, 32, fr0.spec.T, m0, h, prm0, fr0.stamps, fr0.offsets, 1, check=False)
        assert st == B.SRT3D_EBUSY
        a = poll(c2, 1, fr0, prm0)
        B.srt3d_submit(c2, 2, 32, 32, fr0.spec.T, m0, h, prm0, fr0.stamps, fr0.offsets, 1)  # admitted now
        b = poll(c2, 2, fr0, prm0)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    finally:
        B.srt3d_destroy(c2)


def test_injected_allocation_failure_and_recovery(sctx):
    fr, m, prm = frames(1)[0]
    h = synth.impulse_response(fr.spec.T, fr.spec.sigma).astype(np.float32)
    os.environ["SRT3D_FAULT"] = "alloc"
    try:
        st = B.srt3d_submit(sctx, 7, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, fr.stamps, fr.offsets, 1,
                            check=False)
        assert st == B.SRT3D_ENOMEM
    finally:
        del os.environ["SRT3D_FAULT"]
    assert B.srt3d_poll(sctx, 7, 0, *outputs(fr, prm), check=False) == B.SRT3D_ENOTFOUND
    B.srt3d_submit(sctx, 7, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, fr.stamps, fr.offsets, 1)
    poll(sctx, 7, fr, prm)


def test_poll_states_and_errors(sctx):
    fr, m, prm = frames(1)[0]
    h = synth.impulse_response(fr.spec.T, fr.spec.sigma).astype(np.float32)
    o = outputs(fr, prm)
    assert B.srt3d_poll(sctx, 999, 0, *o, check=False) == B.SRT3D_ENOTFOUND
    B.srt3d_submit(sctx, 5, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, fr.stamps, fr.offsets, 0)
    assert B.srt3d_poll(sctx, 5, 0, *o, check=False) == B.SRT3D_EAGAIN
    # a chunk of another shape is refused; the frame stays open
    st = B.srt3d_submit(sctx, 5, fr.spec.rows, fr.spec.cols + 1, fr.spec.T, m, h, prm, fr.stamps, fr.offsets, 1,
                        check=False)
    assert st == B.SRT3D_EINVAL
    empty = np.zeros(fr.spec.num_pixels + 1, np.uint32)
    B.srt3d_submit(sctx, 5, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, np.zeros(0, np.uint16), empty, 1)
    poll(sctx, 5, fr, prm)
    # decreasing offsets are refused synchronously
    bad = fr.offsets.copy()
    bad[2] = bad[3] + 5
    st = B.srt3d_submit(sctx, 6, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, fr.stamps, bad, 1, check=False)
    assert st == B.SRT3D_EINVAL
    # a stamp >= T is reported by poll for that frame only
    st_bad = fr.stamps.copy()
    st_bad[0] = fr.spec.T
    B.srt3d_submit(sctx, 8, fr.spec.rows, fr.spec.cols, fr.spec.T, m, h, prm, st_bad, fr.offsets, 1)
    assert B.srt3d_poll(sctx, 8, 20_000_000, *outputs(fr, prm), check=False) == B.SRT3D_ERANGE
    assert B.srt3d_sync(sctx, check=False) == B.SRT3D_OK


def test_serving_matches_direct_entry_points(sctx):
    # one-shot serving == sketch_stream + finalize + reconstruct on a stream
    fr, m, prm = frames(3)[2]
    submit_all(sctx, 11, fr, m, prm, [(fr.stamps, fr.offsets)])
    a = poll(sctx, 11, fr, prm)
    P, T, K = fr.spec.num_pixels, fr.spec.T, prm.k_max
    S = torch.zeros(P, m, 2, device="cuda")
    n = torch.zeros(P, dtype=torch.int32, device="cuda")
    stamps = torch.from_numpy(fr.stamps.view(np.int16)).cuda()
    offsets = torch.from_numpy(fr.offsets.view(np.int32)).cuda()
    B.srt3d_sketch_stream(sctx, stamps, offsets, T, m, 1, S, n)
    B.srt3d_finalize(sctx, S, n, m, S)
    h = torch.from_numpy(synth.impulse_response(T, fr.spec.sigma).astype(np.float32)).cuda()
    d = torch.zeros(P, K, device="cuda")
    al = torch.zeros(P, K, device="cuda")
    act = torch.zeros(P, K, dtype=torch.uint8, device="cuda")
    a0 = torch.zeros(P, device="cuda")
    B.srt3d_reconstruct(sctx, S, n, fr.spec.rows, fr.spec.cols, T, m, h, prm, d, al, act, a0)
    B.srt3d_sync(sctx)
    assert np.array_equal(a[0], d.cpu().numpy())
    assert np.array_equal(a[1], al.cpu().numpy())
    assert np.array_equal(a[2], act.cpu().numpy())


def test_device_timeout_is_reported_by_that_frames_poll(sctx):
    # Host-side injection: the frame named by SRT3D_FAULT=gridwait:<id> runs its
    # one-launch iteration kernel with a grid-barrier target its grid never
    # reaches and a short wait limit. Every CTA gives up at the first barrier
    # and returns (no fault, no hang); the frame's own error word carries the
    # timeout to its poll. The other frames of the mix are unaffected.
    fs = frames(3)
    alone = []
    for i, (fr, m, prm) in enumerate(fs):
        submit_all(sctx, 600 + i, fr, m, prm, [(fr.stamps, fr.offsets)])
        alone.append(poll(sctx, 600 + i, fr, prm))
    os.environ["SRT3D_FAULT"] = "gridwait:701"
    try:
        for i, (fr, m, prm) in enumerate(fs):
            submit_all(sctx, 700 + i, fr, m, prm, [(fr.stamps, fr.offsets)])
    finally:
        del os.environ["SRT3D_FAULT"]
    for i, (fr, m, prm) in enumerate(fs):
        o = outputs(fr, prm)
        st = B.srt3d_poll(sctx, 700 + i, 20_000_000, *o, check=False)
        if i == 1:
            assert st == B.SRT3D_ETIMEDOUT
        else:
            assert st == B.SRT3D_OK
            for x, y in zip(alone[i], o):
                assert np.array_equal(x, y)
    # the released frame is gone, the context keeps working, nothing leaked
    # into the context's own error word
    assert B.srt3d_poll(sctx, 701, 0, *outputs(*fs[1][::2]), check=False) == B.SRT3D_ENOTFOUND
    fr, m, prm = fs[1]
    submit_all(sctx, 702, fr, m, prm, [(fr.stamps, fr.offsets)])
    for x, y in zip(alone[1], poll(sctx, 702, fr, prm)):
        assert np.array_equal(x, y)
    assert B.srt3d_sync(sctx, check=False) == B.SRT3D_OK
