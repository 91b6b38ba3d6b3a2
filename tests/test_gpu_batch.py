"""Batched uneven frames (srt3d_process_batch): one launch per stage over all
frames, captured into a CUDA graph. Each frame must match the single-frame
entry points (sketch up to the FP32 summation order, reconstruction within the
parity tolerance) and the oracle's photon counts and sketch; a replay of the
graph must reproduce the first call exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import synth

from gpu_util import counts, ctx, dev_offsets, dev_stamps, to_complex  # noqa: F401

pytestmark = pytest.mark.gpu


def uneven_specs(num, seed):
    """Scaled-down version of the uneven-frame workload: sizes, T, m, photon
    density and SBR drawn like the 64-frame batch, sizes divided by 8."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(num):
        n = int(rng.choice([8, 16, 32, 64]))
        T = int(rng.choice([1024, 4096]))
        m = int(rng.choice([4, 16]))
        nbar = float(np.exp(rng.uniform(np.log(10.0), np.log(2000.0))))
        sbr = float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))
        out.append((synth.FrameSpec(rows=n, cols=n + int(rng.integers(0, 5)), T=T, sigma=4.0 if T == 1024 else 6.0,
                                    mean_photons=nbar, sbr=sbr, two_surface_frac=0.1), m))
    return out


def alloc(spec, m, K):
    P = spec.num_pixels
    return dict(z=torch.zeros(P, m, 2, device="cuda"), n=torch.zeros(P, dtype=torch.int32, device="cuda"),
                depth=torch.zeros(P, K, device="cuda"), alpha=torch.zeros(P, K, device="cuda"),
                active=torch.zeros(P, K, dtype=torch.uint8, device="cuda"), alpha0=torch.zeros(P, device="cuda"))


def host(bufs):
    return {k: v.cpu().numpy().copy() for k, v in bufs.items()}


@pytest.mark.parametrize("K,iters,radius,num", [(2, 12, 1, 14), (1, 7, 2, 6), (3, 5, 1, 5)])
def test_batch_matches_single_frame_path(ctx, K, iters, radius, num):
    # all iterations of all frames run in one cooperative launch over the
    # frames' tiles (odd and even iteration counts, radius 1 and 2, K = 1..3)
    prm = B.make_params(iters=iters, k_max=K, radius=radius, d_max=30.0, min_sep=15.0)
    specs = uneven_specs(num, 3 + K)
    frames, keep, outs = [], [], []
    for i, (spec, m) in enumerate(specs):
        fr = synth.make_stream_frame(spec, 500 + i)
        st, off = dev_stamps(fr.stamps), dev_offsets(fr.offsets)
        h = torch.from_numpy(synth.impulse_response(spec.T, spec.sigma).astype(np.float32)).cuda()
        b = alloc(spec, m, K)
        frames.append(B.make_frame(st, off, spec.rows, spec.cols, spec.T, m, h, b["z"], b["n"], b["depth"],
                                   b["alpha"], b["active"], b["alpha0"]))
        keep.append((fr, st, off, h))
        outs.append(b)
    B.srt3d_process_batch(ctx, frames, prm)
    B.srt3d_sync(ctx)
    first = [host(b) for b in outs]
    # graph replay: identical
    for b in outs:
        for v in b.values():
            v.zero_()
    B.srt3d_process_batch(ctx, frames, prm)
    B.srt3d_sync(ctx)
    for a, b in zip(first, outs):
        for k in a:
            assert np.array_equal(a[k], b[k].cpu().numpy()), k
    # each frame against the single-frame entry points and the oracle
    flips = total = 0
    for (spec, m), (fr, st, off, h), a in zip(specs, keep, first):
        P = spec.num_pixels
        S = torch.zeros(P, m, 2, device="cuda")
        n = torch.zeros(P, dtype=torch.int32, device="cuda")
        B.srt3d_sketch_stream(ctx, st, off, spec.T, m, 0, S, n)
        B.srt3d_finalize(ctx, S, n, m, S)
        single = alloc(spec, m, K)
        B.srt3d_reconstruct(ctx, S, n, spec.rows, spec.cols, spec.T, m, h, prm, single["depth"], single["alpha"],
                            single["active"], single["alpha0"])
        B.srt3d_sync(ctx)
        n_ref = np.diff(fr.offsets.astype(np.int64))
        assert np.array_equal(a["n"].view(np.uint32).astype(np.int64), n_ref)
        z_ref = oracle.finalize(*oracle.sketch_stream(fr.stamps, fr.offsets, spec.T, m))
        za = a["z"][..., 0] + 1j * a["z"][..., 1]
        assert np.max(np.abs(za - z_ref)) <= 1e-5
        s = host(single)
        flips += np.count_nonzero(a["active"] != s["active"])
        total += a["active"].size
        both = (a["active"] == 1) & (s["active"] == 1)
        assert np.max(np.abs(a["depth"] - s["depth"])[both], initial=0.0) <= 0.05
    assert flips <= max(2, int(2e-3 * total))


def test_batch_rejects_unsupported_modes(ctx):
    spec, m = uneven_specs(1, 4)[0]
    fr = synth.make_stream_frame(spec, 1)
    h = torch.ones(spec.T, device="cuda")
    b = alloc(spec, m, 1)
    f = B.make_frame(dev_stamps(fr.stamps), dev_offsets(fr.offsets), spec.rows, spec.cols, spec.T, m, h, b["z"],
                     b["n"], b["depth"], b["alpha"], b["active"], b["alpha0"])
    for kw in (dict(init_mode=B.SRT3D_INIT_GIVEN), dict(regularize=0)):
        with pytest.raises(B.SRT3DError) as ei:
            B.srt3d_process_batch(ctx, [f], B.make_params(k_max=1, **kw))
        assert ei.value.status == B.SRT3D_EINVAL
