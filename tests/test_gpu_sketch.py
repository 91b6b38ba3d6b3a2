"""GPU parity of the stream path against the FP64 oracle: photon counts and
histograms bit-exact, sketches within 1e-5 in normalised units (Eq. 3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import synth

from gpu_util import (ctx, counts, csr, dev_hist, dev_offsets, dev_stamps, gpu_sketch_stream,  # noqa: F401
                      sketch_err, to_complex)

pytestmark = pytest.mark.gpu
TOL = 1e-5


def test_sketch_32x32_frame(ctx):
    spec = synth.frame_32x32()
    fr = synth.make_stream_frame(spec, synth.SEED_32x32)
    for m in (4, 10, 32):
        S, n = gpu_sketch_stream(ctx, fr.stamps, fr.offsets, spec.T, m)
        B.srt3d_sync(ctx)
        S_ref, n_ref = oracle.sketch_stream(fr.stamps, fr.offsets, spec.T, m)
        assert np.array_equal(counts(n), n_ref)
        assert sketch_err(S, n, S_ref, n_ref) <= TOL


@pytest.mark.parametrize("T,m,sizes", [
    (2, 1, [1, 0, 3]),
    (7, 6, [0, 0, 1, 2, 9, 0]),
    (1024, 4, [1]),
    (4613, 17, [0, 5, 3000, 1, 77, 0, 256, 255, 257]),
    (4096, 10, [5000, 0, 12, 800]),
    (8192, 16, [100, 2000, 7]),
    (8193, 12, [64, 0, 999]),
    (65536, 32, [1, 4000, 33, 0, 10000]),
])
def test_sketch_edge_cases(ctx, T, m, sizes):
    rng = np.random.default_rng(T + m)
    per = [rng.integers(0, T, size=c) for c in sizes]
    if T == 65536:
        per[1][:4] = [0, 65535, 32768, 1]
    stamps, offsets = csr(per)
    S, n = gpu_sketch_stream(ctx, stamps, offsets, T, m)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= TOL


@pytest.mark.parametrize("T,m,bound", [(4096, 10, 4e-6), (4613, 10, 4e-6), (1024, 32, 2.5e-6), (65535, 32, 2.5e-6)])
def test_sketch_every_phase_single_photon(ctx, T, m, bound):
    """One photon per pixel, every x in [0, T) once: S[x][l-1] is the single
    term e^{i 2 pi l x / T} of Eq. 3, so this bounds the per-term rounding of
    the recurrence between table restarts over all phases."""
    stamps = np.arange(T, dtype=np.uint16)
    offsets = np.arange(T + 1, dtype=np.uint32)
    S, n = gpu_sketch_stream(ctx, stamps, offsets, T, m)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
    assert np.array_equal(counts(n), n_ref)
    assert np.max(np.abs(to_complex(S) - S_ref)) <= bound


@pytest.mark.parametrize("T,m", [(4096, 1), (4613, 2), (1024, 3), (4096, 4), (8192, 4)])
def test_sketch_every_phase_in_whole_words(ctx, T, m):
    """Pixels of 8 equal stamps x in one aligned 16-byte word, every x in
    [0, T): the whole-word path, where at few harmonics part of each word's
    phasors come from the SFU instead of the table. S[x] / 8 is the single
    term e^{i 2 pi l x / T} of Eq. 3 up to the per-term rounding."""
    stamps = np.repeat(np.arange(T, dtype=np.uint16), 8)
    offsets = (8 * np.arange(T + 1)).astype(np.uint32)
    S, n = gpu_sketch_stream(ctx, stamps, offsets, T, m)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
    assert np.array_equal(counts(n), n_ref)
    assert np.max(np.abs(to_complex(S) - S_ref)) / 8 <= 2e-6


def test_sketch_unaligned_stream_base(ctx):
    rng = np.random.default_rng(5)
    T, m = 4096, 10
    per = [rng.integers(0, T, size=c) for c in (300, 0, 17, 1000, 3)]
    stamps, offsets = csr(per)
    for shift in range(1, 8):
        padded = np.concatenate([np.zeros(shift, np.uint16), stamps])
        dev = dev_stamps(padded)[shift:]
        assert dev.data_ptr() % 16 != 0
        S, n = gpu_sketch_stream(ctx, stamps, offsets, T, m, stamps_dev=dev)
        B.srt3d_sync(ctx)
        S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
        assert np.array_equal(counts(n), n_ref)
        assert sketch_err(S, n, S_ref, n_ref) <= TOL


def test_sketch_online_chunks_accumulate(ctx):
    # Sec. 2 online update: two chunks accumulated == one-shot sketch.
    rng = np.random.default_rng(6)
    T, m = 2048, 16
    per = [rng.integers(0, T, size=c) for c in (500, 0, 33, 2500, 1)]
    cut = [rng.integers(0, len(s) + 1) for s in per]
    S = torch.zeros(len(per), m, 2, device="cuda")
    n = torch.zeros(len(per), dtype=torch.int32, device="cuda")
    for part in ([s[:c] for s, c in zip(per, cut)], [s[c:] for s, c in zip(per, cut)]):
        st, off = csr(part)
        B.srt3d_sketch_stream(ctx, dev_stamps(st), dev_offsets(off), T, m, 1, S, n)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(*csr(per), T, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= TOL


@pytest.mark.parametrize("T,m", [(4096, 1), (4096, 10), (1024, 32), (65536, 7)])
def test_sketch_normalised_mode_equals_finalize(ctx, T, m):
    """accumulate = 2 stores z = S / n directly: bit for bit what
    srt3d_finalize gives after an overwriting sketch (empty pixels: 0)."""
    rng = np.random.default_rng(70 + m)
    per = [rng.integers(0, T, size=int(c)) for c in rng.integers(0, 1500, size=50)]
    per[3] = per[3][:0]
    st, off = csr(per)
    P = len(per)
    S = torch.empty(P, m, 2, device="cuda")
    n = torch.empty(P, dtype=torch.int32, device="cuda")
    z = torch.empty(P, m, 2, device="cuda")
    B.srt3d_sketch_stream(ctx, dev_stamps(st), dev_offsets(off), T, m, 0, S, n)
    B.srt3d_finalize(ctx, S, n, m, z)
    z2 = torch.full((P, m, 2), float("nan"), device="cuda")
    n2 = torch.zeros(P, dtype=torch.int32, device="cuda")
    B.srt3d_sketch_stream(ctx, dev_stamps(st), dev_offsets(off), T, m, 2, z2, n2)
    B.srt3d_sync(ctx)
    assert torch.equal(n, n2)
    assert torch.equal(z, z2)


def test_sketch_full_256x256_sampled(ctx):
    # The benchmark's workload at full size; the oracle recomputes a sample of pixels.
    spec = synth.frame_256x256()
    fr = synth.make_stream_frame(spec, synth.SEED_256x256)
    m = 10
    S, n = gpu_sketch_stream(ctx, fr.stamps, fr.offsets, spec.T, m)
    B.srt3d_sync(ctx)
    rng = np.random.default_rng(7)
    pix = np.unique(np.concatenate([rng.choice(spec.num_pixels, 300, replace=False), [0, spec.num_pixels - 1]]))
    per = [fr.stamps[fr.offsets[p]:fr.offsets[p + 1]] for p in pix]
    S_ref, n_ref = oracle.sketch_stream(*csr(per), spec.T, m)
    assert np.array_equal(counts(n)[pix], n_ref)
    assert np.array_equal(counts(n), np.diff(fr.offsets.astype(np.int64)))
    Sg = to_complex(S)[pix]
    assert np.max(np.abs(Sg - S_ref) / np.maximum(n_ref, 1)[:, None]) <= TOL


def test_stamp_out_of_range_is_flagged(ctx):
    stamps, offsets = csr([[1, 2, 3], [5, 16, 7], [0]])
    S, n = gpu_sketch_stream(ctx, stamps, offsets, 16, 3)
    st = B.srt3d_sync(ctx, check=False)
    assert st == B.SRT3D_ERANGE
    S_ref, n_ref = oracle.sketch_stream(*csr([[1, 2, 3], [0]]), 16, 3)
    got = to_complex(S)[[0, 2]]
    assert np.max(np.abs(got - S_ref)) < 1e-5
    assert B.srt3d_sync(ctx, check=False) == B.SRT3D_OK  # flag cleared


def test_malformed_offsets_are_flagged(ctx):
    stamps = np.arange(10, dtype=np.uint16)
    offsets = np.array([0, 6, 4, 10], dtype=np.uint32)
    gpu_sketch_stream(ctx, stamps, offsets, 16, 2)
    assert B.srt3d_sync(ctx, check=False) == B.SRT3D_EOFFSETS
    offsets = np.array([0, 4, 11], dtype=np.uint32)  # beyond num_stamps
    gpu_sketch_stream(ctx, stamps, offsets, 16, 2)
    assert B.srt3d_sync(ctx, check=False) == B.SRT3D_EOFFSETS


def test_invalid_arguments_rejected_synchronously(ctx):
    stamps, offsets = csr([[1]])
    S = torch.zeros(1, 4, 2, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    for T, m in ((0, 4), (65537, 4), (16, 0), (16, 33)):
        with pytest.raises(B.SRT3DError) as ei:
            B.srt3d_sketch_stream(ctx, dev_stamps(stamps), dev_offsets(offsets), T, m, 0, S, n)
        assert ei.value.status == B.SRT3D_EINVAL


@pytest.mark.parametrize("T,sizes", [(1024, [0, 1, 100, 3000]), (4613, [5, 0, 2000]), (65536, [1000, 3, 0]),
                                     (16385, [300, 300]), (5000, [70000, 100]), (4096, [70000, 0, 5]),
                                     (8, [65535, 65536, 1])])
def test_hist_from_stream_bit_exact(ctx, T, sizes):
    rng = np.random.default_rng(T)
    per = [rng.integers(0, T, size=c) for c in sizes]
    per[0] = np.concatenate([per[0], np.full(7, T - 1)]).astype(np.int64)
    stamps, offsets = csr(per)
    hist = torch.empty(len(per), T, dtype=torch.int16, device="cuda")
    B.srt3d_hist_from_stream(ctx, dev_stamps(stamps), dev_offsets(offsets), T, hist)
    B.srt3d_sync(ctx)
    ref = oracle.hist_from_stream(stamps, offsets, T)
    assert np.array_equal(hist.cpu().numpy().view(np.uint16), ref)


def test_hist_from_stream_unaligned_output_bit_exact(ctx):
    # an output row start that is only 2-byte aligned takes the scalar stores
    T = 1024
    rng = np.random.default_rng(11)
    stamps, offsets = csr([rng.integers(0, T, size=c) for c in (500, 0, 77)])
    buf = torch.zeros(3 * T + 1, dtype=torch.int16, device="cuda")
    B.srt3d_hist_from_stream(ctx, dev_stamps(stamps), dev_offsets(offsets), T, buf[1:])
    B.srt3d_sync(ctx)
    assert int(buf[0].item()) == 0
    assert np.array_equal(buf[1:].cpu().numpy().view(np.uint16).reshape(3, T),
                          oracle.hist_from_stream(stamps, offsets, T))


def test_hist_from_stream_32x32_frame_bit_exact(ctx):
    spec = synth.frame_32x32()
    fr = synth.make_stream_frame(spec, synth.SEED_32x32)
    hist = torch.empty(spec.num_pixels, spec.T, dtype=torch.int16, device="cuda")
    B.srt3d_hist_from_stream(ctx, dev_stamps(fr.stamps), dev_offsets(fr.offsets), spec.T, hist)
    B.srt3d_sync(ctx)
    assert np.array_equal(hist.cpu().numpy().view(np.uint16), oracle.hist_from_stream(fr.stamps, fr.offsets, spec.T))


def test_hist_count_overflow_saturates_and_flags(ctx):
    stamps, offsets = csr([np.full(70000, 3), [1]])
    hist = torch.empty(2, 8, dtype=torch.int16, device="cuda")
    B.srt3d_hist_from_stream(ctx, dev_stamps(stamps), dev_offsets(offsets), 8, hist)
    assert B.srt3d_sync(ctx, check=False) == B.SRT3D_ERANGE
    h = hist.cpu().numpy().view(np.uint16)
    assert h[0, 3] == 65535 and h[1, 1] == 1 and h[0].sum() == 65535


def test_finalize_matches_definition(ctx):
    rng = np.random.default_rng(8)
    T, m = 512, 7
    per = [rng.integers(0, T, size=c) for c in (0, 1, 50, 999)]
    stamps, offsets = csr(per)
    S, n = gpu_sketch_stream(ctx, stamps, offsets, T, m)
    z = torch.empty_like(S)
    B.srt3d_finalize(ctx, S, n, m, z)
    B.srt3d_sync(ctx)
    z_ref = oracle.finalize(*oracle.sketch_stream(stamps, offsets, T, m))
    zg = to_complex(z)
    assert np.all(zg[0] == 0)
    assert np.max(np.abs(zg - z_ref)) <= TOL


@pytest.mark.parametrize("P,T,m", [(1, 64, 1), (70, 1024, 4), (129, 4096, 10), (65, 4613, 17), (33, 100, 32)])
def test_hist_sketch_fp32(ctx, P, T, m):
    rng = np.random.default_rng(P * T + m)
    y = rng.poisson(rng.uniform(0.1, 5.0, size=(P, 1)), size=(P, T)).astype(np.uint16)
    y[0, :3] = [60000, 0, 65535]
    S = torch.empty(P, m, 2, device="cuda")
    n = torch.empty(P, dtype=torch.int32, device="cuda")
    B.srt3d_sketch_hist(ctx, dev_hist(y), T, m, B.SRT3D_FP32, S, n)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_hist(y, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= TOL


def test_hist_sketch_fp32_of_stream_histogram_equals_stream_sketch(ctx):
    spec = synth.frame_32x32()
    fr = synth.make_stream_frame(spec, synth.SEED_32x32)
    m = 8
    hist = torch.empty(spec.num_pixels, spec.T, dtype=torch.int16, device="cuda")
    B.srt3d_hist_from_stream(ctx, dev_stamps(fr.stamps), dev_offsets(fr.offsets), spec.T, hist)
    S = torch.empty(spec.num_pixels, m, 2, device="cuda")
    n = torch.empty(spec.num_pixels, dtype=torch.int32, device="cuda")
    B.srt3d_sketch_hist(ctx, hist, spec.T, m, B.SRT3D_FP32, S, n)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(fr.stamps, fr.offsets, spec.T, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= TOL


def test_bounded_device_wait_reports_timeout_and_context_stays_usable(ctx):
    # a grid-barrier wait that can never complete gives up after ~1 ms of SM
    # cycles, latches the device timeout flag and returns; the context keeps
    # working afterwards
    B.srt3d_selftest_wait_timeout(ctx, 2_000_000)
    assert B.srt3d_sync(ctx, check=False) == B.SRT3D_ETIMEDOUT
    assert B.srt3d_sync(ctx, check=False) == B.SRT3D_OK  # the flag was cleared
    rng = np.random.default_rng(8)
    per = [rng.integers(0, 1024, size=c) for c in (5, 300, 0, 17)]
    stamps, offsets = csr(per)
    S, n = gpu_sketch_stream(ctx, stamps, offsets, 1024, 6)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, 1024, 6)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= TOL
    with pytest.raises(B.SRT3DError):
        B.srt3d_selftest_wait_timeout(ctx, 0)
