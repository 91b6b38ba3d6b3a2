"""GPU parity of the tensor-core histogram sketch (tcgen05, Sec. 2 Eqs. 2-3)
against the FP64 oracle. FP16 hi+lo split: <= 1e-4 in normalised units (each
summand of Eq. 3 has modulus 1) and counts bit-exact; BF16: counts exact, the
error is reported and bounded loosely (the BF16 Fourier factors carry 8 bits)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import synth

from gpu_util import counts, csr, ctx, dev_hist, dev_offsets, dev_stamps, sketch_err, to_complex  # noqa: F401

pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-4
BF16_TOL = 2e-2


def run(ctx, y, m, precision):
    P, T = y.shape
    S = torch.full((P, m, 2), float("nan"), device="cuda")
    n = torch.zeros(P, dtype=torch.int32, device="cuda")
    B.srt3d_sketch_hist(ctx, dev_hist(y), T, m, precision, S, n)
    B.srt3d_sync(ctx)
    return S, n


@pytest.mark.parametrize("P,T,m", [(1, 64, 1), (127, 128, 4), (128, 1024, 10), (129, 64, 31), (260, 512, 16),
                                   (300, 4096, 32), (513, 4096, 10)])
def test_fp16_split_matches_oracle(ctx, P, T, m):
    rng = np.random.default_rng(P + T + m)
    y = rng.poisson(rng.uniform(0.2, 6.0, size=(P, 1)), size=(P, T)).astype(np.uint16)
    S, n = run(ctx, y, m, B.SRT3D_FP16_SPLIT)
    S_ref, n_ref = oracle.sketch_hist(y, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= SPLIT_TOL


def test_fp16_split_exact_for_counts_above_2048(ctx):
    # counts > 2048 are split exactly into (y & ~31) + (y & 31)
    P, T, m = 200, 256, 8
    rng = np.random.default_rng(9)
    y = rng.integers(0, 3, size=(P, T)).astype(np.uint16)
    y[0, 5] = 2048
    y[1, 7] = 2049
    y[2, 0] = 65535
    y[3, :] = 40000
    y[150, 200] = 3000
    S, n = run(ctx, y, m, B.SRT3D_FP16_SPLIT)
    S_ref, n_ref = oracle.sketch_hist(y, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= SPLIT_TOL


@pytest.mark.parametrize("precision,tol,values", [
    (B.SRT3D_FP16_SPLIT, SPLIT_TOL, [1, 1022, 1023, 1024, 1025, 1500, 2047, 2048, 2049, 4095, 4096, 65535]),
    (B.SRT3D_BF16, BF16_TOL, [1, 126, 127, 128, 129, 200, 255, 256]),
])
def test_conversion_paths_at_their_count_limits(ctx, precision, tol, values):
    # the converters take a bit-pattern path while every count of a thread's
    # chunk is below 1024 (FP16) / 128 (BF16) and a rounding conversion
    # otherwise; sparse pixels holding one boundary value each make a wrong
    # path choice show up at full weight
    P, T, m = 2 * len(values), 256, 8
    y = np.zeros((P, T), np.uint16)
    rng = np.random.default_rng(21)
    for i, v in enumerate(values):
        y[2 * i, int(rng.integers(0, T))] = v
        b = int(rng.integers(0, T))
        y[2 * i + 1, b] = v
        y[2 * i + 1, (b + 7) % T] = 1
    S, n = run(ctx, y, m, precision)
    S_ref, n_ref = oracle.sketch_hist(y, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= tol


@pytest.mark.parametrize("P,T,m,frac", [(1000, 4096, 32, 0.01), (300, 1024, 10, 1.0), (700, 2048, 3, 0.2)])
def test_fp16_split_counts_above_2048_in_many_stages(ctx, P, T, m, frac):
    # big counts scattered over many tiles and pipeline stages (every stage
    # when frac = 1): the A2 slot shared by the stages must carry exactly the
    # low parts of its own stage
    rng = np.random.default_rng(int(frac * 100) + T)
    y = rng.poisson(3.0, size=(P, T)).astype(np.uint16)
    big = rng.random((P, T)) < frac
    y[big] = rng.integers(2049, 65536, size=int(big.sum())).astype(np.uint16)
    S, n = run(ctx, y, m, B.SRT3D_FP16_SPLIT)
    S_ref, n_ref = oracle.sketch_hist(y, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= SPLIT_TOL


@pytest.mark.parametrize("P,T,m", [(1, 64, 1), (130, 1024, 10), (300, 4096, 32)])
def test_bf16_reported_error(ctx, P, T, m):
    rng = np.random.default_rng(P * 3 + m)
    y = rng.poisson(rng.uniform(0.2, 6.0, size=(P, 1)), size=(P, T)).astype(np.uint16)
    S, n = run(ctx, y, m, B.SRT3D_BF16)
    S_ref, n_ref = oracle.sketch_hist(y, m)
    assert np.array_equal(counts(n), n_ref)
    err = sketch_err(S, n, S_ref, n_ref)
    print(f"BF16 sketch error (normalised) P={P} T={T} m={m}: {err:.3e}")
    assert err <= BF16_TOL


def test_tc_argument_checks(ctx):
    y = np.zeros((4, 100), np.uint16)  # T not a multiple of 64
    S = torch.zeros(4, 4, 2, device="cuda")
    n = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(B.SRT3DError) as ei:
        B.srt3d_sketch_hist(ctx, dev_hist(y), 100, 4, B.SRT3D_FP16_SPLIT, S, n)
    assert ei.value.status == B.SRT3D_EINVAL


def test_full_size_512x512_histograms_sampled(ctx):
    # The histogram workload at full size (512x512 x 4096 bins, 10 000
    # counts/pixel, SBR 0.2, m = 32): every precision on the whole frame, the
    # oracle on a sample of pixels.
    spec = synth.frame_512x512_hist()
    m = 32
    hist, _ = synth.make_hist_frame_torch(spec, synth.SEED_512x512)
    P, T = spec.num_pixels, spec.T
    rng = np.random.default_rng(12)
    pix = np.unique(np.concatenate([rng.choice(P, 96, replace=False), [0, P - 1]]))
    y_s = hist[torch.from_numpy(pix).cuda()].cpu().numpy().view(np.uint16)
    S_ref, n_ref = oracle.sketch_hist(y_s, m)
    for prec, tol in ((B.SRT3D_FP32, 1e-5), (B.SRT3D_FP16_SPLIT, SPLIT_TOL), (B.SRT3D_BF16, BF16_TOL)):
        S = torch.empty(P, m, 2, device="cuda")
        n = torch.empty(P, dtype=torch.int32, device="cuda")
        B.srt3d_sketch_hist(ctx, hist, T, m, prec, S, n)
        B.srt3d_sync(ctx)
        Sg = to_complex(S)[pix]
        assert np.array_equal(counts(n)[pix], n_ref)
        err = np.max(np.abs(Sg - S_ref) / n_ref[:, None])
        print(f"precision {prec}: max normalised error {err:.3e}")
        assert err <= tol
        del S, n
    del hist
    torch.cuda.empty_cache()



@pytest.mark.parametrize("T,m,sizes", [(4096, 10, [1000, 0, 37, 5000, 3]), (1024, 32, [300, 301, 1, 0]),
                                       (64, 3, [0, 12, 7])])
def test_stream_sketch_through_tensor_cores(ctx, T, m, sizes):
    # srt3d_sketch_stream_tc: device histogram of the stamp stream, then the
    # tensor-core sketch; equals the oracle's stream sketch (FP16 split within
    # 1e-5 normalised, counts exact)
    rng = np.random.default_rng(T + m)
    stamps, offsets = csr([rng.integers(0, T, size=c) for c in sizes])
    P = len(sizes)
    S = torch.zeros(P, m, 2, device="cuda")
    n = torch.zeros(P, dtype=torch.int32, device="cuda")
    sd = dev_stamps(stamps) if stamps.size else torch.zeros(8, dtype=torch.int16, device="cuda")[:0]
    off = dev_offsets(offsets)
    B.srt3d_sketch_stream_tc(ctx, sd, off, T, m, B.SRT3D_FP16_SPLIT, S, n)
    B.srt3d_sync(ctx)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
    assert np.array_equal(counts(n), n_ref)
    assert sketch_err(S, n, S_ref, n_ref) <= 1e-5
    with pytest.raises(B.SRT3DError):
        B.srt3d_sketch_stream_tc(ctx, sd, off, 100, m, B.SRT3D_FP16_SPLIT, S, n)


# ----------------------------------------------------------------- fused stream route
def both_stream_routes(ctx, stamps, offsets, T, m, precision=B.SRT3D_FP16_SPLIT, check=True):
    """S, n of srt3d_sketch_stream_tc (histogram through HBM) and of
    srt3d_sketch_stream_tc_fused (histogram stages built in shared memory);
    outputs start as NaN / -1 so that nothing unwritten passes."""
    P = len(offsets) - 1
    sd = dev_stamps(stamps) if stamps.size else torch.zeros(8, dtype=torch.int16, device="cuda")[:0]
    off = dev_offsets(offsets)
    out, status = [], []
    for fn in (B.srt3d_sketch_stream_tc, B.srt3d_sketch_stream_tc_fused):
        S = torch.full((P, m, 2), float("nan"), device="cuda")
        n = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        fn(ctx, sd, off, T, m, precision, S, n)
        status.append(B.srt3d_sync(ctx, check=check))
        out.append((S, n))
    return out, status


def _per_pixel(rng, T, sizes):
    return [rng.integers(0, T, size=c) for c in sizes]


@pytest.mark.parametrize("T,m,sizes", [
    (4096, 10, [1000, 0, 37, 5000, 3]),
    (1024, 32, [300, 301, 1, 0]),
    (64, 3, [0, 12, 7]),
    (4096, 10, "ragged300"),     # three tiles, the last one 44 pixels
    (2048, 16, "chunks"),        # a tile of 45 K stamps: several sort chunks, one pixel spanning three
    (65536, 4, "ragged130"),     # 1024 stages per tile
    (4096, 1, "empty"),          # no stamps at all
])
def test_fused_stream_route_equals_composed_and_oracle(ctx, T, m, sizes):
    # the same integer bin counts enter the same tensor-core products, so S
    # and n equal the composed route's bit for bit; both equal the oracle's
    # stream sketch within the split-FP16 bound (Sec. 2, Eq. 3)
    rng = np.random.default_rng(T + m + 7)
    if sizes == "ragged300":
        per = _per_pixel(rng, T, rng.integers(0, 400, size=300))
    elif sizes == "chunks":
        per = _per_pixel(rng, T, [200] * 127 + [20000])
    elif sizes == "ragged130":
        per = _per_pixel(rng, T, rng.integers(0, 2000, size=130))
    elif sizes == "empty":
        per = [np.zeros(0, np.int64)] * 5
    else:
        per = _per_pixel(rng, T, sizes)
    stamps, offsets = csr(per)
    ((S1, n1), (S2, n2)), _ = both_stream_routes(ctx, stamps, offsets, T, m)
    assert torch.equal(n1, n2)
    assert torch.equal(S1, S2)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
    assert np.array_equal(counts(n2), n_ref)
    assert sketch_err(S2, n2, S_ref, n_ref) <= 1e-5


def test_fused_stream_route_big_bin_counts(ctx):
    # bins above 2048 counts take the exact split A = y & ~31, A2 = y & 31
    T, m = 1024, 12
    rng = np.random.default_rng(3)
    per = [np.full(3000, 17), np.full(2049, 0), rng.integers(0, T, 500),
           np.concatenate([np.full(4100, 1023), rng.integers(0, T, 100)])] + _per_pixel(rng, T, [50] * 200)
    stamps, offsets = csr(per)
    ((S1, n1), (S2, n2)), _ = both_stream_routes(ctx, stamps, offsets, T, m)
    assert torch.equal(n1, n2) and torch.equal(S1, S2)
    S_ref, n_ref = oracle.sketch_stream(stamps, offsets, T, m)
    assert sketch_err(S2, n2, S_ref, n_ref) <= 1e-5


@pytest.mark.parametrize("most", [1500, 60])
def test_fused_stream_route_bf16_equals_composed(ctx, most):
    # dense pixels: stages above 256 entries count in u16 and convert; sparse
    # ones add in BF16 directly
    T, m = 4096, 10
    rng = np.random.default_rng(11 + most)
    per = _per_pixel(rng, T, rng.integers(0, most, size=257))
    stamps, offsets = csr(per)
    ((S1, n1), (S2, n2)), _ = both_stream_routes(ctx, stamps, offsets, T, m, B.SRT3D_BF16)
    assert torch.equal(n1, n2) and torch.equal(S1, S2)


def test_fused_stream_route_error_cases(ctx):
    T, m = 256, 4
    rng = np.random.default_rng(5)
    # a stamp >= T is skipped by both routes and reported
    per = _per_pixel(rng, T, [100, 30, 7])
    per[1] = np.concatenate([per[1], [T, T + 5]])
    stamps, offsets = csr(per)
    ((S1, n1), (S2, n2)), st = both_stream_routes(ctx, stamps, offsets, T, m, check=False)
    assert st == [B.SRT3D_ERANGE, B.SRT3D_ERANGE]
    assert torch.equal(n1, n2) and torch.equal(S1, S2)
    # more than 65535 stamps in a pixel: the fused route counts the first
    # 65535 (the composed route saturates each bin instead); both report it
    per = [rng.integers(0, T, 70000), rng.integers(0, T, 10)]
    stamps, offsets = csr(per)
    (_, (S2, n2)), st = both_stream_routes(ctx, stamps, offsets, T, m, check=False)
    assert st[1] == B.SRT3D_ERANGE
    cut, cut_off = csr([per[0][:65535], per[1]])
    S_ref, n_ref = oracle.sketch_stream(cut, cut_off, T, m)
    assert np.array_equal(counts(n2), n_ref)
    assert sketch_err(S2, n2, S_ref, n_ref) <= 1e-5
    # decreasing offsets: the pixel is left empty and reported
    stamps = np.arange(10, dtype=np.uint16)
    offsets = np.array([0, 6, 4, 10], dtype=np.uint32)
    (_, (S2, n2)), st = both_stream_routes(ctx, stamps, offsets, 64, m, check=False)
    assert st[1] == B.SRT3D_EOFFSETS
    assert counts(n2)[1] == 0
    with pytest.raises(B.SRT3DError):
        B.srt3d_sketch_stream_tc_fused(ctx, dev_stamps(stamps), dev_offsets(offsets), 100, m, B.SRT3D_FP16_SPLIT,
                                       torch.zeros(3, m, 2, device="cuda"),
                                       torch.zeros(3, dtype=torch.int32, device="cuda"))
