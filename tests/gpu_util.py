"""Helpers for the GPU parity tests: host<->device marshalling of CSR frames
and sketches. No arithmetic of the method lives here."""
import numpy as np
import pytest
import torch

from paper_2203_00952_gb300 import binding as B


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def dev_stamps(stamps: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(stamps, dtype=np.uint16).view(np.int16)).cuda()


def dev_offsets(offsets: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.uint32).view(np.int32)).cuda()


def dev_hist(hist: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(hist, dtype=np.uint16).view(np.int16)).cuda()


def to_complex(t: torch.Tensor) -> np.ndarray:
    a = t.detach().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def counts(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32).astype(np.int64)


def csr(per_pixel):
    stamps = (np.concatenate([np.asarray(s, dtype=np.uint16) for s in per_pixel])
              if len(per_pixel) else np.zeros(0, np.uint16))
    offsets = np.zeros(len(per_pixel) + 1, dtype=np.uint32)
    offsets[1:] = np.cumsum([len(s) for s in per_pixel])
    return stamps, offsets


def gpu_sketch_stream(ctx, stamps, offsets, T, m, stamps_dev=None):
    P = len(offsets) - 1
    S = torch.zeros(P, m, 2, device="cuda")
    n = torch.zeros(P, dtype=torch.int32, device="cuda")
    sd = dev_stamps(stamps) if stamps_dev is None else stamps_dev
    if sd.numel() == 0:
        sd = torch.zeros(8, dtype=torch.int16, device="cuda")[:0]
    B.srt3d_sketch_stream(ctx, sd, dev_offsets(offsets), T, m, 0, S, n)
    return S, n


def sketch_err(S_gpu, n_gpu, S_ref, n_ref):
    """Max over entries of |S_gpu - S_ref| / max(n, 1): the error of z in
    normalised units (each summand of Eq. 3 has modulus 1)."""
    Sg = to_complex(S_gpu)
    nn = np.maximum(np.asarray(n_ref, dtype=np.float64), 1.0)[:, None]
    return float(np.max(np.abs(Sg - S_ref) / nn)) if Sg.size else 0.0


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2203_00952_gb300 import build as builder

    builder.build()
    c = B.srt3d_create(0)
    yield c
    B.srt3d_destroy(c)
