"""Helpers shared by the GPU tests (tensor layout only; no solver arithmetic)."""
import numpy as np


def to_cols(x: np.ndarray, ld_pad: int = 0):
    """numpy (N,) or (N, r) -> CUDA float64 tensor (N, r) column major with leading dimension N + ld_pad."""
    import torch

    x2 = x[:, None] if x.ndim == 1 else x
    N, r = x2.shape
    buf = torch.zeros((r, N + ld_pad), dtype=torch.float64, device="cuda")
    buf[:, :N] = torch.from_numpy(np.ascontiguousarray(x2.T)).cuda()
    return buf.T[:N] if ld_pad == 0 else buf.T[:N, :]


def from_cols(t) -> np.ndarray:
    return t.detach().cpu().numpy()


def empty_like_cols(t):
    import torch

    r = t.shape[1]
    ld = t.stride(1)
    buf = torch.zeros((r, ld), dtype=torch.float64, device="cuda")
    return buf.T[: t.shape[0], :]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
