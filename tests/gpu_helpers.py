"""Shared helpers of the GPU parity tests (no method arithmetic here)."""

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03804_gb300 import build, load

    build.build()
    load()
    return torch


def dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def field_maxrel(a, b, floor=0.0):
    """max over components c of max|a_c - b_c| / max|b_c| (the field tolerance measure).

    Components whose reference is identically zero are compared in absolute
    terms against ``floor`` times the largest component magnitude.
    """
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    big = np.abs(b).max()
    worst = 0.0
    for c in range(a.shape[0]):
        ref = np.abs(b[c]).max()
        err = np.abs(a[c] - b[c]).max()
        if ref > 1e-12 * big:
            worst = max(worst, err / ref)
        else:
            worst = max(worst, err / max(big, 1e-300) if floor == 0.0 else err / (floor * big))
    return worst


def pack_tangent(K):
    """(9, 9, ...) tangent to the library's packed (45, ...) upper triangle."""
    rows = []
    for a in range(9):
        for b in range(a, 9):
            rows.append(K[a, b])
    return np.stack(rows)
