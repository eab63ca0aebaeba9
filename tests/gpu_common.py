"""Helpers shared by the GPU parity tests (not collected as tests)."""
import os

import numpy as np
import pytest

import oracle as O

THREADS = max(1, min(16, len(os.sched_getaffinity(0))))


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def dtype_of(prec):
    torch = torch_cuda()
    return torch.float64 if prec == "fp64" else torch.float32


def log_err(name, **vals):
    """Append measured errors to $TNN_PARITY_LOG (if set) for inspection."""
    path = os.environ.get("TNN_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(name + " " + " ".join("%s=%.3e" % (k, v) for k, v in vals.items()) + "\n")


def rel_err(y, ref, z=None):
    """||y - ref||_F / den with den = ||ref|| unless ref is (near) zero
    relative to the input z, then ||z|| (the prox is 1-Lipschitz)."""
    d = np.linalg.norm(np.asarray(y, dtype=np.float64) - ref)
    nr = np.linalg.norm(ref)
    if z is not None and nr < 1e-6 * np.linalg.norm(z):
        return d / max(np.linalg.norm(z), 1e-300)
    return d / max(nr, 1e-300)


def tau_at_quantile(Z, q):
    """Threshold at quantile q of all singular values of the transformed slices
    (oracle DCT + LAPACK singular values)."""
    Zb = O.tube_transform(Z)
    s = np.concatenate([np.linalg.svd(Zb[:, :, k], compute_uv=False) for k in range(Z.shape[2])])
    return float(np.quantile(s, q))
