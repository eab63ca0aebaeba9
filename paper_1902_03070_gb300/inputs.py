"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and assembles them with plain array
operations (rescaling, adding a drift and noise, clipping, smoothing).  It
holds none of the method's arithmetic: wherever a workload needs a DCT
t-product of random factors (a low-tubal-rank core), the caller passes the
t-product routine in, so the CPU oracle and the CUDA library each build the
core with their own code.

Arrays follow the paper's MATLAB layout: shape (n1, n2, n3), Fortran order.

Workloads (seeds: data stream 190203070 + c, mask stream 190203070 + c + 1000):
  1  48x48x16, tubal rank 3, factors i.i.d. N(0,1), 40% observed
  2  144x176x100 video-shaped: rank-10 t-product of U[0,1) factors, min-max
     rescaled to [0,1], plus a per-pixel sinusoid over frames (period 50,
     amplitude U[0,0.05], phase U[0,2pi)), plus N(0, 0.01^2) noise, clipped
     to [0,1]; 20% observed (stands in for the Akiyo/Suzie/Salesman videos)
  3  512x512x31 multispectral-shaped: 5 Gaussian spectral signatures
     (centre U[0,30], width U[2,6]) times smoothed U[0,1) abundance maps
     (Gaussian, sigma 8 px) normalised to sum 1; 10% observed (stands in for
     the CAVE images)
  4  64 tensors, n1, n2 ~ U{32..256}, n3 ~ U{8..64}, rank r ~ U{2..12},
     normal factors of variance r^-1/2 (so each slice product has unit-variance
     entries), plus N(0, 1e-3^2) noise
The observed set is exactly round(p N) positions drawn by a seeded permutation.
"""
import numpy as np

SEED_BASE = 190203070


def rng_data(cfg: int, seed_offset: int = 0):
    return np.random.default_rng(SEED_BASE + cfg + seed_offset)


def rng_mask(cfg: int, seed_offset: int = 0):
    return np.random.default_rng(SEED_BASE + cfg + 1000 + seed_offset)


def uniform_mask(shape, frac, rng):
    """uint8 mask (Fortran order) with exactly round(frac * N) ones at
    positions drawn by a permutation."""
    N = int(np.prod(shape))
    cnt = int(round(frac * N))
    flat = np.zeros(N, dtype=np.uint8)
    flat[rng.permutation(N)[:cnt]] = 1
    return np.asfortranarray(flat.reshape(shape, order="F"))


def fortran(a, dtype=np.float64):
    return np.asfortranarray(np.asarray(a, dtype=dtype))


def lowrank_factors(n1, n2, n3, r, rng, dist="normal", scale=1.0):
    """Two factor tensors (n1 x r x n3) and (r x n2 x n3)."""
    if dist == "normal":
        A = rng.standard_normal((n1, r, n3)) * scale
        F = rng.standard_normal((r, n2, n3)) * scale
    elif dist == "uniform":
        A = rng.random((n1, r, n3)) * scale
        F = rng.random((r, n2, n3)) * scale
    else:
        raise ValueError(dist)
    return fortran(A), fortran(F)


def config1(tprod, seed_offset=0):
    """Returns dict with T (ground truth), B (zero off the mask), mask."""
    rng = rng_data(1, seed_offset)
    A, F = lowrank_factors(48, 48, 16, 3, rng)
    T = fortran(tprod(A, F))
    mask = uniform_mask(T.shape, 0.4, rng_mask(1, seed_offset))
    return {"T": T, "B": fortran(T * mask), "mask": mask,
            "admm": dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=300)}


def config2_parts(n1=144, n2=176, n3=100, rank=10, seed_offset=0):
    rng = rng_data(2, seed_offset)
    A, F = lowrank_factors(n1, n2, n3, rank, rng, dist="uniform")
    amp = rng.uniform(0.0, 0.05, size=(n1, n2))
    phase = rng.uniform(0.0, 2 * np.pi, size=(n1, n2))
    noise = rng.standard_normal((n1, n2, n3)) * 0.01
    return {"A": A, "F": F, "amp": amp, "phase": phase, "noise": noise}


def config2_assemble(core, parts):
    """Rescale the low-rank core to [0,1], add the per-pixel drift of period 50
    frames and the noise, clip to [0,1]."""
    core = np.asarray(core, dtype=np.float64)
    lo, hi = core.min(), core.max()
    X = (core - lo) / (hi - lo if hi > lo else 1.0)
    t = np.arange(core.shape[2], dtype=np.float64)
    X = X + parts["amp"][:, :, None] * np.sin(2 * np.pi * t[None, None, :] / 50.0 + parts["phase"][:, :, None])
    X = X + parts["noise"]
    return fortran(np.clip(X, 0.0, 1.0))


def config2(tprod, n1=144, n2=176, n3=100, seed_offset=0):
    parts = config2_parts(n1, n2, n3, seed_offset=seed_offset)
    T = config2_assemble(tprod(parts["A"], parts["F"]), parts)
    mask = uniform_mask(T.shape, 0.2, rng_mask(2, seed_offset))
    return {"T": T, "B": fortran(T * mask), "mask": mask,
            "admm": dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=200)}


def config3(n1=512, n2=512, n3=31, n_end=5, seed_offset=0):
    from scipy.ndimage import gaussian_filter
    rng = rng_data(3, seed_offset)
    mu = rng.uniform(0.0, 30.0, size=n_end)
    wd = rng.uniform(2.0, 6.0, size=n_end)
    k = np.arange(n3, dtype=np.float64)
    sig = np.exp(-((k[None, :] - mu[:, None]) ** 2) / (2 * wd[:, None] ** 2))  # n_end x n3
    ab = np.stack([gaussian_filter(rng.random((n1, n2)), sigma=8.0, mode="reflect") for _ in range(n_end)])
    ab = ab / ab.sum(axis=0, keepdims=True)
    T = fortran(np.einsum("eij,ek->ijk", ab, sig))
    mask = uniform_mask(T.shape, 0.1, rng_mask(3, seed_offset))
    return {"T": T, "B": fortran(T * mask), "mask": mask,
            "admm": dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=150)}


def config4_shapes(count=64, seed_offset=0):
    rng = rng_data(4, seed_offset)
    out = []
    for _ in range(count):
        n1 = int(rng.integers(32, 257))
        n2 = int(rng.integers(32, 257))
        n3 = int(rng.integers(8, 65))
        r = int(rng.integers(2, 13))
        out.append((n1, n2, n3, r))
    return out


def config4(tprod, count=64, seed_offset=0):
    rng = rng_data(4, 100 + seed_offset)
    tensors = []
    for (n1, n2, n3, r) in config4_shapes(count, seed_offset):
        A, F = lowrank_factors(n1, n2, n3, r, rng, scale=1.0 / np.sqrt(np.sqrt(r)))
        T = np.asarray(tprod(A, F)) + rng.standard_normal((n1, n2, n3)) * 1e-3
        tensors.append(fortran(T))
    return tensors


def config4_tau(n1, n2, noise=1e-3, factor=2.0):
    """Per-tensor threshold of the batched workload: `factor` times the edge
    sqrt(n1) + sqrt(n2) of the singular values of an n1 x n2 slice of i.i.d.
    N(0, noise^2) entries (the orthonormal DCT along tubes keeps the noise
    i.i.d.), so the t-SVT removes the noise and keeps the low-rank part."""
    return float(factor * noise * (np.sqrt(n1) + np.sqrt(n2)))


def random_tensor(shape, rng, dist="normal"):
    if dist == "normal":
        return fortran(rng.standard_normal(shape))
    if dist == "uniform":
        return fortran(rng.random(shape))
    raise ValueError(dist)
