"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws and assembles input tensors; it contains none of the
TT-UTV arithmetic (no factorization, no truncation, no sweep).  Every tensor is
built in FP64 on the host with numpy's PCG64 generator and rounded once to the
requested dtype, so the CUDA path and the oracle decompose exactly the same
values.

Workloads (the structure classes of the paper's experiments, Sec. 4):

* ``gaussian_tt``: Example 1 of Sec. 4.1 -- a signal tensor P contracted from
  i.i.d. N(0,1) TT cores of prescribed ranks, plus Gaussian noise beta*N scaled
  so that ||beta N||_F = rho ||P||_F exactly.
* ``hilbert3``: a smooth function tensor 1/(i+j+k+1) (0-based), the same class
  as Example 2 of Sec. 4.1.
* ``example2``: Example 2 of Sec. 4.1 itself, B(i) = sin(sqrt(sum_k ((i_k-1)/(I-1))^2)),
  1-based indices.
* ``blobs_volume`` / ``observation_mask``: a synthetic MRI-like volume (sum of
  anisotropic Gaussian blobs) and a uniform random observation mask, standing in
  for the BrainWeb volume of the completion experiment (Sec. 4.2.2), which is
  not available here.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_cores", "contract_cores", "gaussian_tt", "hilbert3", "example2",
    "blobs_volume", "observation_mask", "random_indices", "CONFIGS", "make_config",
]


def gaussian_cores(dims, ranks, seed):
    """I.i.d. N(0,1) cores G_k of shape (r_{k-1}, I_k, r_k); ranks includes r_0 = r_d = 1."""
    rng = np.random.default_rng(seed)
    d = len(dims)
    assert len(ranks) == d + 1 and ranks[0] == 1 and ranks[-1] == 1
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(d)]


def contract_cores(cores):
    """Assemble the full tensor from cores (input synthesis only; FP64)."""
    t = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for g in cores[1:]:
        r0, n, r1 = g.shape
        t = (t.reshape(-1, r0) @ g.reshape(r0, n * r1)).reshape(-1, r1)
    return t.reshape([g.shape[1] for g in cores])


def gaussian_tt(dims, ranks, rel_noise, seed, dtype=np.float32):
    """Example-1-style tensor A = P + beta*N with ||beta N|| = rel_noise * ||P|| (Sec. 4.1)."""
    cores = gaussian_cores(dims, ranks, seed)
    p = contract_cores(cores)
    if rel_noise > 0:
        rng = np.random.default_rng(seed + 0x9E3779B9)
        noise = rng.standard_normal(p.shape)
        beta = rel_noise * np.linalg.norm(p.ravel()) / np.linalg.norm(noise.ravel())
        p += beta * noise
        del noise
    return p.astype(dtype, copy=False)


def hilbert3(n=256, dtype=np.float32):
    """A(i,j,k) = 1/(i+j+k+1), i,j,k in 0..n-1, computed in FP64 then rounded."""
    i = np.arange(n, dtype=np.float64)
    s = i[:, None, None] + i[None, :, None] + i[None, None, :]
    return (1.0 / (s + 1.0)).astype(dtype, copy=False)


def example2(I=160, d=4, dtype=np.float64):
    """Example 2 of Sec. 4.1: sin(sqrt(sum_k ((i_k-1)/(I-1))^2)), i_k = 1..I."""
    x2 = (np.arange(I, dtype=np.float64) / (I - 1)) ** 2
    s = np.zeros((1,) * d)
    for k in range(d):
        shape = [1] * d
        shape[k] = I
        s = s + x2.reshape(shape)
    return np.sin(np.sqrt(s)).astype(dtype, copy=False)


def example2_torch(I=160, d=4, device="cuda", dtype=None):
    """example2 built on a torch device (FP64 arithmetic, then cast to dtype):
    the 160^4 tensor is 5.2 GB in FP64, so the GPU tests form it in place."""
    import torch
    x2 = (torch.arange(I, dtype=torch.float64, device=device) / (I - 1)) ** 2
    s = torch.zeros((1,) * d, dtype=torch.float64, device=device)
    for k in range(d):
        shape = [1] * d
        shape[k] = I
        s = s + x2.reshape(shape)
    out = torch.sin(torch.sqrt(s))
    return out if dtype is None else out.to(dtype)


def blobs_volume(shape=(256, 256, 64), nblobs=20, seed=0, dtype=np.float32):
    """Sum of axis-aligned anisotropic Gaussian blobs: centres uniform over the
    volume, per-axis widths U[2,30] voxels, amplitudes U[0.2,1]."""
    rng = np.random.default_rng(seed)
    vol = np.zeros(shape)
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    for _ in range(nblobs):
        c = [rng.uniform(0, s) for s in shape]
        w = [rng.uniform(2.0, 30.0) for _ in shape]
        a = rng.uniform(0.2, 1.0)
        f = [np.exp(-0.5 * ((ax - ci) / wi) ** 2) for ax, ci, wi in zip(axes, c, w)]
        vol += a * f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]
    return vol.astype(dtype, copy=False)


def observation_mask(shape, p_obs=0.3, seed=1):
    """Uniform random observation set Omega: each entry kept with probability p_obs.
    Returns sorted int64 linear (row-major) indices."""
    rng = np.random.default_rng(seed)
    keep = rng.random(int(np.prod(shape))) < p_obs
    return np.flatnonzero(keep).astype(np.int64)


def random_indices(dims, n, seed):
    """n distinct-or-not uniform linear indices into a tensor of shape dims (int64)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, int(np.prod(dims)), size=n, dtype=np.int64)


# The five workloads the sweep is validated and measured on.  Sizes follow the
# paper's synthetic examples (Sec. 4.1) scaled to one GPU.
CONFIGS = {
    "c1": dict(kind="gaussian_tt", dims=(16, 16, 16, 16), ranks=(1, 4, 4, 4, 1),
               rel_noise=1e-8, seed=0, dtype="float64", eps=1e-6),
    "c2": dict(kind="hilbert3", n=256, dtype="float32", eps=1e-6),
    "c3": dict(kind="gaussian_tt", dims=(32, 32, 32, 32, 32), ranks=(1, 20, 20, 20, 20, 1),
               rel_noise=1e-4, seed=0, dtype="float32", eps=1e-3),
    "c4": dict(kind="blobs", shape=(256, 256, 64), nblobs=20, seed=0, p_obs=0.3,
               mask_seed=1, dtype="float32", ranks=(1, 32, 16, 1)),
    # the size and TT ranks of the completion experiment's MRI volume (Sec. 4.2.2:
    # 181 x 217 x 181, ranks (55, 41), 70% of the entries removed), as blobs
    "mri": dict(kind="blobs", shape=(181, 217, 181), nblobs=40, seed=2, p_obs=0.3,
                mask_seed=3, dtype="float32", ranks=(1, 55, 41, 1)),
    "c5": dict(kind="gaussian_tt", dims=(128, 128, 128, 128), ranks=(1, 64, 64, 64, 1),
               rel_noise=1e-3, seed=0, dtype="float32", eps=1e-2),
}


def make_config(name, **override):
    """Build the input tensor of a named workload (FP64 draw, rounded once)."""
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    dt = np.dtype(cfg["dtype"])
    if cfg["kind"] == "gaussian_tt":
        return gaussian_tt(cfg["dims"], cfg["ranks"], cfg["rel_noise"], cfg["seed"], dt)
    if cfg["kind"] == "hilbert3":
        return hilbert3(cfg["n"], dt)
    if cfg["kind"] == "blobs":
        return blobs_volume(cfg["shape"], cfg["nblobs"], cfg["seed"], dt)
    raise ValueError(cfg["kind"])
