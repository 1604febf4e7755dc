"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the method (no sketch, QR, least squares or
core formation): it only builds test tensors, the way the paper's experiments
do (Sec. 4.3-4.4) and the way the workload configurations describe them.

* random_tt: a tensor built by contracting random N(0,1) TT cores of given
  ranks (exactly low TT rank), optionally plus i.i.d. Gaussian noise scaled to
  a relative Frobenius level, rounded to the storage dtype.  The same rounded
  values are handed to both sides.
* hilbert_type: X(i_1..i_d) = 1 / (x_{i_1} + ... + x_{i_d}) with x on a uniform
  grid of [1, 2] including both end points (the 17 GB streaming workload).
* hilbert_paper: the paper's Hilbert tensor 1 / (1 - d + i_1 + ... + i_d),
  1-based (Sec. 4.3).
* gaussian_bumps: sum of N Gaussians exp(-gamma |x - c_j|^2) on the grid
  x = 2 i / n - 1 (Sec. 4.4, second workload of Fig. time2).

All tensors are flat column-major vectors (i_1 fastest).
"""
import numpy as np


def _prod(dims):
    p = 1
    for n in dims:
        p *= int(n)
    return p


def random_tt_cores(dims, ranks, seed=0):
    """Cores G_k of shape (r_{k-1}, n_k, r_k) with i.i.d. N(0,1) entries."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((int(ranks[k]), int(dims[k]), int(ranks[k + 1])))
            for k in range(len(dims))]


def contract_tt(cores):
    """Dense column-major tensor of a list of TT cores (FP64)."""
    L = np.ones((1, 1))
    for G in cores:
        a, n, b = G.shape
        L = (L @ G.reshape((a, n * b), order='F')).reshape((L.shape[0] * n, b), order='F')
    return L[:, 0].copy()


def random_tt(dims, ranks, seed=0, noise=0.0, noise_seed=2, dtype=np.float64):
    """Random-TT tensor (+ relative noise), rounded to `dtype`; returns FP64
    copy of the rounded values and the rounded array itself."""
    x = contract_tt(random_tt_cores(dims, ranks, seed))
    if noise > 0:
        e = np.random.default_rng(noise_seed).standard_normal(x.size)
        x = x + e * (noise * np.linalg.norm(x) / np.linalg.norm(e))
    xr = x.astype(dtype)
    return xr


def hilbert_type(dims, dtype=np.float32, first_last=0, count_last=None):
    """1/(x_{i_1}+...+x_{i_d}), x_i = 1 + i/(n-1); optionally only the slab of
    the last mode [first_last, first_last + count_last).  The sum is formed in
    FP64 left to right (i_1 first), then 1/sum is rounded to `dtype`."""
    dims = [int(n) for n in dims]
    if count_last is None:
        count_last = dims[-1] - first_last
    idx = [None] * (len(dims) - 1) + [np.arange(first_last, first_last + count_last)]
    return hilbert_type_block(dims, idx, dtype)


def hilbert_type_block(dims, idx, dtype=np.float32):
    """The sub-tensor of hilbert_type(dims) at the index sets idx[k] of each
    mode (None = the whole mode), column-major flat, with the same values
    entry for entry (same FP64 summation order and rounding)."""
    dims = [int(n) for n in dims]
    grids = [1.0 + np.arange(n, dtype=np.float64) / max(n - 1, 1) for n in dims]
    grids = [g if ix is None else g[np.asarray(ix, dtype=np.int64)] for g, ix in zip(grids, idx)]
    s = grids[0]
    for k in range(1, len(dims)):
        s = (s[:, None] + grids[k][None, :]).reshape(-1, order='F')
    return (1.0 / s).astype(dtype)


def hilbert_paper(dims, dtype=np.float64):
    """The paper's Hilbert tensor 1/(1 - d + i_1 + ... + i_d), 1-based."""
    dims = [int(n) for n in dims]
    d = len(dims)
    s = np.arange(1, dims[0] + 1, dtype=np.float64)
    for k in range(1, d):
        s = (s[:, None] + np.arange(1, dims[k] + 1, dtype=np.float64)[None, :]).reshape(-1, order='F')
    return (1.0 / (1.0 - d + s)).astype(dtype)


def bump_centres(d, nbumps=100, seed=4):
    """Centres of the Gaussian bumps: nbumps x d, uniform in (-1, 1)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(nbumps, d))


def gaussian_bumps(dims, nbumps=100, gamma=10.0, seed=4, dtype=np.float64):
    """sum_j exp(-gamma sum_k (x_k - c_{j,k})^2), x_k = 2 i_k / n_k - 1,
    centres uniform in (-1, 1)."""
    dims = [int(n) for n in dims]
    C = bump_centres(len(dims), nbumps, seed)
    out = np.zeros(_prod(dims))
    for j in range(nbumps):
        f = np.ones(1)
        for k, n in enumerate(dims):
            x = 2.0 * np.arange(n) / n - 1.0
            f = (f[:, None] * np.exp(-gamma * (x - C[j, k]) ** 2)[None, :]).reshape(-1, order='F')
        out += f
    return out.astype(dtype)


def target_tensor(n_entries, seed=3, dtype=np.float64):
    """The fixed N(0,1) target T of the differentiation loss."""
    return np.random.default_rng(seed).standard_normal(int(n_entries)).astype(dtype)


def batch_specs(count=512, seed=5, cap=2_000_000):
    """Uneven batch of tensor shapes: d ~ U{3..6}, n ~ U{8..32} with n clamped
    to floor(cap^(1/d)), TT ranks ~ U{2..16} per bond, clamped to
    min(N_k, M_k, n_k r_{k-1}, r_{k+1} n_{k+1})."""
    rng = np.random.default_rng(seed)
    specs = []
    for b in range(count):
        d = int(rng.integers(3, 7))
        n = int(rng.integers(8, 33))
        n = min(n, int(np.floor(cap ** (1.0 / d) + 1e-9)))
        dims = [n] * d
        r = [1] + [int(rng.integers(2, 17)) for _ in range(d - 1)] + [1]
        N = [1]
        for m in dims:
            N.append(N[-1] * m)
        for k in range(1, d):
            r[k] = min(r[k], N[k], N[d] // N[k], r[k - 1] * dims[k - 1])
        for k in range(d - 1, 0, -1):
            r[k] = min(r[k], r[k + 1] * dims[k])
        specs.append((dims, r))
    return specs
