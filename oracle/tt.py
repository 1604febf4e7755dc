"""Tensor-train basics and sequential TT-SVD of the oracle (plain NumPy, FP64).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Conventions (Sec. 2.1): a tensor X of size n_1 x ... x n_d is held as a flat
vector in column-major order (i_1 fastest).  The k-th unfolding is
X_k = reshape(X, N_k, M_k) with N_k = n_1...n_k, M_k = n_{k+1}...n_d, i.e. the
same buffer with leading dimension N_k.  A TT core G_k is an array of shape
(r_{k-1}, n_k, r_k) with r_0 = r_d = 1 (Sec. 2.2).
"""
import math
import numpy as np


def prods(dims):
    """N[k] = n_1...n_k for k = 0..d (N[0] = 1)."""
    N = [1]
    for n in dims:
        N.append(N[-1] * int(n))
    return N


def unfold(x, dims, k):
    """X_k = reshape(X, N_k, M_k), column-major (Sec. 2.1)."""
    N = prods(dims)
    return np.asarray(x).reshape((N[k], N[-1] // N[k]), order='F')


def tt_full(cores):
    """Dense column-major vector of the tensor represented by TT cores (Sec. 2.2).

    Contracts left to right: the left interface L_k (N_k x r_k) is
    reshape(L_{k-1} G_k, N_k, r_k) with G_k seen as r_{k-1} x (n_k r_k).
    """
    L = np.ones((1, 1))
    for G in cores:
        r0, n, r1 = G.shape
        L = (L @ G.reshape((r0, n * r1), order='F')).reshape((L.shape[0] * n, r1), order='F')
    return L[:, 0].copy()


def tt_entry(cores, idx):
    """One entry X(i_1..i_d) = G_1(:, i_1, :) ... G_d(:, i_d, :) (Sec. 2.2)."""
    v = np.ones((1,))
    for G, i in zip(cores, idx):
        v = v @ G[:, int(i), :]
    return float(v[0])


def tt_storage(cores_shapes):
    """Number of stored entries sum_k r_{k-1} n_k r_k (Sec. 2.2)."""
    return sum(int(a) * int(b) * int(c) for a, b, c in cores_shapes)


def tt_svd(x, dims, eps):
    """Sequential TT-SVD (Sec. 2.2): every SVD is truncated at an absolute
    Frobenius tolerance eps ||X||_F / sqrt(d-1), which guarantees
    ||X - X~||_F <= eps ||X||_F.  The SVD itself is LAPACK's (numpy)."""
    d = len(dims)
    x = np.asarray(x, dtype=np.float64)
    delta = eps * np.linalg.norm(x) / math.sqrt(max(d - 1, 1))
    cores = []
    C = x.copy()
    r_prev = 1
    for k in range(d - 1):
        n = int(dims[k])
        C = C.reshape((r_prev * n, C.size // (r_prev * n)), order='F')
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]   # tail[r] = ||s[r:]||
        r = len(s)
        for cand in range(1, len(s) + 1):
            t = tail[cand] if cand < len(s) else 0.0
            if t <= delta:
                r = cand
                break
        cores.append(U[:, :r].reshape((r_prev, n, r), order='F'))
        C = (s[:r, None] * Vt[:r, :])
        r_prev = r
    cores.append(C.reshape((r_prev, int(dims[-1]), 1), order='F'))
    return cores
