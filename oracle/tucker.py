"""Tucker2TT of the oracle (plain NumPy, FP64).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Algorithm 3: given an orthogonal Tucker format X = G x_1 A_1 ... x_d A_d
(G: s_1 x ... x s_d, A_j: n_j x s_j with ON columns), take a TT decomposition
H_1..H_d of the small core G and set T_j = H_j x_2 A_j, i.e.
T_j(a, i, c) = sum_s A_j(i, s) H_j(a, s, c).  The TT decomposition of G is the
oracle's PSTT2 (one- or two-pass), so the TT ranks of X~ are those found for G
(the lemma after Algorithm 3: rank X_j = rank G_j).
"""
import numpy as np

from .pstt2 import pstt2


def mode2(core, A):
    """T = H x_2 A for one TT core H (r_{k-1} x s_k x r_k) and A (n_k x s_k)."""
    return np.einsum('is,asc->aic', A, core)


def tucker2tt(G, factors, **pstt2_kw):
    """TT cores of the Tucker tensor (G, factors); G column-major flat with
    dims = [A.shape[1] for A in factors].  Returns (cores, pstt2 result of G)."""
    dims = [int(A.shape[1]) for A in factors]
    o = pstt2(np.asarray(G), dims, **pstt2_kw)
    return [mode2(H, A) for H, A in zip(o['cores'], factors)], o


def unfold2(core):
    """The mode-2 matricization of a TT core: M(i, a + r0 c) = T(a, i, c)."""
    r0, n, r1 = core.shape
    return np.transpose(core, (1, 0, 2)).reshape((n, r0 * r1), order='F')


def tt2tucker(cores, tranks, *, p=5, seed=1):
    """TT2Tucker (Algorithm 4) with the basis of step 2 from sketching: for
    core k, A_k = Q_1 and H_k = Q_1^T (T_k)_(2) (folded back to r_{k-1} x t_k x
    r_k) of the one-sided two-pass PSTT (Algorithm 2, d = 2) of the matrix
    (T_k)_(2) with target rank t_k and test-matrix key seed + k.  Returns
    (H cores, factors A)."""
    from .pstt import pstt
    Hs, As = [], []
    for k, T in enumerate(cores, start=1):
        r0, n, r1 = T.shape
        M = unfold2(T)
        t = min(int(tranks[k - 1]), n, r0 * r1)
        o = pstt(M.reshape(-1, order='F'), [n, r0 * r1], ranks=[1, t, 1], p=p, seed=seed + k)
        A = o['cores'][0].reshape((n, -1), order='F')          # n x t
        H2 = o['cores'][1].reshape((A.shape[1], r0 * r1), order='F')
        Hs.append(np.transpose(H2.reshape((A.shape[1], r0, r1), order='F'), (1, 0, 2)))
        As.append(A)
    return Hs, As
