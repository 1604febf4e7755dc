"""Dense FP64 linear algebra of the oracle: Householder (CP)QR and least squares.

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper obtains the orthonormal bases with a column-pivoted QR (Sec. 3.2,
Algorithm 2: "compute a CPQR of S_j ... set Q_j = Q_j(:, 1:r_j)", citing Chan's
rank-revealing QR).  Its tie-break and sign conventions are not stated; this
oracle uses: the pivot is the remaining column of largest norm, recomputed
from scratch at every step (not downdated); ties go to the lowest index; the
signs are normalised so that diag(R) >= 0.
"""
import math
import numpy as np


def householder_cpqr(A, pivoting=True):
    """Column-pivoted Householder QR, A[:, piv] = Q @ R.

    A: m x n.  Returns (Q, R, piv) with Q m x k orthonormal, R k x n upper
    trapezoidal, k = min(m, n), diag(R) >= 0.  pivoting=False gives the
    unpivoted QR (piv = identity).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    k = min(m, n)
    piv = np.arange(n)
    vs = []
    for i in range(k):
        if pivoting:
            norms = np.sqrt(np.sum(A[i:, i:] ** 2, axis=0))
            j = i + int(np.argmax(norms))  # first maximum: lowest index on ties
            if j != i:
                A[:, [i, j]] = A[:, [j, i]]
                piv[[i, j]] = piv[[j, i]]
        x = A[i:, i]
        nx = math.sqrt(float(np.dot(x, x)))
        if nx == 0.0:
            vs.append(None)
            continue
        alpha = -math.copysign(nx, x[0])
        v = x.copy()
        v[0] -= alpha
        v /= math.sqrt(float(np.dot(v, v)))
        A[i:, i:] -= 2.0 * np.outer(v, v @ A[i:, i:])
        A[i + 1:, i] = 0.0
        vs.append(v)
    R = np.triu(A[:k, :])
    Q = np.eye(m, k)
    for i in reversed(range(k)):
        v = vs[i]
        if v is not None:
            Q[i:, :] -= 2.0 * np.outer(v, v @ Q[i:, :])
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    R = s[:, None] * R
    Q = Q * s[None, :]
    return Q, R, piv


def lstsq_right(S, B):
    """H = argmin ||H B - S||_F for B (r x l, l >= r, full row rank).

    Solved through the QR of B^T: B^T = Q_B R_B, so H = S Q_B R_B^{-T}.
    Returns (H, rdiag) where rdiag is diag(R_B) (zero means B is singular).
    """
    QB, RB, _ = householder_cpqr(B.T, pivoting=False)
    r = B.shape[0]
    RB = RB[:r, :r]
    rdiag = np.diag(RB).copy()
    T = S @ QB[:, :r]                    # N x r
    # H RB^T = T  ->  solve RB H^T = T^T (upper-triangular back substitution)
    Ht = np.zeros((r, S.shape[0]))
    for i in reversed(range(r)):
        acc = T[:, i] - RB[i, i + 1:] @ Ht[i + 1:, :]
        Ht[i, :] = acc / RB[i, i] if RB[i, i] != 0 else np.nan
    return Ht.T, rdiag
