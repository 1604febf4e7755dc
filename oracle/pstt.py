"""One-sided PSTT and PSTT-onepass of the oracle (plain NumPy, FP64).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

PSTT (Algorithm 2) sketches every unfolding from the right, S_j = X_j Omega_j
(j = 1..d-1), keeps Q_j = the first r_j columns of a CPQR of S_j and forms the
cores by eq. (3.1): G_1 = Q_1, G_{k+1} = reshape(Q_k^T reshape(Q_{k+1},
N_k, n_{k+1} r_{k+1})).  Its two-pass last core G_d = Q_{d-1}^T X_{d-1} reads X
again; the single-pass variant (PSTT-onepass, the paragraph after Theorem 3.3)
draws one more Gaussian map Psi_{d-1} (N_{d-1} x (r_{d-1} + p)), sketches
T_{d-1} = Psi_{d-1}^T X_{d-1} in the same pass, and takes
G_d = (Psi_{d-1}^T Q_{d-1})^+ T_{d-1} (eq. "onepass_final_core").

The readings of the two-sided oracle apply unchanged: test matrices
Omega_j = stream j and Psi_{d-1} = stream 64 + d - 1 of oracle.philox (A6),
widths l_j = r_j + p or rmax + p (A3), CPQR pivoting and the eps rank rule
(A4, A5).  The least-squares solve is the same QR of the small factor as the
two-sided middle core.  drm='kr' takes the Khatri-Rao test matrices of
oracle.pstt2 (Omega_j over the modes j+1..d, Psi_{d-1} over 1..d-1): Algorithm 2
"with the Khatri-Rao DRMs" of the paragraph after Theorem 3.3.
"""
import numpy as np

from . import philox
from .linalg import householder_cpqr, lstsq_right
from .pstt2 import clamp_ranks, omega, pick_rank_eps, psi_rounded, sketch_widths
from .tt import prods, unfold


def pstt(x, dims, *, ranks=None, eps=None, rmax=None, p=5, seed=1, test_fmt='f64', drm='gauss'):
    """PSTT (Algorithm 2, two passes): the bases and cores 1..d-1 of
    pstt_onepass, and the last core G_d = Q_{d-1}^T X_{d-1} from a second
    pass over X."""
    o = pstt_onepass(x, dims, ranks=ranks, eps=eps, rmax=rmax, p=p, seed=seed, test_fmt=test_fmt, drm=drm)
    dims = [int(n) for n in dims]
    d = len(dims)
    r = o['r']
    G = o['Q'][d - 1].T @ unfold(x, dims, d - 1)           # r_{d-1} x n_d
    o['cores'][d - 1] = G.reshape((r[d - 1], dims[d - 1], 1), order='F')
    return o


def pstt_onepass(x, dims, *, ranks=None, eps=None, rmax=None, p=5, seed=1, test_fmt='f64', drm='gauss'):
    """PSTT-onepass of the column-major tensor x: fixed ranks
    ([1, r_1, ..., r_{d-1}, 1]) or tolerance mode (eps > 0 with cap rmax).
    Returns a dict with the cores (0-based list, shapes (r_{k-1}, n_k, r_k)),
    the ranks, the bases Q, the sketches S and T, and the last-core factors."""
    dims = [int(n) for n in dims]
    d = len(dims)
    if d < 2:
        raise ValueError("d >= 2 required")
    eps_mode = eps is not None and eps > 0
    if not eps_mode:
        ranks = [int(v) for v in ranks]
        if len(ranks) != d + 1:
            raise ValueError("ranks needs d+1 entries")
        ranks = clamp_ranks(dims, ranks)
    widths = sketch_widths(d, ranks, p, eps_mode, rmax)
    N = prods(dims)
    # one pass: the right sketches of every unfolding and the left sketch of X_{d-1}
    S, Om = {}, {}
    for k in range(1, d):
        Om[k] = philox.round_to(omega(seed, dims, k, widths[k], drm), test_fmt)
        S[k] = unfold(x, dims, k) @ Om[k]
    Psi = psi_rounded(seed, dims, d - 1, widths[d - 1], drm, test_fmt)
    T = Psi.T @ unfold(x, dims, d - 1)                    # l x n_d
    # bases: CPQR of every S_k, rank per A5 in tolerance mode
    r = [1] * (d + 1)
    Q, piv, capped = {}, {}, {}
    for k in range(1, d):
        Qf, Rk, pv = householder_cpqr(S[k])
        rcap = min(N[k], N[d] // N[k])
        if eps_mode:
            rk, cap = pick_rank_eps(Rk, eps, d, rmax, rcap)
        else:
            rk, cap = min(int(ranks[k]), rcap, Qf.shape[1]), False
        r[k], piv[k], capped[k] = rk, pv, cap
        Q[k] = Qf[:, :rk]
    # cores 1..d-1 by eq. (3.1)
    cores = [None] * (d + 1)
    cores[1] = Q[1].reshape((1, dims[0], r[1]), order='F')
    for k in range(2, d):
        W = Q[k - 1].T @ Q[k].reshape((N[k - 1], dims[k - 1] * r[k]), order='F')
        cores[k] = W.reshape((r[k - 1], dims[k - 1], r[k]), order='F')
    # last core: G_d = argmin ||(Psi^T Q_{d-1}) G - T||, i.e. G^T = argmin ||G^T B - T^T||
    # with B = Q_{d-1}^T Psi (r x l)
    B = Q[d - 1].T @ Psi
    Gt, rdiag = lstsq_right(T.T, B)                        # n_d x r_{d-1}
    cores[d] = Gt.T.reshape((r[d - 1], dims[d - 1], 1), order='F')
    return {'r': r, 'Q': Q, 'piv': piv, 'capped': capped, 'S': S, 'T': T, 'Omega': Om, 'Psi': Psi,
            'B': B, 'rdiag': rdiag, 'widths': widths, 'cores': cores[1:]}
