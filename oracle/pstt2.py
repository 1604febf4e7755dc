"""PSTT2 and PSTT2-onepass, step by step, in FP64 (the oracle of the hot path).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module; the product path never does.

What it follows (Sec. 3.2 of the paper):
* Algorithm 2 (PSTT): Gaussian test matrices, sketches S_j = X_j Phi_j, CPQR,
  Q_j = Q(:, 1:r_j), cores by eq. (3.1) ("eq core").
* The two-sided variant PSTT2 (end of Sec. 3.2): split d* = ceil(d/2); column
  bases Q_k for k < d*, row bases P_k for the unfoldings k >= d*; the middle
  core by eq. (3.5) ("PSTT2_final_core", second pass) or, in PSTT2-onepass,
  by an extra sketch of the middle unfolding and a pseudo-inverse as in
  eq. (3.3) ("onepass_final_core").

Readings of the paper taken here (the CUDA path takes the same ones):
* A1  P-indexing: the paper's "P_j for j > d*" is the row basis of X_{j-1};
  row sketches R_k = X_k^T Psi_k cover k = d*..d-1 (the only dimensionally
  consistent reading of eq. (3.5)).
* A2  the one-pass extra sketch is on the column side: S_{d*} = X_{d*} Omega_{d*},
  H = S_{d*} (P_{d*}^T Omega_{d*})^+  (least squares through QR of B^T).
* A3  sketch widths l_k = r_k + p (fixed-rank mode) or rmax + p (eps mode),
  where a requested r_k is first clamped to min(N_k, M_k), the largest rank
  X_k can have (eq. (2.1), r_k <= rank(X_k)).
* A4  CPQR: largest recomputed column norm, lowest index on ties, diag(R)>=0.
* A5  eps-mode rank: smallest r >= 1 with ||R_22^(r)||_F <= eps/sqrt(d-1) ||S||_F,
  capped at rmax (flagged) and at min(N_k, M_k).
* Test matrices: Omega_k = stream k, Psi_k = stream 64 + k (oracle.philox).
  drm='gauss': i.i.d. Gaussian entries (Algorithm 2); drm='kr': Khatri-Rao
  products of per-mode Gaussian factors (eq. (sketch_orig)): Omega_k over the
  modes k+1..d of its rows, Psi_k over the modes 1..k.  With test_fmt rounding
  (the mixed-precision paths) every entry is rounded, except the Khatri-Rao
  Psi_{d-1}, taken mode by mode (psi_rounded).
"""
import math
import numpy as np

from . import philox
from .linalg import householder_cpqr, lstsq_right
from .tt import prods, unfold


def split_index(d):
    """d* = ceil(d/2) (Sec. 3.2, after Theorem 3.3)."""
    return (d + 1) // 2


def pick_rank_eps(R, eps, d, rmax, rcap):
    """A5: smallest r with ||R[r:, r:]||_F <= eps/sqrt(d-1) * ||R||_F."""
    total = math.sqrt(float(np.sum(R ** 2)))
    thr = eps / math.sqrt(max(d - 1, 1)) * total
    kmax = min(R.shape)
    limit = min(rmax, rcap, kmax) if kmax > 0 else 1
    for r in range(1, limit + 1):
        tail = math.sqrt(float(np.sum(R[r:, r:] ** 2)))
        if tail <= thr:
            return r, False
    return max(limit, 1), True


def clamp_ranks(dims, ranks):
    """r_k <= min(N_k, M_k) (eq. (2.1): r_k <= rank(X_k))."""
    N = prods(dims)
    d = len(dims)
    return [1] + [min(int(ranks[k]), N[k], N[d] // N[k]) for k in range(1, d)] + [1]


def sketch_widths(d, ranks, p, eps_mode, rmax):
    """l_k for k = 1..d (index 0 unused); A3."""
    if eps_mode:
        return [None] + [rmax + p] * d
    return [None] + [int(ranks[k]) + p for k in range(1, d)] + [None]


def omega(seed, dims, k, l, drm='gauss'):
    """Omega_k (M_k x l, FP64): the right test matrix of X_k."""
    d = len(dims)
    N = prods(dims)
    if drm == 'kr':
        return philox.kr_test_matrix(seed, philox.STREAM_OMEGA + k, list(range(k + 1, d + 1)), dims[k:], l)
    return philox.test_matrix(seed, philox.STREAM_OMEGA + k, N[d] // N[k], l)


def psi(seed, dims, k, l, drm='gauss'):
    """Psi_k (N_k x l, FP64): the left test matrix of X_k."""
    N = prods(dims)
    if drm == 'kr':
        return philox.kr_test_matrix(seed, philox.STREAM_PSI + k, list(range(1, k + 1)), dims[:k], l,
                                     decreasing=True)
    return philox.test_matrix(seed, philox.STREAM_PSI + k, N[k], l)


def psi_rounded(seed, dims, k, l, drm, fmt):
    """Psi_k as a sketch in arithmetic `fmt` uses it.  Entries are rounded to
    fmt, except the Khatri-Rao Psi_{d-1} of a rounded format, which is taken
    mode by mode as eq. (sketch_orig) writes the Khatri-Rao sketch: the mode-1
    factor rounded to fmt (it enters the product with X) times the rounded
    product of the other factors' rows (the diagonal scaling D), i.e.
    round(F_1(i_1, j)) * round(F_{d-1}(i_{d-1}, j) ... F_2(i_2, j))."""
    d = len(dims)
    if drm == 'kr' and k == d - 1 and fmt not in ('f64', 'f32') and k >= 2:
        s = philox.STREAM_PSI + k
        F1 = philox.round_to(philox.kr_factor(seed, s, 1, dims[0], l), fmt)
        rest = philox.round_to(philox.kr_test_matrix(seed, s, list(range(2, k + 1)), dims[1:k], l,
                                                     decreasing=True), fmt)
        return (F1[None, :, :] * rest[:, None, :]).reshape(-1, l)
    return philox.round_to(psi(seed, dims, k, l, drm), fmt)


def sketches(x, dims, widths, seed, passes, test_fmt='f64', drm='gauss'):
    """Step 2: dense sketches, materialising the test matrices.

    Returns dict with 'S' {k: N_k x l_k} for k < d* (and k = d* in one-pass),
    'R' {k: M_k x l_k} for k = d*..d-1, and the test matrices used.
    test_fmt rounds the test-matrix entries ('f64' keeps them exact); drm
    selects dense Gaussian ('gauss') or Khatri-Rao ('kr') test matrices.
    """
    d = len(dims)
    ds = split_index(d)
    S, R, Om, Ps = {}, {}, {}, {}
    last_col = ds if passes == 1 else ds - 1
    for k in range(1, last_col + 1):
        l = widths[k] if k < ds else widths[ds]
        Om[k] = philox.round_to(omega(seed, dims, k, l, drm), test_fmt)
        S[k] = unfold(x, dims, k) @ Om[k]
    for k in range(ds, d):
        l = widths[k]
        Ps[k] = psi_rounded(seed, dims, k, l, drm, test_fmt)
        R[k] = unfold(x, dims, k).T @ Ps[k]
    return {'S': S, 'R': R, 'Omega': Om, 'Psi': Ps}


def bases(sk, dims, ranks, eps, rmax):
    """Steps 3-4: CPQR of every basis sketch; rank per A5 in eps mode."""
    d = len(dims)
    ds = split_index(d)
    N = prods(dims)
    r = [1] * (d + 1)
    Q, P, piv, Rf, capped = {}, {}, {}, {}, {}
    for k in range(1, d):
        Y = sk['S'][k] if k < ds else sk['R'][k]
        Qf, Rk, pv = householder_cpqr(Y)
        rcap = min(N[k], N[d] // N[k])
        if eps is not None and eps > 0:
            rk, cap = pick_rank_eps(Rk, eps, d, rmax, rcap)
        else:
            rk, cap = min(int(ranks[k]), rcap, Qf.shape[1]), False
        r[k] = rk
        capped[k] = cap
        piv[k] = pv
        Rf[k] = Rk
        if k < ds:
            Q[k] = Qf[:, :rk]
        else:
            P[k] = Qf[:, :rk]
    return r, Q, P, piv, Rf, capped


def outer_cores(dims, r, Q, P):
    """Step 5: G_1 = Q_1, eq. (3.1) for 2 <= k < d*, its row-space mirror for
    d* < k < d, and G_d = P_{d-1}^T."""
    d = len(dims)
    ds = split_index(d)
    N = prods(dims)
    cores = [None] * (d + 1)
    if ds >= 2:
        cores[1] = Q[1].reshape((1, dims[0], r[1]), order='F')
    for k in range(2, ds):
        W = Q[k - 1].T @ Q[k].reshape((N[k - 1], dims[k - 1] * r[k]), order='F')
        cores[k] = W.reshape((r[k - 1], dims[k - 1], r[k]), order='F')
    for k in range(ds + 1, d):
        # G_k(a, i, c) = sum_v P_{k-1}(i + n_k v, a) P_k(v, c)
        nk = dims[k - 1]
        Mk = N[d] // N[k]
        Pm = P[k - 1].reshape((nk, Mk, r[k - 1]), order='F')
        cores[k] = np.einsum('iva,vc->aic', Pm, P[k])
    cores[d] = P[d - 1].T.reshape((r[d - 1], dims[d - 1], 1), order='F')
    return cores


def middle_core_onepass(dims, r, Q, P, S_mid, Om_mid):
    """Step 6 (one-pass): B = P_{d*}^T Omega_{d*}; H = argmin ||H B - S_{d*}||;
    G_{d*} = reshape(Q_{d*-1}^T reshape(H, N_{d*-1}, n_{d*} r_{d*}))."""
    d = len(dims)
    ds = split_index(d)
    N = prods(dims)
    B = P[ds].T @ Om_mid
    H, rdiag = lstsq_right(S_mid, B)
    Ql = Q[ds - 1] if ds >= 2 else np.ones((1, 1))
    W = Ql.T @ H.reshape((N[ds - 1], dims[ds - 1] * r[ds]), order='F')
    return W.reshape((r[ds - 1], dims[ds - 1], r[ds]), order='F'), B, H, rdiag


def middle_core_twopass(x, dims, r, Q, P):
    """Step 7 (two-pass): eq. (3.5), G_{d*} = reshape(X, N_{d*-1}, n_{d*}, M_{d*})
    x_1 Q_{d*-1}^T x_3 P_{d*}^T."""
    d = len(dims)
    ds = split_index(d)
    N = prods(dims)
    X3 = np.asarray(x).reshape((N[ds - 1], dims[ds - 1], N[d] // N[ds]), order='F')
    Ql = Q[ds - 1] if ds >= 2 else np.ones((1, 1))
    return np.einsum('ua,uiv,vc->aic', Ql, X3, P[ds])


def pstt2(x, dims, *, ranks=None, eps=None, rmax=None, p=5, seed=1, passes=1,
          test_fmt='f64', drm='gauss'):
    """PSTT2 (passes=2) or PSTT2-onepass (passes=1) of the column-major tensor x.

    Either fixed ranks (ranks = [1, r_1, ..., r_{d-1}, 1]) or tolerance mode
    (eps > 0 with cap rmax).  Returns a dict with the cores (list, 0-based,
    shapes (r_{k-1}, n_k, r_k)), the ranks, the bases and intermediate state.
    """
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
    ds = split_index(d)
    widths = sketch_widths(d, ranks, p, eps_mode, rmax)
    sk = sketches(x, dims, widths, seed, passes, test_fmt, drm)
    r, Q, P, piv, Rf, capped = bases(sk, dims, ranks, eps if eps_mode else None, rmax)
    cores = outer_cores(dims, r, Q, P)
    out = {'r': r, 'Q': Q, 'P': P, 'piv': piv, 'Rfac': Rf, 'capped': capped,
           'sketch': sk, 'widths': widths}
    if passes == 1:
        Gm, B, H, rdiag = middle_core_onepass(dims, r, Q, P, sk['S'][ds], sk['Omega'][ds][:, :widths[ds]])
        out.update(B=B, H=H, rdiag=rdiag)
    else:
        Gm = middle_core_twopass(x, dims, r, Q, P)
    cores[ds] = Gm
    out['cores'] = cores[1:]
    return out


def pstt2_stream(slabs, dims, *, ranks=None, eps=None, rmax=None, p=5, seed=1, drm='gauss'):
    """PSTT2-onepass over slabs of the last mode (Sec. 4.2, Algorithm 5's
    single stream): each slab (first, count, values) adds its contribution to
    every sketch; only one slab is held at a time.  Same result as pstt2 on
    the whole tensor up to summation order."""
    dims = [int(n) for n in dims]
    d = len(dims)
    ds = split_index(d)
    N = prods(dims)
    eps_mode = eps is not None and eps > 0
    if not eps_mode:
        ranks = clamp_ranks(dims, ranks)
    widths = sketch_widths(d, ranks, p, eps_mode, rmax)
    S = {k: np.zeros((N[k], widths[k] if k < ds else widths[ds])) for k in range(1, ds + 1)}
    R = {k: np.zeros((N[d] // N[k], widths[k])) for k in range(ds, d)}
    Ps = {k: psi(seed, dims, k, widths[k], drm) for k in range(ds, d)}
    Nd1 = N[d - 1]
    for first, count, vals in slabs:
        vals = np.asarray(vals, dtype=np.float64)
        for k in range(1, ds + 1):
            l = S[k].shape[1]
            Mk_slab = (Nd1 // N[k]) * count
            rows = np.arange(Mk_slab, dtype=np.uint64) + np.uint64((Nd1 // N[k]) * first)
            if drm == 'kr':
                Om = omega(seed, dims, k, l, drm)[rows.astype(np.int64)]
            else:
                Om = philox.gaussian(seed, philox.STREAM_OMEGA + k, rows, l)
            S[k] += vals.reshape((N[k], Mk_slab), order='F') @ Om
        for k in range(ds, d):
            Mk_slab = (Nd1 // N[k]) * count
            R[k][(Nd1 // N[k]) * first:(Nd1 // N[k]) * (first + count)] += \
                vals.reshape((N[k], Mk_slab), order='F').T @ Ps[k]
    sk = {'S': S, 'R': R, 'Omega': {}, 'Psi': Ps}
    r, Q, P, piv, Rf, capped = bases(sk, dims, ranks, eps if eps_mode else None, rmax)
    cores = outer_cores(dims, r, Q, P)
    Om_mid = omega(seed, dims, ds, widths[ds], drm)
    Gm, B, H, rdiag = middle_core_onepass(dims, r, Q, P, S[ds], Om_mid)
    cores[ds] = Gm
    return {'r': r, 'Q': Q, 'P': P, 'piv': piv, 'cores': cores[1:], 'sketch': sk,
            'B': B, 'H': H, 'rdiag': rdiag, 'capped': capped}
