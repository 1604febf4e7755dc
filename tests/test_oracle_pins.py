"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a published value,
a library routine that implements a textbook algorithm independently, a
brute-force loop, an exactness theorem of the paper, or its error bound.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import torch

import ttinputs as ti
from oracle import linalg, philox, pstt2 as P, tt


# ---------------------------------------------------------------- Philox
def test_philox_known_answers(golden):
    for row in golden("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in row]
        out = philox.philox4x32_10(*[np.uint64(c) for c in v[:4]], v[4], v[5])
        assert [int(o) for o in out] == v[6:]


def test_gaussian_moments_and_independence():
    z = philox.test_matrix(seed=11, stream=3, nrows=50_000, ncols=8)
    f = z.ravel()
    n = f.size
    assert abs(f.mean()) < 5.0 / math.sqrt(n)
    assert abs(f.var() - 1.0) < 6.0 * math.sqrt(2.0 / n)
    assert abs(np.mean(f ** 4) - 3.0) < 6.0 * math.sqrt(96.0 / n)
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(8))) < 5.0 / math.sqrt(z.shape[0])
    # different streams and seeds are different matrices
    z2 = philox.test_matrix(seed=11, stream=4, nrows=1000, ncols=8)
    z3 = philox.test_matrix(seed=12, stream=3, nrows=1000, ncols=8)
    assert abs(np.corrcoef(z[:1000].ravel(), z2.ravel())[0, 1]) < 0.1
    assert abs(np.corrcoef(z[:1000].ravel(), z3.ravel())[0, 1]) < 0.1


def test_gaussian_rows_are_counter_addressed():
    full = philox.test_matrix(5, 7, 300, 11)
    rows = np.array([299, 0, 17, 17, 128], dtype=np.uint64)
    np.testing.assert_array_equal(philox.gaussian(5, 7, rows, 11), full[rows.astype(int)])
    # column j does not depend on how many columns are requested
    np.testing.assert_array_equal(philox.test_matrix(5, 7, 300, 3), full[:, :3])
    # 64-bit row indices use the high counter word
    big = np.array([2 ** 32 + 5], dtype=np.uint64)
    assert not np.allclose(philox.gaussian(5, 7, big, 4), full[5, :4])


def test_round_to_matches_torch_bf16():
    x = np.random.default_rng(0).standard_normal(10_000) * 10.0 ** np.random.default_rng(1).uniform(-5, 5, 10_000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(philox.round_to(x, "bf16"), ref)


def test_round_to_fp16_matches_numpy_half():
    # numpy's float16 cast (IEEE binary16, nearest-even, subnormals, overflow)
    # as the library reference, over normals, subnormals and the range ends
    rng = np.random.default_rng(3)
    x = rng.standard_normal(20_000) * 2.0 ** rng.uniform(-30, 17, 20_000)
    x = np.concatenate([x, [0.0, -0.0, 65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -24, 2.0 ** -25,
                            3 * 2.0 ** -26, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25, np.inf, -np.inf]])
    f32 = x.astype(np.float32)
    ref = f32.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(philox.round_to(x, "fp16"), ref)
    assert np.isnan(philox.round_to(np.array([np.nan]), "fp16")[0])


def test_round_to_fp16_cases():
    # ties to even at 1 (quantum 2^-10) and in the subnormal range (quantum 2^-24)
    cases = {1.0 + 2.0 ** -11: 1.0, 1.0 + 3 * 2.0 ** -11: 1.0 + 2.0 ** -9, 2.0 ** -25: 0.0,
             3 * 2.0 ** -25: 2.0 ** -23, 65519.0: 65504.0, 65520.0: np.inf, -(1.0 + 2.0 ** -12): -1.0}
    for a, b in cases.items():
        assert philox.round_to(np.array([a]), "fp16")[0] == b
    # relative error at most 2^-11 in the normal range
    x = np.random.default_rng(4).standard_normal(1000)
    x = x[np.abs(x) >= 2.0 ** -14]
    r = philox.round_to(x, "fp16")
    assert np.all(np.abs(r - x) <= 2.0 ** -11 * np.abs(x) * 1.0000001)


def test_round_to_tf32_cases():
    # 1 + 2^-11 is a tie between 1 and 1 + 2^-10 -> even (1); 1 + 3*2^-11 -> 1 + 2^-9
    cases = {1.0 + 2.0 ** -11: 1.0, 1.0 + 3 * 2.0 ** -11: 1.0 + 2.0 ** -9,
             1.0 + 2.0 ** -10: 1.0 + 2.0 ** -10, -(1.0 + 2.0 ** -12): -1.0}
    for a, b in cases.items():
        assert philox.round_to(np.array([a]), "tf32")[0] == b
    x = np.random.default_rng(2).standard_normal(1000)
    r = philox.round_to(x, "tf32")
    assert np.all(np.abs(r - x) <= 2.0 ** -11 * np.abs(x) * 1.0000001)


# ---------------------------------------------------------------- QR / LS
@pytest.mark.parametrize("m,n", [(40, 9), (9, 9), (6, 13), (300, 16)])
def test_cpqr_matches_lapack_geqp3(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n)) * np.geomspace(1, 1e-3, n)[None, :]
    Q, R, piv = linalg.householder_cpqr(A)
    k = min(m, n)
    Qs, Rs, ps = scipy.linalg.qr(A, pivoting=True, mode="economic")
    np.testing.assert_array_equal(piv, ps)
    np.testing.assert_allclose(np.abs(R), np.abs(Rs[:k]), atol=1e-12 * np.abs(Rs).max())
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(Q @ R, A[:, piv], atol=1e-13 * np.abs(A).max())
    assert np.all(np.diag(R) >= 0)
    assert np.all(np.diff(np.abs(np.diag(R))) <= 1e-12)  # rank-revealing order


def test_cpqr_rank_deficient_and_ties():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 7))
    Q, R, piv = linalg.householder_cpqr(A)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-12)
    assert np.abs(R[3:, 3:]).max() < 1e-12 * np.abs(R).max()
    # exact ties: identical columns -> lowest index first
    B = np.tile(rng.standard_normal((10, 1)), (1, 4))
    _, _, pb = linalg.householder_cpqr(B)
    assert pb[0] == 0


def test_lstsq_right_matches_numpy():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((5, 12))
    S = rng.standard_normal((50, 12))
    H, rdiag = linalg.lstsq_right(S, B)
    ref = np.linalg.lstsq(B.T, S.T, rcond=None)[0].T
    np.testing.assert_allclose(H, ref, rtol=1e-11, atol=1e-12)
    assert np.all(rdiag > 0)


# ---------------------------------------------------------------- TT basics
def test_unfold_is_column_major_reshape():
    dims = [3, 4, 2, 5]
    x = np.arange(120, dtype=np.float64)
    for k in range(1, 4):
        Xk = tt.unfold(x, dims, k)
        for idx in [(0, 0, 0, 0), (2, 3, 1, 4), (1, 2, 0, 3)]:
            L = idx[0] + 3 * idx[1] + 12 * idx[2] + 24 * idx[3]
            Nk = int(np.prod(dims[:k]))
            assert Xk[L % Nk, L // Nk] == x[L]


def test_tt_full_matches_brute_force():
    dims, r = [3, 4, 2, 3], [1, 2, 3, 2, 1]
    cores = ti.random_tt_cores(dims, r, seed=9)
    full = tt.tt_full(cores)
    for L in range(full.size):
        rem, idx = L, []
        for n in dims:
            idx.append(rem % n)
            rem //= n
        v = np.ones((1, 1))
        for G, i in zip(cores, idx):
            v = v @ G[:, i, :]
        assert abs(full[L] - v[0, 0]) < 1e-12
    assert tt.tt_storage([g.shape for g in cores]) == 6 + 24 + 12 + 6


def test_table1_storage(golden):
    for d, n, ranks, gb, mb in golden("table1_sizes.txt"):
        d, n = int(d), int(n)
        r = [int(v) for v in ranks.split(",")]
        shapes = [(r[k], n, r[k + 1]) for k in range(d)]
        entries = tt.tt_storage(shapes)
        assert f"{entries * 8 / 2 ** 20:.3g}" == f"{float(mb):.3g}"
        assert f"{8 * n ** d / 2 ** 30:.3g}" == gb


def test_tt_svd_against_dense_svd():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((12, 9)) * np.geomspace(1, 1e-6, 9)[None, :] @ np.linalg.qr(rng.standard_normal((9, 9)))[0]
    x = A.ravel(order="F")
    cores = tt.tt_svd(x, [12, 9], eps=1e-3)
    s = np.linalg.svd(A, compute_uv=False)
    r = cores[0].shape[2]
    err = np.linalg.norm(tt.tt_full(cores) - x)
    assert abs(err - np.sqrt(np.sum(s[r:] ** 2))) < 1e-12 * s[0]
    assert err <= 1e-3 * np.linalg.norm(x)
    assert np.sqrt(np.sum(s[r - 1:] ** 2)) > 1e-3 * np.linalg.norm(x)  # minimal rank


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-8])
def test_tt_svd_error_bound(eps):
    dims = [6, 5, 4, 5]
    x = ti.random_tt(dims, [1, 3, 4, 3, 1], seed=1, noise=1e-5)
    cores = tt.tt_svd(x, dims, eps)
    assert np.linalg.norm(tt.tt_full(cores) - x) <= eps * np.linalg.norm(x) * (1 + 1e-12)


# ---------------------------------------------------------------- PSTT2
@pytest.mark.parametrize("passes", [1, 2])
def test_exact_recovery_config1(passes):
    dims = [16] * 4
    x = ti.random_tt(dims, [1, 3, 4, 3, 1], seed=0)
    o = P.pstt2(x, dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1, passes=passes)
    assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)
    assert [g.shape for g in o["cores"]] == [(1, 16, 4), (4, 16, 4), (4, 16, 4), (4, 16, 1)]


@pytest.mark.parametrize("d", [2, 3, 5, 6, 7])
@pytest.mark.parametrize("passes", [1, 2])
def test_exact_recovery_any_order(d, passes):
    dims = [4 + (k % 3) for k in range(d)]
    r = [1] + [2 + (k % 2) for k in range(d - 1)] + [1]
    x = ti.random_tt(dims, r, seed=d)
    o = P.pstt2(x, dims, ranks=[1] + [4] * (d - 1) + [1], p=3, seed=d + 10, passes=passes)
    assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)


def _proj_terms(x, dims, o):
    d = len(dims)
    ds = P.split_index(d)
    terms = []
    for k in range(1, d):
        Xk = tt.unfold(x, dims, k)
        if k < ds:
            Q = o["Q"][k]
            terms.append(np.linalg.norm(Xk - Q @ (Q.T @ Xk)) ** 2)
        else:
            Pk = o["P"][k]
            terms.append(np.linalg.norm(Xk - (Xk @ Pk) @ Pk.T) ** 2)
    return terms


@pytest.mark.parametrize("seed", range(6))
def test_twopass_deterministic_bound_eq_proj_acc(seed):
    """Theorem 3.2 (eq. proj_acc) with its row-space mirror, per run."""
    dims = [5, 6, 4, 5, 3]
    x = ti.random_tt(dims, [1, 4, 5, 5, 3, 1], seed=seed, noise=1e-2)
    o = P.pstt2(x, dims, ranks=[1, 2, 3, 3, 2, 1], p=2, seed=100 + seed, passes=2)
    err2 = np.linalg.norm(x - tt.tt_full(o["cores"])) ** 2
    assert err2 <= sum(_proj_terms(x, dims, o)) * (1 + 1e-10)


@pytest.mark.parametrize("seed", range(6))
def test_onepass_deterministic_bound(seed):
    """The one-pass bound of Theorem 3.3's proof: the middle term is replaced by
    ||Z_{d*} - X_{d*}||^2 with Z_{d*} = H P_{d*}^T."""
    dims = [5, 6, 4, 5]
    x = ti.random_tt(dims, [1, 4, 5, 3, 1], seed=seed, noise=1e-2)
    o = P.pstt2(x, dims, ranks=[1, 2, 3, 2, 1], p=3, seed=200 + seed, passes=1)
    d, ds = 4, 2
    terms = _proj_terms(x, dims, o)
    Xm = tt.unfold(x, dims, ds)
    terms[ds - 1] = np.linalg.norm(Xm - o["H"] @ o["P"][ds].T) ** 2
    err2 = np.linalg.norm(x - tt.tt_full(o["cores"])) ** 2
    assert err2 <= sum(terms) * (1 + 1e-10)


def test_d2_reduces_to_range_finder():
    """d = 2: two-pass PSTT2 is the randomized range finder on X^T; one-pass is
    S B^+ P^T (the pseudo-inverse form of eq. onepass_final_core)."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 25)) + 1e-3 * rng.standard_normal((30, 25))
    x = A.ravel(order="F")
    r, p = 4, 3
    o2 = P.pstt2(x, [30, 25], ranks=[1, r, 1], p=p, seed=3, passes=2)
    Psi = philox.test_matrix(3, 64 + 1, 30, r + p)
    Qs, _, _ = scipy.linalg.qr(A.T @ Psi, pivoting=True, mode="economic")
    Pr = Qs[:, :r]
    np.testing.assert_allclose(tt.tt_full(o2["cores"]), (A @ Pr @ Pr.T).ravel(order="F"), atol=1e-12)
    o1 = P.pstt2(x, [30, 25], ranks=[1, r, 1], p=p, seed=3, passes=1)
    Om = philox.test_matrix(3, 1, 25, r + p)
    H = (A @ Om) @ np.linalg.pinv(Pr.T @ Om)
    np.testing.assert_allclose(tt.tt_full(o1["cores"]), (H @ Pr.T).ravel(order="F"), atol=1e-11)


def test_expected_error_bound_eq_sketch_bound():
    """eq. (3.2): E||X - X~||^2 <= sum_j (1 + r_j/(p-1)) sum_{k>r_j} sigma_k^2(X_j),
    checked on a seed average (two-pass, where Theorem 3.2's bound applies)."""
    dims = [6, 5, 6]
    x = ti.random_tt(dims, [1, 5, 5, 1], seed=3, noise=5e-2)
    ranks = [1, 2, 2, 1]
    p = 3
    rhs = 0.0
    for k in (1, 2):
        s = np.linalg.svd(tt.unfold(x, dims, k), compute_uv=False)
        rhs += (1 + ranks[k] / (p - 1)) * np.sum(s[ranks[k]:] ** 2)
    errs = [np.linalg.norm(x - tt.tt_full(P.pstt2(x, dims, ranks=ranks, p=p, seed=s, passes=2)["cores"])) ** 2
            for s in range(40)]
    assert np.mean(errs) <= rhs


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_eps_mode_meets_tolerance(eps):
    dims = [8, 7, 6, 7, 8]
    x = ti.random_tt(dims, [1, 3, 4, 4, 3, 1], seed=4, noise=1e-7)
    for passes in (1, 2):
        o = P.pstt2(x, dims, eps=eps, rmax=8, p=6, seed=5, passes=passes)
        assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= eps * np.linalg.norm(x)
        assert o["r"][1:-1] == [3, 4, 4, 3]


def test_sketches_match_brute_force_sums():
    """Step 2 against the definition written as explicit sums over entries."""
    dims = [3, 2, 4, 2]
    x = ti.random_tt(dims, [1, 2, 2, 2, 1], seed=7)
    l = 3
    sk = P.sketches(x, dims, [None, l, l, l, l], seed=9, passes=1)
    N = tt.prods(dims)
    for k, S in sk["S"].items():
        Om = philox.test_matrix(9, k, N[4] // N[k], l)
        ref = np.zeros((N[k], l))
        for L in range(N[4]):
            ref[L % N[k]] += x[L] * Om[L // N[k]]
        np.testing.assert_allclose(S, ref, atol=1e-12)
    for k, R in sk["R"].items():
        Ps = philox.test_matrix(9, 64 + k, N[k], l)
        ref = np.zeros((N[4] // N[k], l))
        for L in range(N[4]):
            ref[L // N[k]] += x[L] * Ps[L % N[k]]
        np.testing.assert_allclose(R, ref, atol=1e-12)


def test_streaming_equals_one_shot():
    dims = [6, 5, 4, 7]
    x = ti.random_tt(dims, [1, 3, 3, 3, 1], seed=8, noise=1e-3)
    full = P.pstt2(x, dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2, passes=1)
    Nd1 = 6 * 5 * 4
    slabs = [(a, c, x[a * Nd1:(a + c) * Nd1]) for a, c in [(4, 3), (0, 2), (2, 2)]]
    st = P.pstt2_stream(slabs, dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2)
    np.testing.assert_allclose(tt.tt_full(st["cores"]), tt.tt_full(full["cores"]), atol=1e-12)


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """A plausible slip in core assembly (a transposed operand) or in the
    middle-core solve (a dropped pseudo-inverse) must break exact recovery."""
    dims = [5, 4, 6, 5]
    x = ti.random_tt(dims, [1, 2, 3, 2, 1], seed=1)
    good = P.pstt2(x, dims, ranks=[1, 3, 3, 3, 1], p=3, seed=4)
    assert np.linalg.norm(x - tt.tt_full(good["cores"])) < 1e-12 * np.linalg.norm(x)

    orig = P.outer_cores

    def swapped(dims_, r, Q, Pb):
        cores = orig(dims_, r, Q, Pb)
        d = len(dims_)
        cores[d - 1] = np.transpose(cores[d - 1], (2, 1, 0)).copy() if cores[d - 1].shape[0] == cores[d - 1].shape[2] else cores[d - 1][::-1].copy()
        return cores

    monkeypatch.setattr(P, "outer_cores", swapped)
    bad = P.pstt2(x, dims, ranks=[1, 3, 3, 3, 1], p=3, seed=4)
    assert np.linalg.norm(x - tt.tt_full(bad["cores"])) > 1e-3 * np.linalg.norm(x)
    monkeypatch.setattr(P, "outer_cores", orig)

    monkeypatch.setattr(P, "lstsq_right", lambda S, B: (S[:, :B.shape[0]], np.ones(B.shape[0])))
    bad2 = P.pstt2(x, dims, ranks=[1, 3, 3, 3, 1], p=3, seed=4)
    assert np.linalg.norm(x - tt.tt_full(bad2["cores"])) > 1e-3 * np.linalg.norm(x)


def test_hilbert_type_block_equals_slices_of_the_whole_tensor():
    """The sub-tensor generator used for sampled checks at full size gives the
    same values, entry for entry, as slicing the whole generated tensor."""
    d = [5, 4, 3, 6]
    x = ti.hilbert_type(d).reshape(d, order="F")
    b = ti.hilbert_type_block(d, [[2], None, [0, 2], None]).reshape((1, 4, 2, 6), order="F")
    assert np.array_equal(b, x[2:3, :, [0, 2], :])
    y = ti.hilbert_type(d, first_last=2, count_last=3).reshape((5, 4, 3, 3), order="F")
    assert np.array_equal(y, x[..., 2:5])


# ------------------------------------------------- one-sided PSTT-onepass
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_pstt_onepass_exact_recovery(d):
    """Exact TT ranks within the sketch: X~ = X to 1e-12 (every Q_j spans the
    column space of X_j, and the last core's least squares is consistent)."""
    from oracle import pstt as PO
    dims = [4 + (k % 3) for k in range(d)]
    r = [1] + [2 + (k % 2) for k in range(d - 1)] + [1]
    x = ti.random_tt(dims, r, seed=30 + d)
    o = PO.pstt_onepass(x, dims, ranks=[1] + [4] * (d - 1) + [1], p=3, seed=d + 40)
    assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)


def test_pstt_onepass_d2_closed_form():
    """d = 2: X~ = Q (Psi^T Q)^+ Psi^T X with Q the first r columns of a
    pivoted QR (LAPACK) of X Omega -- the one-pass range-finder form of
    eq. onepass_final_core, computed here without the oracle's code."""
    from oracle import pstt as PO
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 25)) + 1e-3 * rng.standard_normal((30, 25))
    r, p, seed = 4, 3, 5
    o = PO.pstt_onepass(A.ravel(order="F"), [30, 25], ranks=[1, r, 1], p=p, seed=seed)
    Om = philox.test_matrix(seed, 1, 25, r + p)
    Psi = philox.test_matrix(seed, 64 + 1, 30, r + p)
    Qs, _, _ = scipy.linalg.qr(A @ Om, pivoting=True, mode="economic")
    Q = Qs[:, :r]
    ref = Q @ np.linalg.lstsq(Psi.T @ Q, Psi.T @ A, rcond=None)[0]
    np.testing.assert_allclose(tt.tt_full(o["cores"]), ref.ravel(order="F"), atol=1e-11)


@pytest.mark.parametrize("seed", range(6))
def test_pstt_onepass_deterministic_bound(seed):
    """The bound of the one-pass theorem's proof, per run:
    ||X - X~||^2 <= sum_{j <= d-2} ||(I - Q_j Q_j^T) X_j||^2 + ||Z_{d-1} - X_{d-1}||^2
    with Z_{d-1} = Q_{d-1} (Psi^T Q_{d-1})^+ Psi^T X_{d-1} (formed here with lstsq)."""
    from oracle import pstt as PO
    dims = [5, 6, 4, 5]
    d = 4
    x = ti.random_tt(dims, [1, 4, 5, 3, 1], seed=seed, noise=1e-2)
    o = PO.pstt_onepass(x, dims, ranks=[1, 2, 3, 2, 1], p=3, seed=300 + seed)
    terms = []
    for j in range(1, d - 1):
        Xj = tt.unfold(x, dims, j)
        Qj = o["Q"][j]
        terms.append(np.linalg.norm(Xj - Qj @ (Qj.T @ Xj)) ** 2)
    Xl = tt.unfold(x, dims, d - 1)
    Ql = o["Q"][d - 1]
    Z = Ql @ np.linalg.lstsq(o["Psi"].T @ Ql, o["Psi"].T @ Xl, rcond=None)[0]
    terms.append(np.linalg.norm(Z - Xl) ** 2)
    err2 = np.linalg.norm(x - tt.tt_full(o["cores"])) ** 2
    assert err2 <= sum(terms) * (1 + 1e-10)


def test_pstt_onepass_expected_error_bound():
    """The one-pass theorem: E||X - X~||^2 <= sum_{j <= d-2} (1 + r_j/(p-1)) tail_j
    + (1 + r_{d-1}/(p-1))^2 tail_{d-1}, tail_j = sum_{k > r_j} sigma_k^2(X_j),
    on a seed average."""
    from oracle import pstt as PO
    dims = [6, 5, 6]
    x = ti.random_tt(dims, [1, 5, 5, 1], seed=3, noise=5e-2)
    ranks, p = [1, 2, 2, 1], 4
    rhs = 0.0
    for k in (1, 2):
        s = np.linalg.svd(tt.unfold(x, dims, k), compute_uv=False)
        f = (1 + ranks[k] / (p - 1)) ** (2 if k == 2 else 1)
        rhs += f * np.sum(s[ranks[k]:] ** 2)
    errs = [np.linalg.norm(x - tt.tt_full(PO.pstt_onepass(x, dims, ranks=ranks, p=p, seed=s)["cores"])) ** 2
            for s in range(40)]
    assert np.mean(errs) <= rhs


def test_pstt_onepass_sketches_match_brute_force():
    """The sketches it uses, entry by entry as sums over the tensor's entries
    (S_1 and T_{d-1} = Psi_{d-1}^T X_{d-1} at d = 3)."""
    from oracle import pstt as PO
    dims = [3, 4, 2]
    x = ti.random_tt(dims, [1, 2, 2, 1], seed=9)
    o = PO.pstt_onepass(x, dims, ranks=[1, 2, 2, 1], p=2, seed=4)
    X = x.reshape(dims, order="F")
    Om1 = philox.test_matrix(4, 1, 8, 4)
    Ps2 = philox.test_matrix(4, 64 + 2, 12, 4)
    for i1 in range(3):
        for j in range(4):
            ref = sum(X[i1, i2, i3] * Om1[i2 + 4 * i3, j] for i2 in range(4) for i3 in range(2))
            assert abs(o["S"][1][i1, j] - ref) <= 1e-12 * (1 + abs(ref))
    for j in range(4):
        for i3 in range(2):
            ref = sum(Ps2[i1 + 3 * i2, j] * X[i1, i2, i3] for i1 in range(3) for i2 in range(4))
            assert abs(o["T"][j, i3] - ref) <= 1e-12 * (1 + abs(ref))


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_pstt_twopass_exact_recovery(d):
    from oracle import pstt as PO
    dims = [4 + (k % 3) for k in range(d)]
    r = [1] + [2 + (k % 2) for k in range(d - 1)] + [1]
    x = ti.random_tt(dims, r, seed=50 + d)
    o = PO.pstt(x, dims, ranks=[1] + [4] * (d - 1) + [1], p=3, seed=d + 60)
    assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("seed", range(6))
def test_pstt_twopass_deterministic_bound_eq_proj_acc(seed):
    """Algorithm 2 has Q_j with ON columns for every j, so eq. (proj_acc)
    bounds its error by the projection tails, per run."""
    from oracle import pstt as PO
    dims = [5, 6, 4, 5]
    x = ti.random_tt(dims, [1, 4, 5, 3, 1], seed=seed, noise=1e-2)
    o = PO.pstt(x, dims, ranks=[1, 2, 3, 2, 1], p=2, seed=400 + seed)
    terms = [np.linalg.norm(tt.unfold(x, dims, j) - o["Q"][j] @ (o["Q"][j].T @ tt.unfold(x, dims, j))) ** 2
             for j in range(1, 4)]
    err2 = np.linalg.norm(x - tt.tt_full(o["cores"])) ** 2
    assert err2 <= sum(terms) * (1 + 1e-10)


def test_pstt_twopass_expected_error_bound():
    """Theorem 3.3, eq. (sketch_bound), for Algorithm 2 on a seed average."""
    from oracle import pstt as PO
    dims = [6, 5, 6]
    x = ti.random_tt(dims, [1, 5, 5, 1], seed=3, noise=5e-2)
    ranks, p = [1, 2, 2, 1], 3
    rhs = 0.0
    for k in (1, 2):
        s = np.linalg.svd(tt.unfold(x, dims, k), compute_uv=False)
        rhs += (1 + ranks[k] / (p - 1)) * np.sum(s[ranks[k]:] ** 2)
    errs = [np.linalg.norm(x - tt.tt_full(PO.pstt(x, dims, ranks=ranks, p=p, seed=s)["cores"])) ** 2
            for s in range(40)]
    assert np.mean(errs) <= rhs


# ------------------------------------------------------------- Tucker2TT
def _tucker_tensor(s, n, tt_ranks, seed):
    rng = np.random.default_rng(seed)
    G = ti.random_tt(s, tt_ranks, seed=seed)
    A = [np.linalg.qr(rng.standard_normal((nk, sk)))[0] for nk, sk in zip(n, s)]
    X = G.reshape(s, order="F")
    for k, Ak in enumerate(A):  # dense mode-k products, written independently of the oracle
        X = np.moveaxis(np.tensordot(Ak, X, axes=([1], [k])), 0, k)
    return G, A, X.reshape(-1, order="F")


@pytest.mark.parametrize("passes", [1, 2])
def test_tucker2tt_exact_for_exact_core_ranks(passes):
    """Algorithm 3: a Tucker tensor whose core has exact TT ranks within the
    sketch is reproduced to 1e-12 without forming X."""
    from oracle import tucker as TU
    s, n = [4, 5, 3, 4], [9, 7, 8, 6]
    G, A, X = _tucker_tensor(s, n, [1, 2, 3, 2, 1], seed=21)
    cores, o = TU.tucker2tt(G, A, ranks=[1, 3, 3, 3, 1], p=3, seed=7, passes=passes)
    assert [c.shape[1] for c in cores] == n
    assert np.linalg.norm(tt.tt_full(cores) - X) <= 1e-12 * np.linalg.norm(X)


def test_tucker2tt_ranks_lemma_and_error_equality():
    """The lemma after Algorithm 3 (rank X_j = rank G_j for ON factors), and
    ||X - X~|| = ||G - G~|| (the factors are isometries)."""
    from oracle import tucker as TU
    s, n = [5, 4, 6], [9, 8, 10]
    G, A, X = _tucker_tensor(s, n, [1, 4, 3, 1], seed=22)
    G = G + 1e-3 * np.random.default_rng(3).standard_normal(G.size)
    Xn = G.reshape(s, order="F")
    for k, Ak in enumerate(A):
        Xn = np.moveaxis(np.tensordot(Ak, Xn, axes=([1], [k])), 0, k)
    X = Xn.reshape(-1, order="F")
    for j in (1, 2):
        assert np.linalg.matrix_rank(tt.unfold(X, n, j), tol=1e-10) == \
            np.linalg.matrix_rank(tt.unfold(G, s, j), tol=1e-10)
    cores, o = TU.tucker2tt(G, A, ranks=[1, 2, 2, 1], p=3, seed=8)
    eX = np.linalg.norm(tt.tt_full(cores) - X)
    eG = np.linalg.norm(tt.tt_full(o["cores"]) - G)
    assert abs(eX - eG) <= 1e-12 * np.linalg.norm(X)


def test_mode2_product_matches_dense_mode_product():
    """T_j = H_j x_2 A_j: contracting the new train equals the dense mode-j
    products of the core train's full tensor."""
    from oracle import tucker as TU
    rng = np.random.default_rng(5)
    s, n, r = [3, 4, 2], [5, 6, 7], [1, 2, 3, 1]
    H = [rng.standard_normal((r[k], s[k], r[k + 1])) for k in range(3)]
    A = [rng.standard_normal((n[k], s[k])) for k in range(3)]
    Xg = tt.tt_full(H).reshape(s, order="F")
    for k, Ak in enumerate(A):
        Xg = np.moveaxis(np.tensordot(Ak, Xg, axes=([1], [k])), 0, k)
    got = tt.tt_full([TU.mode2(Hk, Ak) for Hk, Ak in zip(H, A)])
    np.testing.assert_allclose(got, Xg.reshape(-1, order="F"), rtol=0, atol=1e-12)


def test_tt2tucker_exact_and_orthonormal():
    """Algorithm 4 with t_k >= rank (T_k)_(2): the Tucker format reproduces the
    TT tensor to 1e-12 (X = TT(H) x_1 A_1 ... x_d A_d, formed with dense mode
    products), every A_k has orthonormal columns, H_k = T_k x_2 A_k^T."""
    from oracle import tucker as TU
    rng = np.random.default_rng(11)
    n, r = [9, 8, 10, 7], [1, 2, 3, 2, 1]
    T = [rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(4)]
    Hs, As = TU.tt2tucker(T, [r[k] * r[k + 1] for k in range(4)], p=3, seed=5)
    X = tt.tt_full(T)
    Xt = tt.tt_full(Hs).reshape([A.shape[1] for A in As], order="F")
    for k, A in enumerate(As):
        np.testing.assert_allclose(A.T @ A, np.eye(A.shape[1]), atol=1e-12)
        np.testing.assert_allclose(Hs[k], TU.mode2(T[k], A.T), atol=1e-12)
        Xt = np.moveaxis(np.tensordot(A, Xt, axes=([1], [k])), 0, k)
    assert np.linalg.norm(Xt.reshape(-1, order="F") - X) <= 1e-12 * np.linalg.norm(X)


def test_tt2tucker_truncation_error_is_the_projection_error():
    """With orthonormal cores to the left and right of core k (a train in
    mixed-canonical form at k), truncating only A_k costs exactly
    ||(I - A_k A_k^T)(T_k)_(2)||_F."""
    from oracle import tucker as TU
    rng = np.random.default_rng(12)
    n, r = [6, 12, 5], [1, 4, 4, 1]
    T0 = np.linalg.qr(rng.standard_normal((n[0], r[1])))[0].reshape((1, n[0], r[1]), order="F")
    T2 = np.linalg.qr(rng.standard_normal((n[2], r[2])))[0].T.reshape((r[2], n[2], 1), order="F")
    T1 = rng.standard_normal((r[1], n[1], r[2]))
    T = [T0, T1, T2]
    Hs, As = TU.tt2tucker(T, [n[0], 5, n[2]], p=4, seed=9)
    Xt = tt.tt_full(Hs).reshape([A.shape[1] for A in As], order="F")
    for k, A in enumerate(As):
        Xt = np.moveaxis(np.tensordot(A, Xt, axes=([1], [k])), 0, k)
    err = np.linalg.norm(Xt.reshape(-1, order="F") - tt.tt_full(T))
    M = TU.unfold2(T1)
    proj = np.linalg.norm(M - As[1] @ (As[1].T @ M))
    assert abs(err - proj) <= 1e-12 * np.linalg.norm(M)
    assert proj > 0


# ------------------------------------------------- Khatri-Rao test matrices
def _modewise_column_sketch(x, dims, k, F):
    """X_k (F_d (.) ... (.) F_{k+1}) evaluated as eq. (sketch_orig) writes it:
    for every multi-index (l_{k+2}, ..., l_d) the N_k x n_{k+1} block of X_k with
    those indices, times F_{k+1}, times the diagonal matrices of rows l_q of
    F_q, summed -- the Khatri-Rao product is never formed."""
    d = len(dims)
    N = tt.prods(dims)
    nk1 = dims[k]
    rest = dims[k + 1:]
    Xk = tt.unfold(x, dims, k).reshape((N[k], nk1, int(np.prod(rest)) if rest else 1), order="F")
    l = F[k + 1].shape[1]
    out = np.zeros((N[k], l))
    for b, idx in enumerate(np.ndindex(*reversed(rest)) if rest else [()]):
        idx = tuple(reversed(idx))  # (l_{k+2}, ..., l_d), column-major block order
        diag = np.ones(l)
        for q, lq in zip(range(k + 2, d + 1), idx):
            diag = diag * F[q][lq]
        out += (Xk[:, :, b] @ F[k + 1]) * diag[None, :]
    return out


def _modewise_row_sketch(x, dims, k, F):
    """The row-space mirror (X_k^T (F_k (.) ... (.) F_1)): blocks of X_k^T with
    fixed (l_1, ..., l_{k-1}) times F_k, scaled by the rows l_q of F_q."""
    N = tt.prods(dims)
    d = len(dims)
    Xk = tt.unfold(x, dims, k)           # rows (i_1..i_k), i_1 fastest
    lead = dims[:k - 1]
    nk = dims[k - 1]
    Xr = Xk.reshape((N[k - 1], nk, N[d] // N[k]), order="F")
    l = F[k].shape[1]
    out = np.zeros((N[d] // N[k], l))
    for a, idx in enumerate(np.ndindex(*reversed(lead)) if lead else [()]):
        idx = tuple(reversed(idx))  # (l_1, ..., l_{k-1})
        diag = np.ones(l)
        for q, lq in zip(range(1, k), idx):
            diag = diag * F[q][lq]
        out += (Xr[a].T @ F[k]) * diag[None, :]
    return out


@pytest.mark.parametrize("dims", [[3, 4, 2, 3], [2, 3, 2, 3, 2]])
def test_kr_sketches_equal_modewise_products_eq_sketch_orig(dims):
    """The oracle's Khatri-Rao sketches (dense product with the materialised
    test matrix) against eq. (sketch_orig)'s mode-by-mode evaluation with the
    same factors; a Khatri-Rao product with the mode order reversed fails."""
    d = len(dims)
    x = ti.random_tt(dims, [1] + [2] * (d - 1) + [1], seed=11, noise=1e-2)
    l, seed = 5, 13
    sk = P.sketches(x, dims, [None] + [l] * d, seed, 1, drm="kr")
    ds = P.split_index(d)
    for k, S in sk["S"].items():
        F = {q: philox.kr_factor(seed, k, q, dims[q - 1], l) for q in range(k + 1, d + 1)}
        np.testing.assert_allclose(S, _modewise_column_sketch(x, dims, k, F), rtol=1e-12, atol=1e-12)
        if d - k >= 2:
            bad = philox.kr_test_matrix(seed, k, list(range(d, k, -1)), dims[k:][::-1], l)
            assert np.abs(tt.unfold(x, dims, k) @ bad - S).max() > 1e-3
    for k, R in sk["R"].items():
        F = {q: philox.kr_factor(seed, 64 + k, q, dims[q - 1], l) for q in range(1, k + 1)}
        np.testing.assert_allclose(R, _modewise_row_sketch(x, dims, k, F), rtol=1e-12, atol=1e-12)
    assert ds in sk["S"]


def test_kr_factor_rows_are_not_dense_rows():
    """A factor row is a Gaussian row of the same stream at a counter no dense
    test matrix uses (row-high word with the top bit set)."""
    f = philox.kr_factor(5, 3, 2, 7, 6)
    g = philox.gaussian(5, 3, np.arange(7, dtype=np.uint64) + np.uint64((0x80000000 + 2) << 32), 6)
    np.testing.assert_array_equal(f, g)
    dense = philox.test_matrix(5, 3, 7, 6)
    assert not np.any(np.isclose(f, dense))


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("passes", [1, 2])
def test_kr_exact_recovery(d, passes):
    """With target ranks at least the TT ranks, PSTT2 with Khatri-Rao test
    matrices reproduces X (the sketches span the unfoldings' ranges with
    probability one, as with dense Gaussians)."""
    dims = [4 + (k % 3) for k in range(d)]
    r = [1] + [2 + (k % 2) for k in range(d - 1)] + [1]
    x = ti.random_tt(dims, r, seed=d + 20)
    o = P.pstt2(x, dims, ranks=[1] + [4] * (d - 1) + [1], p=3, seed=d + 30, passes=passes, drm="kr")
    assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)


def test_kr_config1_exact_and_different_from_dense():
    dims = [16] * 4
    x = ti.random_tt(dims, [1, 3, 4, 3, 1], seed=0)
    o = P.pstt2(x, dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1, drm="kr")
    g = P.pstt2(x, dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1)
    assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)
    assert np.abs(o["sketch"]["S"][1] - g["sketch"]["S"][1]).max() > 1e-3


def test_kr_d2_is_the_range_finder_with_the_factor():
    """d = 2: each test matrix has a single factor, so PSTT2 with Khatri-Rao
    test matrices is the randomized range finder with those n x l Gaussian
    factors (two-pass: A P P^T with P from the pivoted QR of A^T F)."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((20, 5)) @ rng.standard_normal((5, 18)) + 1e-3 * rng.standard_normal((20, 18))
    x = A.ravel(order="F")
    r, p = 4, 3
    o2 = P.pstt2(x, [20, 18], ranks=[1, r, 1], p=p, seed=4, passes=2, drm="kr")
    Fp = philox.kr_factor(4, 64 + 1, 1, 20, r + p)
    Qs, _, _ = scipy.linalg.qr(A.T @ Fp, pivoting=True, mode="economic")
    Pr = Qs[:, :r]
    np.testing.assert_allclose(tt.tt_full(o2["cores"]), (A @ Pr @ Pr.T).ravel(order="F"), atol=1e-12)
    o1 = P.pstt2(x, [20, 18], ranks=[1, r, 1], p=p, seed=4, passes=1, drm="kr")
    Fo = philox.kr_factor(4, 1, 2, 18, r + p)
    H = (A @ Fo) @ np.linalg.pinv(Pr.T @ Fo)
    np.testing.assert_allclose(tt.tt_full(o1["cores"]), (H @ Pr.T).ravel(order="F"), atol=1e-11)


@pytest.mark.parametrize("seed", range(4))
def test_kr_twopass_deterministic_bound_eq_proj_acc(seed):
    """Theorem 3.2's bound holds for any test matrices, Khatri-Rao included."""
    dims = [5, 6, 4, 5, 3]
    x = ti.random_tt(dims, [1, 4, 5, 5, 3, 1], seed=seed, noise=1e-2)
    o = P.pstt2(x, dims, ranks=[1, 2, 3, 3, 2, 1], p=2, seed=300 + seed, passes=2, drm="kr")
    err2 = np.linalg.norm(x - tt.tt_full(o["cores"])) ** 2
    assert err2 <= sum(_proj_terms(x, dims, o)) * (1 + 1e-10)


def test_kr_streaming_equals_one_shot():
    dims = [6, 5, 4, 7]
    x = ti.random_tt(dims, [1, 3, 3, 3, 1], seed=8, noise=1e-3)
    full = P.pstt2(x, dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2, passes=1, drm="kr")
    Nd1 = 6 * 5 * 4
    slabs = [(a, c, x[a * Nd1:(a + c) * Nd1]) for a, c in [(4, 3), (0, 2), (2, 2)]]
    st = P.pstt2_stream(slabs, dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2, drm="kr")
    np.testing.assert_allclose(tt.tt_full(st["cores"]), tt.tt_full(full["cores"]), atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_kr_one_sided_exact_recovery(d):
    """Algorithm 2 and PSTT-onepass with Khatri-Rao DRMs (the paper's
    substitute for the dense Phi_j) reproduce a random TT of lower rank."""
    dims = [5 + (k % 2) for k in range(d)]
    r = [1] + [2 + (k % 2) for k in range(d - 1)] + [1]
    x = ti.random_tt(dims, r, seed=d + 40)
    tgt = [1] + [4] * (d - 1) + [1]
    from oracle import pstt as PS
    for fn in (PS.pstt_onepass, PS.pstt):
        o = fn(x, dims, ranks=tgt, p=3, seed=d + 50, drm="kr")
        assert np.linalg.norm(x - tt.tt_full(o["cores"])) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
def test_kr_last_row_sketch_mode_by_mode_in_rounded_arithmetic(fmt):
    """The rounded Khatri-Rao Psi_{d-1} of the mixed paths equals eq.
    (sketch_orig)'s mode-by-mode evaluation: each block X(:, w, :)^T times the
    rounded mode-1 factor, scaled column-wise by the rounded product of the
    other modes' rows for that block, summed over the blocks."""
    dims = [5, 3, 4, 6]
    d = len(dims)
    x = ti.random_tt(dims, [1, 2, 2, 2, 1], seed=3, noise=1e-2)
    l, seed = 6, 21
    sk = P.sketches(x, dims, [None] + [l] * d, seed, 1, test_fmt=fmt, drm="kr")
    s = 64 + d - 1
    F1 = philox.round_to(philox.kr_factor(seed, s, 1, dims[0], l), fmt)
    F2 = philox.kr_factor(seed, s, 2, dims[1], l)
    F3 = philox.kr_factor(seed, s, 3, dims[2], l)
    X = x.reshape(dims, order="F")
    ref = np.zeros((dims[3], l))
    for i2 in range(dims[1]):
        for i3 in range(dims[2]):
            scale = philox.round_to(F3[i3] * F2[i2], fmt)
            ref += (X[:, i2, i3, :].T @ F1) * scale[None, :]
    np.testing.assert_allclose(sk["R"][d - 1], ref, rtol=1e-12, atol=1e-12)
    # entries are products of two rounded numbers: exact in FP32, not in fmt
    Ps = sk["Psi"][d - 1]
    assert np.array_equal(Ps.astype(np.float32).astype(np.float64), Ps)
    assert not np.array_equal(philox.round_to(Ps, fmt), Ps)
