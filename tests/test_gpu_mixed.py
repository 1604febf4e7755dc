"""GPU parity of the mixed-precision (TF32 / BF16 / FP16 tensor-core) sketch path.

Bars (derived from the arithmetic):
* test-matrix entries: the FP32 generator differs from the FP64 definition by
  about 1e-7 relative (at most ~1e-5 absolute, only where u is within 1e-5 of
  1 so that |z| is tiny), so after rounding to the MMA type an entry equals
  the oracle's rounded FP64 normal except for rare flips to the neighbouring
  value (< 0.5% of entries, at most one ulp plus 2e-5 absolute);
* sketches: equal to the oracle's FP64 product of the split X (hi + lo in the
  MMA type) with its rounded test matrix; the flips above change a sketch
  entry by about 2^-8 |x w| (BF16), which bounds the relative Frobenius
  difference by 1e-4 and the max-norm difference by 2e-3 of max |S| (FP32
  accumulation inside a tile adds ~1e-7).  FP16 plans split X 2^s (s from
  the largest |X|, the rule of tt_x_scale_log2) and their sketches hold 2^s
  times the values until the finalize: the tests scale them back;
* reconstruction: within 10 eps of the FP64 oracle (relative Frobenius), the
  precision form's stated target.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import philox, pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch, _native as N
from tests.gpu_util import rel, sketch_dict, to_dev

pytestmark = pytest.mark.gpu

PREC = {"tf32": N.TT_PREC_TF32, "bf16": N.TT_PREC_BF16, "fp16": N.TT_PREC_FP16}
ULP = {"tf32": 2.0 ** -10, "bf16": 2.0 ** -7, "fp16": 2.0 ** -10}


def _scale_of(x):
    """FP16 scale exponent: 15 - e with 2^(e-1) <= max |x| < 2^e."""
    m = float(np.max(np.abs(x)))
    return 0 if m == 0.0 else 15 - int(np.frexp(m)[1])


def _mk(dims, prec, x, **kw):
    """TTSketch of precision prec; FP16 plans get the scale of x.  Returns
    (plan, s)."""
    s = _scale_of(x) if prec == "fp16" else 0
    return TTSketch(dims, x_dtype=torch.float32, prec=prec, x_scale_log2=s, **kw), s


def _sketches(t, s):
    """The sketches read between accumulate and finalize, at the scale of X."""
    return {k: v * 2.0 ** -s for k, v in sketch_dict(t).items()}


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16"])
def test_test_matrix_mixed_matches_rounded_oracle(prec):
    nrows, ncols, sid = 20000, 26, 5
    out = torch.empty(nrows * ncols, dtype=torch.float64, device="cuda")
    N.check(N.lib().tt_test_matrix(3, sid, 17, nrows, ncols, PREC[prec], C.c_void_p(out.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream)), "tm")
    got = out.cpu().numpy().reshape(ncols, nrows).T
    ref = philox.round_to(philox.gaussian(3, sid, np.arange(17, 17 + nrows, dtype=np.uint64), ncols), prec)
    diff = np.abs(got - ref)
    assert np.all(diff <= ULP[prec] * np.abs(ref) * 1.0001 + 2e-5)
    assert np.mean(diff > 0) < 5e-3
    assert np.array_equal(philox.round_to(got, prec), got)  # values are exact in the MMA type


def _close_sketch(G, S, what):
    fro = np.linalg.norm(G - S) / np.linalg.norm(S)
    mx = np.max(np.abs(G - S)) / np.max(np.abs(S))
    assert fro <= 1e-4 and mx <= 2e-3, (what, fro, mx)


def _split(x, prec, s=0):
    """X as the sketch kernels see it: hi + lo of X 2^s in the MMA type, at the
    scale of X (s only for FP16)."""
    s = s if prec == "fp16" else 0
    xs = np.asarray(x, dtype=np.float64) * 2.0 ** s
    hi = philox.round_to(xs, prec)
    lo = philox.round_to(xs - hi, prec)
    return (hi + lo) * 2.0 ** -s


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16"])
@pytest.mark.parametrize("dims,r", [([40, 7, 6, 70], [1, 4, 5, 4, 1]), ([9, 8, 7, 6, 5, 9], [1, 5, 6, 6, 5, 5, 1]),
                                    ([130, 100], [1, 6, 1])])
def test_mixed_sketches_match_oracle(prec, dims, r):
    x = ti.random_tt(dims, r, seed=2, noise=1e-6).astype(np.float32)
    target = [1] + [v for v in r[1:-1]] + [1]
    t, s = _mk(dims, prec, x, ranks=target, p=6, seed=4)
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = _sketches(t, s)
    t.finalize()
    xs = _split(x.astype(np.float64), prec, s)
    o = OP.pstt2(xs, dims, ranks=target, p=6, seed=4, passes=1, test_fmt=prec)
    for k, S in o["sketch"]["S"].items():
        _close_sketch(sk[(0, k)], S, ("S", k))
    for k, R in o["sketch"]["R"].items():
        _close_sketch(sk[(1, k)], R, ("R", k))
    st, _ = t.status()
    assert st == 0


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16"])
@pytest.mark.parametrize("case", ["config2_small", "config3_small"])
def test_mixed_within_10eps_of_oracle(prec, case):
    if case == "config2_small":
        dims, eps, p, rmax = [9] * 6, 1e-5, 10, 16
        x = ti.random_tt(dims, [1, 9, 10, 10, 10, 9, 1], seed=0, noise=1e-6).astype(np.float32)
    else:
        dims, eps, p, rmax = [32] * 4, 1e-6, 10, 6
        x = ti.hilbert_type(dims, np.float32)
    x64 = x.astype(np.float64)
    t = _mk(dims, prec, x, eps=eps, rmax=rmax, p=p, seed=1)[0].pstt2(to_dev(x))
    f = TTSketch(dims, eps=eps, rmax=rmax, p=p, seed=1, x_dtype=torch.float32, prec="fp64").pstt2(to_dev(x))
    o = OP.pstt2(x64, dims, eps=eps, rmax=rmax, p=p, seed=1)
    xt = t.reconstruct().cpu().numpy()
    ref = OT.tt_full(o["cores"])
    e_or = rel(xt, ref, x64)
    e_x = rel(xt, x64, x64)
    e_f = rel(xt, f.reconstruct().cpu().numpy(), x64)
    print(f"{case} {prec}: |X~-X~oracle|={e_or:.2e} |X~-X|={e_x:.2e} |X~-X~fp64gpu|={e_f:.2e} ranks={t.status()[1]}")
    assert e_or <= 10 * eps
    assert e_x <= 10 * eps
    assert e_f <= 10 * eps


def test_mixed_streaming_equals_one_shot():
    dims = [24, 10, 12, 20]
    x = ti.random_tt(dims, [1, 3, 4, 3, 1], seed=6, noise=1e-5).astype(np.float32)
    X = to_dev(x)
    one = TTSketch(dims, ranks=[1, 3, 4, 3, 1], p=5, seed=3, prec="bf16").pstt2(X)
    t = TTSketch(dims, ranks=[1, 3, 4, 3, 1], p=5, seed=3, prec="bf16")
    Nd1 = 24 * 10 * 12
    t.begin()
    for first, cnt in [(12, 8), (0, 5), (5, 7)]:
        t.accumulate(X[first * Nd1:(first + cnt) * Nd1].clone(), first, cnt)
    t.finalize()
    # FP32 tile partials differ when the slabs cut the tiles differently
    assert rel(one.reconstruct().cpu().numpy(), t.reconstruct().cpu().numpy(), x) <= 1e-6


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16"])
def test_generic_staged_rows_streaming_match_oracle(prec):
    # n_1 = 70, n_d = 45: the generic tile kernel with staged test-matrix rows
    # (column side: 2 row tiles of i_1 read each row; row side: planes and
    # column tiles), slabs that cut the 32-wide tiles of i_d raggedly
    dims, r = [70, 3, 5, 45], [1, 4, 5, 4, 1]
    x = ti.random_tt(dims, r, seed=8, noise=1e-6).astype(np.float32)
    X = to_dev(x)
    Nd1 = 70 * 3 * 5
    t, s = _mk(dims, prec, x, ranks=r, p=6, seed=9)
    assert t.kernel_kind(15) == 1
    t.begin()
    for first, cnt in [(30, 15), (0, 13), (13, 17)]:
        t.accumulate(X[first * Nd1:(first + cnt) * Nd1].clone(), first, cnt)
    sk = _sketches(t, s)
    t.finalize()
    o = OP.pstt2(_split(x.astype(np.float64), prec, s), dims, ranks=r, p=6, seed=9, passes=1, test_fmt=prec)
    for k, S in o["sketch"]["S"].items():
        _close_sketch(sk[(0, k)], S, ("S", k))
    for k, R in o["sketch"]["R"].items():
        _close_sketch(sk[(1, k)], R, ("R", k))


# ----------------------------------------------------------- tcgen05 kernel
@pytest.mark.parametrize("dims,kw", [
    ([128, 5, 6, 128], dict(ranks=[1, 4, 4, 4, 1], p=4)),            # ragged tiles (5 x 6 planes), l = 8
    ([256, 3, 4, 256], dict(eps=1e-6, rmax=6, p=10)),               # two halves per side, l = 16
    ([256, 7, 128], dict(ranks=[1, 4, 4, 1], p=12)),                # d = 3
])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tcgen05_sketches_match_oracle(dims, kw, prec):
    x = ti.random_tt(dims, [1] + [3] * (len(dims) - 1) + [1], seed=5, noise=1e-5).astype(np.float32)
    t, s = _mk(dims, prec, x, seed=7, **kw)
    assert t.kernel_kind() == 2
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = _sketches(t, s)
    t.finalize()
    st, ranks = t.status()
    assert st in (0, N.TT_WARN_RANK_CAP)
    xs = _split(x.astype(np.float64), prec, s)
    o = OP.pstt2(xs, dims, seed=7, passes=1, test_fmt=prec, **kw)
    for k, S in o["sketch"]["S"].items():
        _close_sketch(sk[(0, k)], S, ("S", k))
    for k, R in o["sketch"]["R"].items():
        _close_sketch(sk[(1, k)], R, ("R", k))


def test_tcgen05_slab_groups_equal_one_shot():
    dims = [128, 3, 2, 256]
    x = ti.random_tt(dims, [1, 3, 3, 2, 1], seed=8, noise=1e-5).astype(np.float32)
    X = to_dev(x)
    one = TTSketch(dims, ranks=[1, 3, 3, 3, 1], p=5, seed=3, prec="bf16")
    assert one.kernel_kind(256) == 2 and one.kernel_kind(128) == 2 and one.kernel_kind(16) == 1
    one.pstt2(X)
    t = TTSketch(dims, ranks=[1, 3, 3, 3, 1], p=5, seed=3, prec="bf16")
    Nd1 = 128 * 3 * 2
    t.begin()
    t.accumulate(X[128 * Nd1:].clone(), 128, 128)
    t.accumulate(X[:128 * Nd1].clone(), 0, 128)
    t.finalize()
    assert rel(one.reconstruct().cpu().numpy(), t.reconstruct().cpu().numpy(), x) <= 1e-6


def test_tcgen05_hilbert_within_10eps():
    dims = [256, 8, 8, 256]
    x = ti.hilbert_type(dims, np.float32)
    t = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="bf16")
    assert t.kernel_kind() == 2
    t.pstt2(to_dev(x))
    f = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="fp64").pstt2(to_dev(x))
    x64 = x.astype(np.float64)
    e_x = rel(t.reconstruct().cpu().numpy(), x64, x64)
    e_f = rel(t.reconstruct().cpu().numpy(), f.reconstruct().cpu().numpy(), x64)
    print(f"tcgen05 hilbert: |X~-X|={e_x:.2e} |X~-X~fp64|={e_f:.2e} ranks={t.status()[1]}")
    assert e_x <= 1e-5 and e_f <= 1e-5


def _sampled_sketch_check(dims, kw, nsamp=6, seed=7):
    """Sketch entries of a multi-tile launch, each computed one by one by the
    oracle (FP64 sums over the whole tensor with the rounded test-matrix rows
    and the split X), at the shapes where CTAs process several tiles."""
    n1, n2, n3, n4 = dims
    Xd = torch.empty(n1 * n2 * n3 * n4, dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, n4, C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    t = TTSketch(dims, seed=seed, prec="bf16", **kw)
    assert t.kernel_kind() == 2
    t.begin()
    t.accumulate(Xd, 0, n4)
    sk = sketch_dict(t)
    x = ti.hilbert_type(dims, np.float32).astype(np.float64)
    xs = _split(x, "bf16").reshape((n1, n2, n3, n4), order="F")
    rng = np.random.default_rng(0)
    l = sk[(0, 1)].shape[1]
    bf = lambda A: philox.round_to(A, "bf16")
    errs = {}
    for _ in range(nsamp):
        i1, i2, i3, i4 = [int(rng.integers(v)) for v in dims]
        # S_1(i1, :) = sum_{i2,i3,i4} X Omega_1[(i2,i3,i4)]
        Om1 = bf(philox.test_matrix(seed, 1, n2 * n3 * n4, l))
        ref = xs[i1].reshape(-1, order="F") @ Om1
        errs.setdefault("S1", []).append(np.abs(sk[(0, 1)][i1] - ref).max() / np.abs(ref).max())
        # S_2(i1 + n1 i2, :) = sum_{i3,i4} X Omega_2[(i3,i4)]
        Om2 = bf(philox.test_matrix(seed, 2, n3 * n4, l))
        ref = xs[i1, i2].reshape(-1, order="F") @ Om2
        errs.setdefault("S2", []).append(np.abs(sk[(0, 2)][i1 + n1 * i2] - ref).max() / np.abs(ref).max())
        # R_2(i3 + n3 i4, :) = sum_{i1,i2} X Psi_2[(i1,i2)]
        Ps2 = bf(philox.test_matrix(seed, 66, n1 * n2, l))
        ref = xs[:, :, i3, i4].reshape(-1, order="F") @ Ps2
        errs.setdefault("R2", []).append(np.abs(sk[(1, 2)][i3 + n3 * i4] - ref).max() / np.abs(ref).max())
        # R_3(i4, :) = sum_{i1,i2,i3} X Psi_3[(i1,i2,i3)]
        Ps3 = bf(philox.test_matrix(seed, 67, n1 * n2 * n3, l))
        ref = xs[:, :, :, i4].reshape(-1, order="F") @ Ps3
        errs.setdefault("R3", []).append(np.abs(sk[(1, 3)][i4] - ref).max() / np.abs(ref).max())
    return {k: max(v) for k, v in errs.items()}


@pytest.mark.parametrize("dims", [[256, 64, 48, 256], [128, 64, 96, 128]])
def test_tcgen05_multitile_sampled_entries(dims):
    """Several tiles per CTA (the run-change flush and the double-buffered row
    accumulators are exercised); entries within the flip bound of the oracle."""
    e = _sampled_sketch_check(dims, dict(eps=1e-6, rmax=6, p=10))
    print("multi-tile sampled max rel err:", e)
    assert all(v <= 2e-3 for v in e.values()), e


@pytest.mark.parametrize("dims", [[256, 64, 48, 256], [128, 64, 96, 128]])
def test_tcgen05_multitile_pipeline_within_10eps(dims):
    """The whole one-pass pipeline at multi-tile shapes: X~ within 10 eps of X
    and of the FP64 path; this also checks that the middle-core solve
    regenerates exactly the test matrix the sketch used (an inconsistent
    B = P^T Omega costs ~1e-5 here)."""
    n1, n2, n3, n4 = dims
    Xd = torch.empty(n1 * n2 * n3 * n4, dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, n4, C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    t = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="bf16")
    assert t.kernel_kind() == 2
    t.pstt2(Xd)
    f = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="fp64").pstt2(Xd)
    e_x = t.error(Xd).cpu().numpy()
    Xf = f.reconstruct(torch.float32)
    e_f = t.error(Xf).cpu().numpy()
    rx, rf = (e_x[0] / e_x[1]) ** 0.5, (e_f[0] / e_x[1]) ** 0.5
    print(f"multi-tile pipeline {dims}: |X~-X|={rx:.2e} |X~-X~fp64|={rf:.2e} ranks={t.status()[1]}")
    assert rx <= 1e-5 and rf <= 1e-5


@pytest.mark.gpu
def test_pinned_host_tensor_read_directly_equals_device_tensor():
    """X in pinned host memory passed straight to the library (the kernels read
    it over the host link) gives the same decomposition as X on the device."""
    dims = [128, 16, 24, 128]
    x = ti.hilbert_type(dims)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    xh = torch.tensor(x, dtype=torch.float32).pin_memory()
    kw = dict(eps=1e-6, rmax=6, p=10, seed=1, x_dtype=torch.float32, prec="bf16")
    a = TTSketch(dims, **kw).pstt2(xd)
    b = TTSketch(dims, **kw)
    b.begin()
    b.accumulate(xh, 0, dims[-1])
    b.finalize()
    torch.cuda.synchronize()
    ra, rb = a.reconstruct(torch.float64).cpu().numpy(), b.reconstruct(torch.float64).cpu().numpy()
    assert a.status()[1] == b.status()[1]
    assert np.linalg.norm(ra - rb) <= 1e-9 * np.linalg.norm(ra)


# --------------------------------------------------------- small-plane kernel
@pytest.mark.parametrize("dims,kw", [
    ([9, 8, 7, 6, 5, 9], dict(eps=1e-5, rmax=6, p=6)),       # d = 6, l = 12; 56 x 30 planes (ragged blocks)
    ([24, 6, 5, 24], dict(eps=1e-5, rmax=16, p=10)),          # l = 26; 6 x 5 planes (ragged blocks)
    ([17, 11, 23], dict(ranks=[1, 4, 4, 1], p=5)),            # d = 3, odd sizes
    ([30, 31], dict(ranks=[1, 5, 1], p=5)),                   # d = 2: one plane
    ([8, 7, 6, 5, 4], dict(eps=1e-5, rmax=8, p=5)),           # d = 5
    ([15, 15, 15, 15, 15, 15], dict(eps=1e-5, rmax=16, p=10)),  # ~21 blocks per CTA: periodic flushes
])
@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_small_plane_sketches_match_oracle(dims, kw, prec):
    """The small-plane kernel (n_1, n_d <= 32): every sketch entry against the
    oracle's FP64 products of the split X with the rounded test matrices."""
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=5, noise=1e-5).astype(np.float32)
    t, s = _mk(dims, prec, x, seed=7, **kw)
    assert t.kernel_kind() == 3
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = _sketches(t, s)
    t.finalize()
    st, _ = t.status()
    assert st in (0, N.TT_WARN_RANK_CAP)
    xs = _split(x.astype(np.float64), prec, s)
    o = OP.pstt2(xs, dims, seed=7, passes=1, test_fmt=prec, **kw)
    for k, S in o["sketch"]["S"].items():
        _close_sketch(sk[(0, k)], S, ("S", k))
    for k, R in o["sketch"]["R"].items():
        _close_sketch(sk[(1, k)], R, ("R", k))


@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_small_plane_within_10eps_of_oracle(prec):
    """The precision-form shape at reduced n: X~ from the small-plane kernel
    within 10 eps of the FP64 oracle's X~ and of X."""
    dims, eps = [10] * 6, 1e-5
    x = ti.random_tt(dims, [1, 10, 10, 10, 10, 10, 1], seed=0, noise=1e-6).astype(np.float32)
    x64 = x.astype(np.float64)
    t = _mk(dims, prec, x, eps=eps, rmax=16, p=10, seed=1)[0]
    assert t.kernel_kind() == 3
    t.pstt2(to_dev(x))
    o = OP.pstt2(x64, dims, eps=eps, rmax=16, p=10, seed=1)
    xt = t.reconstruct().cpu().numpy()
    e_or, e_x = rel(xt, OT.tt_full(o["cores"]), x64), rel(xt, x64, x64)
    print(f"small-plane {prec}: |X~-X~oracle|={e_or:.2e} |X~-X|={e_x:.2e} ranks={t.status()[1]}")
    assert e_or <= 10 * eps and e_x <= 10 * eps


@pytest.mark.parametrize("dims,ranks", [
    ([9, 8, 7, 6, 5, 9], [1, 3, 5, 7, 5, 3, 1]),           # widths 8..12 (padding 16)
    ([4] * 9, [1, 4, 12, 18, 19, 19, 18, 12, 4, 1]),       # the paper's d = 9 rank profile, clamped: widths 14..29
])
@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_small_plane_unequal_widths_match_oracle(dims, ranks, prec):
    """Fixed ranks give each sketch its own width l_k = r_k + p; the
    small-plane kernel pads them all to the widest and writes each sketch's
    own columns: every sketch entry against the oracle."""
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=5, noise=1e-5).astype(np.float32)
    kw = dict(ranks=ranks, p=10)
    t, s = _mk(dims, prec, x, seed=7, **kw)
    assert t.kernel_kind() == 3
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = _sketches(t, s)
    t.finalize()
    widths = {v.shape[1] for v in sk.values()}
    assert len(widths) > 1
    xs = _split(x.astype(np.float64), prec, s)
    o = OP.pstt2(xs, dims, seed=7, passes=1, test_fmt=prec, **kw)
    for k, S in o["sketch"]["S"].items():
        _close_sketch(sk[(0, k)], S, ("S", k))
    for k, R in o["sketch"]["R"].items():
        _close_sketch(sk[(1, k)], R, ("R", k))


@pytest.mark.parametrize("dims,prec", [([256, 64, 48, 256], "bf16"), ([128, 64, 96, 128], "bf16"),
                                       ([128, 64, 96, 128], "fp16")])
def test_tcgen05_multitile_every_sketch_entry(dims, prec):
    """Every entry of every sketch of one multi-tile launch of the plane kernel
    against the oracle's dense FP64 products (the split X, the BF16-rounded
    test matrices).  At these shapes each CTA walks two to three tiles: the
    change of kL block inside a run, the flush of the column accumulators
    after at most 256 MMAs, the double-buffered row accumulators and the
    ragged last kL block (64 = 5 x 12 + 4 at n_1 = 128) all take part."""
    n1, n2, n3, n4 = dims
    Xd = torch.empty(n1 * n2 * n3 * n4, dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, n4, C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    kw = dict(eps=1e-6, rmax=6, p=10)
    s = 16 if prec == "fp16" else 0  # |X| <= 1/4
    t = TTSketch(dims, seed=7, prec=prec, x_scale_log2=s, **kw)
    assert t.kernel_kind() == 2
    t.begin()
    t.accumulate(Xd, 0, n4)
    sk = _sketches(t, s)
    del Xd
    x = ti.hilbert_type(dims, np.float32).astype(np.float64)
    xs = _split(x, prec, s)
    del x
    widths = OP.sketch_widths(4, None, kw["p"], True, kw["rmax"])
    o = OP.sketches(xs, dims, widths, 7, 1, test_fmt=prec)
    for k, S in o["S"].items():
        _close_sketch(sk[(0, k)], S, ("S", k))
    for k, R in o["R"].items():
        _close_sketch(sk[(1, k)], R, ("R", k))
