"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times.

* Streaming workload: Hilbert-type X, d = 4, n = 256 (4.29e9 FP32 entries,
  17.2 GB), eps = 1e-6, rmax = 6, p = 10, seed 1, one accumulate over the whole
  last mode (the tcgen05 plane kernel).  The oracle cannot sketch the whole
  tensor in seconds, so sampled sketch rows are computed one by one: each is an
  FP64 sum over a sub-tensor of X (regenerated on the host from its formula)
  times the oracle's rounded test-matrix rows.  The middle sketches S_2 and R_2
  (test matrices of 65,536 rows) take a few rows each; the outermost S_1 and
  R_3 (16.7 M rows) one row each, in slabs.  Then the whole one-pass pipeline:
  X~ within 10 eps of X and of the FP64 path.  BF16 and FP16 (X 2^16, as
  |X| <= 1/4).
* The same tensor streamed as the benchmark streams it: 16 slabs of 16
  slices (1 GiB each) in shuffled order, Khatri-Rao test matrices, FP16: no
  rank cap, the FP64 path's ranks or at most one more on a bond (the FP32
  accumulation of the tensor cores), X~ within 10 eps of X and of the FP64
  path; with TT_FLAG_SHORT_CHAINS, the FP64 path's ranks and X~ within eps
  of X.
* Precision form: random TT, d = 6, n = 24, internal ranks 10, +1e-6 noise
  (1.91e8 FP32 entries), eps = 1e-5, p = 10, rmax = 16 (the small-plane
  kernel), BF16 and TF32: sampled rows of every sketch (S_1..S_3, R_3..R_5;
  the outermost two one row each, in slabs), and X~ within 10 eps of X and of
  the FP64 path.

Bars as in the multi-tile tests (the rare test-matrix rounding flips bound a
sampled row's max difference by 2e-3 of its max entry).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import philox
from paper_2111_10448_gb300 import TTSketch, _native as N
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

STREAMING = dict(eps=1e-6, rmax=6, p=10, seed=1)
PRECISION = dict(eps=1e-5, rmax=16, p=10, seed=1)


def _split(x, prec, s=0):
    xs = np.asarray(x, dtype=np.float64) * 2.0 ** s
    hi = philox.round_to(xs, prec)
    lo = philox.round_to(xs - hi, prec)
    return (hi + lo) * 2.0 ** -s


S16 = 16  # FP16 scale of the Hilbert-type tensor: |X| <= 1/4, X 2^16 <= 2^14


def _rowerr(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def _tm(seed, stream, rows, l, prec):
    """Rounded oracle test-matrix rows (row indices `rows`)."""
    return philox.round_to(philox.gaussian(seed, stream, np.asarray(rows, dtype=np.uint64), l), prec)


@pytest.fixture(scope="module")
def hilbert256():
    dims = [256] * 4
    Xd = torch.empty(256 ** 4, dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, 256, C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    torch.cuda.synchronize()
    yield dims, Xd
    del Xd
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_streaming_256_sampled_sketch_rows(hilbert256, prec):
    dims, Xd = hilbert256
    n1, n2, n3, n4 = dims
    seed = STREAMING["seed"]
    s = S16 if prec == "fp16" else 0
    t = TTSketch(dims, x_dtype=torch.float32, prec=prec, x_scale_log2=s, **STREAMING)
    assert t.kernel_kind() == 2
    t.begin()
    t.accumulate(Xd, 0, n4)
    sk = {(ty, k): S * 2.0 ** -s for ty, k, S in t.sketches(0)}
    l = sk[(0, 1)].shape[1]
    sub = lambda idx: _split(ti.hilbert_type_block(dims, idx).astype(np.float64), prec, s)
    rng = np.random.default_rng(11)
    errs = {}
    Om2 = _tm(seed, 2, np.arange(n3 * n4), l, prec)
    Ps2 = _tm(seed, 66, np.arange(n1 * n2), l, prec)
    for _ in range(4):
        i1, i2, i3, i4 = [int(rng.integers(v)) for v in dims]
        # S_2(i1 + n1 i2, :) = sum_{i3,i4} X(i1,i2,i3,i4) Omega_2[i3 + n3 i4, :]
        ref = sub([[i1], [i2], None, None]) @ Om2
        got = sk[(0, 2)][i1 + n1 * i2].cpu().numpy()
        errs.setdefault("S2", []).append(_rowerr(got, ref))
        # R_2(i3 + n3 i4, :) = sum_{i1,i2} X(i1,i2,i3,i4) Psi_2[i1 + n1 i2, :]
        ref = sub([None, None, [i3], [i4]]) @ Ps2
        got = sk[(1, 2)][i3 + n3 * i4].cpu().numpy()
        errs.setdefault("R2", []).append(_rowerr(got, ref))
    # outermost sketches: one row each, summed slab by slab in FP64
    i1, i4 = int(rng.integers(n1)), int(rng.integers(n4))
    ref = np.zeros(l)
    for j4 in range(n4):   # S_1(i1, :) = sum X(i1, i2, i3, i4) Omega_1[i2 + n2 i3 + n2 n3 i4, :]
        rows = j4 * n2 * n3 + np.arange(n2 * n3)
        ref += sub([[i1], None, None, [j4]]) @ _tm(seed, 1, rows, l, prec)
    errs["S1"] = [_rowerr(sk[(0, 1)][i1].cpu().numpy(), ref)]
    ref = np.zeros(l)
    for j3 in range(n3):   # R_3(i4, :) = sum X(i1, i2, i3, i4) Psi_3[i1 + n1 i2 + n1 n2 i3, :]
        rows = j3 * n1 * n2 + np.arange(n1 * n2)
        ref += sub([None, None, [j3], [i4]]) @ _tm(seed, 67, rows, l, prec)
    errs["R3"] = [_rowerr(sk[(1, 3)][i4].cpu().numpy(), ref)]
    t.finalize()
    e = {k: max(v) for k, v in errs.items()}
    print(f"256^4 sampled sketch rows {prec}, max rel err:", e)
    assert all(v <= 2e-3 for v in e.values()), e


def test_streaming_256_pipeline_within_10eps(hilbert256):
    dims, Xd = hilbert256
    eps = STREAMING["eps"]
    t = TTSketch(dims, x_dtype=torch.float32, prec="bf16", **STREAMING)
    t.pstt2(Xd)
    st, ranks = t.status()
    assert st in (0, N.TT_WARN_RANK_CAP)
    e_x = t.error(Xd).cpu().numpy()
    f = TTSketch(dims, x_dtype=torch.float32, prec="fp64", **STREAMING).pstt2(Xd)
    Xf = f.reconstruct(torch.float32)
    e_f = t.error(Xf).cpu().numpy()
    del Xf
    rx, rf = (e_x[0] / e_x[1]) ** 0.5, (e_f[0] / e_x[1]) ** 0.5
    print(f"256^4 pipeline: |X~-X|={rx:.2e} |X~-X~fp64|={rf:.2e} ranks={ranks}")
    assert rx <= 10 * eps and rf <= 10 * eps


@pytest.mark.parametrize("short", [False, True])
def test_streaming_256_fp16_slabs_no_rank_cap(hilbert256, short):
    """The benchmark's streaming configuration: FP16 with Khatri-Rao test
    matrices, sixteen 1 GiB slabs of 16 slices in shuffled order.  The FP16
    split (2^-22 relative) resolves the rank threshold eps / sqrt(d - 1):
    status OK (no rank cap), the ranks of the FP64 path or one more on a bond
    (FP32 accumulation noise of the tensor cores near the threshold), X~
    within 10 eps of X and of the FP64 path's X~."""
    dims, Xd = hilbert256
    eps = STREAMING["eps"]
    t = TTSketch(dims, x_dtype=torch.float32, prec="fp16", drm="kr", x_scale_log2=S16, short_chains=short,
                 **STREAMING)
    assert t.kernel_kind(16) == 2
    nd1 = 256 ** 3
    order = list(range(0, 256, 16))
    np.random.default_rng(2).shuffle(order)
    t.begin()
    for a in order:
        t.accumulate(Xd[a * nd1:(a + 16) * nd1], a, 16)
    t.finalize()
    st, ranks = t.status()
    f = TTSketch(dims, x_dtype=torch.float32, prec="fp64", drm="kr", **STREAMING).pstt2(Xd)
    e_x = t.error(Xd).cpu().numpy()
    Xf = f.reconstruct(torch.float32)
    e_f = t.error(Xf).cpu().numpy()
    del Xf
    rx, rf = (e_x[0] / e_x[1]) ** 0.5, (e_f[0] / e_x[1]) ** 0.5
    print(f"256^4 FP16 slabs (short chains {short}): |X~-X|={rx:.2e} |X~-X~fp64|={rf:.2e} ranks={ranks} "
          f"fp64 ranks={f.status()[1]}")
    r64 = f.status()[1]
    assert st == 0 and all(a <= b <= a + 1 for a, b in zip(r64, ranks)), (r64, ranks)
    assert rx <= 10 * eps and rf <= 10 * eps
    if short:
        assert ranks == r64 and rx <= eps


@pytest.fixture(scope="module")
def randomtt24():
    dims = [24] * 6
    x = ti.random_tt(dims, [1, 10, 10, 10, 10, 10, 1], seed=0, noise=1e-6).astype(np.float32)
    return dims, x, to_dev(x)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_precision_24_sampled_sketch_rows(randomtt24, prec):
    dims, x, Xd = randomtt24
    d, n = len(dims), dims[0]
    seed = PRECISION["seed"]
    t = TTSketch(dims, x_dtype=torch.float32, prec=prec, **PRECISION)
    assert t.kernel_kind() == 3
    t.begin()
    t.accumulate(Xd, 0, n)
    sk = {(ty, k): S.cpu().numpy() for ty, k, S in t.sketches(0)}
    t.finalize()
    l = sk[(0, 1)].shape[1]
    xs = x.reshape([n] * d, order="F")
    rng = np.random.default_rng(12)
    split = lambda a: _split(np.asarray(a).reshape(-1, order="F").astype(np.float64), prec)
    errs = {}
    for (ty, k), Sk in sk.items():
        # S_k rows (i_1..i_k): sum over i_{k+1..d} of X Omega_k (n^{d-k} test-matrix rows);
        # R_k rows (i_{k+1..d}): sum over i_{1..k} of X Psi_k (n^k test-matrix rows)
        m = d - k if ty == 0 else k
        stream = k if ty == 0 else 64 + k
        if m <= 4:   # three rows, whole test matrix at once
            W = _tm(seed, stream, np.arange(n ** m), l, prec)
            for _ in range(3):
                lead = [int(v) for v in rng.integers(n, size=k)]
                trail = [int(v) for v in rng.integers(n, size=d - k)]
                if ty == 0:
                    v, row = split(xs[tuple(lead)]), np.ravel_multi_index(lead, [n] * k, order="F")
                else:
                    v, row = split(xs[(Ellipsis,) + tuple(trail)]), np.ravel_multi_index(trail, [n] * (d - k), order="F")
                errs.setdefault(f"{'SR'[ty]}{k}", []).append(_rowerr(Sk[int(row)], v @ W))
        else:        # one row, summed slab by slab over the last summed mode
            ref = np.zeros(l)
            if ty == 0:
                lead = [int(v) for v in rng.integers(n, size=k)]
                row = np.ravel_multi_index(lead, [n] * k, order="F")
                for j in range(n):
                    W = _tm(seed, stream, j * n ** (m - 1) + np.arange(n ** (m - 1)), l, prec)
                    ref += split(xs[tuple(lead)][..., j]) @ W
            else:
                trail = [int(v) for v in rng.integers(n, size=d - k)]
                row = np.ravel_multi_index(trail, [n] * (d - k), order="F")
                for j in range(n):
                    W = _tm(seed, stream, j * n ** (m - 1) + np.arange(n ** (m - 1)), l, prec)
                    ref += split(xs[(Ellipsis, j) + tuple(trail)]) @ W
            errs[f"{'SR'[ty]}{k}"] = [_rowerr(Sk[int(row)], ref)]
    e = {k: max(v) for k, v in errs.items()}
    print(f"24^6 {prec} sampled sketch rows, max rel err:", e)
    assert set(e) == {"S1", "S2", "S3", "R3", "R4", "R5"}
    assert all(v <= 2e-3 for v in e.values()), e


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_precision_24_pipeline_within_10eps(randomtt24, prec):
    dims, x, Xd = randomtt24
    eps = PRECISION["eps"]
    t = TTSketch(dims, x_dtype=torch.float32, prec=prec, **PRECISION).pstt2(Xd)
    f = TTSketch(dims, x_dtype=torch.float32, prec="fp64", **PRECISION).pstt2(Xd)
    e_x = t.error(Xd).cpu().numpy()
    e_f = t.error(f.reconstruct(torch.float32)).cpu().numpy()
    rx, rf = (e_x[0] / e_x[1]) ** 0.5, (e_f[0] / e_x[1]) ** 0.5
    print(f"24^6 {prec} pipeline: |X~-X|={rx:.2e} |X~-X~fp64|={rf:.2e} ranks={t.status()[1]}")
    assert rx <= 10 * eps and rf <= 10 * eps
