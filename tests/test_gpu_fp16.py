"""GPU checks specific to the FP16 sketch precision: X is split as X 2^s
into FP16 hi + lo (s = x_scale_log2, a power of two, so exact), the sketches
are scaled back by 2^-s in FP64 before the bases are formed.

* tt_x_scale_log2 against its rule, s = 15 - e with 2^(e-1) <= max |X| < 2^e,
  computed here with numpy's frexp; zero tensors give 0; an inf or NaN gives
  TT_ERR_NONFINITE.
* A scale that puts |X| 2^s past the FP16 range makes the sketch infinite:
  the finalize reports TT_ERR_NONFINITE in the status word (no fault: inf
  operands are ordinary values to the tensor cores), and the next call on
  the same context computes normally.
* Scale invariance: the result does not depend on s while X 2^s stays in
  the range where the low part of the split is a normal FP16 number (|X 2^s|
  >= 2^-3): same ranks, X~ equal up to FP32 accumulation order (1e-6).
* Resolution: on the Hilbert-type tensor at eps = 1e-6 (d = 4), FP16 stops
  below the rank cap with X~ within eps of X (BF16, printed beside it, stops
  at the cap: its split resolves 2^-17, above eps / sqrt(d - 1)).  With dense
  test matrices the ranks are the FP64 path's.  The tensor cores' FP32
  accumulation adds about 2e-8 relative error per accumulating MMA (measured
  against FP64 products with the kernels' own test matrices), so a bond whose
  FP64 tail lies close to the threshold can take one rank more: the
  Khatri-Rao instance here has its r_2 tail at 0.83 of the threshold, and
  the bar there is "the FP64 ranks or one more".
"""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from paper_2111_10448_gb300 import TTSketch, TTError, x_scale_log2, _native as N
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _rule(x):
    m = float(np.max(np.abs(x)))
    return 0 if m == 0.0 else max(-100, min(100, 15 - int(np.frexp(m)[1])))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_x_scale_log2_follows_its_rule(dtype):
    rng = np.random.default_rng(0)
    for mag in (1e-30, 3e-6, 0.2, 0.25, 1.0, 1.5, 65504.0, 7e9):
        x = rng.standard_normal(100_003) * mag
        xd = torch.tensor(x, dtype=dtype, device="cuda")
        want = _rule(xd.cpu().numpy())
        assert x_scale_log2(xd) == want, mag
    # exact powers of two: max = 2^k gives e = k + 1
    for k in (-3, 0, 7):
        xd = torch.zeros(1000, dtype=dtype, device="cuda")
        xd[517] = -(2.0 ** k)
        assert x_scale_log2(xd) == 15 - (k + 1)
    assert x_scale_log2(torch.zeros(10, dtype=dtype, device="cuda")) == 0
    for bad in (float("inf"), float("nan")):
        xd = torch.ones(4096, dtype=dtype, device="cuda")
        xd[4000] = bad
        with pytest.raises(TTError) as ei:
            x_scale_log2(xd)
        assert ei.value.status == N.TT_ERR_NONFINITE


@pytest.mark.parametrize("dims,kind", [([40, 7, 6, 70], 1), ([24, 6, 5, 24], 3), ([128, 8, 16, 32], 2)])
def test_overflow_past_fp16_range_is_reported(dims, kind):
    """|X| 2^s >= 65520 overflows the FP16 high part: status TT_ERR_NONFINITE
    on the generic, small-plane and slab kernels; afterwards a valid scale on
    the same plan shape computes normally."""
    x = ti.hilbert_type(dims, np.float32)  # |X| <= 1/4
    X = to_dev(x)
    kw = dict(eps=1e-6, rmax=6, p=10, seed=1)
    c = 16 if kind == 2 else dims[-1]
    bad = TTSketch(dims, prec="fp16", x_scale_log2=20, **kw)  # 1/4 2^20 = 262144
    assert bad.kernel_kind(c) == kind
    nd1 = int(np.prod(dims[:-1]))
    bad.begin()
    for a in range(0, dims[-1], c):
        bad.accumulate(X[a * nd1:(a + c) * nd1], a, c)
    bad.finalize()
    st, _ = bad.status()
    assert st == N.TT_ERR_NONFINITE
    good = TTSketch(dims, prec="fp16", x_scale_log2=16, **kw).pstt2(X)
    st, _ = good.status()
    assert st in (0, N.TT_WARN_RANK_CAP)
    e = good.error(X).cpu().numpy()
    assert (e[0] / e[1]) ** 0.5 <= 1e-5


@pytest.mark.parametrize("dims,c", [([256, 16, 16, 64], 16), ([24, 8, 8, 24], 24)])
def test_results_do_not_depend_on_the_scale(dims, c):
    x = ti.hilbert_type(dims, np.float32)  # |X| in [1/8, 1/4]: X 2^s >= 2^-3 for s >= 0
    X = to_dev(x)
    nd1 = int(np.prod(dims[:-1]))
    out = []
    for s in (4, 10, 17):
        t = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=3, prec="fp16", drm="kr", x_scale_log2=s)
        t.begin()
        for a in range(0, dims[-1], c):
            t.accumulate(X[a * nd1:(a + c) * nd1], a, c)
        t.finalize()
        out.append((t.status(), t.reconstruct().cpu().numpy()))
    for (st, xt) in out[1:]:
        assert st == out[0][0]
        assert np.linalg.norm(xt - out[0][1]) <= 1e-6 * np.linalg.norm(x)


@pytest.mark.parametrize("drm", ["gauss", "kr"])
def test_fp16_meets_eps_where_bf16_caps(drm):
    dims = [256, 32, 32, 64]
    Xd = torch.empty(int(np.prod(dims)), dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, dims[-1], C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    kw = dict(eps=1e-6, rmax=6, p=10, seed=1, drm=drm)
    s = x_scale_log2(Xd)
    assert s == 16
    res = {}
    for prec in ("fp64", "bf16", "fp16"):
        t = TTSketch(dims, prec=prec, x_scale_log2=s, **kw)
        nd1 = int(np.prod(dims[:-1]))
        t.begin()
        for a in range(0, dims[-1], 16):
            t.accumulate(Xd[a * nd1:(a + 16) * nd1], a, 16)
        t.finalize()
        e = t.error(Xd).cpu().numpy()
        res[prec] = (t.status(), (e[0] / e[1]) ** 0.5)
    print({k: (v[0], f"{v[1]:.2e}") for k, v in res.items()})
    (st64, r64), e64 = res["fp64"]
    (st16, r16), e16 = res["fp16"]
    assert st64 == 0 and st16 == 0
    if drm == "gauss":
        assert r16 == r64
    else:
        assert all(a <= b <= a + 1 for a, b in zip(r64, r16)), (r64, r16)
    assert e16 <= 1e-6


def test_short_chains_on_the_plane_kernel():
    """TT_FLAG_SHORT_CHAINS on the whole-last-mode plane kernel (its L slots
    flushed after every tile): the same ranks as the default chains and X~
    within 10 eps of X and of the default's X~ (they differ by FP32
    accumulation order only)."""
    dims = [256, 16, 16, 256]
    x = ti.hilbert_type(dims, np.float32)
    X = to_dev(x)
    out = []
    for short in (False, True):
        t = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=2, prec="fp16", x_scale_log2=16, short_chains=short)
        assert t.kernel_kind() == 2
        t.pstt2(X)
        e = t.error(X).cpu().numpy()
        out.append((t.status(), (e[0] / e[1]) ** 0.5, t.reconstruct().cpu().numpy()))
    print([(o[0], f"{o[1]:.2e}") for o in out])
    assert out[0][0][0] == 0 and out[1][0][0] == 0
    assert out[0][1] <= 1e-5 and out[1][1] <= 1e-5
    assert np.linalg.norm(out[0][2] - out[1][2]) <= 1e-5 * np.linalg.norm(x)


@pytest.mark.parametrize("kw", [dict(passes=2), dict(one_sided=True), dict(one_sided=True, passes=2)])
def test_two_pass_and_one_sided_fp16(kw):
    """FP16 sketches feeding the two-pass middle core (a second FP64 pass over
    X itself) and the one-sided PSTT forms: within 10 eps of X and of the FP64
    path with the same options."""
    dims, eps = [9] * 6, 1e-5
    x = ti.random_tt(dims, [1, 9, 10, 10, 10, 9, 1], seed=0, noise=1e-6).astype(np.float32)
    X = to_dev(x)
    s = _rule(x)
    t = TTSketch(dims, eps=eps, rmax=16, p=10, seed=1, prec="fp16", x_scale_log2=s, **kw).pstt2(X)
    f = TTSketch(dims, eps=eps, rmax=16, p=10, seed=1, prec="fp64", x_dtype=torch.float32, **kw).pstt2(X)
    x64 = x.astype(np.float64)
    xt = t.reconstruct().cpu().numpy()
    e_x = np.linalg.norm(xt - x64) / np.linalg.norm(x64)
    e_f = np.linalg.norm(xt - f.reconstruct().cpu().numpy()) / np.linalg.norm(x64)
    print(kw, f"|X~-X|={e_x:.2e} |X~-X~fp64|={e_f:.2e} ranks={t.status()[1]}")
    assert t.status()[0] in (0, N.TT_WARN_RANK_CAP)
    assert e_x <= 10 * eps and e_f <= 10 * eps
