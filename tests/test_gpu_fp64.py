"""GPU parity of the FP64 path against the FP64 oracle, through the C ABI.

Bars: sketches element-wise to 1e-12 relative (FP64 arithmetic, different
summation order); X~ within 1e-10 of the oracle's X~ (relative Frobenius);
exact recovery of random low-rank TT tensors to 1e-12 (Theorems 3.1/3.2)."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import philox, pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch, TTError, _native as N
from tests.gpu_util import rel, sketch_dict, to_dev

pytestmark = pytest.mark.gpu


def test_philox_known_answers_on_device(golden):
    rows = golden("philox4x32_10_kat.txt")
    ctr = np.array([[int(t, 16) for t in r[:4]] for r in rows], dtype=np.uint32)
    for r, c in zip(rows, ctr):
        cd = torch.tensor(c.view(np.int32), device="cuda")
        out = torch.empty(4, dtype=torch.int32, device="cuda")
        N.check(N.lib().tt_philox4x32_10(C.c_void_p(cd.data_ptr()), int(r[4], 16), int(r[5], 16),
                                         C.c_void_p(out.data_ptr()), 1,
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream)), "philox")
        got = out.cpu().numpy().view(np.uint32)
        assert [int(v) for v in got] == [int(t, 16) for t in r[6:10]]


@pytest.mark.parametrize("sid,row0,nrows,ncols", [(3, 0, 1000, 9), (64 + 2, 2 ** 33 - 5, 300, 26), (1, 7, 17, 1)])
def test_test_matrix_fp64_matches_oracle(sid, row0, nrows, ncols):
    out = torch.empty(nrows * ncols, dtype=torch.float64, device="cuda")
    N.check(N.lib().tt_test_matrix(11, sid, row0, nrows, ncols, N.TT_PREC_FP64, C.c_void_p(out.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream)), "tm")
    got = out.cpu().numpy().reshape(ncols, nrows).T
    ref = philox.gaussian(11, sid, np.arange(row0, row0 + nrows, dtype=np.uint64), ncols)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_hilbert_generator_bit_exact():
    dims = [7, 5, 6, 9]
    out = torch.empty(7 * 5 * 6 * 4, dtype=torch.float32, device="cuda")
    n = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, n, 3, 4, C.c_void_p(out.data_ptr()), N.TT_F32,
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)), "gen")
    ref = ti.hilbert_type(dims, np.float32, first_last=3, count_last=4)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def _run_onepass(x, dims, x_dtype=torch.float64, **kw):
    t = TTSketch(dims, x_dtype=x_dtype, prec="fp64", **kw)
    X = to_dev(x, x_dtype)
    t.begin()
    t.accumulate(X, 0, dims[-1])
    sk = sketch_dict(t)
    t.finalize()
    return t, X, sk


@pytest.mark.parametrize("dims,r", [
    ([16, 16, 16, 16], [1, 3, 4, 3, 1]),          # config 1
    ([70, 3, 45], [1, 3, 4, 1]),                  # ragged tiles, d = 3
    ([5, 6, 4, 5, 3], [1, 3, 4, 4, 2, 1]),        # odd d
    ([33, 40], [1, 5, 1]),                        # d = 2
    ([3, 4, 2, 3, 2, 3, 2], [1, 2, 3, 3, 3, 3, 2, 1]),  # d = 7
])
def test_sketches_and_recovery_fp64(dims, r):
    x = ti.random_tt(dims, r, seed=len(dims))
    d = len(dims)
    target = [1] + [min(v + 1, 6) for v in r[1:-1]] + [1]
    t, X, sk = _run_onepass(x, dims, ranks=target, p=4, seed=9)
    o = OP.pstt2(x, dims, ranks=target, p=4, seed=9, passes=1)
    # sketches element-wise
    ds = (d + 1) // 2
    for k, S in o["sketch"]["S"].items():
        G = sk[(0, k)]
        assert G.shape == S.shape
        assert np.max(np.abs(G - S)) <= 1e-12 * np.max(np.abs(S))
    for k, R in o["sketch"]["R"].items():
        G = sk[(1, k)]
        assert np.max(np.abs(G - R)) <= 1e-12 * np.max(np.abs(R))
    # reconstruction: exact recovery and oracle parity
    xt = t.reconstruct().cpu().numpy()
    ref = OT.tt_full(o["cores"])
    assert rel(xt, x, x) <= 1e-12
    assert rel(xt, ref, x) <= 1e-10
    st, ranks = t.status()
    assert st == 0 and ranks == o["r"]
    # fused error kernel agrees with the dense difference
    e2, x2 = t.error(X).cpu().numpy()
    assert abs(x2 - np.sum(x ** 2)) <= 1e-12 * x2
    assert e2 <= 1e-22 * x2


def test_config1_fp32_storage_and_cores_match_oracle():
    dims = [16] * 4
    x = ti.random_tt(dims, [1, 3, 4, 3, 1], seed=0).astype(np.float32)
    t = TTSketch(dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1, x_dtype=torch.float32, prec="fp64")
    t.pstt2(to_dev(x))
    o = OP.pstt2(x.astype(np.float64), dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1)
    assert rel(t.reconstruct().cpu().numpy(), OT.tt_full(o["cores"]), x) <= 1e-10
    assert [g.shape for g in t.core_list()] == [g.shape for g in o["cores"]]


@pytest.mark.parametrize("order", [[(0, 5), (5, 11)], [(9, 7), (0, 4), (4, 5)], [(i, 1) for i in reversed(range(16))]])
def test_streaming_slabs_equal_one_shot(order):
    dims = [9, 7, 8, 16]
    x = ti.random_tt(dims, [1, 3, 3, 3, 1], seed=4, noise=1e-3)
    X = to_dev(x, torch.float64)
    one = TTSketch(dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2, x_dtype=torch.float64).pstt2(X)
    t = TTSketch(dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2, x_dtype=torch.float64)
    Nd1 = 9 * 7 * 8
    t.begin()
    for first, cnt in order:
        t.accumulate(X[first * Nd1:(first + cnt) * Nd1].clone(), first, cnt)
    t.finalize()
    a, b = one.reconstruct().cpu().numpy(), t.reconstruct().cpu().numpy()
    assert rel(a, b, x) <= 1e-12
    o = OP.pstt2(x, dims, ranks=[1, 3, 3, 3, 1], p=4, seed=2)
    assert rel(b, OT.tt_full(o["cores"]), x) <= 1e-10


def test_streaming_bookkeeping_errors():
    dims = [4, 4, 6]
    X = to_dev(np.ones(96), torch.float64)
    t = TTSketch(dims, ranks=[1, 2, 2, 1], p=2, x_dtype=torch.float64)
    with pytest.raises(TTError) as e:
        t.accumulate(X, 0, 6)
    assert e.value.status == N.TT_ERR_STATE
    t.begin()
    t.accumulate(X[:32], 0, 2)
    with pytest.raises(TTError) as e:
        t.accumulate(X[:32], 1, 2)
    assert e.value.status == N.TT_ERR_STATE
    with pytest.raises(TTError) as e:
        t.finalize()
    assert e.value.status == N.TT_ERR_STATE
    with pytest.raises(TTError) as e:
        t.accumulate(X[:32], 5, 2)
    assert e.value.status == N.TT_ERR_INVALID_ARG


@pytest.mark.parametrize("dims,r,eps", [([9, 8, 9, 8, 9, 8], [1, 5, 6, 6, 6, 5, 1], 1e-5),
                                        ([30, 30, 30, 30], [1, 3, 5, 3, 1], 1e-6)])
def test_eps_mode_matches_oracle(dims, r, eps):
    x = ti.random_tt(dims, r, seed=1, noise=1e-7)
    t = TTSketch(dims, eps=eps, rmax=8, p=6, seed=3, x_dtype=torch.float64).pstt2(to_dev(x, torch.float64))
    o = OP.pstt2(x, dims, eps=eps, rmax=8, p=6, seed=3)
    st, ranks = t.status()
    assert ranks == o["r"] and st == 0
    xt = t.reconstruct().cpu().numpy()
    assert rel(xt, OT.tt_full(o["cores"]), x) <= 1e-10
    assert rel(xt, x, x) <= eps


def test_rank_cap_flag():
    dims = [12, 12, 12]
    x = np.random.default_rng(0).standard_normal(12 ** 3)
    t = TTSketch(dims, eps=1e-8, rmax=3, p=4, x_dtype=torch.float64).pstt2(to_dev(x, torch.float64))
    st, ranks = t.status()
    assert st == N.TT_WARN_RANK_CAP and ranks == [1, 3, 3, 1]


@pytest.mark.parametrize("dims,r", [([16, 16, 16, 16], [1, 3, 4, 3, 1]), ([6, 5, 7, 4, 5], [1, 3, 3, 3, 2, 1]),
                                    ([20, 30], [1, 4, 1])])
def test_two_pass_matches_oracle(dims, r):
    x = ti.random_tt(dims, r, seed=3, noise=1e-4)
    target = [1] + [v for v in r[1:-1]] + [1]
    t = TTSketch(dims, ranks=target, p=4, seed=5, passes=2, x_dtype=torch.float64).pstt2(to_dev(x, torch.float64))
    o = OP.pstt2(x, dims, ranks=target, p=4, seed=5, passes=2)
    assert rel(t.reconstruct().cpu().numpy(), OT.tt_full(o["cores"]), x) <= 1e-10
