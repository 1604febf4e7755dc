"""GPU parity of the slab form of the tcgen05 plane kernel: a slab of 16, 32
or 64 last-mode slices of a 4-way tensor (the 1 GiB slabs of the 256^4
streaming workload are 16 slices), accumulated slab by slab in any order.

Every sketch entry after a stream of slabs is compared with the oracle's
dense FP64 products of the split X (hi + lo in BF16, or in FP16 of X 2^s) with
its test matrices rounded the same way, dense Gaussian and Khatri-Rao:
Frobenius 1e-4 and max 2e-3 of
max |S| (the bars and their derivation are those of test_gpu_mixed.py: the
FP32 generator flips a rare rounding decision).  The slab kernel takes the
R_3 products against G planes' blocks at once and keeps the diagonal; a
wrong block choice, row map or flush shows up as O(1) errors here."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import philox, pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch, _native as N
from tests.gpu_util import rel, sketch_dict, to_dev

pytestmark = pytest.mark.gpu


def _split(x, prec="bf16", s=0):
    xs = np.asarray(x, dtype=np.float64) * 2.0 ** s
    hi = philox.round_to(xs, prec)
    return (hi + philox.round_to(xs - hi, prec)) * 2.0 ** -s


def _close(G, S, what):
    fro = np.linalg.norm(G - S) / np.linalg.norm(S)
    mx = np.max(np.abs(G - S)) / np.max(np.abs(S))
    assert fro <= 1e-4 and mx <= 2e-3, (what, fro, mx)


def _slabs(n4, c, seed):
    order = list(range(0, n4, c))
    np.random.default_rng(seed).shuffle(order)
    return [(a, c) for a in order]


@pytest.mark.parametrize("dims,c,kw", [
    ([128, 8, 16, 32], 16, dict(eps=1e-6, rmax=6, p=10)),      # l = 16, one tile
    ([256, 6, 16, 48], 16, dict(ranks=[1, 4, 4, 4, 1], p=4)),  # l = 8, two halves of i_1, ragged kL block
    ([128, 8, 16, 64], 32, dict(eps=1e-6, rmax=6, p=10)),      # c = 32 (G = 4)
    ([256, 4, 8, 64], 64, dict(eps=1e-6, rmax=6, p=10)),       # c = 64 (G = 2)
    ([256, 64, 64, 32], 16, dict(eps=1e-6, rmax=6, p=10)),     # two halves of i_1, 64 tiles
])
@pytest.mark.parametrize("drm", ["gauss", "kr"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_slab_sketches_match_oracle(dims, c, kw, drm, prec):
    _check_slab(dims, c, kw, drm, prec)


def test_slab_multitile_every_sketch_entry():
    """320 tiles (40 kL blocks x 8 kR-group blocks, the last one ragged) over
    the GPU's CTAs: each CTA walks two or three tiles, changes kL block inside
    its run and flushes the column accumulators; every entry against the
    oracle.  With TT_FLAG_SHORT_CHAINS the column accumulators are flushed
    after every two tiles, kL by kL behind the next run."""
    _check_slab([128, 160, 240, 16], 16, dict(eps=1e-6, rmax=6, p=10), "gauss")
    _check_slab([128, 160, 240, 16], 16, dict(eps=1e-6, rmax=6, p=10), "kr", "fp16")
    _check_slab([128, 160, 240, 16], 16, dict(eps=1e-6, rmax=6, p=10, short_chains=True), "kr", "fp16")
    _check_slab([256, 64, 64, 32], 16, dict(eps=1e-6, rmax=6, p=10, short_chains=True), "gauss", "fp16")


def test_slab_headline_launch_shape_every_sketch_entry():
    """The launch shape of the 256^4 stream in 1 GiB slabs, on a 256^3 x 32
    tensor (two 16-slice slabs): 256 kL values x 32 kR groups, FP16 split,
    Khatri-Rao test matrices, eps 1e-6, rmax 6, p 10.  The planner's tile of
    5 kL values leaves a ragged block of one kL value, and each of the 152
    CTAs walks about 11 tiles (55 super-planes, L chains of 176 MMAs); every
    entry of the four sketches against the oracle."""
    _check_slab([256, 256, 256, 32], 16, dict(eps=1e-6, rmax=6, p=10), "kr", "fp16")


def _check_slab(dims, c, kw, drm, prec="bf16"):
    n1, n2, n3, n4 = dims
    x = ti.random_tt(dims, [1, 3, 3, 3, 1], seed=5, noise=1e-5).astype(np.float32)
    X = to_dev(x)
    # FP16: X 2^s below 2^15 (the rule of tt_x_scale_log2)
    s = 15 - int(np.frexp(float(np.max(np.abs(x))))[1]) if prec == "fp16" else 0
    t = TTSketch(dims, seed=7, x_dtype=torch.float32, prec=prec, drm=drm, x_scale_log2=s, **kw)
    assert t.kernel_kind(c) == 2
    nd1 = n1 * n2 * n3
    t.begin()
    for a, cnt in _slabs(n4, c, 1):
        t.accumulate(X[a * nd1:(a + cnt) * nd1].clone(), a, cnt)
    sk = {k: v * 2.0 ** -s for k, v in sketch_dict(t).items()}
    t.finalize()
    st, _ = t.status()
    assert st in (0, N.TT_WARN_RANK_CAP)
    kw = {k: v for k, v in kw.items() if k != "short_chains"}
    widths = OP.sketch_widths(4, OP.clamp_ranks(dims, kw["ranks"]) if "ranks" in kw else None, kw["p"],
                              "eps" in kw, kw.get("rmax"))
    o = OP.sketches(_split(x.astype(np.float64), prec, s), dims, widths, 7, 1, test_fmt=prec, drm=drm)
    for k, S in o["S"].items():
        _close(sk[(0, k)], S, ("S", k))
    for k, R in o["R"].items():
        _close(sk[(1, k)], R, ("R", k))


@pytest.mark.parametrize("drm", ["gauss", "kr"])
def test_slab_stream_equals_whole_tensor(drm):
    """Sixteen-slice slabs in shuffled order against one accumulate of the
    whole last mode (the plane kernel): the decompositions agree to the FP32
    accumulation differences of the two tilings.  Bar 3e-6: both kernels sum
    in FP32 chains of up to 256 MMAs (A14) and the slab kernel stages S_2's
    partials in FP32; at the rank cap (ranks 4-6 resolve the 2^-17 noise of
    the split of X) such perturbations move X~ by ~1e-6, well inside the
    10 eps = 1e-5 that each result keeps to X."""
    dims = [256, 16, 16, 256]
    x = ti.hilbert_type(dims, np.float32)
    X = to_dev(x)
    kw = dict(eps=1e-6, rmax=6, p=10, seed=1, prec="bf16", drm=drm)
    one = TTSketch(dims, **kw)
    assert one.kernel_kind(256) == 2 and one.kernel_kind(16) == 2
    one.pstt2(X)
    t = TTSketch(dims, **kw)
    nd1 = 256 * 16 * 16
    t.begin()
    for a, cnt in _slabs(256, 16, 3):
        t.accumulate(X[a * nd1:(a + cnt) * nd1], a, cnt)
    t.finalize()
    assert t.status()[1] == one.status()[1]
    assert rel(one.reconstruct().cpu().numpy(), t.reconstruct().cpu().numpy(), x) <= 3e-6


@pytest.mark.parametrize("drm", ["gauss", "kr"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_slab_pipeline_within_10eps(drm, prec):
    """The one-pass pipeline fed by 16-slice slabs: X~ within 10 eps of X and
    of the FP64 path with the same test matrices.  FP16 resolves the rank
    threshold eps / sqrt(d - 1): no rank cap, X~ within eps of X, and the FP64
    path's ranks (dense) or at most one more on a bond (Khatri-Rao, whose r_2
    tail on this instance sits at 0.83 of the threshold, inside the FP32
    accumulation noise of the tensor cores)."""
    dims = [256, 32, 32, 128]
    Xd = torch.empty(int(np.prod(dims)), dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, dims[-1], C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    t = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec=prec, drm=drm, x_scale_log2=16)
    nd1 = 256 * 32 * 32
    t.begin()
    for a, cnt in _slabs(128, 16, 5):
        t.accumulate(Xd[a * nd1:(a + cnt) * nd1], a, cnt)
    t.finalize()
    f = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="fp64", drm=drm).pstt2(Xd)
    e_x = t.error(Xd).cpu().numpy()
    e_f = t.error(f.reconstruct(torch.float32)).cpu().numpy()
    rx, rf = (e_x[0] / e_x[1]) ** 0.5, (e_f[0] / e_x[1]) ** 0.5
    print(f"slab pipeline {drm} {prec}: |X~-X|={rx:.2e} |X~-X~fp64|={rf:.2e} ranks={t.status()[1]}")
    assert rx <= 1e-5 and rf <= 1e-5
    if prec == "fp16":
        st, r16 = t.status()
        r64 = f.status()[1]
        assert st == 0 and rx <= 1e-6
        assert r16 == r64 if drm == "gauss" else all(a <= b <= a + 1 for a, b in zip(r64, r16)), (r64, r16)


@pytest.mark.parametrize("drm", ["gauss", "kr"])
def test_mixed_slab_sizes_in_one_stream(drm):
    """Slabs of 16, 128 and 32 slices in one decomposition: the plane kernel
    and the slab kernel share the staging area, and each restages what it
    needs; the result equals one accumulate of the whole tensor up to FP32
    accumulation order (bar 3e-6, as for the sixteen-slice stream above)."""
    dims = [256, 8, 16, 256]
    x = ti.hilbert_type(dims, np.float32)
    X = to_dev(x)
    kw = dict(eps=1e-6, rmax=6, p=10, seed=1, prec="bf16", drm=drm)
    one = TTSketch(dims, **kw).pstt2(X)
    t = TTSketch(dims, **kw)
    nd1 = 256 * 8 * 16
    t.begin()
    for a, cnt in [(0, 16), (128, 128), (16, 32), (48, 16), (64, 64)]:
        t.accumulate(X[a * nd1:(a + cnt) * nd1], a, cnt)
    t.finalize()
    assert t.status()[1] == one.status()[1]
    assert rel(one.reconstruct().cpu().numpy(), t.reconstruct().cpu().numpy(), x) <= 3e-6


def test_staged_r3_blocks_restaged_per_decomposition():
    """Dense test matrices on 16-slice slabs: R_3's 128-row blocks are staged
    in the workspace at the first slab launch of each decomposition.  Runs on
    one caller workspace: fresh; again; after the workspace was overwritten
    and released with tt_workspace_release; after another plan used it and it
    was overwritten.  Every run must reproduce the first (FP32 accumulation
    order only), which is within 10 eps of X."""
    dims = [128, 8, 16, 64]
    x = ti.hilbert_type(dims, np.float32)
    X = to_dev(x)
    kw = dict(eps=1e-6, rmax=6, p=10, seed=1, prec="bf16", drm="gauss")
    A = TTSketch(dims, **kw)
    assert A.kernel_kind(16) == 2
    B = TTSketch([16] * 4, ranks=[1, 4, 4, 4, 1], p=5, seed=1, x_dtype=torch.float64, prec="fp64")
    XB = torch.tensor(ti.random_tt([16] * 4, [1, 3, 4, 3, 1], seed=0), device="cuda")
    ws = torch.empty(max(A.ws_bytes, B.ws_bytes) // 8 + 32, dtype=torch.float64, device="cuda")
    L = N.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: C.c_void_p(t.data_ptr())
    nd1 = 128 * 8 * 16

    def run_A():
        A.cores.fill_(float("nan"))
        N.check(L.tt_pstt2_begin(A.plan, p(ws), s), "begin")
        for a, cnt in _slabs(64, 16, 2):
            N.check(L.tt_pstt2_accumulate(A.plan, p(X[a * nd1:]), a, cnt, p(ws), s), "accumulate")
        N.check(L.tt_pstt2_finalize(A.plan, p(ws), p(A.cores), p(A.ranks), s), "finalize")
        torch.cuda.synchronize()
        return A.reconstruct(torch.float64).cpu().numpy()

    first = run_A()
    assert np.linalg.norm(first - x) / np.linalg.norm(x) <= 1e-5
    got = [run_A()]
    ws.fill_(float("nan"))
    L.tt_workspace_release(p(ws))
    got.append(run_A())
    N.check(L.tt_pstt2(B.plan, p(XB), p(ws), p(B.cores), p(B.ranks), s), "tt_pstt2 B")
    torch.cuda.synchronize()
    ws.fill_(float("nan"))
    got.append(run_A())
    for i, g in enumerate(got):
        assert np.all(np.isfinite(g)), i
        assert np.linalg.norm(g - first) / np.linalg.norm(first) <= 1e-6, i
