"""GPU parity of Khatri-Rao test matrices (TT_FLAG_KR; Sec. 3.2, eq.
(sketch_orig)) against the oracle with drm='kr', through the C ABI, on every
sketch kernel that regenerates test matrices: the FP64 kernel, the generic
tensor-core tile kernel, the small-plane kernel and the tcgen05 plane kernel,
plus the middle-core solve and the backward.

Bars as for dense test matrices: the FP64 path within 1e-10 of the oracle's
X~ (1e-12 of X on exact-rank inputs); mixed sketches equal to the oracle's
FP64 products of the split X with the oracle's Khatri-Rao matrices rounded
to the MMA type up to the rounding-flip bound (the GPU multiplies FP32
factors from the FP32 generator; the product can land on the other side of a
rounding boundary for a small fraction of entries): Frobenius 1e-4, max 2e-3
of max |S|; X~ within 10 eps in tolerance mode; the VJP within 1e-6 (FP64)."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import grad as OG, philox, pstt as PO, pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch, _native as N
from tests.gpu_util import rel, sketch_dict, to_dev

pytestmark = pytest.mark.gpu


def _split(x, prec, s=0):
    """hi + lo of X 2^s in the MMA type, at the scale of X (s: FP16 only)."""
    xs = np.asarray(x, dtype=np.float64) * 2.0 ** s
    hi = philox.round_to(xs, prec)
    lo = philox.round_to(xs - hi, prec)
    return (hi + lo) * 2.0 ** -s


def _scale_of(x, prec):
    """FP16 scale exponent (the rule of tt_x_scale_log2); 0 otherwise."""
    return 15 - int(np.frexp(float(np.max(np.abs(x))))[1]) if prec == "fp16" else 0


def _close(G, S, what):
    fro = np.linalg.norm(G - S) / np.linalg.norm(S)
    mx = np.max(np.abs(G - S)) / np.max(np.abs(S))
    assert fro <= 1e-4 and mx <= 2e-3, (what, fro, mx)


@pytest.mark.parametrize("passes", [1, 2])
def test_fp64_config1_exact_recovery(passes):
    dims = [16] * 4
    x = ti.random_tt(dims, [1, 3, 4, 3, 1], seed=0)
    t = TTSketch(dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1, passes=passes, x_dtype=torch.float64, prec="fp64",
                 drm="kr").pstt2(to_dev(x, torch.float64))
    o = OP.pstt2(x, dims, ranks=[1, 4, 4, 4, 1], p=5, seed=1, passes=passes, drm="kr")
    xt = t.reconstruct().cpu().numpy()
    assert rel(xt, x, x) <= 1e-12
    assert rel(xt, OT.tt_full(o["cores"]), x) <= 1e-10
    assert t.status() == (0, o["r"])


@pytest.mark.parametrize("dims,kw", [
    ([6, 5, 7, 4], dict(ranks=[1, 2, 3, 2, 1], p=4)),
    ([70, 3, 45], dict(ranks=[1, 3, 4, 1], p=5)),
    ([5, 4, 6, 3, 4, 5], dict(eps=1e-6, rmax=6, p=4)),
])
def test_fp64_sketches_and_cores_match_oracle(dims, kw):
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=3, noise=1e-6)
    t = TTSketch(dims, seed=4, x_dtype=torch.float64, prec="fp64", drm="kr", **kw)
    t.begin()
    t.accumulate(to_dev(x, torch.float64), 0, dims[-1])
    sk = sketch_dict(t)
    t.finalize()
    o = OP.pstt2(x, dims, seed=4, drm="kr", **kw)
    for k, S in o["sketch"]["S"].items():
        assert np.abs(sk[(0, k)] - S).max() <= 1e-12 * np.abs(S).max(), ("S", k)
    for k, R in o["sketch"]["R"].items():
        assert np.abs(sk[(1, k)] - R).max() <= 1e-12 * np.abs(R).max(), ("R", k)
    assert t.status()[1] == o["r"]
    assert rel(OT.tt_full(t.core_list(0)), OT.tt_full(o["cores"]), x) <= 1e-10


def test_fp64_streaming_slabs_equal_one_shot():
    dims = [8, 6, 5, 12]
    x = ti.random_tt(dims, [1, 3, 3, 3, 1], seed=6, noise=1e-3)
    X = to_dev(x, torch.float64)
    kw = dict(ranks=[1, 3, 3, 3, 1], p=4, seed=2, x_dtype=torch.float64, prec="fp64", drm="kr")
    one = TTSketch(dims, **kw).pstt2(X)
    t = TTSketch(dims, **kw)
    nd1 = 8 * 6 * 5
    t.begin()
    for a, c in [(7, 5), (0, 3), (3, 4)]:
        t.accumulate(X[a * nd1:(a + c) * nd1].clone(), a, c)
    t.finalize()
    assert rel(one.reconstruct().cpu().numpy(), t.reconstruct().cpu().numpy(), x) <= 1e-12


@pytest.mark.parametrize("dims,kw,kind", [
    ([40, 7, 6, 70], dict(ranks=[1, 4, 5, 4, 1], p=6), 1),             # generic tile kernel
    ([9, 8, 7, 6, 5, 9], dict(eps=1e-5, rmax=6, p=6), 3),              # small-plane kernel
    ([24, 6, 5, 24], dict(eps=1e-5, rmax=16, p=10), 3),                # small-plane, l = 26
    ([256, 3, 4, 256], dict(eps=1e-6, rmax=6, p=10), 2),               # tcgen05 slab kernel, 64 slices a launch
    ([128, 64, 48, 128], dict(eps=1e-6, rmax=6, p=10), 2),             # the same, several tiles a CTA
    ([256, 7, 128], dict(ranks=[1, 4, 4, 1], p=12), 1),                # d = 3: the generic kernel
])
@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_mixed_sketches_match_oracle(dims, kw, kind, prec):
    if kind == 2 and prec == "tf32":
        pytest.skip("the tcgen05 kernels are BF16 / FP16 only")
    if kind == 1 and prec != "bf16" and len(dims) == 3:
        pytest.skip("covered in BF16")
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=5, noise=1e-5).astype(np.float32)
    s = _scale_of(x, prec)
    t = TTSketch(dims, seed=7, x_dtype=torch.float32, prec=prec, drm="kr", x_scale_log2=s, **kw)
    assert t.kernel_kind() == kind
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = {k: v * 2.0 ** -s for k, v in sketch_dict(t).items()}
    t.finalize()
    widths = OP.sketch_widths(d, OP.clamp_ranks(dims, kw["ranks"]) if "ranks" in kw else None, kw["p"],
                              "eps" in kw, kw.get("rmax"))
    o = OP.sketches(_split(x.astype(np.float64), prec, s), dims, widths, 7, 1, test_fmt=prec, drm="kr")
    for k, S in o["S"].items():
        _close(sk[(0, k)], S, ("S", k))
    for k, R in o["R"].items():
        _close(sk[(1, k)], R, ("R", k))


@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_mixed_within_10eps_of_oracle(prec):
    dims, eps = [32] * 4, 1e-6
    x = ti.hilbert_type(dims, np.float32)
    x64 = x.astype(np.float64)
    t = TTSketch(dims, eps=eps, rmax=6, p=10, seed=1, prec=prec, drm="kr",
                 x_scale_log2=_scale_of(x, prec)).pstt2(to_dev(x))
    o = OP.pstt2(x64, dims, eps=eps, rmax=6, p=10, seed=1, drm="kr")
    xt = t.reconstruct().cpu().numpy()
    assert rel(xt, OT.tt_full(o["cores"]), x64) <= 10 * eps
    assert rel(xt, x64, x64) <= 10 * eps


def test_tcgen05_pipeline_within_10eps():
    """The whole one-pass pipeline on the tcgen05 slab kernel (several tiles a
    CTA), Khatri-Rao test matrices: X~ within 10 eps of X and of the FP64 path
    (the middle-core solve regenerates the Khatri-Rao Omega_{d*} the sketch
    used)."""
    dims = [128, 64, 48, 128]
    Xd = torch.empty(int(np.prod(dims)), dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 4)(*dims)
    N.check(N.lib().tt_generate_hilbert_type(4, nn, 0, dims[-1], C.c_void_p(Xd.data_ptr()), N.TT_F32, None), "gen")
    t = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="bf16", drm="kr")
    assert t.kernel_kind() == 2
    t.pstt2(Xd)
    f = TTSketch(dims, eps=1e-6, rmax=6, p=10, seed=1, prec="fp64", drm="kr").pstt2(Xd)
    e_x = t.error(Xd).cpu().numpy()
    e_f = t.error(f.reconstruct(torch.float32)).cpu().numpy()
    rx, rf = (e_x[0] / e_x[1]) ** 0.5, (e_f[0] / e_x[1]) ** 0.5
    print(f"KR plane-kernel pipeline: |X~-X|={rx:.2e} |X~-X~fp64|={rf:.2e} ranks={t.status()[1]}")
    assert rx <= 1e-5 and rf <= 1e-5


@pytest.mark.parametrize("dims,r,target,p", [
    ([8, 8, 8], [1, 4, 4, 1], [1, 2, 2, 1], 5),
    ([6, 5, 7, 4], [1, 3, 4, 3, 1], [1, 2, 3, 2, 1], 4),
])
def test_vjp_matches_oracle(dims, r, target, p):
    x = ti.random_tt(dims, r, seed=4, noise=1e-2)
    t = TTSketch(dims, ranks=target, p=p, seed=2, x_dtype=torch.float64, prec="fp64", drm="kr")
    t.pstt2(to_dev(x, torch.float64))
    _, ranks = t.status()
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=2, drm="kr")
    assert ranks == ref["r"]
    rng = np.random.default_rng(1)
    it = t.items[0]
    dc = np.zeros(t.cores.numel())
    lst = []
    for k in range(1, it["d"] + 1):
        rp0, rp1, n = it["rpad"][k - 1], it["rpad"][k], it["dims"][k - 1]
        g = rng.standard_normal((ranks[k - 1], n, ranks[k]))
        G = np.zeros((rp0, n, rp1))
        G[:ranks[k - 1], :, :ranks[k]] = g
        dc[it["core_off"][k]:it["core_off"][k] + G.size] = G.ravel(order="F")
        lst.append(g)
    dX = torch.empty(x.size, dtype=torch.float64, device="cuda")
    t.backward(torch.tensor(dc, device="cuda"), dX)
    want = OG.cores_vjp(x, dims, ref, lst)
    err = np.linalg.norm(dX.cpu().numpy() - want) / np.linalg.norm(want)
    assert err <= 1e-6, err


@pytest.mark.parametrize("dims,kw", [
    ([6, 5, 4, 7], dict(ranks=[1, 2, 3, 2, 1], p=3)),
    ([8, 7, 6, 5, 9], dict(eps=1e-6, rmax=8, p=4)),
])
def test_one_sided_fp64_matches_oracle(dims, kw):
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=11, noise=1e-6)
    t = TTSketch(dims, seed=5, x_dtype=torch.float64, prec="fp64", one_sided=True, drm="kr", **kw)
    t.pstt2(to_dev(x, torch.float64))
    o = PO.pstt_onepass(x, dims, seed=5, drm="kr", **kw)
    assert t.status()[1] == o["r"]
    assert rel(OT.tt_full(t.core_list(0)), OT.tt_full(o["cores"]), x) <= 1e-10


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_vjp_mixed_matches_rounded_oracle(prec):
    """Mixed-precision backward with Khatri-Rao test matrices (the last row
    sketch mode by mode, as the forward took it) against the oracle gradient
    of the map with the same rounded test matrices."""
    dims, r, target, p = [6, 5, 7, 4], [1, 3, 4, 3, 1], [1, 2, 3, 2, 1], 4
    x = ti.random_tt(dims, r, seed=4, noise=1e-2).astype(np.float32).astype(np.float64)
    t = TTSketch(dims, ranks=target, p=p, seed=2, x_dtype=torch.float32, prec=prec, drm="kr")
    t.pstt2(to_dev(x, torch.float32))
    _, ranks = t.status()
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=2, test_fmt=prec, drm="kr")
    assert ranks == ref["r"]
    rng = np.random.default_rng(1)
    it = t.items[0]
    dc = np.zeros(t.cores.numel())
    lst = []
    for k in range(1, it["d"] + 1):
        rp0, rp1, n = it["rpad"][k - 1], it["rpad"][k], it["dims"][k - 1]
        g = rng.standard_normal((ranks[k - 1], n, ranks[k]))
        G = np.zeros((rp0, n, rp1))
        G[:ranks[k - 1], :, :ranks[k]] = g
        dc[it["core_off"][k]:it["core_off"][k] + G.size] = G.ravel(order="F")
        lst.append(g)
    dX = torch.empty(x.size, dtype=torch.float32, device="cuda")
    t.backward(torch.tensor(dc, device="cuda"), dX)
    want = OG.cores_vjp(x, dims, ref, lst)
    err = np.linalg.norm(dX.double().cpu().numpy() - want) / np.linalg.norm(want)
    print(f"{prec} KR VJP rel err vs rounded oracle: {err:.2e}")
    assert err <= 1e-4, err


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_one_sided_mixed_sketches_match_oracle(prec):
    """One-sided PSTT-onepass, Khatri-Rao: T_{d-1} is the mode-by-mode row
    sketch of X_{d-1}, and its least-squares matrix B uses the same entries."""
    dims, kw = [9, 8, 7, 6, 9], dict(ranks=[1, 3, 5, 4, 3, 1], p=6)
    x = ti.random_tt(dims, [1, 3, 3, 3, 3, 1], seed=12, noise=1e-5).astype(np.float32)
    t = TTSketch(dims, seed=6, x_dtype=torch.float32, prec=prec, one_sided=True, drm="kr", **kw)
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = sketch_dict(t)
    t.finalize()
    o = PO.pstt_onepass(_split(x.astype(np.float64), prec), dims, seed=6, test_fmt=prec, drm="kr", **kw)
    for k, S in o["S"].items():
        _close(sk[(0, k)], S, ("S", k))
    _close(sk[(1, len(dims) - 1)], o["T"].T, "T")
    x64 = x.astype(np.float64)
    f = PO.pstt_onepass(x64, dims, seed=6, drm="kr", **kw)
    assert rel(OT.tt_full(t.core_list(0)), OT.tt_full(f["cores"]), x64) <= 1e-3
