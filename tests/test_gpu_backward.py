"""GPU parity of the backward (adjoint) of the one-pass PSTT2 map and of the
reconstruction, through the C ABI, against the torch-autograd oracle gradient
(oracle/grad.py, itself pinned by finite differences) and against central
finite differences of the GPU forward map.  Bar: 1e-6 relative (the FP64
path; the FP32 storage of X is the same on both sides)."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import grad as OG, philox
from paper_2111_10448_gb300 import PSTT2Fn, TTReconstructFn, TTSketch
from paper_2111_10448_gb300 import _native as NN
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def padded_dcores(t, ranks, rng):
    """Random upstream gradient in the padded core layout, zero outside the
    actual ranks, plus the same as a list of unpadded arrays."""
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
    return dc, lst


@pytest.mark.parametrize("dims,r,target,p", [
    ([8, 8, 8], [1, 4, 4, 1], [1, 2, 2, 1], 5),
    ([6, 5, 7, 4], [1, 3, 4, 3, 1], [1, 2, 3, 2, 1], 4),
    ([5, 4, 6, 3, 4], [1, 3, 3, 3, 2, 1], [1, 2, 3, 2, 2, 1], 4),
    ([9, 11], [1, 4, 1], [1, 3, 1], 3),
    ([70, 3, 45], [1, 3, 4, 1], [1, 3, 3, 1], 4),
])
def test_vjp_matches_oracle(dims, r, target, p):
    x = ti.random_tt(dims, r, seed=4, noise=1e-2)
    t = TTSketch(dims, ranks=target, p=p, seed=2, x_dtype=torch.float64, prec="fp64")
    t.pstt2(to_dev(x, torch.float64))
    _, ranks = t.status()
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=2)
    assert ranks == ref["r"]
    rng = np.random.default_rng(1)
    dc, lst = padded_dcores(t, ranks, rng)
    dX = torch.empty(x.size, dtype=torch.float64, device="cuda")
    t.backward(torch.tensor(dc, device="cuda"), dX)
    got = dX.cpu().numpy()
    want = OG.cores_vjp(x, dims, ref, lst)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-6, err


def _loss_grad_gpu(x, dims, target, p, T, x_dtype=torch.float64, prec="fp64"):
    t = TTSketch(dims, ranks=target, p=p, seed=1, x_dtype=x_dtype, prec=prec, diff=True)
    X = to_dev(x, x_dtype).requires_grad_(True)
    cores = PSTT2Fn.apply(X, t)
    Xt = TTReconstructFn.apply(cores, t, torch.float64)
    L = torch.sum((Xt - torch.tensor(T, device="cuda")) ** 2)
    L.backward()
    return float(L.detach()), X.grad.detach().cpu().numpy().astype(np.float64), t


def test_full_loss_gradient_matches_finite_differences():
    """FP64 central differences (h = 1e-6) of the GPU loss on the d = 3,
    n = 8 instance: rank-(1,4,4,1) cores + 1e-2 noise, target ranks (1,2,2,1)."""
    dims, target, p = [8, 8, 8], [1, 2, 2, 1], 5
    x = ti.random_tt(dims, [1, 4, 4, 1], seed=0, noise=1e-2)
    T = ti.target_tensor(x.size, seed=3)
    L0, g, _ = _loss_grad_gpu(x, dims, target, p, T)
    rng = np.random.default_rng(0)
    h = 1e-6

    def loss_at(xx):
        t = TTSketch(dims, ranks=target, p=p, seed=1, x_dtype=torch.float64, prec="fp64").pstt2(to_dev(xx, torch.float64))
        return float(np.sum((t.reconstruct().cpu().numpy() - T) ** 2))

    idx = rng.choice(x.size, size=30, replace=False)
    fd = np.array([(loss_at(x + h * np.eye(1, x.size, i)[0]) - loss_at(x - h * np.eye(1, x.size, i)[0])) / (2 * h)
                   for i in idx])
    np.testing.assert_allclose(g[idx], fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())
    v = rng.standard_normal(x.size)
    dd = (loss_at(x + h * v) - loss_at(x - h * v)) / (2 * h)
    assert abs(dd - g @ v) <= 1e-6 * abs(dd)
    # and the oracle gradient of the same instance
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=1)
    L1, g1 = OG.loss_and_grad(x, dims, ref, T)
    assert abs(L1 - L0) <= 1e-10 * L1
    assert np.linalg.norm(g - g1) / np.linalg.norm(g1) <= 1e-6


def test_config5_gradient_matches_oracle():
    """d = 5, n = 32, FP32 X from rank-8 random TT cores, fixed N(0,1) target
    T (seed 3), target ranks 8, p = 5: GPU gradient (FP64 path) vs the oracle
    gradient, 1e-6 relative."""
    dims, p = [32] * 5, 5
    x = ti.random_tt(dims, [1, 8, 8, 8, 8, 1], seed=0).astype(np.float32).astype(np.float64)
    T = ti.target_tensor(x.size, seed=3)
    target = [1, 8, 8, 8, 8, 1]
    L0, g, t = _loss_grad_gpu(x.astype(np.float32), dims, target, p, T, x_dtype=torch.float32)
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=1)
    L1, g1 = OG.loss_and_grad(x, dims, ref, T)
    err = np.linalg.norm(g - g1) / np.linalg.norm(g1)
    print(f"config5: L gpu={L0:.10e} oracle={L1:.10e} grad rel err={err:.2e}")
    assert abs(L1 - L0) <= 1e-6 * L1
    assert err <= 1e-6


def test_reconstruct_backward_matches_autograd():
    dims = [5, 6, 4, 7]
    x = ti.random_tt(dims, [1, 3, 3, 3, 1], seed=2, noise=1e-3)
    t = TTSketch(dims, ranks=[1, 3, 3, 3, 1], p=3, seed=4, x_dtype=torch.float64, diff=True).pstt2(to_dev(x, torch.float64))
    T = ti.target_tensor(x.size, seed=5)
    cores = t.cores.clone().requires_grad_(True)
    Xt = TTReconstructFn.apply(cores, t, torch.float64)
    L = torch.sum((Xt - torch.tensor(T, device="cuda")) ** 2)
    L.backward()
    got = cores.grad.cpu().numpy()
    # torch autograd of the padded contraction, on the CPU
    it = t.items[0]
    cc = torch.tensor(t.cores.cpu().numpy(), requires_grad=True)
    Gs = []
    for k in range(1, 5):
        rp0, rp1, n = it["rpad"][k - 1], it["rpad"][k], it["dims"][k - 1]
        off = it["core_off"][k]
        Gs.append(cc[off:off + rp0 * n * rp1].reshape(rp1, n, rp0).permute(2, 1, 0))
    Lt = torch.sum((OG.full_torch(Gs) - torch.tensor(T)) ** 2)
    Lt.backward()
    want = cc.grad.numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-10


@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_vjp_mixed_precision_matches_rounded_oracle(prec):
    """Mixed paths: the adjoint runs in FP32 with the rounded test matrices;
    compared with the oracle gradient of the map whose test matrices are
    rounded to the same type (the FP32 generator flips a few rounding
    decisions, and X is FP32, so the bar is looser than the FP64 path's).
    FP16 plans take the SIMT adjoint; the power-of-two scale of their split
    does not enter the gradient."""
    dims, r, target, p = [6, 5, 7, 4], [1, 3, 4, 3, 1], [1, 2, 3, 2, 1], 4
    x = ti.random_tt(dims, r, seed=4, noise=1e-2).astype(np.float32).astype(np.float64)
    s = 15 - int(np.frexp(float(np.max(np.abs(x))))[1]) if prec == "fp16" else 0
    t = TTSketch(dims, ranks=target, p=p, seed=2, x_dtype=torch.float32, prec=prec, x_scale_log2=s)
    t.pstt2(to_dev(x, torch.float32))
    _, ranks = t.status()
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=2, test_fmt=prec)
    assert ranks == ref["r"]
    dc, lst = padded_dcores(t, ranks, np.random.default_rng(1))
    dX = torch.empty(x.size, dtype=torch.float32, device="cuda")
    t.backward(torch.tensor(dc, device="cuda"), dX)
    got = dX.double().cpu().numpy()
    want = OG.cores_vjp(x, dims, ref, lst)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print(f"{prec} VJP rel err vs rounded oracle: {err:.2e}")
    assert err <= 1e-4, err


def _gpu_test_matrices(ref, dims, seed, prec):
    """The test matrices exactly as the GPU draws them (tt_test_matrix: the
    FP32 generator rounded to the MMA type), in the oracle's layout."""
    code = {"bf16": NN.TT_PREC_BF16, "tf32": NN.TT_PREC_TF32}[prec]
    out = {"Omega": {}, "Psi": {}}
    for key, mats in (("Omega", ref["sketch"]["Omega"]), ("Psi", ref["sketch"]["Psi"])):
        for k, M in mats.items():
            rows, l = M.shape
            sid = k if key == "Omega" else 64 + k
            buf = torch.empty(rows * l, dtype=torch.float64, device="cuda")
            NN.check(NN.lib().tt_test_matrix(seed, sid, 0, rows, l, code, C.c_void_p(buf.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)), "tm")
            out[key][k] = buf.cpu().numpy().reshape(l, rows).T.copy()
    return out


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("dims,r,target,p,slabs", [
    ([12, 10, 9, 8, 14], [1, 3, 4, 4, 3, 1], [1, 2, 3, 3, 2, 1], 5, None),   # widths 7..8, lpad 16
    ([32, 6, 5, 32], [1, 4, 5, 4, 1], [1, 4, 8, 4, 1], 20, [(16, 16), (0, 16)]),  # widths 24..28, lpad 32, streamed
])
def test_tensor_core_sketch_adjoint_matches_rounded_oracle(prec, dims, r, target, p, slabs):
    """The tensor-core sketch adjoint (planes of at most 32 x 32: one warp a
    plane, the split sketch adjoints times the test-matrix rows on mma.sync).
    (1) Against the oracle gradient of the map whose test matrices are the
    GPU's own (exported with tt_test_matrix), linearised where the forward
    linearised: the mixed sketches see X as its two-term split hi + lo in the
    MMA type, so the oracle takes x' = hi + lo.  What is left is FP32
    rounding -- of each FP64 adjoint (split exactly into three terms of the
    MMA type), of the adjoint's accumulation, and of the forward sketches'
    accumulation, which moves the linearisation point by ~2^-24 relative --
    times the conditioning kappa of the gradient map at this instance, which
    the oracle measures (relative change of its gradient over relative change
    of x from x to x'; ~3 on the first instance, ~130 on the second, whose
    middle rank 8 exceeds the tensor's rank 5): bar max(1e-5, 4 2^-24 kappa).
    (2) Against the oracle with its own
    rounded FP64 normals at x: the FP32 generator lands on the other BF16
    neighbour in under 0.5% of the entries (one ulp, 2^-8 relative), which
    moves the gradient by about sqrt(0.005) 2^-8 = 3e-4, and the split of X
    (2^-17) moves it by up to 3e-4 on the second instance, whose middle rank
    of 8 lies above the tensor's rank (the map is ill-conditioned there);
    TF32 is 8 to 40 times closer -- bar 1e-3.  A forward streamed in slabs leaves
    slab-sized staging tables, which the backward restages for the whole
    last mode."""
    x = ti.random_tt(dims, r, seed=4, noise=1e-2).astype(np.float32).astype(np.float64)
    t = TTSketch(dims, ranks=target, p=p, seed=2, x_dtype=torch.float32, prec=prec)
    X = to_dev(x, torch.float32)
    if slabs is None:
        t.pstt2(X)
    else:
        nd1 = int(np.prod(dims[:-1]))
        t.begin()
        for a, c in slabs:
            t.accumulate(X[a * nd1:(a + c) * nd1].clone(), a, c)
        t.finalize()
    _, ranks = t.status()
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=2, test_fmt=prec)
    assert ranks == ref["r"]
    dc, lst = padded_dcores(t, ranks, np.random.default_rng(3))
    dX = torch.full((x.size,), float("nan"), dtype=torch.float32, device="cuda")
    t.backward(torch.tensor(dc, device="cuda"), dX)
    got = dX.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    want = OG.cores_vjp(x, dims, ref, lst)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    own = dict(ref)
    own["sketch"] = dict(ref["sketch"], **_gpu_test_matrices(ref, dims, 2, prec))
    hi = philox.round_to(x, prec)
    xs = hi + philox.round_to(x - hi, prec)
    want_own = OG.cores_vjp(xs, dims, own, lst)
    err_own = np.linalg.norm(got - want_own) / np.linalg.norm(want_own)
    at_x = OG.cores_vjp(x, dims, own, lst)
    kappa = (np.linalg.norm(want_own - at_x) / np.linalg.norm(at_x)) / (np.linalg.norm(xs - x) / np.linalg.norm(x))
    bar = max(1e-5, 4 * 2.0 ** -24 * kappa)
    print(f"{prec} {dims} tensor-core adjoint rel err: vs the oracle with the GPU's test matrices {err_own:.2e} "
          f"(kappa {kappa:.0f}, bar {bar:.1e}), vs the oracle's own {err:.2e}")
    assert err_own <= bar, (err_own, bar)
    assert err <= 1e-3, err
