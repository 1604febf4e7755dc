"""Second workloads of the paper's experiments (Sec. 4.3-4.4): its Hilbert
tensor 1/(1 - d + i_1 + ... + i_d) and the sum of Gaussian bumps, decomposed
in tolerance mode by the FP64 GPU path (parity with the oracle, 1e-10) and by
the BF16 plane kernel (10 eps of the oracle)."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch


def _run(x, dims, prec, **kw):
    xd = torch.tensor(x, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    t = TTSketch(dims, x_dtype=xd.dtype, prec=prec, **kw).pstt2(xd)
    torch.cuda.synchronize()
    return t


@pytest.mark.gpu
@pytest.mark.parametrize("name,dims,eps,rmax", [
    ("hilbert", [20, 20, 20, 20], 1e-8, 12),
    ("bumps", [24, 24, 24], 1e-6, 12),
    ("hilbert", [12, 12, 12, 12, 12], 1e-6, 10),
])
def test_fp64_matches_oracle(name, dims, eps, rmax):
    x = ti.hilbert_paper(dims) if name == "hilbert" else ti.gaussian_bumps(dims, nbumps=6)
    t = _run(x, dims, "fp64", eps=eps, rmax=rmax, p=6, seed=2)
    o = OP.pstt2(x, dims, eps=eps, rmax=rmax, p=6, seed=2)
    st, ranks = t.status()
    assert ranks == o["r"]
    got = OT.tt_full(t.core_list(0))
    nx = np.linalg.norm(x)
    assert np.linalg.norm(got - OT.tt_full(o["cores"])) <= 1e-10 * nx
    if st == 0:
        assert np.linalg.norm(got - x) <= eps * nx


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["hilbert", "bumps"])
def test_bf16_plane_kernel_within_10eps(name):
    dims = [128, 12, 12, 128]
    x = (ti.hilbert_paper(dims) if name == "hilbert" else ti.gaussian_bumps(dims, nbumps=5)).astype(np.float32)
    eps = 1e-5
    t = _run(x, dims, "bf16", eps=eps, rmax=10, p=6, seed=2)     # l = 16: the plane kernel's shape
    assert t.kernel_kind() == 2
    x64 = x.astype(np.float64)
    o = OP.pstt2(x64, dims, eps=eps, rmax=10, p=6, seed=2)
    got = OT.tt_full(t.core_list(0))
    nx = np.linalg.norm(x64)
    err = np.linalg.norm(got - OT.tt_full(o["cores"])) / nx
    print(f"{name}: bf16 plane kernel vs oracle {err:.2e}, ranks {t.status()[1]} / {o['r']}")
    assert err <= 10 * eps


# ------------------------------------------------- device input generators
def _gen(kind, dims, first, count, dtype, **kw):
    import ctypes as C
    from paper_2111_10448_gb300 import _native as N
    inner = int(np.prod(dims[:-1]))
    out = torch.empty(inner * count, dtype=dtype, device="cuda")
    nn = (C.c_int64 * len(dims))(*dims)
    dt = N.TT_F64 if dtype == torch.float64 else N.TT_F32
    if kind == "hilbert":
        st = N.lib().tt_generate_hilbert(len(dims), nn, first, count, C.c_void_p(out.data_ptr()), dt, None)
    else:
        c = np.ascontiguousarray(kw["centres"], dtype=np.float64)
        st = N.lib().tt_generate_gaussian_bumps(len(dims), nn, c.shape[0], kw["gamma"],
                                               c.ctypes.data_as(C.c_void_p), first, count,
                                               C.c_void_p(out.data_ptr()), dt, None)
    N.check(st, kind)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_device_hilbert_equals_host(dtype):
    """The paper's Hilbert tensor on the device, whole and as a slab of the
    last mode, equals the host generator bit for bit (exact integer sum, one
    division, one rounding)."""
    dims = [7, 5, 6, 9]
    npd = np.float64 if dtype == torch.float64 else np.float32
    x = ti.hilbert_paper(dims, dtype=npd).reshape(dims, order="F")
    assert np.array_equal(_gen("hilbert", dims, 0, 9, dtype), x.reshape(-1, order="F"))
    assert np.array_equal(_gen("hilbert", dims, 3, 4, dtype), x[..., 3:7].reshape(-1, order="F"))


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_device_bumps_match_host(dtype):
    """Gaussian bumps on the device against the host generator: the same sum
    order, so the values differ only through the two libraries' exp (FP64:
    1e-14 relative; FP32: at most one rounding step)."""
    dims, nb, gamma = [9, 7, 8], 6, 10.0
    npd = np.float64 if dtype == torch.float64 else np.float32
    x = ti.gaussian_bumps(dims, nbumps=nb, gamma=gamma, seed=4).reshape(dims, order="F")
    c = ti.bump_centres(3, nb, seed=4)
    for first, count in [(0, 8), (2, 3)]:
        got = _gen("bumps", dims, first, count, dtype, centres=c, gamma=gamma).astype(np.float64)
        ref = x[..., first:first + count].reshape(-1, order="F")
        if dtype == torch.float64:
            assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-14
        else:
            assert np.max(np.abs(got - ref.astype(np.float32)) / np.abs(ref)) <= 2 ** -23


@pytest.mark.gpu
@pytest.mark.parametrize("dims,ranks", [
    ([40, 40, 40], [1, 25, 25, 1]),                        # Table 1, d = 3 rank profile
    ([10, 10, 10, 10, 10], [1, 10, 18, 18, 10, 1]),        # Table 1, d = 5 (17 clamped to N_1 = 10)
    ([3] * 9, [1, 3, 9, 18, 19, 19, 18, 9, 3, 1]),         # Table 1, d = 9 (clamped to min(N_k, M_k))
])
def test_table1_rank_profiles_fp64_match_oracle(dims, ranks):
    """Fixed-rank mode with the rank profiles of the paper's Table 1 on the
    paper's Hilbert tensor at reduced n (generated on the device): the FP64
    GPU path equals the oracle to 1e-10."""
    import ctypes as C
    from paper_2111_10448_gb300 import _native as N
    d = len(dims)
    x = ti.hilbert_paper(dims)
    xd = torch.empty(x.size, dtype=torch.float64, device="cuda")
    nn = (C.c_int64 * d)(*dims)
    N.check(N.lib().tt_generate_hilbert(d, nn, 0, dims[-1], C.c_void_p(xd.data_ptr()), N.TT_F64, None), "gen")
    t = TTSketch(dims, ranks=ranks, p=10, seed=2, x_dtype=torch.float64, prec="fp64").pstt2(xd)
    o = OP.pstt2(x, dims, ranks=ranks, p=10, seed=2)
    assert t.status()[1] == o["r"]
    got = OT.tt_full(t.core_list(0))
    ref = OT.tt_full(o["cores"])
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(x)
