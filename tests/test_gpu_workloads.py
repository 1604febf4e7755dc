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
