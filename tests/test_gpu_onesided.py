"""GPU parity of the one-sided PSTT-onepass (Algorithm 2 with the single-pass
last core; TT_FLAG_ONESIDED) against the oracle's pstt_onepass.

Bars as for the two-sided path: FP64 within 1e-10 of the oracle; mixed
precision sketches equal to the oracle's products of the split X with its
rounded test matrices up to the rounding-flip bound, and X~ within 10 eps of
the FP64 oracle in tolerance mode."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import philox, pstt as PO, tt as OT
from paper_2111_10448_gb300 import TTSketch
from tests.gpu_util import rel, sketch_dict, to_dev

pytestmark = pytest.mark.gpu


def _split(x, prec):
    hi = philox.round_to(x, prec)
    lo = philox.round_to(x - hi, prec)
    return hi + lo


def _close(G, S, what):
    fro = np.linalg.norm(G - S) / np.linalg.norm(S)
    mx = np.max(np.abs(G - S)) / np.max(np.abs(S))
    assert fro <= 1e-4 and mx <= 2e-3, (what, fro, mx)


@pytest.mark.parametrize("dims,kw", [
    ([30, 25], dict(ranks=[1, 4, 1], p=3)),                          # d = 2
    ([6, 5, 4, 7], dict(ranks=[1, 2, 3, 2, 1], p=3)),                # fixed ranks
    ([8, 7, 6, 5, 9], dict(eps=1e-6, rmax=8, p=4)),                  # tolerance mode, d = 5
    ([40, 36, 50], dict(ranks=[1, 5, 6, 1], p=5)),                   # n > 32: the generic kernels
])
def test_fp64_matches_oracle(dims, kw):
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=11, noise=1e-6)
    t = TTSketch(dims, seed=5, x_dtype=torch.float64, prec="fp64", one_sided=True, **kw)
    t.pstt2(to_dev(x, torch.float64))
    o = PO.pstt_onepass(x, dims, seed=5, **kw)
    assert t.status()[1] == o["r"]
    got = OT.tt_full(t.core_list(0))
    assert np.linalg.norm(got - OT.tt_full(o["cores"])) <= 1e-10 * np.linalg.norm(x)
    assert [g.shape for g in t.core_list(0)] == [g.shape for g in o["cores"]]


@pytest.mark.parametrize("dims,kw", [
    ([9, 8, 7, 6, 9], dict(ranks=[1, 3, 5, 4, 3, 1], p=6)),          # n <= 32: the small-plane kernel
    ([40, 12, 48], dict(ranks=[1, 4, 4, 1], p=6)),                   # the generic tile kernel
])
@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_sketches_match_oracle(dims, kw, prec):
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=12, noise=1e-5).astype(np.float32)
    t = TTSketch(dims, seed=6, x_dtype=torch.float32, prec=prec, one_sided=True, **kw)
    t.begin()
    t.accumulate(to_dev(x), 0, dims[-1])
    sk = sketch_dict(t)
    t.finalize()
    o = PO.pstt_onepass(_split(x.astype(np.float64), prec), dims, seed=6, test_fmt=prec, **kw)
    assert sorted(sk) == [(0, k) for k in range(1, d)] + [(1, d - 1)]
    for k in range(1, d):
        _close(sk[(0, k)], o["S"][k], ("S", k))
    _close(sk[(1, d - 1)], o["T"].T, "T")


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_within_10eps_of_oracle(prec):
    dims, eps = [10] * 5, 1e-5
    x = ti.random_tt(dims, [1, 6, 8, 8, 6, 1], seed=0, noise=1e-6).astype(np.float32)
    x64 = x.astype(np.float64)
    t = TTSketch(dims, eps=eps, rmax=12, p=10, seed=1, x_dtype=torch.float32, prec=prec, one_sided=True)
    t.pstt2(to_dev(x))
    o = PO.pstt_onepass(x64, dims, eps=eps, rmax=12, p=10, seed=1)
    xt = t.reconstruct().cpu().numpy()
    e_or, e_x = rel(xt, OT.tt_full(o["cores"]), x64), rel(xt, x64, x64)
    print(f"one-sided {prec}: |X~-X~oracle|={e_or:.2e} |X~-X|={e_x:.2e} ranks={t.status()[1]} / {o['r']}")
    assert e_or <= 10 * eps and e_x <= 10 * eps


@pytest.mark.parametrize("dims,kw", [
    ([30, 25], dict(ranks=[1, 4, 1], p=3)),
    ([6, 5, 4, 7], dict(ranks=[1, 2, 3, 2, 1], p=3)),
    ([8, 7, 6, 5, 9], dict(eps=1e-6, rmax=8, p=4)),
    ([40, 36, 50], dict(ranks=[1, 5, 6, 1], p=5)),
])
@pytest.mark.parametrize("xdt", [torch.float64, torch.float32])
def test_twopass_fp64_matches_oracle(dims, kw, xdt):
    """Algorithm 2 proper (one-sided, two passes): the last core from a second
    pass over X, G_d = Q_{d-1}^T X_{d-1}; FP64 within 1e-10 of the oracle."""
    d = len(dims)
    x = ti.random_tt(dims, [1] + [3] * (d - 1) + [1], seed=13, noise=1e-6)
    if xdt == torch.float32:
        x = x.astype(np.float32).astype(np.float64)
    t = TTSketch(dims, seed=5, x_dtype=xdt, prec="fp64", one_sided=True, passes=2, **kw)
    t.pstt2(to_dev(x, xdt))
    o = PO.pstt(x, dims, seed=5, **kw)
    assert t.status()[1] == o["r"]
    got = OT.tt_full(t.core_list(0))
    assert np.linalg.norm(got - OT.tt_full(o["cores"])) <= 1e-10 * np.linalg.norm(x)
