"""Edge cases of the GPU path: the largest sketch width, modes of size one, the
all-zero tensor, and the empty slab."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTError, TTSketch, _native as N
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("passes", [1, 2])
def test_largest_width_64_matches_oracle(passes):
    """l = rmax + p = 64 (TT_MAXL) everywhere: 192-row TSQR leaves at this
    width (three levels for the 576-row sketch), FP64 within 1e-10."""
    dims = [24] * 4
    x = ti.random_tt(dims, [1, 6, 9, 6, 1], seed=2, noise=1e-3)
    kw = dict(eps=1e-9, rmax=54, p=10, seed=4, passes=passes)
    t = TTSketch(dims, x_dtype=torch.float64, prec="fp64", **kw).pstt2(to_dev(x, torch.float64))
    o = OP.pstt2(x, dims, **kw)
    assert max(o["widths"][1:]) == 64
    assert t.status()[1] == o["r"]
    assert rel(t.reconstruct().cpu().numpy(), OT.tt_full(o["cores"]), x) <= 1e-10


def test_largest_width_64_bf16_sketches():
    """The mixed path at width 64 (the generic tile kernel) against the oracle's
    BF16-rounded products."""
    from oracle import philox
    dims = [24] * 4
    x = ti.random_tt(dims, [1, 6, 9, 6, 1], seed=2, noise=1e-3).astype(np.float32)
    kw = dict(eps=1e-6, rmax=54, p=10, seed=4)
    t = TTSketch(dims, x_dtype=torch.float32, prec="bf16", **kw)
    t.begin()
    t.accumulate(to_dev(x), 0, 24)
    sk = {(ty, k): S.cpu().numpy() for ty, k, S in t.sketches(0)}
    t.finalize()
    hi = philox.round_to(x.astype(np.float64), "bf16")
    xs = hi + philox.round_to(x.astype(np.float64) - hi, "bf16")
    o = OP.pstt2(xs, dims, passes=1, test_fmt="bf16", **kw)
    for (ty, k), S in sk.items():
        ref = o["sketch"]["S" if ty == 0 else "R"][k]
        assert S.shape[1] == 64
        assert np.linalg.norm(S - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims,ranks", [([6, 1, 5, 7], [1, 2, 2, 3, 1]), ([1, 9, 8], [1, 1, 3, 1]),
                                        ([7, 6, 1], [1, 3, 1, 1])])
def test_modes_of_size_one(dims, ranks):
    """A mode of size 1 (first, middle or last): ranks clamp through it and the
    decomposition still equals the oracle's."""
    x = ti.random_tt(dims, [1] + [2] * (len(dims) - 1) + [1], seed=6, noise=1e-4)
    t = TTSketch(dims, ranks=ranks, p=3, seed=2, x_dtype=torch.float64, prec="fp64").pstt2(to_dev(x, torch.float64))
    o = OP.pstt2(x, dims, ranks=ranks, p=3, seed=2)
    assert t.status()[1] == o["r"]
    assert rel(t.reconstruct().cpu().numpy(), OT.tt_full(o["cores"]), x) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_zero_tensor_gives_zero_train(prec):
    """X = 0: every sketch is zero; the one-pass solve meets a zero B, which is
    flagged (status bit), and the cores reconstruct to exact zeros (no NaN)."""
    dims = [8, 7, 6, 9]
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.zeros(int(np.prod(dims)), dtype=dt, device="cuda")
    t = TTSketch(dims, ranks=[1, 2, 3, 2, 1], p=3, seed=1, x_dtype=dt, prec=prec).pstt2(X)
    xt = t.reconstruct(torch.float64).cpu().numpy()
    assert np.all(np.isfinite(xt)) and not xt.any()
    err = t.error(X).cpu().numpy()
    assert err[0] == 0.0


def test_empty_slab_is_refused():
    dims = [4, 4, 6]
    X = to_dev(np.ones(96), torch.float64)
    t = TTSketch(dims, ranks=[1, 2, 2, 1], p=2, x_dtype=torch.float64)
    t.begin()
    with pytest.raises(TTError) as e:
        t.accumulate(X[:16], 0, 0)
    assert e.value.status == N.TT_ERR_INVALID_ARG
    t.accumulate(X, 0, 6)   # the plan is still usable
    t.finalize()
    assert t.status()[0] in (0, N.TT_WARN_RANK_CAP)
