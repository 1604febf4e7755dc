"""Checkpoint / resume of a stream (tt_pstt2_export_state / import_state):
half of the slabs on one plan and workspace, the state exported to the host,
the rest on a NEW plan object and workspace after import.  The result equals
the uninterrupted stream's up to summation order (FP64 path: 1e-12; FP16
slab kernel: the FP32 accumulation order, 1e-6 as for any change of slab
order), and the slab bookkeeping travels with the state (a slab added before
the export is refused after the import)."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from paper_2111_10448_gb300 import TTSketch, TTError, _native as N
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,kw,c,bar", [
    ([20, 9, 8, 30], dict(ranks=[1, 4, 5, 4, 1], p=5, prec="fp64", x_dtype=torch.float64), 5, 1e-12),
    ([256, 16, 16, 64], dict(eps=1e-6, rmax=6, p=10, prec="fp16", drm="kr", x_scale_log2=16), 16, 1e-6),
])
def test_resume_equals_uninterrupted_stream(dims, kw, c, bar):
    dt = kw.get("x_dtype", torch.float32)
    x = (ti.random_tt(dims, [1, 3, 3, 3, 1], seed=3, noise=1e-6) if kw["prec"] == "fp64"
         else ti.hilbert_type(dims, np.float32))
    X = to_dev(x, dt)
    nd1 = int(np.prod(dims[:-1]))
    slabs = list(range(0, dims[-1], c))
    one = TTSketch(dims, seed=4, **kw)
    one.begin()
    for a in slabs:
        one.accumulate(X[a * nd1:(a + c) * nd1], a, c)
    one.finalize()
    first = TTSketch(dims, seed=4, **kw)
    first.begin()
    for a in slabs[: len(slabs) // 2]:
        first.accumulate(X[a * nd1:(a + c) * nd1], a, c)
    state = first.export_state()
    del first
    second = TTSketch(dims, seed=4, **kw)
    second.import_state(state)
    with pytest.raises(TTError) as ei:   # already in the state
        second.accumulate(X[:c * nd1], 0, c)
    assert ei.value.status == N.TT_ERR_STATE
    for a in slabs[len(slabs) // 2:]:
        second.accumulate(X[a * nd1:(a + c) * nd1], a, c)
    second.finalize()
    assert second.status() == one.status()
    assert rel(one.reconstruct().cpu().numpy(), second.reconstruct().cpu().numpy(), x) <= bar
    # a state of another problem is refused
    other = TTSketch(dims, seed=5, **kw)
    with pytest.raises(TTError) as ei:
        other.import_state(state)
    assert ei.value.status == N.TT_ERR_INVALID_ARG
