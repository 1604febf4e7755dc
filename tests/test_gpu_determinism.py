"""Run-to-run agreement (the determinism check of the test plan): the same
decomposition twice on the same plan and workspace.  The sketches are summed
with atomics in whatever order the CTAs reach them, so bits may differ; the
results must agree to the summation-order noise of each path (FP64: 1e-12 of
||X||; FP16 slab kernel: FP32 partial sums, 1e-6), with the same ranks."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from paper_2111_10448_gb300 import TTSketch
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,kw,bar", [
    ([24, 10, 12, 20], dict(ranks=[1, 3, 4, 3, 1], p=5, prec="fp64", x_dtype=torch.float64), 1e-12),
    ([256, 16, 16, 64], dict(eps=1e-6, rmax=6, p=10, prec="fp16", drm="kr", x_scale_log2=16), 1e-6),
    ([24, 6, 5, 24], dict(eps=1e-5, rmax=16, p=10, prec="bf16"), 1e-6),
])
def test_two_runs_agree(dims, kw, bar):
    dt = kw.get("x_dtype", torch.float32)
    x = (ti.random_tt(dims, [1, 3, 3, 3, 1], seed=6, noise=1e-6) if dims[0] != 256
         else ti.hilbert_type(dims, np.float32))
    X = to_dev(x, dt)
    t = TTSketch(dims, seed=8, **kw)
    outs = []
    for _ in range(2):
        t.pstt2(X)
        outs.append((t.status(), t.reconstruct().cpu().numpy()))
    assert outs[0][0] == outs[1][0]
    assert np.linalg.norm(outs[0][1] - outs[1][1]) <= bar * np.linalg.norm(x)
