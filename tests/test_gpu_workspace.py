"""Plans taking turns on one caller workspace.

The workspace holds the device tables of the plan that last used it; the
library re-sends a plan's tables whenever the workspace last held another
plan's, and refuses calls that would read state another plan has replaced.
Each decomposition is checked against the FP64 oracle."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch, _native as N


def _p(t):
    return C.c_void_p(t.data_ptr())


def _s():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _cases():
    dA = [16] * 4
    xA = ti.random_tt(dA, [1, 3, 4, 3, 1], seed=0)
    kA = dict(ranks=[1, 4, 4, 4, 1], p=5, seed=1)
    dB = [128, 16, 24, 128]
    xB = ti.hilbert_type(dB, np.float32)
    kB = dict(eps=1e-6, rmax=6, p=10, seed=1)
    A = TTSketch(dA, x_dtype=torch.float64, prec="fp64", **kA)
    B = TTSketch(dB, x_dtype=torch.float32, prec="bf16", **kB)
    refA = OT.tt_full(OP.pstt2(xA, dA, **kA)["cores"])
    refB = OT.tt_full(OP.pstt2(xB.astype(np.float64), dB, **kB)["cores"])
    return [(A, torch.tensor(xA, device="cuda"), refA, 1e-10),
            (B, torch.tensor(xB, device="cuda"), refB, 1e-5)]


@pytest.mark.gpu
def test_plans_alternating_on_one_workspace_match_the_oracle():
    cases = _cases()
    nbytes = max(t.ws_bytes for t, *_ in cases)
    ws = torch.empty(nbytes // 8 + 32, dtype=torch.float64, device="cuda")
    L = N.lib()
    for t, X, ref, tol in cases + cases[::-1] + cases:
        t.cores.fill_(float("nan"))
        N.check(L.tt_pstt2(t.plan, _p(X), _p(ws), _p(t.cores), _p(t.ranks), _s()), "tt_pstt2")
        torch.cuda.synchronize()
        got = t.reconstruct(torch.float64).cpu().numpy()  # (its own workspace)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, (t.dims, err)


@pytest.mark.gpu
def test_state_replaced_by_another_plan_is_refused():
    (A, XA, refA, tolA), (B, XB, _, _) = _cases()
    nbytes = max(A.ws_bytes, B.ws_bytes)
    ws = torch.empty(nbytes // 8 + 32, dtype=torch.float64, device="cuda")
    L = N.lib()
    nd1 = 16 ** 3
    # a streaming decomposition of A whose workspace B takes over midway
    N.check(L.tt_pstt2_begin(A.plan, _p(ws), _s()), "begin")
    N.check(L.tt_pstt2_accumulate(A.plan, _p(XA[:8 * nd1]), 0, 8, _p(ws), _s()), "acc")
    N.check(L.tt_pstt2(B.plan, _p(XB), _p(ws), _p(B.cores), _p(B.ranks), _s()), "B")
    assert L.tt_pstt2_accumulate(A.plan, _p(XA[8 * nd1:]), 8, 8, _p(ws), _s()) == N.TT_ERR_STATE
    assert L.tt_pstt2_finalize(A.plan, _p(ws), _p(A.cores), _p(A.ranks), _s()) == N.TT_ERR_STATE
    # accumulate on a workspace other than the one begun on
    N.check(L.tt_pstt2_begin(A.plan, _p(ws), _s()), "begin")
    assert L.tt_pstt2_accumulate(A.plan, _p(XA), 0, 16, _p(A.ws), _s()) == N.TT_ERR_STATE
    # the backward needs this plan's forward state in this workspace
    N.check(L.tt_pstt2(A.plan, _p(XA), _p(ws), _p(A.cores), _p(A.ranks), _s()), "A")
    dX = torch.empty_like(XA)
    dc = torch.randn_like(A.cores)
    N.check(L.tt_pstt2_backward(A.plan, _p(ws), _p(dc), _p(dX), _s()), "backward")
    assert L.tt_pstt2_backward(A.plan, _p(A.ws), _p(dc), _p(dX), _s()) == N.TT_ERR_STATE
    N.check(L.tt_pstt2(B.plan, _p(XB), _p(ws), _p(B.cores), _p(B.ranks), _s()), "B")
    assert L.tt_pstt2_backward(A.plan, _p(ws), _p(dc), _p(dX), _s()) == N.TT_ERR_STATE
    # after a release the next call sends the tables again and works
    torch.cuda.synchronize()
    L.tt_workspace_release(_p(ws))
    N.check(L.tt_pstt2(A.plan, _p(XA), _p(ws), _p(A.cores), _p(A.ranks), _s()), "A")
    torch.cuda.synchronize()
    got = A.reconstruct(torch.float64).cpu().numpy()
    assert np.linalg.norm(got - refA) / np.linalg.norm(refA) <= tolA


def test_release_and_state_checks_need_no_device():
    """Host-side: release of unknown or NULL addresses is a no-op; a backward
    before any forward and an accumulate before begin are refused before
    anything reaches a device."""
    L = N.lib()
    L.tt_workspace_release(None)
    L.tt_workspace_release(C.c_void_p(4096))
    q = N.make_problem([8, 8, 8], ranks=[1, 2, 2, 1], p=3, seed=1)
    h = C.c_void_p()
    N.check(L.tt_sketch_plan(C.byref(q), C.byref(h)), "plan")
    try:
        dummy = C.c_void_p(256)
        assert L.tt_pstt2_backward(h, dummy, dummy, dummy, None) == N.TT_ERR_STATE
        assert L.tt_pstt2_accumulate(h, dummy, 0, 8, dummy, None) == N.TT_ERR_STATE
        assert L.tt_pstt2_finalize(h, dummy, dummy, dummy, None) == N.TT_ERR_STATE
    finally:
        L.tt_plan_destroy(h)
