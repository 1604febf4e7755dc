"""tt_pstt2_noalloc: the one-shot forward with the workspace in the library's
fixed device array, checked against tt_pstt2 with a caller workspace on the
same plan and input (two calls in a row, and alternating plans so that the
plan tables must be re-sent).  Collected last on purpose: it must also pass
after every other GPU test has run in the same process."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from paper_2111_10448_gb300 import TTSketch, _native as N

# status bits of the call -> the tt_status that tt_query_status reports
# (1 rank cap -> TT_WARN_RANK_CAP = 7, 2 singular -> 5, 4 timeout -> 6)

SCRATCH_BYTES = 32 << 20


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _noalloc(t, X, cores, ranks, status):
    return N.lib().tt_pstt2_noalloc(t.plan, _ptr(X), _ptr(cores), _ptr(ranks),
                                    _ptr(status) if status is not None else None, None)


def _cases():
    # plain FP64 (d=4, n=16, true ranks (1,3,4,3,1), target 4, p 5) and a
    # BF16 shape served by the tensor-core plane kernel
    x1 = ti.random_tt([16] * 4, [1, 3, 4, 3, 1], seed=0)
    yield "fp64", torch.tensor(x1, dtype=torch.float64, device="cuda"), dict(
        dims=[16] * 4, ranks=[1, 4, 4, 4, 1], p=5, seed=1, x_dtype=torch.float64)
    dims = [128, 16, 24, 128]
    x2 = ti.hilbert_type(dims)
    yield "bf16", torch.tensor(x2, dtype=torch.float32, device="cuda"), dict(
        dims=dims, eps=1e-6, rmax=6, p=10, seed=1, x_dtype=torch.float32, prec="bf16")


@pytest.mark.gpu
def test_noalloc_matches_caller_workspace_two_calls_in_a_row():
    for name, X, kw in _cases():
        dims = kw.pop("dims")
        t = TTSketch(dims, **kw).pstt2(X)
        torch.cuda.synchronize()
        st_ref, ranks_ref = t.status()
        ref = t.reconstruct(torch.float64).cpu().numpy()
        nrm = np.linalg.norm(ref)
        tol = 1e-12 if name == "fp64" else 1e-9
        for call in range(2):
            cores = torch.full_like(t.cores, float("nan"))
            ranks = torch.full_like(t.ranks, -1)
            status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            N.check(_noalloc(t, X, cores, ranks, status), "tt_pstt2_noalloc")
            torch.cuda.synchronize()
            assert ranks.cpu().tolist() == t.ranks.cpu().tolist(), (name, call)
            bits = int(status.item())
            decoded = 5 if bits & 2 else 6 if bits & 4 else 7 if bits & 1 else 0
            assert decoded == st_ref, (name, call, bits, st_ref)
            got = t.reconstruct(torch.float64, cores=cores).cpu().numpy()
            err = np.linalg.norm(got - ref) / nrm
            assert err <= tol, (name, call, err)


@pytest.mark.gpu
def test_backward_after_noalloc_is_refused():
    """The no-alloc call keeps its saved state in the library array, which no
    caller can name: a backward on any caller workspace afterwards is
    refused, even one that held this plan's state from an earlier forward."""
    name, X, kw = next(_cases())
    dims = kw.pop("dims")
    t = TTSketch(dims, **kw).pstt2(X)
    dc = torch.zeros_like(t.cores)
    dX = torch.empty_like(X)
    t.backward(dc, dX)  # accepted: the forward state is in t.ws
    cores = torch.zeros_like(t.cores)
    ranks = torch.zeros_like(t.ranks)
    N.check(_noalloc(t, X, cores, ranks, None), "tt_pstt2_noalloc")
    st = N.lib().tt_pstt2_backward(t.plan, _ptr(t.ws), _ptr(dc), _ptr(dX), None)
    assert st == N.TT_ERR_STATE
    torch.cuda.synchronize()


@pytest.mark.gpu
def test_noalloc_alternating_plans_resend_tables():
    cases = list(_cases())
    runs = []
    for name, X, kw in cases:
        kw = dict(kw)
        dims = kw.pop("dims")
        t = TTSketch(dims, **kw).pstt2(X)
        torch.cuda.synchronize()
        runs.append((name, X, t, t.reconstruct(torch.float64).cpu().numpy()))
    for name, X, t, ref in runs + runs[::-1] + runs:
        cores = torch.zeros_like(t.cores)
        ranks = torch.zeros_like(t.ranks)
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        N.check(_noalloc(t, X, cores, ranks, status), "tt_pstt2_noalloc")
        torch.cuda.synchronize()
        got = t.reconstruct(torch.float64, cores=cores).cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= (1e-12 if name == "fp64" else 1e-9), (name, err)


def test_noalloc_refuses_a_workspace_above_the_fixed_size():
    """Refused before anything touches a device (so it runs without a GPU)."""
    pr = N.make_problem([256, 256, 256, 256], eps=1e-6, rmax=6, p=10, seed=1)
    h = C.c_void_p()
    N.check(N.lib().tt_sketch_plan(C.byref(pr), C.byref(h)), "plan")
    try:
        ws = C.c_size_t()
        N.check(N.lib().tt_plan_sizes(h, C.byref(ws), None, None), "sizes")
        assert ws.value > SCRATCH_BYTES
        dummy = C.c_void_p(256)
        assert N.lib().tt_pstt2_noalloc(h, dummy, dummy, dummy, None, None) == N.TT_ERR_UNSUPPORTED
        assert N.lib().tt_pstt2_noalloc(h, None, dummy, dummy, None, None) == N.TT_ERR_INVALID_ARG
    finally:
        N.lib().tt_plan_destroy(h)
