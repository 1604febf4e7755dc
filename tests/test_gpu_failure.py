"""Failure detection without a GPU fault: the bounded wait of the kernels
gives up on an mbarrier that nothing arrives at, raises the timeout bit, and
the context stays usable."""
import ctypes as C

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as OT
from paper_2111_10448_gb300 import TTSketch, _native as N


def test_selftest_rejects_bad_arguments():
    st = C.c_void_p(256)
    assert N.lib().tt_selftest_wait_timeout(0, st, None) == N.TT_ERR_INVALID_ARG
    assert N.lib().tt_selftest_wait_timeout(10**10, st, None) == N.TT_ERR_INVALID_ARG
    assert N.lib().tt_selftest_wait_timeout(1000, None, None) == N.TT_ERR_INVALID_ARG


@pytest.mark.gpu
def test_bounded_wait_gives_up_and_context_survives():
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    N.check(N.lib().tt_selftest_wait_timeout(2_000_000, C.c_void_p(st.data_ptr()), None), "selftest")
    torch.cuda.synchronize()
    assert int(st.item()) == 4
    # the context still runs a decomposition correctly
    x = ti.random_tt([16] * 4, [1, 3, 4, 3, 1], seed=0)
    t = TTSketch([16] * 4, ranks=[1, 4, 4, 4, 1], p=5, seed=1, x_dtype=torch.float64)
    t.pstt2(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    assert t.status()[0] == 0
    got = OT.tt_full(t.core_list(0))
    assert np.linalg.norm(got - x) <= 1e-12 * np.linalg.norm(x)
