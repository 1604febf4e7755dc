"""GPU parity of Tucker2TT (Algorithm 3): the decomposition of the Tucker
core by the library, then the per-core mode-2 products (tt_core_mode2),
against the oracle (FP64 within 1e-10)."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as OT, tucker as TU
from paper_2111_10448_gb300 import tucker2tt

pytestmark = pytest.mark.gpu


def _case(s, n, ranks, seed, noise):
    rng = np.random.default_rng(seed)
    G = ti.random_tt(s, ranks, seed=seed, noise=noise)
    A = [np.linalg.qr(rng.standard_normal((nk, sk)))[0] for nk, sk in zip(n, s)]
    return G, A


def _trim(cores, r):
    return [c.cpu().numpy()[:r[k], :, :r[k + 1]] for k, c in enumerate(cores)]


@pytest.mark.parametrize("s,n,kw", [
    ([4, 5, 3, 4], [9, 7, 8, 6], dict(ranks=[1, 3, 3, 3, 1], p=3)),
    ([6, 5, 6], [40, 33, 50], dict(eps=1e-8, rmax=6, p=4)),
    ([5, 4, 6, 5, 4], [11, 9, 12, 10, 8], dict(ranks=[1, 3, 4, 4, 3, 1], p=4, passes=2)),
])
def test_tucker2tt_matches_oracle(s, n, kw):
    d = len(s)
    G, A = _case(s, n, [1] + [3] * (d - 1) + [1], seed=31, noise=1e-4)
    cores, t = tucker2tt(torch.tensor(G, device="cuda"), [torch.tensor(a, device="cuda") for a in A],
                         prec="fp64", seed=9, **kw)
    ref, o = TU.tucker2tt(G, A, seed=9, **kw)
    r = t.status()[1]
    assert r == o["r"]
    got = OT.tt_full(_trim(cores, r))
    want = OT.tt_full(ref)
    assert [c.shape[1] for c in cores] == n
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_core_mode2_padded_rows_stay_zero():
    """The padded rank rows and columns of a core stay zero in its product."""
    rng = np.random.default_rng(2)
    H = np.zeros((4, 3, 5))
    H[:2, :, :3] = rng.standard_normal((2, 3, 3))
    A = rng.standard_normal((7, 3))
    import ctypes as C
    from paper_2111_10448_gb300 import _native as N
    Hd = torch.tensor(H.reshape(-1, order="F"), device="cuda")
    Ad = torch.tensor(A.reshape(-1, order="F"), device="cuda")
    Td = torch.empty(4 * 7 * 5, dtype=torch.float64, device="cuda")
    N.check(N.lib().tt_core_mode2(C.c_void_p(Hd.data_ptr()), 4, 3, 5, C.c_void_p(Ad.data_ptr()), 7,
                                  C.c_void_p(Td.data_ptr()), None), "mode2")
    T = Td.cpu().numpy().reshape((4, 7, 5), order="F")
    np.testing.assert_allclose(T, TU.mode2(H, A), rtol=0, atol=1e-13)
    assert not T[2:].any() and not T[:, :, 3:].any()


@pytest.mark.parametrize("tr", [[2, 6, 6, 2], [2, 4, 3, 2]])
def test_tt2tucker_matches_oracle(tr):
    """TT2Tucker (Algorithm 4): the factors and Tucker-core train against the
    oracle (FP64 within 1e-10), exact when t_k >= rank (T_k)_(2)."""
    from paper_2111_10448_gb300 import tt2tucker
    rng = np.random.default_rng(4)
    n, r = [9, 12, 10, 7], [1, 2, 3, 2, 1]
    T = [rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(4)]
    Hs, As = tt2tucker([torch.tensor(t, device="cuda") for t in T], tr, p=4, seed=3)
    Hr, Ar = TU.tt2tucker(T, tr, p=4, seed=3)
    for k in range(4):
        t = Ar[k].shape[1]
        A = As[k].cpu().numpy()
        H = Hs[k].cpu().numpy()
        assert np.abs(A[:, t:]).max(initial=0.0) == 0.0 and np.abs(H[:, t:, :]).max(initial=0.0) == 0.0
        np.testing.assert_allclose(A[:, :t], Ar[k], rtol=0, atol=1e-10)
        np.testing.assert_allclose(H[:, :t, :], Hr[k], rtol=0, atol=1e-10 * np.abs(Hr[k]).max())
    Xt = OT.tt_full([h.cpu().numpy() for h in Hs]).reshape([a.shape[1] for a in As], order="F")
    for k, A in enumerate(As):
        Xt = np.moveaxis(np.tensordot(A.cpu().numpy(), Xt, axes=([1], [k])), 0, k)
    X = OT.tt_full(T)
    err = np.linalg.norm(Xt.reshape(-1, order="F") - X) / np.linalg.norm(X)
    if tr == [2, 6, 6, 2]:
        assert err <= 1e-12
    print(f"tt2tucker t={tr}: |X~-X|/|X| = {err:.2e}")
