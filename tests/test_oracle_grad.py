"""Pins of the reference gradient (oracle/grad.py): the torch map equals the
NumPy oracle's forward map, and its autograd gradient matches FP64 central
finite differences of the NumPy oracle (which recomputes its own pivots)."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import grad as OG, pstt2 as OP, tt as OT


def fd_instance():
    """d = 3, n = 8: rank-(1,4,4,1) cores plus 1e-2 relative noise, target
    ranks (1,2,2,1), p = 5, so that the map truncates (non-trivial)."""
    dims = [8, 8, 8]
    x = ti.random_tt(dims, [1, 4, 4, 1], seed=0, noise=1e-2)
    return dims, x, [1, 2, 2, 1], 5


def test_torch_map_equals_numpy_oracle():
    for dims, r, target in [([8, 8, 8], [1, 4, 4, 1], [1, 2, 2, 1]), ([5, 4, 6, 3, 4], [1, 3, 3, 3, 2, 1], [1, 2, 3, 2, 2, 1]),
                            ([7, 9], [1, 3, 1], [1, 2, 1])]:
        x = ti.random_tt(dims, r, seed=3, noise=1e-2)
        ref = OG.forward_ref(x, dims, ranks=target, p=4, seed=2)
        ct = OG.cores_torch(torch.tensor(x), dims, ref)
        full_t = OG.full_torch(ct).numpy()
        np.testing.assert_allclose(full_t, OT.tt_full(ref["cores"]), atol=1e-12 * np.abs(x).max())
        for a, b in zip(ct, ref["cores"]):
            np.testing.assert_allclose(a.numpy(), b, atol=1e-11)


def test_gradient_matches_central_finite_differences():
    dims, x, target, p = fd_instance()
    T = ti.target_tensor(x.size, seed=3)
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=1)
    L0, g = OG.loss_and_grad(x, dims, ref, T)

    def loss_np(xx):
        o = OP.pstt2(xx, dims, ranks=target, p=p, seed=1, passes=1)
        return float(np.sum((OT.tt_full(o["cores"]) - T) ** 2))

    assert abs(loss_np(x) - L0) <= 1e-12 * L0
    rng = np.random.default_rng(0)
    h = 1e-6
    idx = rng.choice(x.size, size=40, replace=False)
    fd = np.array([(loss_np(x + h * np.eye(1, x.size, i)[0]) - loss_np(x - h * np.eye(1, x.size, i)[0])) / (2 * h)
                   for i in idx])
    np.testing.assert_allclose(g[idx], fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())
    # a random direction (all entries at once)
    v = rng.standard_normal(x.size)
    dd = (loss_np(x + h * v) - loss_np(x - h * v)) / (2 * h)
    assert abs(dd - g @ v) <= 1e-6 * abs(dd)


def test_planted_gradient_mistake_is_caught(monkeypatch):
    """Dropping the sign normalisation of the QR changes nothing (gauge), but a
    transposed least-squares solve must break the finite-difference pin."""
    dims, x, target, p = fd_instance()
    T = ti.target_tensor(x.size, seed=3)
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=1)
    orig = torch.linalg.solve
    monkeypatch.setattr(torch.linalg, "solve", lambda A, B: orig(A.T + 0.01 * torch.eye(A.shape[0], dtype=A.dtype), B))
    L1, _ = OG.loss_and_grad(x, dims, ref, T)
    o = OP.pstt2(x, dims, ranks=target, p=p, seed=1, passes=1)
    L0 = float(np.sum((OT.tt_full(o["cores"]) - T) ** 2))
    assert abs(L1 - L0) > 1e-6 * L0


def test_gradient_with_khatri_rao_test_matrices_matches_finite_differences():
    """The same pin with Khatri-Rao test matrices (the map depends on them only
    through the sketches, so the adjoint has the same form)."""
    dims, x, target, p = fd_instance()
    T = ti.target_tensor(x.size, seed=3)
    ref = OG.forward_ref(x, dims, ranks=target, p=p, seed=1, drm="kr")
    L0, g = OG.loss_and_grad(x, dims, ref, T)

    def loss_np(xx):
        o = OP.pstt2(xx, dims, ranks=target, p=p, seed=1, passes=1, drm="kr")
        return float(np.sum((OT.tt_full(o["cores"]) - T) ** 2))

    assert abs(loss_np(x) - L0) <= 1e-12 * L0
    rng = np.random.default_rng(1)
    h = 1e-6
    v = rng.standard_normal(x.size)
    dd = (loss_np(x + h * v) - loss_np(x - h * v)) / (2 * h)
    assert abs(dd - g @ v) <= 1e-6 * abs(dd)
    idx = rng.choice(x.size, size=20, replace=False)
    fd = np.array([(loss_np(x + h * np.eye(1, x.size, i)[0]) - loss_np(x - h * np.eye(1, x.size, i)[0])) / (2 * h)
                   for i in idx])
    np.testing.assert_allclose(g[idx], fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())
