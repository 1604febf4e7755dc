"""Reference gradient of the PSTT2-onepass map (torch CPU float64 autograd).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The one-pass map X -> TT cores (Sec. 3.2: sketches, QR of the selected
pivot columns, the least-squares middle core of eq. (3.3), the core products
of eq. (3.1) and its row mirror) is smooth once the column pivots and the
ranks are frozen at the values of a forward run.  This module writes that map
with plain torch operations (matmul, torch.linalg.qr, torch.linalg.solve) on
the oracle's dense test matrices and lets torch.autograd differentiate it.
It shares nothing with the CUDA path.

Index maps (column-major, Sec. 2.1): a flat tensor x gives the unfolding
X_k[u, v] = x[u + N_k v], i.e. x.reshape(M_k, N_k).T in torch's row-major
terms; a matrix whose rows are indexed u + N_{k-1} i reshapes to [i, u, .]
with .reshape(n_k, N_{k-1}, .).

Pinned by central finite differences of the NumPy oracle's own forward map
(oracle.pstt2, which recomputes its pivots): tests/test_oracle_grad.py.
"""
import numpy as np
import torch

from .pstt2 import pstt2, split_index
from .tt import prods

F64 = torch.float64


def _qr_pos(A):
    """Reduced QR with diag(R) >= 0."""
    Q, R = torch.linalg.qr(A, mode="reduced")
    s = torch.sign(torch.diagonal(R))
    s = torch.where(s == 0, torch.ones_like(s), s)
    return Q * s[None, :]


def cores_torch(x, dims, ref):
    """The one-pass cores (list of [a, i, c] tensors) as a function of x
    (torch float64, flat column-major), with the pivots, ranks and test
    matrices of the forward run `ref` (an oracle.pstt2 result)."""
    dims = [int(n) for n in dims]
    d = len(dims)
    ds = split_index(d)
    N = prods(dims)
    r = ref["r"]
    Om, Ps = ref["sketch"]["Omega"], ref["sketch"]["Psi"]

    def unf(k):
        return x.reshape(N[d] // N[k], N[k]).T

    Q, P = {}, {}
    for k in range(1, d):
        if k < ds:
            Y = unf(k) @ torch.as_tensor(Om[k], dtype=F64)
        else:
            Y = unf(k).T @ torch.as_tensor(Ps[k], dtype=F64)
        A = Y[:, torch.as_tensor(np.asarray(ref["piv"][k][:r[k]]))]
        (Q if k < ds else P)[k] = _qr_pos(A)

    cores = [None] * (d + 1)
    if ds >= 2:
        cores[1] = Q[1].unsqueeze(0)
    for k in range(2, ds):
        cores[k] = torch.einsum("ua,iuc->aic", Q[k - 1], Q[k].reshape(dims[k - 1], N[k - 1], r[k]))
    for k in range(ds + 1, d):
        Mk = N[d] // N[k]
        cores[k] = torch.einsum("via,vc->aic", P[k - 1].reshape(Mk, dims[k - 1], r[k - 1]), P[k])
    cores[d] = P[d - 1].T.unsqueeze(2)
    Omd = torch.as_tensor(Om[ds], dtype=F64)
    S = unf(ds) @ Omd
    B = P[ds].T @ Omd
    H = torch.linalg.solve(B @ B.T, B @ S.T).T          # argmin ||H B - S||
    Ql = Q[ds - 1] if ds >= 2 else torch.ones(1, 1, dtype=F64)
    cores[ds] = torch.einsum("ua,iuc->aic", Ql, H.reshape(dims[ds - 1], N[ds - 1], r[ds]))
    return cores[1:]


def full_torch(cores):
    """Column-major flat tensor of TT cores: L_k[u + N_{k-1} i, c] =
    sum_a L_{k-1}[u, a] G_k[a, i, c]."""
    L = torch.ones(1, 1, dtype=F64)
    for G in cores:
        T = torch.einsum("ua,aic->iuc", L, G)
        L = T.reshape(T.shape[0] * T.shape[1], T.shape[2])
    return L[:, 0]


def loss_and_grad(x, dims, ref, target):
    """L = ||X~(x) - T||_F^2 and dL/dx (numpy float64), pivots/ranks frozen."""
    xt = torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    L = torch.sum((full_torch(cores_torch(xt, dims, ref)) - torch.as_tensor(target, dtype=F64)) ** 2)
    L.backward()
    return float(L.detach()), xt.grad.numpy().copy()


def cores_vjp(x, dims, ref, dcores):
    """sum_k <dcores_k, d cores_k / dx> (numpy float64)."""
    xt = torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    cores = cores_torch(xt, dims, ref)
    s = sum(torch.sum(G * torch.as_tensor(np.asarray(g), dtype=F64)) for G, g in zip(cores, dcores))
    s.backward()
    return xt.grad.numpy().copy()


def forward_ref(x, dims, *, ranks, p, seed, test_fmt="f64", drm="gauss"):
    """A forward oracle run whose pivots and ranks freeze the map."""
    return pstt2(x, dims, ranks=ranks, p=p, seed=seed, passes=1, test_fmt=test_fmt, drm=drm)
