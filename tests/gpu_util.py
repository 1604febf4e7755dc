"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch


def to_dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def rel(a, b, ref):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(ref)))


def sketch_dict(t, item=0):
    """{(type, k): host array} of every sketch in the workspace."""
    return {(ty, k): S.cpu().numpy().copy() for ty, k, S in t.sketches(item)}
