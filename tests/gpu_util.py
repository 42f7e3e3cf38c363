"""Helpers shared by the GPU parity tests."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32_nodes(x):
    """Nodes as the FP32 path sees them, returned in FP64 for the oracle."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def cplx_dev(z, dtype=None):
    import torch
    dtype = dtype or torch.complex64
    return torch.from_numpy(np.ascontiguousarray(np.asarray(z, dtype=np.complex128))).to(
        device="cuda", dtype=dtype).contiguous()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)
