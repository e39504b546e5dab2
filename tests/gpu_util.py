"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel_err(a, b, scale=None):
    """max |a - b| / max(|b|, scale) elementwise (scale defaults to 1)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.maximum(np.abs(b), 1.0 if scale is None else scale)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    d = np.where(both_inf, 0.0, np.abs(a - b))
    return float(np.max(d / s)) if d.size else 0.0


def soa(theta_rows):
    import torch
    return torch.tensor(np.ascontiguousarray(np.asarray(theta_rows).T), dtype=torch.float64,
                        device="cuda")
