"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def obj_tensor():
    import torch
    return torch.zeros(1, dtype=torch.float64, device="cuda")
