"""Helpers shared by the GPU parity tests (marshalling only)."""

import numpy as np
import torch


def dev():
    return torch.device("cuda:0")


def t32(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=dev())


def t64(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=dev())


def np64(t):
    return t.detach().double().cpu().numpy()


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)


def product_bound(X, F, rtol):
    """Elementwise tolerance rtol * (|X| |F|) for a product accumulated in float32."""
    return rtol * (np.abs(X) @ np.abs(F)) + 1e-30
