"""Helpers shared by the GPU tests (no arithmetic of the method)."""
import numpy as np
import torch

DEV = torch.device("cuda:0")


def T(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def N(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
