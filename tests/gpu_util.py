"""Helpers for the GPU tests (numpy views of device results)."""
import numpy as np


def np_(t):
    return t.detach().cpu().numpy()


def colmajor_np(t):
    """numpy copy of a column-major device matrix."""
    return np.asfortranarray(np_(t))
