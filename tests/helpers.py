"""Shared helpers of the test-suite (no method arithmetic)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def to_np(t):
    try:
        return t.detach().cpu().numpy().astype(np.float64)
    except AttributeError:
        return np.asarray(t, dtype=np.float64)


PHYS = dict(tau=0.6, gravity=1e-5, density_contrast=1.0, settling_velocity=1e-3, diffusivity=1e-3)
