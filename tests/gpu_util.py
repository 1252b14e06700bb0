"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def sim(w, precision="fp32", capacity=None, **kw):
    need_gpu()
    from paper_2409_11470_gb300.binding import Simulation
    return Simulation(w, capacity=capacity, precision=precision, **kw)


def rows(off, idx):
    return [np.sort(idx[off[a]:off[a + 1]]) for a in range(len(off) - 1)]


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def with_velocities(w, sigma=0.1, seed=1):
    rng = np.random.default_rng(seed)
    n = len(w["p"]["x"])
    for f in ("vx", "vy", "vz"):
        w["p"][f] = rng.normal(0.0, sigma, n)
    return w
