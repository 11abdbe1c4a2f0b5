"""Sampled scenario paths for the scenario-tree construction (paper §6.2:
10^4 Monte-Carlo scenarios of the day-ahead price from a fitted time-series
model).  The model of the paper (an ARIMA fit to the EXAA prices) is not
available; the stand-in is an AR(1) deviation of the log price around the
generator's lognormal level with a daily profile, seeded.  Returns paths of
shape (S, N, dim): dim independent series (dim = 1: the price)."""
from __future__ import annotations

import numpy as np


def make_price_paths(S: int, N: int = 24, dim: int = 1, seed: int = 5, phi: float = 0.8,
                     sigma: float = 0.3, hour0: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    hours = hour0 + np.arange(1, N + 1)
    profile = 0.2 * np.sin(2.0 * np.pi * (hours - 6) / 24.0)
    dev = np.zeros((S, dim))
    out = np.empty((S, N, dim))
    innov = sigma * np.sqrt(1.0 - phi * phi)
    for t in range(N):
        dev = phi * dev + innov * rng.standard_normal((S, dim))
        out[:, t, :] = 0.1 * np.exp(profile[t] + dev)
    return out
