"""Shared helpers of the parity tests: oracle reference runs and comparisons."""
from __future__ import annotations

import numpy as np

import oracle as O


def psnr(est: np.ndarray, ref: np.ndarray, mask: np.ndarray) -> float:
    """10 log10(255^2 / MSE), MSE pooled over the masked (loss) pixels."""
    d = (est - ref)[mask]
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(255.0 ** 2 / mse)


class OracleSetup:
    """Oracle dictionary, weights and tables of one workload (shared pattern)."""

    def __init__(self, basis, M, N, rho_hat, support, numeric=None, tables=True):
        self.phi = O.dictionary(basis, M, N, numeric)
        self.dup = O.find_duplicates(self.phi)
        self.w = O.weights(M, N, rho_hat, support)
        self.support = support
        if tables:
            self.C, self.D = O.fase_tables(self.phi, self.w)

    def se(self, s, gamma, I):
        return O.se_original(self.phi, self.w, s, gamma, I, self.dup)

    def fase_batch(self, s, gamma, I, nthreads=0):
        return O.fase_batch(self.phi, self.w, self.C, self.D, s, gamma, I, self.dup, nthreads)


def first_near_tie(margin: np.ndarray, tau: float) -> int:
    """Index of the first iteration whose oracle tie margin is <= tau (len if none)."""
    bad = np.nonzero(margin <= tau)[0]
    return int(bad[0]) if len(bad) else len(margin)


def coef_rel_err(c: np.ndarray, c_ref: np.ndarray) -> np.ndarray:
    """|c - c_ref| / max(|c_ref|, 1e-12 max|c_ref|) per iteration."""
    floor = 1e-12 * np.max(np.abs(c_ref)) if c_ref.size else 0.0
    return np.abs(c - c_ref) / np.maximum(np.abs(c_ref), floor)
