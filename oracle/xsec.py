"""Reweighted cross sections and their errors (oracle; test infrastructure only).

Sec. 3.1.2 of the paper: for a sample with cross section sigma and error dsigma,
original weights w_i and reweighted weights w'_i (i = 1..N),

    sigma'  = C sum_i w'_i,                C the sample's normalisation,
    dsigma' = dsigma * (1/N) sum_i w'_i / w_i  +  sigma * std(w'),

and when dsigma' comes out infinite, NaN or non-positive it is replaced by
dsigma times the larger of sigma'/sigma and sigma/sigma'.

Readings (the paper leaves them open):
  * C = sigma / sum_i w_i, so that the original weights reproduce sigma;
  * std is the population standard deviation, sqrt((1/N) sum (w' - mean w')^2);
  * the mean of w'/w runs over the events with w_i != 0 (the ratio is undefined
    for the others);
  * the formula is applied as printed, including its units (the second term
    multiplies sigma by a spread of weights).
"""
from __future__ import annotations

import math

import numpy as np


def reweighted_xsec(w: np.ndarray, w_new: np.ndarray, sigma: float, dsigma: float):
    """w: [N] original weights; w_new: [N, k] reweighted weights.
    Returns (sigma' [k], dsigma' [k], fallback [k] bool)."""
    w = np.asarray(w, dtype=np.float64)
    w_new = np.asarray(w_new, dtype=np.float64)
    if w_new.ndim == 1:
        w_new = w_new[:, None]
    n = w.shape[0]
    c = sigma / np.sum(w)
    sig = c * np.sum(w_new, axis=0)
    nz = w != 0.0
    mean_ratio = np.mean(w_new[nz] / w[nz][:, None], axis=0) if np.any(nz) else np.full(w_new.shape[1], np.nan)
    std = np.sqrt(np.mean((w_new - np.mean(w_new, axis=0)) ** 2, axis=0))
    dsig = dsigma * mean_ratio + sigma * std
    fallback = ~np.isfinite(dsig) | (dsig <= 0.0)
    out = dsig.copy()
    for j in np.nonzero(fallback)[0]:
        r1 = sig[j] / sigma if sigma != 0.0 else math.inf
        r2 = sigma / sig[j] if sig[j] != 0.0 else math.inf
        out[j] = dsigma * max(r1, r2)
    assert n == w_new.shape[0]
    return sig, out, fallback
