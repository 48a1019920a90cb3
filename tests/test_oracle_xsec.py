"""The reweighted cross-section oracle (Sec. 3.1.2) against closed forms and
brute force (CPU)."""
import math

import numpy as np

from oracle import xsec


def test_unchanged_weights_reproduce_the_sample():
    w = np.full(1000, 2.5)
    s, ds, fb = xsec.reweighted_xsec(w, w[:, None], 7.0, 0.3)
    assert np.allclose(s, 7.0, rtol=1e-15) and np.allclose(ds, 0.3, rtol=1e-15) and not fb.any()


def test_uniform_scaling():
    """w' = lam w with equal weights: sigma' = lam sigma, std = 0, dsigma' = lam dsigma."""
    w = np.full(512, 0.25)
    lam = np.array([0.5, 2.0, 3.0])
    s, ds, fb = xsec.reweighted_xsec(w, w[:, None] * lam[None, :], 4.0, 0.1)
    assert np.allclose(s, 4.0 * lam, rtol=1e-15) and np.allclose(ds, 0.1 * lam, rtol=1e-14)


def test_brute_force_loop():
    g = np.random.default_rng(3)
    w = g.uniform(0.5, 1.5, 200)
    w[7] = 0.0                               # excluded from the ratio mean only
    wn = w[:, None] * g.uniform(0.8, 1.2, (200, 3))
    sigma, dsigma = 12.0, 0.4
    s, ds, _ = xsec.reweighted_xsec(w, wn, sigma, dsigma)
    for j in range(3):
        tot = 0.0
        for i in range(200):
            tot += wn[i, j]
        c = sigma / sum(w)
        assert math.isclose(s[j], c * tot, rel_tol=1e-13)
        ratios = [wn[i, j] / w[i] for i in range(200) if w[i] != 0.0]
        mean = tot / 200
        var = sum((wn[i, j] - mean) ** 2 for i in range(200)) / 200
        assert math.isclose(ds[j], dsigma * sum(ratios) / len(ratios) + sigma * math.sqrt(var), rel_tol=1e-12)


def test_fallback_for_non_positive_or_non_finite_errors():
    w = np.full(10, 1.0)
    # all new weights zero: sigma' = 0, dsigma' = 0 -> fallback, sigma / sigma' is infinite
    s, ds, fb = xsec.reweighted_xsec(w, np.zeros((10, 1)), 2.0, 0.2)
    assert s[0] == 0.0 and fb[0] and math.isinf(ds[0])
    # a NaN weight poisons dsigma' -> fallback to dsigma times the larger ratio
    wn = np.full((10, 1), 3.0)
    wn[4, 0] = np.nan
    s, ds, fb = xsec.reweighted_xsec(w, wn, 2.0, 0.2)
    assert fb[0] and math.isnan(s[0]) and math.isnan(ds[0])
    # w' = w / 4: dsigma' = dsigma / 4 > 0, no fallback; w' = -w: dsigma' = -dsigma <= 0
    # falls back to dsigma times the larger of sigma'/sigma and sigma/sigma' (both -1 here)
    s, ds, fb = xsec.reweighted_xsec(w, np.full((10, 1), 0.25), 2.0, 0.2)
    assert not fb[0] and math.isclose(ds[0], 0.05, rel_tol=1e-15)
    s, ds, fb = xsec.reweighted_xsec(w, np.full((10, 1), -1.0), 2.0, 0.2)
    assert fb[0] and s[0] == -2.0 and math.isclose(ds[0], -0.2, rel_tol=1e-15)


def test_invariances():
    """Permuting events changes nothing; splitting a sample into two halves and
    summing their sigma' (same C) gives the whole."""
    g = np.random.default_rng(8)
    w = g.uniform(0.1, 2.0, 300)
    wn = w[:, None] * g.uniform(0.5, 1.5, (300, 4))
    s, ds, _ = xsec.reweighted_xsec(w, wn, 5.0, 0.5)
    perm = g.permutation(300)
    s2, ds2, _ = xsec.reweighted_xsec(w[perm], wn[perm], 5.0, 0.5)
    assert np.allclose(s, s2, rtol=1e-14) and np.allclose(ds, ds2, rtol=1e-13)
    c = 5.0 / w.sum()
    assert np.allclose(s, c * (wn[:150].sum(0) + wn[150:].sum(0)), rtol=1e-14)
