"""Seeded input generators: conservation, on-shell masses, determinism (CPU)."""
import numpy as np
import pytest

from paper_2510_05100_b300 import phase_space as ps


def _mdot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


@pytest.mark.parametrize("proc,masses", [
    ("ee_mumu", [0, 0, 0, 0]),
    ("gg_ttx", [0, 0, 173, 173]),
    ("qq_ttx", [0, 0, 173, 173]),
    ("qq_ttxg", [0, 0, 173, 173, 0]),
    ("gg_ttxg", [0, 0, 173, 173, 0]),
    ("gg_ttxgg", [0, 0, 173, 173, 0, 0]),
])
def test_conservation_and_masses(proc, masses):
    p = ps.make_events(proc, 2000, 5)
    assert p.shape == (2000, len(masses), 4)
    tot = p[:, 0] + p[:, 1] - p[:, 2:].sum(axis=1)
    assert np.max(np.abs(tot)) < 1e-9 * np.max(p[:, :, 0])
    for i, m in enumerate(masses):
        m2 = _mdot(p[:, i], p[:, i])
        assert np.max(np.abs(m2 - m * m)) < 1e-8 * np.max(p[:, i, 0] ** 2)
    assert np.all(p[:, :, 0] > 0)


def test_deterministic_by_seed():
    a = ps.make_events("gg_ttxg", 100, 3)
    b = ps.make_events("gg_ttxg", 100, 3)
    c = ps.make_events("gg_ttxg", 100, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_sqrt_s_ranges():
    for proc, lo, hi in (("gg_ttx", 347.0, 3000.0), ("gg_ttxg", 400.0, 4000.0), ("gg_ttxgg", 500.0, 5000.0)):
        p = ps.make_events(proc, 4000, 9)
        rs = p[:, 0, 0] + p[:, 1, 0]
        assert rs.min() >= lo * (1 - 1e-12) and rs.max() <= hi * (1 + 1e-12)


def test_grids():
    assert len(ps.grid_gg_ttx()) == 8 and len(ps.grid_gg_ttxg()) == 16 and len(ps.grid_64()) == 64
    g = ps.grid_gg_ttxg()
    assert g[0] == dict(mt=171.0, wt=0.0, alphas=0.112) and g[-1]["mt"] == 175.0
    assert len({pt["mt"] for pt in ps.grid_64()}) == 8
