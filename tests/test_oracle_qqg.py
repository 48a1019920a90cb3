"""The q q~ -> t t~ g oracle against what physics fixes (CPU only).

Gauge invariance of every colour component (a dropped diagram, a wrong sign,
propagator or colour factor of one diagram breaks it), the soft-gluon limit
against the pinned q q~ -> t t~ oracle times eikonal factors with colour
correlators computed here (fixes the overall normalisation), Lorentz invariance
and the exact alpha_s^3 scaling.
"""
import itertools

import numpy as np
import pytest

import physics_pins as pp
from oracle import qq, qqg
from paper_2510_05100_b300 import phase_space as ps

MT = 173.0
AS = 0.118


@pytest.mark.parametrize("hel", [(1, -1, 1, -1, 1), (-1, 1, 1, 1, -1), (1, -1, -1, 1, -1), (-1, 1, -1, -1, 1)])
def test_gauge_invariance_every_colour_component(hel):
    p = ps.make_events("qq_ttxg", 8, 21)
    phys = qqg.colour_amplitude(p, MT, hel)
    gauge = qqg.colour_amplitude(p, MT, hel, eps_override=p[:, 4])
    scale = np.max(np.abs(phys)) * np.max(p[:, 4, 0])
    assert np.max(np.abs(gauge)) < 1e-13 * scale
    assert np.max(np.abs(phys)) > 0.0


def test_colour_conservation_of_the_correlators():
    corr, resid = pp.qq_qq_colour_correlators()
    assert resid < 1e-14
    assert np.allclose(np.diag(corr), 4.0 / 3.0)          # T_i^2 = C_F
    assert np.allclose(corr.sum(axis=1), 0.0, atol=1e-14)  # sum_j T_i . T_j = 0


@pytest.mark.parametrize("omega_frac", [1e-5])
def test_soft_gluon_limit(omega_frac):
    ev, born = pp.soft_qq_ttg_events(6, 22, MT, 900.0, omega_frac)
    corr, _ = pp.qq_qq_colour_correlators()
    got = qqg.me2(ev, MT, 0.0, AS)
    ref = pp.soft_eikonal(ev[:, :4], ev[:, 4], corr, AS) * qq.me2(born, MT, 0.0, AS)
    assert np.max(np.abs(got / ref - 1.0)) < 1e-4   # measured 1.4e-6 at omega = 1e-5 sqrt(s)


def test_lorentz_invariance():
    p = ps.make_events("qq_ttxg", 4, 23)
    m = qqg.me2(p, MT, 0.0, AS)
    q = pp.boost(pp.rotate(p, pp.random_rotation(4)), [0.25, -0.3, 0.4])
    assert np.max(np.abs(qqg.me2(q, MT, 0.0, AS) / m - 1.0)) < 1e-12


def test_alphas_cubed_scaling_and_width():
    p = ps.make_events("qq_ttxg", 4, 24)
    m = qqg.me2(p, MT, 0.0, AS)
    assert np.allclose(qqg.me2(p, MT, 0.0, 0.124) / m, (0.124 / AS) ** 3, rtol=1e-13)
    assert np.min(np.abs(qqg.me2(p, MT, 1.5, AS) / m - 1.0)) > 0.0   # the width enters the top propagators


def test_wrong_particle_count_rejected():
    with pytest.raises(ValueError):
        qqg.me2(np.zeros((2, 4, 4)), MT, 0.0, AS)
