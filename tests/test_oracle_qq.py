"""The q q~ -> t t~ oracle against results fixed by physics (CPU only).

Pins: the Combridge closed form (massive, light and massless top), the trace
form at a changed top mass on kept momenta (checks the mass convention of the
external spinors), the colour factor (N^2 - 1)/4, chirality conservation of the
massless light-quark current, Lorentz invariance and the exact alpha_s^2 scaling
of the reweighting ratio.
"""
import itertools

import numpy as np
import pytest

import physics_pins as pp
from oracle import qq, reweight
from paper_2510_05100_b300 import phase_space as ps

MT = 173.0
AS = 0.118


def test_colour_factor_is_quadratic_casimir_sum():
    # sum_{a,b} tr(t^a t^b) tr(t^b t^a) = sum_{a,b} (delta^ab / 2)^2 = (N^2 - 1) / 4
    assert abs(qq.colour_factor() - 2.0) < 1e-14


@pytest.mark.parametrize("mt", [MT, 10.0, 0.0])
def test_qq_ttx_combridge(mt):
    p = ps.two_body_events(256, 3, mt, mt, 2 * mt + 1.0, 3000.0)
    m = qq.me2(p, mt, 0.0, AS)
    ref = pp.qq_qq_combridge(p, mt, AS)
    assert np.max(np.abs(m / ref - 1.0)) < 1e-13


def test_massless_limit_textbook():
    """m = 0: (4/9) g^4 (t^2 + u^2) / s^2 (Ellis, Stirling & Webber Table 7.1)."""
    p = ps.two_body_events(64, 4, 0.0, 0.0, 10.0, 3000.0)
    s = pp.mdot(p[:, 0] + p[:, 1], p[:, 0] + p[:, 1])
    t = pp.mdot(p[:, 0] - p[:, 2], p[:, 0] - p[:, 2])
    u = pp.mdot(p[:, 0] - p[:, 3], p[:, 0] - p[:, 3])
    g4 = (4.0 * np.pi * AS) ** 2
    ref = g4 * 4.0 / 9.0 * (t * t + u * u) / (s * s)
    assert np.max(np.abs(qq.me2(p, 0.0, 0.0, AS) / ref - 1.0)) < 1e-13


@pytest.mark.parametrize("m_new", [171.0, 175.0, 150.0])
def test_changed_mass_on_kept_momenta_trace_form(m_new):
    """At a new top mass the spinors are those of the light-cone-shifted momenta; the
    trace form needs no momentum conservation, so it pins that convention."""
    p = ps.make_events("qq_ttx", 128, 5)
    m = qq.me2(p, m_new, 0.0, AS)
    pt = pp.light_cone_mass_shift(p[:, 2], m_new)
    ptb = pp.light_cone_mass_shift(p[:, 3], m_new)
    ref = pp.qq_qq_trace(p[:, 0], p[:, 1], pt, ptb, m_new, AS)
    assert np.max(np.abs(m / ref - 1.0)) < 1e-13
    # and it differs from the on-shell value at the original mass
    assert np.min(np.abs(m / qq.me2(p, MT, 0.0, AS) - 1.0)) > 1e-6


def test_chirality_conservation_of_massless_current():
    """A vector current of massless q, q~ vanishes unless their helicities are opposite."""
    p = ps.make_events("qq_ttx", 16, 6)
    amps = qq.amplitudes(p, MT)
    big = np.max(np.abs(amps))
    for i, (l1, l2, _, _) in enumerate(itertools.product((-1, 1), repeat=4)):
        if l1 == l2:
            assert np.max(np.abs(amps[:, i])) < 1e-13 * big
        else:
            assert np.min(np.abs(amps[:, i])) > 0.0


def test_lorentz_invariance():
    p = ps.make_events("qq_ttx", 8, 7)
    m = qq.me2(p, MT, 0.0, AS)
    q = pp.boost(pp.rotate(p, pp.random_rotation(5)), [0.2, 0.4, -0.5])
    assert np.max(np.abs(qq.me2(q, MT, 0.0, AS) / m - 1.0)) < 1e-12


def test_alphas_scaling_and_width_independence():
    p = ps.make_events("qq_ttx", 8, 8)
    out = reweight.reweight("qq_ttx", p, np.ones(8), dict(mt=MT, wt=0.0, alphas=AS),
                            [dict(mt=MT, wt=0.0, alphas=0.124), dict(mt=MT, wt=1.5, alphas=AS)])
    assert np.allclose(out[:, 0], (0.124 / AS) ** 2, rtol=1e-13)
    assert np.array_equal(out[:, 1], np.ones(8))


def test_wrong_particle_count_rejected():
    with pytest.raises(ValueError):
        qq.me2(np.zeros((2, 5, 4)), MT, 0.0, AS)
