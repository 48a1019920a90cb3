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


# ---- the crossings into q g, g q, q~ g, g q~ and q~ q channels ----
CROSSED = ["qg_ttxq", "gq_ttxq", "qxg_ttxqx", "gqx_ttxqx"]
GLUON_IN = {"qg_ttxq": 1, "gq_ttxq": 0, "qxg_ttxqx": 1, "gqx_ttxqx": 0}


def test_identity_crossing_is_the_direct_channel():
    p = ps.make_events("qq_ttxg", 4, 31)
    for hel in itertools.product((-1, 1), repeat=5):
        assert np.array_equal(qqg.amplitudes_crossed("qq_ttxg", p, MT, 0.7, AS, hel),
                              qqg.amplitudes(p, MT, 0.7, AS, hel))
    swapped = p[:, [1, 0, 2, 3, 4]]
    assert np.allclose(qqg.me2_crossed("qxq_ttxg", swapped, MT, 0.7, AS), qqg.me2(p, MT, 0.7, AS), rtol=1e-14)


@pytest.mark.parametrize("process", CROSSED)
def test_crossed_gauge_invariance(process):
    """eps of the incoming gluon -> its momentum: every colour component vanishes
    (a wrong momentum flow in any propagator or in the three-gluon vertex breaks it)."""
    p = ps.make_events("qq_ttxg", 6, 32)
    ig = GLUON_IN[process]
    phys, gauge = [], []
    for hel in itertools.product((-1, 1), repeat=5):
        phys.append(np.max(np.abs(qqg.colour_amplitude(p, MT, hel, process=process))))
        gauge.append(np.max(np.abs(qqg.colour_amplitude(p, MT, hel, eps_override=p[:, ig], process=process))))
    assert max(phys) > 0.0
    assert max(gauge) < 1e-13 * max(phys) * np.max(p[:, ig, 0])


@pytest.mark.parametrize("process", ["qg_ttxq", "qxg_ttxqx"])
@pytest.mark.parametrize("x", [0.35, 0.7])
def test_initial_state_collinear_limit(process, x):
    """The outgoing light parton collinear to the incoming gluon (g -> q q~ splitting,
    the parton entering the hard process carries x p_g): |M|^2 -> 8 pi alpha_s P(x) /
    (x 2 p_g.p_c) |M_Born|^2 with the textbook splitting function and the q q~ -> t t~
    trace form (no azimuthal correlation for a quark entering the hard process).  This
    fixes the 1/96 spin-colour average, the crossed wavefunctions and the flow
    momenta; the deviation falls linearly with the angle."""
    dev = []
    for theta in (1e-3, 1e-4):
        ev = pp.collinear_initial_events(4, 33, MT, 1500.0, x, theta)
        got = qqg.me2_crossed(process, ev, MT, 0.0, AS)
        t = 2.0 * pp.mdot(ev[:, 1], ev[:, 4])
        if process == "qg_ttxq":    # q(pa) q~(x pb) -> t t~
            born = pp.qq_qq_trace(ev[:, 0], x * ev[:, 1], ev[:, 2], ev[:, 3], MT, AS)
        else:                       # q(x pb) q~(pa) -> t t~
            born = pp.qq_qq_trace(x * ev[:, 1], ev[:, 0], ev[:, 2], ev[:, 3], MT, AS)
        ref = 8.0 * np.pi * AS * pp.splitting_g_to_qq(x) / (x * t) * born
        dev.append(np.max(np.abs(got / ref - 1.0)))
    assert dev[1] < 2e-4          # measured 3e-5 .. 9e-5 at theta = 1e-4
    assert dev[1] < 0.2 * dev[0]


def test_charge_conjugation_and_beam_swap():
    """q~ g -> t t~ q~ is q g -> t t~ q with t and t~ exchanged (C invariance of QCD),
    width included; g q and g q~ are q g and q~ g with the beams exchanged."""
    p = ps.make_events("qq_ttxg", 6, 34)
    qb = qqg.me2_crossed("qxg_ttxqx", p, MT, 1.3, AS)
    assert np.allclose(qb, qqg.me2_crossed("qg_ttxq", p[:, [0, 1, 3, 2, 4]], MT, 1.3, AS), rtol=1e-13)
    sw = p[:, [1, 0, 2, 3, 4]]
    assert np.allclose(qqg.me2_crossed("gq_ttxq", sw, MT, 1.3, AS), qqg.me2_crossed("qg_ttxq", p, MT, 1.3, AS),
                       rtol=1e-14)
    assert np.allclose(qqg.me2_crossed("gqx_ttxqx", sw, MT, 1.3, AS), qb, rtol=1e-14)


@pytest.mark.parametrize("process", CROSSED)
def test_crossed_lorentz_invariance_and_scaling(process):
    p = ps.make_events("qq_ttxg", 4, 35)
    m = qqg.me2_crossed(process, p, MT, 0.0, AS)
    q = pp.boost(pp.rotate(p, pp.random_rotation(5)), [-0.2, 0.35, 0.3])
    assert np.max(np.abs(qqg.me2_crossed(process, q, MT, 0.0, AS) / m - 1.0)) < 1e-12
    assert np.allclose(qqg.me2_crossed(process, p, MT, 0.0, 0.124) / m, (0.124 / AS) ** 3, rtol=1e-13)


@pytest.mark.parametrize("x", [0.4, 0.75])
def test_forward_quark_limit(x):
    """The outgoing quark collinear to the incoming one (q -> q g*, the gluon with x p_q
    entering g g -> t t~): averaged over the quark's azimuth, |M|^2 -> 8 pi alpha_s
    P_gq(x) / (x 2 p_q.p_q') |M(g g -> t t~)|^2 with the Combridge closed form.  This
    pins the t-channel gluon of the crossed light line, three-gluon vertex included;
    before the average the azimuthal spin correlation of the gluon is visible."""
    ev = pp.forward_quark_events(8, 36, MT, 1500.0, x, 1e-3)
    got = qqg.me2_crossed("qg_ttxq", ev, MT, 0.0, AS)
    t = 2.0 * pp.mdot(ev[:, 0], ev[:, 4])
    born = pp.gg_qq_combridge(np.stack([x * ev[:, 0], ev[:, 1], ev[:, 2], ev[:, 3]], axis=1), MT, AS)
    ratio = got / (8.0 * np.pi * AS * pp.splitting_q_to_g(x) / (x * t) * born)
    assert abs(np.mean(ratio) - 1.0) < 2e-6     # measured 4e-8 .. 2e-7 at theta = 1e-3
    assert np.std(ratio) > 1e-2                  # the cos(2 phi) correlation
