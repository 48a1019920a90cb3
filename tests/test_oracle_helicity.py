"""Helicity-exclusive |M_h|^2 of the oracle against closed forms (CPU only).

e+e- -> mu+mu-: each of the 16 configurations against the textbook chiral form;
q q~ -> t t~: each configuration against the centre-of-mass helicity amplitudes
(opposite top helicities (1 +- cos)^2, equal ones (1 - beta^2) sin^2) at the top
mass and near the massless limit; both: the terms add up to the helicity sum, and
parity maps a configuration to its mirror.
"""
import itertools

import numpy as np
import pytest

import physics_pins as pp
from oracle import ee, qq, reweight
from paper_2510_05100_b300 import phase_space as ps

CONFIGS = np.array(list(itertools.product((-1, 1), repeat=4)))


def every_config(n):
    """Each event repeated once per configuration: momenta index and helicities."""
    return np.repeat(np.arange(n), 16), np.tile(CONFIGS, (n, 1))


def test_ee_per_configuration_closed_form():
    p = ps.make_events("ee_mumu", 32, 101)
    idx, hel = every_config(32)
    pt = ps.EE_ORIGINAL
    got = ee.me2_helicity(p[idx], pt["mz"], pt["wz"], pt["sw2"], pt["alpha"], hel)
    ref = pp.ee_mumu_helicity_closed_form(p[idx], hel, pt["mz"], pt["wz"], pt["sw2"], pt["alpha"])
    scale = np.max(ref)
    assert np.max(np.abs(got - ref)) < 1e-13 * scale
    nz = ref > 0
    assert np.sum(nz) == 4 * 32 and np.max(np.abs(got[nz] / ref[nz] - 1.0)) < 1e-12


@pytest.mark.parametrize("mt", [173.0, 1.0])
def test_qq_per_configuration_cm_helicity_amplitudes(mt):
    p = ps.two_body_events(32, 102, mt, mt, 2 * mt + 1.0, 3000.0)
    idx, hel = every_config(32)
    got = qq.me2_helicity(p[idx], mt, 0.0, 0.118, hel)
    ref = pp.qq_qq_helicity_cm(p[idx], hel, mt, 0.118)
    scale = np.max(ref)
    assert np.max(np.abs(got - ref)) < 1e-12 * scale
    # the 16 terms add up to the Combridge form
    tot = got.reshape(32, 16).sum(axis=1)
    assert np.max(np.abs(tot / pp.qq_qq_combridge(p, mt, 0.118) - 1.0)) < 1e-13


@pytest.mark.parametrize("proc", ["ee_mumu", "qq_ttx"])
def test_terms_sum_to_the_helicity_sum_and_parity(proc):
    p = ps.make_events(proc, 24, 103)
    orig = ps.EE_ORIGINAL if proc == "ee_mumu" else dict(mt=171.0, wt=0.0, alphas=0.118)
    idx, hel = every_config(24)
    terms = reweight.me2_helicity(proc, p[idx], orig, hel).reshape(24, 16)
    assert np.max(np.abs(terms.sum(axis=1) / reweight.me2(proc, p, orig) - 1.0)) < 1e-13
    if proc == "qq_ttx":
        # QCD conserves parity: flipping every helicity leaves each term unchanged
        flipped = reweight.me2_helicity(proc, p[idx], orig, -hel).reshape(24, 16)
        assert np.max(np.abs(flipped - terms)) < 1e-12 * np.max(terms)


def test_exclusive_ratio_and_zero_rule():
    p = ps.make_events("qq_ttx", 40, 104)
    hel = np.random.default_rng(5).choice([-1, 1], size=(40, 4))
    w = np.random.default_rng(6).uniform(0.5, 2.0, 40)
    orig = dict(mt=173.0, wt=0.0, alphas=0.118)
    out = reweight.reweight_helicity("qq_ttx", p, hel, w, orig, [orig, dict(mt=173.0, wt=0.0, alphas=0.124)])
    zero = hel[:, 0] == hel[:, 1]            # equal q, q~ helicities: |M_h|^2 = 0 -> weight 0
    assert np.all(out[zero] == 0.0)
    assert np.allclose(out[~zero, 0], w[~zero], rtol=1e-14)
    assert np.allclose(out[~zero, 1], w[~zero] * (0.124 / 0.118) ** 2, rtol=1e-13)


@pytest.mark.parametrize("proc", ["ee_mumu", "qq_ttx"])
def test_vanishing_configurations_are_exact_zeros(proc):
    """The configurations chirality forbids are exact zeros after the residue cut, and
    no physical configuration comes anywhere near the cut."""
    p = ps.make_events(proc, 64, 105)
    orig = ps.EE_ORIGINAL if proc == "ee_mumu" else dict(mt=173.0, wt=0.0, alphas=0.118)
    idx, hel = every_config(64)
    terms = reweight.me2_helicity(proc, p[idx], orig, hel).reshape(64, 16)
    forbidden = (CONFIGS[:, 0] == CONFIGS[:, 1]) | ((CONFIGS[:, 2] == CONFIGS[:, 3]) if proc == "ee_mumu" else False)
    assert np.all(terms[:, forbidden] == 0.0)
    rel = terms[:, ~forbidden] / reweight.me2(proc, p, orig)[:, None]
    assert np.min(rel) > 1e6 * reweight.ZERO_TERM


def test_qq_ttxg_terms_sum_to_the_helicity_sum_and_zeros():
    """q q~ -> t t~ g: the 32 configuration terms add up to the helicity sum, the
    configurations with equal light-quark helicities are exact zeros after the residue
    cut, and QCD's parity maps each term to its mirror."""
    from oracle import qqg
    p = ps.make_events("qq_ttxg", 6, 106)
    orig = dict(mt=173.0, wt=0.0, alphas=0.118)
    confs = np.array(list(itertools.product((-1, 1), repeat=5)))
    idx = np.repeat(np.arange(6), 32)
    hel = np.tile(confs, (6, 1))
    terms = reweight.me2_helicity("qq_ttxg", p[idx], orig, hel).reshape(6, 32)
    assert np.max(np.abs(terms.sum(axis=1) / qqg.me2(p, 173.0, 0.0, 0.118) - 1.0)) < 1e-13
    forbidden = confs[:, 0] == confs[:, 1]
    assert np.all(terms[:, forbidden] == 0.0) and np.all(terms[:, ~forbidden] > 0.0)
    mirror = reweight.me2_helicity("qq_ttxg", p[idx], orig, -hel).reshape(6, 32)
    assert np.max(np.abs(mirror - terms)) < 1e-12 * np.max(terms)


@pytest.mark.parametrize("proc,npart,n", [("gg_ttx", 4, 6), ("gg_ttxg", 5, 4), ("gg_ttxgg", 6, 2)])
def test_gg_terms_sum_to_the_helicity_sum_and_parity(proc, npart, n):
    """The g g processes' per-event helicity terms: over every configuration they add up to
    the helicity sum, and parity (every 3-momentum reversed, every helicity flipped) maps
    each term onto its mirror; at a shifted top mass (the spinors' light-cone convention)."""
    p = ps.make_events(proc, n, 105)
    pt = dict(mt=171.0, wt=0.0, alphas=0.118)
    cfg = np.array(list(itertools.product((-1, 1), repeat=npart)), dtype=np.int8)
    idx, hel = np.repeat(np.arange(n), len(cfg)), np.tile(cfg, (n, 1))
    terms = reweight.me2_helicity(proc, p[idx], pt, hel).reshape(n, -1)
    assert np.max(np.abs(terms.sum(axis=1) / reweight.me2(proc, p, pt) - 1.0)) < 1e-13
    mirror = p.copy()
    mirror[..., 1:] *= -1.0
    flipped = reweight.me2_helicity(proc, mirror[idx], pt, -hel).reshape(n, -1)
    assert np.max(np.abs(flipped - terms)) < 1e-13 * np.max(terms)
