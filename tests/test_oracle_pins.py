"""The oracle against results fixed by physics and mathematics (CPU only).

Each pin is chosen so that a plausible mistake in the oracle fails it:
a dropped diagram, a wrong vertex sign or colour factor, a transposed
operand in the colour contraction, a wrong averaging factor, or a broken
spinor/polarisation construction.
"""
import itertools
import math

import numpy as np
import pytest

import physics_pins as pp
from oracle import colour, ee, qcd, reweight
from oracle.lorentz import GAMMA, bar, mdot, polarisation, slash, spinor_u, spinor_v
from paper_2510_05100_b300 import phase_space as ps

MT = 173.0
AS = 0.118


# ---------------------------------------------------------------- building blocks
def test_dirac_algebra_clifford():
    """{gamma^mu, gamma^nu} = 2 g^{mu nu}."""
    g = np.diag([1.0, -1.0, -1.0, -1.0])
    for mu in range(4):
        for nu in range(4):
            anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(anti, 2.0 * g[mu, nu] * np.eye(4), atol=1e-15)


def test_spinor_completeness_and_dirac_equation():
    """sum_s u ubar = p-slash + m, sum_s v vbar = p-slash - m, (p-slash - m) u = 0."""
    p = ps.two_body_events(5, 7, MT, MT, 400.0, 2000.0)[:, 2]
    ss_u = sum(np.einsum("ni,nj->nij", spinor_u(p, MT, l), bar(spinor_u(p, MT, l))) for l in (-1, 1))
    ss_v = sum(np.einsum("ni,nj->nij", spinor_v(p, MT, l), bar(spinor_v(p, MT, l))) for l in (-1, 1))
    ps_ = slash(p)
    assert np.allclose(ss_u, ps_ + MT * np.eye(4), rtol=0, atol=1e-10)
    assert np.allclose(ss_v, ps_ - MT * np.eye(4), rtol=0, atol=1e-10)
    for l in (-1, 1):
        r = np.einsum("nij,nj->ni", ps_ - MT * np.eye(4), spinor_u(p, MT, l))
        assert np.max(np.abs(r)) < 1e-9


def test_spinor_off_shell_mass_convention():
    """With mass m != sqrt(p^2) the spinors are those of p~ (same direction, same E+|p|)."""
    p = ps.two_body_events(4, 8, MT, MT, 400.0, 2000.0)[:, 2]
    m = 171.0
    pabs = np.linalg.norm(p[:, 1:], axis=1)
    wp2 = p[:, 0] + pabs
    wm2 = m * m / wp2
    pt = np.empty_like(p)
    pt[:, 0] = 0.5 * (wp2 + wm2)
    pt[:, 1:] = p[:, 1:] / pabs[:, None] * (0.5 * (wp2 - wm2))[:, None]
    assert np.allclose(mdot(pt, pt), m * m, rtol=1e-12)
    ss = sum(np.einsum("ni,nj->nij", spinor_u(p, m, l), bar(spinor_u(p, m, l))) for l in (-1, 1))
    assert np.allclose(ss, slash(pt) + m * np.eye(4), atol=1e-10)


def test_polarisation_vectors():
    k = ps.two_body_events(6, 9, 0.0, 0.0, 100.0, 1000.0)[:, 2]
    k = np.concatenate([k, np.array([[5.0, 0, 0, 5.0], [5.0, 0, 0, -5.0]])])
    for lam in (-1, 1):
        e = polarisation(k, lam)
        assert np.max(np.abs(mdot(e, k))) < 1e-12
        assert np.allclose(mdot(e, e.conj()), -1.0)
    # completeness in the transverse plane: sum_l eps eps^* = -g + (k n + n k)/(k.n) for n=(1,0,0,0)-k-hat..
    e_p, e_m = polarisation(k, 1), polarisation(k, -1)
    ss = np.einsum("ni,nj->nij", e_p, e_p.conj()) + np.einsum("ni,nj->nij", e_m, e_m.conj())
    khat = k[:, 1:] / np.linalg.norm(k[:, 1:], axis=1)[:, None]
    proj = np.eye(3)[None] - np.einsum("ni,nj->nij", khat, khat)
    assert np.allclose(ss[:, 1:, 1:], proj, atol=1e-12)


def test_su3_generators():
    t, f = colour.T, colour.F
    assert np.allclose(np.einsum("aij,bji->ab", t, t), 0.5 * np.eye(8))
    comm = np.einsum("aij,bjk->abik", t, t) - np.einsum("bij,ajk->abik", t, t)
    assert np.allclose(comm, 1j * np.einsum("abc,cik->abik", f, t))
    assert np.allclose(np.einsum("aij,ajk->ik", t, t), 4.0 / 3.0 * np.eye(3))   # C_F
    assert np.allclose(np.einsum("acd,bcd->ab", f, f), 3.0 * np.eye(8))          # C_A


# ---------------------------------------------------------------- diagram counts
@pytest.mark.parametrize("ngl,count", [(2, 3), (3, 16), (4, 123)])
def test_diagram_counts(ngl, count):
    assert len(qcd.diagrams(ngl)) == count


def test_colour_matrix_hermitian_psd_and_trace():
    for ngl in (2, 3):
        g = qcd.colour_matrix(ngl)
        assert np.allclose(g, g.conj().T)
        w = np.linalg.eigvalsh(g)
        assert w.min() > -1e-10 * w.max()


# ---------------------------------------------------------------- closed forms
def test_ee_mumu_qed_limit():
    """Z decoupled (mZ -> huge): e^4 (1 + cos^2 theta)."""
    p = ps.ee_mumu_events(64, 1)
    alpha = 1.0 / 132.507
    m = ee.me2(p, mz=1e9, wz=0.0, sw2=0.2312, alpha=alpha)
    ref = pp.qed_limit_closed_form(p, alpha)
    assert np.max(np.abs(m / ref - 1.0)) < 1e-9     # Z residue ~ s/mZ^2 = 2.5e-13


@pytest.mark.parametrize("point", [ps.EE_ORIGINAL, ps.EE_NEW])
def test_ee_mumu_photon_z_closed_form(point):
    p = ps.ee_mumu_events(256, 1)
    m = ee.me2(p, point["mz"], point["wz"], point["sw2"], point["alpha"])
    ref = pp.ee_mumu_closed_form(p, point["mz"], point["wz"], point["sw2"], point["alpha"])
    assert np.max(np.abs(m / ref - 1.0)) < 1e-13


def test_ee_mumu_resonance_peak():
    """At sqrt(s) = mZ the Z term dominates the photon term by ~ (mZ/GZ)^2 g^4 factors."""
    p = ps.ee_mumu_events(16, 3, sqrt_s=91.1876)
    pt = ps.EE_ORIGINAL
    m = ee.me2(p, pt["mz"], pt["wz"], pt["sw2"], pt["alpha"])
    ref = pp.ee_mumu_closed_form(p, pt["mz"], pt["wz"], pt["sw2"], pt["alpha"])
    assert np.max(np.abs(m / ref - 1.0)) < 1e-13


@pytest.mark.parametrize("mt", [MT, 10.0, 0.0])
def test_gg_ttx_combridge(mt):
    p = ps.two_body_events(256, 2, mt, mt, 2 * mt + 1.0, 3000.0)
    m = qcd.me2(p, mt, 0.0, AS)
    ref = pp.gg_qq_combridge(p, mt, AS)
    # the closed form cancels rho - rho^2/(4 t1 t2) against t1^2 + t2^2 near the
    # beam axis for light quarks (t1 t2 ~ m^2/s): allow its own rounding there
    assert np.max(np.abs(m / ref - 1.0)) < (1e-13 if mt > 100 else 5e-12)


def test_gg_qqg_parke_taylor_massless():
    p = ps.gg_tt_jets_events(64, 21, 1, 50.0, 4000.0, mt=0.0)
    m = qcd.me2(p, 0.0, 0.0, AS)
    ref = pp.parke_taylor_me2(pp.rotate(p, pp.random_rotation(5)), AS)
    rel = np.abs(m / ref - 1.0)
    assert np.max(rel) < 1e-11


@pytest.mark.slow
def test_gg_qqgg_per_helicity_mhv():
    """Every MHV, anti-MHV and vanishing helicity configuration of g g -> q q~ g g."""
    p = ps.gg_tt_jets_events(3, 22, 2, 50.0, 5000.0, mt=0.0)
    pr = pp.rotate(p, pp.random_rotation(6))
    # scale: the helicity-summed, colour-summed value of each event
    scale = qcd.me2(p, 0.0, 0.0, AS) * 4.0 * 64.0 * 2.0
    checked = 0
    for hg in itertools.product((-1, 1), repeat=4):
        for lt in (-1, 1):
            for ltb in (-1, 1):
                ref = pp.parke_taylor_helicity(pr, AS, lt, ltb, (-hg[0], -hg[1], hg[2], hg[3]))
                if ref is None:
                    continue
                o = qcd.me2_helicity(p, 0.0, 0.0, AS, hg, lt, ltb)
                assert np.max(np.abs(o - ref) / scale) < 1e-12, (hg, lt, ltb)
                checked += 1
    assert checked == 52


# ---------------------------------------------------------------- invariances
def _gauge_residual(p, which, hel, lt, ltb, mt):
    """max over colour configurations |M(eps->k)| / sum_terms |K_t||L_t|."""
    npart = p.shape[1]
    ngl = npart - 2
    terms = qcd.diagram_terms(ngl)
    kmat = np.stack([qcd.term_colour(t, ngl).reshape(-1) for t in terms])   # [T, C]
    g = math.sqrt(4 * math.pi * AS)
    rows = [0, 1] + list(range(4, npart))
    p_out = [-p[:, 0], -p[:, 1]] + [p[:, r] for r in range(4, npart)]
    eps = []
    for k, (row, lam) in enumerate(zip(rows, hel)):
        e = polarisation(p[:, row], lam)
        e = e if k < 2 else e.conj()
        if k == which:
            e = p[:, row].astype(complex)
        eps.append(e)
    kin = qcd._Kinematics(p_out, eps, g)
    ub = bar(spinor_u(p[:, 2], mt, lt))
    v = spinor_v(p[:, 3], mt, ltb)
    lmat = np.stack([qcd._line_amplitude(t, kin, ub, v, p[:, 2], mt, 0.0) for t in terms], 1)
    full = lmat @ kmat
    scale = np.abs(lmat) @ np.abs(kmat)
    return np.max(np.abs(full) / np.max(scale, axis=1, keepdims=True))


@pytest.mark.parametrize("proc", ["gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_gauge_invariance(proc):
    """eps -> k for any one gluon makes every colour component of M vanish."""
    p = ps.make_events(proc, 3, 31)
    ngl = p.shape[1] - 2
    rng = np.random.default_rng(1)
    for which in range(ngl):
        hel = tuple(int(h) for h in rng.choice([-1, 1], ngl))
        r = _gauge_residual(p, which, hel, int(rng.choice([-1, 1])), int(rng.choice([-1, 1])), MT)
        assert r < 1e-13, (which, r)


@pytest.mark.parametrize("proc", ["gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_lorentz_invariance(proc):
    p = ps.make_events(proc, 4, 41)
    m = qcd.me2(p, MT, 0.0, AS)
    q = pp.boost(pp.rotate(p, pp.random_rotation(3)), [0.3, -0.2, 0.6])
    mq = qcd.me2(q, MT, 0.0, AS)
    assert np.max(np.abs(mq / m - 1.0)) < 1e-12


@pytest.mark.parametrize("proc", ["gg_ttxg", "gg_ttxgg"])
def test_bose_symmetry(proc):
    p = ps.make_events(proc, 4, 51)
    m = qcd.me2(p, MT, 0.0, AS)
    sw = p.copy()
    sw[:, [0, 1]] = p[:, [1, 0]]
    # swapped legs change the rounding order of strongly cancelling diagram sums
    assert np.max(np.abs(qcd.me2(sw, MT, 0.0, AS) / m - 1.0)) < 1e-12
    if p.shape[1] == 6:
        sw = p.copy()
        sw[:, [4, 5]] = p[:, [5, 4]]
        assert np.max(np.abs(qcd.me2(sw, MT, 0.0, AS) / m - 1.0)) < 1e-12


def test_rotation_invariance_off_shell_mass():
    """With m != sqrt(p_t^2) the result is still rotation invariant (p~ is built covariantly
    under rotations) but not boost invariant."""
    p = ps.make_events("gg_ttxg", 4, 61)
    m = qcd.me2(p, 171.0, 0.0, AS)
    q = pp.rotate(p, pp.random_rotation(9))
    assert np.max(np.abs(qcd.me2(q, 171.0, 0.0, AS) / m - 1.0)) < 1e-12


# ---------------------------------------------------------------- coupling scaling and the ratio
@pytest.mark.parametrize("proc,n", [("gg_ttx", 2), ("gg_ttxg", 3)])
def test_alphas_scaling_exact(proc, n):
    """Tree amplitudes with n+... external gluons scale as g_s^(n_gluons): ratio = (as'/as)^n."""
    p = ps.make_events(proc, 8, 71)
    w = np.ones(8)
    out = reweight.reweight(proc, p, w, dict(mt=MT, wt=0.0, alphas=AS),
                            [dict(mt=MT, wt=0.0, alphas=0.124)])
    assert np.allclose(out[:, 0], (0.124 / AS) ** n, rtol=1e-13)


def test_unit_ratio_and_zero_convention():
    p = ps.make_events("gg_ttx", 6, 81)
    w = np.linspace(0.5, 2.0, 6)
    orig = dict(mt=MT, wt=0.0, alphas=AS)
    out = reweight.reweight("gg_ttx", p, w, orig, [orig])
    assert np.array_equal(out[:, 0], w)
    # 1/0 -> 0: an event with |M|^2 = 0 gets weight 0
    r = reweight.ratio_epilogue(np.array([1.0, 2.0]), np.array([0.0, 2.0]), np.array([[3.0, 4.0]]))
    assert r[0, 0] == 0.0 and r[1, 0] == 4.0


def test_mass_change_moves_weights():
    p = ps.make_events("gg_ttx", 4, 91)
    out = reweight.reweight("gg_ttx", p, np.ones(4), dict(mt=MT, wt=0.0, alphas=AS),
                            [dict(mt=171.0, wt=0.0, alphas=AS), dict(mt=175.0, wt=0.0, alphas=AS)])
    assert np.all(np.isfinite(out)) and np.all(out > 0)
    assert not np.allclose(out[:, 0], 1.0)


def test_top_width_enters_propagators():
    """Gamma_t only shifts propagator poles: a small width changes |M|^2 slightly, never by much."""
    p = ps.make_events("gg_ttxg", 4, 95)
    m0 = qcd.me2(p, MT, 0.0, AS)
    m1 = qcd.me2(p, MT, 1.5, AS)
    rel = np.abs(m1 / m0 - 1.0)
    assert np.all(rel > 0) and np.all(rel < 0.1)


def test_massless_lepton_currents_vanish_for_equal_helicities():
    """Helicity filtering of e+e- -> mu+mu- rests on this: a chiral current of a massless
    fermion-antifermion pair vanishes unless their helicities are opposite, so only 4 of
    the 16 configurations contribute."""
    from oracle.lorentz import PL, PR
    p = ps.make_events("ee_mumu", 16, 91)
    scale = np.max(np.abs(p))
    for proj in (PL, PR):
        mats = np.einsum("mij,jk->mik", GAMMA, proj)
        for l1 in (-1, 1):
            for l2 in (-1, 1):
                je = np.einsum("ni,mij,nj->nm", bar(spinor_v(p[:, 0], 0.0, l1)), mats, spinor_u(p[:, 1], 0.0, l2))
                jm = np.einsum("ni,mij,nj->nm", bar(spinor_u(p[:, 3], 0.0, l2)), mats, spinor_v(p[:, 2], 0.0, l1))
                if l1 == l2:
                    assert np.max(np.abs(je)) < 1e-13 * scale and np.max(np.abs(jm)) < 1e-13 * scale
    # and the surviving configurations carry all of |M|^2: both chiralities of opposite pairs
    n_nonzero = 0
    for l1, l2 in itertools.product((-1, 1), repeat=2):
        j = np.einsum("ni,mij,nj->nm", bar(spinor_v(p[:, 0], 0.0, l1)), GAMMA, spinor_u(p[:, 1], 0.0, l2))
        n_nonzero += int(np.max(np.abs(j)) > 1e-6 * scale)
    assert n_nonzero == 2


# ---------------------------------------------------------------- the condition estimate kappa
def test_condition_gg_ttx_brute_force():
    """kappa = sum_h sum_st |Re(conj(A_s) G_st A_t)| / |M|^2 against an independent
    diagram-by-diagram evaluation (Dirac representation, own helicity spinors, circular
    polarisations and colour tensors); that evaluation itself reproduces the Combridge
    |M|^2, so its three diagrams carry the right relative signs and colour factors.  A
    dropped sign of the colour matrix, a wrong index set of the pair sum or a sum taken
    after the helicity sum would each move kappa away from it."""
    p = ps.make_events("gg_ttx", 12, 5)
    kappa = qcd.condition(p, MT, 0.0, AS)
    for e in range(len(p)):
        x = pp.gg_qq_pair_terms(p[e], MT, AS)
        total = x.sum()
        assert abs(total / 256.0 / pp.gg_qq_combridge(p[e:e + 1], MT, AS)[0] - 1.0) < 1e-13
        assert abs(kappa[e] / (np.abs(x).sum() / abs(total)) - 1.0) < 1e-12, e


@pytest.mark.parametrize("proc", ["gg_ttxg", "gg_ttxgg"])
def test_condition_bounds_and_invariances(proc):
    """kappa >= 1 (triangle inequality) and > 1 whenever diagrams interfere; unchanged by
    alpha_s (every term carries the same power of g_s) and by a rotation of the event (a
    rotation multiplies each helicity amplitude by a phase common to all diagrams, so
    every term Re(conj(A_s) G_st A_t) is kept; a boost is not such a symmetry of a single
    diagram, whose polarisations change gauge)."""
    p = ps.make_events(proc, 3, 81)
    k = qcd.condition(p, MT, 0.0, AS)
    assert np.all(k > 1.0 + 1e-6)
    assert np.max(np.abs(qcd.condition(p, MT, 0.0, 0.124) / k - 1.0)) < 1e-12
    q = pp.rotate(p, pp.random_rotation(17))
    assert np.max(np.abs(qcd.condition(q, MT, 0.0, AS) / k - 1.0)) < 1e-9


def test_condition_predicts_fp64_rounding():
    """kappa as a rounding bound: the FP64 oracle's own relative error, measured against the
    same diagrams evaluated in extended precision (np.longdouble, eps 1.1e-19), stays below
    64 eps kappa on every event, and is of the size kappa predicts.  Events 75 and 146 of
    the seeded 512-event g g -> t t~ g g sample are its worst conditioned (kappa ~ 6e4 and
    7e3); the six others are typical (kappa < 100)."""
    mom = ps.make_events("gg_ttxgg", 512, 3)
    idx = np.array([75, 146, 0, 100, 200, 300, 400, 511])
    eps = np.finfo(np.float64).eps
    for mt in (MT, 170.0):
        m64 = qcd.me2(mom[idx], mt, 0.0, AS)
        mld = qcd.me2(mom[idx].astype(np.longdouble), mt, 0.0, AS)
        kappa = qcd.condition(mom[idx], mt, 0.0, AS)
        err = np.abs(m64 / mld - 1.0).astype(np.float64)
        assert np.all(err <= 64.0 * eps * kappa), (mt, err, kappa)
        assert kappa[0] > 1e4 and kappa[1] > 1e3 and np.all(kappa[2:] < 100.0)
        assert err[0] > 1e-2 * eps * kappa[0]          # the worst event's error is kappa's size
        assert np.all(err[2:] < 1e-14)                 # typical events: a few eps
