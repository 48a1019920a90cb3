"""Helicity-exclusive reweighting on the GPU vs the oracle, through the C ABI (needs a B300).

Each event carries a random helicity configuration, forbidden ones included (they
must give weight 0).  Tolerance: the helicity sum's (FP64 1e-12, q q~ -> t t~ mixed
1e-5), or, for a term far below its event's helicity sum, the conditioning bound
64 eps (sqrt(kappa_0) + sqrt(kappa_j)) with kappa = |M|^2 / |M_h|^2 at each point:
the amplitude components are of the size of the whole sum's, so the absolute rounding
of a small A_h is a relative error of about eps |A_typical| / |A_h| on |A_h|^2.
"""
import numpy as np
import pytest

from rexlib import ensure_built, helicity_tolerance
from oracle import reweight as oracle_rw
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QCD_ORIG = dict(mt=173.0, wt=0.0, alphas=0.118)


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(proc, n, seed):
    mom = ps.make_events(proc, n, seed)
    hel = np.random.default_rng(seed).choice(np.array([-1, 1], dtype=np.int8), size=(n, 4))
    w = np.random.default_rng(seed + 1).uniform(-0.5, 2.0, n)
    if proc == "ee_mumu":
        return mom, hel, w, ps.EE_ORIGINAL, [ps.EE_NEW, dict(ps.EE_NEW, mz=91.5), ps.EE_ORIGINAL]
    pts = ps.grid_gg_ttxg()[::3] + [QCD_ORIG, dict(mt=173.0, wt=0.0, alphas=0.124), dict(mt=168.0, wt=1.3, alphas=0.12)]
    return mom, hel, w, QCD_ORIG, pts


@pytest.mark.parametrize("proc,precision,tol", [("ee_mumu", 0, 1e-12), ("qq_ttx", 0, 1e-12), ("qq_ttx", 1, 1e-5)])
def test_parity_with_forbidden_configurations(rex, proc, precision, tol):
    n = 777   # several tiles, ragged tail
    mom, hel, w, orig, pts = case(proc, n, 61)
    p = rex.Process(proc, precision)
    p.set_params(orig)
    got = p.reweight_helicity(dev(mom), dev(hel), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight_helicity(proc, mom, hel, w, orig, pts)
    zero = ref[:, 0] == 0.0
    assert np.any(zero) and np.all(got[zero] == 0.0)
    eps = np.finfo(np.float64 if precision == 0 else np.float32).eps / 2
    bound = helicity_tolerance(proc, mom, hel, orig, pts, tol, eps)
    err = np.abs(got - ref) / np.where(ref != 0.0, np.abs(ref), 1.0)
    assert np.all(err[~zero] < bound[~zero])
    # most terms meet the helicity sum's tolerance outright
    assert np.mean(err[~zero] < tol) > 0.99
    # an unchanged point keeps the weight exactly (0 for a forbidden configuration)
    j = [i for i, pt in enumerate(pts) if pt == orig][0]
    assert np.array_equal(got[~zero, j], w[~zero])


def test_summing_configurations_gives_the_helicity_sum(rex):
    """|M|^2 at a new point as the sum over the 16 configurations of
    w_h' = |M_h'|^2 / |M_0|^2 ... checked through the weights: sum_h w'_h |M_h,0|^2 = w' |M_0|^2."""
    n = 64
    mom = ps.make_events("qq_ttx", n, 62)
    idx = np.repeat(np.arange(n), 16)
    confs = np.array(np.meshgrid(*[[-1, 1]] * 4, indexing="ij")).reshape(4, -1).T.astype(np.int8)
    hel = np.tile(confs, (n, 1))
    pts = [dict(mt=170.0, wt=0.0, alphas=0.118)]
    p = rex.Process("qq_ttx", 0)
    p.set_params(QCD_ORIG)
    wh = p.reweight_helicity(dev(mom[idx]), dev(hel), dev(np.ones(16 * n)), pts).cpu().numpy()[:, 0]
    m0h = oracle_rw.me2_helicity("qq_ttx", mom[idx], QCD_ORIG, hel)
    summed = (wh * m0h).reshape(n, 16).sum(axis=1) / oracle_rw.me2("qq_ttx", mom, QCD_ORIG)
    ws = p.reweight(dev(mom), dev(np.ones(n)), pts).cpu().numpy()[:, 0]
    assert np.max(np.abs(summed / ws - 1.0)) < 1e-12


def test_unsupported_processes_raise(rex):
    """The crossings of q q~ -> t t~ g evaluate only the helicity sum."""
    p = rex.Process("qg_ttxq", 0)
    p.set_params(QCD_ORIG)
    mom = dev(ps.make_events("qq_ttxg", 4, 1))
    with pytest.raises(rex.RexError):
        p.reweight_helicity(mom, dev(np.ones((4, 5), dtype=np.int8)), dev(np.ones(4)), [QCD_ORIG])


GG_NPART = {"gg_ttx": 4, "gg_ttxg": 5, "gg_ttxgg": 6}


def extended_reference(proc, mom, hel, w, pts):
    """The oracle's exclusive weights evaluated in extended precision (np.longdouble): a
    small helicity term carries the FP64 rounding of its diagrams' sum, relative error up
    to ~ eps sum_d |A_d| / |A_h| (7e-10 on one g g -> t t~ g term here), beyond what the
    small-term bound allows; the extended evaluation removes it from the reference."""
    ref = oracle_rw.reweight_helicity(proc, mom.astype(np.longdouble), hel, w, QCD_ORIG, pts)
    return np.asarray(ref, dtype=np.float64)


@pytest.mark.parametrize("proc,precision,tol,n", [("gg_ttx", 0, 1e-12, 300), ("gg_ttx", 1, 1e-5, 300),
                                                  ("gg_ttxg", 0, 1e-12, 97), ("gg_ttxg", 1, 1e-3, 97),
                                                  ("gg_ttxg", 2, 1e-12, 97),
                                                  ("gg_ttxgg", 0, 1e-12, 13), ("gg_ttxgg", 1, 1e-3, 13)])
def test_gg_exclusive_parity(rex, proc, precision, tol, n):
    """g g -> t t~ (+ g, + g g): each event with a random configuration of all its
    helicities.  The kernels sum real linear gluon polarisations; the exclusive tile
    combines its lanes' jamps into the helicity amplitude of the event's configuration
    (e_lambda ~ e1 -/+ i lambda e2).  Against the oracle's per-configuration terms,
    with the helicity sum's tolerance or the small-term conditioning bound."""
    npart = GG_NPART[proc]
    mom = ps.make_events(proc, n, 65)
    hel = np.random.default_rng(65).choice(np.array([-1, 1], dtype=np.int8), size=(n, npart))
    w = np.random.default_rng(66).uniform(0.5, 2.0, n)
    pts = ps.grid_gg_ttxg()[::3] + [QCD_ORIG, dict(mt=172.0, wt=1.2, alphas=0.121)]
    p = rex.Process(proc, precision)
    p.set_params(QCD_ORIG)
    got = p.reweight_helicity(dev(mom), dev(hel), dev(w), pts).cpu().numpy()
    ref = extended_reference(proc, mom, hel, w, pts)
    # g g -> t t~: four of the sixteen configurations are forbidden by angular momentum in
    # the on-shell 2 -> 2 kinematics; on FP64 momenta they are zero to ~1e-17 of the sum,
    # and the kernel reports them as 0 (the 1/0 -> 0 rule) at every point
    zero = np.zeros(n, dtype=bool)
    if proc == "gg_ttx":
        ext = mom.astype(np.longdouble)
        frac = oracle_rw.me2_helicity(proc, ext, QCD_ORIG, hel) / oracle_rw.me2(proc, ext, QCD_ORIG)
        zero = np.asarray(frac, dtype=np.float64) < 1e-12
        assert np.any(zero)
    assert np.all(got[zero] == 0.0)
    eps = {0: np.finfo(np.float64).eps / 2, 1: np.finfo(np.float32).eps / 2, 2: 2.0 ** -48}[precision]
    bound = helicity_tolerance(proc, mom, hel, QCD_ORIG, pts, tol, eps)
    err = np.abs(got[~zero] / ref[~zero] - 1.0)
    assert np.all(err < bound[~zero]), (np.max(err), np.max(err / bound[~zero]))
    assert np.mean(err < tol) > 0.9
    j = pts.index(QCD_ORIG)
    kept = ~zero & (got[:, j] != 0.0)         # FP32 returns a term below 1e-11 of its scale as 0
    assert np.mean(kept[~zero]) > 0.95
    assert np.array_equal(got[kept, j], w[kept])   # an unchanged point keeps the weight exactly


@pytest.mark.parametrize("precision", [0, 1])
def test_gg_ttxg_configurations_sum_to_the_helicity_sum(rex, precision):
    """sum_h w'_h |M_h,0|^2 = w' |M_0|^2 over the 32 configurations of each event, with
    the GPU's exclusive and helicity-summed weights."""
    n = 24
    mom = ps.make_events("gg_ttxg", n, 67)
    confs = np.array(np.meshgrid(*[[-1, 1]] * 5, indexing="ij")).reshape(5, -1).T.astype(np.int8)
    idx = np.repeat(np.arange(n), 32)
    hel = np.tile(confs, (n, 1))
    pts = [dict(mt=170.0, wt=0.0, alphas=0.118)]
    p = rex.Process("gg_ttxg", precision)
    p.set_params(QCD_ORIG)
    wh = p.reweight_helicity(dev(mom[idx]), dev(hel), dev(np.ones(32 * n)), pts).cpu().numpy()[:, 0]
    m0h = oracle_rw.me2_helicity("gg_ttxg", mom[idx], QCD_ORIG, hel)
    summed = (wh * m0h).reshape(n, 32).sum(axis=1) / oracle_rw.me2("gg_ttxg", mom, QCD_ORIG)
    ws = p.reweight(dev(mom), dev(np.ones(n)), pts).cpu().numpy()[:, 0]
    assert np.max(np.abs(summed / ws - 1.0)) < (1e-12 if precision == 0 else 1e-4)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-4)])
def test_qq_ttxg_exclusive_parity(rex, precision, tol):
    """q q~ -> t t~ g, each event with a random configuration of its 5 helicities (the
    gluon's in the helicity basis), against the oracle's per-configuration terms."""
    n = 150
    mom = ps.make_events("qq_ttxg", n, 63)
    hel = np.random.default_rng(63).choice(np.array([-1, 1], dtype=np.int8), size=(n, 5))
    w = np.random.default_rng(64).uniform(0.5, 2.0, n)
    pts = ps.grid_gg_ttxg()[::3] + [QCD_ORIG, dict(mt=172.0, wt=1.2, alphas=0.121)]
    p = rex.Process("qq_ttxg", precision)
    p.set_params(QCD_ORIG)
    got = p.reweight_helicity(dev(mom), dev(hel), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight_helicity("qq_ttxg", mom, hel, w, QCD_ORIG, pts)
    zero = ref[:, 0] == 0.0
    assert np.any(zero) and np.all(got[zero] == 0.0)
    eps = np.finfo(np.float64 if precision == 0 else np.float32).eps / 2
    bound = helicity_tolerance("qq_ttxg", mom, hel, QCD_ORIG, pts, tol, eps)
    err = np.abs(got - ref) / np.where(ref != 0.0, np.abs(ref), 1.0)
    assert np.all(err[~zero] < bound[~zero])


def test_full_size_exclusive_headline_workload(rex):
    """The helicity-exclusive leg of bench.py at its full size and in its launch: 2^20
    g g -> t t~ g events (the headline sample, seed 3) x the 16 headline points, each
    event with a random configuration (seed 203).  FP64 against the extended-precision
    oracle on sampled events; mixed against FP64 at every event, within
    max(1e-3, 64 eps32 (sqrt(kappa_0) + sqrt(kappa_j))).  kappa_0 = |M_0|^2 / |M_h,0|^2
    comes from the oracle for the events beyond 1e-3, and kappa_j = kappa_0 w'_j / w'_h,j
    from the FP64 summed and exclusive weights (the ratio of the two reweightings is
    kappa_j / kappa_0)."""
    n = 1 << 20
    mom = ps.make_events("gg_ttxg", n, 3)
    hel = np.random.default_rng(203).choice(np.array([-1, 1], dtype=np.int8), size=(n, 5))
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()
    dm, dh, dw = dev(mom), dev(hel), dev(w)
    exact = rex.Process("gg_ttxg", 0)
    exact.set_params(QCD_ORIG)
    fp64 = exact.reweight_helicity(dm, dh, dw, pts).cpu().numpy()
    mixed_p = rex.Process("gg_ttxg", 1)
    mixed_p.set_params(QCD_ORIG)
    mixed = mixed_p.reweight_helicity(dm, dh, dw, pts).cpu().numpy()

    rng = np.random.default_rng(7)
    idx = np.concatenate([rng.choice(n, 22, replace=False), [0, n - 1]])
    ref = extended_reference("gg_ttxg", mom[idx], hel[idx], w[idx], pts)
    bound = helicity_tolerance("gg_ttxg", mom[idx], hel[idx], QCD_ORIG, pts, 1e-12, np.finfo(np.float64).eps / 2)
    assert np.all(np.abs(fp64[idx] / ref - 1.0) < bound)

    both = (fp64 != 0.0) & (mixed != 0.0)
    assert np.all((fp64 == 0.0) == (mixed == 0.0)) or np.mean(both) > 0.999
    err = np.where(both, np.abs(mixed / np.where(both, fp64, 1.0) - 1.0), 0.0)
    far = np.nonzero(np.any(err > 1e-3, axis=1))[0]
    assert len(far) <= n // 100, len(far)           # small terms only (1.5e-3 of the events here)
    if len(far):
        summed = exact.reweight(dev(mom[far]), dev(w[far]), pts).cpu().numpy()
        m0 = oracle_rw.me2("gg_ttxg", mom[far], QCD_ORIG)
        m0h = oracle_rw.me2_helicity("gg_ttxg", mom[far], QCD_ORIG, hel[far])
        k0 = m0 / m0h
        nz = fp64[far] != 0.0
        kj = np.where(nz, k0[:, None] * summed / np.where(nz, fp64[far], 1.0), np.inf)
        bound = np.maximum(1e-3, 64.0 * (np.finfo(np.float32).eps / 2) * (np.sqrt(k0)[:, None] + np.sqrt(kj)))
        assert np.all(err[far] < bound), np.max(err[far] / bound)
    exact.close()
    mixed_p.close()
