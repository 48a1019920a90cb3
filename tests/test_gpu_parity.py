"""CUDA path vs the FP64 oracle, through the C ABI (needs a B300).

Tolerances:
* FP64 mode: 1e-12 relative per event on |M|^2 and on every new weight.
* unchanged parameter point: new weight == input weight exactly (same mass
  slot, same coupling factor, w * (x / x) = w).
* mixed mode (FP32 amplitudes): the bound measured per process, see MIXED_TOL.
"""
import math

import numpy as np
import pytest

from rexlib import ensure_built
from oracle import reweight as oracle_rw
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
# Stated bound on the relative error of a new weight in mixed precision (FP32
# currents and spinor chains, FP64 invariants, colour form in FP32 or on tensor
# cores as FP16 hi+lo, FP64 helicity sum and ratio).  The largest errors seen
# against the FP64 kernel over 2^20 (gg_ttx, gg_ttxg) and 2^16 (gg_ttxgg) events
# are 7.4e-7, 1.4e-4 and 6.8e-5; the bounds keep a factor of 7 or more above them.
MIXED_TOL = {"gg_ttx": 1e-5, "gg_ttxg": 1e-3, "gg_ttxgg": 1e-3}

ORIG_QCD = dict(mt=173.0, wt=0.0, alphas=0.118)
SIZES = {"ee_mumu": 300, "gg_ttx": 101, "gg_ttxg": 53, "gg_ttxgg": 19}
NGLUON = {"gg_ttx": 2, "gg_ttxg": 3, "gg_ttxgg": 4}


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def original(proc):
    return ps.EE_ORIGINAL if proc == "ee_mumu" else ORIG_QCD


def new_points(proc):
    if proc == "ee_mumu":
        return [ps.EE_NEW]
    if proc == "gg_ttx":
        return ps.grid_gg_ttx()
    if proc == "gg_ttxg":
        return ps.grid_gg_ttxg()
    return [dict(mt=171.0, wt=0.0, alphas=0.118), dict(mt=175.0, wt=0.0, alphas=0.124),
            dict(mt=173.0, wt=0.0, alphas=0.112)]


def make(proc, rex, precision=0):
    p = rex.Process(proc, precision)
    p.set_params(original(proc))
    return p


def rel(a, b):
    return np.abs(a / b - 1.0)


@pytest.mark.parametrize("proc", ["ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_me2_parity_fp64(rex, proc):
    n = SIZES[proc]
    mom = ps.make_events(proc, n, 101)
    p = make(proc, rex)
    for pt in [original(proc)] + new_points(proc)[:2]:
        got = p.me2(dev(mom), pt).cpu().numpy()
        ref = oracle_rw.me2(proc, mom, pt)
        assert np.max(rel(got, ref)) < FP64_TOL, (proc, pt, np.max(rel(got, ref)))


@pytest.mark.parametrize("proc", ["ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_reweight_parity_fp64(rex, proc):
    n = SIZES[proc]
    mom = ps.make_events(proc, n, 202)
    w = np.random.default_rng(3).uniform(0.5, 2.0, n)
    pts = new_points(proc)
    p = make(proc, rex)
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight(proc, mom, w, original(proc), pts)
    assert got.shape == (n, len(pts))
    assert np.max(rel(got, ref)) < FP64_TOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("proc", ["ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_unchanged_point_gives_input_weight_exactly(rex, proc, precision):
    if proc == "ee_mumu" and precision == 1:
        pytest.skip("ee_mumu is FP64 only")
    n = SIZES[proc]
    mom = ps.make_events(proc, n, 303)
    w = np.random.default_rng(4).uniform(0.5, 2.0, n)
    p = make(proc, rex, precision)
    got = p.reweight(dev(mom), dev(w), [original(proc)] * 3).cpu().numpy()
    assert np.array_equal(got, np.repeat(w[:, None], 3, axis=1))


@pytest.mark.parametrize("proc", ["gg_ttx", "gg_ttxg"])
def test_alphas_only_points_scale_exactly(rex, proc):
    n = SIZES[proc]
    mom = ps.make_events(proc, n, 404)
    w = np.ones(n)
    p = make(proc, rex)
    got = p.reweight(dev(mom), dev(w), [dict(mt=173.0, wt=0.0, alphas=0.124)]).cpu().numpy()
    assert np.allclose(got, (0.124 / 0.118) ** NGLUON[proc], rtol=1e-14, atol=0)


def test_dedupe_matches_per_point_evaluation_bitwise(rex):
    mom = dev(ps.make_events("gg_ttxg", 77, 505))
    w = dev(np.linspace(0.5, 1.5, 77))
    pts = ps.grid_gg_ttxg()
    a = make("gg_ttxg", rex)
    b = make("gg_ttxg", rex)
    b.set_flags(rex.FLAG_NO_DEDUPE)
    assert torch.equal(a.reweight(mom, w, pts), b.reweight(mom, w, pts))


def test_point_lists_longer_than_one_launch(rex):
    """300 points with 75 distinct masses: several launches, columns stitched."""
    n = 40
    mom = ps.make_events("gg_ttx", n, 606)
    w = np.ones(n)
    mts = np.linspace(165.0, 180.0, 75)
    pts = [dict(mt=float(mts[i % 75]), wt=0.0, alphas=0.110 + 0.0001 * (i % 4)) for i in range(300)]
    p = make("gg_ttx", rex)
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    sub = [0, 1, 63, 64, 74, 75, 150, 255, 256, 299]
    ref = oracle_rw.reweight("gg_ttx", mom, w, ORIG_QCD, [pts[i] for i in sub])
    assert np.max(rel(got[:, sub], ref)) < FP64_TOL


def test_top_width(rex):
    n = 33
    mom = ps.make_events("gg_ttxg", n, 707)
    w = np.ones(n)
    orig = dict(mt=173.0, wt=1.4, alphas=0.118)
    pts = [dict(mt=172.0, wt=1.3, alphas=0.118), dict(mt=174.0, wt=0.0, alphas=0.120)]
    p = rex.Process("gg_ttxg")
    p.set_params(orig)
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight("gg_ttxg", mom, w, orig, pts)
    assert np.max(rel(got, ref)) < FP64_TOL


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17])
def test_ragged_tails(rex, n):
    mom = ps.make_events("gg_ttxg", n, 808)
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()[:5]
    p = make("gg_ttxg", rex)
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight("gg_ttxg", mom, w, ORIG_QCD, pts)
    assert np.max(rel(got, ref)) < FP64_TOL


def test_empty_inputs_leave_outputs_untouched(rex):
    p = make("gg_ttxg", rex)
    mom = dev(ps.make_events("gg_ttxg", 4, 1))
    w = dev(np.ones(4))
    out = torch.full((4, 2), 7.0, dtype=torch.float64, device="cuda")
    p.reweight(mom[:0], w[:0], ps.grid_gg_ttxg()[:2], w_out=out[:0])
    p.reweight(mom, w, [], w_out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)


def test_nonfinite_momenta_give_nan_for_that_event_only(rex):
    mom = ps.make_events("gg_ttxg", 20, 909)
    mom[5, 4, 1] = np.nan
    p = make("gg_ttxg", rex)
    got = p.reweight(dev(mom), dev(np.ones(20)), ps.grid_gg_ttxg()[:3]).cpu().numpy()
    assert np.all(np.isnan(got[5]))
    assert np.all(np.isfinite(np.delete(got, 5, axis=0)))


def test_host_entry_point_matches_device_entry_point(rex):
    n = 90
    mom = ps.make_events("gg_ttxg", n, 111)
    w = np.random.default_rng(5).uniform(0.5, 2.0, n)
    pts = ps.grid_gg_ttxg()
    p = make("gg_ttxg", rex)
    dev_out = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    host_out = np.zeros((n, len(pts)))
    p.reweight_host(mom, w, pts, host_out)
    assert np.array_equal(dev_out, host_out)


@pytest.mark.parametrize("proc,precision", [("gg_ttx", 1), ("qq_ttx", 0), ("ee_mumu", 0)])
def test_host_entry_point_pipelines_chunks(rex, proc, precision):
    """rex_reweight_host in chunks of 2^16 events on two streams: 4 chunks and a ragged
    tail, from page-locked and from pageable host arrays, bitwise equal to one device
    launch; then a smaller call on the same handle (buffers already grown)."""
    n = 3 * (1 << 16) + 4321
    mom = ps.make_events(proc, n, 112)
    w = np.random.default_rng(6).uniform(0.5, 2.0, n)
    pts = ps.grid_gg_ttx()[:5] if proc != "ee_mumu" else [ps.EE_NEW, ps.EE_ORIGINAL]
    p = rex.Process(proc, precision)
    p.set_params(ps.EE_ORIGINAL if proc == "ee_mumu" else ORIG_QCD)
    ref = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    pinned = [torch.from_numpy(a).pin_memory() for a in (mom, w)]
    out_pinned = torch.zeros((n, len(pts)), dtype=torch.float64).pin_memory()
    p.reweight_host(pinned[0], pinned[1], pts, out_pinned)
    assert np.array_equal(out_pinned.numpy(), ref)
    out = np.zeros((n, len(pts)))
    p.reweight_host(mom, w, pts, out)
    assert np.array_equal(out, ref)
    small = np.zeros((1000, len(pts)))
    p.reweight_host(mom[:1000], w[:1000], pts, small)
    assert np.array_equal(small, ref[:1000])
    p.close()


@pytest.mark.parametrize("proc", ["gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_mixed_precision_error_bound(rex, proc):
    n = SIZES[proc] * 2
    mom = ps.make_events(proc, n, 222)
    w = np.ones(n)
    pts = new_points(proc)
    p = make(proc, rex, precision=1)
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight(proc, mom, w, ORIG_QCD, pts)
    err = np.max(rel(got, ref))
    assert err < MIXED_TOL[proc], err


def test_full_size_workload_sampled(rex):
    """The benchmark workload (2^20 g g -> t t~ g events, 16 points) in the launch
    configuration the benchmark times, checked on sampled events."""
    n = 1 << 20
    mom = ps.make_events("gg_ttxg", n, 3)
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()
    p = make("gg_ttxg", rex)
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.random.default_rng(6).choice(n, 24, replace=False)
    idx = np.concatenate([idx, [0, n - 1]])
    ref = oracle_rw.reweight("gg_ttxg", mom[idx], w[idx], ORIG_QCD, pts)
    assert np.max(rel(got[idx], ref)) < FP64_TOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("proc", ["gg_ttx", "gg_ttxg", "gg_ttxgg"])
def test_every_kernel_variant(rex, proc, precision):
    """Each thread-mapping variant against the oracle (FP64) or the mixed bound."""
    n = SIZES[proc]
    mom = ps.make_events(proc, n, 515)
    w = np.random.default_rng(8).uniform(0.5, 2.0, n)
    pts = new_points(proc)[:4]
    ref = oracle_rw.reweight(proc, mom, w, ORIG_QCD, pts)
    p = make(proc, rex, precision)
    tol = FP64_TOL if precision == 0 else MIXED_TOL[proc]
    assert p.num_variants == 9
    for v in range(p.num_variants):
        p.variant = v
        got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
        assert np.max(rel(got, ref)) < tol, (v, np.max(rel(got, ref)))
        same = p.reweight(dev(mom), dev(w), [ORIG_QCD]).cpu().numpy()
        assert np.array_equal(same[:, 0], w), v


def test_autotune_picks_the_fastest_variant(rex):
    n = 1 << 14
    mom = dev(ps.make_events("gg_ttxg", n, 616))
    w = dev(np.ones(n))
    out = torch.empty((n, 16), dtype=torch.float64, device="cuda")
    p = make("gg_ttxg", rex, 1)
    ms = p.autotune(mom, w, ps.grid_gg_ttxg(), out)
    assert len(ms) == 9 and all(t > 0 for t in ms)
    assert p.variant == int(np.argmin(ms))
    with pytest.raises(rex.RexError):
        p.variant = 9


def test_fp64_tolerance_rule_on_ill_conditioned_events(rex):
    """The tolerance rule of the exact mode: an (event, point) may miss 1e-12 only if
    the oracle's condition estimate explains it, err <= 64 eps (kappa_0 + kappa_j).
    Events 75 and 146 of the seeded 512-event g g -> t t~ g g sample are the two
    that miss 1e-12 (5.2e-12 at point 13 and 1.0e-12 at point 51, kappa ~ 6e4 and
    7e3); six well-conditioned events of the same sample are checked beside them."""
    from oracle import qcd
    mom = ps.make_events("gg_ttxgg", 512, 3)
    grid = ps.grid_64()
    idx = np.array([75, 146, 0, 100, 200, 300, 400, 511])
    pts = [grid[13], grid[51]]
    got = make("gg_ttxgg", rex).reweight(dev(mom[idx]), dev(np.ones(len(idx))), pts).cpu().numpy()
    ref = oracle_rw.reweight("gg_ttxgg", mom[idx], np.ones(len(idx)), ORIG_QCD, pts)
    err = rel(got, ref)
    eps = np.finfo(float).eps
    worst = 0.0
    for i, j in zip(*np.nonzero(err > FP64_TOL)):
        k0 = qcd.condition(mom[idx[i]:idx[i] + 1], ORIG_QCD["mt"], 0.0, ORIG_QCD["alphas"])[0]
        kj = qcd.condition(mom[idx[i]:idx[i] + 1], pts[j]["mt"], 0.0, pts[j]["alphas"])[0]
        assert err[i, j] <= 64 * eps * (k0 + kj), (idx[i], j, err[i, j], k0, kj)
        worst = max(worst, err[i, j])
    assert np.all(err[2:] < FP64_TOL)          # the well-conditioned events meet 1e-12 outright


def test_fp64_ill_conditioned_events_against_extended_precision(rex):
    """The same eight events against the oracle's diagrams evaluated in extended precision
    (np.longdouble), which removes the FP64 oracle's own rounding (6.3e-12 on event 75):
    the kernel's error is then its own, and it stays within 64 eps (kappa_0 + kappa_j)."""
    from oracle import qcd
    mom = ps.make_events("gg_ttxgg", 512, 3)
    grid = ps.grid_64()
    idx = np.array([75, 146, 0, 100, 200, 300, 400, 511])
    pts = [grid[13], grid[51]]
    got = make("gg_ttxgg", rex).reweight(dev(mom[idx]), dev(np.ones(len(idx))), pts).cpu().numpy()
    ext = mom[idx].astype(np.longdouble)
    m0 = qcd.me2(ext, ORIG_QCD["mt"], 0.0, ORIG_QCD["alphas"])
    eps = np.finfo(float).eps
    k0 = qcd.condition(mom[idx], ORIG_QCD["mt"], 0.0, ORIG_QCD["alphas"])
    for j, pt in enumerate(pts):
        ref = (qcd.me2(ext, pt["mt"], 0.0, pt["alphas"]) / m0).astype(np.float64)
        kj = qcd.condition(mom[idx], pt["mt"], 0.0, pt["alphas"])
        err = np.abs(got[:, j] / ref - 1.0)
        assert np.all(err <= 64 * eps * (k0 + kj)), (j, err, k0, kj)
        assert np.all(err[2:] < FP64_TOL)


def test_full_size_ee_every_event(rex):
    """e+e- -> mu+mu-: the full 4096-event sample at the new electroweak point, every event
    against the oracle."""
    mom = ps.make_events("ee_mumu", 4096, 1)
    w = np.ones(4096)
    got = make("ee_mumu", rex).reweight(dev(mom), dev(w), [ps.EE_NEW]).cpu().numpy()
    ref = oracle_rw.reweight("ee_mumu", mom, w, ps.EE_ORIGINAL, [ps.EE_NEW])
    assert np.max(rel(got, ref)) < FP64_TOL


def test_full_size_gg_ttx_sampled(rex):
    """g g -> t t~ at 2^20 events x 8 points: the FP64 kernel on sampled events against the
    oracle, the mixed kernel against the FP64 one at every event."""
    n = 1 << 20
    mom = ps.make_events("gg_ttx", n, 2)
    w = np.ones(n)
    pts = ps.grid_gg_ttx()
    dm, dw = dev(mom), dev(w)
    got = make("gg_ttx", rex).reweight(dm, dw, pts).cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.concatenate([np.random.default_rng(8).choice(n, 32, replace=False), [0, n - 1]])
    ref = oracle_rw.reweight("gg_ttx", mom[idx], w[idx], ORIG_QCD, pts)
    assert np.max(rel(got[idx], ref)) < FP64_TOL
    mixed = make("gg_ttx", rex, precision=1).reweight(dm, dw, pts).cpu().numpy()
    assert np.max(rel(mixed, got)) < MIXED_TOL["gg_ttx"]


def test_full_size_gg_ttxg_mixed_every_event(rex):
    """The headline workload (2^20 g g -> t t~ g events x 16 points) in mixed precision against
    the FP64 kernel at every event (the FP64 kernel is checked against the oracle above)."""
    n = 1 << 20
    mom = ps.make_events("gg_ttxg", n, 3)
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()
    dm, dw = dev(mom), dev(w)
    exact = make("gg_ttxg", rex).reweight(dm, dw, pts).cpu().numpy()
    mixed = make("gg_ttxg", rex, precision=1).reweight(dm, dw, pts).cpu().numpy()
    assert np.max(rel(mixed, exact)) < MIXED_TOL["gg_ttxg"]
