"""q q~ -> t t~ on the GPU vs the FP64 oracle, through the C ABI (needs a B300).

Tolerances:
* FP64 mode: 1e-12 relative per event on |M|^2 and on every new weight (one
  diagram, a helicity sum of non-negative terms: the condition number of the
  oracle's sum is 1, and the kernel's C0 + C2 m^2 + C4 m^4 form adds a few
  roundings).
* mixed mode (FP32 spinors and currents, FP64 s, polynomial and ratio): 1e-5.
* unchanged parameter point: new weight == input weight exactly.
"""
import numpy as np
import pytest

from rexlib import ensure_built
from oracle import qq as oracle_qq
from oracle import reweight as oracle_rw
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5
ORIG = dict(mt=173.0, wt=0.0, alphas=0.118)
PROC = "qq_ttx"


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(rex, precision=0):
    p = rex.Process(PROC, precision)
    p.set_params(ORIG)
    return p


def rel(a, b):
    return np.abs(a / b - 1.0)


def points():
    # the 64-point (mt, alphas) grid plus points with a top width (no effect here)
    return ps.grid_64()[::3] + [dict(mt=171.0, wt=1.4, alphas=0.118), dict(mt=173.0, wt=2.0, alphas=0.121)]


def test_single_kernel_variant(rex):
    p = make(rex)
    assert p.num_variants == 1 and p.variant == 0
    with pytest.raises(Exception):
        p.variant = 1


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_me2_parity(rex, precision, tol):
    n = 301   # three tiles of 128, ragged tail of 45
    mom = ps.make_events(PROC, n, 31)
    p = make(rex, precision)
    for pt in (ORIG, dict(mt=168.0, wt=0.0, alphas=0.125)):
        got = p.me2(dev(mom), pt).cpu().numpy()
        ref = oracle_qq.me2(mom, pt["mt"], pt["wt"], pt["alphas"])
        assert np.max(rel(got, ref)) < tol


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_reweight_parity(rex, precision, tol):
    n = 515
    mom = ps.make_events(PROC, n, 32)
    w = np.random.default_rng(3).uniform(-1.0, 2.0, n)
    pts = points()
    got = make(rex, precision).reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight(PROC, mom, w, ORIG, pts)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < tol


@pytest.mark.parametrize("precision", [0, 1])
def test_unchanged_point_and_alphas_scaling(rex, precision):
    n = 200
    mom = ps.make_events(PROC, n, 33)
    w = np.random.default_rng(4).uniform(0.5, 2.0, n)
    pts = [ORIG, dict(mt=173.0, wt=0.0, alphas=0.124), dict(mt=173.0, wt=3.0, alphas=0.118)]
    got = make(rex, precision).reweight(dev(mom), dev(w), pts).cpu().numpy()
    assert np.array_equal(got[:, 0], w)
    assert np.max(rel(got[:, 1], w * (0.124 / 0.118) ** 2)) < 1e-14
    assert np.array_equal(got[:, 2], w)   # the width enters no propagator


@pytest.mark.parametrize("n", [1, 2, 127, 128, 129])
def test_ragged_tails(rex, n):
    mom = ps.make_events(PROC, n, 34)
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()
    got = make(rex).reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight(PROC, mom, w, ORIG, pts)
    assert np.max(rel(got, ref)) < FP64_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_empty_inputs_and_nonfinite_events(rex, precision):
    p = make(rex, precision)
    mom = ps.make_events(PROC, 40, 35)
    out = torch.full((40, 2), 7.0, dtype=torch.float64, device="cuda")
    p.reweight(dev(mom)[:0], dev(np.ones(40))[:0], ps.grid_gg_ttx()[:2], w_out=out[:0])
    p.reweight(dev(mom), dev(np.ones(40)), [], w_out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    mom[9, 2, 3] = np.nan
    mom[17, 0, 0] = np.inf
    pts = ps.grid_gg_ttx()[:3] + [ORIG, dict(mt=173.0, wt=0.0, alphas=0.121)]   # incl. same-mass points
    got = p.reweight(dev(mom), dev(np.ones(40)), pts).cpu().numpy()
    assert np.all(np.isnan(got[[9, 17]]))
    assert np.all(np.isfinite(np.delete(got, [9, 17], axis=0)))


def test_full_size_workload_sampled(rex):
    """2^20 events and 16 points (the g g -> t t~ g benchmark shape) on the FP64 kernel,
    sampled events against the oracle; the mixed kernel against the FP64 one everywhere."""
    n = 1 << 20
    mom = ps.make_events(PROC, n, 36)
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()
    dm, dw = dev(mom), dev(w)
    got = make(rex).reweight(dm, dw, pts).cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.concatenate([np.random.default_rng(7).choice(n, 32, replace=False), [0, 127, 128, n - 1]])
    ref = oracle_rw.reweight(PROC, mom[idx], w[idx], ORIG, pts)
    assert np.max(rel(got[idx], ref)) < FP64_TOL
    mixed = make(rex, 1).reweight(dm, dw, pts).cpu().numpy()
    assert np.max(rel(mixed, got)) < MIXED_TOL


def test_integer_alu_conversions_round_like_ieee(rex):
    """The mixed tile's FP64 -> FP32 conversion (round to nearest even, flush below
    2^-126) and the exact FP32 -> FP64 one, against numpy's IEEE casts."""
    rng = np.random.default_rng(9)
    x = np.concatenate([
        rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
        # ties: values exactly half-way between two FP32 numbers, both parities
        (np.arange(1, 2001, dtype=np.float64) + 0.5) * 2.0 ** -23 + 1.0,
        -(np.arange(1, 2001, dtype=np.float64) + 0.5) * 2.0 ** -23 - 1.0,
        np.nextafter(np.float64(np.finfo(np.float32).max), np.inf) * np.array([1.0, -1.0]),
        np.array([0.0, -0.0, 1.0, -2.5, 3.4e38, 3.5e38, -1e39, 1.2e-38, 1.1754943508222875e-38,
                  1e-40, -1e-45, 1e-300, np.inf, -np.inf, np.nan, 173.0, 0.118]),
    ])
    f32, f64, fin = rex.probe_convert(torch.from_numpy(x).cuda())
    f32, f64, fin = f32.cpu().numpy(), f64.cpu().numpy(), fin.cpu().numpy()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    tiny = np.abs(x) < 2.0 ** -126
    ref[tiny] = np.copysign(np.float32(0.0), x[tiny]).astype(np.float32)
    nan = np.isnan(x)
    assert np.all(np.isnan(f32[nan])) and np.all(np.isnan(f64[nan]))
    assert np.array_equal(f32[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    assert np.array_equal(f64[~nan].view(np.uint64), ref[~nan].astype(np.float64).view(np.uint64))
    # the momentum conversion (finiteness checked per event) agrees wherever it is defined
    ok = np.isfinite(x) & (np.abs(x) < 2.0 ** 128)
    assert np.array_equal(fin[ok].view(np.uint32), ref[ok].view(np.uint32))
