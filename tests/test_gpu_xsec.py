"""Reweighted cross sections on the GPU (rex_xsec_*) against the oracle of
Sec. 3.1.2 (needs a B300).  FP64 throughout; the tolerance 1e-12 is the exact
mode's, the accumulation order is fixed (bitwise reproducible)."""
import numpy as np
import pytest

from rexlib import ensure_built
from oracle import xsec as oracle_xsec
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def sample(n, k, seed, zeros=True):
    g = np.random.default_rng(seed)
    w = g.uniform(0.2, 3.0, n)
    if zeros and n >= 50:
        w[g.choice(n, n // 50, replace=False)] = 0.0
    wn = w[:, None] * g.lognormal(0.0, 0.3, (n, k))
    wn[w == 0.0] = 0.0
    return w, wn


def run(rex, w, wn, sigma, dsigma, splits=None):
    x = rex.XSec(wn.shape[1])
    dw, dwn = torch.from_numpy(w).cuda(), torch.from_numpy(np.ascontiguousarray(wn)).cuda()
    bounds = [0] + list(splits or []) + [w.shape[0]]
    for a, b in zip(bounds[:-1], bounds[1:]):
        x.accumulate(dw[a:b], dwn[a:b])
    out = x.result(sigma, dsigma)
    x.close()
    return out


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("n,k", [(1, 1), (37, 5), (10007, 37), (70001, 64)])
def test_matches_the_oracle(rex, n, k):
    w, wn = sample(n, k, n)
    s, ds, fb = run(rex, w, wn, 3.7, 0.21)
    rs, rds, rfb = oracle_xsec.reweighted_xsec(w, wn, 3.7, 0.21)
    assert np.array_equal(fb, rfb)
    assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL


def test_accumulation_over_calls_and_bitwise_reproducibility(rex):
    w, wn = sample(50000, 16, 4)
    whole = run(rex, w, wn, 1.0, 0.05)
    parts = run(rex, w, wn, 1.0, 0.05, splits=[1, 4097, 4098, 30000])
    again = run(rex, w, wn, 1.0, 0.05, splits=[1, 4097, 4098, 30000])
    rs, rds, _ = oracle_xsec.reweighted_xsec(w, wn, 1.0, 0.05)
    for s, ds, _ in (whole, parts):
        assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL
    assert np.array_equal(parts[0], again[0]) and np.array_equal(parts[1], again[1])


def test_fallback_branch(rex):
    w = np.full(300, 1.0)
    wn = np.stack([np.full(300, 0.25), np.full(300, -1.0), np.zeros(300)], axis=1)
    s, ds, fb = run(rex, w, wn, 2.0, 0.2)
    rs, rds, rfb = oracle_xsec.reweighted_xsec(w, wn, 2.0, 0.2)
    assert list(fb) == [False, True, True] and np.array_equal(fb, rfb)
    assert np.allclose(s, rs, rtol=TOL) and ds[0] == pytest.approx(rds[0], rel=TOL)
    assert ds[1] == pytest.approx(-0.2, rel=TOL) and np.isinf(ds[2])


def test_nonfinite_weight_poisons_only_its_point(rex):
    w, wn = sample(1000, 3, 9, zeros=False)
    wn[17, 1] = np.nan
    s, ds, fb = run(rex, w, wn, 1.0, 0.1)
    assert np.isnan(s[1]) and fb[1] and not fb[0] and not fb[2]
    rs, rds, _ = oracle_xsec.reweighted_xsec(w, wn, 1.0, 0.1)
    assert np.max(rel(s[[0, 2]], rs[[0, 2]])) < TOL


def test_empty_call_is_a_no_op(rex):
    w, wn = sample(500, 4, 2)
    x = rex.XSec(4)
    dw, dwn = torch.from_numpy(w).cuda(), torch.from_numpy(wn).cuda()
    x.accumulate(dw[:0], dwn[:0])
    x.accumulate(dw, dwn)
    s, ds, _ = x.result(1.0, 0.1)
    rs, rds, _ = oracle_xsec.reweighted_xsec(w, wn, 1.0, 0.1)
    assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL
    x.reset()
    x.accumulate(dw[:250], dwn[:250])
    s2, _, _ = x.result(1.0, 0.1)
    rs2, _, _ = oracle_xsec.reweighted_xsec(w[:250], wn[:250], 1.0, 0.1)
    assert np.max(rel(s2, rs2)) < TOL
    x.close()


def test_on_the_benchmark_weights(rex):
    """The reduction on the output of the benchmark's launch (2^20 g g -> t t~ g
    events x 16 points); the unchanged-mass, unchanged-alphas column does not exist
    in this grid, so every column is a genuine reweighting."""
    n = 1 << 20
    mom = torch.from_numpy(ps.make_events("gg_ttxg", n, 3)).cuda()
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    p = rex.Process("gg_ttxg", 0)
    p.set_params(mt=173.0, wt=0.0, alphas=0.118)
    pts = ps.grid_gg_ttxg()
    wn = p.reweight(mom, w, pts)
    x = rex.XSec(len(pts))
    x.accumulate(w, wn)
    s, ds, fb = x.result(10.0, 0.3)
    x.close()
    rs, rds, rfb = oracle_xsec.reweighted_xsec(w.cpu().numpy(), wn.cpu().numpy(), 10.0, 0.3)
    assert np.array_equal(fb, rfb) and not fb.any()
    assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL


def test_state_round_trip_and_merge_of_two_accumulators(rex):
    """Two accumulators over the halves of a sample (as two GPUs would hold them),
    their states merged on the host and loaded into a third: the result of the whole
    sample.  A state read and written back is unchanged, bit for bit."""
    w, wn = sample(30001, 12, 21)
    dw, dwn = torch.from_numpy(w).cuda(), torch.from_numpy(wn).cuda()
    a, b, c = rex.XSec(12), rex.XSec(12), rex.XSec(12)
    a.accumulate(dw[:14000], dwn[:14000])
    b.accumulate(dw[14000:], dwn[14000:])
    sa, sb = a.get_state(), b.get_state()
    c.set_state(rex.xsec_merge_states(sa, sb, 12))
    s, ds, fb = c.result(4.0, 0.2)
    rs, rds, rfb = oracle_xsec.reweighted_xsec(w, wn, 4.0, 0.2)
    assert np.array_equal(fb, rfb)
    assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL
    a.set_state(sa)
    assert np.array_equal(a.get_state(), sa)
    for x in (a, b, c):
        x.close()


@pytest.mark.parametrize("scale", [1e-250, 1e-30, 1e30, 1e250])
def test_uniformly_scaled_weights(rex, scale):
    """The double-float sums scale each thread's values by a power of two near its first
    value, so weights of any common magnitude keep the exact mode's tolerance."""
    w, wn = sample(20000, 8, 12)
    s, ds, fb = run(rex, w, wn * scale, 1.0, 0.1)
    rs, rds, rfb = oracle_xsec.reweighted_xsec(w, wn * scale, 1.0, 0.1)
    assert np.array_equal(fb, rfb)
    assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL


def test_values_beyond_the_double_float_range_take_the_fp64_path(rex):
    """Blocks holding a value further than 2^40 from its thread's scale, a subnormal or
    a tiny input weight are summed in FP64 instead (same tolerance); the others stay in
    double-float."""
    w, wn = sample(9000, 6, 13, zeros=False)
    wn[5, 2] *= 1e20               # 2^66 above its neighbours
    wn[2100, 0] = 1e-310           # subnormal
    w[4500] = 1e-30                # reciprocal beyond 2^60
    wn[4500] *= 1e-30
    s, ds, fb = run(rex, w, wn, 1.0, 0.1)
    rs, rds, rfb = oracle_xsec.reweighted_xsec(w, wn, 1.0, 0.1)
    assert np.array_equal(fb, rfb)
    assert np.max(rel(s, rs)) < TOL and np.max(rel(ds, rds)) < TOL
