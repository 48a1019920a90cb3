"""The crossed q q~ -> t t~ g channels on the GPU vs the FP64 oracle, through the C ABI
(needs a B300).

Each channel (q~ q, q g, g q, q~ g, g q~ initial states) runs the q q~ -> t t~ g kernels
with the event's partons read into the direct channel's slots; the oracle evaluates
each channel from its own external wavefunctions.  Tolerances as for the direct
channel: FP64 1e-12 relative per weight, mixed precision 1e-4 on the samples.  A
crossed light line exchanges a t-channel gluon, t = (p_in - p_out)^2 of the light
quark, and for a forward quark the Feynman-gauge diagrams on it cancel to
|t| / s_hat of their size: rounding is amplified by kappa = s_hat / |t|.  The
mixed-against-FP64 check over every event of a large sample therefore holds each
event to max(1e-4, 4 * 2^-24 * kappa) and at most 1e-3 of the events above 1e-4.
"""
import numpy as np
import pytest

from rexlib import ensure_built
from oracle import reweight as oracle_rw
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-4
ORIG = dict(mt=173.0, wt=0.0, alphas=0.118)
CROSSED = ["qxq_ttxg", "qg_ttxq", "gq_ttxq", "qxg_ttxqx", "gqx_ttxqx"]


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(rex, proc, precision=0):
    p = rex.Process(proc, precision)
    p.set_params(ORIG)
    return p


def rel(a, b):
    return np.abs(a / b - 1.0)


def mdot(a):
    return a[:, 0] ** 2 - a[:, 1] ** 2 - a[:, 2] ** 2 - a[:, 3] ** 2


def points():
    return ps.grid_gg_ttxg() + [dict(mt=172.0, wt=1.4, alphas=0.118), ORIG, dict(mt=173.0, wt=0.0, alphas=0.124)]


@pytest.mark.parametrize("proc", CROSSED)
@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_me2_and_reweight_parity(rex, proc, precision, tol):
    n = 75   # 3 tiles of 32, ragged tail
    mom = ps.make_events(proc, n, 81)
    p = make(rex, proc, precision)
    for pt in (ORIG, dict(mt=169.0, wt=1.0, alphas=0.125)):
        got = p.me2(dev(mom), pt).cpu().numpy()
        ref = oracle_rw.me2(proc, mom, pt)
        assert np.max(rel(got, ref)) < tol
    w = np.random.default_rng(11).uniform(-1.0, 2.0, n)
    pts = points()
    got = p.reweight(dev(mom), dev(w), pts).cpu().numpy()
    ref = oracle_rw.reweight(proc, mom, w, ORIG, pts)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < tol
    j = pts.index(ORIG)
    assert np.array_equal(got[:, j], w)
    assert np.max(rel(got[:, j + 1], w * (0.124 / 0.118) ** 3)) < 1e-14


@pytest.mark.parametrize("proc", ["qg_ttxq", "qxg_ttxqx"])
def test_mixed_against_fp64_at_scale(rex, proc):
    """2^18 events x 16 points: mixed against FP64 at every event, FP64 against the
    oracle on sampled events."""
    n = 1 << 18
    mom = ps.make_events(proc, n, 82)
    w = np.ones(n)
    pts = ps.grid_gg_ttxg()
    dm, dw = dev(mom), dev(w)
    exact = make(rex, proc).reweight(dm, dw, pts).cpu().numpy()
    idx = np.concatenate([np.random.default_rng(12).choice(n, 10, replace=False), [0, n - 1]])
    assert np.max(rel(exact[idx], oracle_rw.reweight(proc, mom[idx], w[idx], ORIG, pts))) < FP64_TOL
    mixed = make(rex, proc, 1).reweight(dm, dw, pts).cpu().numpy()
    err = np.max(rel(mixed, exact), axis=1)
    kappa = mdot(mom[:, 0] + mom[:, 1]) / np.abs(mdot(mom[:, 0] - mom[:, 4]))
    bound = np.maximum(MIXED_TOL, 4.0 * 2.0 ** -24 * kappa)
    over = float(np.mean(err > MIXED_TOL))
    print(f"{proc} mixed vs FP64 max rel err {err.max():.3e} (kappa {kappa[np.argmax(err)]:.3e}), "
          f"max err / bound {np.max(err / bound):.3f}, fraction above {MIXED_TOL:g}: {over:.2e}")
    assert np.all(err < bound)
    assert over < 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_every_channel_in_one_persistent_launch(rex, precision):
    """A p p -> t t~ + jet sample: g g, q q~ and four crossed channels as batches of one
    persistent multi-process launch, each equal to its own single-process launch."""
    pts = ps.grid_gg_ttxg()
    batches, single = [], []
    for i, (proc, n) in enumerate((("gg_ttxg", 40), ("qq_ttxg", 33), ("qg_ttxq", 65), ("gq_ttxq", 31),
                                   ("qxg_ttxqx", 47), ("gqx_ttxqx", 1))):
        p = make(rex, proc, precision)
        dm = dev(ps.make_events(proc, n, 90 + i))
        dw = torch.ones(n, dtype=torch.float64, device="cuda")
        batches.append((p, dm, dw, torch.zeros((n, len(pts)), dtype=torch.float64, device="cuda")))
        single.append(p.reweight(dm, dw, pts).cpu().numpy())
    m = rex.Multi(precision)
    m.reweight(batches, pts)
    torch.cuda.synchronize()
    for b, ref in zip(batches, single):
        assert np.max(rel(b[3].cpu().numpy(), ref)) < 1e-13
    m.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_pp_ttxj_sample(rex, precision):
    """The benchmark's four-channel p p -> t t~ + jet sample (2^20 events, 16 points) in
    one persistent launch, as it is timed: FP64 against the oracle on sampled events of
    every channel; mixed against each channel's own single-process launch."""
    spec = (("gg_ttxg", 786432, 13), ("qg_ttxq", 131072, 15), ("qxg_ttxqx", 65536, 16), ("qq_ttxg", 65536, 14))
    pts = ps.grid_gg_ttxg()
    batches, moms = [], []
    for proc, n, seed in spec:
        p = make(rex, proc, precision)
        mom = ps.make_events(proc, n, seed)
        moms.append(mom)
        batches.append((p, dev(mom), torch.ones(n, dtype=torch.float64, device="cuda"),
                        torch.zeros((n, len(pts)), dtype=torch.float64, device="cuda")))
    m = rex.Multi(precision)
    m.reweight(batches, pts)
    torch.cuda.synchronize()
    for (proc, n, _), mom, b in zip(spec, moms, batches):
        got = b[3].cpu().numpy()
        if precision == 0:
            idx = np.concatenate([np.random.default_rng(13).choice(n, 5, replace=False), [0, n - 1]])
            ref = oracle_rw.reweight(proc, mom[idx], np.ones(len(idx)), ORIG, pts)
            assert np.max(rel(got[idx], ref)) < FP64_TOL, proc
        else:
            single = b[0].reweight(b[1], b[2], pts).cpu().numpy()
            assert np.max(rel(got, single)) < 1e-13, proc
    m.close()
