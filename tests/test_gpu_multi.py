"""Persistent multi-process launch vs the single-process entry point and the
oracle, through the C ABI (needs a B300)."""
import numpy as np
import pytest

from rexlib import ensure_built
from oracle import reweight as oracle_rw
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORIG_QCD = dict(mt=173.0, wt=0.0, alphas=0.118)
SIZES = {"ee_mumu": 150, "gg_ttx": 101, "gg_ttxg": 53, "gg_ttxgg": 19, "qq_ttx": 300}


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def points(k):
    g = ps.grid_64()
    return [dict(g[(7 * j) % 64], **ps.EE_NEW) for j in range(k)]


def setup(rex, precision, seed=11):
    out = []
    for proc, n in SIZES.items():
        mom = ps.make_events(proc, n, seed + n)
        w = np.random.default_rng(n).uniform(0.5, 2.0, n)
        p = rex.Process(proc, 0 if proc == "ee_mumu" else precision)   # ee_mumu: FP64 only
        p.set_params(ps.EE_ORIGINAL if proc == "ee_mumu" else ORIG_QCD)
        out.append((proc, p, mom, w))
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_multi_matches_single_process_launches(rex, precision, mode):
    pts = points(9)
    items = setup(rex, precision)
    m = rex.Multi(precision, mode)
    batches, single = [], []
    for proc, p, mom, w in items:
        dm, dw = dev(mom), dev(w)
        wo = torch.zeros((mom.shape[0], len(pts)), dtype=torch.float64, device="cuda")
        batches.append((p, dm, dw, wo))
        single.append(p.reweight(dm, dw, pts).cpu().numpy())
    m.reweight(batches, pts)
    torch.cuda.synchronize()
    for (proc, p, mom, w), b, ref in zip(items, batches, single):
        got = b[3].cpu().numpy()
        assert np.max(np.abs(got / ref - 1.0)) < 1e-13, proc
        if precision == 0:
            orc = oracle_rw.reweight(proc, mom, w, ps.EE_ORIGINAL if proc == "ee_mumu" else ORIG_QCD, pts[:3])
            assert np.max(np.abs(got[:, :3] / orc - 1.0)) < 1e-12, proc


@pytest.mark.parametrize("mode", [0, 1])
def test_multi_graph_replay_and_point_chunks(rex, mode):
    """70 points: two launches per call (64 + 6) in persistent mode; a captured graph
    (fork-join of streams in stream mode) replays them."""
    pts = points(70)
    items = setup(rex, 1, seed=21)
    m = rex.Multi(1, mode)
    batches, refs = [], []
    for proc, p, mom, w in items:
        dm, dw = dev(mom), dev(w)
        batches.append((p, dm, dw, torch.zeros((mom.shape[0], 70), dtype=torch.float64, device="cuda")))
        refs.append(p.reweight(dm, dw, pts).cpu().numpy())
    m.capture(batches, pts)
    for b in batches:
        b[3].zero_()
    m.replay()
    torch.cuda.synchronize()
    for b, ref in zip(batches, refs):
        assert np.max(np.abs(b[3].cpu().numpy() / ref - 1.0)) < 1e-13


def test_multi_validation(rex):
    pts = points(2)
    m = rex.Multi(0)
    p64 = rex.Process("gg_ttx", 0)
    p64.set_params(ORIG_QCD)
    pmx = rex.Process("gg_ttx", 1)
    pmx.set_params(ORIG_QCD)
    mom = dev(ps.make_events("gg_ttx", 4, 1))
    w = dev(np.ones(4))
    wo = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(rex.RexError):
        m.reweight([], pts)
    with pytest.raises(rex.RexError):
        m.reweight([(pmx, mom, w, wo)], pts)          # precision mismatch
    ee = [rex.Process("ee_mumu", 0) for _ in range(2)]
    for e in ee:
        e.set_params(ps.EE_ORIGINAL)
    emom = dev(ps.make_events("ee_mumu", 4, 1))
    with pytest.raises(rex.RexError):
        m.reweight([(ee[0], emom, w, wo), (ee[1], emom, w, wo)], pts)
    with pytest.raises(rex.RexError):
        m.replay()                                    # nothing captured
    m.reweight([(p64, mom[:0], w[:0], wo[:0])], pts)  # empty batch: no-op
    m.reweight([(p64, mom, w, wo)], [])               # no points: no-op
    # a NULL parameter array with k = 1 is rejected before any point is read
    import ctypes
    lib = rex.load()
    barr = (rex.Batch * 1)(rex.Batch(p64._h.value, mom.data_ptr(), w.data_ptr(), 4, wo.data_ptr()))
    assert lib.rex_reweight_multi(m._h, barr, 1, None, 1, None) == rex.REX_EINVAL
    assert b"null parameter array" in lib.rex_last_error()
    assert lib.rex_multi_capture(m._h, barr, 1, None, 1) == rex.REX_EINVAL
    assert lib.rex_reweight_multi_noalloc(barr, 1, None, 1, 0, None) == rex.REX_EINVAL
    assert b"null parameter array" in lib.rex_last_error()


@pytest.mark.parametrize("subset", [("gg_ttx", "qq_ttx"), ("ee_mumu", "gg_ttx", "qq_ttx"),
                                    ("gg_ttx", "gg_ttxg", "qq_ttx"), ("gg_ttxgg", "qq_ttx")])
@pytest.mark.parametrize("precision", [0, 1])
def test_register_classes(rex, subset, precision):
    """The heaviest process of a launch picks the persistent kernel's register class
    (light: e+e-, g g -> t t~, q q~ -> t t~; + g g -> t t~ g; + g g -> t t~ g g); every
    class gives the single-process results."""
    pts = points(16)
    items = [it for it in setup(rex, precision, seed=31) if it[0] in subset]
    m = rex.Multi(precision)
    batches, single = [], []
    for proc, p, mom, w in items:
        dm, dw = dev(mom), dev(w)
        batches.append((p, dm, dw, torch.zeros((mom.shape[0], len(pts)), dtype=torch.float64, device="cuda")))
        single.append(p.reweight(dm, dw, pts).cpu().numpy())
    m.reweight(batches, pts)
    torch.cuda.synchronize()
    for (proc, *_), b, ref in zip(items, batches, single):
        assert np.max(np.abs(b[3].cpu().numpy() / ref - 1.0)) < 1e-13, proc
    m.close()


def test_config4_full_size_persistent_graph(rex):
    """The multi-process workload at full size in the launch configuration the benchmark
    times: 10k e+e- + 1M g g -> t t~ + 500k g g -> t t~ g + 100k g g -> t t~ g g, 64 points,
    one captured persistent launch in mixed precision.  Every batch against its own
    single-process launch at every event, sampled events against the oracle."""
    mixed_tol = {"ee_mumu": 1e-12, "gg_ttx": 1e-5, "gg_ttxg": 1e-3, "gg_ttxgg": 1e-3}
    pts = [dict(p, **ps.EE_NEW) for p in ps.grid_64()]
    spec = (("ee_mumu", 10_000, 41), ("gg_ttx", 1_000_000, 42), ("gg_ttxg", 500_000, 43), ("gg_ttxgg", 100_000, 44))
    batches, data = [], []
    for proc, n, seed in spec:
        p = rex.Process(proc, 0 if proc == "ee_mumu" else 1)
        orig = ps.EE_ORIGINAL if proc == "ee_mumu" else ORIG_QCD
        p.set_params(orig)
        mom = ps.make_events(proc, n, seed)
        dm, dw = dev(mom), torch.ones(n, dtype=torch.float64, device="cuda")
        batches.append((p, dm, dw, torch.zeros((n, 64), dtype=torch.float64, device="cuda")))
        data.append((proc, p, mom, orig, dm, dw))
    m = rex.Multi(1)
    m.capture(batches, pts)
    m.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    for (proc, p, mom, orig, dm, dw), b in zip(data, batches):
        got = b[3].cpu().numpy()
        single = p.reweight(dm, dw, pts).cpu().numpy()
        assert np.max(np.abs(got / single - 1.0)) < 1e-13, proc
        ns = 3 if proc == "gg_ttxgg" else 12
        idx = rng.choice(mom.shape[0], ns, replace=False)
        kp = pts if proc != "gg_ttxgg" else pts[::8]
        cols = list(range(64)) if proc != "gg_ttxgg" else list(range(0, 64, 8))
        ref = oracle_rw.reweight(proc, mom[idx], np.ones(ns), orig, kp)
        assert np.max(np.abs(got[idx][:, cols] / ref - 1.0)) < mixed_tol[proc], proc
    m.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_slot_groups_and_autotune(rex, precision):
    """Slot groups split each g g tile's mass slots over several work items (1, 3 and 8
    groups of the 16-mass point list, a ragged split included): every weight equals the
    single-process launch's; the autotuner times its six candidates and keeps one."""
    g = ps.grid_64()
    pts = [dict(g[j], **ps.EE_NEW) for j in range(0, 64, 4)]     # 8 masses x 2 alphas
    items = setup(rex, precision, seed=41)
    batches, single = [], []
    for proc, p, mom, w in items:
        dm, dw = dev(mom), dev(w)
        batches.append((p, dm, dw, torch.zeros((mom.shape[0], len(pts)), dtype=torch.float64, device="cuda")))
        single.append(p.reweight(dm, dw, pts).cpu().numpy())
    m = rex.Multi(precision)
    assert m.slot_groups == 1
    for groups in (3, 8, 1):
        m.slot_groups = groups
        for b in batches:
            b[3].zero_()
        m.reweight(batches, pts)
        torch.cuda.synchronize()
        for (proc, *_), b, ref in zip(items, batches, single):
            assert np.max(np.abs(b[3].cpu().numpy() / ref - 1.0)) < 1e-13, (proc, groups)
    with pytest.raises(rex.RexError):
        m.slot_groups = 0
    with pytest.raises(rex.RexError):
        m.slot_groups = 17
    ms = m.autotune(batches, pts)
    assert len(ms) == 6 and all(t > 0 for t in ms)
    assert m.slot_groups == (1, 2, 3, 4, 6, 8)[int(np.argmin(ms))]
    m.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_measured_tile_costs_order_the_launch(rex, precision, tmp_path):
    """rex_multi_autotune measures one tile's time per tile kind (seven batches, six
    kinds: the crossed q g channel has a tile of its own) and the persistent launch
    then hands out its items by those costs.  The order changes no weight: estimated,
    measured and reversed costs give bitwise the same outputs.  The tuning cache
    stores the costs and restores them into a new handle without timing."""
    from paper_2510_05100_b300 import tune_cache
    pts = points(16)
    items = setup(rex, precision, seed=23)
    for proc, n in (("qq_ttxg", 77), ("qg_ttxq", 45)):
        p = rex.Process(proc, precision)
        p.set_params(ORIG_QCD)
        items.append((proc, p, ps.make_events(proc, n, 300 + n), np.random.default_rng(n).uniform(0.5, 2.0, n)))
    batches = [(p, dev(mom), dev(w), torch.zeros((mom.shape[0], len(pts)), dtype=torch.float64, device="cuda"))
               for _, p, mom, w in items]
    m = rex.Multi(precision)
    assert all(m.tile_cost(b[0]) == 0.0 for b in batches)

    def run(handle):
        for b in batches:
            b[3].zero_()
        handle.reweight(batches, pts)
        torch.cuda.synchronize()
        return [b[3].cpu().numpy().copy() for b in batches]

    estimated = run(m)
    m.autotune(batches, pts)
    cost = {name: m.tile_cost(b[0]) for (name, *_), b in zip(items, batches)}
    assert all(c > 0 for c in cost.values()), cost
    assert cost["gg_ttxgg"] > cost["gg_ttxg"] > cost["gg_ttx"], cost
    m.slot_groups = 1
    measured = run(m)
    for (name, *_), b in zip(items, batches):
        m.set_tile_cost(b[0], 1.0 / cost[name])          # the opposite order
    reversed_ = run(m)
    for a, b, c in zip(estimated, measured, reversed_):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    m.set_tile_cost(batches[0][0], 0.0)
    assert m.tile_cost(batches[0][0]) == 0.0
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(rex.RexError):
            m.set_tile_cost(batches[0][0], bad)
    m.close()

    path = str(tmp_path / "tune.json")
    m1 = rex.Multi(precision)
    e1 = tune_cache.autotune_multi(m1, batches, pts, path)
    m2 = rex.Multi(precision)
    e2 = tune_cache.autotune_multi(m2, batches, pts, path)
    assert not e1["cached"] and e2["cached"] and m2.slot_groups == m1.slot_groups
    for b in batches:
        assert m2.tile_cost(b[0]) == m1.tile_cost(b[0]) > 0
    m1.close()
    m2.close()
    for _, p, *_ in items:
        p.close()
