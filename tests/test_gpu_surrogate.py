"""Surrogate MLP kernels vs the FP64 oracle MLP, training, and the exact fallback (needs a B300).

BF16 tolerance: the GPU keeps weights W1..W4 and every activation and gradient
between layers in BF16 (8-bit mantissa, unit roundoff 2^-9) and accumulates in
FP32.  Against the FP64 oracle evaluated on the same BF16-rounded weights and
features, the loss agrees to 2e-2 and each layer's gradient to 5e-2 relative
(L2 norm).  Against a reference that rounds at the same points as the kernels
the agreement is 1e-2 on every gradient block.
"""
import math
import time

import numpy as np
import pytest

from rexlib import ensure_built
from oracle import mlp
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORIG = dict(mt=173.0, wt=0.0, alphas=0.118)


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def bf16(x):
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((a >> 16) & 1) + np.uint32(0x7FFF)
    return ((a + r) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)


def to_flat(params):
    """Oracle [(W, b)] (W1 22 x 256) -> the library's flat layout (W1 padded to 32 rows)."""
    parts = []
    for i, (w, b) in enumerate(params):
        if i == 0:
            w = np.vstack([w, np.zeros((32 - w.shape[0], w.shape[1]))])
        parts += [w.reshape(-1), b]
    return np.concatenate(parts).astype(np.float32)


def from_flat(flat):
    out, o = [], 0
    for rows, cols in ((32, 256), (256, 256), (256, 256), (256, 256), (256, 2)):
        w = flat[o:o + rows * cols].reshape(rows, cols).astype(np.float64)
        o += rows * cols
        b = flat[o:o + cols].astype(np.float64)
        o += cols
        out.append([w[:22] if rows == 32 else w, b])
    return out


def sample_inputs(n, seed):
    g = np.random.default_rng(seed)
    mom = ps.make_events("gg_ttxg", n, seed)
    mt = g.uniform(170.0, 176.0, n)
    al = g.uniform(0.110, 0.126, n)
    ratio = np.exp(g.normal(0.0, 0.2, n))
    return mom, mt, al, ratio


def emulated_loss_grad(params, x, t):
    """The kernels' arithmetic in numpy: BF16 inputs, weights W1..W4, activations and
    gradients between layers; FP32-like accumulation (done in FP64 here)."""
    hs, zs = [bf16(x)], []
    for i, (w, b) in enumerate(params[:4]):
        z = hs[-1] @ bf16(w) + b
        zs.append(z)
        hs.append(bf16(mlp.gelu(z)))
    out = hs[-1] @ params[4][0] + params[4][1]
    n = x.shape[0]
    res = out[:, 0] - t
    tgt = np.abs(res)
    loss = np.mean(res * res + (out[:, 1] - tgt) ** 2)
    dout = np.stack([2 * res / n, 2 * (out[:, 1] - tgt) / n], axis=1)
    grads = [None] * 5
    grads[4] = [hs[4].T @ dout, dout.sum(0)]
    dz = bf16((dout @ params[4][0].T) * mlp.gelu_grad(zs[3]))
    for i in range(3, -1, -1):
        grads[i] = [hs[i].T @ dz, dz.sum(0)]
        if i > 0:
            dz = bf16((dz @ bf16(params[i][0]).T) * mlp.gelu_grad(zs[i - 1]))
    return loss, grads


@pytest.mark.parametrize("power", [0, 3])
def test_loss_and_gradients_match_the_oracle(rex, power):
    n = 256
    mom, mt, al, ratio = sample_inputs(n, 5)
    params = mlp.init_params(7)
    for i in range(4):                       # make W1..W4 exactly representable in BF16
        params[i][0] = bf16(params[i][0])
    s = rex.Surrogate(0)
    s.set_exact_alphas(0.118, power)
    s.set_weights(to_flat(params))
    loss_gpu, g_gpu = s.loss_grad(torch.from_numpy(mom).cuda(), torch.from_numpy(ratio).cuda(),
                                  torch.from_numpy(mt).cuda(), torch.from_numpy(al).cuda())
    x = bf16(mlp.features(mom, mt, al))
    t = mlp.target(ratio, al, 0.118, power).astype(np.float32).astype(np.float64)
    loss_ref, g_ref = mlp.loss_and_grad(params, x, t)
    loss_emu, g_emu = emulated_loss_grad(params, x, t)
    gg = from_flat(g_gpu)
    assert abs(loss_gpu / loss_ref - 1) < 2e-2
    assert abs(loss_gpu / loss_emu - 1) < 1e-3
    for i in range(5):
        for j in range(2):
            a, r, e = gg[i][j], g_ref[i][j], g_emu[i][j]
            assert np.linalg.norm(a - r) / np.linalg.norm(r) < 5e-2, (i, j)
            assert np.linalg.norm(a - e) / np.linalg.norm(e) < 1e-2, (i, j)
    # padded rows of W1 get exactly zero gradient
    assert np.all(g_gpu[22 * 256:32 * 256] == 0.0)


@pytest.fixture(scope="module")
def trained(rex):
    """A surrogate trained on exact FP64 ratios of 8192 g g -> t t~ g events x 16 points."""
    pts = ps.grid_gg_ttxg()
    n = 8192
    mom = torch.from_numpy(ps.make_events("gg_ttxg", n, 31)).cuda()
    exact = rex.Process("gg_ttxg", 0)
    exact.set_params(ORIG)
    ratio = exact.reweight(mom, torch.ones(n, dtype=torch.float64, device="cuda"), pts)
    s = rex.Surrogate(1)
    s.set_exact_alphas(0.118, 3)             # |M|^2 ~ alphas^3: the network learns the mt part
    losses = s.train(mom, ratio, pts, steps=600, batch=4096, lr=1e-3, seed=3)
    return s, exact, pts, losses


def test_training_reduces_the_loss(rex, trained):
    s, _, _, losses = trained
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()


@pytest.mark.parametrize("kernel", ["fused", "layered"])
def test_inference_matches_the_oracle_forward(rex, trained, kernel):
    s, _, pts, _ = trained
    s.set_kernel(rex.SURROGATE_FUSED if kernel == "fused" else rex.SURROGATE_LAYERED)
    n = 64
    mom = ps.make_events("gg_ttxg", n, 77)
    pred = torch.empty((n, len(pts)), dtype=torch.float32, device="cuda")
    errp = torch.empty((n, len(pts)), dtype=torch.float32, device="cuda")
    s.reweight(torch.from_numpy(mom).cuda(), None, pts, pred=pred, err=errp)
    params = from_flat(s.get_weights())
    for i in range(4):
        params[i][0] = bf16(params[i][0])
    mt = np.array([p["mt"] for p in pts])
    al = np.array([p["alphas"] for p in pts])
    x = bf16(mlp.features(np.repeat(mom, len(pts), axis=0), np.tile(mt, n), np.tile(al, n)))
    out, _ = mlp.forward(params, x)
    ref = out[:, 0].reshape(n, len(pts)) + mlp.coupling_part(al, 0.118, 3)[None, :]
    scale = np.abs(ref).max() + 1e-3
    assert np.max(np.abs(pred.cpu().numpy() - ref)) < 2e-2 * scale + 2e-3
    s.set_kernel(rex.SURROGATE_FUSED)


@pytest.mark.parametrize("n,k", [(1, 1), (37, 5), (300, 16), (20011, 16)])
def test_fused_and_layered_kernels_agree(rex, trained, n, k):
    """The tcgen05 kernel against the layer-by-layer one on ragged tile counts (n k
    not a multiple of 128), a single partial tile, and more tiles than SMs.  Both
    round activations to BF16, so a rounding flip of an activation may differ
    between the two FP32 summation orders; the bound is a few BF16 ulps of the
    output's scale."""
    s, _, _, _ = trained
    g = np.random.default_rng(n)
    pts = [dict(mt=float(m), wt=0.0, alphas=float(a))
           for m, a in zip(g.uniform(170.0, 176.0, k), g.uniform(0.110, 0.126, k))]
    mom = torch.from_numpy(ps.make_events("gg_ttxg", n, 1000 + n)).cuda()
    w = torch.from_numpy(g.uniform(0.5, 2.0, n)).cuda()
    outs = {}
    for kind in (rex.SURROGATE_FUSED, rex.SURROGATE_LAYERED):
        s.set_kernel(kind)
        pred = torch.full((n, k), float("nan"), dtype=torch.float32, device="cuda")
        err = torch.full((n, k), float("nan"), dtype=torch.float32, device="cuda")
        w_out = torch.full((n, k), float("nan"), dtype=torch.float64, device="cuda")
        s.reweight(mom, w, pts, tau=float("inf"), w_out=w_out, pred=pred, err=err)
        outs[kind] = (pred, err, w_out)
    s.set_kernel(rex.SURROGATE_FUSED)
    (pf, ef, wf), (pl, el, wl) = outs[rex.SURROGATE_FUSED], outs[rex.SURROGATE_LAYERED]
    for a in (pf, ef, wf):
        assert torch.isfinite(a).all()
    scale = float(pl.abs().max()) + 1e-2
    assert float((pf - pl).abs().max()) < 2e-2 * scale
    assert float((ef - el).abs().max()) < 2e-2 * (float(el.abs().max()) + 1e-2)
    assert torch.allclose(wf, w[:, None] * torch.exp(pf.double()), rtol=1e-6, atol=0)   # exp in FP32


def test_fallback_extremes(rex, trained):
    s, exact, pts, _ = trained
    n = 300
    mom = torch.from_numpy(ps.make_events("gg_ttxg", n, 88)).cuda()
    w = torch.from_numpy(np.random.default_rng(2).uniform(0.5, 2.0, n)).cuda()
    ref = exact.reweight(mom, w, pts)
    out = torch.empty_like(ref)
    nfb = s.reweight(mom, w, pts, tau=-1.0, exact=exact, w_out=out)      # every event falls back
    assert nfb == n and torch.equal(out, ref)
    pred = torch.empty((n, len(pts)), dtype=torch.float32, device="cuda")
    nfb = s.reweight(mom, w, pts, tau=float("inf"), exact=exact, w_out=out, pred=pred)
    assert nfb == 0
    assert torch.allclose(out, w[:, None] * torch.exp(pred.double()), rtol=1e-6, atol=0)   # exp in FP32


def test_what_the_surrogate_gains_over_the_exact_path(rex, trained):
    """What the trained network buys against the method without it, on the same
    events and points: the network alone (fused tcgen05 kernel) must beat the exact
    FP64 kernel, and the fallback bookkeeping must hold (flagged events exact).
    The exact mixed-precision kernel is timed beside them for the record: on B300
    it stays faster than the 4 x 256 network (about 4e5 tensor flops per pair
    against about 1e4 FP32 flops for the exact g g -> t t~ g amplitudes)."""
    s, exact, pts, _ = trained
    n = 1 << 15
    mom = torch.from_numpy(ps.make_events("gg_ttxg", n, 99)).cuda()
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    ref = exact.reweight(mom, w, pts)
    mixed = rex.Process("gg_ttxg", 1)
    mixed.set_params(ORIG)
    out = torch.empty_like(ref)
    errp = torch.empty((n, len(pts)), dtype=torch.float32, device="cuda")
    tau = 0.02
    nfb = s.reweight(mom, w, pts, tau=tau, exact=exact, w_out=out, err=errp)
    rel = (out / ref - 1).abs()
    flagged_ev = (errp > tau).any(dim=1)
    assert nfb == int(flagged_ev.sum())
    assert torch.all(rel[flagged_ev] == 0)                   # fallback rows are exact
    torch.cuda.synchronize()

    def clock(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / 3

    t_net = clock(lambda: s.reweight(mom, w, pts, tau=float("inf"), w_out=out))
    t_fp64 = clock(lambda: exact.reweight(mom, w, pts, w_out=out))
    t_fb = clock(lambda: s.reweight(mom, w, pts, tau=tau, exact=exact, w_out=out))
    t_mix = clock(lambda: mixed.reweight(mom, w, pts))
    print(f"\nnetwork only: {t_net * 1e3:.2f} ms, with fallback (tau {tau}): {t_fb * 1e3:.2f} ms, "
          f"exact FP64: {t_fp64 * 1e3:.2f} ms, exact mixed: {t_mix * 1e3:.2f} ms; "
          f"fallback {nfb}/{n} events, max rel err {float(rel.max()):.3e}, median {float(rel.median()):.3e}")
    assert t_net < t_fp64


def soft_collinear_y(mom):
    """The guard variable, written out here: min over i in {1, 2, t, t~} of 2 k.p_i / s_hat."""
    def dot(a, b):
        return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)
    shat = dot(mom[:, 0] + mom[:, 1], mom[:, 0] + mom[:, 1])
    return 2.0 * np.min(np.stack([dot(mom[:, 4], mom[:, i]) for i in range(4)]), axis=0) / shat


def test_calibrated_fallback_holds_the_stated_bound_on_held_out_events(rex, trained):
    """The stated error bound of the surrogate: calibrated on one held-out set (tau on the
    error head and the soft/collinear guard, at most 5e-4 of the kept pairs off by more
    than the bound in |log w|), it keeps the escape rate of the pairs it does not send
    back to the exact path at or below 1e-3 on an independent held-out seed, measured
    against the FP64 kernel; every fallback row is exact."""
    _, exact, pts, _ = trained
    # a network trained as far as the bound needs (65536 events x 16 points, 4000 steps:
    # a few seconds); the module's small fixture network would send every event back
    n_tr = 1 << 16
    mom_tr = torch.from_numpy(ps.make_events("gg_ttxg", n_tr, 4040)).cuda()
    ratio = exact.reweight(mom_tr, torch.ones(n_tr, dtype=torch.float64, device="cuda"), pts)
    s = rex.Surrogate(2)
    s.set_exact_alphas(0.118, 3)
    for steps, lr in ((2500, 1e-3), (1500, 3e-4)):
        s.train(mom_tr, ratio, pts, steps=steps, batch=8192, lr=lr, seed=5)
    bound = 3e-2
    n = 1 << 15
    mom_cal = torch.from_numpy(ps.make_events("gg_ttxg", n, 4141)).cuda()
    cal = s.calibrate(exact, mom_cal, pts, bound, 5e-4)
    assert cal["escape_rate"] <= 5e-4 and 0.0 <= cal["fallback_rate"] < 1.0, cal
    mom_np = ps.make_events("gg_ttxg", n, 4242)
    mom = torch.from_numpy(mom_np).cuda()
    w = torch.from_numpy(np.random.default_rng(3).uniform(0.5, 2.0, n)).cuda()
    ref = exact.reweight(mom, w, pts)
    out = torch.empty_like(ref)
    errp = torch.empty((n, len(pts)), dtype=torch.float32, device="cuda")
    nfb = s.reweight(mom, w, pts, tau=cal["tau"], exact=exact, w_out=out, err=errp)
    flagged = (errp > cal["tau"]).any(dim=1).cpu().numpy() | ~(soft_collinear_y(mom_np) >= cal["guard"])
    assert nfb == int(flagged.sum())
    dlog = (out / ref).log().abs().cpu().numpy()
    assert np.all(dlog[flagged] == 0.0)                       # fallback rows are the exact ones
    kept = dlog[~flagged]
    escape = float((kept > bound).mean())
    print(f"\ncalibration: tau {cal['tau']:.4g}, guard {cal['guard']:.4g}, fallback {cal['fallback_rate']:.3f}; "
          f"held-out: fallback {nfb / n:.3f}, escape {escape:.2e}, max kept {kept.max():.3g}")
    assert kept.size > 0 and escape <= 1e-3
    s.close()


def test_guard_validation(rex, trained):
    s = trained[0]
    with pytest.raises(rex.RexError):
        s.set_guard(-0.1)
    with pytest.raises(rex.RexError):
        s.set_guard(1.0)
    s.set_guard(0.0)


def test_save_and_load_round_trip(rex, trained, tmp_path):
    """A saved network loads into a fresh handle with identical weights, coupling
    setting and predictions; a foreign file is refused."""
    s, _, pts, _ = trained
    path = str(tmp_path / "net.bin")
    s.save(path)
    t = rex.Surrogate(99)
    t.load(path)
    assert np.array_equal(t.get_weights(), s.get_weights())
    mom = torch.from_numpy(ps.make_events("gg_ttxg", 64, 5)).cuda()
    a = torch.empty((64, len(pts)), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    s.reweight(mom, None, pts, pred=a)
    t.reweight(mom, None, pts, pred=b)
    assert torch.equal(a, b)
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(b"not a network")
    with pytest.raises(rex.RexError):
        t.load(bad)
    t.close()
