"""The FP64 surrogate MLP oracle against independent checks (CPU)."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_values_and_derivative():
    z = np.linspace(-8.0, 8.0, 4001)
    g = mlp.gelu(z)
    # the tanh form stays within 4.8e-4 of the exact z Phi(z) (Hendrycks & Gimpel)
    assert np.max(np.abs(g - z * norm.cdf(z))) < 4.8e-4
    # tanh is odd: gelu(z) - gelu(-z) = z; gelu(0) = 0; saturation at both ends
    assert np.allclose(g - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([20.0]))[0] - 20.0) < 1e-12 and abs(mlp.gelu(np.array([-20.0]))[0]) < 1e-12
    h = 1e-6
    zz = np.array([-3.0, -1.0, 0.0, 0.5, 2.0, 6.0])
    fd = (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(zz), fd, rtol=1e-8, atol=1e-10)
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5


def _small():
    p = mlp.init_params(3, nin=5, width=7, nlayer=2, nout=2)
    g = np.random.default_rng(4)
    x = g.normal(size=(9, 5))
    t = g.normal(size=9)
    return p, x, t


def test_gradients_match_central_finite_differences():
    """The error head's target is a stop-gradient: freeze it at the base point."""
    params, x, t = _small()
    out, _ = mlp.forward(params, x)
    frozen = np.abs(out[:, 0] - t)
    _, grads = mlp.loss_and_grad(params, x, t, frozen)
    _, grads_default = mlp.loss_and_grad(params, x, t)
    for a, b in zip(grads, grads_default):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    h = 1e-6
    worst = 0.0
    for li, (w, b) in enumerate(params):
        for arr, garr in ((w, grads[li][0]), (b, grads[li][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = mlp.loss_and_grad(params, x, t, frozen)
                arr[idx] = old - h
                lm, _ = mlp.loss_and_grad(params, x, t, frozen)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                scale = max(abs(fd), abs(garr[idx]), 1e-8)
                worst = max(worst, abs(fd - garr[idx]) / scale)
    assert worst < 1e-6


def test_forward_is_the_layer_composition():
    params, x, _ = _small()
    out, _ = mlp.forward(params, x)
    h = x
    for w, b in params[:-1]:
        z = h @ w + b
        # (1 + tanh(u)) / 2 = 1 / (1 + exp(-2u)): the tanh-form GELU as z times a logistic
        h = z / (1.0 + np.exp(-2.0 * math.sqrt(2.0 / math.pi) * (z + 0.044715 * z ** 3)))
    ref = h @ params[-1][0] + params[-1][1]
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-14)


def test_adam_first_step_is_lr_times_sign():
    """After one step from zero moments, Adam moves every parameter by lr * g/(|g| + eps')."""
    params = [[np.array([[1.0, -2.0]]), np.array([0.5, 0.0])]]
    grads = [[np.array([[0.3, -0.01]]), np.array([-4.0, 0.0])]]
    opt = mlp.Adam(params, lr=0.01)
    opt.update(params, grads)
    assert np.allclose(params[0][0], [[1.0 - 0.01, -2.0 + 0.01]], rtol=1e-9)
    assert np.allclose(params[0][1], [0.5 + 0.01, 0.0], rtol=1e-9)


def test_training_reduces_loss_on_a_smooth_target():
    g = np.random.default_rng(0)
    x = g.uniform(-1, 1, (256, 4))
    t = np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2]
    params = mlp.init_params(1, nin=4, width=32, nlayer=2, nout=2)
    opt = mlp.Adam(params, lr=3e-3)
    l0, _ = mlp.loss_and_grad(params, x, t)
    for _ in range(300):
        l, gr = mlp.loss_and_grad(params, x, t)
        opt.update(params, gr)
    assert l < 0.1 * l0


def test_features_layout():
    p = np.arange(2 * 5 * 4, dtype=float).reshape(2, 5, 4) * 100.0
    x = mlp.features(p, np.array([173.0, 176.0]), np.array([0.118, 0.126]))
    assert x.shape == (2, 22)
    assert np.allclose(x[1, :20], p[1].reshape(20) * 1e-3)
    assert np.allclose(x[:, 20], [0.0, 1.0]) and np.allclose(x[:, 21], [0.0, 1.0])


def test_coupling_part_removes_the_exact_alphas_dependence():
    """With the coupling part removed, the target of an alphas-only reweighting is
    zero: the oracle's |M|^2 scales exactly as alphas^3 for g g -> t t~ g."""
    from oracle import reweight
    from paper_2510_05100_b300 import phase_space as ps
    p = ps.make_events("gg_ttxg", 3, 12)
    orig = dict(mt=173.0, wt=0.0, alphas=0.118)
    pts = [dict(mt=173.0, wt=0.0, alphas=a) for a in (0.110, 0.121, 0.126)]
    r = reweight.reweight("gg_ttxg", p, np.ones(3), orig, pts)
    al = np.array([q["alphas"] for q in pts])[None, :]
    t = mlp.target(r, al, 0.118, 3)
    assert np.max(np.abs(t)) < 1e-13
    # the full log ratio is recovered by adding the part back
    assert np.allclose(t + mlp.coupling_part(al, 0.118, 3), np.log(r), rtol=0, atol=1e-15)
    # power 0 leaves the target as log(ratio)
    assert np.array_equal(mlp.target(r, al, 0.118, 0), np.log(r))
