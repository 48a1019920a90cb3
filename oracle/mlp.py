"""FP64 reference MLP for the reweighting surrogate (oracle; test infrastructure).

The surrogate predicts r = log(|M(p; theta)|^2 / |M(p; theta_0)|^2) for an event p
and a parameter point theta, plus an estimate of its own absolute error.  The
paper has no learned component; this is the plain definition that the GPU
training and inference kernels are checked against:

    x  = [features(p) (20), features(theta) (2)]                       (22)
    h1 = gelu(x  W1 + b1)        W1: 22 x 256
    h2 = gelu(h1 W2 + b2)        W2: 256 x 256
    h3 = gelu(h2 W3 + b3)
    h4 = gelu(h3 W4 + b4)
    [y, e] = h4 W5 + b5          W5: 256 x 2   (prediction, error estimate)

gelu(z) = z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2: the tanh form of the
Gaussian error linear unit (Hendrycks & Gimpel 2016), which stays within 4.8e-4
of z Phi(z).  The GPU kernels evaluate tanh with the hardware approximation.

Loss of a batch of n samples with targets t:
    L = 1/n sum_i [ (y_i - t_i)^2 + (e_i - |y_i - t_i|)^2 ],
where the error head's target |y_i - t_i| is treated as a constant (no gradient
flows from the second term into y).

Exact coupling part (optional): tree-level |M|^2 is proportional to alphas^n
(n = 3 for g g -> t t~ g), so log r = n log(alphas / alphas0) + f(p, mt).  With
n > 0 the network's target is t = log r - n log(alphas / alphas0), and the
prediction of log r is y + n log(alphas / alphas0).

Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
theta <- theta - lr (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps).
"""
from __future__ import annotations

import math

import numpy as np

WIDTH = 256
NLAYER = 4          # hidden layers
NIN = 22
NOUT = 2


GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    """d gelu / dz = (1 + t)/2 + z (1 - t^2) sqrt(2/pi) (1 + 3 a z^2) / 2, t = tanh(u(z))."""
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def init_params(seed: int = 0, nin: int = NIN, width: int = WIDTH, nlayer: int = NLAYER, nout: int = NOUT):
    """He-normal weights, zero biases; list of (W, b) for nlayer hidden layers + head."""
    g = np.random.Generator(np.random.PCG64(seed))
    dims = [nin] + [width] * nlayer + [nout]
    params = []
    for a, b in zip(dims[:-1], dims[1:]):
        params.append([g.normal(0.0, math.sqrt(2.0 / a), (a, b)), np.zeros(b)])
    return params


def forward(params, x):
    """Returns (outputs [n, 2], cache of (input, pre-activation) per layer)."""
    cache = []
    h = x
    for i, (w, b) in enumerate(params):
        z = h @ w + b
        cache.append((h, z))
        h = gelu(z) if i < len(params) - 1 else z
    return h, cache


def loss_and_grad(params, x, t, err_target=None):
    """Mean loss and its gradient with respect to every (W, b).

    err_target: the error head's target; None means |y - t| of this forward pass,
    held constant (stop-gradient) in the derivative."""
    out, cache = forward(params, x)
    n = x.shape[0]
    y, e = out[:, 0], out[:, 1]
    res = y - t
    tgt_e = np.abs(res) if err_target is None else err_target
    loss = float(np.mean(res * res + (e - tgt_e) ** 2))
    dout = np.zeros_like(out)
    dout[:, 0] = 2.0 * res / n
    dout[:, 1] = 2.0 * (e - tgt_e) / n
    grads = [None] * len(params)
    d = dout
    for i in range(len(params) - 1, -1, -1):
        h, z = cache[i]
        if i < len(params) - 1:
            d = d * gelu_grad(z)
        grads[i] = [h.T @ d, d.sum(axis=0)]
        d = d @ params[i][0].T
    return loss, grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
        self.v = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
        self.step = 0

    def update(self, params, grads):
        self.step += 1
        c1 = 1.0 - self.b1 ** self.step
        c2 = 1.0 - self.b2 ** self.step
        for p, g, m, v in zip(params, grads, self.m, self.v):
            for i in range(2):
                m[i] = self.b1 * m[i] + (1.0 - self.b1) * g[i]
                v[i] = self.b2 * v[i] + (1.0 - self.b2) * g[i] * g[i]
                p[i] = p[i] - self.lr * (m[i] / c1) / (np.sqrt(v[i] / c2) + self.eps)


# ---------------------------------------------------------------------------
# input features (fixed affine maps; shared definition with the GPU kernels'
# feature step is by specification, not by code)
# ---------------------------------------------------------------------------
MOM_SCALE = 1.0e-3          # GeV -> TeV
MT_REF, MT_SCALE = 173.0, 1.0 / 3.0
AS_REF, AS_SCALE = 0.118, 1.0 / 0.008


def features(p: np.ndarray, mt: np.ndarray, alphas: np.ndarray) -> np.ndarray:
    """[n, 22]: the 20 momentum components (E, px, py, pz of 5 particles) in TeV,
    (mt - 173)/3, (alphas - 0.118)/0.008."""
    n = p.shape[0]
    x = np.empty((n, NIN))
    x[:, :20] = p.reshape(n, 20) * MOM_SCALE
    x[:, 20] = (np.asarray(mt) - MT_REF) * MT_SCALE
    x[:, 21] = (np.asarray(alphas) - AS_REF) * AS_SCALE
    return x


def coupling_part(alphas, alphas0: float, power: int):
    """n log(alphas / alphas0): the exact alphas dependence of the log ratio."""
    return power * np.log(np.asarray(alphas, dtype=np.float64) / alphas0)


def target(ratio, alphas, alphas0: float = 0.118, power: int = 0):
    """Training target: log(ratio) minus the exact coupling part."""
    return np.log(np.asarray(ratio, dtype=np.float64)) - coupling_part(alphas, alphas0, power)
