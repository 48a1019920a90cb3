"""q q~ -> t t~ from its one Feynman diagram (oracle; test infrastructure only).

The quark-initiated leading-order channel of p p -> t t~; with g g -> t t~ it
forms a multi-channel sample of the kind the runtime comparison reweights
(Sec. 4.2, where p may be any massless QCD parton): a massless light quark q(1)
and antiquark q~(2) annihilate
into an s-channel gluon that makes the top pair t(3) t~(4).  Feynman rules as
in the g g -> t t~ (+ n g) oracle (Peskin & Schroeder Fig. 16.7, Feynman gauge):

    M = [vbar(p2) (i g gamma^mu t^a) u(p1)] (-i g_{mu nu} / s) [ubar(p3) (i g gamma^nu t^a) v(p4)],
    s = (p1 + p2)^2.

The kinematic part L_h = J_in(h) . J_out(h) (Minkowski product of the two
fermion currents) is evaluated with explicit 4x4 Dirac matrices for each of the
16 helicity configurations h; the colour factor is the explicit sum over every
colour index of |sum_a t^a_{j i} t^a_{k l}|^2.  Then

    sum |M|^2 = g^4 / s^2 * C * sum_h |L_h|^2,

averaged by 1/4 (quark spins) and 1/9 (quark colours).  The top width enters
no propagator of this diagram and is ignored.  The top spinors take the mass of
the parameter point on the kept momenta (the on-shell projection of the
Lorentz module).

Particle order in the momentum array: q(1) q~(2) t(3) t~(4), the incoming pair
with their physical (incoming) momenta.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .colour import T
from .lorentz import GAMMA, bar, mdot, spinor_u, spinor_v


def colour_factor() -> float:
    """sum over i, j, k, l of |sum_a t^a_{j i} t^a_{k l}|^2 (q colour i, q~ j, t k, t~ l)."""
    amp = np.einsum("aji,akl->ijkl", T, T)
    return float(np.real(np.sum(amp * amp.conj())))


def _current(left: np.ndarray, right: np.ndarray) -> np.ndarray:
    """left-bar gamma^mu right for row spinors left (already barred) and column right: [N, 4]."""
    return np.einsum("ni,mij,nj->nm", left, GAMMA, right)


def amplitudes(p: np.ndarray, mt: float) -> np.ndarray:
    """L_h = J_in . J_out for the 16 helicity configurations (l1, l2, l3, l4), [N, 16] complex."""
    p = np.asarray(p, dtype=np.float64)
    out = []
    for l1, l2, l3, l4 in itertools.product((-1, 1), repeat=4):
        j_in = _current(bar(spinor_v(p[:, 1], 0.0, l2)), spinor_u(p[:, 0], 0.0, l1))
        j_out = _current(bar(spinor_u(p[:, 2], mt, l3)), spinor_v(p[:, 3], mt, l4))
        out.append(mdot(j_in, j_out))
    return np.stack(out, axis=1)


def me2_helicity(p: np.ndarray, mt: float, wt: float, alphas: float, hel: np.ndarray) -> np.ndarray:
    """The term of the helicity sum (me2 = sum over configurations) of each event's own
    configuration hel[N, 4] = (l1, l2, l3, l4), helicities +1/-1 of q, q~, t, t~ in the
    frame of the momenta (wt unused)."""
    del wt
    p = np.asarray(p, dtype=np.float64)
    hel = np.asarray(hel)
    g2 = 4.0 * math.pi * alphas
    q = p[:, 0] + p[:, 1]
    s = mdot(q, q)
    amps = amplitudes(p, mt)   # [N, 16] in itertools.product((-1, 1), repeat=4) order
    out = np.zeros(p.shape[0])
    for i, conf in enumerate(itertools.product((-1, 1), repeat=4)):
        sel = np.all(hel == np.array(conf), axis=1)
        out[sel] = (g2 * g2 * colour_factor() * np.abs(amps[sel, i]) ** 2 / (s[sel] * s[sel]) / 36.0)
    return out


def me2(p: np.ndarray, mt: float, wt: float, alphas: float) -> np.ndarray:
    """Spin/colour summed and averaged |M|^2 for q q~ -> t t~, one point (wt unused)."""
    del wt
    p = np.asarray(p, dtype=np.float64)
    if p.ndim != 3 or p.shape[1] != 4:
        raise ValueError("q q~ -> t t~ expects momenta [N, 4, 4]")
    g2 = 4.0 * math.pi * alphas
    q = p[:, 0] + p[:, 1]
    s = mdot(q, q)
    amps = amplitudes(p, mt)
    hsum = np.sum(np.abs(amps) ** 2, axis=1)
    return g2 * g2 * colour_factor() * hsum / (s * s) / 36.0
