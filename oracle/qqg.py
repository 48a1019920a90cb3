"""q q~ -> t t~ g from its five Feynman diagrams (oracle; test infrastructure only).

The quark-initiated p p -> t t~ + jet channel (the runtime comparison of Sec. 4.2
reweights samples with up to one jet of any massless QCD parton).  Particles:
q(1) q~(2) in (physical momenta), t(3) t~(4) g(5) out.  Feynman rules as in the
other QCD oracles (Peskin & Schroeder Fig. 16.7, Feynman gauge): vertex
i g gamma^mu t^a, quark propagator i (q-slash + m) / (q^2 - m^2), gluon propagator
-i g_{mu nu} delta^{ab} / q^2, three-gluon vertex
g f^{abc} [g^{mu nu}(k - p)^rho + g^{nu rho}(p - q)^mu + g^{rho mu}(q - k)^nu] with
every momentum flowing into the vertex.

With s = (p1 + p2)^2 and s' = (p3 + p4)^2 the diagrams are, light line read from
vbar(p2) to u(p1), top line from ubar(p3) to v(p4):
  D1 gluon off the quark:    vbar2 (g gamma^mu t^b) S(p1 - k) (g eps* t^a) u1 . G(s') . ubar3 (g gamma_mu t^b) v4
  D2 gluon off the antiquark: vbar2 (g eps* t^a) S(k - p2) (g gamma^mu t^b) u1 . G(s') . ubar3 (...) v4
  D3 gluon off the top:      vbar2 (g gamma^mu t^b) u1 . G(s) . ubar3 (g eps* t^a) S(p3 + k) (g gamma_mu t^b) v4
  D4 gluon off the antitop:  ... ubar3 (g gamma_mu t^b) S(-p4 - k) (g eps* t^a) v4
  D5 three-gluon vertex:     J_in^mu G(s) V_{mu rho nu}(q, -k, -q') eps*^rho G(s') J_out^nu, colour f^{bac}
(each vertex carrying its factor i and each propagator its i or -i).  Colour
tensors K_d[a, i1, j2, i3, j4] are built from t^a and f^abc; the colour sum is
sum_{d,d'} conj(A_d) G_dd' A_d' with G = conj(K) K^T over every index.  Summed over
the 32 helicity configurations, averaged by 1/4 (spins) and 1/9 (quark colours).
Top spinors follow the Lorentz module's mass convention; the width enters the top
propagators as q^2 - m^2 + i m Gamma.

The crossed channels with one light quark line (q g -> t t~ q, q~ g -> t t~ q~, the
beam-swapped g q, g q~ and q~ q) are the same five diagrams with each external
state's own wavefunction and the momenta along the fermion-number flow
(CROSSINGS, amplitudes_crossed); the colour sum is the same, the average 1/96 for
q g (1/4 spins, 1/3 quark and 1/8 gluon colours).
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np

from .colour import F, T
from .lorentz import GAMMA, bar, mdot, polarisation, slash, spinor_u, spinor_v


@functools.lru_cache(maxsize=None)
def colour_tensors() -> np.ndarray:
    """K[d, a, i1, j2, i3, j4] for the five diagrams."""
    tt = np.einsum("bij,ajk->baik", T, T)      # (t^b t^a)_{ik}
    k1 = np.einsum("bajk,blm->akjlm", tt, T)   # (t^b t^a)_{j2 i1} (t^b)_{i3 j4}
    k2 = np.einsum("abjk,blm->akjlm", tt, T)   # (t^a t^b)_{j2 i1} (t^b)_{i3 j4}
    k3 = np.einsum("bjk,ablm->akjlm", T, tt)   # (t^b)_{j2 i1} (t^a t^b)_{i3 j4}
    k4 = np.einsum("bjk,balm->akjlm", T, tt)   # (t^b)_{j2 i1} (t^b t^a)_{i3 j4}
    k5 = np.einsum("bac,bjk,clm->akjlm", F, T, T)
    return np.stack([k1, k2, k3, k4, k5])


@functools.lru_cache(maxsize=None)
def colour_matrix() -> np.ndarray:
    k = colour_tensors().reshape(5, -1)
    return k.conj() @ k.T


def _real(p) -> np.ndarray:
    """Momenta as a real array: FP64, unless they are given in extended precision
    (np.longdouble), which is then kept through every step (a reference free of the
    FP64 evaluation's own rounding, for ill-conditioned events)."""
    p = np.asarray(p)
    return p if p.dtype == np.longdouble else p.astype(np.float64)


def _chain(left: np.ndarray, mats: list, right: np.ndarray) -> np.ndarray:
    """left-row . (product of [N,4,4] matrices) . right-column, [N]."""
    m = mats[0]
    for x in mats[1:]:
        m = np.einsum("nij,njk->nik", m, x)
    return np.einsum("ni,nij,nj->n", left, m, right)


def _vector_chain(left: np.ndarray, before: list, after: list, right: np.ndarray) -> np.ndarray:
    """left . B gamma^mu A . right for every mu (upper index), [N, 4]."""
    n = left.shape[0]
    eye = np.broadcast_to(np.eye(4, dtype=complex), (n, 4, 4))
    out = np.empty((n, 4), dtype=np.result_type(left, right, complex))
    for mu in range(4):
        g = np.broadcast_to(GAMMA[mu], (n, 4, 4))
        out[:, mu] = _chain(left, (before or [eye]) + [g] + (after or [eye]), right)
    return out


def _diagrams(q1, q2, p3, p4, k, left, right, ub3, v4, eps, mt, wt, alphas) -> np.ndarray:
    """The five diagram amplitudes [N, 5] of one light line read from the row spinor
    left to the column spinor right, momenta along the fermion-number flow: q1 enters
    the line at right, q2 at left, and the gluon leaves it with momentum k and vector
    eps (eps* of an outgoing gluon, eps of an incoming one with k = -its momentum)."""
    g = math.sqrt(4.0 * math.pi * alphas)
    n = left.shape[0]
    es = slash(eps)
    q = q1 + q2
    qp = p3 + p4
    s, sp = mdot(q, q), mdot(qp, qp)
    m1 = np.eye(4) * mt
    j_in = _vector_chain(left, [], [], right)
    j_out = _vector_chain(ub3, [], [], v4)
    # D1, D2: emission from the light line (massless propagators)
    a1 = q1 - k
    c1 = _vector_chain(left, [], [slash(a1), es], right) / mdot(a1, a1)[:, None]
    a2 = k - q2
    c2 = _vector_chain(left, [es, slash(a2)], [], right) / mdot(a2, a2)[:, None]
    # D3, D4: emission from the top line
    a3 = p3 + k
    d3 = mdot(a3, a3) - mt * mt + 1j * mt * wt
    c3 = _vector_chain(ub3, [es, slash(a3) + m1], [], v4) / d3[:, None]
    a4 = -p4 - k
    d4 = mdot(a4, a4) - mt * mt + 1j * mt * wt
    c4 = _vector_chain(ub3, [], [slash(a4) + m1, es], v4) / d4[:, None]
    cf = -1j * g ** 3        # (i g)^3 x i (fermion propagator) x (-i) (gluon propagator)
    amp = np.empty((n, 5), dtype=np.result_type(left, right, complex))
    amp[:, 0] = cf * mdot(c1, j_out) / sp
    amp[:, 1] = cf * mdot(c2, j_out) / sp
    amp[:, 2] = cf * mdot(j_in, c3) / s
    amp[:, 3] = cf * mdot(j_in, c4) / s
    # D5: (i g)^2 x g (vertex) x (-i)^2 (two gluon propagators) = g^3
    v = (mdot(j_in, eps) * mdot(q + k, j_out) + mdot(eps, j_out) * mdot(j_in, qp - k)
         - mdot(j_in, j_out) * mdot(eps, qp + q))
    amp[:, 4] = g ** 3 * v / (s * sp)
    return amp


def amplitudes(p: np.ndarray, mt: float, wt: float, alphas: float, hel: tuple, eps_override=None) -> np.ndarray:
    """The five diagram amplitudes [N, 5] of one helicity configuration
    hel = (l1, l2, l3, l4, lg); eps_override replaces the gluon's eps* (gauge checks)."""
    p = _real(p)
    l1, l2, l3, l4, lg = hel
    p1, p2, p3, p4, k = p[:, 0], p[:, 1], p[:, 2], p[:, 3], p[:, 4]
    eps = polarisation(k, lg).conj() if eps_override is None else eps_override.astype(complex)
    return _diagrams(p1, p2, p3, p4, k, bar(spinor_v(p2, 0.0, l2)), spinor_u(p1, 0.0, l1),
                     bar(spinor_u(p3, mt, l3)), spinor_v(p4, mt, l4), eps, mt, wt, alphas)


# The crossings of q q~ -> t t~ g into the other p p -> t t~ + jet channels with a
# light quark line.  Record order: the two incoming partons, t, t~, the outgoing
# parton.  Each entry: (indices of the incoming quark, incoming antiquark, outgoing
# quark, outgoing antiquark, incoming gluon, outgoing gluon; None where absent) and
# the spin-colour average (1/4 for the spins, 1/9 for a q q~ pair, 1/24 for q g).
CROSSINGS = {
    "qq_ttxg": ((0, 1, None, None, None, 4), 36.0),
    "qxq_ttxg": ((1, 0, None, None, None, 4), 36.0),
    "qg_ttxq": ((0, None, 4, None, 1, None), 96.0),
    "gq_ttxq": ((1, None, 4, None, 0, None), 96.0),
    "qxg_ttxqx": ((None, 0, None, 4, 1, None), 96.0),
    "gqx_ttxqx": ((None, 1, None, 4, 0, None), 96.0),
}


def amplitudes_crossed(process: str, p: np.ndarray, mt: float, wt: float, alphas: float, hel: tuple,
                       eps_override=None) -> np.ndarray:
    """The five diagram amplitudes [N, 5] of one channel of CROSSINGS from the Feynman
    rules of its own external states (Peskin & Schroeder Sec. 4.7): an incoming
    quark gives u, an outgoing quark ubar, an incoming antiquark vbar, an outgoing
    antiquark v, an outgoing gluon eps*, an incoming gluon eps.  hel: the helicities
    of the record's particles in record order.  The light line runs along the
    fermion-number flow from the quark entering the diagram (an incoming quark or
    an outgoing antiquark, momentum q1) to the one leaving it (momentum -q2)."""
    p = _real(p)
    (iq, iqb, oq, oqb, ig, og), _ = CROSSINGS[process]
    if iq is not None:
        right, q1 = spinor_u(p[:, iq], 0.0, hel[iq]), p[:, iq]
    else:
        right, q1 = spinor_v(p[:, oqb], 0.0, hel[oqb]), -p[:, oqb]
    if iqb is not None:
        left, q2 = bar(spinor_v(p[:, iqb], 0.0, hel[iqb])), p[:, iqb]
    else:
        left, q2 = bar(spinor_u(p[:, oq], 0.0, hel[oq])), -p[:, oq]
    if og is not None:
        k, eps = p[:, og], polarisation(p[:, og], hel[og]).conj()
    else:
        k, eps = -p[:, ig], polarisation(p[:, ig], hel[ig])
    if eps_override is not None:
        eps = eps_override.astype(complex)
    return _diagrams(q1, q2, p[:, 2], p[:, 3], k, left, right, bar(spinor_u(p[:, 2], mt, hel[2])),
                     spinor_v(p[:, 3], mt, hel[3]), eps, mt, wt, alphas)


def me2_crossed(process: str, p: np.ndarray, mt: float, wt: float, alphas: float) -> np.ndarray:
    """Spin/colour summed and averaged |M|^2 of one channel of CROSSINGS, one point."""
    p = _real(p)
    if p.ndim != 3 or p.shape[1] != 5:
        raise ValueError(f"{process} expects momenta [N, 5, 4]")
    gm = colour_matrix()
    total = np.zeros(p.shape[0], dtype=p.dtype)
    for hel in itertools.product((-1, 1), repeat=5):
        a = amplitudes_crossed(process, p, mt, wt, alphas, hel)
        total += np.real(np.einsum("ns,st,nt->n", a.conj(), gm, a))
    return total / CROSSINGS[process][1]


def me2(p: np.ndarray, mt: float, wt: float, alphas: float) -> np.ndarray:
    """Spin/colour summed and averaged |M|^2 for q q~ -> t t~ g, one point."""
    p = _real(p)
    if p.ndim != 3 or p.shape[1] != 5:
        raise ValueError("q q~ -> t t~ g expects momenta [N, 5, 4]")
    gm = colour_matrix()
    total = np.zeros(p.shape[0], dtype=p.dtype)
    for hel in itertools.product((-1, 1), repeat=5):
        a = amplitudes(p, mt, wt, alphas, hel)
        total += np.real(np.einsum("ns,st,nt->n", a.conj(), gm, a))
    return total / 36.0


def me2_helicity(p: np.ndarray, mt: float, wt: float, alphas: float, hel: np.ndarray) -> np.ndarray:
    """The term of the helicity sum (me2 = sum over configurations, same 1/36) of each
    event's own configuration hel[N, 5] = (l1, l2, l3, l4, lg): helicities of q, q~, t,
    t~ and the gluon in the frame of the momenta."""
    p = _real(p)
    hel = np.asarray(hel)
    gm = colour_matrix()
    out = np.zeros(p.shape[0], dtype=p.dtype)
    for conf in itertools.product((-1, 1), repeat=5):
        sel = np.all(hel == np.array(conf), axis=1)
        if np.any(sel):
            a = amplitudes(p[sel], mt, wt, alphas, conf)
            out[sel] = np.real(np.einsum("ns,st,nt->n", a.conj(), gm, a)) / 36.0
    return out


def colour_amplitude(p: np.ndarray, mt: float, hel: tuple, eps_override=None, alphas: float = 0.118,
                     process: str = "qq_ttxg") -> np.ndarray:
    """sum_d K_d A_d: the colour-dressed amplitude [N, 8, 3, 3, 3, 3] of one configuration
    (hel in record order) of q q~ -> t t~ g or one of its CROSSINGS."""
    if process == "qq_ttxg":
        a = amplitudes(p, mt, 0.0, alphas, hel, eps_override)
    else:
        a = amplitudes_crossed(process, p, mt, 0.0, alphas, hel, eps_override)
    return np.einsum("nd,dajklm->najklm", a, colour_tensors())
