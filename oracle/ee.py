"""e+(1) e-(2) -> mu+(3) mu-(4) through photon and Z exchange (oracle).

Feynman rules (massless leptons, Feynman-gauge propagators; the q^mu q^nu part
of the Z propagator vanishes against the conserved massless currents):

* photon-fermion vertex    -i e Q_f gamma^mu
* Z-fermion vertex         -i (e / (s_W c_W)) gamma^mu (g_L^f P_L + g_R^f P_R),
                           g_L = T3 - Q s_W^2,  g_R = -Q s_W^2
* photon propagator        -i g_{mu nu} / q^2
* Z propagator             -i g_{mu nu} / (q^2 - m_Z^2 + i m_Z Gamma_Z)

Electroweak inputs are independent: alpha, m_Z, Gamma_Z, sin^2 theta_W, with
c_W^2 = 1 - s_W^2.  The amplitude is
    iM = [vbar(p1) V_mu u(p2)] D^{mu nu}(s) [ubar(p4) V_nu v(p3)]
summed over the two exchanged bosons; |M|^2 is summed over the 16 helicity
configurations and averaged by 1/4.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .lorentz import GAMMA, PL, PR, bar, mdot, spinor_u, spinor_v

Q_LEPTON = -1.0
T3_LEPTON = -0.5


def _vector_current(left: np.ndarray, right: np.ndarray, cl: float, cr: float) -> np.ndarray:
    """left^bar gamma^mu (cl P_L + cr P_R) right, as an upper-index 4-vector [N, 4]."""
    chiral = cl * PL + cr * PR
    mats = np.einsum("mij,jk->mik", GAMMA, chiral)
    return np.einsum("ni,mij,nj->nm", left, mats, right)


def me2_helicity(p: np.ndarray, mz: float, wz: float, sw2: float, alpha: float, hel: np.ndarray) -> np.ndarray:
    """The term of the helicity sum (me2 = sum over configurations, same 1/4) of each
    event's own configuration hel[N, 4] = (l1, l2, l3, l4), helicities +1/-1 of
    e+, e-, mu+, mu- in the frame of the momenta."""
    p = np.asarray(p, dtype=np.float64)
    hel = np.asarray(hel)
    out = np.zeros(p.shape[0])
    for conf in itertools.product((-1, 1), repeat=4):
        sel = np.all(hel == np.array(conf), axis=1)
        if np.any(sel):
            out[sel] = _config_me2(p[sel], mz, wz, sw2, alpha, conf)
    return out


def _config_me2(p, mz, wz, sw2, alpha, conf):
    e = math.sqrt(4.0 * math.pi * alpha)
    cw2 = 1.0 - sw2
    gz = e / math.sqrt(sw2 * cw2)
    gl = T3_LEPTON - Q_LEPTON * sw2
    gr = -Q_LEPTON * sw2
    p1, p2, p3, p4 = p[:, 0], p[:, 1], p[:, 2], p[:, 3]
    q = p1 + p2
    s = mdot(q, q)
    l1, l2, l3, l4 = conf
    vb1 = bar(spinor_v(p1, 0.0, l1))
    u2 = spinor_u(p2, 0.0, l2)
    v3 = spinor_v(p3, 0.0, l3)
    ub4 = bar(spinor_u(p4, 0.0, l4))
    amp = (-1j / s) * mdot(-1j * e * Q_LEPTON * _vector_current(vb1, u2, 1.0, 1.0),
                           -1j * e * Q_LEPTON * _vector_current(ub4, v3, 1.0, 1.0))
    amp = amp + (-1j / (s - mz * mz + 1j * mz * wz)) * mdot(-1j * gz * _vector_current(vb1, u2, gl, gr),
                                                            -1j * gz * _vector_current(ub4, v3, gl, gr))
    return np.abs(amp) ** 2 / 4.0


def me2(p: np.ndarray, mz: float, wz: float, sw2: float, alpha: float) -> np.ndarray:
    p = np.asarray(p, dtype=np.float64)
    e = math.sqrt(4.0 * math.pi * alpha)
    cw2 = 1.0 - sw2
    gz = e / math.sqrt(sw2 * cw2)
    gl = T3_LEPTON - Q_LEPTON * sw2
    gr = -Q_LEPTON * sw2
    p1, p2, p3, p4 = p[:, 0], p[:, 1], p[:, 2], p[:, 3]
    q = p1 + p2
    s = mdot(q, q)
    d_a = -1j / s
    d_z = -1j / (s - mz * mz + 1j * mz * wz)
    total = np.zeros(p.shape[0])
    for l1, l2, l3, l4 in itertools.product((-1, 1), repeat=4):
        vb1 = bar(spinor_v(p1, 0.0, l1))
        u2 = spinor_u(p2, 0.0, l2)
        v3 = spinor_v(p3, 0.0, l3)
        ub4 = bar(spinor_u(p4, 0.0, l4))
        amp = np.zeros(p.shape[0], dtype=complex)
        # photon
        je = -1j * e * Q_LEPTON * _vector_current(vb1, u2, 1.0, 1.0)
        jm = -1j * e * Q_LEPTON * _vector_current(ub4, v3, 1.0, 1.0)
        amp += d_a * mdot(je, jm)
        # Z
        je = -1j * gz * _vector_current(vb1, u2, gl, gr)
        jm = -1j * gz * _vector_current(ub4, v3, gl, gr)
        amp += d_z * mdot(je, jm)
        total += np.abs(amp) ** 2
    return total / 4.0
