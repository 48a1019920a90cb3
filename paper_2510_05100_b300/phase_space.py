"""Seeded synthetic parton-level events (inputs only; no matrix-element arithmetic).

Both the CUDA path and the CPU oracle consume what this module produces, so it
holds nothing of the reweighting method itself: only phase-space point
generation and the parameter grids.  Events are returned as float64 arrays of
shape ``[nev, npart, 4]`` with components ordered (E, px, py, pz), the per-parton
``(t, x, y, z)`` order of the Rex SoA momentum vectors (paper Sec. 2.1.1, Table 2).

Workloads (all in the partonic centre-of-mass frame, no cuts):

* ``ee_mumu``: e+(1) e-(2) -> mu+(3) mu-(4), sqrt(s)=500 GeV, massless, e+ along
  +z, e- along -z; cos(theta) uniform in [-1, 1] where theta is the angle between
  mu- and e-, phi uniform in [0, 2 pi).
* ``gg_ttx``: g(1) g(2) -> t(3) t~(4); sqrt(s_hat) log-uniform, isotropic top.
* ``qq_ttx``: q(1) q~(2) -> t(3) t~(4), massless light quarks; the same
  two-body kinematics as ``gg_ttx``.
* ``qq_ttxg``: q(1) q~(2) -> t(3) t~(4) g(5); the ``gg_ttxg`` kinematics.  Its
  crossed channels ``qxq_ttxg``, ``qg_ttxq``, ``gq_ttxq``, ``qxg_ttxqx`` and
  ``gqx_ttxqx`` (the two incoming partons, t, t~, the outgoing light parton) take
  the same kinematics: every external light parton is massless.
* ``gg_ttxg`` / ``gg_ttxgg``: g g -> t t~ g (g): massive RAMBO (Kleiss, Stirling,
  Ellis, Comput. Phys. Commun. 40 (1986) 359) at log-uniform sqrt(s_hat).

Random numbers come from numpy's PCG64 generator with an explicit seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MT_DEFAULT = 173.0
ALPHAS_DEFAULT = 0.118

# Electroweak reference point for e+e- -> mu+mu- (photon + Z).
EE_ORIGINAL = dict(mz=91.1876, wz=2.4952, sw2=0.2312, alpha=1.0 / 132.507)
EE_NEW = dict(mz=91.0, wz=2.6, sw2=0.2300, alpha=1.0 / 132.507)

QQ_TTXG_CROSSINGS = ("qq_ttxg", "qxq_ttxg", "qg_ttxq", "gq_ttxq", "qxg_ttxqx", "gqx_ttxqx")
PROCESS_NPART = {"ee_mumu": 4, "gg_ttx": 4, "qq_ttx": 4, "gg_ttxg": 5, "gg_ttxgg": 6,
                 **{name: 5 for name in QQ_TTXG_CROSSINGS}}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _beams(sqrt_s: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two massless beams along +z and -z, each carrying sqrt(s)/2."""
    n = sqrt_s.shape[0]
    e = 0.5 * sqrt_s
    b1 = np.zeros((n, 4))
    b2 = np.zeros((n, 4))
    b1[:, 0] = e
    b1[:, 3] = e
    b2[:, 0] = e
    b2[:, 3] = -e
    return b1, b2


def ee_mumu_events(nev: int, seed: int = 1, sqrt_s: float = 500.0) -> np.ndarray:
    """e+(1) e-(2) -> mu+(3) mu-(4) at fixed sqrt(s), massless leptons."""
    g = _rng(seed)
    cos_t = g.uniform(-1.0, 1.0, nev)
    phi = g.uniform(0.0, 2.0 * math.pi, nev)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    e = 0.5 * sqrt_s
    p = np.zeros((nev, 4, 4))
    p[:, 0] = [e, 0.0, 0.0, e]        # e+ along +z
    p[:, 1] = [e, 0.0, 0.0, -e]       # e- along -z
    # mu- direction n with n . (-z) = cos(theta)
    n = np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), -cos_t], axis=1)
    p[:, 3, 0] = e
    p[:, 3, 1:] = e * n
    p[:, 2, 0] = e
    p[:, 2, 1:] = -e * n
    return p


def log_uniform(g: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(g.uniform(math.log(lo), math.log(hi), n))


def two_body_events(nev: int, seed: int, m3: float, m4: float,
                    rs_lo: float, rs_hi: float) -> np.ndarray:
    """Massless beams -> two bodies of masses m3, m4, isotropic in the CM frame."""
    g = _rng(seed)
    rs = log_uniform(g, rs_lo, rs_hi, nev)
    cos_t = g.uniform(-1.0, 1.0, nev)
    phi = g.uniform(0.0, 2.0 * math.pi, nev)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    s = rs * rs
    # Kallen function for the final-state momentum
    lam = (s - (m3 + m4) ** 2) * (s - (m3 - m4) ** 2)
    pabs = np.sqrt(np.maximum(lam, 0.0)) / (2.0 * rs)
    e3 = (s + m3 * m3 - m4 * m4) / (2.0 * rs)
    e4 = (s + m4 * m4 - m3 * m3) / (2.0 * rs)
    n = np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)
    b1, b2 = _beams(rs)
    p = np.zeros((nev, 4, 4))
    p[:, 0] = b1
    p[:, 1] = b2
    p[:, 2, 0] = e3
    p[:, 2, 1:] = pabs[:, None] * n
    p[:, 3, 0] = e4
    p[:, 3, 1:] = -pabs[:, None] * n
    return p


def rambo_massive(g: np.random.Generator, rs: np.ndarray,
                  masses: list[float]) -> np.ndarray:
    """RAMBO: n final-state momenta, total (rs, 0, 0, 0), given masses.

    Massless RAMBO (isotropic q_i with energies from -log(r1 r2), conformal
    transformation to the CM frame), followed by the massive rescaling
    p_i = (sqrt(m_i^2 + xi^2 E_i^2), xi * p_i) with xi solved by Newton
    iteration from sum_i sqrt(m_i^2 + xi^2 E_i^2) = rs.
    """
    nev = rs.shape[0]
    n = len(masses)
    r = g.uniform(0.0, 1.0, (nev, n, 4))
    c = 2.0 * r[..., 0] - 1.0
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    f = 2.0 * math.pi * r[..., 1]
    q0 = -np.log(np.maximum(r[..., 2] * r[..., 3], 1e-300))
    q = np.empty((nev, n, 4))
    q[..., 0] = q0
    q[..., 1] = q0 * s * np.cos(f)
    q[..., 2] = q0 * s * np.sin(f)
    q[..., 3] = q0 * c
    qs = q.sum(axis=1)                                   # [nev, 4]
    qm = np.sqrt(np.maximum(qs[:, 0] ** 2 - (qs[:, 1:] ** 2).sum(axis=1), 0.0))
    b = -qs[:, 1:] / qm[:, None]
    gam = qs[:, 0] / qm
    a = 1.0 / (1.0 + gam)
    x = rs / qm
    bq = (b[:, None, :] * q[..., 1:]).sum(axis=2)        # [nev, n]
    p = np.empty((nev, n, 4))
    p[..., 0] = x[:, None] * (gam[:, None] * q[..., 0] + bq)
    p[..., 1:] = x[:, None, None] * (q[..., 1:] + b[:, None, :] * q[..., 0:1]
                                     + a[:, None, None] * bq[..., None] * b[:, None, :])
    m = np.asarray(masses, dtype=np.float64)
    if np.all(m == 0.0):
        return p
    e0 = p[..., 0].copy()
    xi = np.sqrt(np.maximum(0.0, 1.0 - (m.sum() / rs) ** 2))
    for _ in range(60):
        en = np.sqrt(m[None, :] ** 2 + (xi[:, None] * e0) ** 2)
        fval = en.sum(axis=1) - rs
        dval = (xi[:, None] * e0 ** 2 / en).sum(axis=1)
        step = fval / dval
        xi = xi - step
        if np.max(np.abs(step)) < 1e-15:
            break
    out = np.empty_like(p)
    out[..., 0] = np.sqrt(m[None, :] ** 2 + (xi[:, None] * e0) ** 2)
    out[..., 1:] = xi[:, None, None] * p[..., 1:]
    return out


def gg_tt_jets_events(nev: int, seed: int, njets: int, rs_lo: float, rs_hi: float,
                      mt: float = MT_DEFAULT) -> np.ndarray:
    """g(1) g(2) -> t(3) t~(4) + njets gluons via massive RAMBO."""
    g = _rng(seed)
    rs = log_uniform(g, rs_lo, rs_hi, nev)
    fin = rambo_massive(g, rs, [mt, mt] + [0.0] * njets)
    b1, b2 = _beams(rs)
    p = np.empty((nev, 4 + njets, 4))
    p[:, 0] = b1
    p[:, 1] = b2
    p[:, 2:] = fin
    return p


@dataclass(frozen=True)
class Workload:
    process: str
    nev: int
    seed: int
    description: str


def make_events(process: str, nev: int, seed: int, mt: float = MT_DEFAULT) -> np.ndarray:
    """The standard synthetic sample for each process (see module docstring)."""
    if process == "ee_mumu":
        return ee_mumu_events(nev, seed)
    if process in ("gg_ttx", "qq_ttx"):
        return two_body_events(nev, seed, mt, mt, 2.0 * mt + 1.0, 3000.0)
    if process == "gg_ttxg" or process in QQ_TTXG_CROSSINGS:
        return gg_tt_jets_events(nev, seed, 1, 400.0, 4000.0, mt)
    if process == "gg_ttxgg":
        return gg_tt_jets_events(nev, seed, 2, 500.0, 5000.0, mt)
    raise ValueError(f"unknown process {process!r}")


def qcd_grid(n_mt: int, mt_lo: float, mt_hi: float,
             n_as: int, as_lo: float, as_hi: float) -> list[dict]:
    """mt-major grid of (mt, alphas) parameter points; top width 0."""
    mts = np.linspace(mt_lo, mt_hi, n_mt)
    als = np.linspace(as_lo, as_hi, n_as) if n_as > 1 else np.array([as_lo])
    return [dict(mt=float(m), wt=0.0, alphas=float(a)) for m in mts for a in als]


def grid_gg_ttx() -> list[dict]:
    """8 points: mt in linspace(171, 175, 4) x alphas in {0.112, 0.124}."""
    return qcd_grid(4, 171.0, 175.0, 2, 0.112, 0.124)


def grid_gg_ttxg() -> list[dict]:
    """16 points: mt in linspace(171, 175, 4) x alphas in linspace(0.112, 0.124, 4)."""
    return qcd_grid(4, 171.0, 175.0, 4, 0.112, 0.124)


def grid_64() -> list[dict]:
    """64 points: mt in linspace(170, 176, 8) x alphas in linspace(0.110, 0.126, 8)."""
    return qcd_grid(8, 170.0, 176.0, 8, 0.110, 0.126)


def qcd_original(mt: float = MT_DEFAULT, alphas: float = ALPHAS_DEFAULT) -> dict:
    return dict(mt=mt, wt=0.0, alphas=alphas)
