"""Reweighting epilogue and process dispatch (oracle).

w'_{e,j} = w_e |M(p_e; theta_j)|^2 / |M(p_e; theta_0)|^2  (paper Sec. 3, the
weight factorisation), with the teaRex normaliser convention (Sec. 3.1.1):
the normaliser is 1/|M|^2 with 1/0 mapped to 0, so an event whose original
|M|^2 is zero gets new weights 0.  Helicity-exclusive reweighting (the
alternative to the helicity-summed default, Sec. 4.1.2) takes the same ratio of
the event's own helicity configuration.
"""
from __future__ import annotations

import numpy as np

from . import ee, qcd, qq, qqg

QCD_PROCESSES = {"gg_ttx": 4, "gg_ttxg": 5, "gg_ttxgg": 6}


def me2(process: str, p: np.ndarray, point: dict) -> np.ndarray:
    """|M|^2 per event for one parameter point (dict of named parameters)."""
    if process == "ee_mumu":
        return ee.me2(p, point["mz"], point["wz"], point["sw2"], point["alpha"])
    if process in QCD_PROCESSES:
        if p.shape[1] != QCD_PROCESSES[process]:
            raise ValueError(f"{process} expects {QCD_PROCESSES[process]} particles")
        return qcd.me2(p, point["mt"], point.get("wt", 0.0), point["alphas"])
    if process == "qq_ttx":
        return qq.me2(p, point["mt"], point.get("wt", 0.0), point["alphas"])
    if process == "qq_ttxg":
        return qqg.me2(p, point["mt"], point.get("wt", 0.0), point["alphas"])
    if process in qqg.CROSSINGS:
        return qqg.me2_crossed(process, p, point["mt"], point.get("wt", 0.0), point["alphas"])
    raise ValueError(f"unknown process {process!r}")


# A configuration that vanishes identically (a massless fermion pair of equal
# helicities in a vector current) comes out of the explicit spinors as a rounding
# residue of about 1e-32 of the event's helicity sum; below this fraction a term is
# taken as the exact zero it is (physical terms, helicity flips ~ m^2/s included,
# are many orders above it).
ZERO_TERM = 1e-24


def me2_helicity(process: str, p: np.ndarray, point: dict, hel: np.ndarray) -> np.ndarray:
    """The helicity-sum term of each event's own helicity configuration hel[N, npart]
    (processes whose amplitudes are evaluated in a helicity basis)."""
    if process == "ee_mumu":
        m = ee.me2_helicity(p, point["mz"], point["wz"], point["sw2"], point["alpha"], hel)
    elif process == "qq_ttx":
        m = qq.me2_helicity(p, point["mt"], point.get("wt", 0.0), point["alphas"], hel)
    elif process == "qq_ttxg":
        m = qqg.me2_helicity(p, point["mt"], point.get("wt", 0.0), point["alphas"], hel)
    elif process in QCD_PROCESSES:
        m = qcd.me2_helicity_per_event(p, point["mt"], point.get("wt", 0.0), point["alphas"], hel)
    else:
        raise ValueError(f"no helicity-exclusive evaluation for {process!r}")
    return np.where(m < ZERO_TERM * me2(process, p, point), 0.0, m)


def reweight_helicity(process: str, p: np.ndarray, hel: np.ndarray, w_in: np.ndarray, original: dict,
                      points: list[dict]) -> np.ndarray:
    """Helicity-exclusive new weights [N, k]: w |M_h(theta_j)|^2 / |M_h(theta_0)|^2 with h
    the event's own configuration, and 0 where |M_h(theta_0)|^2 == 0."""
    m0 = me2_helicity(process, p, original, hel)
    mk = (np.stack([me2_helicity(process, p, pt, hel) for pt in points]) if points
          else np.zeros((0, p.shape[0])))
    return ratio_epilogue(w_in, m0, mk)


def ratio_epilogue(w_in: np.ndarray, me2_orig: np.ndarray, me2_new: np.ndarray) -> np.ndarray:
    """w_in * me2_new / me2_orig, and 0 where me2_orig == 0.  Shapes [N], [N], [k, N] -> [N, k]."""
    w_in = np.asarray(w_in, dtype=np.float64)
    zero = me2_orig == 0.0
    safe = np.where(zero, 1.0, me2_orig)
    out = w_in[None, :] * (me2_new / safe[None, :])
    out[:, zero] = 0.0
    return out.T.copy()


def reweight(process: str, p: np.ndarray, w_in: np.ndarray, original: dict,
             points: list[dict]) -> np.ndarray:
    """New weights [N, k] for k parameter points."""
    m0 = me2(process, p, original)
    mk = np.stack([me2(process, p, pt) for pt in points]) if points else np.zeros((0, p.shape[0]))
    return ratio_epilogue(w_in, m0, mk)
