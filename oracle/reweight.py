"""Reweighting epilogue and process dispatch (oracle).

w'_{e,j} = w_e |M(p_e; theta_j)|^2 / |M(p_e; theta_0)|^2  (paper Sec. 3, the
weight factorisation), with the teaRex normaliser convention (Sec. 3.1.1):
the normaliser is 1/|M|^2 with 1/0 mapped to 0, so an event whose original
|M|^2 is zero gets new weights 0.
"""
from __future__ import annotations

import numpy as np

from . import ee, qcd, qq

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
    raise ValueError(f"unknown process {process!r}")


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
