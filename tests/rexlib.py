"""Shared helpers for tests that load the CUDA library."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rex.h")
TOOLING_HEADER = os.path.join(ROOT, "include", "rex_tooling.h")


def ensure_built():
    from paper_2510_05100_b300 import build, rex
    if not os.path.exists(rex.LIB_PATH):
        build.build()
    return rex


def declared_symbols(header=HEADER):
    text = open(header).read()
    return sorted(set(re.findall(r"^(?:int64_t|int|void|const char \*)\s*\*?\s*(rex_\w+)\s*\(", text, re.M)))


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


gpu = pytest.mark.gpu


def helicity_tolerance(proc, mom, hel, orig, pts, floor, eps):
    """Per (event, point) bound on the relative error of a helicity-exclusive weight:
    max(floor, 64 eps (sqrt(kappa_0) + sqrt(kappa_j))), kappa = |M|^2 / |M_h|^2 at
    each point (the oracle's values)."""
    import numpy as np
    from oracle import reweight as oracle_rw

    def sqrt_kappa(pt):
        mh = oracle_rw.me2_helicity(proc, mom, pt, hel)
        return np.sqrt(oracle_rw.me2(proc, mom, pt) / np.where(mh > 0, mh, np.inf))
    k0 = sqrt_kappa(orig)
    kj = np.stack([sqrt_kappa(pt) for pt in pts], axis=1)
    return np.maximum(floor, 64.0 * eps * (k0[:, None] + kj))
