"""Shared helpers for tests that load the CUDA library."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rex.h")


def ensure_built():
    from paper_2510_05100_b300 import build, rex
    if not os.path.exists(rex.LIB_PATH):
        build.build()
    return rex


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int64_t|int|void|const char \*)\s*\*?\s*(rex_\w+)\s*\(", text, re.M)))


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


gpu = pytest.mark.gpu
