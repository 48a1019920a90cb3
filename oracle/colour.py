"""SU(3) generators and structure constants as explicit matrices (oracle).

t^a = lambda^a / 2 with the Gell-Mann matrices lambda^a, so tr(t^a t^b) = delta^ab / 2,
and [t^a, t^b] = i f^abc t^c, hence f^abc = -2 i tr([t^a, t^b] t^c).
"""
from __future__ import annotations

import numpy as np

NC = 3
NADJ = 8


def gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


T = gell_mann() / 2.0


def structure_constants() -> np.ndarray:
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = -2j * np.einsum("abik,cki->abc", comm, T)
    assert np.max(np.abs(f.imag)) < 1e-14
    return f.real


F = structure_constants()
