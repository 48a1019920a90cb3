"""Minkowski and Dirac algebra, external spinors and polarisation vectors (oracle).

Conventions (Peskin & Schroeder, "An Introduction to QFT", Ch. 3):
metric diag(+1, -1, -1, -1); chiral basis
    gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]],
    sigma^mu = (1, sigma_i), sigmabar^mu = (1, -sigma_i),
so that the upper two components are left-handed.

External fermions (P&S eq. 3.50 and 3.62):
    u(p, xi) = ( sqrt(p.sigma) xi,  sqrt(p.sigmabar) xi )
    v(p, eta) = ( sqrt(p.sigma) eta, -sqrt(p.sigmabar) eta )
with xi a helicity eigenvector along p-hat and eta = xi of opposite helicity.
The square root of the 2x2 Hermitian matrix M = p.sigma (det M = m^2) is taken
from the Cayley-Hamilton identity sqrt(M) = (M + m 1) / sqrt(tr M + 2 m).

Mass used in external spinors when a parameter point changes the mass while
the momenta are kept (the paper's reweighting passes only momenta to the
amplitude, Sec. 4.1.3): the spinor is the standard one of the on-shell momentum
    p~ = (E~, |p~| p-hat),  E~ + |p~| = E + |p|,  E~ - |p~| = m^2 / (E + |p|),
i.e. same direction and same light-cone component E + |p| as p, mass m.
When p^2 = m^2 this is p itself.
"""
from __future__ import annotations

import numpy as np

METRIC = np.diag([1.0, -1.0, -1.0, -1.0])

_I2 = np.eye(2, dtype=complex)
_SX = np.array([[0, 1], [1, 0]], dtype=complex)
_SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
_SZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = [_I2, _SX, _SY, _SZ]

GAMMA = np.zeros((4, 4, 4), dtype=complex)
for _mu in range(4):
    _sig = PAULI[_mu]
    _sigbar = PAULI[_mu] if _mu == 0 else -PAULI[_mu]
    GAMMA[_mu, :2, 2:] = _sig
    GAMMA[_mu, 2:, :2] = _sigbar
GAMMA5 = np.diag([-1.0, -1.0, 1.0, 1.0]).astype(complex)
PL = 0.5 * (np.eye(4) - GAMMA5)
PR = 0.5 * (np.eye(4) + GAMMA5)


def mdot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Minkowski product a.b over the last axis (no complex conjugation)."""
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def slash(a: np.ndarray) -> np.ndarray:
    """gamma^mu a_mu for upper-index components a[..., 4] -> [..., 4, 4]."""
    a_low = a * np.array([1.0, -1.0, -1.0, -1.0])
    return np.einsum("...m,mij->...ij", a_low.astype(complex), GAMMA)


def bar(psi: np.ndarray) -> np.ndarray:
    """Dirac adjoint psi^dagger gamma^0 of column spinors psi[..., 4]."""
    return np.einsum("...i,ij->...j", psi.conj(), GAMMA[0])


def _sigma_dot(p: np.ndarray, sign: float) -> np.ndarray:
    """p.sigma (sign=+1) or p.sigmabar (sign=-1) as [..., 2, 2]: p^0 1 - sign p_vec.sigma_vec."""
    out = p[..., 0, None, None] * _I2
    for i in range(1, 4):
        out = out - sign * p[..., i, None, None] * PAULI[i]
    return out


def _sqrt_psd2(m: np.ndarray, det_sqrt: np.ndarray) -> np.ndarray:
    """sqrt of Hermitian PSD 2x2 matrices with sqrt(det) given (Cayley-Hamilton)."""
    tr = np.real(m[..., 0, 0] + m[..., 1, 1])
    den = np.sqrt(tr + 2.0 * det_sqrt)
    return (m + det_sqrt[..., None, None] * _I2) / den[..., None, None]


def angles(p: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Polar and azimuthal angle of the 3-momentum (theta=0, phi=0 for p=0)."""
    pabs = np.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2 + p[..., 3] ** 2)
    safe = np.where(pabs > 0, pabs, 1.0)
    cos_t = np.where(pabs > 0, p[..., 3] / safe, 1.0)
    theta = np.arccos(np.clip(cos_t, -1.0, 1.0))
    phi = np.arctan2(p[..., 2], p[..., 1])
    return theta, phi


def helicity_xi(p: np.ndarray, lam: int) -> np.ndarray:
    """Two-spinor with (p-hat . sigma) xi = lam xi (P&S problem 3.x basis)."""
    theta, phi = angles(p)
    c = np.cos(theta / 2.0)
    s = np.sin(theta / 2.0)
    if lam > 0:
        xi = np.stack([c + 0j, np.exp(1j * phi) * s], axis=-1)
    else:
        xi = np.stack([-np.exp(-1j * phi) * s, c + 0j], axis=-1)
    return xi


def onshell_projection(p: np.ndarray, m: float) -> np.ndarray:
    """p~: same direction and E+|p| as p, mass m (see module docstring)."""
    pabs = np.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2 + p[..., 3] ** 2)
    wp2 = p[..., 0] + pabs
    wm2 = m * m / wp2
    e_t = 0.5 * (wp2 + wm2)
    k_t = 0.5 * (wp2 - wm2)
    safe = np.where(pabs > 0, pabs, 1.0)
    out = np.empty_like(p)
    out[..., 0] = e_t
    for i in range(1, 4):
        out[..., i] = np.where(pabs > 0, p[..., i] / safe * k_t, 0.0)
    return out


def spinor_u(p: np.ndarray, m: float, lam: int) -> np.ndarray:
    """u(p~, xi_lam) as [..., 4] complex."""
    pt = onshell_projection(p, m)
    xi = helicity_xi(p, lam)
    msq = np.full(p.shape[:-1], abs(m))
    up = _sqrt_psd2(_sigma_dot(pt, +1.0), msq)
    dn = _sqrt_psd2(_sigma_dot(pt, -1.0), msq)
    return np.concatenate([np.einsum("...ij,...j->...i", up, xi),
                           np.einsum("...ij,...j->...i", dn, xi)], axis=-1)


def spinor_v(p: np.ndarray, m: float, lam: int) -> np.ndarray:
    """v(p~, eta) for an antifermion of helicity lam, eta = xi_{-lam}, as [..., 4]."""
    pt = onshell_projection(p, m)
    eta = helicity_xi(p, -lam)
    msq = np.full(p.shape[:-1], abs(m))
    up = _sqrt_psd2(_sigma_dot(pt, +1.0), msq)
    dn = _sqrt_psd2(_sigma_dot(pt, -1.0), msq)
    return np.concatenate([np.einsum("...ij,...j->...i", up, eta),
                           -np.einsum("...ij,...j->...i", dn, eta)], axis=-1)


def polarisation(k: np.ndarray, lam: int) -> np.ndarray:
    """Helicity polarisation vector eps^mu(k, lam) = -(lam e_theta + i e_phi)/sqrt(2).

    e_theta, e_phi are the spherical unit vectors of k-hat; eps is transverse
    (eps^0 = 0, eps.k = 0) and normalised eps.eps^* = -1.
    """
    theta, phi = angles(k)
    ct, st = np.cos(theta), np.sin(theta)
    cp, sp = np.cos(phi), np.sin(phi)
    e_th = np.stack([np.zeros_like(ct), ct * cp, ct * sp, -st], axis=-1)
    e_ph = np.stack([np.zeros_like(ct), -sp, cp, np.zeros_like(ct)], axis=-1)
    return -(lam * e_th + 1j * e_ph) / np.sqrt(2.0)
