"""Minkowski algebra, Dirac matrices, helicity spinors and polarisation vectors.

Oracle module (test infrastructure only).  Everything is numpy FP64 /
complex128, vectorised over a leading event axis.

Conventions (textbook; the paper states its wavefunctions in Sect. 4.1):
  * metric (+,-,-,-); a four-vector is an array [..., 4] = (E, px, py, pz)
  * chiral (Weyl) basis: gamma^0 = [[0,1],[1,0]], gamma^k = [[0,s_k],[-s_k,0]],
    gamma_5 = diag(-1,-1,1,1); P_L = (1-gamma_5)/2 keeps the upper two components
  * u(p,l) = ( sqrt(E - l|p|) xi_l , sqrt(E + l|p|) xi_l )
    v(p,l) = ( -l sqrt(E + l|p|) xi_-l , l sqrt(E - l|p|) xi_-l )
    with xi_l the two-component helicity eigenstate along p (l = +-1 is twice
    the helicity) -- the spinors the paper calls u(p, nHEL/2), v(p, nHEL/2)
  * eps(k, +-1) = (0, -+ e_theta - i e_phi)/sqrt(2), eps(k, 0) = (|k|, E k^)/m;
    an incoming vector boson carries eps, an outgoing one eps^* (Sect. 4.1)

Parity: pinned by tests/test_oracle_lorentz.py (Dirac equation, helicity
eigenvalue, normalisation, completeness relations, transversality).
"""
import numpy as np

METRIC = np.array([1.0, -1.0, -1.0, -1.0])

_I2 = np.eye(2, dtype=complex)
_Z2 = np.zeros((2, 2), dtype=complex)
PAULI = [
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
]

# gamma^mu with an upper index, shape (4, 4, 4): [mu, row, col]
GAMMA = np.array(
    [np.block([[_Z2, _I2], [_I2, _Z2]])]
    + [np.block([[_Z2, s], [-s, _Z2]]) for s in PAULI]
)
GAMMA5 = np.diag([-1.0, -1.0, 1.0, 1.0]).astype(complex)
PL = 0.5 * (np.eye(4) - GAMMA5)
PR = 0.5 * (np.eye(4) + GAMMA5)
GAMMA0 = GAMMA[0]


def mdot(a, b):
    """Minkowski product a.b over the last axis (no complex conjugation)."""
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def lower(a):
    """a_mu from a^mu."""
    return a * METRIC


def slash(a):
    """gamma^mu a_mu for a contravariant (possibly complex) vector, [..., 4] -> [..., 4, 4]."""
    return np.einsum("...m,mij->...ij", lower(a).astype(complex), GAMMA)


def _angles(p):
    """Polar and azimuthal angle of the three-momentum (z axis for p = 0)."""
    px, py, pz = p[..., 1], p[..., 2], p[..., 3]
    r = np.sqrt(px * px + py * py + pz * pz)
    theta = np.arctan2(np.sqrt(px * px + py * py), pz)
    phi = np.arctan2(py, px)
    return r, theta, phi


def helicity_xi(p, lam):
    """Two-component eigenstate of (p^ . sigma) with eigenvalue lam (= +-1)."""
    _, th, ph = _angles(p)
    c, s = np.cos(th / 2), np.sin(th / 2)
    if lam == 1:
        return np.stack([c + 0j, np.exp(1j * ph) * s], axis=-1)
    return np.stack([-np.exp(-1j * ph) * s, c + 0j], axis=-1)


def _sqrt_pos(x):
    return np.sqrt(np.maximum(x, 0.0))


def u_spinor(p, lam):
    """Dirac spinor u(p, lam/2) of a fermion with four-momentum p (p^2 = m^2)."""
    r, _, _ = _angles(p)
    E = p[..., 0]
    xi = helicity_xi(p, lam)
    a = _sqrt_pos(E - lam * r)[..., None]
    b = _sqrt_pos(E + lam * r)[..., None]
    return np.concatenate([a * xi, b * xi], axis=-1)


def v_spinor(p, lam):
    """Dirac spinor v(p, lam/2) of an antifermion with four-momentum p."""
    r, _, _ = _angles(p)
    E = p[..., 0]
    eta = helicity_xi(p, -lam)
    a = _sqrt_pos(E + lam * r)[..., None]
    b = _sqrt_pos(E - lam * r)[..., None]
    return np.concatenate([-lam * a * eta, lam * b * eta], axis=-1)


def bar(psi):
    """Dirac adjoint psi^dagger gamma^0 as a row spinor [..., 4]."""
    return np.einsum("...i,ij->...j", psi.conj(), GAMMA0)


def polarisation(k, lam, mass=0.0):
    """eps^mu(k, lam) for lam = +1, -1 (and 0 when mass > 0); complex [..., 4]."""
    r, th, ph = _angles(k)
    if lam == 0:
        E = k[..., 0]
        out = np.zeros(k.shape, dtype=complex)
        safe = np.where(r > 0, r, 1.0)
        out[..., 0] = r / mass
        for j in range(3):
            nj = np.where(r > 0, k[..., j + 1] / safe, 1.0 if j == 2 else 0.0)
            out[..., j + 1] = E * nj / mass
        return out
    e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=-1)
    e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=-1)
    eps3 = (-lam * e_th - 1j * e_ph) / np.sqrt(2.0)
    return np.concatenate([np.zeros(k.shape[:-1] + (1,), dtype=complex), eps3], axis=-1)


def boost(p, beta):
    """Active Lorentz boost of four-vectors p [..., 4] by velocity beta [3] (|beta| < 1)."""
    beta = np.asarray(beta, dtype=float)
    b2 = float(beta @ beta)
    g = 1.0 / np.sqrt(1.0 - b2)
    bp = p[..., 1:] @ beta
    E = g * (p[..., 0] + bp)
    coef = np.where(b2 > 0, (g - 1.0) * bp / (b2 if b2 > 0 else 1.0), 0.0) + g * p[..., 0]
    vec = p[..., 1:] + coef[..., None] * beta
    return np.concatenate([E[..., None], vec], axis=-1)


def rotate(p, R):
    """Rotate the three-vector part of p [..., 4] by the 3x3 matrix R."""
    return np.concatenate([p[..., :1], p[..., 1:] @ R.T], axis=-1)
