"""Pins of the oracle's spinors and polarisation vectors against their defining equations."""
import numpy as np
import pytest

from oracle.lorentz import (GAMMA, GAMMA0, METRIC, bar, boost, mdot, polarisation, slash,
                            u_spinor, v_spinor)


def _momenta(rng, m, n=32, extra=()):
    p3 = rng.normal(size=(n, 3)) * 300.0
    p3 = np.concatenate([p3] + [np.array(extra, dtype=float).reshape(-1, 3)], axis=0) if extra else p3
    E = np.sqrt(m * m + (p3 ** 2).sum(axis=1))
    return np.concatenate([E[:, None], p3], axis=1)


SPECIAL = [[0, 0, -200.0], [0, 0, 200.0], [1e-3, 0, -200.0], [0, 5.0, 0]]


@pytest.mark.parametrize("m", [0.0, 175.0])
def test_dirac_equation(m):
    rng = np.random.default_rng(1)
    p = _momenta(rng, m, extra=SPECIAL)
    ps = slash(p)
    one = np.eye(4)
    for lam in (-1, 1):
        u = u_spinor(p, lam)
        v = v_spinor(p, lam)
        r_u = np.einsum("nij,nj->ni", ps - m * one, u)
        r_v = np.einsum("nij,nj->ni", ps + m * one, v)
        scale = p[:, :1]
        assert np.abs(r_u / scale).max() < 1e-12
        assert np.abs(r_v / scale).max() < 1e-12


@pytest.mark.parametrize("m", [0.0, 80.4])
def test_helicity_eigenvalue(m):
    """Sigma . p^ u(p, l) = l u(p, l);  for v the spin is opposite: Sigma . p^ v = -l v."""
    rng = np.random.default_rng(2)
    p = _momenta(rng, m, extra=SPECIAL)
    n = p[:, 1:] / np.linalg.norm(p[:, 1:], axis=1, keepdims=True)
    pauli = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    Sig = np.einsum("nk,kij->nij", n, np.array(pauli))
    S4 = np.zeros((p.shape[0], 4, 4), dtype=complex)
    S4[:, :2, :2] = Sig
    S4[:, 2:, 2:] = Sig
    for lam in (-1, 1):
        u = u_spinor(p, lam)
        v = v_spinor(p, lam)
        assert np.abs(np.einsum("nij,nj->ni", S4, u) - lam * u).max() < 1e-9
        assert np.abs(np.einsum("nij,nj->ni", S4, v) + lam * v).max() < 1e-9


@pytest.mark.parametrize("m", [0.0, 175.0])
def test_normalisation_and_completeness(m):
    rng = np.random.default_rng(3)
    p = _momenta(rng, m, extra=SPECIAL)
    su = 0
    sv = 0
    for lam in (-1, 1):
        u, v = u_spinor(p, lam), v_spinor(p, lam)
        assert np.allclose(np.einsum("ni,ni->n", bar(u), u), 2 * m, atol=1e-9)
        assert np.allclose(np.einsum("ni,ni->n", bar(v), v), -2 * m, atol=1e-9)
        assert np.allclose(np.einsum("ni,ni->n", u.conj(), u), 2 * p[:, 0])
        su = su + np.einsum("ni,nj->nij", u, bar(u))
        sv = sv + np.einsum("ni,nj->nij", v, bar(v))
    one = np.eye(4)
    scale = p[:, 0][:, None, None]
    assert np.abs((su - (slash(p) + m * one)) / scale).max() < 1e-12
    assert np.abs((sv - (slash(p) - m * one)) / scale).max() < 1e-12


@pytest.mark.parametrize("m", [0.0, 80.4])
def test_polarisation_vectors(m):
    rng = np.random.default_rng(4)
    k = _momenta(rng, m, extra=SPECIAL)
    hels = (-1, 1) if m == 0 else (-1, 0, 1)
    proj = 0
    for lam in hels:
        e = polarisation(k, lam, mass=m)
        assert np.abs(mdot(k, e) / k[:, 0]).max() < 1e-12          # transversality
        assert np.allclose(mdot(e, e.conj()), -1.0, atol=1e-12)     # normalisation
        proj = proj + np.einsum("ni,nj->nij", e, e.conj())
        # helicity: (J . k^) eps = lam eps with (J_k)_{ij} = -i eps_{kij} on the spatial part
        n = k[:, 1:] / np.linalg.norm(k[:, 1:], axis=1, keepdims=True)
        J = np.zeros((3, 3, 3), dtype=complex)
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    J[a, b, c] = -1j * (a - b) * (b - c) * (c - a) / 2  # -i eps_{abc}
        Jn = np.einsum("nk,kij->nij", n, J)
        assert np.abs(np.einsum("nij,nj->ni", Jn, e[:, 1:]) - lam * e[:, 1:]).max() < 1e-12
    g = np.diag(METRIC)
    if m > 0:
        target = -g[None] + np.einsum("ni,nj->nij", k, k) / (m * m)
        assert np.abs(proj - target).max() < 1e-9 * np.abs(target).max()
    else:
        n = k[:, 1:] / np.linalg.norm(k[:, 1:], axis=1, keepdims=True)
        target = np.eye(3)[None] - np.einsum("ni,nj->nij", n, n)
        assert np.abs(proj[:, 1:, 1:] - target).max() < 1e-12


def test_boost_preserves_invariants():
    rng = np.random.default_rng(5)
    p = _momenta(rng, 10.0)
    q = _momenta(rng, 3.0)
    b = np.array([0.3, -0.5, 0.6])
    assert np.allclose(mdot(boost(p, b), boost(q, b)), mdot(p, q), rtol=1e-12)
