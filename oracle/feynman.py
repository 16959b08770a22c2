"""Textbook Feynman-rule building blocks (numpy, FP64, vectorised over events).

Oracle module (test infrastructure only).  Every function returns a factor of
"i M" exactly as the Feynman rules write it (vertex factors and propagators
carry their own factors of i); the caller divides the product by i.

Rules (the Lagrangians of Sect. 4.2, Eqs. 22-40, written in the textbook
form with D_mu = d_mu - i g_s t^a A^a_mu):
  fermion propagator        i (qslash + m) / (q^2 - m^2 + i m w)
  massless vector (Feynman) -i g^{mu nu} / q^2
  massive vector (unitary)  -i (g^{mu nu} - q^mu q^nu / (m^2 - i m w)) / (q^2 - m^2 + i m w)
  scalar                    i / (q^2 - m^2 + i m w)
  FFV vertex                i gamma^mu (gL P_L + gR P_R)
  ggg vertex (all momenta incoming, colour f^{abc} stripped)
      g_s [ g^{mu nu}(k1-k2)^rho + g^{nu rho}(k2-k3)^mu + g^{rho mu}(k3-k1)^nu ]

Parity: pinned through the processes built from them (closed forms, Ward
identity, boost invariance) in tests/test_oracle_processes.py.
"""
import numpy as np

from .lorentz import GAMMA, PL, PR, mdot, slash


def den(q2, m, w):
    return q2 - m * m + 1j * m * w


def fermion_prop(q, m=0.0, w=0.0):
    """i (qslash + m) / (q^2 - m^2 + i m w), [N, 4, 4]."""
    num = slash(q) + m * np.eye(4)
    return 1j * num / den(mdot(q, q), m, w)[..., None, None]


def vector_prop(q, X, m=0.0, w=0.0):
    """Apply the vector propagator to a vertex output X^nu (upper index) -> upper index."""
    q2 = mdot(q, q)
    if m == 0.0:
        return -1j * X / q2[..., None]
    mc2 = m * m - 1j * m * w
    Y = X - q * (mdot(q, X) / mc2)[..., None]
    return -1j * Y / den(q2, m, w)[..., None]


def scalar_prop(q, m, w=0.0):
    return 1j / den(mdot(q, q), m, w)


def chiral(gl, gr):
    return gl * PL + gr * PR


def ffv_current(row, col, gl, gr):
    """J^mu = row . (i gamma^mu (gl P_L + gr P_R)) . col  (upper index), [N, 4]."""
    G = np.einsum("mij,jk->mik", GAMMA, chiral(gl, gr))
    return 1j * np.einsum("ni,mij,nj->nm", row, G, col)


def vector_insertion(X, gl, gr):
    """i Xslash (gl P_L + gr P_R) for a vector wavefunction X^mu, [N, 4, 4]."""
    return 1j * slash(X) @ chiral(gl, gr)


def fermion_line(row, col, p_start, inserts, m=0.0, w=0.0):
    """row . Gamma_n S(q_{n-1}) ... S(q_1) Gamma_1 . col.

    col is the spinor at the start of the fermion-number arrow, carrying
    momentum p_start along the arrow; inserts is an ordered list of
    (Gamma_k [N,4,4], Q_k [N,4]) with Q_k the four-momentum that leaves the
    line at insertion k.  The propagator after insertion k carries
    q_k = p_start - Q_1 - ... - Q_k and mass m, width w.
    """
    vec = col
    q = p_start.copy()
    for k, (G, Q) in enumerate(inserts):
        vec = np.einsum("nij,nj->ni", G, vec)
        q = q - Q
        if k < len(inserts) - 1:
            vec = np.einsum("nij,nj->ni", fermion_prop(q, m, w), vec)
    return np.einsum("ni,ni->n", row, vec)


def vvv_out(V1, k1, V2, k2, k3, g):
    """ggg vertex with legs 1, 2 contracted: output vector (upper index) for leg 3.

    All three momenta incoming to the vertex.
    """
    d12 = (k1 - k2)
    d23 = (k2 - k3)
    d31 = (k3 - k1)
    return g * (mdot(V1, V2)[..., None] * d12 + V2 * mdot(d23, V1)[..., None] + V1 * mdot(d31, V2)[..., None])
