"""Input preparation shared by the parity tests (no part of the method's arithmetic).

RAMBO's boosts, in FP64, leave a generated point off shell by up to ~1e-11 relative and unbalanced
by up to ~1e-9 GeV.  An evaluator that reads a mass from the energy and one that reads it from the
parameter card, or that routes an internal momentum through the other side of a diagram, then
legitimately differ at that level.  The parity tests therefore hand both sides momenta that are on
shell and balanced to FP64 rounding.
"""
import numpy as np


def consistent(P, masses):
    """P [N, n_ext, 4] with two massless incoming partons along +z and -z, made consistent to FP64
    rounding: the final-state three-momenta are kept except the last leg's transverse components,
    which are set by transverse balance; every final energy is recomputed on shell from masses
    (one per leg, incoming first); the incoming energies are re-solved from the final state's total
    energy and longitudinal momentum."""
    Q = np.array(P, dtype=np.float64, copy=True)
    m = np.asarray(masses, dtype=np.float64)
    Q[:, -1, 1:3] = -Q[:, 2:-1, 1:3].sum(axis=1)
    for k in range(2, Q.shape[1]):
        Q[:, k, 0] = np.sqrt(m[k] * m[k] + np.sum(Q[:, k, 1:] ** 2, axis=1))
    E = Q[:, 2:, 0].sum(axis=1)
    pz = Q[:, 2:, 3].sum(axis=1)
    ea, eb = 0.5 * (E + pz), 0.5 * (E - pz)
    Q[:, 0] = 0.0
    Q[:, 1] = 0.0
    Q[:, 0, 0], Q[:, 0, 3] = ea, ea
    Q[:, 1, 0], Q[:, 1, 3] = eb, -eb
    return Q


def conditioning(fn, P, ref, par, draws=4, seed=123):
    """The oracle's own spread under relative perturbations of its input momenta at the FP64
    rounding level (2^-52): how far any FP64 evaluation of P can be expected to move."""
    rng = np.random.default_rng(seed)
    spread = np.zeros_like(ref)
    for _ in range(draws):
        Q = P * (1 + 2.0 ** -52 * rng.standard_normal(P.shape))
        spread = np.maximum(spread, np.abs(fn(Q, par) - ref))
    return spread
