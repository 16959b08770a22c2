"""SU(3) colour by brute force over explicit generator components.

Oracle module (test infrastructure only).  t^a = lambda^a / 2 (Gell-Mann), so
Tr(t^a t^b) = delta^{ab}/2, and f^{abc} = -2i Tr([t^a, t^b] t^c).  Colour sums
are plain sums over all external colour indices of explicit tensors; no
Fierz identity or colour-basis algebra is used.  (The paper defers colour
summation to its QCD companion paper, Sect. 2; this is the plain definition.)

Parity: pinned by tests/test_oracle_colour.py (Lie algebra, normalisation,
Casimirs, known 2x2 colour matrix of q qbar g g, symmetry/PSD of the
six-gluon trace matrix, U(1) decoupling); colour_projector against colour_sum
in tests/test_oracle_vjets.py.
"""
import itertools
import numpy as np

_L = np.zeros((8, 3, 3), dtype=complex)
_L[0][0, 1] = _L[0][1, 0] = 1
_L[1][0, 1], _L[1][1, 0] = -1j, 1j
_L[2][0, 0], _L[2][1, 1] = 1, -1
_L[3][0, 2] = _L[3][2, 0] = 1
_L[4][0, 2], _L[4][2, 0] = -1j, 1j
_L[5][1, 2] = _L[5][2, 1] = 1
_L[6][1, 2], _L[6][2, 1] = -1j, 1j
_L[7][0, 0] = _L[7][1, 1] = 1 / np.sqrt(3)
_L[7][2, 2] = -2 / np.sqrt(3)

T = _L / 2.0  # t^a_{ij}, shape (8, 3, 3)

F = np.real(-2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T)))


def colour_sum(amps, tensors):
    """sum over all colour indices c of | sum_d c_d[c] A_d |^2.

    amps: list of D complex arrays [N]; tensors: list of D explicit colour
    tensors of identical shape (one axis per coloured external leg).  The
    colour-dressed amplitude is formed for every colour assignment and its
    modulus squared summed: the plain definition, with no colour matrix.
    """
    C = np.array([t.ravel() for t in tensors])  # [D, n_colours]
    A = np.stack(amps, axis=0)                   # [D, N]
    M = C.T @ A                                   # [n_colours, N]
    return np.sum(np.abs(M) ** 2, axis=0)


def colour_projector(tensors):
    """B (r x D) with sum over all colour indices c of |sum_d c_d[c] A_d|^2 = |B A|^2 for explicit
    diagram colour tensors c_d: the rows of the SVD C = U S Vh of the D x n_c matrix of tensors span
    the colour space the diagrams reach and C^T A = Vh^T S U^T A, so |C^T A| = |S U^T A| and
    B = S U^T (singular values above 1e-12 of the largest).  Taken once per process; per point and
    helicity the diagrams still combine linearly before the square, as in colour_sum.  (Vh^T has
    orthonormal columns, so |Vh^T y| = |y|.)"""
    C = np.array([t.ravel() for t in tensors])
    U, S, _ = np.linalg.svd(C, full_matrices=False)   # C = U S Vh: C^T A = Vh^T (S U^T A)
    keep = S > 1e-12 * S[0]
    return S[keep, None] * U[:, keep].T


def colour_norm(amps, B):
    """|B A|^2 summed over the colour components, for amps [D] of arrays [N]."""
    A = np.stack(amps, axis=0)
    return np.sum(np.abs(B @ A) ** 2, axis=0)


def trace_product(labels_matrices):
    """Tr of a product of 3x3 matrices."""
    M = np.eye(3, dtype=complex)
    for m in labels_matrices:
        M = M @ m
    return np.trace(M)


def gluon_trace_matrix(n):
    """C_{sigma,tau} = sum_{a_1..a_n} Tr(T^{a_1} T^{a_sigma2}..) Tr(T^{a_1} T^{a_tau2}..)^*

    with T^a = sqrt(2) t^a (Tr(T^a T^b) = delta^{ab}) and sigma, tau running
    over the (n-1)! orderings of legs 2..n (leg 1 first).  Returns
    (orderings, C).  Evaluated as a contraction of explicit generator
    components: every adjoint index a_k is summed with the 81-component
    tensor W_{ij,kl} = sum_a T^a_{ij} (T^a_{kl})^*.
    """
    Tn = np.sqrt(2.0) * T
    orders = [(0,) + p for p in itertools.permutations(range(1, n))]
    W = np.einsum("aij,akl->ijkl", Tn, Tn.conj())
    m = len(orders)
    index = {o: k for k, o in enumerate(orders)}
    # brute-force row for sigma = identity ordering
    row = np.zeros(m, dtype=complex)
    letters = "abcdefghijklmnopqrstuvwxyz"
    for t_, tau in enumerate(orders):
        pos_t = {leg: k for k, leg in enumerate(tau)}
        subs = []
        for leg in range(n):
            ps, pt = leg, pos_t[leg]
            subs.append(letters[ps] + letters[(ps + 1) % n] + letters[n + pt] + letters[n + (pt + 1) % n])
        row[t_] = np.einsum(",".join(subs) + "->", *([W] * n), optimize="greedy")
    # the sum over dummy colour labels is invariant under relabelling the legs,
    # so C(sigma, tau) = C(id, tau relabelled by leg -> position in sigma)
    C = np.zeros((m, m), dtype=complex)
    for s, sig in enumerate(orders):
        pos_s = {leg: k for k, leg in enumerate(sig)}
        for t_, tau in enumerate(orders):
            C[s, t_] = row[index[tuple(pos_s[leg] for leg in tau)]]
    return orders, C
