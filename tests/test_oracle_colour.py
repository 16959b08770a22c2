"""Pins of the oracle's explicit SU(3) generators and brute-force colour sums."""
import itertools

import numpy as np

from oracle import colour


def test_lie_algebra_and_normalisation():
    T, F = colour.T, colour.F
    # Tr(t^a t^b) = delta/2 and [t^a, t^b] = i f^{abc} t^c
    assert np.allclose(np.einsum("aij,bji->ab", T, T), 0.5 * np.eye(8))
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    assert np.allclose(comm, 1j * np.einsum("abc,cik->abik", F, T))
    # totally antisymmetric, textbook values f^{123} = 1, f^{458} = sqrt(3)/2
    for p in itertools.permutations(range(3)):
        sign = np.linalg.det(np.eye(3)[list(p)])
        assert np.allclose(np.transpose(F, p), sign * F)
    assert np.isclose(F[0, 1, 2], 1.0)
    assert np.isclose(F[3, 4, 7], np.sqrt(3) / 2)
    # Casimirs C_F = 4/3, C_A = 3
    assert np.allclose(np.einsum("aij,ajk->ik", T, T), 4.0 / 3.0 * np.eye(3))
    assert np.allclose(np.einsum("acd,bcd->ab", F, F), 3.0 * np.eye(8))


def test_qqbar_gg_colour_matrix():
    """K for the colour strings (t^a t^b)_{ji}, (t^b t^a)_{ji}: [[16/3, -2/3], [-2/3, 16/3]]."""
    from oracle.processes import _colour_string
    cab = _colour_string([0, 1], 2)
    cba = _colour_string([1, 0], 2)
    C = np.array([c.ravel() for c in (cab, cba)])
    K = C @ C.conj().T
    assert np.allclose(K, [[16 / 3, -2 / 3], [-2 / 3, 16 / 3]])
    # f^{a0 a1 c} t^c = -i [t^a0, t^a1]; _colour_string([1, 0]) is (t^a0 t^a1) (gluon 1 inserted first)
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    assert np.allclose(cG, -1j * (cba - cab))


def test_four_gluon_trace_matrix_closed_form():
    """Tr(T T) = delta normalisation: Mangano-Parke closed forms for n = 4, N = 3."""
    orders, C = colour.gluon_trace_matrix(4)
    N = 3.0
    diag = (N * N - 1) * (N ** 4 - 3 * N * N + 3) / N ** 2
    adjacent = (N * N - 1) * (3 - N * N) / N ** 2
    reflected = (N * N - 1) * (N * N + 3) / N ** 2
    for s, a in enumerate(orders):
        for t, b in enumerate(orders):
            if a == b:
                want = diag
            elif b == (a[0],) + tuple(reversed(a[1:])):
                want = reflected
            else:
                want = adjacent
            assert np.isclose(C[s, t].real, want) and abs(C[s, t].imag) < 1e-12


def test_six_gluon_trace_matrix_properties():
    orders, C = colour.gluon_trace_matrix(6)
    assert C.shape == (120, 120)
    assert np.allclose(C, C.conj().T)
    assert np.abs(C.imag).max() < 1e-10
    assert np.linalg.eigvalsh(C).min() > -1e-9
    # rational with denominator dividing N^4 = 81
    assert np.abs(C.real * 81 - np.round(C.real * 81)).max() < 1e-8
    # second brute-force route for a few entries: explicit loop over all 8^6 colour labels
    Tn = np.sqrt(2.0) * colour.T
    labels = np.array(list(itertools.product(range(8), repeat=6)))

    def traces(order):
        M = Tn[labels[:, order[0]]]
        for leg in order[1:]:
            M = M @ Tn[labels[:, leg]]
        return np.trace(M, axis1=1, axis2=2)

    t0 = traces(orders[0])
    for t in (0, 1, 7, 59, 119):
        direct = np.sum(t0 * traces(orders[t]).conj())
        assert np.isclose(direct, C[0, t], rtol=1e-10, atol=1e-8)
    s = orders.index((0, 2, 4, 1, 5, 3))
    t = orders.index((0, 5, 1, 3, 2, 4))
    assert np.isclose(np.sum(traces(orders[s]) * traces(orders[t]).conj()), C[s, t], rtol=1e-10, atol=1e-8)


def test_u1_decoupling():
    """Sum of traces with one leg at every position of a fixed cyclic order of the rest vanishes."""
    Tn = np.sqrt(2.0) * colour.T
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = rng.integers(0, 8, size=4)
        # Tr(T^x T^a T^b T^c) + Tr(T^a T^x T^b T^c) + ... with x -> identity (U(1)) equals N-independent
        # cyclic-sum identity: sum over insertions of the identity gives 4 Tr(T^a T^b T^c); replace the
        # U(1) generator by 1/sqrt(N) * identity and check sum_positions Tr(...) = 4 Tr(abc)/sqrt(N)
        mats = [Tn[a[0]], Tn[a[1]], Tn[a[2]]]
        u1 = np.eye(3) / np.sqrt(3)
        tot = 0
        for pos in range(3):
            seq = mats[:pos] + [u1] + mats[pos:]
            tot += np.trace(seq[0] @ seq[1] @ seq[2] @ seq[3])
        assert np.isclose(tot, 3 * np.trace(mats[0] @ mats[1] @ mats[2]) / np.sqrt(3))
