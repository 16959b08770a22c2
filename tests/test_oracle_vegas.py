"""Pins of the oracle's adaptive grid (oracle.vegas, VEGAS of Lepage 1978).

The map is pinned by the change of variables it must preserve (exact integrals
of polynomials through random grids), the equal-bin grid is the identity, and
refinement by its fixed points: a flat histogram leaves any grid unchanged, and
for f(x) = 2x the grid approaches the density proportional to |f| (edges
sqrt(k/N)).  End to end, the adapted sigma-hat of u u~ > e+ e- agrees with the
closed-form integral and its error falls below that of uniform sampling.
"""
import math

import numpy as np
import pytest

from oracle import vegas, xsec
from oracle.sm import SMParams

PAR = SMParams()


def random_grid(rng, D, N):
    w = rng.uniform(0.2, 1.0, size=(D, N))
    e = np.concatenate([np.zeros((D, 1)), np.cumsum(w, axis=1)], axis=1)
    return e / e[:, -1:]


def test_equal_bins_are_the_identity():
    g = vegas.uniform_grid(3, 16)
    y = np.random.default_rng(1).random((1000, 3))
    x, jac, b = vegas.vegas_map(g, y)
    assert np.abs(x - y).max() < 1e-15
    assert np.abs(jac - 1).max() < 1e-14
    assert np.array_equal(b, np.floor(y * 16).astype(int))


@pytest.mark.parametrize("seed", [2, 3])
def test_change_of_variables_is_exact(seed):
    """int_0^1 J(y) f(x(y)) dy = int_0^1 f(x) dx for a polynomial f, per y-bin by Gauss-Legendre."""
    rng = np.random.default_rng(seed)
    N = 12
    g = random_grid(rng, 1, N)
    c = rng.normal(size=6)  # f(x) = sum c_k x^k
    xq, wq = np.polynomial.legendre.leggauss(8)
    total = 0.0
    for i in range(N):
        y = (i + 0.5 * (xq + 1)) / N          # Gauss points inside y-bin i
        x, jac, b = vegas.vegas_map(g, y[:, None])
        assert np.all(b[:, 0] == i)
        f = np.polyval(c[::-1], x[:, 0])
        total += np.sum(0.5 * wq / N * jac * f)
    exact = sum(ck / (k + 1) for k, ck in enumerate(c))
    assert total == pytest.approx(exact, rel=1e-13, abs=1e-13)


def test_map_is_monotone_and_covers_the_unit_interval():
    rng = np.random.default_rng(4)
    g = random_grid(rng, 2, 20)
    y = np.sort(rng.random((5000, 1)), axis=0).repeat(2, axis=1)
    x, jac, _ = vegas.vegas_map(g, y)
    assert np.all(np.diff(x, axis=0) >= 0)
    assert np.all((x > 0) & (x < 1)) and np.all(jac > 0)


def test_flat_histogram_keeps_the_grid():
    rng = np.random.default_rng(5)
    g = random_grid(rng, 3, 10)
    new = vegas.refine(g, np.ones((3, 10)), alpha=1.5)
    assert np.abs(new - g).max() < 1e-15


def test_refinement_invariants_and_empty_dimensions():
    rng = np.random.default_rng(6)
    g = vegas.uniform_grid(3, 16)
    d = rng.random((3, 16)) ** 4
    d[2] = 0.0
    new = vegas.refine(g, d, alpha=1.0)
    assert np.all(new[:, 0] == 0) and np.all(new[:, -1] == 1)
    assert np.all(np.diff(new, axis=1) > 0)
    assert np.array_equal(new[2], g[2])                 # no points: unchanged
    assert not np.allclose(new[0], g[0])


def test_grid_approaches_the_density_of_abs_f():
    """f(x) = 2x: points uniform in y give bin sums proportional to width * int_bin f^2 dx,
    equal when the bin density is proportional to |f| (edges sqrt(k/N)).  Ten refinements
    bring the grid there (the three-point smoothing shifts the first edge slightly), with
    bins narrowing where f grows.  (Smoothing hides an alternating bin pattern from the sums,
    so far longer exact-sum iterations drift; in use VEGAS runs a few iterations.)"""
    N = 32
    g = vegas.uniform_grid(1, N)
    for _ in range(10):
        x = g[0]
        d = (x[1:] - x[:-1]) * (4.0 / 3.0) * (x[1:] ** 3 - x[:-1] ** 3)
        g = vegas.refine(g, d[None, :], alpha=1.0)
    target = np.sqrt(np.arange(N + 1) / N)
    assert np.abs(g[0] - target).max() < 0.03
    assert np.abs(g[0] - target)[4:].max() < 0.01
    assert np.all(np.diff(np.diff(g[0][1:])) < 0)


def test_histogram_sums_squared_weights_per_bin():
    bins = np.array([[0, 2], [1, 2], [0, 0]])
    w = np.array([1.0, 2.0, 3.0])
    h = vegas.histogram(2, 3, bins, w)
    assert np.array_equal(h, [[10.0, 4.0, 0.0], [9.0, 0.0, 5.0]])


def test_adapted_sigma_matches_closed_form_and_reduces_the_error():
    """u u~ > e+ e- at 500 GeV: five adaptation rounds, then sigma-hat against the
    Gauss-Legendre integral of the closed form, and its error against uniform sampling."""
    from oracle import processes as pr
    kin = {"kind": "2to2", "sqrt_s": 500.0}
    n = 4000
    grid = vegas.uniform_grid(xsec.grid_dims(kin), 16)
    for it in range(5):
        P, W, S, T, bins = xsec.generate_grid(kin, PAR, 0, np.arange(it * n, (it + 1) * n), grid)
        w = W * pr.uux_epem(P, PAR) / (2 * S) * 0.3893793721e9
        grid = vegas.refine(grid, vegas.histogram(2, 16, bins, w), alpha=1.5)
    ev = np.arange(10 ** 6, 10 ** 6 + n)
    P, W, S, T, _ = xsec.generate_grid(kin, PAR, 0, ev, grid)
    sig, err = xsec.estimate(*[xsec.accumulate(pr.uux_epem(P, PAR), W, S, T, 1.0)[k] for k in (0, 1, 3)])
    P0, W0, S0, T0 = xsec.generate(kin, PAR, 0, ev)
    sig0, err0 = xsec.estimate(*[xsec.accumulate(pr.uux_epem(P0, PAR), W0, S0, T0, 1.0)[k] for k in (0, 1, 3)])
    x, wq = np.polynomial.legendre.leggauss(64)
    Q = np.zeros((64, 4, 4))
    Q[:, 0] = [250, 0, 0, 250]
    Q[:, 1] = [250, 0, 0, -250]
    Q[:, 3, 0] = 250
    Q[:, 3, 1] = 250 * np.sqrt(1 - x * x)
    Q[:, 3, 3] = 250 * x
    Q[:, 2, 0] = 250
    Q[:, 2, 1:] = -Q[:, 3, 1:]
    exact = np.sum(wq * pr.uux_epem(Q, PAR) / (32 * math.pi * 500.0 ** 2) * 0.3893793721e9)
    assert abs(sig - exact) < 4 * err
    assert err < 0.6 * err0
