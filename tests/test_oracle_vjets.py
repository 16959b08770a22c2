"""Pins of the oracle's V + n jets processes (qqx_v_ng: q q~' > V + n gluons, every Feynman diagram,
the paper's Sect. 2.1 V + jets family): u d~ > W+ g g g and u u~ > Z g g g.

- The colour projector (an orthonormal basis of the colour space the diagrams span) gives the
  explicit sum over all colour indices, for random amplitudes.
- The same generic code at n = 1 and n = 2 equals the hand-written q q~ > V g (closed form) and
  q q~ > V g g oracles, point by point: couplings, colour tensors, signs and normalisation.
- n = 3: the Ward identity of each gluon (eps -> k gives zero on exactly on-shell inputs), which
  fixes the diagrams with two three-gluon vertices and the four-gluon vertex against the rest and
  fails when the four-gluon diagrams are dropped; Bose symmetry under every permutation of the
  gluons; boosts.
"""
import itertools

import numpy as np
import pytest

from oracle import colour, processes as pr
from oracle.sm import SMParams
from test_oracle_chains import _massive_points

PAR = SMParams()


def test_colour_projector_equals_the_explicit_colour_sum():
    rng = np.random.default_rng(700)
    for n in (2, 3):
        if n == 2:
            ts = [pr._colour_string([0, 1], 2), pr._colour_string([1, 0], 2),
                  pr._colour_string(["G"], 2, with_f=(0, 1))]
        else:
            ts = [pr._colour_string(list(o), 3) for o in itertools.permutations(range(3))][:4]
        B = colour.colour_projector(ts)
        A = [rng.normal(size=7) + 1j * rng.normal(size=7) for _ in ts]
        assert np.allclose(colour.colour_norm(A, B), colour.colour_sum(A, ts), rtol=1e-12)


@pytest.mark.parametrize("boson", ["w", "z"])
def test_generic_code_equals_the_one_and_two_gluon_oracles(boson):
    mV = PAR.mW if boson == "w" else PAR.mZ
    gl, gr = (PAR.g / np.sqrt(2.0), 0.0) if boson == "w" else pr._z_couplings("u", PAR)
    one = pr.udx_wpg if boson == "w" else pr.uux_zg
    two = pr.udx_wpgg if boson == "w" else pr.uux_zgg
    P1 = _massive_points(600.0, (mV, 0.0), 8, seed=710)
    assert np.allclose(pr.qqx_v_ng(P1, PAR, gl, gr, mV), one(P1, PAR), rtol=1e-12, atol=0)
    P2 = _massive_points(600.0, (mV, 0.0, 0.0), 8, seed=711)
    assert np.allclose(pr.qqx_v_ng(P2, PAR, gl, gr, mV), two(P2, PAR), rtol=1e-12, atol=0)


@pytest.mark.parametrize("which", ["udx_wpggg", "uux_zggg"])
def test_three_gluons_ward_bose_and_boosts(which):
    f = getattr(pr, which)
    mV = PAR.mW if which == "udx_wpggg" else PAR.mZ
    P = _massive_points(800.0, (mV, 0.0, 0.0, 0.0), 5, seed=720)
    ref = f(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (3, 4, 5):
        bad = f(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2), bad / (ref * P[:, leg, 0] ** 2)
    for perm in itertools.permutations((3, 4, 5)):
        assert np.allclose(f(P[:, [0, 1, 2] + list(perm)], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(f(random_lorentz(P, 721), PAR), ref, rtol=1e-10)


def test_ward_identity_catches_dropped_four_gluon_diagrams(monkeypatch):
    orig = pr._gluon_blocks
    monkeypatch.setattr(pr, "_gluon_blocks", lambda legs: [b for b in orig(legs) if b[0] != "quartic"])
    monkeypatch.setattr(pr, "_VJETS", {})
    P = _massive_points(800.0, (PAR.mW, 0.0, 0.0, 0.0), 3, seed=730)
    ref = pr.udx_wpggg(P, PAR)
    bad = pr.udx_wpggg(P, PAR, eps_override={3: P[:, 3]})
    assert np.all(np.abs(bad) > 1e-6 * ref * P[:, 3, 0] ** 2)
