"""Pins of the oracle's one-fermion-line engine (fermion_line_process: a quark line with colourless
bosons and up to three incoming or outgoing gluons, every Feynman diagram) and of the process built on
it, g g > t t~ H g (H t t~ plus one jet, the paper's Sect. 2 Htt~ + jets family).

- The engine equals three independently written oracles point by point: g g > t t~ H (eight
  diagrams written out), g g > t t~ g (eighteen diagram terms written out, the four-gluon vertex
  among them) and u d~ > W+ g g g (q q~ > V + n gluons): crossing (incoming and outgoing gluons, a
  quark or antiquark at either end of the line), massive internal fermions with widths, scalar and
  vector insertions.
- g g > t t~ H g: the Ward identity of each gluon at zero top width (fixed-width top propagators break
  it at O(m Gamma / (p^2 - m^2))), Bose symmetry of the incoming gluons, boosts.
- V V plus jets (u u~ > Z Z g g) on the same engine: equal to u u~ > Z Z (closed form) and u u~ > Z Z g
  with no and one gluon; Ward identity of each gluon, Bose symmetry of the gluons and of the Z bosons,
  boosts.
- H V plus jets (u d~ > W+ H g g, the W* > W+ H insertion) on the same engine: equal to u d~ > W+ H
  (closed form) and u d~ > W+ H g with no and one gluon; Ward identity of each gluon, Bose symmetry,
  boosts.
- W+ W- plus jets (u u~ > W+ W- g g): the t-channel W pair in the order its d quark fixes, or an
  s-channel photon or Z into the W W V vertex, as alternatives whose diagrams add: equal to u u~ > W+ W-
  and u u~ > W+ W- g with no and one gluon; Ward identity of each gluon, Bose symmetry, boosts.
- W+ Z plus jets (u d~ > W+ Z g g): the Z with the u couplings before the W emission, with the d
  couplings after it, or an s-channel W into W W Z; equal to u d~ > W+ Z and u d~ > W+ Z g with no and
  one gluon; Ward identity of each gluon, Bose symmetry, boosts.
- H V plus three jets (u d~ > W+ H g g g): Ward identity of each gluon (fails without the four-gluon
  lines), Bose symmetry of the gluons, boosts.
- Four gluons (g g > t t~ g g, t t~ plus two jets): the recursive gluon trees built for three gluons
  reproduce g g > t t~ g, the vectorised colour tensors equal the explicit loop, and g g > t t~ g g
  satisfies each gluon's Ward identity at zero top width, Bose symmetry and boosts.
- WBF H plus jets on two quark lines (us_dch_ng, u s > d c H + n gluons): equal to u s > d c H and
  u s > d c H g at n = 0, 1; at n = 2 the Ward identity of each gluon (fails without the three-gluon
  pair lines), Bose symmetry, boosts.
"""
import numpy as np
import pytest

from oracle import processes as pr
from oracle.sm import SMParams
from test_oracle_chains import _massive_points

PAR = SMParams()


def test_engine_equals_the_written_out_oracles():
    mt = PAR.mt
    P = _massive_points(1000.0, (mt, mt, PAR.mH), 6, seed=800)
    got = pr.fermion_line_process(P, PAR, (3, "v"), (2, "ubar"), [dict(leg=4, kind="S", y=-mt / PAR.vev)],
                                  [(0, True), (1, True)], mt, PAR.wt, 1.0 / 256.0)
    assert np.allclose(got, pr.gg_ttxh(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(1000.0, (mt, mt, 0.0), 6, seed=801)
    got = pr.fermion_line_process(P, PAR, (3, "v"), (2, "ubar"), [], [(0, True), (1, True), (4, False)],
                                  mt, PAR.wt, 1.0 / 256.0)
    assert np.allclose(got, pr.gg_ttxg(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(800.0, (PAR.mW, 0.0, 0.0, 0.0), 6, seed=802)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"),
                                  [dict(leg=2, kind="V", gl=PAR.g / np.sqrt(2.0), gr=0.0, mass=PAR.mW)],
                                  [(3, False), (4, False), (5, False)], 0.0, 0.0, 1.0 / 36.0)
    assert np.allclose(got, pr.udx_wpggg(P, PAR), rtol=1e-12, atol=0)


def test_ttxhg_ward_bose_and_boosts():
    P = _massive_points(1500.0, (PAR.mt, PAR.mt, PAR.mH, 0.0), 5, seed=803)
    ref0 = pr.gg_ttxhg(P, PAR, widths=False)
    assert np.all(ref0 > 0) and np.all(np.isfinite(ref0))
    for leg in (0, 1, 5):
        bad = pr.gg_ttxhg(P, PAR, eps_override={leg: P[:, leg]}, widths=False)
        assert np.all(np.abs(bad) < 1e-24 * ref0 * P[:, leg, 0] ** 2)
    ref = pr.gg_ttxhg(P, PAR)
    assert np.allclose(pr.gg_ttxhg(P[:, [1, 0, 2, 3, 4, 5]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.gg_ttxhg(random_lorentz(P, 804), PAR), ref, rtol=1e-10)


def test_ward_identity_catches_dropped_triple_gluon_lines(monkeypatch):
    """Without the diagrams whose three gluons join through two three-gluon vertices the gluon Ward
    identity fails (a planted mistake in the engine's diagram set)."""
    orig = pr._gluon_blocks
    monkeypatch.setattr(pr, "_gluon_blocks", lambda legs: [b for b in orig(legs) if b[0] != "triple"])
    monkeypatch.setattr(pr, "_VJETS", {})
    P = _massive_points(1500.0, (PAR.mt, PAR.mt, PAR.mH, 0.0), 3, seed=805)
    ref0 = pr.gg_ttxhg(P, PAR, widths=False)
    bad = pr.gg_ttxhg(P, PAR, eps_override={5: P[:, 5]}, widths=False)
    assert np.all(np.abs(bad) > 1e-8 * ref0 * P[:, 5, 0] ** 2)


# ---------------------------------------------------------------------------
# WBF H plus jets: two quark lines (us_dch_ng)
# ---------------------------------------------------------------------------
def test_wbf_lines_equal_the_zero_and_one_gluon_oracles():
    """The two-line code with no gluon equals u s > d c H (closed-form pinned) and with one gluon
    u s > d c H g (Ward- and soft-limit-pinned), point by point."""
    P = _massive_points(1000.0, (0.0, 0.0, PAR.mH), 6, seed=900)
    assert np.allclose(pr.us_dch_ng(P, PAR), pr.us_dch(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(1000.0, (0.0, 0.0, PAR.mH, 0.0), 6, seed=901)
    assert np.allclose(pr.us_dch_ng(P, PAR), pr.us_dchg(P, PAR), rtol=1e-12, atol=0)


def test_wbf_h_two_jets_ward_bose_and_boosts():
    P = _massive_points(1000.0, (0.0, 0.0, PAR.mH, 0.0, 0.0), 5, seed=902)
    ref = pr.us_dchgg(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (5, 6):
        bad = pr.us_dchgg(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(pr.us_dchgg(P[:, [0, 1, 2, 3, 4, 6, 5]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.us_dchgg(random_lorentz(P, 903), PAR), ref, rtol=1e-10)


def test_wbf_ward_identity_catches_dropped_pair_lines(monkeypatch):
    """Without the diagrams whose two gluons join through the three-gluon vertex the Ward identity of
    a gluon fails."""
    orig = pr._gluon_blocks
    monkeypatch.setattr(pr, "_gluon_blocks", lambda legs: [b for b in orig(legs) if b[0] != "pair"])
    monkeypatch.setattr(pr, "_VJETS", {})
    P = _massive_points(1000.0, (0.0, 0.0, PAR.mH, 0.0, 0.0), 3, seed=904)
    ref = pr.us_dchgg(P, PAR)
    bad = pr.us_dchgg(P, PAR, eps_override={5: P[:, 5]})
    assert np.all(np.abs(bad) > 1e-8 * ref * P[:, 5, 0] ** 2)


# ---------------------------------------------------------------------------
# V V plus jets on the one-line engine: u u~ > Z Z g g
# ---------------------------------------------------------------------------
def test_zz_plus_jets_engine_equals_the_zero_and_one_gluon_oracles():
    gl, gr = pr._z_couplings("u", PAR)
    z = [dict(leg=k, kind="V", gl=gl, gr=gr, mass=PAR.mZ) for k in (2, 3)]
    P = _massive_points(500.0, (PAR.mZ, PAR.mZ), 6, seed=950)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), z, [], 0.0, 0.0, 1.0 / 36.0)
    assert np.allclose(got, pr.uux_zz(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(500.0, (PAR.mZ, PAR.mZ, 0.0), 6, seed=951)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), z, [(4, False)], 0.0, 0.0, 1.0 / 36.0)
    assert np.allclose(got, pr.uux_zzg(P, PAR), rtol=1e-12, atol=0)


def test_zzgg_ward_bose_and_boosts():
    P = _massive_points(600.0, (PAR.mZ, PAR.mZ, 0.0, 0.0), 5, seed=952)
    ref = pr.uux_zzgg(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (4, 5):
        bad = pr.uux_zzgg(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(pr.uux_zzgg(P[:, [0, 1, 2, 3, 5, 4]], PAR), ref, rtol=1e-12)
    assert np.allclose(pr.uux_zzgg(P[:, [0, 1, 3, 2, 4, 5]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.uux_zzgg(random_lorentz(P, 953), PAR), ref, rtol=1e-10)


# ---------------------------------------------------------------------------
# H V plus jets on the one-line engine: u d~ > W+ H g g (a W* > W+ H insertion)
# ---------------------------------------------------------------------------
def _wh(par):
    return dict(kind="VS", legs=(2, 3), gl=par.g / np.sqrt(2.0), gr=0.0, mass=par.mW, width=par.wW, gvvs=par.gwwh)


def test_wh_plus_jets_engine_equals_the_zero_and_one_gluon_oracles():
    P = _massive_points(500.0, (PAR.mW, PAR.mH), 6, seed=960)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), [_wh(PAR)], [], 0.0, 0.0, 1.0 / 36.0)
    assert np.allclose(got, pr.udx_wph(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(600.0, (PAR.mW, PAR.mH, 0.0), 6, seed=961)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), [_wh(PAR)], [(4, False)], 0.0, 0.0, 1.0 / 36.0)
    assert np.allclose(got, pr.udx_wphg(P, PAR), rtol=1e-12, atol=0)


def test_whgg_ward_bose_and_boosts():
    P = _massive_points(700.0, (PAR.mW, PAR.mH, 0.0, 0.0), 5, seed=962)
    ref = pr.udx_wphgg(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (4, 5):
        bad = pr.udx_wphgg(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(pr.udx_wphgg(P[:, [0, 1, 2, 3, 5, 4]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.udx_wphgg(random_lorentz(P, 963), PAR), ref, rtol=1e-10)


# ---------------------------------------------------------------------------
# W+ W- plus jets: t-channel W pair in fixed order, or an s-channel photon or Z (alternatives)
# ---------------------------------------------------------------------------
def test_wpwm_plus_jets_engine_equals_the_zero_and_one_gluon_oracles():
    alts = pr.wpwm_line_alternatives(PAR)
    P = _massive_points(500.0, (PAR.mW, PAR.mW), 6, seed=970)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), None, [], 0.0, 0.0, 1.0 / 36.0,
                                  alternatives=alts, keep_order=True)
    assert np.allclose(got, pr.uux_wpwm(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(600.0, (PAR.mW, PAR.mW, 0.0), 6, seed=971)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), None, [(4, False)], 0.0, 0.0, 1.0 / 36.0,
                                  alternatives=alts, keep_order=True)
    assert np.allclose(got, pr.uux_wpwmg(P, PAR), rtol=1e-12, atol=0)


def test_wpwmgg_ward_bose_and_boosts():
    # points whose gluons pass the jet cuts (pT > 20 GeV): a gluon nearly collinear with a quark makes an
    # almost on-shell propagator that amplifies rounding in the individual diagrams
    P = _massive_points(700.0, (PAR.mW, PAR.mW, 0.0, 0.0), 16, seed=972)
    pt = np.hypot(P[:, 4:, 1], P[:, 4:, 2])
    P = P[np.all(pt > 20.0, axis=1)][:5]
    assert len(P) == 5
    ref = pr.uux_wpwmgg(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (4, 5):
        bad = pr.uux_wpwmgg(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(pr.uux_wpwmgg(P[:, [0, 1, 2, 3, 5, 4]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.uux_wpwmgg(random_lorentz(P, 973), PAR), ref, rtol=1e-10)


# ---------------------------------------------------------------------------
# W+ Z plus jets: the Z with the u couplings before the W emission, the d couplings after it, or an
# s-channel W into W W Z
# ---------------------------------------------------------------------------
def test_wpz_plus_jets_engine_equals_the_zero_and_one_gluon_oracles():
    alts = pr.wpz_line_alternatives(PAR)
    P = _massive_points(500.0, (PAR.mW, PAR.mZ), 6, seed=980)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), None, [], 0.0, 0.0, 1.0 / 36.0,
                                  alternatives=alts, keep_order=True)
    assert np.allclose(got, pr.udx_wpz(P, PAR), rtol=1e-12, atol=0)
    P = _massive_points(600.0, (PAR.mW, PAR.mZ, 0.0), 6, seed=981)
    got = pr.fermion_line_process(P, PAR, (0, "u"), (1, "vbar"), None, [(4, False)], 0.0, 0.0, 1.0 / 36.0,
                                  alternatives=alts, keep_order=True)
    assert np.allclose(got, pr.udx_wpzg(P, PAR), rtol=1e-12, atol=0)


def test_wpzgg_ward_bose_and_boosts():
    P = _massive_points(700.0, (PAR.mW, PAR.mZ, 0.0, 0.0), 16, seed=982)
    pt = np.hypot(P[:, 4:, 1], P[:, 4:, 2])
    P = P[np.all(pt > 20.0, axis=1)][:5]
    assert len(P) == 5
    ref = pr.udx_wpzgg(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (4, 5):
        bad = pr.udx_wpzgg(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(pr.udx_wpzgg(P[:, [0, 1, 2, 3, 5, 4]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.udx_wpzgg(random_lorentz(P, 983), PAR), ref, rtol=1e-10)


def test_whggg_ward_bose_and_boosts():
    """H V plus three jets (the engine with three gluons and the W* > W+ H insertion)."""
    P = _massive_points(900.0, (PAR.mW, PAR.mH, 0.0, 0.0, 0.0), 16, seed=990)
    pt = np.hypot(P[:, 4:, 1], P[:, 4:, 2])
    P = P[np.all(pt > 20.0, axis=1)][:4]
    assert len(P) == 4
    ref = pr.udx_wphggg(P, PAR)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    for leg in (4, 5, 6):
        bad = pr.udx_wphggg(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(np.abs(bad) < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(pr.udx_wphggg(P[:, [0, 1, 2, 3, 6, 4, 5]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.udx_wphggg(random_lorentz(P, 991), PAR), ref, rtol=1e-10)


def test_whggg_ward_identity_catches_dropped_four_gluon_lines(monkeypatch):
    orig = pr._gluon_blocks
    monkeypatch.setattr(pr, "_gluon_blocks", lambda legs: [b for b in orig(legs) if b[0] != "quartic"])
    monkeypatch.setattr(pr, "_VJETS", {})
    P = _massive_points(900.0, (PAR.mW, PAR.mH, 0.0, 0.0, 0.0), 3, seed=992)
    ref = pr.udx_wphggg(P, PAR)
    bad = pr.udx_wphggg(P, PAR, eps_override={4: P[:, 4]})
    assert np.all(np.abs(bad) > 1e-8 * ref * P[:, 4, 0] ** 2)


# ---------------------------------------------------------------------------
# four gluons: recursive gluon trees and vectorised colour tensors (t t~ plus two jets)
# ---------------------------------------------------------------------------
def test_gluon_trees_at_three_gluons_reproduce_gg_ttxg(monkeypatch):
    """The recursive trees (three- and four-gluon vertices joining sub-blocks) built for a set of three
    gluons in place of the written-out triple and quartic blocks give g g > t t~ g point by point: the
    tree currents, their momenta and their colour (adjoint vectors) as the four-gluon case uses them."""
    orig = pr._gluon_blocks
    monkeypatch.setattr(pr, "_gluon_blocks", lambda legs: pr._gluon_trees(legs) if len(legs) == 3 else orig(legs))
    monkeypatch.setattr(pr, "_VJETS", {})
    P = _massive_points(1000.0, (PAR.mt, PAR.mt, 0.0), 5, seed=801)
    got = pr.fermion_line_process(P, PAR, (3, "v"), (2, "ubar"), [], [(0, True), (1, True), (4, False)],
                                  PAR.mt, PAR.wt, 1.0 / 256.0)
    assert np.allclose(got, pr.gg_ttxg(P, PAR), rtol=1e-12, atol=0)


def test_vectorised_colour_tensor_equals_the_explicit_loop():
    import itertools
    rng = np.random.default_rng(11)
    for blocks in ([("g", 2), ("pair", (0, 1))], [("quartic", ((0, 1, 2), 1))], [("triple", (0, 2, 1))],
                   [("g", 1), ("g", 0), ("g", 2)]):
        T3 = pr._line_colour_tensor(blocks, 3)
        for _ in range(20):
            a = tuple(int(x) for x in rng.integers(0, 8, 3))
            M = np.eye(3, dtype=complex)
            for k, sp in blocks:
                M = pr._block_colour(k, sp, a) @ M
            assert np.allclose(T3[(slice(None), slice(None)) + a], M.T, atol=1e-14)
    assert len(pr._gluon_trees((0, 1, 2, 3))) == 45   # 15 cubic trees, 10 with a quartic vertex x 3


def test_ttxgg_ward_bose_and_boosts():
    P = _massive_points(1500.0, (PAR.mt, PAR.mt, 0.0, 0.0), 12, seed=1000)
    pt = np.hypot(P[:, 4:, 1], P[:, 4:, 2])
    P = P[np.all(pt > 20.0, axis=1)][:3]
    assert len(P) == 3
    ref0 = pr.gg_ttxgg(P, PAR, widths=False)
    assert np.all(ref0 > 0) and np.all(np.isfinite(ref0))
    for leg in (0, 5):
        bad = pr.gg_ttxgg(P, PAR, eps_override={leg: P[:, leg]}, widths=False)
        assert np.all(np.abs(bad) < 1e-24 * ref0 * P[:, leg, 0] ** 2)
    ref = pr.gg_ttxgg(P, PAR)
    assert np.allclose(pr.gg_ttxgg(P[:, [0, 1, 2, 3, 5, 4]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.gg_ttxgg(random_lorentz(P, 1001), PAR), ref, rtol=1e-10)
