"""Pins of the paper's phase-space parametrisation (Eq. 13, App. A.1, Eq. 17, App. A.2) and its cuts
(Eqs. 8-11), as the oracle implements them at fixed partonic energy.

- Two bodies: the weights integrate (Gauss-Legendre over the pT uniform, split where the rapidity
  range starts to bind) to the closed form of the massless two-body phase space inside the pT and
  rapidity ranges, (c_lo - c_hi) / (8 pi), c = min(tanh y_max, sqrt(1 - 4 pT^2 / s)).
- Three and four massless bodies: the weights' mean equals RAMBO's volume times its acceptance of
  the same ranges (statistical, independent samples).
- A resonance object: the weights' mean equals the resonance-mapped RAMBO estimate of the same
  integral (statistical).
- Every point conserves momentum and is on shell; the free objects respect their ranges.
- The cuts of Eqs. 8-11 on configurations whose answers follow from the definitions by hand.
"""
import math

import numpy as np
import pytest

from oracle import phasespace as ps

W = 1000.0


def _obj(legs, y_max, pt_min, pt_max, **kw):
    d = dict(legs=legs, y_max=y_max, pt_min=pt_min, pt_max=pt_max)
    d.update(kw)
    return d


@pytest.mark.parametrize("y_max,pt_max", [(5.0, 400.0), (1.0, 400.0), (0.7, 450.0), (0.5, 300.0)])
def test_two_body_weights_integrate_to_the_closed_form(y_max, pt_max):
    pt_min = 20.0
    objs = [_obj((0,), y_max, pt_min, pt_max), _obj((1,), y_max, pt_min, pt_max)]
    L0, L1 = math.log(pt_min ** 2), math.log(pt_max ** 2)
    # the rapidity bound starts to cut at pT_b = (w / 2) / cosh(y_max): split the quadrature there
    ptb = 0.5 * W / math.cosh(y_max)
    cuts = [0.0, 1.0]
    if pt_min < ptb < pt_max:
        cuts = [0.0, (math.log(ptb ** 2) - L0) / (L1 - L0), 1.0]
    x, wq = np.polynomial.legendre.leggauss(200)
    tot = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        uu = a + (b - a) * (x + 1) / 2
        for branch in (0.25, 0.75):  # the two rapidity solutions, each chosen with probability 1/2
            u = np.zeros((len(uu), 3))
            u[:, 0], u[:, 1], u[:, 2] = uu, 0.3, branch
            _, w, _ = ps.ypt_phi(W, objs, 2, u)
            tot += 0.5 * (b - a) / 2 * np.sum(wq * w)
    c = lambda pt: min(math.tanh(y_max), math.sqrt(max(1.0 - 4.0 * pt * pt / (W * W), 0.0)))
    ref = (c(pt_min) - c(pt_max)) / (8.0 * math.pi)
    if ref == 0.0:
        assert tot == 0.0
    else:
        assert tot == pytest.approx(ref, rel=1e-10)


def _ranges_ok(pf, objs):
    ok = np.ones(pf.shape[0], dtype=bool)
    for o in objs:
        p = pf[:, o["legs"][0]] if len(o["legs"]) == 1 else pf[:, o["legs"][0]] + pf[:, o["legs"][1]]
        pt = np.hypot(p[:, 1], p[:, 2])
        y = 0.5 * np.log((p[:, 0] + p[:, 3]) / (p[:, 0] - p[:, 3]))
        ok &= (np.abs(y) <= o["y_max"]) & (pt >= o["pt_min"]) & (pt <= o["pt_max"])
    return ok


@pytest.mark.parametrize("nf", [3, 4])
def test_massless_weights_against_rambo(nf):
    objs = [_obj((k,), 2.0, 30.0, 450.0) for k in range(nf)]
    n = 2000000
    rng = np.random.default_rng(40 + nf)
    pf, w, ok = ps.ypt_phi(W, objs, nf, rng.random((n, ps.ypt_uniforms(objs))))
    assert np.all(_ranges_ok(pf[ok], objs))
    est, err = w.mean(), w.std() / math.sqrt(n)
    q, wr = ps.rambo_massless(W, nf, rng.random((n, 4 * nf)))
    acc = _ranges_ok(q, objs)
    ref, rerr = wr[0] * acc.mean(), wr[0] * acc.std() / math.sqrt(n)
    assert abs(est - ref) < 5.0 * math.hypot(err, rerr), (est, err, ref, rerr)
    assert err < 0.02 * est


def test_resonance_object_against_resonance_rambo():
    """u d~ > e+ ve g g layout: gluons (2, 3) of the final legs free, the W -> e+ ve pair (0, 1) the
    balancing resonance object; the same integral from the resonance-mapped RAMBO."""
    objs = [_obj((2,), 2.5, 20.0, 480.0), _obj((3,), 2.5, 20.0, 480.0),
            _obj((0, 1), 4.0, 0.0, 480.0, res_mass=80.4, res_width=2.085)]
    n = 400000
    rng = np.random.default_rng(50)
    pf, w, ok = ps.ypt_phi(W, objs, 4, rng.random((n, ps.ypt_uniforms(objs))))
    assert np.all(_ranges_ok(pf[ok], objs))
    est, err = w.mean(), w.std() / math.sqrt(n)
    q, wr, okr = ps.rambo_resonance(W, 4, 80.4, 2.085, rng.random((n, 15)))
    acc = okr & _ranges_ok(q, objs)
    vals = np.where(acc, wr, 0.0)
    ref, rerr = vals.mean(), vals.std() / math.sqrt(n)
    assert abs(est - ref) < 5.0 * math.hypot(err, rerr), (est, err, ref, rerr)


def test_points_conserve_momentum_and_are_on_shell():
    objs = [_obj((0,), 2.5, 20.0, 480.0), _obj((3,), 2.5, 20.0, 480.0, mass=5.0),
            _obj((1, 2), 3.0, 0.0, 480.0, res_mass=91.19, res_width=2.5)]
    u = np.random.default_rng(60).random((5000, ps.ypt_uniforms(objs)))
    pf, w, ok = ps.ypt_phi(W, objs, 4, u)
    assert ok.mean() > 0.3
    pf = pf[ok]
    tot = pf.sum(axis=1)
    assert np.abs(tot - np.array([W, 0, 0, 0])).max() < 1e-9 * W
    m2 = pf[:, :, 0] ** 2 - (pf[:, :, 1:] ** 2).sum(axis=2)
    assert np.abs(m2[:, [0, 1, 2]]).max() < 1e-9 * W * W
    assert np.abs(m2[:, 3] - 25.0).max() < 1e-9 * W * W


def _jet(pt, eta, phi):
    return np.array([pt * math.cosh(eta), pt * math.cos(phi), pt * math.sin(phi), pt * math.sinh(eta)])


def test_paper_cuts_by_hand():
    J, B, L = ps.JET, ps.BJET, ps.LEPTON
    cases = [
        # two jets at pT 30 and 25: pT_ij = 25 Delta R; Delta R 0.7 -> 17.5 fails, 0.9 -> 22.5 passes
        ([_jet(30, 0.0, 0.0), _jet(25, 0.7, 0.0)], [J, J], False),
        ([_jet(30, 0.0, 0.0), _jet(25, 0.0, 0.9)], [J, J], True),
        ([_jet(30, 0.3, 0.5), _jet(25, 0.3 + 0.6, 0.5 + 0.6)], [J, J], True),   # Delta R = 0.849: 21.2
        ([_jet(30, 0.3, 0.5), _jet(25, 0.3 + 0.5, 0.5 + 0.5)], [J, J], False),  # Delta R = 0.707: 17.7
        # jets reach |eta| < 5, b jets and leptons |eta| < 2.5; all pT > 20
        ([_jet(30, 4.9, 0.0), _jet(30, -4.9, 3.0)], [J, J], True),
        ([_jet(30, 5.1, 0.0), _jet(30, 0.0, 3.0)], [J, J], False),
        ([_jet(30, 2.6, 0.0), _jet(30, 0.0, 3.0)], [B, J], False),
        ([_jet(30, 2.4, 0.0), _jet(30, 0.0, 3.0)], [L, J], True),
        ([_jet(19.9, 0.0, 0.0), _jet(30, 0.0, 3.0)], [L, J], False),
        # leptons and b jets are not isolated: close to a jet is allowed
        ([_jet(30, 0.0, 0.0), _jet(30, 0.05, 0.05)], [L, J], True),
        ([_jet(30, 0.0, 0.0), _jet(30, 0.05, 0.05)], [B, J], True),
        # a leg without a class is not cut
        ([_jet(1.0, 7.0, 0.0), _jet(30, 0.0, 3.0)], [0, J], True),
    ]
    for legs, cls, want in cases:
        P = np.array(legs)[None]
        assert bool(ps.pass_paper_cuts(P, cls)[0]) == want, (cls, want)
