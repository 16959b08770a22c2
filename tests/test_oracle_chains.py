"""Pins that tie the oracle's multi-leg processes to simpler, independently pinned ones.

- u s > d c h h: its W W > h h core (the code it runs) against the zero-momentum Higgs
  theorem: a Higgs boson of zero four-momentum couples like a shift of the vacuum value v,
  so the W W H H Green function with one such Higgs equals the v-derivative of the W W H
  Green function (every coupling and every mass, m_W^2 = g^2 v^2 / 4 and the Higgs curvature
  m_H^2(v) = lambda (3 v^2 - v0^2), differentiated).  Each of the four diagrams is one term
  of that derivative, so a wrong sign or coupling in any of them fails.
- u d~ > e+ ve g g: its normalisation through the soft-gluon chain u d~ > e+ ve (closed form)
  <- u d~ > e+ ve g <- u d~ > e+ ve g g, with the colour-correlated eikonal factor of three
  coloured partons.
- g g > g g g g: the Ward identity of each final gluon (the NMHV helicities included).
"""
import math

import numpy as np
import pytest

from oracle import phasespace as ps, processes as pr
from oracle.feynman import ffv_current, vector_prop
from oracle.lorentz import bar, boost, mdot, u_spinor
from oracle.sm import SMParams

PAR = SMParams()


# ---------------------------------------------------------------------------
# u s > d c h h: zero-momentum Higgs theorem for the W W > h h core
# ---------------------------------------------------------------------------
def _currents(n, seed):
    """Off-shell W momenta q1, q2 from u > d and s > c quark lines, and their V-A currents."""
    rng = np.random.default_rng(seed)
    def massless(E, c, phi):
        s = np.sqrt(1 - c * c)
        return np.stack([E, E * s * np.cos(phi), E * s * np.sin(phi), E * c], axis=1)
    p0 = massless(rng.uniform(200, 400, n), np.full(n, 1.0), np.zeros(n))
    p1 = massless(rng.uniform(200, 400, n), np.full(n, -1.0), np.zeros(n))
    p2 = massless(rng.uniform(100, 200, n), rng.uniform(-0.8, 0.8, n), rng.uniform(0, 6.28, n))
    p3 = massless(rng.uniform(100, 200, n), rng.uniform(-0.8, 0.8, n), rng.uniform(0, 6.28, n))
    gw = PAR.g / math.sqrt(2.0)
    J1 = ffv_current(bar(u_spinor(p2, -1)), u_spinor(p0, -1), gw, 0.0)
    J2 = ffv_current(bar(u_spinor(p3, -1)), u_spinor(p1, -1), gw, 0.0)
    return p0 - p2, p1 - p3, J1, J2


def _wwh_green(v, q1, q2, J1, J2, pA, par, v0):
    """W W H Green function with propagators on every leg, as a function of the vacuum value v at
    fixed g, lambda and v0: i g m_W(v) (D_W(q1) J1).(D_W(q2) J2) times i / (pA^2 - m_H^2(v))."""
    mw = par.g * v / 2.0
    lam = par.mH ** 2 / (2.0 * v0 ** 2)
    mh2 = lam * (3.0 * v * v - v0 * v0)
    W1 = vector_prop(q1, J1, mw, 0.0)
    W2 = vector_prop(q2, J2, mw, 0.0)
    return 1j * par.g * mw * mdot(W1, W2) * 1j / (mdot(pA, pA) - mh2)


def _let_residual(par):
    q1, q2, J1, J2 = _currents(6, seed=301)
    pA = q1 + q2  # the zero-momentum Higgs takes nothing
    v0 = par.vev
    # v-derivative by Richardson-extrapolated central differences
    def d(h):
        return (_wwh_green(v0 + h, q1, q2, J1, J2, pA, par, v0) - _wwh_green(v0 - h, q1, q2, J1, J2, pA, par, v0)) / (2 * h)
    h = 1e-3 * v0
    deriv = (4 * d(h / 2) - d(h)) / 3
    W1 = vector_prop(q1, J1, par.mW, 0.0)
    W2 = vector_prop(q2, J2, par.mW, 0.0)
    pieces = pr._ww_hh(W1, q1, W2, q2, pA, np.zeros_like(pA), par)
    four = sum(pieces) * 1j / (mdot(pA, pA) - par.mH ** 2)
    scale = sum(np.abs(x) for x in pieces) * np.abs(1.0 / (mdot(pA, pA) - par.mH ** 2))
    return np.abs(four - deriv) / scale, pieces


def test_us_dchh_core_zero_momentum_higgs_theorem():
    par0 = PAR.with_(wW=0.0, wH=0.0)
    res, pieces = _let_residual(par0)
    assert np.all(res < 1e-8), res
    # every diagram contributes at this kinematics, so each is tested
    tot = sum(np.abs(x) for x in pieces)
    for x in pieces:
        assert np.all(np.abs(x) > 1e-3 * tot)


@pytest.mark.parametrize("plant", ["s_channel_sign", "contact_dropped", "t_channel_sign"])
def test_us_dchh_core_theorem_catches_planted_mistakes(monkeypatch, plant):
    """A flipped s-channel Higgs term, a dropped contact term or a flipped W-exchange term planted in
    the oracle's core makes the theorem fail, and u s > d c h h runs that core."""
    orig = pr._ww_hh
    sign = {"s_channel_sign": (1, -1, 1, 1), "contact_dropped": (0, 1, 1, 1), "t_channel_sign": (1, 1, -1, -1)}[plant]
    monkeypatch.setattr(pr, "_ww_hh", lambda *a: [s * x for s, x in zip(sign, orig(*a))])
    res, _ = _let_residual(PAR.with_(wW=0.0, wH=0.0))
    assert np.all(res > 1e-3)
    # and the process changes with it
    u = np.random.default_rng(20).uniform(0.02, 0.98, (4, 16))
    pf, _ = ps.rambo_massive(1000.0, [0.0, 0.0, PAR.mH, PAR.mH], u)
    P = np.zeros((4, 6, 4))
    P[:, 0], P[:, 1] = ps.incoming(1000.0, 4)
    P[:, 2:] = pf
    planted = pr.us_dchh(P)
    monkeypatch.setattr(pr, "_ww_hh", orig)
    assert np.all(np.abs(planted / pr.us_dchh(P) - 1) > 1e-6)


# ---------------------------------------------------------------------------
# soft-gluon chain of u d~ > e+ ve g g
# ---------------------------------------------------------------------------
def _add_soft_gluon(base, k):
    """Append a gluon of momentum k to a massless final state: the final momenta of base are scaled
    to the invariant mass of P - k and boosted to its rest frame's motion (exact momentum
    conservation, every leg on shell, tending to base as k -> 0)."""
    n, m = base.shape[:2]
    P = base[:, 0] + base[:, 1]
    Q = P - k
    rs = np.sqrt(mdot(P, P))
    rq = np.sqrt(mdot(Q, Q))
    out = np.zeros((n, m + 1, 4))
    out[:, :2] = base[:, :2]
    for i in range(n):
        fin = base[i, 2:] * (rq[i] / rs[i])  # base is in the centre-of-mass frame
        out[i, 2:m] = boost(fin, Q[i, 1:] / Q[i, 0])
    out[:, m] = k
    return out


def _soft_dev(f_hard, f_soft, base, eik, nhat, ws):
    m2 = f_hard(base, PAR)
    devs = []
    for w in ws:
        k = np.concatenate([[w], w * nhat])[None, :].repeat(len(base), 0)
        Q = _add_soft_gluon(base, k)
        # the hard |M|^2 is taken at base, which Q without its gluon tends to as w -> 0
        devs.append(np.max(np.abs(f_soft(Q, PAR) / (eik(Q, k) * m2) - 1)))
    return devs


def _two_body(sqrt_s, n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.9, 0.9, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    E = sqrt_s / 2
    s = np.sqrt(1 - c * c)
    P = np.zeros((n, 4, 4))
    P[:, 0] = [E, 0, 0, E]
    P[:, 1] = [E, 0, 0, -E]
    P[:, 2] = np.stack([np.full(n, E), E * s * np.cos(phi), E * s * np.sin(phi), E * c], axis=1)
    P[:, 3] = P[:, 2] * np.array([1, -1, -1, -1])
    return P


def _S(Q, i, j, k):
    return mdot(Q[:, i], Q[:, j]) / (mdot(Q[:, i], k) * mdot(Q[:, j], k))


def test_udx_epveg_soft_limit_ward_and_boosts():
    """u d~ > e+ ve g: as the gluon's energy w -> 0, |M|^2 -> gs^2 C_F 2 S_{u d~} |M|^2(u d~ > e+ ve),
    the deviation falling in proportion to w; eps -> k gives zero; Lorentz invariance."""
    # e+ ve near the W pole, where the process is largest
    base = _two_body(PAR.mW + 0.7, 5, seed=310)
    nhat = np.array([0.6, 0.0, 0.8])
    eik = lambda Q, k: PAR.gs ** 2 * (4.0 / 3.0) * 2 * _S(Q, 0, 1, k)
    devs = _soft_dev(pr.udx_epve, pr.udx_epveg, base, eik, nhat, (1e-3, 1e-4))
    assert devs[1] < 1e-3 and devs[1] < devs[0] / 5, devs
    P = np.zeros((6, 5, 4))
    u = np.random.default_rng(311).uniform(0.02, 0.98, (6, 12))
    P[:, 0], P[:, 1] = ps.incoming(500.0, 6)
    P[:, 2:], _ = ps.rambo_massless(500.0, 3, u)
    ref = pr.udx_epveg(P, PAR)
    assert np.all(pr.udx_epveg(P, PAR, eps_override=P[:, 4]) <= 1e-24 * ref * P[:, 4, 0] ** 2)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.udx_epveg(random_lorentz(P, 312), PAR), ref, rtol=1e-11)


def _qqg_eikonal(Q, k, g_leg):
    """Colour-correlated eikonal factor of a soft gluon off q (leg 0), q~ (leg 1) and a gluon:
    -2 gs^2 sum_{i<j} T_i.T_j S_ij with T_q.T_q~ = (C_A - 2 C_F)/2 = 1/6, T_q.T_g = T_q~.T_g =
    -C_A/2 = -3/2 (colour conservation among the three partons)."""
    return PAR.gs ** 2 * (3.0 * _S(Q, 0, g_leg, k) + 3.0 * _S(Q, 1, g_leg, k) - _S(Q, 0, 1, k) / 3.0)


def _w1j_points(n, seed, sqrt_s=400.0):
    """u d~ > e+ ve g points with the e+ ve mass near the W pole (where W + jets is largest)."""
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    for i in range(n):
        mw = PAR.mW + rng.uniform(-2, 2)
        c, phi = rng.uniform(-0.8, 0.8), rng.uniform(0, 2 * np.pi)
        s = math.sqrt(1 - c * c)
        Eg = (sqrt_s ** 2 - mw ** 2) / (2 * sqrt_s)
        g = np.array([Eg, Eg * s * math.cos(phi), Eg * s * math.sin(phi), Eg * c])
        W = np.array([sqrt_s, 0, 0, 0]) - g
        c2, phi2 = rng.uniform(-0.9, 0.9), rng.uniform(0, 2 * np.pi)
        s2 = math.sqrt(1 - c2 * c2)
        e = 0.5 * mw * np.array([1, s2 * math.cos(phi2), s2 * math.sin(phi2), c2])
        nu = e * np.array([1, -1, -1, -1])
        P[i, 2] = boost(e[None], W[1:] / W[0])[0]
        P[i, 3] = boost(nu[None], W[1:] / W[0])[0]
        P[i, 4] = g
    return P


def test_udx_epvegg_soft_limit_against_udx_epveg():
    """u d~ > e+ ve g g with either gluon soft: |M|^2 -> eikonal(q, q~, g) |M|^2(u d~ > e+ ve g), the
    deviation falling in proportion to the soft gluon's energy.  Together with the previous pin this
    fixes the normalisation that the Ward identity, Bose symmetry and boosts leave free."""
    base = _w1j_points(5, seed=320)
    nhat = np.array([0.48, -0.36, 0.8])
    devs = _soft_dev(pr.udx_epveg, pr.udx_epvegg, base, lambda Q, k: _qqg_eikonal(Q, k, 4), nhat, (1e-2, 1e-3))
    assert devs[1] < 1e-3 and devs[1] < devs[0] / 5, devs
    # the other gluon soft (Bose symmetry of the pair)
    swap = lambda Q, par: pr.udx_epvegg(Q[:, [0, 1, 2, 3, 5, 4]], par)
    devs = _soft_dev(pr.udx_epveg, swap, base, lambda Q, k: _qqg_eikonal(Q, k, 4), nhat, (1e-2, 1e-3))
    assert devs[1] < 1e-3, devs


def test_udx_epvegg_soft_limit_catches_a_dropped_coupling(monkeypatch):
    """Every gluon vertex of u d~ > e+ ve g g planted without its gs (a uniform factor: the Ward
    identity, Bose symmetry and boosts still hold) fails the soft-limit pin."""
    base = _w1j_points(3, seed=321)
    nhat = np.array([0.48, -0.36, 0.8])
    ref_soft = lambda Q, par: pr.udx_epvegg(Q, par)
    gs = PAR.gs
    vi, vo = pr.vector_insertion, pr.vvv_out
    m2_base = pr.udx_epveg(base, PAR)
    monkeypatch.setattr(pr, "vector_insertion", lambda X, gl, gr: vi(X, gl / gs, gr / gs) if gl == gr == gs else vi(X, gl, gr))
    monkeypatch.setattr(pr, "vvv_out", lambda a, b, c, d, e, g: vo(a, b, c, d, e, g / gs if g == gs else g))
    k = np.concatenate([[1e-3], 1e-3 * nhat])[None, :].repeat(3, 0)
    Q = _add_soft_gluon(base, k)
    ratio = ref_soft(Q, PAR) / (_qqg_eikonal(Q, k, 4) * m2_base)
    assert np.all(np.abs(ratio - 1) > 0.1)


# ---------------------------------------------------------------------------
# six gluons: Ward identity of every final gluon
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("leg", [2, 5])
def test_six_gluon_ward_identity(leg):
    """g g > g g g g with one gluon's polarisation replaced by its momentum: every helicity
    combination of the other five (MHV and NMHV alike) gives zero."""
    u = np.random.default_rng(330).uniform(0.02, 0.98, (2, 16))
    P = np.zeros((2, 6, 4))
    P[:, 0], P[:, 1] = ps.incoming(1500.0, 2)
    P[:, 2:], _ = ps.rambo_massless(1500.0, 4, u)
    ref = pr.gluons(P)
    bad = pr.gluons(P, eps_override={leg: P[:, leg]})
    assert np.all(bad < 1e-24 * ref * P[:, leg, 0] ** 2)


# ---------------------------------------------------------------------------
# V + 2 jets and WBF H + 1 jet: Ward identity, Bose symmetry, soft limits, boosts
# ---------------------------------------------------------------------------
def _add_soft_massive(base, k, masses):
    """Append a gluon of momentum k to a final state with the given masses (base in its centre-of-mass
    frame): the final three-momenta are scaled by the xi with sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = M_Q,
    M_Q the invariant mass of P - k, and boosted to P - k (momentum conservation and masses exact,
    tending to base as k -> 0)."""
    n, m = base.shape[:2]
    P = base[:, 0] + base[:, 1]
    Q = P - k
    MQ = np.sqrt(mdot(Q, Q))
    out = np.zeros((n, m + 1, 4))
    out[:, :2] = base[:, :2]
    ms = np.asarray(masses, dtype=float)
    for i in range(n):
        q3 = base[i, 2:, 1:]
        a2 = (q3 ** 2).sum(axis=1)
        xi = 1.0
        for _ in range(60):  # Newton on f(xi) = sum sqrt(m^2 + xi^2 a2) - MQ
            e = np.sqrt(ms ** 2 + xi * xi * a2)
            xi -= (e.sum() - MQ[i]) / (xi * (a2 / e).sum())
        fin = np.zeros((m - 2, 4))
        fin[:, 1:] = xi * q3
        fin[:, 0] = np.sqrt(ms ** 2 + xi * xi * a2)
        out[i, 2:m] = boost(fin, Q[i, 1:] / Q[i, 0])
    out[:, m] = k
    return out


def _massive_points(sqrt_s, masses, n, seed):
    from kinematics import consistent
    u = np.random.default_rng(seed).uniform(0.05, 0.95, (n, 4 * len(masses)))
    pf, _ = ps.rambo_massive(sqrt_s, list(masses), u)
    P = np.zeros((n, len(masses) + 2, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return consistent(P, (0.0, 0.0) + tuple(masses))


@pytest.mark.parametrize("which", ["udx_wpgg", "uux_zgg"])
def test_v_plus_two_jets_ward_bose_soft_and_boosts(which):
    """q q~ > V g g: each gluon's eps -> k gives zero (exactly on-shell inputs); swapping the gluons
    leaves |M|^2 unchanged; either gluon soft: |M|^2 -> eikonal(q, q~, g) |M|^2(q q~ > V g) (closed
    form), the deviation falling in proportion to its energy; boosts."""
    f = getattr(pr, which)
    f0 = {"udx_wpgg": pr.udx_wpg, "uux_zgg": pr.uux_zg}[which]
    mV = PAR.mW if which == "udx_wpgg" else PAR.mZ
    P = _massive_points(600.0, (mV, 0.0, 0.0), 4, seed=400)
    ref = f(P, PAR)
    for leg in (3, 4):
        bad = f(P, PAR, eps_override={leg: P[:, leg]})
        assert np.all(bad < 1e-24 * ref * P[:, leg, 0] ** 2)
    assert np.allclose(f(P[:, [0, 1, 2, 4, 3]], PAR), ref, rtol=1e-12)
    from test_oracle_processes import random_lorentz
    assert np.allclose(f(random_lorentz(P, 401), PAR), ref, rtol=1e-10)
    base = _massive_points(600.0, (mV, 0.0), 4, seed=402)
    m2 = f0(base, PAR)
    nhat = np.array([0.48, -0.36, 0.8])
    devs = []
    for w in (1e-2, 1e-3):
        k = np.concatenate([[w], w * nhat])[None, :].repeat(len(base), 0)
        Q = _add_soft_massive(base, k, (mV, 0.0))
        devs.append(np.max(np.abs(f(Q, PAR) / (_qqg_eikonal(Q, k, 3) * m2) - 1)))
    assert devs[1] < 1e-3 and devs[1] < devs[0] / 5, devs


def test_wbf_higgs_plus_jet_ward_soft_and_boosts():
    """u s > d c H g: the gluon's eps -> k gives zero (exactly on-shell inputs); as the gluon gets soft,
    |M|^2 -> g_s^2 2 C_F (S_ud + S_sc) |M|^2(u s > d c H) (the two lines' colours do not interfere,
    Tr t^a = 0), the deviation falling in proportion to its energy; boosts."""
    P = _massive_points(1000.0, (0.0, 0.0, PAR.mH, 0.0), 4, seed=410)
    ref = pr.us_dchg(P, PAR)
    bad = pr.us_dchg(P, PAR, eps_override=P[:, 5])
    assert np.all(bad < 1e-24 * ref * P[:, 5, 0] ** 2)
    from test_oracle_processes import random_lorentz
    assert np.allclose(pr.us_dchg(random_lorentz(P, 411), PAR), ref, rtol=1e-10)
    base = _massive_points(1000.0, (0.0, 0.0, PAR.mH), 4, seed=412)
    m2 = pr.us_dch(base, PAR)
    nhat = np.array([0.6, 0.0, 0.8])
    devs = []
    for w in (1e-2, 1e-3):
        k = np.concatenate([[w], w * nhat])[None, :].repeat(len(base), 0)
        Q = _add_soft_massive(base, k, (0.0, 0.0, PAR.mH))
        eik = PAR.gs ** 2 * (4.0 / 3.0) * 2 * (_S(Q, 0, 2, k) + _S(Q, 1, 3, k))
        devs.append(np.max(np.abs(pr.us_dchg(Q, PAR) / (eik * m2) - 1)))
    assert devs[1] < 1e-3 and devs[1] < devs[0] / 5, devs
