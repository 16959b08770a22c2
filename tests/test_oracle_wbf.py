"""Pins of the oracle's weak-boson-fusion multi-Higgs processes (Sect. 2.10: u d > u d + HH(H),
and u s > d c h h h by W+ W- fusion alone) and of the complex-mass option (Sect. 7.11).

- The generic V V > n H core (vv_higgs) at n = 2 equals the separately pinned W W > h h core.
- The zero-momentum Higgs theorem links every n to n - 1: a Higgs of zero four-momentum couples
  like a shift of the vacuum value v, so the V V + (n+1) H Green function with one such Higgs is
  the v-derivative of the V V + n H Green function (m_V = g_V v / 2, the Higgs curvature
  m_H^2(v) = lambda (3 v^2 - v0^2), H H H = -6 lambda v, H H H H = -6 lambda, V V H = g_V m_V(v),
  V V H H = g_V^2 / 2).  Checked for W and Z at n = 1 -> 2 and 2 -> 3; a wrong sign or coupling
  of the quartic Higgs vertex fails it.
- u d > u d h: closed form.  With conserved massless currents the vector propagators act as
  g^{mu nu} / D, every helicity amplitude is (V V H coupling) J1.J2 / (D1 D2), and the
  chiral Fierz identity turns the W-fusion spinor product of the left-handed lines into minus the
  Z-fusion one, so the exchange sign makes the two interfere constructively:
    LL: 16 (p0.p1)(p2.p3) (9 |a_L|^2 + 9 |b|^2 + 6 Re a_L b*),  RR: 16 (p0.p1)(p2.p3) 9 |a_R|^2,
    LR, RL: 16 (p0.p3)(p1.p2) 9 |a_LR|^2, |a_RL|^2, averaged by 1/36,
  a = g_ZZH g^u g^d / (D_Z(p0-p2) D_Z(p1-p3)), b = g_WWH (g^2/2) / (D_W(p0-p3) D_W(p1-p2)).
  This fixes the lines, couplings, colour and the relative sign the n = 2, 3 processes share.
- The W-fusion channel of u d > u d h (h) equals u s > d c h (h) with the outgoing quarks
  exchanged.
- Complex-mass option: at 16 and 32 TeV (fixed angles) the complex-mass |M|^2 of the HHH
  processes stays at the zero-width one, while the fixed-width one (the same widths, real
  couplings) grows with the energy (the gauge cancellation broken at O(Gamma/m)); a complex-mass
  card whose V V H coupling is kept real grows the same way.
- Higgs permutations and boosts.
"""
import math

import numpy as np
import pytest

from oracle import phasespace as ps, processes as pr
from oracle.feynman import den, ffv_current, vector_prop
from oracle.lorentz import bar, boost, mdot, u_spinor
from oracle.sm import SMParams

PAR = SMParams()


def _points(sqrt_s, nh, n, seed):
    from kinematics import consistent
    masses = [0.0, 0.0] + [PAR.mH] * nh
    u = np.random.default_rng(seed).uniform(0.05, 0.95, (n, 4 * len(masses)))
    pf, _ = ps.rambo_massive(sqrt_s, masses, u)
    P = np.zeros((n, len(masses) + 2, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return consistent(P, (0.0, 0.0) + tuple(masses))


def _line_currents(seed, n=6, z=False):
    """Off-shell boson momenta q1, q2 from two quark lines and their currents (left-handed W lines,
    or Z lines with the u and d couplings)."""
    rng = np.random.default_rng(seed)

    def massless(E, c, phi):
        s = np.sqrt(1 - c * c)
        return np.stack([E, E * s * np.cos(phi), E * s * np.sin(phi), E * c], axis=1)
    p0 = massless(rng.uniform(300, 500, n), np.full(n, 1.0), np.zeros(n))
    p1 = massless(rng.uniform(300, 500, n), np.full(n, -1.0), np.zeros(n))
    p2 = massless(rng.uniform(100, 200, n), rng.uniform(-0.8, 0.8, n), rng.uniform(0, 6.28, n))
    p3 = massless(rng.uniform(100, 200, n), rng.uniform(-0.8, 0.8, n), rng.uniform(0, 6.28, n))
    if z:
        c1, c2 = pr._z_couplings("u", PAR), pr._z_couplings("d", PAR)
    else:
        c1 = c2 = (PAR.g / math.sqrt(2.0), 0.0)
    J1 = ffv_current(bar(u_spinor(p2, -1)), u_spinor(p0, -1), *c1)
    J2 = ffv_current(bar(u_spinor(p3, -1)), u_spinor(p1, -1), *c2)
    return p0 - p2, p1 - p3, J1, J2


# ---------------------------------------------------------------------------
# the generic core
# ---------------------------------------------------------------------------
def test_core_at_two_higgs_equals_the_ww_hh_core():
    P = _points(1000.0, 2, 8, seed=401)
    p = [P[:, k] for k in range(6)]
    q1, q2 = p[0] - p[2], p[1] - p[3]
    gw = PAR.g / math.sqrt(2.0)
    for h in ((-1, -1, -1, -1),):
        W1 = vector_prop(q1, ffv_current(bar(u_spinor(p[2], h[2])), u_spinor(p[0], h[0]), gw, 0.0), PAR.mW, PAR.wW)
        W2 = vector_prop(q2, ffv_current(bar(u_spinor(p[3], h[3])), u_spinor(p[1], h[1]), gw, 0.0), PAR.mW, PAR.wW)
        a = sum(pr._ww_hh(W1, q1, W2, q2, p[4], p[5], PAR))
        b = pr.vv_higgs(W1, q1, W2, q2, [p[4], p[5]], pr.wbf_couplings(PAR, "w"))
        assert np.allclose(b, a, rtol=1e-13, atol=0)


def _cp(v, v0, gV, mH0):
    lam = mH0 ** 2 / (2.0 * v0 ** 2)
    mV = gV * v / 2.0
    return dict(mV=mV, wV=0.0, gvvh=gV * mV, gvvhh=gV * gV / 2.0, mH=math.sqrt(lam * (3 * v * v - v0 * v0)), wH=0.0,
                ghhh=-6.0 * lam * v, ghhhh=-6.0 * lam)


def _green(v, v0, gV, q1, q2, J1, J2, pH, flip_quartic=False):
    """V V + n H Green function with propagators on every leg, at vacuum value v."""
    cp = _cp(v, v0, gV, PAR.mH)
    if flip_quartic:
        cp["ghhhh"] = -cp["ghhhh"]
    V1 = vector_prop(q1, J1, cp["mV"], 0.0)
    V2 = vector_prop(q2, J2, cp["mV"], 0.0)
    G = pr.vv_higgs(V1, q1, V2, q2, pH, cp)
    for p in pH:
        G = G * 1j / (mdot(p, p) - cp["mH"] ** 2)
    return G


def _let_residual(n, z, flip_quartic=False):
    """|G_{n+1}(pH, 0) - dG_n/dv| / |G_{n+1}| with the zero-momentum leg amputated."""
    q1, q2, J1, J2 = _line_currents(500 + n + 10 * z, n=64, z=z)
    gV = PAR.gz if z else PAR.g
    v0 = PAR.vev
    rng = np.random.default_rng(600 + n)
    Q = q1 + q2
    pH = []
    for k in range(n - 1):  # off-shell Higgs legs that share Q; the last one takes the rest
        pH.append(Q * rng.uniform(0.2, 0.4) + rng.normal(0.0, 30.0, Q.shape))
    pH.append(Q - sum(pH) if pH else Q.copy())
    # keep points whose propagators are all well away from their poles (the finite difference in v
    # moves the poles by about 1 %): every Higgs line (one leg or a set of legs) from m_H^2 and every
    # internal boson line from m_V^2, by 30 % at least
    mV = gV * v0 / 2.0
    far = np.ones(len(Q), dtype=bool)
    for S in pr._subsets(frozenset(range(n))):
        pS = sum(pH[k] for k in S)
        far &= np.abs(mdot(pS, pS) / PAR.mH ** 2 - 1.0) > 0.3
        if len(S) < n:
            r = q1 - pS
            far &= np.abs(mdot(r, r) / mV ** 2 - 1.0) > 0.3
    idx = np.nonzero(far)[0][:6]
    assert len(idx) == 6
    q1, q2, J1, J2 = q1[idx], q2[idx], J1[idx], J2[idx]
    Q = Q[idx]
    pH = [x[idx] for x in pH]

    def d(h):
        return (_green(v0 + h, v0, gV, q1, q2, J1, J2, pH) - _green(v0 - h, v0, gV, q1, q2, J1, J2, pH)) / (2 * h)
    h = 1e-3 * v0
    deriv = (4 * d(h / 2) - d(h)) / 3
    cp = _cp(v0, v0, gV, PAR.mH)
    if flip_quartic:
        cp["ghhhh"] = -cp["ghhhh"]
    V1 = vector_prop(q1, J1, cp["mV"], 0.0)
    V2 = vector_prop(q2, J2, cp["mV"], 0.0)
    G1 = pr.vv_higgs(V1, q1, V2, q2, pH + [np.zeros_like(Q)], cp)
    for p in pH:
        G1 = G1 * 1j / (mdot(p, p) - cp["mH"] ** 2)
    return np.abs(G1 - deriv) / np.abs(G1)


@pytest.mark.parametrize("n,z", [(1, False), (1, True), (2, False), (2, True)])
def test_core_zero_momentum_higgs_theorem(n, z):
    res = _let_residual(n, z)
    assert np.all(res < 1e-7), res


@pytest.mark.parametrize("z", [False, True])
def test_core_theorem_catches_a_flipped_quartic_higgs_vertex(z):
    """The theorem at n = 2 -> 3 involves the H H H H vertex: flipping its sign on the three-Higgs
    side (but not in the derivative, where it does not enter) fails it."""
    res = _let_residual(2, z, flip_quartic=True)
    assert np.all(res > 1e-3), res


# ---------------------------------------------------------------------------
# u d > u d h: closed form; the W channel against u s > d c h (h)
# ---------------------------------------------------------------------------
def test_ud_udh_closed_form():
    for par in (PAR, PAR.with_cms()):
        P = _points(1000.0, 1, 40, seed=410)
        p = [P[:, k] for k in range(5)]
        d = lambda a, b: mdot(p[a], p[b])
        (gLu, gRu), (gLd, gRd) = pr._z_couplings("u", par), pr._z_couplings("d", par)
        DZ = den(mdot(p[0] - p[2], p[0] - p[2]), par.mZ, par.wZ) * den(mdot(p[1] - p[3], p[1] - p[3]), par.mZ, par.wZ)
        DW = den(mdot(p[0] - p[3], p[0] - p[3]), par.mW, par.wW) * den(mdot(p[1] - p[2], p[1] - p[2]), par.mW, par.wW)
        gzzh, gwwh = par.gzzh, par.gwwh
        aL, aR = gzzh * gLu * gLd / DZ, gzzh * gRu * gRd / DZ
        aLR, aRL = gzzh * gLu * gRd / DZ, gzzh * gRu * gLd / DZ
        b = gwwh * (par.g ** 2 / 2.0) / DW
        st = 16.0 * d(0, 1) * d(2, 3)
        su = 16.0 * d(0, 3) * d(1, 2)
        want = (st * (9 * abs(aL) ** 2 + 9 * abs(b) ** 2 + 6 * np.real(aL * np.conj(b)) + 9 * abs(aR) ** 2)
                + su * 9 * (abs(aLR) ** 2 + abs(aRL) ** 2)) / 36.0
        assert np.allclose(pr.ud_udh(P, par), want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("nh", [1, 2])
def test_w_channel_equals_us_dc(nh):
    P = _points(1000.0, nh, 12, seed=420 + nh)
    swap = [0, 1, 3, 2] + list(range(4, 4 + nh))
    ref = (pr.us_dch if nh == 1 else pr.us_dchh)(P[:, swap])
    assert np.allclose(pr.ud_udh_n(P, PAR, bosons=("w",)), ref, rtol=1e-12, atol=0)


def test_us_dchhh_equals_the_w_channel_of_ud_udhhh():
    P = _points(1500.0, 3, 6, seed=430)
    assert np.allclose(pr.ud_udh_n(P, PAR, bosons=("w",)), pr.us_dchhh(P[:, [0, 1, 3, 2, 4, 5, 6]]), rtol=1e-12)


# ---------------------------------------------------------------------------
# symmetries
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fn,nh", [(pr.ud_udhh, 2), (pr.ud_udhhh, 3), (pr.us_dchhh, 3)])
def test_higgs_permutations_and_boosts(fn, nh):
    P = _points(1500.0, nh, 5, seed=440 + nh)
    ref = fn(P)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    perm = [0, 1, 2, 3] + list(range(4, 4 + nh))[::-1]
    assert np.allclose(fn(P[:, perm]), ref, rtol=1e-11)
    beta = np.array([0.3, -0.5, 0.6])
    assert np.allclose(fn(boost(P, beta)), ref, rtol=1e-9)


def test_cms_card():
    c = PAR.with_cms()
    assert c.mW == pytest.approx(PAR.cw * PAR.mZ) and c.wW == pytest.approx(PAR.cw * PAR.wZ)
    assert c.muW ** 2 == pytest.approx(complex(c.mW ** 2, -c.mW * c.wW), rel=1e-14)
    assert c.muW ** 2 == pytest.approx(PAR.cw ** 2 * c.muZ ** 2, rel=1e-14)
    assert c.vev == pytest.approx(2 * c.muW / c.g)
    # at zero widths the complex-mass card is the fixed-width card with the tied W mass
    P = _points(1500.0, 3, 4, seed=450)
    z = c.with_(wW=0.0, wZ=0.0)
    f = PAR.with_(mW=c.mW, wW=0.0, wZ=0.0)
    assert np.allclose(pr.ud_udhhh(P, z), pr.ud_udhhh(P, f), rtol=1e-13)


# ---------------------------------------------------------------------------
# complex-mass option: the high-energy behaviour
# ---------------------------------------------------------------------------
def _fixed_angles(E, nh, n=4, seed=5):
    """A fixed-angle family: one massless configuration scaled to the energy E, the Higgs bosons
    made massive by the common three-momentum factor xi (directions and momentum balance kept)."""
    u = np.random.default_rng(seed).uniform(0.05, 0.95, (n, 4 * (2 + nh)))
    q, _ = ps.rambo_massless(1.0, 2 + nh, u)
    ms = np.array([0.0, 0.0] + [PAR.mH] * nh)
    P = np.zeros((n, 4 + nh, 4))
    P[:, 0], P[:, 1] = ps.incoming(E, n)
    for i in range(n):
        q3 = E * q[i, :, 1:]
        a2 = (q3 ** 2).sum(axis=1)
        xi = 1.0
        for _ in range(60):
            e = np.sqrt(ms ** 2 + xi * xi * a2)
            xi -= (e.sum() - E) / (xi * (a2 / e).sum())
        P[i, 2:, 1:] = xi * q3
        P[i, 2:, 0] = np.sqrt(ms ** 2 + xi * xi * a2)
    return P


@pytest.mark.parametrize("fn", [pr.us_dchhh, pr.ud_udhhh])
def test_complex_mass_restores_the_high_energy_behaviour(fn, monkeypatch):
    cms = PAR.with_cms()
    zero = cms.with_(wW=0.0, wZ=0.0)
    fw = PAR.with_(mW=cms.mW, wW=cms.wW)   # the same masses and widths, real couplings
    P16, P32 = _fixed_angles(16e3, 3), _fixed_angles(32e3, 3)
    z16, z32 = fn(P16, zero), fn(P32, zero)
    c16, c32 = fn(P16, cms), fn(P32, cms)
    f16, f32 = fn(P16, fw), fn(P32, fw)
    assert np.allclose(c16, z16, rtol=0.03) and np.allclose(c32, z32, rtol=0.03)
    assert np.all(f32 > 10 * z32)
    assert np.all(f32 / f16 > 2 * z32 / z16)   # s^3 |M|^2 grows with the energy in the fixed-width scheme
    # a complex-mass card with a real V V H coupling breaks the cancellation the same way
    monkeypatch.setattr(SMParams, "gwwh", property(lambda self: self.g * self.mW))
    monkeypatch.setattr(SMParams, "gzzh", property(lambda self: self.gz * self.mZ))
    assert np.all(fn(P32, cms) > 10 * z32)


# ---------------------------------------------------------------------------
# u u > u u + Higgs bosons: Z Z fusion with the outgoing quarks exchanged
# ---------------------------------------------------------------------------
def test_uu_uuh_closed_form():
    """Per helicity the amplitude is g_ZZH g^{h0} g^{h1} times a spinor product over the Z
    denominators.  Same-chirality lines: both pairings contribute, and by the chiral Fierz identity
    the exchanged product is minus the direct one, so with the exchange sign
      16 (p0.p1)(p2.p3) (g_L^4 + g_R^4) |g_ZZH|^2 (9/|Dt|^2 + 9/|Du|^2 + 6 Re 1/(Dt Du*));
    opposite chiralities: only the pairing that keeps each line's helicity,
      16 (p0.p3)(p1.p2) 9 |g_ZZH g_L g_R / Dt|^2 x 2 and 16 (p0.p2)(p1.p3) 9 |g_ZZH g_L g_R / Du|^2 x 2,
    Dt = D_Z(p0 - p2) D_Z(p1 - p3), Du = D_Z(p0 - p3) D_Z(p1 - p2); averaged by 1/36."""
    for par in (PAR, PAR.with_cms()):
        P = _points(1000.0, 1, 40, seed=470)
        p = [P[:, k] for k in range(5)]
        d = lambda a, b: mdot(p[a], p[b])
        gL, gR = pr._z_couplings("u", par)
        Dt = den(mdot(p[0] - p[2], p[0] - p[2]), par.mZ, par.wZ) * den(mdot(p[1] - p[3], p[1] - p[3]), par.mZ, par.wZ)
        Du = den(mdot(p[0] - p[3], p[0] - p[3]), par.mZ, par.wZ) * den(mdot(p[1] - p[2], p[1] - p[2]), par.mZ, par.wZ)
        g2 = abs(par.gzzh) ** 2
        same = 16 * d(0, 1) * d(2, 3) * (gL ** 4 + gR ** 4) * g2 * (
            9 / np.abs(Dt) ** 2 + 9 / np.abs(Du) ** 2 + 6 * np.real(1 / (Dt * np.conj(Du))))
        opp = 2 * 9 * g2 * gL ** 2 * gR ** 2 * (16 * d(0, 3) * d(1, 2) / np.abs(Dt) ** 2
                                                   + 16 * d(0, 2) * d(1, 3) / np.abs(Du) ** 2)
        assert np.allclose(pr.uu_uuh_n(P, par), (same + opp) / 36.0, rtol=1e-12, atol=0)


@pytest.mark.parametrize("nh", [2, 3])
def test_uu_uu_higgs_fermi_symmetry_permutations_and_boosts(nh):
    P = _points(1500.0, nh, 5, seed=480 + nh)
    ref = pr.uu_uuh_n(P)
    assert np.all(ref > 0) and np.all(np.isfinite(ref))
    assert np.allclose(pr.uu_uuh_n(P[:, [0, 1, 3, 2] + list(range(4, 4 + nh))]), ref, rtol=1e-12)
    assert np.allclose(pr.uu_uuh_n(P[:, [1, 0, 2, 3] + list(range(4, 4 + nh))]), ref, rtol=1e-12)
    assert np.allclose(pr.uu_uuh_n(P[:, [0, 1, 2, 3] + list(range(4, 4 + nh))[::-1]]), ref, rtol=1e-11)
    assert np.allclose(pr.uu_uuh_n(boost(P, np.array([0.2, 0.4, -0.5]))), ref, rtol=1e-9)
