"""Pins of the oracle's Philox stream, phase-space generators, cuts and MC estimate."""
import math

import numpy as np
import pytest

from oracle import phasespace as ps, xsec
from oracle.lorentz import mdot
from oracle.sm import SMParams

PAR = SMParams()


def test_philox_matches_numpy_library():
    """numpy.random.Philox is Philox4x64-10; it increments its counter before each block."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        ctr[0] = ctr[0] & np.uint64(0x7FFFFFFFFFFFFFF0)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        lib = np.random.Philox(counter=ctr, key=key).random_raw(8)
        c1 = ctr.copy()
        c1[0] += np.uint64(1)
        c2 = ctr.copy()
        c2[0] += np.uint64(2)
        mine = ps.philox4x64_10(np.stack([c1, c2]), key)
        assert np.array_equal(mine.ravel(), lib)


def test_uniforms_are_halves_of_the_library_words():
    """Uniform i of a draw is the low (even i) or high (odd i) 32 bits w of word (i % 8) // 2 of
    Philox block i // 8, as (w + 1/2) 2^-32; the words from numpy's library Philox4x64-10."""
    seed, ev, att = 987654321, 4242, 5
    u = ps.uniforms(seed, np.array([ev]), np.array([att]), 21)[0]
    key = np.array([seed, 0], dtype=np.uint64)
    for i in range(21):
        ctr = np.array([ev - 1, att, i // 8, 0], dtype=np.uint64)  # the library steps the counter first
        word = int(np.random.Philox(counter=ctr, key=key).random_raw(4)[(i % 8) // 2])
        w = (word >> 32) if i % 2 else (word & 0xFFFFFFFF)
        assert u[i] == (w + 0.5) / 2.0 ** 32


def test_uniforms_range_and_moments():
    u = ps.uniforms(7, np.arange(20000), np.zeros(20000), 8)
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005
    assert abs((u * u).mean() - 1 / 3) < 0.005
    # distinct attempts give distinct streams
    u1 = ps.uniforms(7, np.arange(100), np.ones(100), 8)
    assert not np.allclose(u[:100], u1)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_rambo_massless(n):
    w = 1000.0
    u = ps.uniforms(1, np.arange(500), np.zeros(500), 4 * n)
    p, wt = ps.rambo_massless(w, n, u)
    tot = p.sum(axis=1)
    assert np.allclose(tot, [w, 0, 0, 0], atol=1e-9 * w)
    assert np.abs(mdot(p, p)).max() < 1e-9 * w * w
    assert np.all(p[..., 0] > 0)
    vol = (2 * math.pi) ** (4 - 3 * n) * (math.pi / 2) ** (n - 1) * w ** (2 * n - 4) / (
        math.factorial(n - 1) * math.factorial(n - 2))
    assert np.allclose(wt, vol)
    if n == 2:
        assert np.isclose(vol, 1 / (8 * math.pi))


def test_rambo_flat_distributions():
    """n=2: isotropic; n=3: flat Dalitz plot, <x_i> = 2/3, <x_i^2> = 1/2 (x = 2E/w)."""
    N = 40000
    u = ps.uniforms(2, np.arange(N), np.zeros(N), 8)
    p, _ = ps.rambo_massless(500.0, 2, u)
    c = p[:, 0, 3] / p[:, 0, 0]
    assert abs(c.mean()) < 0.02 and abs((c * c).mean() - 1 / 3) < 0.01
    u = ps.uniforms(3, np.arange(N), np.zeros(N), 12)
    p, _ = ps.rambo_massless(500.0, 3, u)
    x = 2 * p[:, :, 0] / 500.0
    assert np.allclose(x.mean(axis=0), 2 / 3, atol=0.01)
    assert np.allclose((x * x).mean(axis=0), 0.5, atol=0.01)


def test_rambo_massive():
    w = 1000.0
    u = ps.uniforms(4, np.arange(200), np.zeros(200), 8)
    m1, m2 = 125.0, 300.0
    p, wt = ps.rambo_massive(w, [m1, m2], u)
    assert np.allclose(p.sum(axis=1), [w, 0, 0, 0], atol=1e-9 * w)
    assert np.allclose(mdot(p[:, 0], p[:, 0]), m1 * m1, rtol=1e-10)
    assert np.allclose(mdot(p[:, 1], p[:, 1]), m2 * m2, rtol=1e-10)
    k = math.sqrt((w * w - (m1 + m2) ** 2) * (w * w - (m1 - m2) ** 2)) / (2 * w)
    assert np.allclose(wt, k / (4 * math.pi * w), rtol=1e-12)
    # three massive bodies: volume against direct two-step integration
    N = 200000
    u = ps.uniforms(5, np.arange(N), np.zeros(N), 12)
    ms = [125.0, 125.0, 0.0]
    p, wt = ps.rambo_massive(w, ms, u)
    vol_mc = wt.mean()
    # dPhi_3 = int ds23/(2 pi) Phi_2(w; m1, sqrt(s23)) Phi_2(sqrt(s23); m2, m3)
    s = np.linspace((ms[1] + ms[2]) ** 2, (w - ms[0]) ** 2, 200001)
    lam = lambda a, b, c: a * a + b * b + c * c - 2 * a * b - 2 * b * c - 2 * a * c
    f = (np.sqrt(np.maximum(lam(w * w, ms[0] ** 2, s), 0)) / (8 * math.pi * w * w)
         * np.sqrt(np.maximum(lam(s, ms[1] ** 2, ms[2] ** 2), 0)) / (8 * math.pi * s)) / (2 * math.pi)
    vol = np.trapezoid(f, s)
    assert abs(vol_mc / vol - 1) < 0.01


def test_breit_wigner_jacobian():
    """Mean of the Eq. 16 Jacobian over uniform theta equals the s range / (2 pi)."""
    m, w = 175.0, 1.5
    u = (np.arange(200000) + 0.5) / 200000
    s, jac = ps.bw_sample(m, w, u)
    t0, t1 = ps.bw_range(m, w)
    s_lo, s_hi = m * m + m * w * math.tan(t0), m * m + m * w * math.tan(t1)
    assert np.isclose(jac.mean() * 2 * math.pi, s_hi - s_lo, rtol=1e-6)
    assert np.isclose(s_hi - m * m, 20 * m * w)
    # the range rule min(20, m/Gamma)
    assert np.isclose(math.tan(ps.bw_range(10.0, 2.0)[1]), 5.0)


def test_ttbar_chain_kinematics():
    N = 2000
    u = ps.uniforms(2, np.arange(N), np.zeros(N), 16)
    P, wt, ok, shat = ps.ttbar_dilepton(u, PAR, (400.0, 2000.0))
    P, wt, shat = P[ok], wt[ok], shat[ok]
    assert ok.mean() > 0.5
    fin = P[:, 2:].sum(axis=1)
    ini = P[:, 0] + P[:, 1]
    assert np.allclose(fin, ini, atol=1e-9 * 2000)
    assert np.abs(mdot(P[:, 2:], P[:, 2:])).max() < 1e-8
    t = P[:, 2] + P[:, 3] + P[:, 4]
    tb = P[:, 5] + P[:, 6] + P[:, 7]
    W = P[:, 3] + P[:, 4]
    for v, m, g in ((t, PAR.mt, PAR.wt), (tb, PAR.mt, PAR.wt), (W, PAR.mW, PAR.wW)):
        s = mdot(v, v)
        assert np.all(np.abs(s - m * m) <= 20 * m * g * (1 + 1e-9))
    assert np.all(wt > 0)
    assert np.all((np.sqrt(shat) >= 400) & (np.sqrt(shat) <= 2000))


def test_cut_definitions():
    def mom(pt_, eta_, phi_):
        return np.array([pt_ * math.cosh(eta_), pt_ * math.cos(phi_), pt_ * math.sin(phi_), pt_ * math.sinh(eta_)])

    base = [mom(50, 0.0, 0.0), mom(50, 1.0, 2.0)]
    P = np.array([[np.zeros(4), np.zeros(4)] + base])
    assert ps.pass_cuts(P, [2, 3], 20.0, 2.5, 0.4)[0]
    for bad in (mom(19.9, 0.5, 4.0), mom(50, 2.51, 4.0), mom(50, -2.51, 4.0), mom(50, 0.2, 0.3)):
        P = np.array([[np.zeros(4), np.zeros(4)] + base + [bad]])
        assert not ps.pass_cuts(P, [2, 3, 4], 20.0, 2.5, 0.4)[0]
    # Delta R across the phi = +-pi seam
    P = np.array([[np.zeros(4), np.zeros(4), mom(50, 0, math.pi - 0.1), mom(50, 0, -math.pi + 0.1)]])
    assert not ps.pass_cuts(P, [2, 3], 20.0, 2.5, 0.4)[0]
    assert np.isclose(ps.delta_r(P[:, 2], P[:, 3])[0], 0.2)


def test_mc_estimate_two_body_closed_form():
    """sigma-hat(u u~ > e+ e-) from the resampled generator against the integral of the
    closed-form dsigma/dcos(theta) (Gauss-Legendre), within 4 standard errors."""
    from oracle import processes as pr
    kin = {"kind": "2to2", "sqrt_s": 500.0}
    P, W, S, tries = xsec.generate(kin, PAR, 0, np.arange(20000))
    me2 = pr.uux_epem(P, PAR)
    sw, sw2, nacc, ntry = xsec.accumulate(me2, W, S, tries, 1.0)
    sig, err = xsec.estimate(sw, sw2, ntry)
    x, wq = np.polynomial.legendre.leggauss(64)
    Q = np.zeros((64, 4, 4))
    Q[:, 0] = [250, 0, 0, 250]
    Q[:, 1] = [250, 0, 0, -250]
    Q[:, 3, 0] = 250
    Q[:, 3, 1] = 250 * np.sqrt(1 - x * x)
    Q[:, 3, 3] = 250 * x
    Q[:, 2, 0] = 250
    Q[:, 2, 1:] = -Q[:, 3, 1:]
    dsig = pr.uux_epem(Q, PAR) / (32 * math.pi * 500.0 ** 2) * 0.3893793721e9
    exact = np.sum(wq * dsig)
    assert abs(sig - exact) < 4 * err
    assert err / sig < 0.02


def test_per_event_massive_rambo_matches_rambo_massive():
    u = ps.uniforms(5, np.arange(500), np.zeros(500), 12)
    masses = [125.0, 0.0, 30.0]
    p1, w1 = ps.rambo_massive(1000.0, masses, u)
    p2, w2 = ps.rambo_massive_events(1000.0, np.tile(masses, (500, 1)), u)
    assert np.array_equal(p1, p2) and np.array_equal(w1, w2)


def test_resonance_generator_kinematics():
    """App. A.2 resonance mapping: momentum conservation, massless particles, the pair mass in the
    Breit-Wigner window of Eq. 16."""
    m, g = 80.4, 2.085
    u = ps.uniforms(6, np.arange(4000), np.zeros(4000), 16)
    pf, wt, ok = ps.rambo_resonance(1000.0, 4, m, g, u)
    assert ok.all() and np.all(wt > 0)
    tot = pf.sum(axis=1)
    assert np.abs(tot - [1000.0, 0, 0, 0]).max() < 1e-9
    m2 = pf[..., 0] ** 2 - (pf[..., 1:] ** 2).sum(axis=-1)
    assert np.abs(m2).max() < 1e-7 * 1000.0 ** 2
    pr = pf[:, 0] + pf[:, 1]
    s = pr[:, 0] ** 2 - (pr[:, 1:] ** 2).sum(axis=1)
    assert np.all(np.abs(s - m * m) / (m * g) < 20.0 + 1e-6)


@pytest.mark.parametrize("shape", ["flat", "breit-wigner"])
def test_resonance_generator_factorises_phase_space(shape):
    """dPhi_4 = dPhi_3(R, 3, 4) ds/(2 pi) dPhi_2(R -> 1 2): the integral over the Breit-Wigner
    window of s_12 agrees between the resonance generator and plain massless RAMBO (statistical,
    4 standard errors), for a flat and a resonant integrand."""
    w, nf, m, g = 1000.0, 4, 80.4, 2.085
    n = 200000

    def integrand(pf):
        pr = pf[:, 0] + pf[:, 1]
        s = pr[:, 0] ** 2 - (pr[:, 1:] ** 2).sum(axis=1)
        inside = np.abs(s - m * m) / (m * g) < 20.0
        f = (m * g) ** 2 / ((s - m * m) ** 2 + (m * g) ** 2) if shape == "breit-wigner" else np.ones_like(s)
        return np.where(inside, f, 0.0)

    u = ps.uniforms(7, np.arange(n), np.zeros(n), 4 * nf)
    pf, wt, ok = ps.rambo_resonance(w, nf, m, g, u)
    a = np.where(ok, wt, 0.0) * integrand(pf)
    u2 = ps.uniforms(8, np.arange(n), np.zeros(n), 4 * nf)
    p2, w2 = ps.rambo_massless(w, nf, u2)
    b = w2 * integrand(p2)
    ma, ea = a.mean(), a.std() / math.sqrt(n)
    mb, eb = b.mean(), b.std() / math.sqrt(n)
    assert abs(ma - mb) < 4 * math.hypot(ea, eb)
    if shape == "breit-wigner":
        assert ea < 0.1 * eb  # the mapped generator flattens the resonance
