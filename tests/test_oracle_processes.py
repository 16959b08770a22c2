"""Pins of the oracle's |M|^2: closed forms, Parke-Taylor, Ward identity, Bose symmetry, boosts."""
import itertools
import math

import numpy as np
import pytest

from oracle import colour, phasespace as ps, processes as pr
from oracle.lorentz import boost, mdot, rotate
from oracle.sm import CHARGE, T3, SMParams

PAR = SMParams()


def two_to_two(sqrt_s, n, m3=0.0, m4=0.0, seed=0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.95, 0.95, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    s = sqrt_s ** 2
    pabs = math.sqrt((s - (m3 + m4) ** 2) * (s - (m3 - m4) ** 2)) / (2 * sqrt_s)
    P = np.zeros((n, 4, 4))
    P[:, 0] = [sqrt_s / 2, 0, 0, sqrt_s / 2]
    P[:, 1] = [sqrt_s / 2, 0, 0, -sqrt_s / 2]
    nvec = np.stack([np.sqrt(1 - c * c) * np.cos(phi), np.sqrt(1 - c * c) * np.sin(phi), c], axis=1)
    P[:, 2, 0] = math.sqrt(m3 * m3 + pabs * pabs)
    P[:, 2, 1:] = pabs * nvec
    P[:, 3, 0] = math.sqrt(m4 * m4 + pabs * pabs)
    P[:, 3, 1:] = -pabs * nvec
    return P


def rambo_points(sqrt_s, n_final, n, seed=0):
    u = np.random.default_rng(seed).uniform(0.01, 0.99, (n, 4 * n_final))
    pf, _ = ps.rambo_massless(sqrt_s, n_final, u)
    P = np.zeros((n, n_final + 2, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return P


def random_lorentz(P, seed):
    rng = np.random.default_rng(seed)
    beta = rng.normal(size=3)
    beta *= 0.9 / np.linalg.norm(beta)
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return rotate(boost(P, beta), R)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def test_uux_epem_closed_form():
    """u u~ > gamma/Z > e+ e-: helicity-amplitude closed form, theta = angle(e-, u)."""
    P = two_to_two(500.0, 64, seed=1)
    s = 500.0 ** 2
    c = P[:, 3, 3] / P[:, 3, 0]
    sw2 = PAR.sw2
    cw2 = 1 - sw2
    e = PAR.e
    prop = s / (s - PAR.mZ ** 2 + 1j * PAR.mZ * PAR.wZ)

    def g(f, chir):
        return T3[f] - CHARGE[f] * sw2 if chir == "L" else -CHARGE[f] * sw2

    A = {(i, j): CHARGE["u"] * CHARGE["e"] + g("u", i) * g("e", j) / (sw2 * cw2) * prop
         for i in "LR" for j in "LR"}
    want = (e ** 4 / 12.0) * ((1 + c) ** 2 * (abs(A["L", "L"]) ** 2 + abs(A["R", "R"]) ** 2)
                             + (1 - c) ** 2 * (abs(A["L", "R"]) ** 2 + abs(A["R", "L"]) ** 2))
    got = pr.uux_epem(P)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    # QED limit: Z switched off
    qed = PAR.with_(mZ=1e9, wZ=0.0)
    want_qed = e ** 4 * CHARGE["u"] ** 2 * (1 + c * c) / 3.0
    assert np.allclose(pr.uux_epem(P, qed), want_qed, rtol=1e-9)


def test_udx_epve_closed_form():
    """u d~ > W+ > e+ ve: avg|M|^2 = g^4/3 (p_u.p_e)(p_d.p_v) / |s - mW^2 + i mW GW|^2."""
    P = two_to_two(300.0, 64, seed=2)
    s = 300.0 ** 2
    D = abs(s - PAR.mW ** 2 + 1j * PAR.mW * PAR.wW) ** 2
    want = PAR.g ** 4 / 3.0 * mdot(P[:, 0], P[:, 2]) * mdot(P[:, 1], P[:, 3]) / D
    assert np.allclose(pr.udx_epve(P), want, rtol=1e-12)


def test_uux_gg_closed_form():
    P = two_to_two(1000.0, 64, seed=3)
    s = 1e6
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    want = PAR.gs ** 4 * ((32 / 27) * (t * t + u * u) / (t * u) - (8 / 3) * (t * t + u * u) / (s * s))
    assert np.allclose(pr.uux_gg(P), want, rtol=1e-12)


def test_gg_ttx_closed_form():
    mt = PAR.mt
    P = two_to_two(800.0, 64, m3=mt, m4=mt, seed=4)
    s = 800.0 ** 2
    t1 = 2 * mdot(P[:, 0], P[:, 2]) / s
    t2 = 2 * mdot(P[:, 1], P[:, 2]) / s
    rho = 4 * mt * mt / s
    want = PAR.gs ** 4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    assert np.allclose(pr.gg_ttx(P, widths=False), want, rtol=1e-12)


def test_gg_gg_closed_form():
    P = two_to_two(1500.0, 64, seed=5)
    s = 1500.0 ** 2
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    want = 4.5 * PAR.gs ** 4 * (3 - t * u / s ** 2 - s * u / t ** 2 - s * t / u ** 2)
    assert np.allclose(pr.gluons(P), want, rtol=1e-12)


# ---------------------------------------------------------------------------
# Parke-Taylor MHV amplitudes for 5 and 6 gluons
# ---------------------------------------------------------------------------
def _angle_products(K):
    """<ij> for all-outgoing massless momenta K [n, N, 4] (negative energies continued by i)."""
    n = K.shape[0]
    lam = []
    for k in range(n):
        sgn = np.sign(K[k][:, 0])
        q = K[k] * sgn[:, None]
        kp = q[:, 0] + q[:, 3]
        km = q[:, 0] - q[:, 3]
        big = kp > km
        kp_, km_ = np.where(big, kp, 1.0), np.where(big, 1.0, km)
        # the two forms differ by a phase only; pick the one without a small denominator
        l0 = np.where(big, np.sqrt(kp_) + 0j, (q[:, 1] - 1j * q[:, 2]) / np.sqrt(km_))
        l1 = np.where(big, (q[:, 1] + 1j * q[:, 2]) / np.sqrt(kp_), np.sqrt(km_) + 0j)
        fac = np.where(sgn < 0, 1j, 1.0)
        lam.append(np.stack([l0 * fac, l1 * fac], axis=1))
    ang = np.zeros((n, n, K.shape[1]), dtype=complex)
    for i in range(n):
        for j in range(n):
            ang[i, j] = lam[i][:, 0] * lam[j][:, 1] - lam[i][:, 1] * lam[j][:, 0]
    return ang


@pytest.mark.parametrize("n_final", [3, 4])
def test_mhv_parke_taylor(n_final):
    n = n_final + 2
    P = rambo_points(1500.0, n_final, 16, seed=6)
    K = np.stack([-P[:, 0], -P[:, 1]] + [P[:, k] for k in range(2, n)], axis=0)
    ang = _angle_products(K)
    assert np.allclose(np.abs(ang[0, 2]) ** 2, np.abs(2 * mdot(K[0], K[2])), rtol=1e-10)
    orders, C = colour.gluon_trace_matrix(n)
    g = PAR.gs
    for neg in [(0, 1), (0, 3), (2, 4)]:
        # outgoing helicities: legs in `neg` negative, the rest positive
        out_hel = [(-1 if k in neg else 1) for k in range(n)]
        phys = [(-h if k < 2 else h) for k, h in enumerate(out_hel)]
        E = []
        from oracle.lorentz import polarisation
        for k in range(n):
            eps = polarisation(P[:, k], phys[k])
            E.append(eps if k < 2 else eps.conj())
        _, A = pr.gluon_partial_amplitudes(K, np.stack(E), g)
        i, j = neg
        pt = []
        for o in orders:
            d = 1.0
            for a in range(n):
                d = d * ang[o[a], o[(a + 1) % n]]
            pt.append(g ** (n - 2) * ang[i, j] ** 4 / d)
        pt = np.array(pt)
        assert np.allclose(np.abs(A), np.abs(pt), rtol=1e-10)
        m2_or = np.real(np.einsum("sn,st,tn->n", A, C, A.conj()))
        m2_pt = np.real(np.einsum("sn,st,tn->n", pt, C, pt.conj()))
        assert np.allclose(m2_or, m2_pt, rtol=1e-10)


def test_all_plus_and_one_minus_vanish():
    P = rambo_points(1500.0, 4, 8, seed=7)
    _, ph = pr.gluons(P, per_helicity=True)
    tot = sum(ph.values())
    for h, v in ph.items():
        out = [(-x if k < 2 else x) for k, x in enumerate(h)]
        if sum(1 for x in out if x < 0) <= 1 or sum(1 for x in out if x > 0) <= 1:
            assert np.all(v < 1e-20 * tot)


# ---------------------------------------------------------------------------
# gauge invariance, Bose symmetry, Lorentz invariance
# ---------------------------------------------------------------------------
def test_ward_identity_w2j():
    P = rambo_points(1000.0, 4, 16, seed=8)
    ref = pr.udx_epvegg(P)
    for leg in (4, 5):
        bad = pr.udx_epvegg(P, eps_override={leg: P[:, leg]})
        # eps -> k scales the amplitude by ~E: amplitude-level residual below 1e-12
        assert np.all(bad < 1e-24 * ref * P[:, leg, 0] ** 2)


def test_ward_identity_gluons():
    P = rambo_points(1500.0, 3, 8, seed=9)
    ref = pr.gluons(P)
    bad = pr.gluons(P, eps_override={3: P[:, 3]})
    assert np.all(bad < 1e-24 * ref * P[:, 3, 0] ** 2)


def _ttbar_points(n, seed, par=PAR):
    u = np.random.default_rng(seed).uniform(0.02, 0.98, (4 * n, 16))
    P, wt, ok, _ = ps.ttbar_dilepton(u, par, (400.0, 2000.0))
    return P[ok][:n]


def test_ward_identity_ttbar_zero_width():
    """The resonant subset alone is not gauge invariant; the full set of gluon
    attachments to the b~ -> t~ ... t -> b line is, at zero widths."""
    par0 = PAR.with_(wt=0.0, wW=0.0)
    # points drawn with broad resonances, away from the poles the zero-width amplitude has
    P = _ttbar_points(8, 10, par=PAR.with_(wt=40.0, wW=25.0))
    ref = pr.gg_ttx_dilep(P, par0, all_attachments=True)
    for leg in (0, 1):
        bad = pr.gg_ttx_dilep(P, par0, eps_override={leg: P[:, leg]}, all_attachments=True)
        # near-collinear b-g propagators condition the cancellation; the resonant subset
        # alone leaves residuals of order 1e-3 here, a wrong sign or vertex O(1)
        assert np.all(bad < 1e-14 * ref * P[:, leg, 0] ** 2)


def test_bose_symmetry():
    P = rambo_points(1000.0, 4, 16, seed=11)
    Q = P[:, [0, 1, 2, 3, 5, 4]]
    assert np.allclose(pr.udx_epvegg(P), pr.udx_epvegg(Q), rtol=1e-12)
    P = _ttbar_points(8, 12)
    Q = P[:, [1, 0, 2, 3, 4, 5, 6, 7]]
    assert np.allclose(pr.gg_ttx_dilep(P), pr.gg_ttx_dilep(Q), rtol=1e-11)
    P = rambo_points(1500.0, 4, 4, seed=13)
    ref = pr.gluons(P)
    for perm in ([0, 1, 3, 2, 5, 4], [1, 0, 5, 4, 3, 2]):
        assert np.allclose(pr.gluons(P[:, perm]), ref, rtol=1e-11)


@pytest.mark.parametrize("name", ["u u~ > e+ e-", "u d~ > e+ ve g g", "g g > t t~ > b e+ ve b~ e- ve~",
                                  "u s > d c h h", "g g > g g g"])
def test_lorentz_invariance(name):
    if name == "u u~ > e+ e-":
        P = two_to_two(500.0, 16, seed=14)
    elif name == "g g > t t~ > b e+ ve b~ e- ve~":
        P = _ttbar_points(8, 15)
    elif name == "u s > d c h h":
        u = np.random.default_rng(16).uniform(0.02, 0.98, (16, 16))
        pf, _ = ps.rambo_massive(1000.0, [0.0, 0.0, PAR.mH, PAR.mH], u)
        P = np.zeros((16, 6, 4))
        P[:, 0], P[:, 1] = ps.incoming(1000.0, 16)
        P[:, 2:] = pf
    elif name == "g g > g g g":
        P = rambo_points(1500.0, 3, 8, seed=17)
    else:
        P = rambo_points(1000.0, 4, 16, seed=18)
    f = pr.PROCESSES[name]
    if name == "g g > t t~ > b e+ ve b~ e- ve~":
        # the doubly-resonant subset is not gauge invariant, so its helicity sum depends on the
        # frame that defines the gluon helicity vectors (eps^0 = 0): rotations only.  The full
        # attachment set at zero widths is gauge invariant and boost invariant.
        R, _ = np.linalg.qr(np.random.default_rng(19).normal(size=(3, 3)))
        assert np.allclose(f(rotate(P, R)), f(P), rtol=5e-11)
        par0 = PAR.with_(wt=0.0, wW=0.0)
        P = _ttbar_points(8, 15, par=PAR.with_(wt=40.0, wW=25.0))
        a = pr.gg_ttx_dilep(P, par0, all_attachments=True)
        b = pr.gg_ttx_dilep(random_lorentz(P, 19), par0, all_attachments=True)
        assert np.allclose(a, b, rtol=1e-8)
        return
    assert np.allclose(f(random_lorentz(P, 19)), f(P), rtol=5e-11)


def test_us_dchh_positive_and_finite():
    u = np.random.default_rng(20).uniform(0.02, 0.98, (32, 16))
    pf, _ = ps.rambo_massive(1000.0, [0.0, 0.0, PAR.mH, PAR.mH], u)
    P = np.zeros((32, 6, 4))
    P[:, 0], P[:, 1] = ps.incoming(1000.0, 32)
    P[:, 2:] = pf
    m2 = pr.us_dchh(P)
    assert np.all(np.isfinite(m2)) and np.all(m2 > 0)
    # symmetric under exchange of the two Higgs bosons
    assert np.allclose(pr.us_dchh(P[:, [0, 1, 2, 3, 5, 4]]), m2, rtol=1e-12)


def _ww_hh_point(par, w, c=0.3, phi=0.7):
    E = w / 2
    pw = math.sqrt(E * E - par.mW ** 2)
    ph = math.sqrt(E * E - par.mH ** 2)
    s = math.sqrt(1 - c * c)
    P = np.zeros((1, 4, 4))
    P[0, 0] = [E, 0, 0, pw]
    P[0, 1] = [E, 0, 0, -pw]
    P[0, 2] = [E, ph * s * math.cos(phi), ph * s * math.sin(phi), ph * c]
    P[0, 3] = [E, -P[0, 2, 1], -P[0, 2, 2], -P[0, 2, 3]]
    return P


def test_ww_hh_gauge_cancellation():
    """W_L W_L > h h: each diagram grows like s/mW^2, their sum tends to a finite
    constant (the Goldstone-boson amplitude of the equivalence theorem) only when the
    couplings g mW, g^2/2 and -3 mH^2/v and the unitary-gauge propagator are mutually
    consistent; a 10% error in any of them leaves a sum growing like s.  Zero W width:
    a fixed width in the t-channel W propagator spoils the cancellation (the effect the
    paper discusses for multi-Higgs production)."""
    par0 = PAR.with_(wW=0.0)
    vals = []
    for w in (1e4, 1e5, 1e6):
        amps = pr.wpwm_hh_amplitudes(_ww_hh_point(par0, w), (0, 0), par0)
        tot = sum(amps)[0]
        big = max(abs(a[0]) for a in amps)
        assert abs(tot) < 1e-3 * big or w == 1e4
        vals.append(tot)
    assert abs(vals[-1] / vals[-2] - 1) < 0.01
    assert abs(vals[-1]) < 10.0


def _ww_point(sqrt_s, cth, par=PAR):
    """u u~ > W+ W- at fixed sqrt(s) and cos(theta) of the W+ (one point)."""
    E = 0.5 * sqrt_s
    k = math.sqrt(E * E - par.mW ** 2)
    st = math.sqrt(1 - cth * cth)
    P = np.zeros((1, 4, 4))
    P[0, 0] = [E, 0, 0, E]
    P[0, 1] = [E, 0, 0, -E]
    P[0, 2] = [E, k * st, 0, k * cth]
    P[0, 3] = [E, -k * st, 0, -k * cth]
    return P


def test_uux_wpwm_gauge_cancellation():
    """Longitudinal W+ W- from u u~: the t-channel quark-exchange diagram grows like s/mW^2, and only
    with the WWA and WWZ couplings e and g cos(theta_W), the -i phase and the (W-, W+, V)
    orientation of the WWV vertex relative to the fermion couplings do the photon and Z diagrams
    cancel that growth: the summed |M|^2 tends to a constant while the t-channel amplitude alone
    rises a hundredfold per decade of sqrt(s).  Zero widths (a fixed Z width leaves a remainder
    growing like s)."""
    par0 = PAR.with_(wZ=0.0, wW=0.0)
    vals, tch = [], []
    for rs in (5e3, 5e4, 5e5):
        P = _ww_point(rs, 0.3, par0)
        m2 = 0.0
        for hf in itertools.product((-1, 1), (-1, 1)):
            a = pr.uux_wpwm_amplitudes(P, hf + (0, 0), par0)
            m2 += abs(sum(a)[0]) ** 2
        vals.append(m2)
        tch.append(abs(pr.uux_wpwm_amplitudes(P, (-1, 1, 0, 0), par0)[0][0]))
    assert tch[1] / tch[0] > 90 and tch[2] / tch[1] > 90
    assert abs(vals[2] / vals[1] - 1) < 1e-3 and abs(vals[1] / vals[0] - 1) < 0.05
    # the opposite phase of the WWV vertex (equivalently the opposite orientation) does not cancel
    P = _ww_point(5e4, 0.3, par0)
    a = pr.uux_wpwm_amplitudes(P, (-1, 1, 0, 0), par0)
    flipped = abs((a[0] - a[1] - a[2])[0]) ** 2
    assert flipped > 1e3 * vals[1]


def test_uux_wpwm_polarisation_sum_and_boosts():
    """The helicity sum over the three W polarisations equals the contraction of the amplitude
    tensor with -g^{mu nu} + k^mu k^nu / mW^2 for each W, and the summed |M|^2 is invariant under
    random Lorentz transformations."""
    P = two_to_two(800.0, 50, PAR.mW, PAR.mW, seed=5)
    ref = pr.uux_wpwm(P, PAR)
    # tensor form: amplitude as a function of the W polarisation vectors (basis vectors e_mu)
    from oracle.lorentz import bar, u_spinor, v_spinor
    from oracle.feynman import fermion_line, vector_insertion, vector_prop, vvv_out, ffv_current
    g = np.diag([1.0, -1.0, -1.0, -1.0])
    p = [P[:, k] for k in range(4)]
    gw = PAR.g / np.sqrt(2.0)
    q = p[0] + p[1]
    tot = 0.0
    for hf in itertools.product((-1, 1), (-1, 1)):
        u = u_spinor(p[0], hf[0])
        vb = bar(v_spinor(p[1], hf[1]))
        T = np.zeros((P.shape[0], 4, 4), dtype=complex)
        for mu in range(4):
            for nu in range(4):
                ep = np.zeros((P.shape[0], 4), dtype=complex)
                em = np.zeros((P.shape[0], 4), dtype=complex)
                ep[:, mu] = 1.0
                em[:, nu] = 1.0
                a = fermion_line(vb, u, p[0], [(vector_insertion(ep, gw, 0.0), p[2]),
                                               (vector_insertion(em, gw, 0.0), p[3])])
                X = vvv_out(em, -p[3], ep, -p[2], q, 1.0)
                ga = PAR.e * CHARGE["u"]
                gl, gr = PAR.gz * (T3["u"] - CHARGE["u"] * PAR.sw2), PAR.gz * (-CHARGE["u"] * PAR.sw2)
                a = a - 1j * PAR.e * mdot(X, vector_prop(q, ffv_current(vb, u, ga, ga)))
                a = a - 1j * PAR.g * PAR.cw * mdot(X, vector_prop(q, ffv_current(vb, u, gl, gr), PAR.mZ, PAR.wZ))
                T[:, mu, nu] = a / 1j
        # M = sum_ab eps+*^a eps-*^b T_ab; sum over polarisations of eps*^a eps^c = -g^{ac} + k^a k^c / m^2
        Pp = -g[None] + np.einsum("ni,nj->nij", p[2], p[2]) / PAR.mW ** 2
        Pm = -g[None] + np.einsum("ni,nj->nij", p[3], p[3]) / PAR.mW ** 2
        tot = tot + np.einsum("nab,ncd,nac,nbd->n", T, T.conj(), Pp, Pm).real
    tens = 3.0 * tot / 36.0
    assert np.allclose(tens, ref, rtol=1e-11)
    Q = random_lorentz(P, seed=6)
    assert np.allclose(pr.uux_wpwm(Q, PAR), ref, rtol=1e-10)


def test_udx_wpz_gauge_cancellation_and_boosts():
    """u d~ > W+ Z, longitudinal W and Z: the Z-from-u, Z-from-d and s-channel-W diagrams each grow like
    s/mW^2, and their sum stays finite only with the Z couplings of the two quark lines, the W
    propagator and the WWZ vertex of uux_wpwm_amplitudes (incoming W+ as V1) mutually consistent;
    the opposite WWZ phase grows like s^2 in |M|^2.  Zero widths.  The helicity sum is Lorentz
    invariant."""
    par0 = PAR.with_(wZ=0.0, wW=0.0)
    vals = []
    for rs in (5e3, 5e4, 5e5):
        mW, mZ = par0.mW, par0.mZ
        E3 = (rs * rs + mW * mW - mZ * mZ) / (2 * rs)
        k = math.sqrt(E3 * E3 - mW * mW)
        P = np.zeros((1, 4, 4))
        P[0, 0] = [rs / 2, 0, 0, rs / 2]
        P[0, 1] = [rs / 2, 0, 0, -rs / 2]
        P[0, 2] = [E3, k * math.sqrt(1 - 0.09), 0, k * 0.3]
        P[0, 3] = [rs - E3, -k * math.sqrt(1 - 0.09), 0, -k * 0.3]
        m2 = 0.0
        for hf in itertools.product((-1, 1), (-1, 1)):
            m2 += abs(sum(pr.udx_wpz_amplitudes(P, hf + (0, 0), par0))[0]) ** 2
        a = pr.udx_wpz_amplitudes(P, (-1, 1, 0, 0), par0)
        assert min(abs(x[0]) for x in a) > 1e3 * math.sqrt(m2) or rs == 5e3
        vals.append((m2, abs((a[0] + a[1] - a[2])[0]) ** 2))
    assert abs(vals[2][0] / vals[1][0] - 1) < 1e-3 and abs(vals[1][0] / vals[0][0] - 1) < 0.01
    assert vals[1][1] > 1e6 * vals[1][0]
    P = two_to_two(700.0, 40, PAR.mW, PAR.mZ, seed=8)
    ref = pr.udx_wpz(P, PAR)
    assert np.allclose(pr.udx_wpz(random_lorentz(P, seed=9), PAR), ref, rtol=1e-10)


def test_uu_uu_closed_form():
    """u u > u u (identical quarks): the spin- and colour-averaged |M|^2 of t- and u-channel gluon
    exchange alone, g_s^4 [4/9 ((s^2 + u^2)/t^2 + (s^2 + t^2)/u^2) - 8/27 s^2/(u t)], whose
    interference term carries the relative minus sign of the exchanged identical fermions and the
    colour factor Tr(t^a t^b t^a t^b); photon exchange alone, the Moller form times the colour
    factors 1 and 1/3; the full gluon + photon + Z result is Lorentz invariant."""
    P = two_to_two(400.0, 200, seed=4)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    ref = pr.uu_uu(P, PAR, bosons=("g",))
    cf = PAR.gs ** 4 * (4 / 9 * ((s * s + u * u) / t ** 2 + (s * s + t * t) / u ** 2) - 8 / 27 * s * s / (u * t))
    assert np.allclose(ref, cf, rtol=1e-12, atol=0)
    # photon alone: the Moller form with colour factors 1 (direct) and 1/3 (interference)
    eq4 = (PAR.e * CHARGE["u"]) ** 4
    ref = pr.uu_uu(P, PAR, bosons=("a",))
    cf = eq4 * (2 * ((s * s + u * u) / t ** 2 + (s * s + t * t) / u ** 2) + 4 / 3 * s * s / (u * t))
    assert np.allclose(ref, cf, rtol=1e-12, atol=0)
    # all bosons: Lorentz invariant, and different from the pure-QCD value by the electroweak terms
    full = pr.uu_uu(P, PAR)
    assert np.allclose(pr.uu_uu(random_lorentz(P, seed=10), PAR), full, rtol=1e-10)
    assert not np.allclose(full, pr.uu_uu(P, PAR, bosons=("g",)), rtol=1e-3)


def test_uux_zz_closed_form():
    """u u~ > Z Z: per point, (gL^4 + gR^4)/3 [t/u + u/t + 4 mZ^2 s/(t u) - mZ^4 (1/t^2 + 1/u^2)] (spin
    sum 4, colour sum 3, average 1/36), and symmetric under the exchange of the two Z bosons."""
    P = two_to_two(500.0, 100, PAR.mZ, PAR.mZ, seed=4)
    ref = pr.uux_zz(P, PAR)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    m2 = PAR.mZ ** 2
    gl = PAR.gz * (T3["u"] - CHARGE["u"] * PAR.sw2)
    gr = PAR.gz * (-CHARGE["u"] * PAR.sw2)
    cf = (gl ** 4 + gr ** 4) / 3.0 * (t / u + u / t + 4 * m2 * s / (t * u) - m2 * m2 * (1 / t ** 2 + 1 / u ** 2))
    assert np.allclose(ref, cf, rtol=1e-12, atol=0)
    assert np.allclose(pr.uux_zz(P[:, [0, 1, 3, 2]], PAR), ref, rtol=1e-12)


def test_uux_zh_closed_form():
    """u u~ > Z H through the s-channel Z: the spin trace with the Z polarisation sum gives, per point,
    g_ZZH^2 (gL^2 + gR^2) [s/2 + 2 (p1.k)(p2.k)/mZ^2] / (6 ((s - mZ^2)^2 + mZ^2 wZ^2)) (colour sum 3,
    average 1/36; the q q/mZ^2 part of the propagator vanishes on the massless current)."""
    P = two_to_two(600.0, 100, PAR.mZ, PAR.mH, seed=11)
    ref = pr.uux_zh(P, PAR)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    k = P[:, 2]
    gl = PAR.gz * (T3["u"] - CHARGE["u"] * PAR.sw2)
    gr = PAR.gz * (-CHARGE["u"] * PAR.sw2)
    m2 = PAR.mZ ** 2
    cf = ((PAR.gz * PAR.mZ) ** 2 * (gl ** 2 + gr ** 2) * (s / 2 + 2 * mdot(P[:, 0], k) * mdot(P[:, 1], k) / m2)
          / (6.0 * ((s - m2) ** 2 + m2 * PAR.wZ ** 2)))
    assert np.allclose(ref, cf, rtol=1e-12, atol=0)


def test_udx_wph_closed_form():
    """u d~ > W+ H through the s-channel W: the trace of the purely left-handed current with the W
    polarisation sum gives, per point, g_WWH^2 gW^2 [s/2 + 2 (p1.k)(p2.k)/mW^2] / (6 ((s - mW^2)^2 +
    mW^2 wW^2)), gW = g/sqrt2 (the ZH form with gL = gW, gR = 0)."""
    P = two_to_two(600.0, 100, PAR.mW, PAR.mH, seed=12)
    ref = pr.udx_wph(P, PAR)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    k = P[:, 2]
    m2 = PAR.mW ** 2
    cf = ((PAR.g * PAR.mW) ** 2 * (PAR.g ** 2 / 2) * (s / 2 + 2 * mdot(P[:, 0], k) * mdot(P[:, 1], k) / m2)
          / (6.0 * ((s - m2) ** 2 + m2 * PAR.wW ** 2)))
    assert np.allclose(ref, cf, rtol=1e-12, atol=0)


def _wwa_points(sqrt_s, n, seed, par=PAR):
    """u u~ > W+ W- gamma points from the oracle's massive RAMBO (masses mW, mW, 0)."""
    u = np.random.default_rng(seed).uniform(0.01, 0.99, (n, 12))
    pf, _ = ps.rambo_massive(sqrt_s, [par.mW, par.mW, 0.0], u)
    P = np.zeros((n, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return P


def test_uux_wpwma_ward_identity():
    """The photon's polarisation replaced by its momentum: with zero W and Z widths the fifteen
    diagrams of u u~ > W+ W- gamma sum to zero for every helicity of the quarks and W bosons, to
    rounding of the individual diagrams; without the two quartic diagrams, or with the quartic
    vertex's sign flipped, the sum is of the order of the diagrams."""
    P = _wwa_points(700.0, 40, seed=21)
    k = P[:, 4].astype(complex)
    for h in itertools.product((-1, 1), (-1, 1), (-1, 0, 1), (-1, 0, 1)):
        a = pr.uux_wpwma_amplitudes(P, h + (1,), PAR, eps_override=k, widths=False)
        allv = [x for v in a.values() for x in v]
        scale = sum(abs(x) for x in allv)
        tot = sum(allv)
        assert np.all(abs(tot) <= 1e-12 * scale)
        if h[2] == 0 and h[3] == 0 and h[0] != h[1]:
            noq = sum(x for key, v in a.items() if key != "quart" for x in v)
            assert np.all(abs(noq) > 1e-6 * scale)
            flip = noq - sum(a["quart"])
            assert np.all(abs(flip) > 1e-6 * scale)


def test_uux_wpwma_soft_photon_limit():
    """As the photon's energy w goes to zero, |M|^2(u u~ > W+ W- gamma) summed over the photon's
    helicities tends to -J.J |M|^2(u u~ > W+ W-) with the eikonal current J = e sum_i eta_i Q_i p_i /
    (p_i.k) over the four charged legs (eta = -1 incoming, +1 outgoing), the deviation falling in
    proportion to w.  Zero W width: a fixed width regulates the W propagator next to the emitted soft
    photon (1 / (2 p.k + i mW wW)) and removes the W terms of the eikonal limit."""
    par = PAR.with_(wW=0.0)
    base = two_to_two(500.0, 8, par.mW, par.mW, seed=22)
    m2 = pr.uux_wpwm(base, par)
    nhat = np.array([0.48, -0.6, 0.64])
    devs = []
    for w in (1e-1, 1e-2):
        P = np.zeros((8, 5, 4))
        P[:, :2] = base[:, :2]
        kph = np.concatenate([[w], w * nhat])
        Qv = base[:, 0] + base[:, 1] - kph
        Q2 = mdot(Qv, Qv)
        pst = np.sqrt(Q2 / 4 - par.mW ** 2)
        d = base[:, 2, 1:] / np.linalg.norm(base[:, 2, 1:], axis=1)[:, None]
        rest = np.zeros((8, 2, 4))
        rest[:, 0, 0] = rest[:, 1, 0] = np.sqrt(Q2) / 2
        rest[:, 0, 1:] = pst[:, None] * d
        rest[:, 1, 1:] = -pst[:, None] * d
        for i in range(8):
            beta = Qv[i, 1:] / Qv[i, 0]
            P[i, 2:4] = boost(rest[i], beta)
        P[:, 4] = kph
        assert np.allclose(P[:, 0] + P[:, 1], P[:, 2:].sum(axis=1), atol=1e-9)
        m3 = pr.uux_wpwma(P, par)
        qs = [(-1, CHARGE["u"], P[:, 0]), (-1, -CHARGE["u"], P[:, 1]), (1, 1.0, P[:, 2]), (1, -1.0, P[:, 3])]
        J = sum(eta * qc * p / mdot(p, P[:, 4])[:, None] for eta, qc, p in qs) * par.e
        soft = -mdot(J, J) * m2
        devs.append(np.max(np.abs(m3 / soft - 1)))
    assert devs[1] < 2e-3 and devs[1] < devs[0] / 5


def test_uux_wpwma_boosts():
    """|M|^2 of u u~ > W+ W- gamma is invariant under random Lorentz transformations."""
    P = _wwa_points(600.0, 12, seed=23)
    assert np.allclose(pr.uux_wpwma(random_lorentz(P, seed=24), PAR), pr.uux_wpwma(P, PAR), rtol=1e-10)


def _ttxh_points(sqrt_s, n, seed, mh=PAR.mH):
    u = np.random.default_rng(seed).uniform(0.01, 0.99, (n, 12))
    pf, _ = ps.rambo_massive(sqrt_s, [PAR.mt, PAR.mt, mh], u)
    P = np.zeros((n, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return P


def test_gg_ttxh_ward_identity():
    """Either gluon's polarisation replaced by its momentum: with zero top width the eight diagrams of
    g g > t t~ H sum to zero for every helicity of the other gluon and the tops."""
    P = _ttxh_points(1000.0, 20, seed=31)
    ref = pr.gg_ttxh(P, PAR, per_helicity=True, widths=False)
    for leg in (0, 1):
        ward = pr.gg_ttxh(P, PAR, per_helicity=True, widths=False, eps_override=(leg, P[:, leg].astype(complex)))
        for h, v in ward.items():
            assert np.all(np.abs(v) <= 1e-20 * np.abs(ref[h]) + 1e-24 * max(abs(x).max() for x in ref.values()))


def test_gg_ttxh_soft_higgs_limit():
    """A soft massless scalar emitted from the external top lines: as its energy w goes to zero, |M|^2
    of g g > t t~ H tends to (mt/v)^2 mt^2 [1/(p_t.k) + 1/(p_t~.k)]^2 |M|^2(g g > t t~), the deviation
    falling in proportion to w (the Higgs mass enters the amplitude only through its momentum)."""
    par = PAR
    base = two_to_two(800.0, 6, par.mt, par.mt, seed=32)
    m2 = pr.gg_ttx(base, par, widths=False)
    nhat = np.array([0.36, 0.48, -0.8])
    devs = []
    for w in (1e-1, 1e-2):
        P = np.zeros((6, 5, 4))
        P[:, :2] = base[:, :2]
        k = np.concatenate([[w], w * nhat])
        Qv = base[:, 0] + base[:, 1] - k
        Q2 = mdot(Qv, Qv)
        pst = np.sqrt(Q2 / 4 - par.mt ** 2)
        d = base[:, 2, 1:] / np.linalg.norm(base[:, 2, 1:], axis=1)[:, None]
        rest = np.zeros((6, 2, 4))
        rest[:, 0, 0] = rest[:, 1, 0] = np.sqrt(Q2) / 2
        rest[:, 0, 1:] = pst[:, None] * d
        rest[:, 1, 1:] = -pst[:, None] * d
        for i in range(6):
            P[i, 2:4] = boost(rest[i], Qv[i, 1:] / Qv[i, 0])
        P[:, 4] = k
        m3 = pr.gg_ttxh(P, par, widths=False)
        eik = (par.mt / par.vev) * par.mt * (1 / mdot(P[:, 2], k) + 1 / mdot(P[:, 3], k))
        devs.append(np.max(np.abs(m3 / (eik ** 2 * m2) - 1)))
    assert devs[1] < 2e-3 and devs[1] < devs[0] / 5


def test_gg_ttxh_bose_and_boosts():
    """Swapping the two gluons leaves |M|^2 unchanged; so do random Lorentz transformations."""
    P = _ttxh_points(900.0, 10, seed=33)
    ref = pr.gg_ttxh(P, PAR)
    assert np.allclose(pr.gg_ttxh(P[:, [1, 0, 2, 3, 4]], PAR), ref, rtol=1e-11)
    assert np.allclose(pr.gg_ttxh(random_lorentz(P, seed=34), PAR), ref, rtol=1e-10)


def test_hh_hh_closed_form():
    """h h > h h from the potential lambda (H^dag H - v^2/2)^2 with mH^2 = 2 lambda v^2: the h^3 and
    h^4 terms lambda v h^3 + lambda/4 h^4 give M = -6 lambda - (6 lambda v)^2 sum_{x=s,t,u} 1/(x - mH^2)
    at zero Higgs width.  Per point at 1e-12, and the high-energy limit (the contact term alone)."""
    par = PAR.with_(wH=0.0)
    P = np.zeros((40, 4, 4))
    rs = np.linspace(300.0, 3000.0, 40)
    rng = np.random.default_rng(41)
    for i, w in enumerate(rs):
        P[i] = two_to_two(w, 1, par.mH, par.mH, seed=int(rng.integers(1 << 30)))[0]
        pin = math.sqrt(w * w / 4 - par.mH ** 2)
        P[i, 0] = [w / 2, 0, 0, pin]
        P[i, 1] = [w / 2, 0, 0, -pin]
    lam = par.mH ** 2 / (2 * par.vev ** 2)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    m2 = par.mH ** 2
    M = -6 * lam - (6 * lam * par.vev) ** 2 * (1 / (s - m2) + 1 / (t - m2) + 1 / (u - m2))
    assert np.allclose(pr.hh_hh(P, par), M ** 2, rtol=1e-12, atol=0)
    Q = two_to_two(1e6, 4, par.mH, par.mH, seed=42)
    pin = math.sqrt(1e12 / 4 - par.mH ** 2)
    Q[:, 0] = [5e5, 0, 0, pin]
    Q[:, 1] = [5e5, 0, 0, -pin]
    assert np.allclose(pr.hh_hh(Q, par), 36 * lam ** 2, rtol=1e-3)


@pytest.mark.parametrize("which", ["w", "z"])
def test_qqx_vg_closed_form(which):
    """q q~' > V g with an on-shell massive V: the spin- and colour-averaged |M|^2 is
    (4/9) (gL^2 + gR^2) gs^2 (t^2 + u^2 + 2 s mV^2) / (t u), the massive-V form of the textbook
    q q~ > gamma g result (8/9) e^2 eq^2 gs^2 (t/u + u/t); t = (p_q - p_V)^2, u = (p_q - p_g)^2."""
    if which == "w":
        mV, gl, gr, fn = PAR.mW, PAR.g / math.sqrt(2.0), 0.0, pr.udx_wpg
    else:
        mV, fn = PAR.mZ, pr.uux_zg
        gl = PAR.gz * (T3["u"] - CHARGE["u"] * PAR.sw2)
        gr = PAR.gz * (-CHARGE["u"] * PAR.sw2)
    P = two_to_two(400.0, 64, mV, 0.0, seed=61)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    want = (4.0 / 9.0) * (gl ** 2 + gr ** 2) * PAR.gs ** 2 * (t * t + u * u + 2 * s * mV ** 2) / (t * u)
    assert np.allclose(fn(P, PAR), want, rtol=1e-12, atol=0)


def test_ug_wpd_crossed_closed_form():
    """u g > W+ d is u d~ > W+ g crossed (the d~ and the gluon exchanged, one fermion crossed: sign -1).
    The q q~ invariants map as s -> u, t -> t, u -> s, so summed over spins and colours it is
    -(4/9)(36)(gL^2)(gs^2)(s^2 + t^2 + 2 u mW^2)/(s t), averaged over 4 spins and 24 colours, with
    s = (p_u + p_g)^2, t = (p_u - p_W)^2, u = (p_u - p_d)^2."""
    mW, gl = PAR.mW, PAR.g / math.sqrt(2.0)
    P = two_to_two(400.0, 64, mW, 0.0, seed=71)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    summed = -(4.0 / 9.0) * 36.0 * gl ** 2 * PAR.gs ** 2 * (s * s + t * t + 2 * u * mW ** 2) / (s * t)
    assert np.allclose(pr.ug_wpd(P, PAR), summed / 96.0, rtol=1e-12, atol=0)


def _zzg_points(sqrt_s, n, seed):
    u = np.random.default_rng(seed).uniform(0.01, 0.99, (n, 12))
    pf, _ = ps.rambo_massive(sqrt_s, [PAR.mZ, PAR.mZ, 0.0], u)
    P = np.zeros((n, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return P


def test_uux_zzg_ward_soft_and_boosts():
    """u u~ > Z Z g: the gluon's polarisation replaced by its momentum gives zero; as the gluon's energy
    w goes to zero |M|^2 tends to gs^2 C_F 2 (p_u.p_u~) / ((p_u.k)(p_u~.k)) |M|^2(u u~ > Z Z), the
    deviation falling in proportion to w; and |M|^2 is Lorentz invariant."""
    P = _zzg_points(600.0, 20, seed=72)
    ref = pr.uux_zzg(P, PAR)
    ward = pr.uux_zzg(P, PAR, eps_override=P[:, 4].astype(complex))
    assert np.all(np.abs(ward) <= 1e-24 * ref)
    assert np.allclose(pr.uux_zzg(random_lorentz(P, seed=73), PAR), ref, rtol=1e-10)
    base = two_to_two(500.0, 6, PAR.mZ, PAR.mZ, seed=74)
    m2 = pr.uux_zz(base, PAR)
    nhat = np.array([0.6, 0.0, 0.8])
    devs = []
    for w in (1e-1, 1e-2):
        Q = np.zeros((6, 5, 4))
        Q[:, :2] = base[:, :2]
        k = np.concatenate([[w], w * nhat])
        Qv = base[:, 0] + base[:, 1] - k
        Q2 = mdot(Qv, Qv)
        pst = np.sqrt(Q2 / 4 - PAR.mZ ** 2)
        d = base[:, 2, 1:] / np.linalg.norm(base[:, 2, 1:], axis=1)[:, None]
        rest = np.zeros((6, 2, 4))
        rest[:, 0, 0] = rest[:, 1, 0] = np.sqrt(Q2) / 2
        rest[:, 0, 1:] = pst[:, None] * d
        rest[:, 1, 1:] = -pst[:, None] * d
        for i in range(6):
            Q[i, 2:4] = boost(rest[i], Qv[i, 1:] / Qv[i, 0])
        Q[:, 4] = k
        eik = PAR.gs ** 2 * (4.0 / 3.0) * 2 * mdot(Q[:, 0], Q[:, 1]) / (mdot(Q[:, 0], k) * mdot(Q[:, 1], k))
        devs.append(np.max(np.abs(pr.uux_zzg(Q, PAR) / (eik * m2) - 1)))
    assert devs[1] < 2e-3 and devs[1] < devs[0] / 5


def _ttxg_points(sqrt_s, n, seed):
    u = np.random.default_rng(seed).uniform(0.01, 0.99, (n, 12))
    pf, _ = ps.rambo_massive(sqrt_s, [PAR.mt, PAR.mt, 0.0], u)
    P = np.zeros((n, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    return P


@pytest.mark.parametrize("leg", [0, 1, 4])
def test_gg_ttxg_ward_identity(leg):
    """g g > t t~ g: any gluon's polarisation replaced by its momentum (zero top width) gives zero once
    all sixteen diagrams are summed: the three-gluon, four-gluon and quark-gluon rules must agree in
    sign and strength.  Dropping the four-gluon diagram breaks it."""
    P = _ttxg_points(1000.0, 4, seed=81)
    ref = pr.gg_ttxg(P, PAR, widths=False)
    ward = pr.gg_ttxg(P, PAR, widths=False, eps_override=(leg, P[:, leg].astype(complex)))
    assert np.all(np.abs(ward) <= 1e-20 * ref)


def test_gg_ttxg_bose_and_boosts():
    """Swapping the incoming gluons leaves |M|^2 unchanged; so do random Lorentz transformations."""
    P = _ttxg_points(900.0, 3, seed=82)
    ref = pr.gg_ttxg(P, PAR)
    assert np.allclose(pr.gg_ttxg(P[:, [1, 0, 2, 3, 4]], PAR), ref, rtol=1e-11)
    assert np.allclose(pr.gg_ttxg(random_lorentz(P, seed=83), PAR), ref, rtol=1e-10)


def test_gg_ttxg_ward_identity_needs_the_four_gluon_vertex(monkeypatch):
    """The Ward identity of g g > t t~ g fails when the four-gluon diagram is dropped or its sign
    flipped (a mistake planted in the oracle), so the pin above constrains that vertex."""
    P = _ttxg_points(1000.0, 3, seed=81)
    k4 = (4, P[:, 4].astype(complex))
    orig = pr._vvvv_out
    for planted in (lambda a, b, c: tuple(0 * x for x in orig(a, b, c)),
                    lambda a, b, c: tuple(-x for x in orig(a, b, c))):
        monkeypatch.setattr(pr, "_vvvv_out", planted)
        ref = pr.gg_ttxg(P, PAR, widths=False)
        assert np.all(np.abs(pr.gg_ttxg(P, PAR, widths=False, eps_override=k4)) > 1e-3 * ref)


def test_ttbar_chain_narrow_width_factorisation():
    """Integrated over the full six-body phase space at fixed sqrt(s) = 1 TeV, g g > t t~ > b e+ ve
    b~ e- ve~ factorises into the on-shell g g > t t~ phase-space integral times the square of the
    branching ratio B = [Gamma(t > b W) / wt] [Gamma(W > e ve) / wW], computed from the same couplings
    (Gamma(t > b W) = g^2 mt^3 (1 - r)^2 (1 + 2r) / (64 pi mW^2), r = mW^2/mt^2; Gamma(W > e ve) =
    g^2 mW / (48 pi)), times the fraction (2/pi) atan(20) of each Breit-Wigner inside the generator's
    window of 20 widths.  This pins the decay chain's normalisation (couplings, propagators, phase-space
    weights) against the closed-form-pinned g g > t t~.  The finite widths (wt/mt ~ 1 %, wW/mW ~ 3 %)
    and the Monte Carlo error (~2 % at 6,000 points) bound the agreement; 8 % is allowed."""
    par = PAR
    rs = 1000.0
    n = 6000
    u = np.random.default_rng(5).uniform(0.0, 1.0, (n, 16))
    P, wt, ok, _ = ps.ttbar_dilepton(u, par, (rs, rs))
    f = np.zeros(n)
    f[ok] = pr.gg_ttx_dilep(P[ok], par) * wt[ok]
    i6 = f.mean()
    x, wq = np.polynomial.legendre.leggauss(64)
    beta = math.sqrt(1 - 4 * par.mt ** 2 / rs ** 2)
    Q = np.zeros((64, 4, 4))
    Q[:, 0] = [rs / 2, 0, 0, rs / 2]
    Q[:, 1] = [rs / 2, 0, 0, -rs / 2]
    Q[:, 2, 0] = Q[:, 3, 0] = rs / 2
    Q[:, 2, 1] = beta * rs / 2 * np.sqrt(1 - x * x)
    Q[:, 2, 3] = beta * rs / 2 * x
    Q[:, 3, 1:] = -Q[:, 2, 1:]
    i2 = beta / (8 * math.pi) * 0.5 * np.sum(wq * pr.gg_ttx(Q, par, widths=False))
    g2 = par.g ** 2
    r = par.mW ** 2 / par.mt ** 2
    gamma_tbw = g2 * par.mt ** 3 * (1 - r) ** 2 * (1 + 2 * r) / (64 * math.pi * par.mW ** 2)
    gamma_wen = g2 * par.mW / (48 * math.pi)
    B = gamma_tbw / par.wt * gamma_wen / par.wW
    window = (2 / math.pi) * math.atan(20.0)
    assert abs(i6 / (i2 * B ** 2 * window ** 4) - 1) < 0.08


def _soft_emission_points(base, w, nhat, m2, m3):
    """2 -> 3 points from 2 -> 2 points: a massless emission of energy w along nhat, the two final
    particles (masses m2, m3) recoiling in their rest frame along the original direction."""
    n = base.shape[0]
    P = np.zeros((n, 5, 4))
    P[:, :2] = base[:, :2]
    k = np.concatenate([[w], w * np.asarray(nhat)])
    Qv = base[:, 0] + base[:, 1] - k
    Q2 = mdot(Qv, Qv)
    rq = np.sqrt(Q2)
    pst = np.sqrt((Q2 - (m2 + m3) ** 2) * (Q2 - (m2 - m3) ** 2)) / (2 * rq)
    d = base[:, 2, 1:] / np.linalg.norm(base[:, 2, 1:], axis=1)[:, None]
    rest = np.zeros((n, 2, 4))
    rest[:, 0, 0] = np.sqrt(m2 * m2 + pst * pst)
    rest[:, 1, 0] = np.sqrt(m3 * m3 + pst * pst)
    rest[:, 0, 1:] = pst[:, None] * d
    rest[:, 1, 1:] = -pst[:, None] * d
    for i in range(n):
        P[i, 2:4] = boost(rest[i], Qv[i, 1:] / Qv[i, 0])
    P[:, 4] = k
    return P


@pytest.mark.parametrize("which", ["zh", "wh", "wz", "ww"])
def test_v_pair_plus_gluon_ward_soft_and_boosts(which):
    """u u~ > Z H g, u d~ > W+ H g, u d~ > W+ Z g and u u~ > W+ W- g: the gluon's Ward identity; as the gluon's energy w goes to zero
    |M|^2 tends to gs^2 C_F 2 (p_q.p_q~) / ((p_q.k)(p_q~.k)) times |M|^2 without the gluon, the
    deviation falling in proportion to w; Lorentz invariance."""
    if which == "zh":
        fn, base_fn, m2, m3 = pr.uux_zhg, pr.uux_zh, PAR.mZ, PAR.mH
    elif which == "wh":
        fn, base_fn, m2, m3 = pr.udx_wphg, pr.udx_wph, PAR.mW, PAR.mH
    elif which == "wz":
        fn, base_fn, m2, m3 = pr.udx_wpzg, pr.udx_wpz, PAR.mW, PAR.mZ
    else:
        fn, base_fn, m2, m3 = pr.uux_wpwmg, pr.uux_wpwm, PAR.mW, PAR.mW
    u = np.random.default_rng(91).uniform(0.01, 0.99, (12, 12))
    pf, _ = ps.rambo_massive(600.0, [m2, m3, 0.0], u)
    P = np.zeros((12, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(600.0, 12)
    P[:, 2:] = pf
    ref = fn(P, PAR)
    assert np.all(np.abs(fn(P, PAR, eps_override=P[:, 4].astype(complex))) <= 1e-20 * ref)
    assert np.allclose(fn(random_lorentz(P, seed=92), PAR), ref, rtol=1e-10)
    base = two_to_two(500.0, 6, m2, m3, seed=93)
    mb = base_fn(base, PAR)
    devs = []
    for w in (1e-1, 1e-2):
        Q = _soft_emission_points(base, w, [0.0, 0.6, 0.8], m2, m3)
        k = Q[:, 4]
        eik = PAR.gs ** 2 * (4.0 / 3.0) * 2 * mdot(Q[:, 0], Q[:, 1]) / (mdot(Q[:, 0], k) * mdot(Q[:, 1], k))
        devs.append(np.max(np.abs(fn(Q, PAR) / (eik * mb) - 1)))
    assert devs[1] < 2e-3 and devs[1] < devs[0] / 5


@pytest.mark.parametrize("which", ["w", "z"])
def test_gg_vqqx_ward_bose_and_boosts(which):
    """g g > W+ d u~ and g g > Z u u~: either gluon's polarisation replaced by its momentum gives zero once the six
    quark-line orderings and the two s-channel-gluon diagrams are summed; the gluons are
    interchangeable; |M|^2 is Lorentz invariant.  The external quarks are put exactly on shell
    (E = |p|): an external massless spinor of a momentum with p^2 = eps E^2 breaks the identity at
    sqrt(eps), and RAMBO's rescaling leaves eps ~ 1e-15."""
    fn, mV = (pr.gg_wpdux, PAR.mW) if which == "w" else (pr.gg_zuux, PAR.mZ)
    u = np.random.default_rng(101).uniform(0.01, 0.99, (10, 12))
    pf, _ = ps.rambo_massive(700.0, [mV, 0.0, 0.0], u)
    P = np.zeros((10, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(700.0, 10)
    P[:, 2:] = pf
    for k in (3, 4):
        P[:, k, 0] = np.linalg.norm(P[:, k, 1:], axis=1)
    ref = fn(P, PAR)
    for leg in (0, 1):
        assert np.all(np.abs(fn(P, PAR, eps_override=(leg, P[:, leg].astype(complex)))) <= 1e-20 * ref)
    assert np.allclose(fn(P[:, [1, 0, 2, 3, 4]], PAR), ref, rtol=1e-11)
    assert np.allclose(fn(random_lorentz(P, seed=102), PAR), ref, rtol=1e-10)


def test_uux_ttx_closed_forms():
    """u u~ > t t~: with F = (mt^2 - t)^2 + (mt^2 - u)^2 + 2 mt^2 s, the gluon exchange alone gives
    (4/9) gs^4 F / s^2 and the photon exchange alone 2 e^4 Qu^2 Qt^2 F / s^2 (colour factors 2 and
    9 over 36, the massive-final-state QED trace); the gluon does not interfere with the photon or
    the Z (colour orthogonality); |M|^2 is Lorentz invariant."""
    mt = PAR.mt
    P = two_to_two(900.0, 40, mt, mt, seed=111)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    F = (mt * mt - t) ** 2 + (mt * mt - u) ** 2 + 2 * mt * mt * s
    assert np.allclose(pr.uux_ttx(P, PAR, bosons=("g",)), (4.0 / 9.0) * PAR.gs ** 4 * F / s ** 2, rtol=1e-12)
    qa = PAR.e ** 2 * CHARGE["u"] * CHARGE["t"]
    assert np.allclose(pr.uux_ttx(P, PAR, bosons=("a",)), 2 * qa ** 2 * F / s ** 2, rtol=1e-12)
    full = pr.uux_ttx(P, PAR)
    assert np.allclose(full, pr.uux_ttx(P, PAR, bosons=("g",)) + pr.uux_ttx(P, PAR, bosons=("a", "z")), rtol=1e-12)
    assert np.allclose(pr.uux_ttx(random_lorentz(P, seed=112), PAR), full, rtol=1e-10)


def test_uux_ttxg_ward_and_boosts():
    """u u~ > t t~ g: the gluon's polarisation replaced by its momentum gives zero (zero top width)
    once the thirteen diagrams are summed; |M|^2 is Lorentz invariant."""
    u = np.random.default_rng(121).uniform(0.01, 0.99, (8, 12))
    pf, _ = ps.rambo_massive(1000.0, [PAR.mt, PAR.mt, 0.0], u)
    P = np.zeros((8, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(1000.0, 8)
    P[:, 2:] = pf
    P[:, 4, 0] = np.linalg.norm(P[:, 4, 1:], axis=1)
    ref = pr.uux_ttxg(P, PAR, widths=False)
    ward = pr.uux_ttxg(P, PAR, widths=False, eps_override=P[:, 4].astype(complex))
    assert np.all(np.abs(ward) <= 1e-20 * ref)
    full = pr.uux_ttxg(P, PAR)
    assert np.allclose(pr.uux_ttxg(random_lorentz(P, seed=122), PAR), full, rtol=1e-10)


def test_us_dch_closed_form():
    """u s > d c H through W+ W- fusion: the two left-handed currents give
    sum_spins |[d gamma^mu P_L u][c gamma_mu P_L s]|^2 = 16 (p_u.p_s)(p_d.p_c) (the V-A trace of muon
    decay with P_L = (1 - gamma5)/2), so |M|^2 = (9/36) gWWH^2 gW^4 16 (p_u.p_s)(p_d.p_c) /
    (|q1^2 - mW^2 + i mW wW|^2 |q2^2 - mW^2 + i mW wW|^2), q1 = p_u - p_d, q2 = p_s - p_c (the
    propagators' q q / mW^2 terms vanish on the conserved massless currents)."""
    u = np.random.default_rng(131).uniform(0.01, 0.99, (30, 12))
    pf, _ = ps.rambo_massive(1000.0, [0.0, 0.0, PAR.mH], u)
    P = np.zeros((30, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(1000.0, 30)
    P[:, 2:] = pf
    for k in (2, 3):
        P[:, k, 0] = np.linalg.norm(P[:, k, 1:], axis=1)
    gw2 = PAR.g ** 2 / 2
    q1 = P[:, 0] - P[:, 2]
    q2 = P[:, 1] - P[:, 3]
    den = lambda q: (mdot(q, q) - PAR.mW ** 2) ** 2 + (PAR.mW * PAR.wW) ** 2
    want = (9.0 / 36.0) * (PAR.g * PAR.mW) ** 2 * gw2 ** 2 * 16 * mdot(P[:, 0], P[:, 1]) * mdot(P[:, 2], P[:, 3]) \
        / (den(q1) * den(q2))
    assert np.allclose(pr.us_dch(P, PAR), want, rtol=1e-10)


def _wa_points(rs, cos_uph, phi):
    """u d~ > W+ gamma in the CM frame with the photon at angle theta to the u (cos theta = cos_uph)."""
    n = len(cos_uph)
    pabs = (rs ** 2 - PAR.mW ** 2) / (2 * rs)
    P = np.zeros((n, 4, 4))
    P[:, 0] = [rs / 2, 0, 0, rs / 2]
    P[:, 1] = [rs / 2, 0, 0, -rs / 2]
    s_ = np.sqrt(1 - cos_uph ** 2)
    P[:, 3] = np.stack([np.full(n, pabs), pabs * s_ * np.cos(phi), pabs * s_ * np.sin(phi), pabs * cos_uph], axis=1)
    P[:, 2, 0] = math.sqrt(PAR.mW ** 2 + pabs ** 2)
    P[:, 2, 1:] = -P[:, 3, 1:]
    return P


def test_udx_wpa_radiation_zero():
    """u d~ > W+ gamma has the radiation amplitude zero: at zero W width every helicity amplitude
    vanishes when the photon leaves at cos theta = -1/3 to the u direction (the point where the photon
    couplings of the u, the d~ and the W, weighted by their eikonal factors, cancel; Mikaelian, Samuel
    and Sahdev 1979).  It needs the WWA vertex with the quark couplings' sign and strength."""
    rng = np.random.default_rng(141)
    for rs in (300.0, 600.0, 2000.0):
        phi = rng.uniform(0, 2 * np.pi, 5)
        at_zero = pr.udx_wpa(_wa_points(rs, np.full(5, -1.0 / 3.0), phi), PAR, widths=False)
        away = pr.udx_wpa(_wa_points(rs, np.full(5, 0.5), phi), PAR, widths=False)
        assert np.all(at_zero <= 1e-20 * away)
        assert np.all(pr.udx_wpa(_wa_points(rs, np.full(5, -0.2), phi), PAR, widths=False) > 1e-3 * away)


@pytest.mark.parametrize("which", ["za", "aa"])
def test_uux_va_closed_form(which):
    """u u~ > Z gamma and u u~ > gamma gamma: the q q~ > V g form with the gluon replaced by a photon,
    the colour factor C_F N_c = 4 by N_c = 3: (1/3)(gL^2 + gR^2) e^2 Qu^2 (t^2 + u^2 + 2 s mV^2)/(t u);
    for two photons (2/3) e^4 Qu^4 (t/u + u/t), the textbook q q~ > gamma gamma result."""
    qa = PAR.e * CHARGE["u"]
    if which == "za":
        mV, fn = PAR.mZ, pr.uux_za
        gl = PAR.gz * (T3["u"] - CHARGE["u"] * PAR.sw2)
        gr = PAR.gz * (-CHARGE["u"] * PAR.sw2)
    else:
        mV, fn, gl, gr = 0.0, pr.uux_aa, qa, qa
    P = two_to_two(400.0, 64, mV, 0.0, seed=151)
    s = mdot(P[:, 0] + P[:, 1], P[:, 0] + P[:, 1])
    t = mdot(P[:, 0] - P[:, 2], P[:, 0] - P[:, 2])
    u = mdot(P[:, 0] - P[:, 3], P[:, 0] - P[:, 3])
    want = (1.0 / 3.0) * (gl ** 2 + gr ** 2) * qa ** 2 * (t * t + u * u + 2 * s * mV ** 2) / (t * u)
    assert np.allclose(fn(P, PAR), want, rtol=1e-12, atol=0)
    if which == "aa":
        assert np.allclose(want, (2.0 / 3.0) * qa ** 4 * (t / u + u / t), rtol=1e-12)


# ---------------------------------------------------------------------------
# NMHV six-gluon amplitudes: the soft-gluon limit of every colour-ordered amplitude
# ---------------------------------------------------------------------------
def test_nmhv_six_gluon_soft_limit():
    """A colour-ordered amplitude with a soft positive-helicity gluon s between its neighbours a and b
    tends to g <a b> / (<a s> <s b>) times the amplitude without s (the universal soft factor in the
    normalisation of the Parke-Taylor pin above), with a deviation that falls in proportion to the
    soft energy.  With three negative helicities among the six, every one of the 120 orderings of
    this NMHV helicity reduces to a five-gluon anti-MHV amplitude, itself pinned by Parke-Taylor."""
    from test_oracle_chains import _add_soft_massive
    from oracle.lorentz import polarisation
    g = PAR.gs
    base = rambo_points(1500.0, 3, 6, seed=31)
    out_hel = [-1, -1, 1, -1, 1]                    # five hard gluons (outgoing convention)

    def amps(P, hels):
        n = P.shape[1]
        K = np.stack([-P[:, 0], -P[:, 1]] + [P[:, k] for k in range(2, n)], axis=0)
        phys = [(-h if k < 2 else h) for k, h in enumerate(hels)]
        E = []
        for k in range(n):
            eps = polarisation(P[:, k], phys[k])
            E.append(eps if k < 2 else eps.conj())
        orders, A = pr.gluon_partial_amplitudes(K, np.stack(E), g)
        return K, orders, A

    _, orders5, A5 = amps(base, out_hel)
    index5 = {o: i for i, o in enumerate(orders5)}
    nhat = np.array([0.36, -0.48, 0.8])
    devs = []
    for lam in (1e-4, 1e-5):
        w = lam * 1500.0
        k = np.concatenate([[w], w * nhat])[None, :].repeat(len(base), 0)
        P6 = _add_soft_massive(base, k, (0.0, 0.0, 0.0))
        K6, orders6, A6 = amps(P6, out_hel + [1])
        ang = _angle_products(K6)
        dev = 0.0
        for i6, o in enumerate(orders6):
            pos = o.index(5)
            a, b = o[pos - 1], o[(pos + 1) % 6]
            o5 = tuple(x for x in o if x != 5)
            soft = g * np.abs(ang[a, b] / (ang[a, 5] * ang[5, b]))
            want = soft * np.abs(A5[index5[o5]])
            dev = max(dev, float(np.max(np.abs(np.abs(A6[i6]) / want - 1))))
        devs.append(dev)
    assert devs[1] < 1e-3 and devs[1] < devs[0] / 5, devs
