"""Counter-based random numbers, phase-space generators, cuts and the MC sum.

Oracle module (test infrastructure only), numpy FP64.

Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) written
from its published definition: ten rounds of
    (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
with the key bumped by the Weyl constants between rounds.  Event i, attempt
a, block j uses counter (i, a, j, 0) and key (seed, 0); each block gives four
64-bit words, each word two 32-bit deviates (low half first) mapped to doubles
in (0, 1) as (w + 1/2) 2^-32 -- 32-bit deviates like those of the paper's
generator (App. B).  Uniform i of a draw is half i % 2 of word (i % 8) // 2 of
block i // 8.

Generators (the paper's own parametrisation, App. A, is replaced by the
workload's stated generators; the Breit-Wigner mapping is the paper's Eq. 16):
  two_to_two_massless : cos(theta) ~ U[-1,1], phi ~ U[0, 2 pi)
  rambo_massless      : RAMBO (Kleiss, Stirling, Ellis 1986), flat n-body
  ttbar_dilepton      : sqrt(s) ~ U[a,b], Breit-Wigner t, t~, W+, W- virtualities
                        (Eq. 16, range |s-m^2|/(m Gamma) < min(20, m/Gamma),
                        App. A.2), isotropic two-body decays in each rest frame
  rambo_massive       : RAMBO with the massive rescaling (Kleiss et al. 1986)
  ypt_phi             : the paper's y, pT, phi parametrisation at fixed sqrt(s) (Eq. 13,
                        App. A.1) with the pT mapping of Eq. 17 and Breit-Wigner resonance
                        objects (App. A.2)
Cuts: the workloads' form pT > pt_min, |eta| < eta_max, Delta R > dr_min; and the paper's
selection of Eqs. 8-11 (pass_paper_cuts: jets with the Durham pT_ij, b jets, leptons).
A point failing the cuts (or the kinematic limits) is redrawn with the next
attempt number; the MC estimate divides by the number of tries (Eq. 4
integrated with the efficiency included).

Parity: pinned by tests/test_oracle_phasespace.py (Philox against numpy's
library Philox4x64, RAMBO volume/momentum conservation/masslessness,
two-body volume, Breit-Wigner Jacobian against direct integration, cut
definitions by brute force).
"""
import math
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """(high, low) 64-bit halves of the 128-bit product of uint64 arrays."""
    a_lo, a_hi = a & _M32, a >> _S32
    b_lo, b_hi = b & _M32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _M32) + (hl & _M32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(ctr, key):
    """ctr: uint64 [N, 4]; key: uint64 [N, 2] (or [2]); returns uint64 [N, 4]."""
    with np.errstate(over="ignore"):
        c = [ctr[:, k].astype(np.uint64) for k in range(4)]
        key = np.broadcast_to(np.asarray(key, dtype=np.uint64), (ctr.shape[0], 2))
        k0, k1 = key[:, 0].copy(), key[:, 1].copy()
        for r in range(10):
            hi0, lo0 = _mulhilo(M0, c[0])
            hi1, lo1 = _mulhilo(M1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            if r < 9:
                k0 = k0 + W0
                k1 = k1 + W1
        return np.stack(c, axis=1)


def to_unit32(w):
    """uint32 values (held in uint64) -> doubles in (0, 1): (w + 0.5) * 2^-32."""
    return (w.astype(np.float64) + 0.5) * (2.0 ** -32)


def uniforms(seed, event, attempt, n):
    """[N, n] doubles for events `event` at attempts `attempt` (uniform i: block i // 8,
    word (i % 8) // 2, its low 32 bits for even i, its high 32 bits for odd i)."""
    event = np.asarray(event, dtype=np.uint64)
    attempt = np.asarray(attempt, dtype=np.uint64)
    N = event.shape[0]
    nb = (n + 7) // 8
    out = np.empty((N, 8 * nb))
    for j in range(nb):
        ctr = np.stack([event, attempt, np.full(N, j, dtype=np.uint64), np.zeros(N, dtype=np.uint64)], axis=1)
        o = philox4x64_10(ctr, np.array([seed, 0], dtype=np.uint64))
        halves = np.stack([o & np.uint64(0xFFFFFFFF), o >> np.uint64(32)], axis=2).reshape(N, 8)
        out[:, 8 * j:8 * j + 8] = to_unit32(halves)
    return out[:, :n]


# ---------------------------------------------------------------------------
# generators
# ---------------------------------------------------------------------------
def incoming(w, N):
    """Beam partons along +z and -z, each with energy w/2."""
    pa = np.zeros((N, 4))
    pb = np.zeros((N, 4))
    pa[:, 0] = pa[:, 3] = 0.5 * w
    pb[:, 0] = 0.5 * w
    pb[:, 3] = -0.5 * w
    return pa, pb


def two_to_two_massless(w, u):
    """Legs (a, b, 3, 4): leg 4 at (cos theta = 2u0-1, phi = 2 pi u1), leg 3 opposite.

    Returns momenta [N, 4, 4] and the two-body volume 1/(8 pi)."""
    N = u.shape[0]
    c = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * math.pi * u[:, 1]
    s = np.sqrt(np.maximum(1.0 - c * c, 0.0))
    E = 0.5 * w
    P = np.zeros((N, 4, 4))
    P[:, 0], P[:, 1] = incoming(w, N)
    n = np.stack([s * np.cos(phi), s * np.sin(phi), c], axis=1)
    P[:, 3, 0] = E
    P[:, 3, 1:] = E * n
    P[:, 2, 0] = E
    P[:, 2, 1:] = -E * n
    return P, np.full(N, 1.0 / (8.0 * math.pi))


def rambo_volume(w, n):
    """Massless n-body volume with the (2 pi) factors of Eq. 5."""
    return ((2 * math.pi) ** (4 - 3 * n) * (math.pi / 2) ** (n - 1) * w ** (2 * n - 4)
            / (math.factorial(n - 1) * math.factorial(n - 2)))


def rambo_massless(w, n, u):
    """RAMBO: n massless momenta with total (w, 0, 0, 0); u [N, 4n] (4 per particle).

    Particle k: c = 2u-1, phi = 2 pi u', q0 = -ln(u'' u'''), q = q0 (1, s cos phi,
    s sin phi, c); then the conformal boost + scaling that brings sum q to (w,0,0,0).
    """
    N = u.shape[0]
    q = np.zeros((N, n, 4))
    for k in range(n):
        c = 2.0 * u[:, 4 * k] - 1.0
        phi = 2.0 * math.pi * u[:, 4 * k + 1]
        q0 = -np.log(u[:, 4 * k + 2] * u[:, 4 * k + 3])
        s = np.sqrt(np.maximum(1.0 - c * c, 0.0))
        q[:, k, 0] = q0
        q[:, k, 1] = q0 * s * np.cos(phi)
        q[:, k, 2] = q0 * s * np.sin(phi)
        q[:, k, 3] = q0 * c
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(axis=1))
    b = -Q[:, 1:] / M[:, None]
    gam = Q[:, 0] / M
    a = 1.0 / (1.0 + gam)
    x = w / M
    bq = np.einsum("nj,nkj->nk", b, q[:, :, 1:])
    p = np.zeros_like(q)
    p[:, :, 0] = x[:, None] * (gam[:, None] * q[:, :, 0] + bq)
    p[:, :, 1:] = x[:, None, None] * (q[:, :, 1:] + b[:, None, :] * q[:, :, :1] + (a[:, None] * bq)[:, :, None] * b[:, None, :])
    return p, np.full(N, rambo_volume(w, n))


def rambo_massive(w, masses, u, iterations=40):
    """Massive RAMBO: massless RAMBO followed by the rescaling p -> (sqrt(m^2 + xi^2 |p|^2), xi p)
    with xi solved by Newton iteration from sum E = w; weight per Kleiss et al. (1986)."""
    n = len(masses)
    p, wt0 = rambo_massless(w, n, u)
    m = np.asarray(masses, dtype=float)
    if not np.any(m > 0):
        return p, wt0
    E0 = p[:, :, 0]
    xi = np.full(p.shape[0], math.sqrt(max(1.0 - (m.sum() / w) ** 2, 0.0)))
    for _ in range(iterations):
        Ek = np.sqrt(m[None, :] ** 2 + (xi[:, None] * E0) ** 2)
        f = Ek.sum(axis=1) - w
        df = (xi[:, None] * E0 ** 2 / Ek).sum(axis=1)
        xi = xi - f / df
    Ek = np.sqrt(m[None, :] ** 2 + (xi[:, None] * E0) ** 2)
    out = np.empty_like(p)
    out[:, :, 0] = Ek
    out[:, :, 1:] = xi[:, None, None] * p[:, :, 1:]
    absk = xi[:, None] * E0
    # Kleiss et al.: W_massive = W_massless * xi^(2n-3) * prod(|k|/E) * w / sum(|k|^2/E)
    wt = wt0 * xi ** (2 * n - 3) * np.prod(absk / Ek, axis=1) * w / (absk ** 2 / Ek).sum(axis=1)
    return out, wt


def rambo_massive_events(w, masses, u, iterations=40):
    """rambo_massive with per-event masses [N, n] (same Newton solve and weight, row by row)."""
    m = np.asarray(masses, dtype=float)
    N, n = m.shape
    p, wt0 = rambo_massless(w, n, u)
    E0 = p[:, :, 0]
    xi = np.sqrt(np.maximum(1.0 - (m.sum(axis=1) / w) ** 2, 0.0))
    for _ in range(iterations):
        Ek = np.sqrt(m ** 2 + (xi[:, None] * E0) ** 2)
        f = Ek.sum(axis=1) - w
        df = (xi[:, None] * E0 ** 2 / Ek).sum(axis=1)
        xi = xi - f / df
    Ek = np.sqrt(m ** 2 + (xi[:, None] * E0) ** 2)
    out = np.empty_like(p)
    out[:, :, 0] = Ek
    out[:, :, 1:] = xi[:, None, None] * p[:, :, 1:]
    absk = xi[:, None] * E0
    wt = wt0 * xi ** (2 * n - 3) * np.prod(absk / Ek, axis=1) * w / (absk ** 2 / Ek).sum(axis=1)
    return out, wt


def rambo_resonance(w, nf, m, width, u):
    """nf massless final particles, the first two the decay products of a resonance of mass m and
    width `width` (App. A.2): dPhi_nf = dPhi_{nf-1}(R, 3..nf) ds/(2 pi) dPhi_2(R -> 1 2), with
    s = p_R^2 Breit-Wigner mapped (Eq. 16 range, bw_sample) and an isotropic decay at rest.
    u [N, 4 nf]: 4 RAMBO uniforms per particle of (R, 3, ..., nf), then theta, then the decay
    direction (cos = 2u - 1, phi = 2 pi u) of particle 1.
    Returns (pf [N, nf, 4] in the order 1, 2, 3, ..., nf; weight [N]; ok [N])."""
    N = u.shape[0]
    k = 4 * (nf - 1)
    s, jac = bw_sample(m, width, u[:, k])
    M = np.sqrt(np.maximum(s, 0.0))
    ok = (s > 0) & (M < w)
    Mr = np.where(ok, M, 0.5 * w)  # rejected rows get a harmless mass; their weight is unused
    masses = np.zeros((N, nf - 1))
    masses[:, 0] = Mr
    q, wt = rambo_massive_events(w, masses, u[:, :k])
    p1s, p2s, pabs = _iso_pair(Mr, np.zeros(N), np.zeros(N), 2.0 * u[:, k + 1] - 1.0, 2.0 * math.pi * u[:, k + 2])
    pf = np.empty((N, nf, 4))
    pf[:, 0] = _boost_from_rest(p1s, q[:, 0], Mr)
    pf[:, 1] = _boost_from_rest(p2s, q[:, 0], Mr)
    pf[:, 2:] = q[:, 1:]
    wt = wt * jac * pabs / (4.0 * math.pi * Mr)
    return pf, wt, ok


def _lam(a, b, c):
    return a * a + b * b + c * c - 2 * a * b - 2 * b * c - 2 * c * a


def _boost_from_rest(pstar, P, M):
    """Take pstar [N,4] from the rest frame of a system with lab momentum P [N,4], mass M [N]."""
    E = (P[:, 0] * pstar[:, 0] + (P[:, 1:] * pstar[:, 1:]).sum(axis=1)) / M
    coef = ((P[:, 1:] * pstar[:, 1:]).sum(axis=1) / (P[:, 0] + M) + pstar[:, 0]) / M
    out = np.empty_like(pstar)
    out[:, 0] = E
    out[:, 1:] = pstar[:, 1:] + coef[:, None] * P[:, 1:]
    return out


def _iso_pair(M, m1, m2, c, phi):
    """Two-body decay at rest: (p1*, p2*, |p*|) for daughter masses m1, m2, direction of 1."""
    pabs = np.sqrt(np.maximum(_lam(M * M, m1 * m1, m2 * m2), 0.0)) / (2.0 * M)
    s = np.sqrt(np.maximum(1.0 - c * c, 0.0))
    n = np.stack([s * np.cos(phi), s * np.sin(phi), c], axis=1)
    p1 = np.concatenate([np.sqrt(m1 * m1 + pabs * pabs)[:, None], pabs[:, None] * n], axis=1)
    p2 = np.concatenate([np.sqrt(m2 * m2 + pabs * pabs)[:, None], -pabs[:, None] * n], axis=1)
    return p1, p2, pabs


def bw_range(m, w, cap=20.0):
    """theta range of Eq. 16 for |s - m^2|/(m w) < min(cap, m/w) (App. A.2)."""
    x = min(cap, m / w)
    return -math.atan(x), math.atan(x)


def bw_sample(m, w, u):
    """s = m^2 + m w tan(theta), theta uniform in the App. A.2 range; returns (s, ds Jacobian / (2 pi))."""
    t0, t1 = bw_range(m, w)
    th = t0 + (t1 - t0) * u
    s = m * m + m * w * np.tan(th)
    jac = (t1 - t0) * ((s - m * m) ** 2 + (m * w) ** 2) / (m * w)
    return s, jac / (2.0 * math.pi)


def ttbar_dilepton(u, par, sqrt_s_range):
    """g g > t t~ > (b e+ ve)(b~ e- ve~); u [N, 16]. Returns (P [N,8,4], weight [N], ok [N], shat [N]).

    Draw order: sqrt(s), s_t, s_t~, s_W+, s_W-, top direction (cos, phi), b in
    the t frame, e+ in the W+ frame, b~ in the t~ frame, e- in the W- frame.
    weight = dPhi_2(s; t, t~) * prod ds/(2 pi) * dPhi_2(t; b, W+) dPhi_2(W+; e+, ve)
             * dPhi_2(t~; b~, W-) dPhi_2(W-; e-, ve~)   (Eq. 15, App. A.2)
    A point is kept only if sqrt(s_W) <= sqrt(s_t) for both tops and
    sqrt(s_t) + sqrt(s_t~) <= sqrt(s).
    """
    N = u.shape[0]
    lo, hi = sqrt_s_range
    rs = lo + (hi - lo) * u[:, 0]
    shat = rs * rs
    st, jt = bw_sample(par.mt, par.wt, u[:, 1])
    stb, jtb = bw_sample(par.mt, par.wt, u[:, 2])
    swp, jwp = bw_sample(par.mW, par.wW, u[:, 3])
    swm, jwm = bw_sample(par.mW, par.wW, u[:, 4])
    ok = (st > 0) & (stb > 0) & (swp > 0) & (swm > 0)
    st_ = np.where(ok, st, 1.0)
    stb_ = np.where(ok, stb, 1.0)
    swp_ = np.where(ok, swp, 1.0)
    swm_ = np.where(ok, swm, 1.0)
    mt_, mtb_, mwp_, mwm_ = np.sqrt(st_), np.sqrt(stb_), np.sqrt(swp_), np.sqrt(swm_)
    ok &= (mwp_ <= mt_) & (mwm_ <= mtb_) & (mt_ + mtb_ <= rs)
    two_pi = 2.0 * math.pi
    zeros = np.zeros(N)
    P = np.zeros((N, 8, 4))
    P[:, 0], P[:, 1] = incoming(rs, N)
    # production in the CM frame
    pt_, ptb_, k_prod = _iso_pair(rs, mt_, mtb_, 2 * u[:, 5] - 1, two_pi * u[:, 6])
    # t -> b W+
    b_, wp_, k_t = _iso_pair(mt_, zeros, mwp_, 2 * u[:, 7] - 1, two_pi * u[:, 8])
    b_ = _boost_from_rest(b_, pt_, mt_)
    wp_ = _boost_from_rest(wp_, pt_, mt_)
    # W+ -> e+ ve
    ep_, ve_, k_wp = _iso_pair(mwp_, zeros, zeros, 2 * u[:, 9] - 1, two_pi * u[:, 10])
    ep_ = _boost_from_rest(ep_, wp_, mwp_)
    ve_ = _boost_from_rest(ve_, wp_, mwp_)
    # t~ -> b~ W-
    bb_, wm_, k_tb = _iso_pair(mtb_, zeros, mwm_, 2 * u[:, 11] - 1, two_pi * u[:, 12])
    bb_ = _boost_from_rest(bb_, ptb_, mtb_)
    wm_ = _boost_from_rest(wm_, ptb_, mtb_)
    # W- -> e- ve~
    em_, vb_, k_wm = _iso_pair(mwm_, zeros, zeros, 2 * u[:, 13] - 1, two_pi * u[:, 14])
    em_ = _boost_from_rest(em_, wm_, mwm_)
    vb_ = _boost_from_rest(vb_, wm_, mwm_)
    for k, v in enumerate([b_, ep_, ve_, bb_, em_, vb_]):
        P[:, 2 + k] = v

    def phi2(k, M):
        return k / (4.0 * math.pi * M)

    wt = (phi2(k_prod, rs) * jt * jtb * jwp * jwm
          * phi2(k_t, mt_) * phi2(k_wp, mwp_) * phi2(k_tb, mtb_) * phi2(k_wm, mwm_))
    wt = np.where(ok, wt, 0.0)
    return P, wt, ok, shat


# ---------------------------------------------------------------------------
# the paper's parametrisation at fixed sqrt(s): rapidity, transverse momentum and azimuth
# (Eq. 13, App. A.1), the pT mapping of Eq. 17 and Breit-Wigner resonances (App. A.2)
# ---------------------------------------------------------------------------
def ypt_uniforms(objects):
    """Uniforms one y/pT/phi draw takes: 3 n - 3 for n objects, plus 3 per resonance object."""
    n = len(objects)
    return 3 * n - 3 + 3 * sum(1 for o in objects if len(o["legs"]) == 2)


def ypt_phi(w, objects, nf, u):
    """Momenta of nf final legs at partonic energy w in the centre-of-mass frame.

    objects: the n objects of the n-body phase space in generation order, each a dict with
      legs      (k,) one final leg (index among the final legs), or (k1, k2) a resonance decaying to two
                massless legs;
      mass      mass of a one-leg object; res_mass, res_width of a resonance;
      y_max     |y| < y_max;  pt_min, pt_max  pT range.
    Following App. A.1, dPhi_n = (2 pi)^(4 - 3n) 2^-n prod dy_i d^2 pT_i delta^4(P - sum p): the first
    n - 2 objects take y uniform in [-y_max, y_max], the first n - 1 take ln(pT^2 + m^2) uniform over
    their pT range (Eq. 17: d pT^2 = (pT^2 + m^2) d ln(pT^2 + m^2), m^2 = s_k for a resonance) and phi
    uniform; the last object's pT balances the others.  With the energy fixed (no x_a, x_b
    integration), the light-cone components P+- = sum mT_i exp(+-y_i) = w fix the rapidities of the
    last two objects (two solutions, one chosen by a uniform; Jacobian 2 mT_a mT_b |sinh(y_b - y_a)|).
    Their y_max and the last object's pT range hold a posteriori.  A resonance object (App. A.2):
    s = p^2 Breit-Wigner mapped (Eq. 16 range, bw_sample), isotropic two-body decay at rest.
    Uniform order: the resonances' s, the free rapidities, (pT, phi) of the first n - 1 objects, the
    solution, then each resonance's decay direction (cos = 2u - 1, phi = 2 pi u).
    Returns (pf [N, nf, 4], weight [N], ok [N])."""
    N = u.shape[0]
    n = len(objects)
    k = 0
    m2 = np.zeros((N, n))
    wt = np.ones(N)
    ok = np.ones(N, dtype=bool)
    for j, o in enumerate(objects):
        if len(o["legs"]) == 2:
            s, jac = bw_sample(o["res_mass"], o["res_width"], u[:, k])
            k += 1
            ok &= s > 0
            m2[:, j] = np.where(s > 0, s, 1.0)
            wt = wt * jac
        else:
            m2[:, j] = o.get("mass", 0.0) ** 2
    y = np.zeros((N, n))
    for j in range(n - 2):
        Y = objects[j]["y_max"]
        y[:, j] = (2.0 * u[:, k] - 1.0) * Y
        k += 1
        wt = wt * 2.0 * Y
    px = np.zeros((N, n))
    py = np.zeros((N, n))
    for j in range(n - 1):
        o = objects[j]
        L0 = np.log(o["pt_min"] ** 2 + m2[:, j])
        L1 = np.log(o["pt_max"] ** 2 + m2[:, j])
        L = L0 + u[:, k] * (L1 - L0)
        pt2 = np.maximum(np.exp(L) - m2[:, j], 0.0)
        ph = 2.0 * math.pi * u[:, k + 1]
        k += 2
        px[:, j] = np.sqrt(pt2) * np.cos(ph)
        py[:, j] = np.sqrt(pt2) * np.sin(ph)
        wt = wt * math.pi * (pt2 + m2[:, j]) * (L1 - L0)
    px[:, n - 1] = -px[:, : n - 1].sum(axis=1)
    py[:, n - 1] = -py[:, : n - 1].sum(axis=1)
    mt = np.sqrt(px ** 2 + py ** 2 + m2)
    # light-cone components P+- = mT exp(+-y) of the free objects; energies and longitudinal
    # momenta are formed from them, E = (P+ + P-)/2, pz = (P+ - P-)/2, so that the balance
    # sum P+- = w also holds for the stored momenta (E - pz of a forward particle is not a
    # difference of two large numbers)
    lp = np.zeros((N, n))
    lm = np.zeros((N, n))
    lp[:, : n - 2] = mt[:, : n - 2] * np.exp(y[:, : n - 2])
    lm[:, : n - 2] = mt[:, : n - 2] * np.exp(-y[:, : n - 2])
    Ap = w - lp[:, : n - 2].sum(axis=1)
    Am = w - lm[:, : n - 2].sum(axis=1)
    ok &= (Ap > 0) & (Am > 0)
    a, b = mt[:, n - 2], mt[:, n - 1]
    M2 = Ap * Am
    c = M2 + a * a - b * b
    D = c * c - 4.0 * M2 * a * a
    ok &= D >= 0
    root = np.sqrt(np.maximum(D, 0.0))
    # the two roots of Am X^2 - c X + a^2 Ap = 0: the larger without cancellation, the smaller from
    # the product of the roots a^2 Ap / Am (c - root loses the digits the balance of P- needs)
    Ams = np.where(Am > 0, Am, 1.0)
    big = (c + root) / (2.0 * Ams)
    small = a * a * Ap / (Ams * np.where(big > 0, big, 1.0))
    X = np.where(u[:, k] < 0.5, big, small)
    k += 1
    Z = Ap - X
    ok &= (X > 0) & (Z > 0)
    Xs, Zs = np.where(X > 0, X, 1.0), np.where(Z > 0, Z, 1.0)
    y[:, n - 2] = np.log(Xs / a)
    y[:, n - 1] = np.log(Zs / b)
    lp[:, n - 2], lm[:, n - 2] = Xs, a * a / Xs
    lp[:, n - 1], lm[:, n - 1] = Zs, b * b / Zs
    # Jacobian 2 mT_a mT_b |sinh(y_b - y_a)| with exp(y_b - y_a) = (Z a) / (X b)
    r = (Zs * a) / (Xs * b)
    J = a * b * np.abs(r - 1.0 / r)
    ok &= J > 0
    wt = wt * 2.0 / np.where(J > 0, J, 1.0) * 2.0
    for j in (n - 2, n - 1):
        ok &= np.abs(y[:, j]) <= objects[j]["y_max"]
    ptn = np.hypot(px[:, n - 1], py[:, n - 1])
    ok &= (ptn >= objects[n - 1]["pt_min"]) & (ptn <= objects[n - 1]["pt_max"])
    wt = wt * (2.0 * math.pi) ** (4 - 3 * n) * 2.0 ** (-n)
    E = 0.5 * (lp + lm)
    pz = 0.5 * (lp - lm)
    pf = np.zeros((N, nf, 4))
    for j, o in enumerate(objects):
        Pj = np.stack([E[:, j], px[:, j], py[:, j], pz[:, j]], axis=1)
        if len(o["legs"]) == 1:
            pf[:, o["legs"][0]] = Pj
    for j, o in enumerate(objects):
        if len(o["legs"]) == 2:
            M = np.sqrt(m2[:, j])
            Pj = np.stack([E[:, j], px[:, j], py[:, j], pz[:, j]], axis=1)
            p1, p2, pabs = _iso_pair(M, np.zeros(N), np.zeros(N), 2.0 * u[:, k] - 1.0, 2.0 * math.pi * u[:, k + 1])
            k += 2
            pf[:, o["legs"][0]] = _boost_from_rest(p1, Pj, M)
            pf[:, o["legs"][1]] = _boost_from_rest(p2, Pj, M)
            wt = wt * pabs / (4.0 * math.pi * M)
    return pf, np.where(ok, wt, 0.0), ok


# ---------------------------------------------------------------------------
# cuts
# ---------------------------------------------------------------------------
def pt(p):
    return np.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2)


def eta(p):
    """Pseudorapidity 1/2 ln((|p|+pz)/(|p|-pz))."""
    a = np.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2 + p[..., 3] ** 2)
    return 0.5 * np.log((a + p[..., 3]) / (a - p[..., 3]))


def phi(p):
    return np.arctan2(p[..., 2], p[..., 1])


def delta_r(p1, p2):
    dphi = np.abs(phi(p1) - phi(p2))
    dphi = np.where(dphi > math.pi, 2 * math.pi - dphi, dphi)
    return np.sqrt((eta(p1) - eta(p2)) ** 2 + dphi ** 2)


def pass_cuts(P, legs, pt_min, eta_max, dr_min):
    """All of legs have pT > pt_min and |eta| < eta_max, every pair Delta R > dr_min."""
    ok = np.ones(P.shape[0], dtype=bool)
    for k in legs:
        ptk = pt(P[:, k])
        ok &= ptk > pt_min
        with np.errstate(divide="ignore", invalid="ignore"):
            ok &= np.abs(eta(P[:, k])) < eta_max
    for i in range(len(legs)):
        for j in range(i + 1, len(legs)):
            with np.errstate(divide="ignore", invalid="ignore"):
                ok &= delta_r(P[:, legs[i]], P[:, legs[j]]) > dr_min
    return ok


# the paper's selection (Eqs. 8-11): jets |eta| < 5, pT > 20, and pT_ij = min(pT_i, pT_j) Delta R_ij > 20
# for every pair of jets (the Durham relative transverse momentum); b jets from top decays |eta| < 2.5,
# pT > 20, and charged leptons |eta| < 2.5, pT > 20, neither isolated
PAPER_CUTS = {"jet_pt": 20.0, "jet_eta": 5.0, "jet_ptij": 20.0, "b_pt": 20.0, "b_eta": 2.5, "lep_pt": 20.0,
              "lep_eta": 2.5}
JET, BJET, LEPTON = 1, 2, 3


def pass_paper_cuts(P, leg_class, c=PAPER_CUTS):
    """leg_class: per leg of P, 0 (no cut), JET, BJET or LEPTON."""
    ok = np.ones(P.shape[0], dtype=bool)
    jets = [k for k, cl in enumerate(leg_class) if cl == JET]
    with np.errstate(divide="ignore", invalid="ignore"):
        for k, cl in enumerate(leg_class):
            if cl == 0:
                continue
            ptmin, etamax = {JET: (c["jet_pt"], c["jet_eta"]), BJET: (c["b_pt"], c["b_eta"]),
                             LEPTON: (c["lep_pt"], c["lep_eta"])}[cl]
            ok &= (pt(P[:, k]) > ptmin) & (np.abs(eta(P[:, k])) < etamax)
        for i in range(len(jets)):
            for j in range(i + 1, len(jets)):
                a, b = P[:, jets[i]], P[:, jets[j]]
                ok &= np.minimum(pt(a), pt(b)) * delta_r(a, b) > c["jet_ptij"]
    return ok
