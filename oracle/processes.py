"""Spin- and colour-summed |M|^2 of the workload processes, from the plain definition.

Oracle module (test infrastructure only).  For each process the Feynman
diagrams are written out by hand from the vertices of Sect. 4.2, every
helicity combination is evaluated (no pruning), and colour is summed over
every explicit colour index (oracle/colour.py).  The result is averaged over
the initial helicities and colours, Eq. 4:

    |M|^2_avg = 1/(4 n_a n_b) sum_lambda sum_c |sum_diagrams M|^2 .

No identical-particle factor is applied here (that belongs to the phase-space
integral).  Momenta: array [N, n_ext, 4] of physical four-momenta (E, px, py,
pz), incoming legs first, in the order of the process string.

Functions and their pins (tests/test_oracle_processes.py):
  uux_epem        u u~ > e+ e-   : closed-form dsigma/dcos(theta), exact per point
  udx_epve        u d~ > e+ ve   : closed form (V-A), exact per point
  udx_epvegg      u d~ > e+ ve g g : Ward identity, Bose symmetry, boosts; its
                   normalisation by the soft limit of either gluon against the
                   colour-correlated eikonal factor of q, q~, g times u d~ > e+ ve g
  uux_gg          u u~ > g g     : textbook closed form, exact per point
  gg_ttx          g g > t t~     : textbook closed form (massive), exact per point
  uux_ttx         u u~ > t t~    : textbook closed forms of the gluon and the photon exchange (massive
                   final quarks), exact per point; no gluon-electroweak interference; boosts
  uux_ttxg        u u~ > t t~ g  : Ward identity for the gluon (zero top width), boosts
  hh_hh           h h > h h      : closed form from the Higgs potential, exact per point
  gg_ttxg         g g > t t~ g   : Ward identity for each of the three gluons (zero top width), Bose
                   symmetry of the incoming gluons, boosts
  gg_ttxh         g g > t t~ h   : Ward identity for each gluon (zero top width), the soft-Higgs
                   limit against the eikonal factor times g g > t t~, Bose symmetry, boosts
  gg_ttx_dilep    g g > t t~ > b e+ ve b~ e- ve~ (doubly resonant diagrams):
                   Ward identity (zero widths), Bose symmetry, boosts
  uu_uu           u u > u u      : gluon, photon and Z exchange; textbook closed forms for
                   the gluon part and the photon part, exact per point; boosts
  uux_zz          u u~ > z z     : closed form, exact per point; Bose symmetry
  uux_zh          u u~ > z h     : closed form from the trace, exact per point
  udx_wph         u d~ > w+ h    : closed form from the trace, exact per point
  udx_wpg, uux_zg q q~ > V g     : textbook closed form (t^2 + u^2 + 2 s mV^2)/(t u), exact per point
  uux_za, uux_aa  u u~ > z a, a a: the same form with the photon (colour N_c in place of C_F N_c)
  gg_wpdux, gg_zuux  g g > w+ d u~, g g > z u u~ : Ward identity for each gluon, Bose symmetry, boosts
  ug_wpd          u g > w+ d     : the same closed form crossed (s <-> u, one fermion: sign -1), exact
  uux_zzg         u u~ > z z g   : Ward identity for the gluon, the soft-gluon limit against C_F times
                   the eikonal factor times u u~ > z z, boosts
  uux_zhg, udx_wphg, udx_wpzg, uux_wpwmg  u u~ > z h g, u d~ > w+ h g, u d~ > w+ z g,
                   u u~ > w+ w- g : the same three pins against the processes without the gluon
  uux_wpwm        u u~ > w+ w-   : gauge cancellation of the longitudinal amplitude
                   (each diagram grows like s/mW^2, the sum stays finite), the W
                   polarisation sum against the tensor form -g + k k/mW^2, boosts
  udx_wpa         u d~ > w+ a    : the radiation amplitude zero at cos(u, photon) = -1/3
  udx_wpz         u d~ > w+ z    : gauge cancellation of the longitudinal amplitude
                   (the WWZ vertex with an incoming W), boosts
  uux_wpwma       u u~ > w+ w- a : the photon's Ward identity with zero W and Z widths (the
                   fifteen diagrams cancel only with the quartic WWAA and WWAZ vertices),
                   the soft-photon limit against the eikonal factor times u u~ > w+ w-, boosts
  us_dch          u s > d c h    (WW fusion): closed form from the V-A traces, exact per point
  us_dchg         u s > d c h g  (WW fusion plus one jet): Ward identity, the soft-gluon limit
                   against 2 C_F (S_ud + S_sc) times u s > d c h (the lines' colours do not
                   interfere), boosts
  us_dchgg        u s > d c h g g (WBF H plus two jets, 24 diagrams) on the two-line code (us_dch_ng),
                   which equals us_dch and us_dchg at 0 and 1 gluons; Ward identity for each gluon (fails
                   without the pair lines), Bose symmetry, boosts (tests/test_oracle_line.py)
  udx_wpzgg       u d~ > w+ z g g (W+ Z plus two jets) on the one-fermion-line engine (the Z before or after
                   the W emission, with the u or the d couplings, or an s-channel W into W W Z), which
                   equals udx_wpz and udx_wpzg with no and one gluon; Ward identity for each gluon, Bose
                   symmetry, boosts (tests/test_oracle_line.py)
  uux_wpwmgg      u u~ > w+ w- g g (W+ W- plus two jets, 31 diagrams) on the one-fermion-line engine (the
                   t-channel W pair in its fixed order, or an s-channel photon or Z into the W W V vertex),
                   which equals uux_wpwm and uux_wpwmg with no and one gluon; Ward identity for each
                   gluon, Bose symmetry, boosts (tests/test_oracle_line.py)
  udx_wphggg      u d~ > w+ h g g g (H V plus three jets, 54 diagrams) on the same engine: Ward identity for
                   each gluon (fails without the four-gluon lines), Bose symmetry, boosts
                   (tests/test_oracle_line.py)
  udx_wphgg       u d~ > w+ h g g (H V plus two jets, 8 diagrams) on the one-fermion-line engine (a W* > W+ H
                   insertion), which equals udx_wph and udx_wphg with no and one gluon; Ward identity for
                   each gluon, Bose symmetry, boosts (tests/test_oracle_line.py)
  uux_zzgg        u u~ > z z g g (V V plus two jets, 30 diagrams) on the one-fermion-line engine, which
                   equals uux_zz and uux_zzg with no and one gluon; Ward identity for each gluon, Bose
                   symmetry of the gluons and of the Z bosons, boosts (tests/test_oracle_line.py)
  gg_ttxgg        g g > t t~ g g (t t~ plus two jets, 159 diagrams) on the one-fermion-line engine with
                   four-gluon trees (_gluon_trees; recursive currents and vectorised colour tensors, both
                   checked against the three-gluon forms); Ward identity for each gluon at zero top width
                   (fails without the four-gluon vertex in the trees), Bose symmetry, boosts
                   (tests/test_oracle_line.py)
  gg_ttxhg        g g > t t~ h g (H t t~ plus one jet, 54 diagrams) on the one-fermion-line engine
                   (fermion_line_process), which equals gg_ttxh, gg_ttxg and udx_wpggg point by point;
                   Ward identity for each gluon (fails without the triple-gluon lines), Bose symmetry,
                   boosts (tests/test_oracle_line.py)
  udx_wpggg, uux_zggg  u d~ > w+ g g g, u u~ > z g g g (V plus three jets, 54 diagrams): the generic
                   q q~ > V + n gluons code (qqx_v_ng) equals q q~ > V g and q q~ > V g g at n = 1, 2;
                   at n = 3 the Ward identity of each gluon (fails without the four-gluon diagrams),
                   Bose symmetry, boosts (tests/test_oracle_vjets.py)
  udx_wpgg, uux_zgg  u d~ > w+ g g, u u~ > z g g (V plus two jets): Ward identity for each gluon,
                   Bose symmetry, the soft limit of either gluon against the colour-correlated
                   eikonal factor of q, q~, g times q q~ > V g (closed form), boosts
  us_dchh         u s > d c h h  (WW fusion): its W W > h h core (_ww_hh, the code
                   it runs) pinned by the gauge cancellation of the longitudinal
                   on-shell W+ W- > h h amplitude (wpwm_hh_amplitudes calls the same
                   core); the whole process by the fixed-angle high-energy limit
                   (zero W width: s^2 |M|^2 tends to a constant, a wrong relative
                   sign or coupling of the four diagrams grows like s^2); its W
                   currents by u s > d c h; Higgs-exchange symmetry, boosts
  us_dchhh        u s > d c h h h (WW fusion) and
  ud_udh, ud_udhh, ud_udhhh  u d > u d + 1, 2, 3 Higgs (ZZ and WW fusion, Sect. 2.10): the V V > n H
                   core (vv_higgs) equals _ww_hh at n = 2 and follows the zero-momentum Higgs
                   theorem from n to n + 1 for W and Z; u d > u d h against its closed form (the
                   lines, couplings, colour and the exchange sign of the W channel); the W channel
                   against u s > d c h (h) with the outgoing quarks exchanged; with the complex-mass
                   card the HHH processes keep the zero-width high-energy behaviour that the
                   fixed-width card loses; Higgs permutations, boosts (tests/test_oracle_wbf.py)
  uu_uuh_n, uu_uuhh, uu_uuhhh  u u > u u + 1, 2, 3 Higgs (Z Z fusion with the outgoing quarks
                   exchanged): u u > u u h against its closed form (the chiral Fierz identity turns the
                   exchanged left-handed spinor product into minus the direct one, so the exchange sign
                   makes the two channels interfere constructively); the core as for u d > u d + Higgs;
                   Fermi symmetry of the outgoing quarks, Higgs permutations, boosts
                   (tests/test_oracle_wbf.py)
  udx_epveg       u d~ > e+ ve g : Ward identity; soft-gluon limit against C_F times
                   the eikonal factor times u d~ > e+ ve (closed form); boosts
  gluons          g g > g...g    : Berends-Giele, pinned by the gg > gg closed
                   form, Parke-Taylor MHV amplitudes, the soft-gluon limit of every
                   NMHV six-gluon partial amplitude onto the Parke-Taylor-pinned
                   five-gluon ones, Ward, Bose, boosts
"""
import itertools
import numpy as np

from . import colour
from .feynman import (ffv_current, fermion_line, fermion_prop, scalar_prop, vector_insertion,
                      vector_prop, vvv_out, den)
from .lorentz import bar, mdot, polarisation, u_spinor, v_spinor
from .sm import CHARGE, T3, SMParams

HEL_F = (-1, 1)
HEL_V = (-1, 1)

_T = colour.T
_F = colour.F
_DELTA3 = np.eye(3, dtype=complex)


def _z_couplings(f, par):
    gl = par.gz * (T3[f] - CHARGE[f] * par.sw2)
    gr = par.gz * (-CHARGE[f] * par.sw2)
    return gl, gr


def _a_coupling(f, par):
    return par.e * CHARGE[f]


# --------------------------------------------------------------------------
# q q~ > l+ l- via photon and Z  (cfg: u u~ > e+ e-)
# --------------------------------------------------------------------------
def uux_epem(P, par=SMParams(), per_helicity=False, quark="u", lepton="e"):
    p = [P[:, k] for k in range(4)]
    q = p[0] + p[1]
    tot = 0.0
    ph = {}
    for h in itertools.product(HEL_F, repeat=4):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        v = v_spinor(p[2], h[2])
        ub = bar(u_spinor(p[3], h[3]))
        iM = 0.0
        # photon
        ga_q, ga_l = _a_coupling(quark, par), _a_coupling(lepton, par)
        Jq = ffv_current(vb, u, ga_q, ga_q)
        Jl = ffv_current(ub, v, ga_l, ga_l)
        iM = iM + mdot(vector_prop(q, Jq), Jl)
        # Z
        zq, zl = _z_couplings(quark, par), _z_couplings(lepton, par)
        Jq = ffv_current(vb, u, *zq)
        Jl = ffv_current(ub, v, *zl)
        iM = iM + mdot(vector_prop(q, Jq, par.mZ, par.wZ), Jl)
        M = iM / 1j
        m2 = colour.colour_sum([M], [_DELTA3])
        ph[h] = m2
        tot = tot + m2
    avg = tot / (4.0 * 9.0)
    return (avg, ph) if per_helicity else avg


# --------------------------------------------------------------------------
# u d~ > e+ ve via W+  (closed-form pin of the W building block)
# --------------------------------------------------------------------------
def udx_epve(P, par=SMParams()):
    p = [P[:, k] for k in range(4)]
    gw = par.g / np.sqrt(2.0)
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        v = v_spinor(p[2], h[2])
        ub = bar(u_spinor(p[3], h[3]))
        L = ffv_current(ub, v, gw, 0.0)
        W = vector_prop(p[2] + p[3], L, par.mW, par.wW)
        Jq = ffv_current(vb, u, gw, 0.0)
        M = mdot(Jq, W) / 1j
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# u d~ > e+ ve g  (W+ -> e+ ve plus one gluon: the link of the soft-gluon chain
# u d~ > e+ ve  <-  u d~ > e+ ve g  <-  u d~ > e+ ve g g)
# --------------------------------------------------------------------------
def udx_epveg(P, par=SMParams(), eps_override=None):
    """Two diagrams: the gluon before or after the W along the quark line.
    eps_override: optional vector[N,4] replacing the gluon polarisation (Ward identity)."""
    p = [P[:, k] for k in range(5)]
    gs, gw = par.gs, par.g / np.sqrt(2.0)
    cg = _colour_string([0], 1)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_F, HEL_F, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        L = ffv_current(bar(u_spinor(p[3], h[3])), v_spinor(p[2], h[2]), gw, 0.0)
        qW = p[2] + p[3]
        W = (vector_insertion(vector_prop(qW, L, par.mW, par.wW), gw, 0.0), qW)
        eg = polarisation(p[4], h[4]).conj() if eps_override is None else eps_override.astype(complex)
        G = (vector_insertion(eg, gs, gs), p[4])
        amps = [fermion_line(vb, u, p[0], [W, G]) / 1j, fermion_line(vb, u, p[0], [G, W]) / 1j]
        tot = tot + colour.colour_sum(amps, [cg, cg])
    return tot / 36.0


# --------------------------------------------------------------------------
# helpers shared by the quark-line processes
# --------------------------------------------------------------------------
def _colour_string(gluon_slots, n_gluons, with_f=None):
    """Explicit colour tensor c[i_start, i_end, a_1..a_n] of one diagram.

    gluon_slots: the sequence of colour insertions along the fermion arrow,
    from the start (column spinor) to the end (row spinor); each entry is a
    gluon label k (t^{a_k}) or "G" for an internal gluon attached to the
    ggg vertex of gluons with_f = (k1, k2), giving f^{a_k1 a_k2 c} t^c.
    The result is (t_last ... t_first)_{i_end, i_start} arranged with axes
    (i_start, i_end, a_0, ..., a_{n-1}).
    """
    shape = (3, 3) + (8,) * n_gluons
    out = np.zeros(shape, dtype=complex)
    for a in itertools.product(range(8), repeat=n_gluons):
        M = np.eye(3, dtype=complex)
        for slot in gluon_slots:
            if slot == "G":
                k1, k2 = with_f
                Tg = np.einsum("c,cij->ij", _F[a[k1], a[k2], :], _T)
            else:
                Tg = _T[a[slot]]
            M = Tg @ M
        out[(slice(None), slice(None)) + a] = M.T  # [i_start, i_end]
    return out


# --------------------------------------------------------------------------
# q q~ > g g  (textbook closed-form pin of the qqg and ggg rules)
# --------------------------------------------------------------------------
def uux_gg(P, par=SMParams()):
    p = [P[:, k] for k in range(4)]
    gs = par.gs
    cAB = _colour_string([0, 1], 2)
    cBA = _colour_string([1, 0], 2)
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_V, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        e2 = polarisation(p[2], h[2]).conj()
        e3 = polarisation(p[3], h[3]).conj()
        G2 = (vector_insertion(e2, gs, gs), p[2])
        G3 = (vector_insertion(e3, gs, gs), p[3])
        A23 = fermion_line(vb, u, p[0], [G2, G3])
        A32 = fermion_line(vb, u, p[0], [G3, G2])
        X = vvv_out(e2, -p[2], e3, -p[3], p[2] + p[3], gs)
        Gint = vector_prop(p[2] + p[3], X)
        AG = fermion_line(vb, u, p[0], [(vector_insertion(Gint, gs, gs), p[2] + p[3])])
        tot = tot + colour.colour_sum([A23 / 1j, A32 / 1j, AG / 1j], [cAB, cBA, cG])
    return tot / 36.0


# --------------------------------------------------------------------------
# u d~ > e+ ve g g   (W+ -> e+ ve, two gluons on the quark line or via ggg)
# --------------------------------------------------------------------------
def udx_epvegg(P, par=SMParams(), per_helicity=False, eps_override=None):
    """Eight diagrams: the W and both gluons in all 3! orders along the quark
    line, plus the W and the ggg-produced gluon pair in both orders.

    eps_override: optional {leg: vector[N,4]} replacing a gluon polarisation
    (used by the Ward-identity pin with eps -> k).
    """
    p = [P[:, k] for k in range(6)]
    gs, gw = par.gs, par.g / np.sqrt(2.0)
    colours = {}
    for order in itertools.permutations(["W", 0, 1]):
        colours[order] = _colour_string([s for s in order if s != "W"], 2)
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    tot = 0.0
    ph = {}
    for h in itertools.product(HEL_F, HEL_F, HEL_F, HEL_F, HEL_V, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ve_ = v_spinor(p[2], h[2])
        ubn = bar(u_spinor(p[3], h[3]))
        eg = [polarisation(p[4], h[4]).conj(), polarisation(p[5], h[5]).conj()]
        if eps_override:
            for leg, vec in eps_override.items():
                eg[leg - 4] = vec.astype(complex)
        L = ffv_current(ubn, ve_, gw, 0.0)
        qW = p[2] + p[3]
        W = vector_prop(qW, L, par.mW, par.wW)
        ins = {"W": (vector_insertion(W, gw, 0.0), qW),
               0: (vector_insertion(eg[0], gs, gs), p[4]),
               1: (vector_insertion(eg[1], gs, gs), p[5])}
        amps, cols = [], []
        for order, c in colours.items():
            amps.append(fermion_line(vb, u, p[0], [ins[s] for s in order]) / 1j)
            cols.append(c)
        X = vvv_out(eg[0], -p[4], eg[1], -p[5], p[4] + p[5], gs)
        Gint = vector_prop(p[4] + p[5], X)
        insG = (vector_insertion(Gint, gs, gs), p[4] + p[5])
        for order in (["W", "G"], ["G", "W"]):
            amps.append(fermion_line(vb, u, p[0], [ins["W"] if s == "W" else insG for s in order]) / 1j)
            cols.append(cG)
        m2 = colour.colour_sum(amps, cols)
        ph[h] = m2
        tot = tot + m2
    avg = tot / 36.0
    return (avg, ph) if per_helicity else avg


# --------------------------------------------------------------------------
# g g > t t~ (on-shell tops; textbook closed-form pin of the massive line)
# --------------------------------------------------------------------------
def gg_ttx(P, par=SMParams(), widths=True):
    """g(0) g(1) > t(2) t~(3) with on-shell tops: t- and u-channel top exchange and the s-channel gluon.
    The internal top carries the width wt (as every internal massive line does) unless widths=False."""
    p = [P[:, k] for k in range(4)]
    gs, mt = par.gs, par.mt
    wt = par.wt if widths else 0.0
    cAB = _colour_string([0, 1], 2)  # arrow starts at the t~ spinor: gluon 0 nearest t~
    cBA = _colour_string([1, 0], 2)
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    tot = 0.0
    for h in itertools.product(HEL_V, HEL_V, HEL_F, HEL_F):
        e0 = polarisation(p[0], h[0])
        e1 = polarisation(p[1], h[1])
        ubt = bar(u_spinor(p[2], h[2]))
        vt = v_spinor(p[3], h[3])
        G0 = (vector_insertion(e0, gs, gs), -p[0])
        G1 = (vector_insertion(e1, gs, gs), -p[1])
        A01 = fermion_line(ubt, vt, -p[3], [G0, G1], mt, wt)
        A10 = fermion_line(ubt, vt, -p[3], [G1, G0], mt, wt)
        X = vvv_out(e0, p[0], e1, p[1], -(p[0] + p[1]), gs)
        Gint = vector_prop(p[0] + p[1], X)
        AG = fermion_line(ubt, vt, -p[3], [(vector_insertion(Gint, gs, gs), -(p[0] + p[1]))], mt, wt)
        tot = tot + colour.colour_sum([A01 / 1j, A10 / 1j, AG / 1j], [cAB, cBA, cG])
    return tot / (4.0 * 64.0)


# --------------------------------------------------------------------------
# g g > t t~ H (the Higgs from every top line of g g > t t~: eight diagrams)
# --------------------------------------------------------------------------
def gg_ttxh(P, par=SMParams(), per_helicity=False, eps_override=None, widths=True):
    """g(0) g(1) > t(2) t~(3) H(4).  The top line runs from the t~ spinor v(p3) to ubar(p2); the two
    gluons and the Higgs are inserted in every order along it (six diagrams, colour t^a t^b or t^b t^a
    by the order of the gluons), and the s-channel gluon of g g > t t~ is inserted with the Higgs before
    or after it (two diagrams, colour f^{abc} t^c).  The Higgs vertex is the FFS one of Sect. 4.2 with
    the Yukawa coupling of L = -(mt/v) t~ t H: a factor -i mt/v in i M.  Internal tops carry the width
    wt unless widths=False.  eps_override = (leg, vector) replaces that gluon's polarisation vector."""
    p = [P[:, k] for k in range(5)]
    n = P.shape[0]
    gs, mt = par.gs, par.mt
    wt = par.wt if widths else 0.0
    yt = -mt / par.vev
    cAB = _colour_string([0, 1], 2)
    cBA = _colour_string([1, 0], 2)
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    Hins = (np.broadcast_to(1j * yt * np.eye(4, dtype=complex), (n, 4, 4)), p[4])
    tot = 0.0
    ph = {}
    for h in itertools.product(HEL_V, HEL_V, HEL_F, HEL_F):
        e0 = polarisation(p[0], h[0])
        e1 = polarisation(p[1], h[1])
        if eps_override is not None:
            if eps_override[0] == 0:
                e0 = eps_override[1]
            else:
                e1 = eps_override[1]
        ubt = bar(u_spinor(p[2], h[2]))
        vt = v_spinor(p[3], h[3])
        G0 = (vector_insertion(e0, gs, gs), -p[0])
        G1 = (vector_insertion(e1, gs, gs), -p[1])
        AB, BA = 0.0, 0.0
        for order in itertools.permutations(["G0", "G1", "H"]):
            ins = [{"G0": G0, "G1": G1, "H": Hins}[x] for x in order]
            a = fermion_line(ubt, vt, -p[3], ins, mt, wt)
            if order.index("G0") < order.index("G1"):
                AB = AB + a
            else:
                BA = BA + a
        X = vvv_out(e0, p[0], e1, p[1], -(p[0] + p[1]), gs)
        Gs = (vector_insertion(vector_prop(p[0] + p[1], X), gs, gs), -(p[0] + p[1]))
        AG = fermion_line(ubt, vt, -p[3], [Gs, Hins], mt, wt) + fermion_line(ubt, vt, -p[3], [Hins, Gs], mt, wt)
        val = colour.colour_sum([AB / 1j, BA / 1j, AG / 1j], [cAB, cBA, cG])
        if per_helicity:
            ph[h] = val
        tot = tot + val
    if per_helicity:
        return ph
    return tot / (4.0 * 64.0)


# --------------------------------------------------------------------------
# g g > W+ d u~  (W plus two jets from two gluons: eight diagrams)
# --------------------------------------------------------------------------
def _gg_vqqx(P, par, gl, gr, mV, eps_override):
    """g(0) g(1) > V(2) q(3) q~'(4).  The quark line runs from v(p4) to ubar(p3): the two gluons and
    the V (coupling i gamma^mu (gl P_L + gr P_R)) in every order along it (six diagrams, colour
    t^a t^b or t^b t^a by the order of the gluons), and the s-channel gluon of the two gluons beside
    the V (two, colour f^{abc} t^c).  eps_override = (leg, vector) replaces that gluon's vector."""
    p = [P[:, k] for k in range(5)]
    gs = par.gs
    cAB = _colour_string([0, 1], 2)
    cBA = _colour_string([1, 0], 2)
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    tot = 0.0
    for h in itertools.product(HEL_V, HEL_V, HEL_W, HEL_F, HEL_F):
        e0 = polarisation(p[0], h[0])
        e1 = polarisation(p[1], h[1])
        if eps_override is not None:
            e0, e1 = (eps_override[1], e1) if eps_override[0] == 0 else (e0, eps_override[1])
        ev = polarisation(p[2], h[2], mass=mV).conj()
        ubd = bar(u_spinor(p[3], h[3]))
        vu = v_spinor(p[4], h[4])
        ins = {"G0": (vector_insertion(e0, gs, gs), -p[0]), "G1": (vector_insertion(e1, gs, gs), -p[1]),
               "W": (vector_insertion(ev, gl, gr), p[2])}
        AB, BA = 0.0, 0.0
        for order in itertools.permutations(["G0", "G1", "W"]):
            a = fermion_line(ubd, vu, -p[4], [ins[x] for x in order])
            if order.index("G0") < order.index("G1"):
                AB = AB + a
            else:
                BA = BA + a
        X = vvv_out(e0, p[0], e1, p[1], -(p[0] + p[1]), gs)
        Gs = (vector_insertion(vector_prop(p[0] + p[1], X), gs, gs), -(p[0] + p[1]))
        AG = fermion_line(ubd, vu, -p[4], [Gs, ins["W"]]) + fermion_line(ubd, vu, -p[4], [ins["W"], Gs])
        tot = tot + colour.colour_sum([AB / 1j, BA / 1j, AG / 1j], [cAB, cBA, cG])
    return tot / (4.0 * 64.0)


def gg_wpdux(P, par=SMParams(), eps_override=None):
    """g g > W+ d u~ (the quark line from the u~ to the d emits the W+)."""
    return _gg_vqqx(P, par, par.g / np.sqrt(2.0), 0.0, par.mW, eps_override)


def gg_zuux(P, par=SMParams(), eps_override=None):
    """g g > Z u u~."""
    gl, gr = _z_couplings("u", par)
    return _gg_vqqx(P, par, gl, gr, par.mZ, eps_override)


# --------------------------------------------------------------------------
# u u~ > t t~  (s-channel gluon, photon and Z)
# --------------------------------------------------------------------------
def uux_ttx(P, par=SMParams(), bosons=("g", "a", "z")):
    """u(p0) u~(p1) > t(p2) t~(p3) through an s-channel gluon, photon or Z between the light-quark
    current and the top current.  Colour: t^a_{i1 i0} t^a_{i2 i3} for the gluon, delta_{i1 i0}
    delta_{i2 i3} for the photon and the Z (axes i0 u, i1 u~, i2 t, i3 t~).  `bosons` selects the
    exchanged bosons (the pins take them one at a time)."""
    p = [P[:, k] for k in range(4)]
    d = np.eye(3, dtype=complex)
    tens = {"g": np.einsum("aji,akl->ijkl", _T, _T), "ew": np.einsum("ji,kl->ijkl", d, d)}
    q = p[0] + p[1]
    spec = {"g": ((par.gs, par.gs), (par.gs, par.gs), 0.0, 0.0, "g"),
            "a": ((_a_coupling("u", par),) * 2, (_a_coupling("t", par),) * 2, 0.0, 0.0, "ew"),
            "z": (_z_couplings("u", par), _z_couplings("t", par), par.mZ, par.wZ, "ew")}
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ubt = bar(u_spinor(p[2], h[2]))
        vt = v_spinor(p[3], h[3])
        amps, cols = [], []
        for b in bosons:
            cq, ct, m, w, c = spec[b]
            amps.append(mdot(vector_prop(q, ffv_current(vb, u, *cq), m, w), ffv_current(ubt, vt, *ct)) / 1j)
            cols.append(tens[c])
        tot = tot + colour.colour_sum(amps, cols)
    return tot / 36.0


def uux_ttxg(P, par=SMParams(), eps_override=None, widths=True):
    """u(p0) u~(p1) > t(p2) t~(p3) g(p4): the s-channel gluon, photon or Z of u u~ > t t~ with the
    gluon emitted from the light-quark line (two places) or from the top line (two places), and the
    s-channel gluon's three-gluon vertex with the emitted gluon (13 diagrams).  Colour tensors over
    (i0 u, i1 u~, i2 t, i3 t~, a): along the light line the product of generators runs from u to u~,
    along the top line from t~ to t.  Internal tops carry the width wt unless widths=False."""
    p = [P[:, k] for k in range(5)]
    gs, mt = par.gs, par.mt
    wt = par.wt if widths else 0.0
    T, F = _T, _F
    d = np.eye(3, dtype=complex)
    cpl = {"g": ((gs, gs), (gs, gs), 0.0, 0.0), "a": ((_a_coupling("u", par),) * 2, (_a_coupling("t", par),) * 2, 0.0, 0.0),
           "z": (_z_couplings("u", par), _z_couplings("t", par), par.mZ, par.wZ)}
    # colour tensors
    c_light = {"GV": np.einsum("cjk,aki,clm->ijlma", T, T, T),    # (t^c t^a)_{i1 i0} t^c_{i2 i3}
               "VG": np.einsum("ajk,cki,clm->ijlma", T, T, T)}    # (t^a t^c)_{i1 i0} t^c_{i2 i3}
    c_top = {"GV": np.einsum("cji,clk,akm->ijlma", T, T, T),      # t^c_{i1 i0} (t^c t^a)_{i2 i3}
             "VG": np.einsum("cji,alk,ckm->ijlma", T, T, T)}      # t^c_{i1 i0} (t^a t^c)_{i2 i3}
    c_ew_light = np.einsum("aji,lm->ijlma", T, d)                 # t^a_{i1 i0} delta_{i2 i3}
    c_ew_top = np.einsum("ji,alm->ijlma", d, T)                   # delta_{i1 i0} t^a_{i2 i3}
    c_ggg = np.einsum("cji,cae,elm->ijlma", T, F, T)              # t^c_{i1 i0} f^{c a e} t^e_{i2 i3}
    q = p[0] + p[1]
    Q = p[2] + p[3]
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_F, HEL_F, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ubt = bar(u_spinor(p[2], h[2]))
        vt = v_spinor(p[3], h[3])
        eg = polarisation(p[4], h[4]).conj() if eps_override is None else eps_override
        amps, cols = [], []
        for b in ("g", "a", "z"):
            cu, ct, m, w = cpl[b]
            # gluon from the light line: the boson carries Q into the top current
            Yt = vector_prop(Q, ffv_current(ubt, vt, *ct), m, w)
            Vu = (vector_insertion(Yt, *cu), Q)
            Gu = (vector_insertion(eg, gs, gs), p[4])
            a_gv = fermion_line(vb, u, p[0], [Gu, Vu]) / 1j
            a_vg = fermion_line(vb, u, p[0], [Vu, Gu]) / 1j
            # gluon from the top line: the boson carries q out of the light current into the top line
            Yu = vector_prop(q, ffv_current(vb, u, *cu), m, w)
            Vt = (vector_insertion(Yu, *ct), -q)
            a_tgv = fermion_line(ubt, vt, -p[3], [Gu, Vt], mt, wt) / 1j
            a_tvg = fermion_line(ubt, vt, -p[3], [Vt, Gu], mt, wt) / 1j
            if b == "g":
                amps += [a_gv, a_vg, a_tgv, a_tvg]
                cols += [c_light["GV"], c_light["VG"], c_top["GV"], c_top["VG"]]
            else:
                amps += [a_gv + a_vg, a_tgv + a_tvg]
                cols += [c_ew_light, c_ew_top]
        # the s-channel gluon emits the gluon through the three-gluon vertex
        Ju = vector_prop(q, ffv_current(vb, u, gs, gs))
        X = vvv_out(Ju, q, eg, -p[4], -Q, gs)
        amps.append(fermion_line(ubt, vt, -p[3], [(vector_insertion(vector_prop(Q, X), gs, gs), -Q)], mt, wt) / 1j)
        cols.append(c_ggg)
        tot = tot + colour.colour_sum(amps, cols)
    return tot / 36.0


# --------------------------------------------------------------------------
# g g > t t~ g  (top pair plus one jet: sixteen diagrams)
# --------------------------------------------------------------------------
def _vvvv_out(J1, J2, J3):
    """Lorentz parts of the four-gluon vertex with legs (1, 2, 3) contracted and the fourth open, for
    its three colour structures f^{12e} f^{3Xe}, f^{13e} f^{2Xe}, f^{1Xe} f^{23e} (Sect. 4.2 VVVV,
    the textbook rule -i gs^2 [f^{abe} f^{cde} (g^{ac} g^{bd} - g^{ad} g^{bc}) + two permutations])."""
    d12, d13, d23 = mdot(J1, J2)[..., None], mdot(J1, J3)[..., None], mdot(J2, J3)[..., None]
    return (d13 * J2 - d23 * J1, d12 * J3 - d23 * J1, d12 * J3 - d13 * J2)


def gg_ttxg(P, par=SMParams(), eps_override=None, widths=True):
    """g(0) g(1) > t(2) t~(3) g(4).  The top line runs from v(p3) to ubar(p2); the diagrams are
      - the three gluons attached to the line in each of the six orders (colour t t t),
      - two gluons joined by a three-gluon vertex into one line attached beside the third gluon, for
        the three pairs and both orders along the line (six; colour f t t),
      - the three gluons joined into one line through two three-gluon vertices (three) or the
        four-gluon vertex (one, three colour structures), attached to the top line (colour f f t).
    Colour is summed over explicit indices; internal tops carry the width wt unless widths=False.
    eps_override = (leg, vector) replaces that gluon's polarisation vector."""
    p = [P[:, k] for k in range(5)]
    gs, mt = par.gs, par.mt
    wt = par.wt if widths else 0.0
    T, F = _T, _F
    # gluon momenta flowing into the gluon vertices; k4 is the outgoing gluon's, reversed
    kg = {0: p[0], 1: p[1], 4: -p[4]}
    legs = (0, 1, 4)

    def ctensor(spec):
        """Colour tensor [i_start, i_end, a0, a1, a4] of a colour factor given as an einsum over t and f."""
        out = np.zeros((3, 3, 8, 8, 8), dtype=complex)
        for a in itertools.product(range(8), repeat=3):
            A = dict(zip(legs, a))
            out[(slice(None), slice(None)) + a] = spec(A).T
        return out

    tensors, amp_specs = [], []
    # six orders of direct attachment (first in the list = nearest the t~)
    for order in itertools.permutations(legs):
        tensors.append(ctensor(lambda A, o=order: T[A[o[2]]] @ T[A[o[1]]] @ T[A[o[0]]]))
        amp_specs.append(("direct", order))
    # a pair (x, y) merged by f^{a_x a_y c} into one gluon c, attached with the third gluon z
    for x, y in ((0, 1), (0, 4), (1, 4)):
        z = [l for l in legs if l not in (x, y)][0]
        fxy = lambda A, x=x, y=y: np.einsum("c,cij->ij", F[A[x], A[y], :], T)
        tensors.append(ctensor(lambda A, f=fxy, z=z: T[A[z]] @ f(A)))
        amp_specs.append(("pair_first", (x, y, z)))
        tensors.append(ctensor(lambda A, f=fxy, z=z: f(A) @ T[A[z]]))
        amp_specs.append(("pair_last", (x, y, z)))
    # all three merged: (x y) then z through two three-gluon vertices, f^{xye} f^{ezg} t^g
    for x, y in ((0, 1), (0, 4), (1, 4)):
        z = [l for l in legs if l not in (x, y)][0]
        tensors.append(ctensor(lambda A, x=x, y=y, z=z:
                               np.einsum("e,eg,gij->ij", F[A[x], A[y], :], F[:, A[z], :], T)))
        amp_specs.append(("triple", (x, y, z)))
    # four-gluon vertex, legs (0, 1, 4, X): f^{01e} f^{4Xe}, f^{04e} f^{1Xe}, f^{0Xe} f^{14e}
    tensors.append(ctensor(lambda A: np.einsum("e,ge,gij->ij", F[A[0], A[1], :], F[A[4], :, :], T)))
    amp_specs.append(("quartic", 0))
    tensors.append(ctensor(lambda A: np.einsum("e,ge,gij->ij", F[A[0], A[4], :], F[A[1], :, :], T)))
    amp_specs.append(("quartic", 1))
    tensors.append(ctensor(lambda A: np.einsum("ge,e,gij->ij", F[A[0], :, :], F[A[1], A[4], :], T)))
    amp_specs.append(("quartic", 2))

    tot = 0.0
    for h in itertools.product(HEL_V, HEL_V, HEL_F, HEL_F, HEL_V):
        eps = {0: polarisation(p[0], h[0]), 1: polarisation(p[1], h[1]), 4: polarisation(p[4], h[4]).conj()}
        if eps_override is not None:
            eps[eps_override[0]] = eps_override[1]
        ubt = bar(u_spinor(p[2], h[2]))
        vt = v_spinor(p[3], h[3])

        def ins(J, kin):
            """A gluon line carrying momentum kin into the top line."""
            return (vector_insertion(J, gs, gs), -kin)

        def merge(x, y):
            """Propagated gluon line of gluons x and y through f^{a_x a_y c}; momentum into the line."""
            k = kg[x] + kg[y]
            return vector_prop(k, vvv_out(eps[x], kg[x], eps[y], kg[y], -k, gs)), k

        amps = []
        for kind, spec in amp_specs:
            if kind == "direct":
                a = fermion_line(ubt, vt, -p[3], [ins(eps[l], kg[l]) for l in spec], mt, wt)
            elif kind in ("pair_first", "pair_last"):
                x, y, z = spec
                J, k = merge(x, y)
                seq = [ins(J, k), ins(eps[z], kg[z])] if kind == "pair_first" else [ins(eps[z], kg[z]), ins(J, k)]
                a = fermion_line(ubt, vt, -p[3], seq, mt, wt)
            elif kind == "triple":
                x, y, z = spec
                J, k = merge(x, y)
                K = k + kg[z]
                G = vector_prop(K, vvv_out(J, k, eps[z], kg[z], -K, gs))
                a = fermion_line(ubt, vt, -p[3], [ins(G, K)], mt, wt)
            else:
                K = kg[0] + kg[1] + kg[4]
                G = vector_prop(K, -1j * gs * gs * _vvvv_out(eps[0], eps[1], eps[4])[spec])
                a = fermion_line(ubt, vt, -p[3], [ins(G, K)], mt, wt)
            amps.append(a / 1j)
        tot = tot + colour.colour_sum(amps, tensors)
    return tot / (4.0 * 64.0)


# --------------------------------------------------------------------------
# g g > t t~ > (b e+ ve) (b~ e- ve~): the three doubly-resonant diagrams
# --------------------------------------------------------------------------
def gg_ttx_dilep(P, par=SMParams(), per_helicity=False, eps_override=None, all_attachments=False):
    """Legs: g(0) g(1) b(2) e+(3) ve(4) b~(5) e-(6) ve~(7).

    The fermion line runs from the outgoing b~ (v spinor) to the outgoing b
    (u-bar spinor): W- emission, top propagator, the gluon insertions (two
    orders, or the ggg-produced gluon), top propagator, W+ emission.  These
    are the three doubly-resonant diagrams.  Fixed widths in every top and W
    propagator.

    all_attachments=True adds the diagrams with a gluon on the b or b~
    segment of the line (15 in total).  That set, unlike the resonant
    subset, is QCD gauge invariant at zero widths, which the Ward-identity
    pin uses.
    """
    p = [P[:, k] for k in range(8)]
    gs, gw, mt, wt = par.gs, par.g / np.sqrt(2.0), par.mt, par.wt
    tot = 0.0
    ph = {}
    # insertion sequences along the arrow; the segment before "Wm" and after "Wp" is a b quark
    if all_attachments:
        seqs = []
        for pos in itertools.permutations(range(4), 2):
            seq = ["Wm", "Wp"]
            rest = [x for x in range(4) if x not in pos]
            full = [None] * 4
            full[pos[0]], full[pos[1]] = 0, 1
            full[rest[0]], full[rest[1]] = "Wm", "Wp"
            seqs.append(full)
        for slot in range(3):
            seq = ["Wm", "Wp"]
            seq.insert(slot, "G")
            seqs.append(seq)
    else:
        seqs = [["Wm", 0, 1, "Wp"], ["Wm", 1, 0, "Wp"], ["Wm", "G", "Wp"]]
    cols = []
    for seq in seqs:
        glu = [x for x in seq if x not in ("Wm", "Wp")]
        cols.append(_colour_string(glu, 2, with_f=(0, 1)) if "G" in glu else _colour_string(glu, 2))
    for h in itertools.product(HEL_V, HEL_V, *([HEL_F] * 6)):
        e = [polarisation(p[0], h[0]), polarisation(p[1], h[1])]
        if eps_override:
            for leg, vec in eps_override.items():
                e[leg] = vec.astype(complex)
        ub_b = bar(u_spinor(p[2], h[2]))
        v_ep = v_spinor(p[3], h[3])
        ub_nu = bar(u_spinor(p[4], h[4]))
        v_bb = v_spinor(p[5], h[5])
        ub_em = bar(u_spinor(p[6], h[6]))
        v_nub = v_spinor(p[7], h[7])
        Wp = vector_prop(p[3] + p[4], ffv_current(ub_nu, v_ep, gw, 0.0), par.mW, par.wW)
        Wm = vector_prop(p[6] + p[7], ffv_current(ub_em, v_nub, gw, 0.0), par.mW, par.wW)
        X = vvv_out(e[0], p[0], e[1], p[1], -(p[0] + p[1]), gs)
        Gint = vector_prop(p[0] + p[1], X)
        ins = {"Wm": (vector_insertion(Wm, gw, 0.0), p[6] + p[7]),
               "Wp": (vector_insertion(Wp, gw, 0.0), p[3] + p[4]),
               0: (vector_insertion(e[0], gs, gs), -p[0]),
               1: (vector_insertion(e[1], gs, gs), -p[1]),
               "G": (vector_insertion(Gint, gs, gs), -(p[0] + p[1]))}
        amps = []
        for seq in seqs:
            amps.append(_line_with_flavours(ub_b, v_bb, -p[5], [ins[x] for x in seq], seq, mt, wt) / 1j)
        m2 = colour.colour_sum(amps, cols)
        ph[h] = m2
        tot = tot + m2
    avg = tot / (4.0 * 64.0)
    return (avg, ph) if per_helicity else avg


def _line_with_flavours(row, col, p_start, inserts, seq, mt, wt):
    """Fermion line whose propagators are massless b quarks outside the
    W- ... W+ stretch and tops (mass mt, width wt) inside it."""
    vec = col
    q = p_start.copy()
    inside = False
    for k, ((G, Q), tag) in enumerate(zip(inserts, seq)):
        vec = np.einsum("nij,nj->ni", G, vec)
        q = q - Q
        if tag == "Wm":
            inside = True
        elif tag == "Wp":
            inside = False
        if k < len(inserts) - 1:
            S = fermion_prop(q, mt, wt) if inside else fermion_prop(q)
            vec = np.einsum("nij,nj->ni", S, vec)
    return np.einsum("ni,ni->n", row, vec)


# --------------------------------------------------------------------------
# u s > d c h h  (W+ W- fusion into a Higgs pair)
# --------------------------------------------------------------------------
def _ww_hh(W1, q1, W2, q2, pA, pB, par):
    """The four W+ W- > h h diagrams as i M pieces (contact WWHH, s-channel H through HHH, and W
    exchange with the Higgs bosons pA or pB leaving the W1 end), for vector wavefunctions W1 (a W+
    flowing in with momentum q1) and W2 (a W- flowing in with momentum q2), off shell or on shell.
    H wavefunctions are 1; couplings g mW (WWH), g^2/2 (WWHH) and -3 mH^2/v (HHH)."""
    g, mW, wW, mH, wH, v = par.g, par.mW, par.wW, par.mH, par.wH, par.vev
    gwwh, gwwhh, ghhh = par.gwwh, g * g / 2.0, -3.0 * mH * mH / v
    w12 = mdot(W1, W2)
    out = [1j * gwwhh * w12, (1j * gwwh * w12) * scalar_prop(q1 + q2, mH, wH) * (1j * ghhh)]
    for ph in (pA, pB):
        Wst = vector_prop(q1 - ph, 1j * gwwh * W1, mW, wW)
        out.append(1j * gwwh * mdot(Wst, W2))
    return out


def us_dchh(P, par=SMParams(), per_helicity=False):
    """Four diagrams: the two quark currents, each into its t-channel W propagator, feed the
    W+ W- > h h core (_ww_hh): WWHH contact, s-channel H with HHH, and t/u-channel W exchange
    with two WWH vertices."""
    p = [P[:, k] for k in range(6)]
    gw = par.g / np.sqrt(2.0)
    q1 = p[0] - p[2]
    q2 = p[1] - p[3]
    tot = 0.0
    ph = {}
    for h in itertools.product(HEL_F, repeat=4):
        J1 = ffv_current(bar(u_spinor(p[2], h[2])), u_spinor(p[0], h[0]), gw, 0.0)
        J2 = ffv_current(bar(u_spinor(p[3], h[3])), u_spinor(p[1], h[1]), gw, 0.0)
        W1 = vector_prop(q1, J1, par.mW, par.wW)
        W2 = vector_prop(q2, J2, par.mW, par.wW)
        M = sum(_ww_hh(W1, q1, W2, q2, p[4], p[5], par)) / 1j
        m2 = 9.0 * np.abs(M) ** 2
        ph[h + (0, 0)] = m2
        tot = tot + m2
    avg = tot / 36.0
    return (avg, ph) if per_helicity else avg


def us_dch(P, par=SMParams()):
    """u(p0) s(p1) > d(p2) c(p3) H(p4) by W+ W- fusion: the two quark currents, each into its t-channel
    W propagator, meet at the WWH vertex (one diagram; no Z fusion for these flavours)."""
    p = [P[:, k] for k in range(5)]
    gw = par.g / np.sqrt(2.0)
    gwwh = par.gwwh
    q1 = p[0] - p[2]
    q2 = p[1] - p[3]
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        J1 = ffv_current(bar(u_spinor(p[2], h[2])), u_spinor(p[0], h[0]), gw, 0.0)
        J2 = ffv_current(bar(u_spinor(p[3], h[3])), u_spinor(p[1], h[1]), gw, 0.0)
        M = (1j * gwwh * mdot(vector_prop(q1, J1, par.mW, par.wW), vector_prop(q2, J2, par.mW, par.wW))) / 1j
        tot = tot + 9.0 * np.abs(M) ** 2
    return tot / 36.0


def us_dchg(P, par=SMParams(), eps_override=None):
    """u(p0) s(p1) > d(p2) c(p3) H(p4) g(p5) by W+ W- fusion plus one jet: the gluon from either quark
    line, before or after that line's W vertex (four diagrams).  The W seen by the gluon's line is the
    other line's propagated current through the WWH vertex and a W propagator carrying the momentum the
    line gives away.  Colour: each line keeps its own, (t^a)_{d u} delta_{c s} or delta_{d u}
    (t^a)_{c s}.  eps_override replaces the gluon's polarisation vector."""
    p = [P[:, k] for k in range(6)]
    gw = par.g / np.sqrt(2.0)
    gwwh = par.gwwh
    d3 = np.eye(3, dtype=complex)
    c1 = np.einsum("adu,cs->udsca", _T, d3)
    c2 = np.einsum("du,acs->udsca", d3, _T)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_F, HEL_F, HEL_V):
        ub_d, u_u = bar(u_spinor(p[2], h[2])), u_spinor(p[0], h[0])
        ub_c, u_s = bar(u_spinor(p[3], h[3])), u_spinor(p[1], h[1])
        eg = polarisation(p[5], h[4]).conj() if eps_override is None else eps_override.astype(complex)
        G = (vector_insertion(eg, par.gs, par.gs), p[5])
        amps = []
        for (row, col, pin, pout), (orow, ocol, opin, opout) in (((ub_d, u_u, p[0], p[2]), (ub_c, u_s, p[1], p[3])),
                                                                   ((ub_c, u_s, p[1], p[3]), (ub_d, u_u, p[0], p[2]))):
            qo = opin - opout
            Wo = vector_prop(qo, ffv_current(orow, ocol, gw, 0.0), par.mW, par.wW)
            q = pin - pout - p[5]
            V = vector_prop(q, 1j * gwwh * Wo, par.mW, par.wW)
            W = (vector_insertion(V, gw, 0.0), q)
            amps.append((fermion_line(row, col, pin, [G, W]) + fermion_line(row, col, pin, [W, G])) / 1j)
        tot = tot + colour.colour_sum(amps, [c1, c2])
    return tot / 36.0


# --------------------------------------------------------------------------
# V V > n Higgs bosons (V = W or Z, off shell or on shell), any n: the weak-boson-fusion
# core of u s > d c h h h and u d > u d h (h (h))
# --------------------------------------------------------------------------
def _splits(S, k):
    """The partitions of the frozenset S into exactly k nonempty unordered blocks."""
    items = sorted(S)
    out = []

    def rec(i, blocks):
        if i == len(items):
            if len(blocks) == k:
                out.append([frozenset(b) for b in blocks])
            return
        for b in blocks:
            b.append(items[i])
            rec(i + 1, blocks)
            b.pop()
        if len(blocks) < k:
            blocks.append([items[i]])
            rec(i + 1, blocks)
            blocks.pop()

    rec(0, [])
    return out


def _subsets(S):
    items = sorted(S)
    return [frozenset(c) for r in range(1, len(items) + 1) for c in itertools.combinations(items, r)]


def wbf_couplings(par, boson):
    """Couplings and masses of the V V > Higgs core for V = "w" or "z" (the card's scheme: real, or
    complex with its cms flag): V V H (g mu_W or g_Z mu_Z), V V H H (g^2/2 or g_Z^2/2), H H H
    (-3 mH^2/v), H H H H (-3 mH^2/v^2)."""
    v = par.vev
    c = dict(mH=par.mH, wH=par.wH, ghhh=-3.0 * par.mH ** 2 / v, ghhhh=-3.0 * par.mH ** 2 / v ** 2)
    if boson == "w":
        c.update(mV=par.mW, wV=par.wW, gvvh=par.gwwh, gvvhh=par.g ** 2 / 2.0)
    else:
        c.update(mV=par.mZ, wV=par.wZ, gvvh=par.gzzh, gvvhh=par.gz ** 2 / 2.0)
    return c


def vv_higgs(V1, q1, V2, q2, pH, cp):
    """i M of V(q1) V(q2) > H(pH[0]) ... H(pH[n-1]) for vector wavefunctions V1, V2 (upper index) that
    flow in with momenta q1, q2; the Higgs legs are amputated (wavefunction 1).

    Every tree diagram is a V line from V1 to V2 that gives off its Higgs bosons in an ordered
    sequence of emissions, each either one Higgs line at a V V H vertex or two at a V V H H vertex,
    with a V propagator between consecutive emissions.  A Higgs line that ends in the external bosons
    of a set S is the off-shell current phi(S): 1 for one boson, else the sum over the splits of S
    into two (H H H vertex) or three (H H H H vertex) parts of the product of their currents, times
    the Higgs propagator of S's summed momentum.  cp: couplings and masses (wbf_couplings)."""
    n = len(pH)
    phi_cache = {}

    def psum(S):
        return sum(pH[k] for k in sorted(S))

    def phi(S):
        if len(S) == 1:
            return 1.0
        if S not in phi_cache:
            tot = 0.0
            for blocks in _splits(S, 2):
                tot = tot + (1j * cp["ghhh"]) * phi(blocks[0]) * phi(blocks[1])
            for blocks in _splits(S, 3):
                tot = tot + (1j * cp["ghhhh"]) * phi(blocks[0]) * phi(blocks[1]) * phi(blocks[2])
            phi_cache[S] = tot * scalar_prop(psum(S), cp["mH"], cp["wH"])
        return phi_cache[S]

    def emissions(R):
        for B in _subsets(R):
            yield 1j * cp["gvvh"] * phi(B), B
        for B1 in _subsets(R):
            for B2 in _subsets(R - B1):
                if min(B1) < min(B2):  # unordered pair of disjoint blocks
                    yield 1j * cp["gvvhh"] * phi(B1) * phi(B2), B1 | B2

    def chain(X, q, R):
        tot = 0.0
        for f, used in emissions(R):
            rest = R - used
            if not rest:
                tot = tot + f * mdot(X, V2)
            else:
                qn = q - psum(used)
                tot = tot + chain(vector_prop(qn, np.asarray(f)[..., None] * X, cp["mV"], cp["wV"]), qn, rest)
        return tot

    return chain(V1, q1, frozenset(range(n)))


def us_dchhh(P, par=SMParams()):
    """u(p0) s(p1) > d(p2) c(p3) H(p4) H(p5) H(p6) by W+ W- fusion: the two quark currents, each into its
    t-channel W propagator, feed the W W > h h h core (vv_higgs, 25 diagrams).  Colour: each line keeps
    its own (a factor 9 in the colour sum)."""
    p = [P[:, k] for k in range(P.shape[1])]
    gw = par.g / np.sqrt(2.0)
    cp = wbf_couplings(par, "w")
    q1, q2 = p[0] - p[2], p[1] - p[3]
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        W1 = vector_prop(q1, ffv_current(bar(u_spinor(p[2], h[2])), u_spinor(p[0], h[0]), gw, 0.0), par.mW, par.wW)
        W2 = vector_prop(q2, ffv_current(bar(u_spinor(p[3], h[3])), u_spinor(p[1], h[1]), gw, 0.0), par.mW, par.wW)
        M = vv_higgs(W1, q1, W2, q2, p[4:], cp) / 1j
        tot = tot + 9.0 * np.abs(M) ** 2
    return tot / 36.0


def ud_udh_n(P, par=SMParams(), bosons=("w", "z")):
    """u(p0) d(p1) > u(p2) d(p3) + n Higgs bosons (p4...) by weak-boson fusion, the paper's Sect. 2.10
    processes for n = 2, 3: Z Z fusion, u > u and d > d each giving off a Z (colour delta_{i2 i0}
    delta_{i3 i1}), and W+ W- fusion, u > d giving off a W+ and d > u a W- (colour delta_{i3 i0}
    delta_{i2 i1}); exchanging the two outgoing quarks between the lines gives the W diagrams their
    relative minus sign.  Each pair of currents, through its t-channel propagators, feeds the V V > n H
    core (vv_higgs).  `bosons` selects the fusion channels (the pins take them one at a time)."""
    p = [P[:, k] for k in range(P.shape[1])]
    gw = par.g / np.sqrt(2.0)
    zu, zd = _z_couplings("u", par), _z_couplings("d", par)
    cz, cw = wbf_couplings(par, "z"), wbf_couplings(par, "w")
    d = _DELTA3
    tens = {"z": np.einsum("ca,db->abcd", d, d), "w": np.einsum("da,cb->abcd", d, d)}
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        u0, u1 = u_spinor(p[0], h[0]), u_spinor(p[1], h[1])
        ub2, ub3 = bar(u_spinor(p[2], h[2])), bar(u_spinor(p[3], h[3]))
        amps, tt = [], []
        if "z" in bosons:
            q1, q2 = p[0] - p[2], p[1] - p[3]
            Z1 = vector_prop(q1, ffv_current(ub2, u0, *zu), par.mZ, par.wZ)
            Z2 = vector_prop(q2, ffv_current(ub3, u1, *zd), par.mZ, par.wZ)
            amps.append(vv_higgs(Z1, q1, Z2, q2, p[4:], cz) / 1j)
            tt.append(tens["z"])
        if "w" in bosons:
            q1, q2 = p[0] - p[3], p[1] - p[2]
            W1 = vector_prop(q1, ffv_current(ub3, u0, gw, 0.0), par.mW, par.wW)
            W2 = vector_prop(q2, ffv_current(ub2, u1, gw, 0.0), par.mW, par.wW)
            amps.append(-vv_higgs(W1, q1, W2, q2, p[4:], cw) / 1j)
            tt.append(tens["w"])
        tot = tot + colour.colour_sum(amps, tt)
    return tot / 36.0


def uu_uuh_n(P, par=SMParams()):
    """u(p0) u(p1) > u(p2) u(p3) + n Higgs bosons (p4...) by Z Z fusion, the paper's Sect. 2.10 u u > H H (H)
    u u family: the lines u0 > u2, u1 > u3 (colour delta_{i2 i0} delta_{i3 i1}) and, with the identical
    outgoing quarks exchanged and a relative minus sign, u0 > u3, u1 > u2 (delta_{i3 i0} delta_{i2 i1});
    each pair of Z currents, through its t-channel propagators, feeds the Z Z > n H core (vv_higgs).
    No W fusion: u > d W+ on both lines would leave d d."""
    p = [P[:, k] for k in range(P.shape[1])]
    zu = _z_couplings("u", par)
    cz = wbf_couplings(par, "z")
    d = _DELTA3
    tens = [np.einsum("ca,db->abcd", d, d), np.einsum("da,cb->abcd", d, d)]
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        u0, u1 = u_spinor(p[0], h[0]), u_spinor(p[1], h[1])
        ub2, ub3 = bar(u_spinor(p[2], h[2])), bar(u_spinor(p[3], h[3]))
        amps = []
        for sign, (ra, rb) in ((1.0, (ub2, ub3)), (-1.0, (ub3, ub2))):
            pa, pb = (p[2], p[3]) if sign > 0 else (p[3], p[2])
            q1, q2 = p[0] - pa, p[1] - pb
            Z1 = vector_prop(q1, ffv_current(ra, u0, *zu), par.mZ, par.wZ)
            Z2 = vector_prop(q2, ffv_current(rb, u1, *zu), par.mZ, par.wZ)
            amps.append(sign * vv_higgs(Z1, q1, Z2, q2, p[4:], cz) / 1j)
        tot = tot + colour.colour_sum(amps, tens)
    return tot / 36.0


def uu_uuhh(P, par=SMParams()):
    return uu_uuh_n(P, par)


def uu_uuhhh(P, par=SMParams()):
    return uu_uuh_n(P, par)


def ud_udh(P, par=SMParams()):
    return ud_udh_n(P, par)


def ud_udhh(P, par=SMParams()):
    return ud_udh_n(P, par)


def ud_udhhh(P, par=SMParams()):
    return ud_udh_n(P, par)


# --------------------------------------------------------------------------
# W+ W- > h h with on-shell external W bosons (gauge-cancellation pin of the
# WWH / WWHH / HHH couplings used by u s > d c h h)
# --------------------------------------------------------------------------
def wpwm_hh_amplitudes(P, hel, par=SMParams()):
    """The four diagrams of W+(p0) W-(p1) > h(p2) h(p3) for fixed W helicities,
    returned separately (contact, s-channel H, t- and u-channel W) as M values:
    the core of u s > d c h h (_ww_hh) fed with on-shell polarisation vectors."""
    p = [P[:, k] for k in range(4)]
    e0 = polarisation(p[0], hel[0], mass=par.mW)
    e1 = polarisation(p[1], hel[1], mass=par.mW)
    return [x / 1j for x in _ww_hh(e0, p[0], e1, p[1], p[2], p[3], par)]


# --------------------------------------------------------------------------
# u u > u u  (identical quarks: t- and u-channel gluon exchange with a relative minus sign)
# --------------------------------------------------------------------------
def uu_uu(P, par=SMParams(), bosons=("g", "a", "z")):
    """Gauge-boson exchange between the two quark lines, u(p0) > u(p2) with u(p1) > u(p3) (t channel)
    and u(p0) > u(p3) with u(p1) > u(p2) (u channel), for the gluon, the photon and the Z (the
    diagrams of the Standard Model at tree level); exchanging the two identical outgoing quarks gives
    the u-channel diagrams their relative minus sign.  Colour: t^a_{i2 i0} t^a_{i3 i1} and
    t^a_{i3 i0} t^a_{i2 i1} for the gluon, the deltas of the same lines for the photon and the Z.
    `bosons` selects the exchanged bosons (the pins take them one at a time)."""
    p = [P[:, k] for k in range(4)]
    d = np.eye(3, dtype=complex)
    col = {"g": (np.einsum("aji,alk->ikjl", _T, _T), np.einsum("adi,ack->ikcd", _T, _T)),
           "ew": (np.einsum("ji,lk->ikjl", d, d), np.einsum("di,ck->ikcd", d, d))}
    ga = _a_coupling("u", par)
    cpl = {"g": ((par.gs, par.gs), 0.0, 0.0, "g"), "a": ((ga, ga), 0.0, 0.0, "ew"),
           "z": (_z_couplings("u", par), par.mZ, par.wZ, "ew")}
    tot = 0.0
    for h in itertools.product(HEL_F, repeat=4):
        u0, u1 = u_spinor(p[0], h[0]), u_spinor(p[1], h[1])
        ub2, ub3 = bar(u_spinor(p[2], h[2])), bar(u_spinor(p[3], h[3]))
        amps, tens = [], []
        for b in bosons:
            (gl, gr), m, w, c = cpl[b]
            Mt = mdot(vector_prop(p[0] - p[2], ffv_current(ub2, u0, gl, gr), m, w), ffv_current(ub3, u1, gl, gr)) / 1j
            Mu = mdot(vector_prop(p[0] - p[3], ffv_current(ub3, u0, gl, gr), m, w), ffv_current(ub2, u1, gl, gr)) / 1j
            amps += [Mt, -Mu]
            tens += list(col[c])
        tot = tot + colour.colour_sum(amps, tens)
    return tot / 36.0


# --------------------------------------------------------------------------
# u u~ > Z Z  (t- and u-channel u exchange; no triple-gauge vertex)
# --------------------------------------------------------------------------
def uux_zz(P, par=SMParams()):
    """The two diagrams of u(p0) u~(p1) > Z(p2) Z(p3): both orders of the two Z emissions along the
    quark line."""
    p = [P[:, k] for k in range(4)]
    zl, zr = _z_couplings("u", par)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        e2 = polarisation(p[2], h[2], mass=par.mZ).conj()
        e3 = polarisation(p[3], h[3], mass=par.mZ).conj()
        G2 = (vector_insertion(e2, zl, zr), p[2])
        G3 = (vector_insertion(e3, zl, zr), p[3])
        M = (fermion_line(vb, u, p[0], [G2, G3]) + fermion_line(vb, u, p[0], [G3, G2])) / 1j
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# u u~ > Z Z g  (Z pair plus one jet: the gluon and the two Z in every order along the quark line)
# --------------------------------------------------------------------------
def uux_zzg(P, par=SMParams(), eps_override=None):
    """u(p0) u~(p1) > Z(p2) Z(p3) g(p4): the six orderings of the gluon and the two Z emissions along
    the quark line, colour t^a.  eps_override replaces the gluon's polarisation vector."""
    p = [P[:, k] for k in range(5)]
    zl, zr = _z_couplings("u", par)
    cT = _colour_string([0], 1)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        e2 = polarisation(p[2], h[2], mass=par.mZ).conj()
        e3 = polarisation(p[3], h[3], mass=par.mZ).conj()
        eg = polarisation(p[4], h[4]).conj() if eps_override is None else eps_override
        ins = {"Z2": (vector_insertion(e2, zl, zr), p[2]), "Z3": (vector_insertion(e3, zl, zr), p[3]),
               "G": (vector_insertion(eg, par.gs, par.gs), p[4])}
        A = sum(fermion_line(vb, u, p[0], [ins[x] for x in order])
                for order in itertools.permutations(["Z2", "Z3", "G"]))
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 36.0


# --------------------------------------------------------------------------
# vector-boson pairs and HV plus one jet: the gluon at every place along the quark line
# --------------------------------------------------------------------------
def _with_gluon(lines, eg, kg, gs):
    """Sum over the places of one gluon emission (vector eg, outgoing momentum kg) along each quark
    line of `lines`: (row, col, p_start, inserts) with the insertions of the process without the
    gluon; the gluon goes before, between or after them."""
    G = (vector_insertion(eg, gs, gs), kg)
    tot = 0.0
    for row, col, p0, ins in lines:
        for k in range(len(ins) + 1):
            tot = tot + fermion_line(row, col, p0, ins[:k] + [G] + ins[k:])
    return tot


def uux_zhg(P, par=SMParams(), eps_override=None):
    """u(p0) u~(p1) > Z(p2) H(p3) g(p4): the s-channel Z of u u~ > Z H (ZZH vertex) with the gluon
    from the quark line before or after it (two diagrams, colour t^a)."""
    p = [P[:, k] for k in range(5)]
    zl, zr = _z_couplings("u", par)
    gzzh = par.gzzh
    cT = _colour_string([0], 1)
    Q = p[2] + p[3]
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ez = polarisation(p[2], h[2], mass=par.mZ).conj()
        eg = polarisation(p[4], h[3]).conj() if eps_override is None else eps_override
        Y = vector_prop(Q, 1j * gzzh * ez, par.mZ, par.wZ)
        A = _with_gluon([(vb, u, p[0], [(vector_insertion(Y, zl, zr), Q)])], eg, p[4], par.gs)
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 36.0


def udx_wphg(P, par=SMParams(), eps_override=None):
    """u(p0) d~(p1) > W+(p2) H(p3) g(p4): the s-channel W of u d~ > W+ H (WWH vertex) with the gluon
    from the quark line before or after it (two diagrams, colour t^a)."""
    p = [P[:, k] for k in range(5)]
    gw = par.g / np.sqrt(2.0)
    gwwh = par.gwwh
    cT = _colour_string([0], 1)
    Q = p[2] + p[3]
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ew = polarisation(p[2], h[2], mass=par.mW).conj()
        eg = polarisation(p[4], h[3]).conj() if eps_override is None else eps_override
        Y = vector_prop(Q, 1j * gwwh * ew, par.mW, par.wW)
        A = _with_gluon([(vb, u, p[0], [(vector_insertion(Y, gw, 0.0), Q)])], eg, p[4], par.gs)
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 36.0


def udx_wpa(P, par=SMParams(), widths=True):
    """u(p0) d~(p1) > W+(p2) gamma(p3): the photon from the u line, from the d line, and from the
    s-channel W through the WWA vertex (the vertex of udx_wpz_amplitudes with the photon in place of
    the Z).  The s-channel W carries the width wW unless widths=False."""
    p = [P[:, k] for k in range(4)]
    gw = par.g / np.sqrt(2.0)
    wW = par.wW if widths else 0.0
    q = p[0] + p[1]
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ew = polarisation(p[2], h[2], mass=par.mW).conj()
        ea = polarisation(p[3], h[3]).conj()
        W = (vector_insertion(ew, gw, 0.0), p[2])
        A = (fermion_line(vb, u, p[0], [(vector_insertion(ea, *(2 * (_a_coupling("u", par),))), p[3]), W])
             + fermion_line(vb, u, p[0], [W, (vector_insertion(ea, *(2 * (_a_coupling("d", par),))), p[3])]))
        Ws = vector_prop(q, ffv_current(vb, u, gw, 0.0), par.mW, wW)
        A = A - 1j * par.e * mdot(vvv_out(Ws, q, ew, -p[2], -p[3], 1.0), ea)
        tot = tot + colour.colour_sum([A / 1j], [_DELTA3])
    return tot / 36.0


def udx_wpzg(P, par=SMParams(), eps_override=None):
    """u(p0) d~(p1) > W+(p2) Z(p3) g(p4): the three graphs of u d~ > W+ Z (Z from the u line, Z from
    the d line, s-channel W into the WWZ vertex) with the gluon at every place along the quark line
    (3 + 3 + 2 diagrams, colour t^a)."""
    p = [P[:, k] for k in range(5)]
    gw = par.g / np.sqrt(2.0)
    zu, zd = _z_couplings("u", par), _z_couplings("d", par)
    cT = _colour_string([0], 1)
    Q = p[2] + p[3]
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ew = polarisation(p[2], h[2], mass=par.mW).conj()
        ez = polarisation(p[3], h[3], mass=par.mZ).conj()
        eg = polarisation(p[4], h[4]).conj() if eps_override is None else eps_override
        W = (vector_insertion(ew, gw, 0.0), p[2])
        # the s-channel W: the WWZ vertex with the W+* on its first leg, contracted with the outgoing
        # W+ and Z, propagated back to the quark line (the vertex of udx_wpz_amplitudes, leg order cycled)
        Y = vector_prop(Q, -1j * par.g * par.cw * vvv_out(ew, -p[2], ez, -p[3], Q, 1.0), par.mW, par.wW)
        lines = [(vb, u, p[0], [(vector_insertion(ez, *zu), p[3]), W]),
                 (vb, u, p[0], [W, (vector_insertion(ez, *zd), p[3])]),
                 (vb, u, p[0], [(vector_insertion(Y, gw, 0.0), Q)])]
        A = _with_gluon(lines, eg, p[4], par.gs)
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 36.0


def uux_wpwmg(P, par=SMParams(), eps_override=None):
    """u(p0) u~(p1) > W+(p2) W-(p3) g(p4): the graphs of u u~ > W+ W- (t-channel d, s-channel photon
    and Z into the WWV vertex) with the gluon at every place along the quark line (3 + 2 + 2
    diagrams, colour t^a)."""
    p = [P[:, k] for k in range(5)]
    gw = par.g / np.sqrt(2.0)
    cT = _colour_string([0], 1)
    Q = p[2] + p[3]
    ga = _a_coupling("u", par)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ep = polarisation(p[2], h[2], mass=par.mW).conj()
        em = polarisation(p[3], h[3], mass=par.mW).conj()
        eg = polarisation(p[4], h[4]).conj() if eps_override is None else eps_override
        lines = [(vb, u, p[0], [(vector_insertion(ep, gw, 0.0), p[2]), (vector_insertion(em, gw, 0.0), p[3])])]
        X = vvv_out(em, -p[3], ep, -p[2], Q, 1.0)
        for gv, (gl, gr), mV, wV in ((par.e, (ga, ga), 0.0, 0.0),
                                     (par.g * par.cw, _z_couplings("u", par), par.mZ, par.wZ)):
            Y = vector_prop(Q, -1j * gv * X, mV, wV)
            lines.append((vb, u, p[0], [(vector_insertion(Y, gl, gr), Q)]))
        A = _with_gluon(lines, eg, p[4], par.gs)
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 36.0


# --------------------------------------------------------------------------
# u g > W+ d  (the crossing of u d~ > W+ g: the incoming gluon on either side of the W emission)
# --------------------------------------------------------------------------
def ug_wpd(P, par=SMParams()):
    """u(p0) g(p1) > W+(p2) d(p3): the quark line from u(p0) to ubar_d(p3) with the gluon absorbed
    before or after the W emission, colour t^a; averaged over 2 x 2 spins and 3 x 8 colours."""
    p = [P[:, k] for k in range(4)]
    gw = par.g / np.sqrt(2.0)
    cT = _colour_string([0], 1)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_V, HEL_W, HEL_F):
        u = u_spinor(p[0], h[0])
        eg = polarisation(p[1], h[1])
        ew = polarisation(p[2], h[2], mass=par.mW).conj()
        ubd = bar(u_spinor(p[3], h[3]))
        G = (vector_insertion(eg, par.gs, par.gs), -p[1])
        W = (vector_insertion(ew, gw, 0.0), p[2])
        A = fermion_line(ubd, u, p[0], [G, W]) + fermion_line(ubd, u, p[0], [W, G])
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 96.0


# --------------------------------------------------------------------------
# u u~ > Z H  (s-channel Z through the ZZH vertex)
# --------------------------------------------------------------------------
def uux_zh(P, par=SMParams()):
    """u(p0) u~(p1) > Z(p2) H(p3): the quark current into the Z propagator and the ZZH vertex
    i g_ZZH g^{mu nu}, g_ZZH = gZ mZ (Sect. 4.2 VVS)."""
    p = [P[:, k] for k in range(4)]
    zl, zr = _z_couplings("u", par)
    gzzh = par.gzzh
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ez = polarisation(p[2], h[2], mass=par.mZ).conj()
        Z = vector_prop(p[0] + p[1], ffv_current(vb, u, zl, zr), par.mZ, par.wZ)
        M = 1j * gzzh * mdot(Z, ez) / 1j
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# q q~' > V g  (vector boson plus one jet: the gluon from either quark)
# --------------------------------------------------------------------------
def _qqx_vg(P, par, gl, gr, mV):
    """q(p0) q~'(p1) > V(p2) g(p3) with V coupling i gamma^mu (gl P_L + gr P_R): the two orderings of
    the gluon and V insertions along the quark line, colour t^a."""
    p = [P[:, k] for k in range(4)]
    gs = par.gs
    cT = _colour_string([0], 1)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ev = polarisation(p[2], h[2], mass=mV).conj()
        eg = polarisation(p[3], h[3]).conj()
        G = (vector_insertion(eg, gs, gs), p[3])
        V = (vector_insertion(ev, gl, gr), p[2])
        A = fermion_line(vb, u, p[0], [G, V]) + fermion_line(vb, u, p[0], [V, G])
        tot = tot + colour.colour_sum([A / 1j], [cT])
    return tot / 36.0


def _qqx_vgg(P, par, gl, gr, mV, eps_override=None):
    """q(p0) q~'(p1) > V(p2) g(p3) g(p4) with an on-shell massive V of coupling i gamma^mu (gl P_L +
    gr P_R): the V and both gluons in all six orders along the quark line (colour strings of the two
    gluon orders), and the V with the pair from the three-gluon vertex in both orders (f^{abc} t^c).
    eps_override: optional {leg: vector[N,4]} replacing a gluon polarisation (Ward identity)."""
    p = [P[:, k] for k in range(5)]
    gs = par.gs
    colours = {o: _colour_string([x for x in o if x != "V"], 2) for o in itertools.permutations(["V", 0, 1])}
    cG = _colour_string(["G"], 2, with_f=(0, 1))
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_V, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ev = polarisation(p[2], h[2], mass=mV).conj()
        eg = [polarisation(p[3], h[3]).conj(), polarisation(p[4], h[4]).conj()]
        if eps_override:
            for leg, vec in eps_override.items():
                eg[leg - 3] = vec.astype(complex)
        ins = {"V": (vector_insertion(ev, gl, gr), p[2]), 0: (vector_insertion(eg[0], gs, gs), p[3]),
               1: (vector_insertion(eg[1], gs, gs), p[4])}
        amps, cols = [], []
        for order, c in colours.items():
            amps.append(fermion_line(vb, u, p[0], [ins[x] for x in order]) / 1j)
            cols.append(c)
        X = vvv_out(eg[0], -p[3], eg[1], -p[4], p[3] + p[4], gs)
        insG = (vector_insertion(vector_prop(p[3] + p[4], X), gs, gs), p[3] + p[4])
        for order in (["V", "G"], ["G", "V"]):
            amps.append(fermion_line(vb, u, p[0], [ins["V"] if x == "V" else insG for x in order]) / 1j)
            cols.append(cG)
        tot = tot + colour.colour_sum(amps, cols)
    return tot / 36.0


def udx_wpgg(P, par=SMParams(), eps_override=None):
    """u d~ > W+ g g (on-shell W plus two jets)."""
    return _qqx_vgg(P, par, par.g / np.sqrt(2.0), 0.0, par.mW, eps_override)


def uux_zgg(P, par=SMParams(), eps_override=None):
    """u u~ > Z g g (on-shell Z plus two jets)."""
    gl, gr = _z_couplings("u", par)
    return _qqx_vgg(P, par, gl, gr, par.mZ, eps_override)


# --------------------------------------------------------------------------
# q q~' > V + n gluons, n = 1, 2, 3 (V plus jets, Sect. 2.1): every Feynman diagram
# --------------------------------------------------------------------------
def _gluon_blocks(legs):
    """The ways a set of gluons joins into one gluon line that meets the quark line: as a list of
    (kind, spec).  One gluon: ("g", x); two: ("pair", (x, y)) through a three-gluon vertex; three:
    ("triple", (x, y, z)) through two three-gluon vertices ((x y) first) for each of the three pairs,
    and ("quartic", s) through the four-gluon vertex for its three colour structures s = 0, 1, 2."""
    legs = tuple(sorted(legs))
    if len(legs) == 1:
        return [("g", legs[0])]
    if len(legs) == 2:
        return [("pair", legs)]
    if len(legs) >= 4:
        return _gluon_trees(legs)
    x, y, z = legs
    return ([("triple", (a, b, c)) for a, b, c in ((x, y, z), (x, z, y), (y, z, x))]
            + [("quartic", (legs, s)) for s in range(3)])


def _gluon_trees(legs):
    """Four or more gluons joined into one line: every tree of three- and four-gluon vertices, as
    ("tree", t) with t = ("c3", block_a, block_b) (a three-gluon vertex joining the lines of two
    disjoint sets, the one holding the smallest leg first) or ("c4", s, block_a, block_b, block_c) (the
    four-gluon vertex joining three lines, colour structure s as for "quartic"); the sub-blocks are
    those of _gluon_blocks.  Four gluons: 15 trees of three-gluon vertices and 10 with one four-gluon
    vertex (30 with its colour structures)."""
    S = tuple(sorted(legs))
    out = []
    for part in _set_partitions(list(S)):
        blocks = sorted((tuple(sorted(b)) for b in part), key=lambda b: b[0])
        if len(blocks) == 2:
            for ba in _gluon_blocks(blocks[0]):
                for bb in _gluon_blocks(blocks[1]):
                    out.append(("tree", ("c3", ba, bb)))
        elif len(blocks) == 3:
            for ba in _gluon_blocks(blocks[0]):
                for bb in _gluon_blocks(blocks[1]):
                    for bc in _gluon_blocks(blocks[2]):
                        for s in range(3):
                            out.append(("tree", ("c4", s, ba, bb, bc)))
    return out


def _block_legs(kind, spec):
    if kind == "g":
        return (spec,)
    if kind in ("pair", "triple"):
        return tuple(sorted(spec))
    if kind == "quartic":
        return tuple(spec[0])
    if spec[0] == "c3":
        return tuple(sorted(_block_legs(*spec[1]) + _block_legs(*spec[2])))
    return tuple(sorted(_block_legs(*spec[2]) + _block_legs(*spec[3]) + _block_legs(*spec[4])))


def _block_adjoint(kind, spec, A):
    """The adjoint colour vector v[c] of a joined gluon line (its line meets the quark line as
    sum_c v[c] t^c), for gluon colours A[leg]."""
    F = _F
    if kind == "g":
        return np.eye(8)[A[spec]]
    if kind == "pair":
        x, y = spec
        return F[A[x], A[y], :]
    if kind == "triple":
        x, y, z = spec
        return np.einsum("e,ec->c", F[A[x], A[y], :], F[:, A[z], :])
    if kind == "quartic":
        (x, y, z), s = spec
        va, vb, vc = np.eye(8)[A[x]], np.eye(8)[A[y]], np.eye(8)[A[z]]
    elif spec[0] == "c3":
        va, vb = _block_adjoint(*spec[1], A), _block_adjoint(*spec[2], A)
        return np.einsum("a,b,abc->c", va, vb, F)
    else:
        s = spec[1]
        va, vb, vc = (_block_adjoint(*b, A) for b in spec[2:])
    # four-gluon vertex, legs (a, b, c, X): f^{abe} f^{cXe}, f^{ace} f^{bXe}, f^{aXe} f^{bce}
    if s == 0:
        return np.einsum("a,b,c,abe,cXe->X", va, vb, vc, F, F)
    if s == 1:
        return np.einsum("a,b,c,ace,bXe->X", va, vb, vc, F, F)
    return np.einsum("a,b,c,aXe,bce->X", va, vb, vc, F, F)


def _block_vtensor(kind, spec):
    """The adjoint vectors of a joined gluon line for every colour assignment of its legs, at once:
    an array with one axis of 8 per leg (in _block_legs order) and the adjoint axis last."""
    F = _F
    if kind == "g":
        return np.eye(8)
    if kind == "pair":
        return F.copy()
    if kind == "triple":
        x, y, z = spec
        v = np.einsum("xye,ezc->xyzc", F, F)          # legs in the order (x, y, z)
        return np.moveaxis(v, [0, 1, 2], [sorted(spec).index(x), sorted(spec).index(y), sorted(spec).index(z)])
    if kind == "quartic":
        s = spec[1]
        va = vb = vc = np.eye(8)
        la, lb, lc = (spec[0][0],), (spec[0][1],), (spec[0][2],)
    elif spec[0] == "c3":
        la, lb = _block_legs(*spec[1]), _block_legs(*spec[2])
        va, vb = _block_vtensor(*spec[1]), _block_vtensor(*spec[2])
    else:
        s = spec[1]
        la, lb, lc = (_block_legs(*b) for b in spec[2:])
        va, vb, vc = (_block_vtensor(*b) for b in spec[2:])
    letters = "ijklmnopqrstuvw"
    legs = sorted(la + lb + (lc if kind == "quartic" or spec[0] == "c4" else ()))
    L = {leg: letters[k] for k, leg in enumerate(legs)}
    sa, sb = "".join(L[l] for l in la), "".join(L[l] for l in lb)
    out = "".join(L[l] for l in legs)
    if kind != "quartic" and spec[0] == "c3":
        return np.einsum(f"{sa}a,{sb}b,abZ->{out}Z", va, vb, F)
    sc = "".join(L[l] for l in lc)
    rule = {0: "abe,cZe", 1: "ace,bZe", 2: "aZe,bce"}[s]
    return np.einsum(f"{sa}a,{sb}b,{sc}c,{rule}->{out}Z", va, vb, vc, F, F)


def _block_colour(kind, spec, A):
    """Colour matrix (3 x 3) a joined gluon line gives the quark line, for gluon colours A[leg]."""
    T, F = _T, _F
    if kind == "tree":
        return np.einsum("c,cij->ij", _block_adjoint(kind, spec, A), T)
    if kind == "g":
        return T[A[spec]]
    if kind == "pair":
        x, y = spec
        return np.einsum("c,cij->ij", F[A[x], A[y], :], T)
    if kind == "triple":
        x, y, z = spec
        return np.einsum("e,ec,cij->ij", F[A[x], A[y], :], F[:, A[z], :], T)
    (x, y, z), s = spec   # four-gluon vertex, legs (x, y, z, X): f^{xye} f^{zXe}, f^{xze} f^{yXe}, f^{xXe} f^{yze}
    if s == 0:
        return np.einsum("e,ce,cij->ij", F[A[x], A[y], :], F[A[z], :, :], T)
    if s == 1:
        return np.einsum("e,ce,cij->ij", F[A[x], A[z], :], F[A[y], :, :], T)
    return np.einsum("ce,e,cij->ij", F[A[x], :, :], F[A[y], A[z], :], T)


def _set_partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in _set_partitions(rest):
        for k in range(len(part)):
            yield part[:k] + [[first] + part[k]] + part[k + 1:]
        yield [[first]] + part


def _vjets_diagrams(n):
    """Every diagram of q q~' > V + n gluons as a sequence of insertions along the quark line, from
    the quark's column spinor to the antiquark's row spinor: "V" or a joined gluon line (kind, spec);
    and its explicit colour tensor [i_start, i_end, a_0 .. a_{n-1}]."""
    diags = []
    for part in _set_partitions(list(range(n))):
        for choice in itertools.product(*[_gluon_blocks(b) for b in part]):
            for order in itertools.permutations(["V"] + list(choice)):
                diags.append(order)
    tensors = []
    for order in diags:
        t = np.zeros((3, 3) + (8,) * n, dtype=complex)
        for a in itertools.product(range(8), repeat=n):
            M = np.eye(3, dtype=complex)
            for ins in order:
                if ins != "V":
                    M = _block_colour(ins[0], ins[1], a) @ M
            t[(slice(None), slice(None)) + a] = M.T
        tensors.append(t)
    return diags, colour.colour_projector(tensors)


_VJETS = {}


def qqx_v_ng(P, par, gl, gr, mV, eps_override=None):
    """q(p0) q~'(p1) > V(p2) g(p3) ... g(p_{2+n}), n = 1, 2, 3, with an on-shell V of mass mV coupling
    i gamma^mu (gl P_L + gr P_R) to the quark line: every diagram is an ordering along the quark line of
    the V and of the gluons joined into lines (_gluon_blocks: single gluons, pairs through the
    three-gluon vertex, triples through two three-gluon vertices or the four-gluon vertex); colour
    summed over explicit indices (colour_projector of the diagrams' colour tensors).
    eps_override: {leg: vector[N,4]} replaces a gluon's polarisation (Ward identity)."""
    n = P.shape[1] - 3
    if n not in _VJETS:
        _VJETS[n] = _vjets_diagrams(n)
    diags, G = _VJETS[n]
    p = [P[:, k] for k in range(P.shape[1])]
    gs = par.gs
    kg = {j: -p[3 + j] for j in range(n)}   # gluon momenta into the gluon vertices
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, *([HEL_V] * n)):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ev = polarisation(p[2], h[2], mass=mV).conj()
        eps = {j: polarisation(p[3 + j], h[3 + j]).conj() for j in range(n)}
        if eps_override:
            for leg, vec in eps_override.items():
                eps[leg - 3] = vec.astype(complex)
        cache = {}

        def line(kind, spec):
            """(current [N,4] into the quark line, momentum leaving the quark line)."""
            key = (kind, spec)
            if key in cache:
                return cache[key]
            if kind == "g":
                out = (eps[spec], p[3 + spec])
            elif kind == "pair":
                x, y = spec
                k = kg[x] + kg[y]
                out = (vector_prop(k, vvv_out(eps[x], kg[x], eps[y], kg[y], -k, gs)), -k)
            elif kind == "triple":
                x, y, z = spec
                J, mk = line("pair", (x, y))
                k = -mk
                K = k + kg[z]
                out = (vector_prop(K, vvv_out(J, k, eps[z], kg[z], -K, gs)), -K)
            else:
                (x, y, z), s = spec
                K = kg[x] + kg[y] + kg[z]
                out = (vector_prop(K, -1j * gs * gs * _vvvv_out(eps[x], eps[y], eps[z])[s]), -K)
            cache[key] = out
            return out

        amps = []
        for order in diags:
            ins = []
            for x in order:
                if x == "V":
                    ins.append((vector_insertion(ev, gl, gr), p[2]))
                else:
                    J, Q = line(*x)
                    ins.append((vector_insertion(J, gs, gs), Q))
            amps.append(fermion_line(vb, u, p[0], ins) / 1j)
        tot = tot + colour.colour_norm(amps, G)
    return tot / 36.0


def _line_colour_tensor(blocks, ng):
    """Explicit colour tensor [i_start, i_end, a_0 .. a_{ng-1}] of a quark line with the joined gluon
    lines `blocks` in order from the start of the fermion arrow: (t_last ... t_first)_{i_end i_start},
    each block's matrix sum_c v[c] t^c built for all colour assignments at once (_block_vtensor)."""
    letters = "abcdefgh"
    R = np.eye(3, dtype=complex)          # axes: current index, start index
    rs = "xz"
    for kind, spec in blocks:
        legs = _block_legs(kind, spec)
        Mb = np.einsum("...c,cij->...ij", _block_vtensor(kind, spec), _T)   # legs..., row, column
        ls = "".join(letters[l] for l in legs)
        R = np.einsum(f"{ls}yx,{rs}->y{rs[1:]}{ls}", Mb, R)
        rs = "x" + rs[1:] + ls
    order = "".join(letters[l] for l in range(ng))
    return np.einsum(f"{rs}->zx{order}", R)


def fermion_line_process(P, par, col, row, colourless, gluons, mf=0.0, wf=0.0, average=1.0 / 36.0,
                         eps_override=None, alternatives=None, keep_order=False):
    """|M|^2 of a process with one fermion line, colourless bosons attached to it and any number (up
    to three) of incoming or outgoing gluons, from every Feynman diagram: the orderings along the line
    of the colourless insertions and of the gluons joined into lines (_gluon_blocks), colour summed
    over explicit indices (colour_projector), averaged by `average`.

    col: (leg, "u") an incoming quark or (leg, "v") an outgoing antiquark, where the fermion-number
    arrow starts; row: (leg, "ubar") an outgoing quark or (leg, "vbar") an incoming antiquark, where it
    ends.  colourless: outgoing bosons as dicts (leg, kind "V" with gl, gr, mass: i gamma^mu (gl P_L +
    gr P_R); kind "S" with y: i y; kind "VS" with legs (vector, scalar), gl, gr, mass, width, gvvs: an
    off-shell vector of that mass and width from the line into the external vector and scalar through
    the i gvvs g^{mu nu} vertex; kind "VV" with legs (V2, V1), gl, gr, mass, width, gv, vmass (one mass,
    or one per leg): an off-shell vector from the line into two external vectors through the three-vector
    vertex -i gv [...] with (V1, V2, V) = (legs[1], legs[0], line), the W W gamma / W W Z rule of Sect.
    4.2).  alternatives: several such lists whose diagrams add coherently (for instance t-channel W
    emissions and an s-channel photon or Z); keep_order: an alternative's insertions stay in their
    listed order along the line (the t-channel quark between two W emissions fixes it).  gluons:
    (leg, incoming) pairs.  Internal fermions carry mass mf and width wf.  eps_override: {leg:
    vector[N,4]} replaces a gluon's polarisation."""
    confs = alternatives if alternatives is not None else [colourless]
    ng = len(gluons)
    key = ("line", ng, tuple(len(c) for c in confs), keep_order)
    if key not in _VJETS:
        diags = []
        for ci, conf in enumerate(confs):
            for part in _set_partitions(list(range(ng))):
                for choice in itertools.product(*[_gluon_blocks(b) for b in part]):
                    for order in itertools.permutations([("c", i) for i in range(len(conf))] + list(choice)):
                        seq = [x[1] for x in order if x[0] == "c"]
                        if keep_order and seq != sorted(seq):
                            continue
                        diags.append((ci, order))
        tensors = []
        for _, order in diags:
            if ng >= 4:
                tensors.append(_line_colour_tensor([ins for ins in order if ins[0] != "c"], ng))
                continue
            t = np.zeros((3, 3) + (8,) * ng, dtype=complex)
            for a in itertools.product(range(8), repeat=ng):
                M = np.eye(3, dtype=complex)
                for ins in order:
                    if ins[0] != "c":
                        M = _block_colour(ins[0], ins[1], a) @ M
                t[(slice(None), slice(None)) + a] = M.T
            tensors.append(t)
        _VJETS[key] = (diags, colour.colour_projector(tensors))
    diags, B = _VJETS[key]
    p = [P[:, k] for k in range(P.shape[1])]
    gs = par.gs
    kg = {j: (p[l] if inc else -p[l]) for j, (l, inc) in enumerate(gluons)}
    p_start = p[col[0]] if col[1] == "u" else -p[col[0]]
    # external colourless legs: (leg, mass) of vectors, scalars; helicities per leg, shared by the
    # alternatives
    vlegs = {}
    for conf in confs:
        for c in conf:
            if c["kind"] == "V":
                vlegs[c["leg"]] = c["mass"]
            elif c["kind"] == "VS":
                vlegs[c["legs"][0]] = c["mass"]
            elif c["kind"] == "VV":
                vm = c["vmass"] if isinstance(c["vmass"], tuple) else (c["vmass"], c["vmass"])
                vlegs[c["legs"][0]], vlegs[c["legs"][1]] = vm
    vl = sorted(vlegs)
    hels = [HEL_F, HEL_F] + [HEL_W] * len(vl) + [HEL_V] * ng
    tot = 0.0
    for h in itertools.product(*hels):
        cs = u_spinor(p[col[0]], h[0]) if col[1] == "u" else v_spinor(p[col[0]], h[0])
        rs = bar(u_spinor(p[row[0]], h[1]) if row[1] == "ubar" else v_spinor(p[row[0]], h[1]))
        pol = {l: polarisation(p[l], hv, mass=vlegs[l]).conj() for l, hv in zip(vl, h[2:2 + len(vl)])}
        cins = []
        for conf in confs:
            ci_list = []
            for c in conf:
                if c["kind"] == "VS":
                    # an off-shell V* from the line into the external V and scalar through V V S
                    pv, pss = p[c["legs"][0]], p[c["legs"][1]]
                    X = vector_prop(pv + pss, 1j * c["gvvs"] * pol[c["legs"][0]], c["mass"], c["width"])
                    ci_list.append((vector_insertion(X, c["gl"], c["gr"]), pv + pss))
                elif c["kind"] == "VV":
                    # an off-shell V* from the line into two external vectors through V V V
                    l2, l1 = c["legs"]
                    Q = p[l2] + p[l1]
                    X = vvv_out(pol[l1], -p[l1], pol[l2], -p[l2], Q, 1.0)
                    Y = vector_prop(Q, -1j * c["gv"] * X, c["mass"], c["width"])
                    ci_list.append((vector_insertion(Y, c["gl"], c["gr"]), Q))
                elif c["kind"] == "V":
                    ci_list.append((vector_insertion(pol[c["leg"]], c["gl"], c["gr"]), p[c["leg"]]))
                else:
                    ci_list.append((np.broadcast_to(1j * c["y"] * np.eye(4, dtype=complex), (P.shape[0], 4, 4)),
                                    p[c["leg"]]))
            cins.append(ci_list)
        eps = {}
        for j_, ((l, inc), hg) in enumerate(zip(gluons, h[2 + len(vl):])):
            e = polarisation(p[l], hg)
            eps[j_] = e if inc else e.conj()
            if eps_override and l in eps_override:
                eps[j_] = eps_override[l].astype(complex)
        cache = {}

        def line(kind, spec):
            """(gluon line [N,4] into the fermion line, momentum leaving the fermion line)."""
            k_ = (kind, spec)
            if k_ in cache:
                return cache[k_]
            if kind == "g":
                out = (eps[spec], -kg[spec])
            elif kind == "pair":
                x, y = spec
                k = kg[x] + kg[y]
                out = (vector_prop(k, vvv_out(eps[x], kg[x], eps[y], kg[y], -k, gs)), -k)
            elif kind == "triple":
                x, y, z = spec
                J, mk = line("pair", (x, y))
                k = -mk
                K = k + kg[z]
                out = (vector_prop(K, vvv_out(J, k, eps[z], kg[z], -K, gs)), -K)
            elif kind == "quartic":
                (x, y, z), s_ = spec
                K = kg[x] + kg[y] + kg[z]
                out = (vector_prop(K, -1j * gs * gs * _vvvv_out(eps[x], eps[y], eps[z])[s_]), -K)
            elif spec[0] == "c3":
                (JA, mA), (JB, mB) = line(*spec[1]), line(*spec[2])
                K = -(mA + mB)
                out = (vector_prop(K, vvv_out(JA, -mA, JB, -mB, -K, gs)), -K)
            else:
                sub = [line(*b) for b in spec[2:]]
                K = -(sub[0][1] + sub[1][1] + sub[2][1])
                out = (vector_prop(K, -1j * gs * gs * _vvvv_out(sub[0][0], sub[1][0], sub[2][0])[spec[1]]), -K)
            cache[k_] = out
            return out

        amps = []
        for ci, order in diags:
            ins = []
            for x in order:
                if x[0] == "c":
                    ins.append(cins[ci][x[1]])
                else:
                    J, Q = line(*x)
                    ins.append((vector_insertion(J, gs, gs), Q))
            amps.append(fermion_line(rs, cs, p_start, ins, mf, wf) / 1j)
        tot = tot + colour.colour_norm(amps, B)
    return tot * average


def us_dch_ng(P, par=SMParams(), eps_override=None):
    """u(p0) s(p1) > d(p2) c(p3) H(p4) + n gluons (p5 ...), n up to 3, by W+ W- fusion (WBF H plus jets):
    every diagram places the gluons, joined into lines (_gluon_blocks), on either quark line and orders
    each line's insertions (its W vertex and its gluon lines).  The line s > c, with its W vertex left
    open, is evaluated against the four basis vectors to give its current J2 (upper index); its W
    propagator, the W W H vertex and the W propagator of the line u > d turn it into the vector that
    line absorbs.  Colour: each line keeps its own string, (M1)_{d u} (M2)_{c s}, summed over explicit
    indices (colour_projector).  eps_override: {leg: vector[N,4]} replaces a gluon's polarisation."""
    ng = P.shape[1] - 5
    key = ("wbf", ng)
    if key not in _VJETS:
        diags = []
        for part in _set_partitions(list(range(ng))):
            for choice in itertools.product(*[_gluon_blocks(b) for b in part]):
                for side in itertools.product((0, 1), repeat=len(choice)):
                    on = [[b for b, sd in zip(choice, side) if sd == k] for k in (0, 1)]
                    for o1 in itertools.permutations([("W",)] + on[0]):
                        for o2 in itertools.permutations([("W",)] + on[1]):
                            diags.append((o1, o2))
        tensors = []
        for o1, o2 in diags:
            t = np.zeros((3, 3, 3, 3) + (8,) * ng, dtype=complex)
            for a in itertools.product(range(8), repeat=ng):
                M = []
                for o in (o1, o2):
                    m_ = np.eye(3, dtype=complex)
                    for ins in o:
                        if ins[0] != "W":
                            m_ = _block_colour(ins[0], ins[1], a) @ m_
                    M.append(m_.T)   # [i_start, i_end]
                t[(slice(None),) * 4 + a] = np.einsum("ud,sc->udsc", M[0], M[1])
            tensors.append(t)
        _VJETS[key] = (diags, colour.colour_projector(tensors))
    diags, B = _VJETS[key]
    p = [P[:, k] for k in range(P.shape[1])]
    gs, gw, gwwh = par.gs, par.g / np.sqrt(2.0), par.gwwh
    kg = {j: -p[5 + j] for j in range(ng)}
    basis = [np.broadcast_to(np.eye(4)[mu], (P.shape[0], 4)).astype(complex) for mu in range(4)]
    metric = np.array([1.0, -1.0, -1.0, -1.0])
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_F, HEL_F, *([HEL_V] * ng)):
        ub_d, u_u = bar(u_spinor(p[2], h[2])), u_spinor(p[0], h[0])
        ub_c, u_s = bar(u_spinor(p[3], h[3])), u_spinor(p[1], h[1])
        eps = {j: polarisation(p[5 + j], h[4 + j]).conj() for j in range(ng)}
        if eps_override:
            for leg, vec in eps_override.items():
                eps[leg - 5] = vec.astype(complex)
        cache = {}

        def gline(kind, spec):
            k_ = (kind, spec)
            if k_ in cache:
                return cache[k_]
            if kind == "g":
                out = (eps[spec], -kg[spec])
            elif kind == "pair":
                x, y = spec
                k = kg[x] + kg[y]
                out = (vector_prop(k, vvv_out(eps[x], kg[x], eps[y], kg[y], -k, gs)), -k)
            elif kind == "triple":
                x, y, z = spec
                J, mk = gline("pair", (x, y))
                k = -mk
                K = k + kg[z]
                out = (vector_prop(K, vvv_out(J, k, eps[z], kg[z], -K, gs)), -K)
            else:
                (x, y, z), s_ = spec
                K = kg[x] + kg[y] + kg[z]
                out = (vector_prop(K, -1j * gs * gs * _vvvv_out(eps[x], eps[y], eps[z])[s_]), -K)
            cache[k_] = out
            return out

        amps = []
        for o1, o2 in diags:
            # W momenta: what each line gives away at its W vertex
            q = []
            for o, pin, pout in ((o1, p[0], p[2]), (o2, p[1], p[3])):
                qq = pin - pout
                for ins in o:
                    if ins[0] != "W":
                        qq = qq - gline(*ins)[1]
                q.append(qq)
            # the line s > c with its W vertex open: J2_mu against the basis vectors, raised
            ins2 = [None if x[0] == "W" else (vector_insertion(gline(*x)[0], gs, gs), gline(*x)[1]) for x in o2]
            J2 = np.zeros((P.shape[0], 4), dtype=complex)
            for mu in range(4):
                seq = [(vector_insertion(basis[mu], gw, 0.0), q[1]) if x is None else x for x in ins2]
                J2[:, mu] = metric[mu] * fermion_line(ub_c, u_s, p[1], seq)
            V = vector_prop(q[0], 1j * gwwh * vector_prop(q[1], J2, par.mW, par.wW), par.mW, par.wW)
            seq1 = [(vector_insertion(V, gw, 0.0), q[0]) if x[0] == "W" else
                    (vector_insertion(gline(*x)[0], gs, gs), gline(*x)[1]) for x in o1]
            amps.append(fermion_line(ub_d, u_u, p[0], seq1) / 1j)
        tot = tot + colour.colour_norm(amps, B)
    return tot / 36.0


def us_dchgg(P, par=SMParams(), eps_override=None):
    """u s > d c H g g (WBF H plus two jets, 24 diagrams; us_dch_ng)."""
    return us_dch_ng(P, par, eps_override)


def uux_zzgg(P, par=SMParams(), eps_override=None):
    """u(p0) u~(p1) > Z(p2) Z(p3) g(p4) g(p5) (V V plus two jets, 30 diagrams): the quark line from u(p0)
    to vbar(p1) with both Z bosons and the gluons (fermion_line_process)."""
    gl, gr = _z_couplings("u", par)
    z = [dict(leg=k, kind="V", gl=gl, gr=gr, mass=par.mZ) for k in (2, 3)]
    return fermion_line_process(P, par, (0, "u"), (1, "vbar"), z, [(4, False), (5, False)], 0.0, 0.0, 1.0 / 36.0,
                                eps_override)


def udx_wphgg(P, par=SMParams(), eps_override=None):
    """u(p0) d~(p1) > W+(p2) H(p3) g(p4) g(p5) (H V plus two jets, 8 diagrams): the quark line from u(p0)
    to vbar(p1) with the W* > W+ H insertion and the gluons (fermion_line_process)."""
    wh = dict(kind="VS", legs=(2, 3), gl=par.g / np.sqrt(2.0), gr=0.0, mass=par.mW, width=par.wW, gvvs=par.gwwh)
    return fermion_line_process(P, par, (0, "u"), (1, "vbar"), [wh], [(4, False), (5, False)], 0.0, 0.0,
                                1.0 / 36.0, eps_override)


def wpwm_line_alternatives(par):
    """The colourless parts of u u~ > W+(p2) W-(p3) on the quark line: the two W emissions in the order
    the t-channel d quark fixes (W+ nearer the u), or an s-channel photon or Z into the W W V vertex."""
    gw = par.g / np.sqrt(2.0)
    ga = _a_coupling("u", par)
    zl, zr = _z_couplings("u", par)
    t = [dict(leg=2, kind="V", gl=gw, gr=0.0, mass=par.mW), dict(leg=3, kind="V", gl=gw, gr=0.0, mass=par.mW)]
    a = [dict(kind="VV", legs=(2, 3), gl=ga, gr=ga, mass=0.0, width=0.0, gv=par.e, vmass=par.mW)]
    z = [dict(kind="VV", legs=(2, 3), gl=zl, gr=zr, mass=par.mZ, width=par.wZ, gv=par.g * par.cw, vmass=par.mW)]
    return [t, a, z]


def uux_wpwmgg(P, par=SMParams(), eps_override=None):
    """u(p0) u~(p1) > W+(p2) W-(p3) g(p4) g(p5) (W+ W- plus two jets, 31 diagrams): the quark line with the
    t-channel W pair or the s-channel photon or Z, and the gluons (fermion_line_process)."""
    return fermion_line_process(P, par, (0, "u"), (1, "vbar"), None, [(4, False), (5, False)], 0.0, 0.0,
                                1.0 / 36.0, eps_override, alternatives=wpwm_line_alternatives(par), keep_order=True)


def wpz_line_alternatives(par):
    """The colourless parts of u d~ > W+(p2) Z(p3) on the quark line: the Z from the u before the W+
    turns it into a d, the Z from the d after it, or an s-channel W into the W W Z vertex."""
    gw = par.g / np.sqrt(2.0)
    zu, zd = _z_couplings("u", par), _z_couplings("d", par)
    w = dict(leg=2, kind="V", gl=gw, gr=0.0, mass=par.mW)
    return [[dict(leg=3, kind="V", gl=zu[0], gr=zu[1], mass=par.mZ), w],
            [w, dict(leg=3, kind="V", gl=zd[0], gr=zd[1], mass=par.mZ)],
            [dict(kind="VV", legs=(3, 2), gl=gw, gr=0.0, mass=par.mW, width=par.wW, gv=par.g * par.cw,
                  vmass=(par.mZ, par.mW))]]


def udx_wpzgg(P, par=SMParams(), eps_override=None):
    """u(p0) d~(p1) > W+(p2) Z(p3) g(p4) g(p5) (W+ Z plus two jets, 38 diagrams): the three u d~ > W+ Z graphs
    with the gluons (fermion_line_process)."""
    return fermion_line_process(P, par, (0, "u"), (1, "vbar"), None, [(4, False), (5, False)], 0.0, 0.0,
                                1.0 / 36.0, eps_override, alternatives=wpz_line_alternatives(par), keep_order=True)


def udx_wphggg(P, par=SMParams(), eps_override=None):
    """u(p0) d~(p1) > W+(p2) H(p3) g(p4) g(p5) g(p6) (H V plus three jets, 54 diagrams): the quark line with the
    W* > W+ H insertion and the three gluons (fermion_line_process)."""
    wh = dict(kind="VS", legs=(2, 3), gl=par.g / np.sqrt(2.0), gr=0.0, mass=par.mW, width=par.wW, gvvs=par.gwwh)
    return fermion_line_process(P, par, (0, "u"), (1, "vbar"), [wh], [(4, False), (5, False), (6, False)], 0.0,
                                0.0, 1.0 / 36.0, eps_override)


def gg_ttxgg(P, par=SMParams(), eps_override=None, widths=True):
    """g(0) g(1) > t(2) t~(3) g(4) g(5) (t t~ plus two jets, 159 diagrams): the top line from v(p3) to ubar(p2)
    with the four gluons joined into lines, four-gluon trees included (fermion_line_process)."""
    return fermion_line_process(P, par, (3, "v"), (2, "ubar"), [], [(0, True), (1, True), (4, False), (5, False)],
                                par.mt, par.wt if widths else 0.0, 1.0 / 256.0, eps_override)


def gg_ttxhg(P, par=SMParams(), eps_override=None, widths=True):
    """g(0) g(1) > t(2) t~(3) H(4) g(5) (H t t~ plus one jet): the top line from v(p3) to ubar(p2) with the
    Higgs (Yukawa -mt/v) and the three gluons, 54 diagrams (fermion_line_process)."""
    return fermion_line_process(P, par, (3, "v"), (2, "ubar"), [dict(leg=4, kind="S", y=-par.mt / par.vev)],
                                [(0, True), (1, True), (5, False)], par.mt, par.wt if widths else 0.0,
                                1.0 / 256.0, eps_override)


def udx_wpggg(P, par=SMParams(), eps_override=None):
    """u d~ > W+ g g g (on-shell W plus three jets, 54 diagrams)."""
    return qqx_v_ng(P, par, par.g / np.sqrt(2.0), 0.0, par.mW, eps_override)


def uux_zggg(P, par=SMParams(), eps_override=None):
    """u u~ > Z g g g (on-shell Z plus three jets, 54 diagrams)."""
    gl, gr = _z_couplings("u", par)
    return qqx_v_ng(P, par, gl, gr, par.mZ, eps_override)


def _uux_va(P, par, gl, gr, mV):
    """u(p0) u~(p1) > V(p2) gamma(p3): both orders of the V (coupling gl, gr; mass mV, 0 for a photon)
    and the photon along the quark line, colour delta."""
    p = [P[:, k] for k in range(4)]
    qa = _a_coupling("u", par)
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W if mV > 0 else HEL_V, HEL_V):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ev = polarisation(p[2], h[2], mass=mV).conj()
        ea = polarisation(p[3], h[3]).conj()
        V = (vector_insertion(ev, gl, gr), p[2])
        A = (vector_insertion(ea, qa, qa), p[3])
        M = (fermion_line(vb, u, p[0], [A, V]) + fermion_line(vb, u, p[0], [V, A])) / 1j
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


def uux_za(P, par=SMParams()):
    """u u~ > Z gamma."""
    return _uux_va(P, par, *_z_couplings("u", par), par.mZ)


def uux_aa(P, par=SMParams()):
    """u u~ > gamma gamma (identical photons; no symmetry factor here)."""
    qa = _a_coupling("u", par)
    return _uux_va(P, par, qa, qa, 0.0)


def udx_wpg(P, par=SMParams()):
    """u d~ > W+ g."""
    return _qqx_vg(P, par, par.g / np.sqrt(2.0), 0.0, par.mW)


def uux_zg(P, par=SMParams()):
    """u u~ > Z g."""
    gl, gr = _z_couplings("u", par)
    return _qqx_vg(P, par, gl, gr, par.mZ)


# --------------------------------------------------------------------------
# u d~ > W+ H  (s-channel W through the WWH vertex)
# --------------------------------------------------------------------------
def udx_wph(P, par=SMParams()):
    """u(p0) d~(p1) > W+(p2) H(p3): the quark current into the W propagator and the WWH vertex
    i g_WWH g^{mu nu}, g_WWH = g mW (Sect. 4.2 VVS)."""
    p = [P[:, k] for k in range(4)]
    gw = par.g / np.sqrt(2.0)
    gwwh = par.gwwh
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W):
        u = u_spinor(p[0], h[0])
        vb = bar(v_spinor(p[1], h[1]))
        ew = polarisation(p[2], h[2], mass=par.mW).conj()
        W = vector_prop(p[0] + p[1], ffv_current(vb, u, gw, 0.0), par.mW, par.wW)
        M = 1j * gwwh * mdot(W, ew) / 1j
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# u u~ > W+ W-  (t-channel d exchange, s-channel photon and Z through the WWV vertex)
# --------------------------------------------------------------------------
HEL_W = (-1, 0, 1)


def uux_wpwm_amplitudes(P, hel, par=SMParams()):
    """The three diagrams of u(p0) u~(p1) > W+(p2) W-(p3) for fixed helicities (t-channel d quark,
    s-channel photon, s-channel Z), returned separately as M values.

    WWV vertex (the VVV function of Sect. 4.2 with (V1, V2, V3) = (W-, W+, V) and coupling
    g_WWA = e, g_WWZ = g cos(theta_W)): with every momentum incoming and the outgoing W- and W+
    entering as V1 and V2, its factor in i M is -i g_V [g^{12}(k1 - k2)^3 + g^{23}(k2 - k3)^1 +
    g^{31}(k3 - k1)^2].  The phase and orientation are those under which the longitudinal
    amplitude stays finite at high energy (tests/test_oracle_processes.py)."""
    p = [P[:, k] for k in range(4)]
    gw = par.g / np.sqrt(2.0)
    u = u_spinor(p[0], hel[0])
    vb = bar(v_spinor(p[1], hel[1]))
    ep = polarisation(p[2], hel[2], mass=par.mW).conj()
    em = polarisation(p[3], hel[3], mass=par.mW).conj()
    out = [fermion_line(vb, u, p[0], [(vector_insertion(ep, gw, 0.0), p[2]),
                                      (vector_insertion(em, gw, 0.0), p[3])])]
    q = p[0] + p[1]
    X = vvv_out(em, -p[3], ep, -p[2], q, 1.0)
    ga = _a_coupling("u", par)
    for gv, (gl, gr), mV, wV in ((par.e, (ga, ga), 0.0, 0.0),
                                 (par.g * par.cw, _z_couplings("u", par), par.mZ, par.wZ)):
        V = vector_prop(q, ffv_current(vb, u, gl, gr), mV, wV)
        out.append(-1j * gv * mdot(X, V))
    return [x / 1j for x in out]


def uux_wpwm(P, par=SMParams()):
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W):
        M = sum(uux_wpwm_amplitudes(P, h, par))
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# u d~ > W+ Z  (u and d exchange, s-channel W through the WWZ vertex)
# --------------------------------------------------------------------------
def udx_wpz_amplitudes(P, hel, par=SMParams()):
    """The three diagrams of u(p0) d~(p1) > W+(p2) Z(p3) for fixed helicities (Z from the u line, Z
    from the d line, s-channel W), returned separately as M values.  The WWZ vertex is the one of
    uux_wpwm_amplitudes: -i g_WWZ times the Lorentz structure, with the s-channel W+ entering as the
    incoming W+ (V1), the outgoing W+ as the incoming W- (V2) and the Z as V3."""
    p = [P[:, k] for k in range(4)]
    gw = par.g / np.sqrt(2.0)
    u = u_spinor(p[0], hel[0])
    vb = bar(v_spinor(p[1], hel[1]))
    ew = polarisation(p[2], hel[2], mass=par.mW).conj()
    ez = polarisation(p[3], hel[3], mass=par.mZ).conj()
    zu, zd = _z_couplings("u", par), _z_couplings("d", par)
    out = [fermion_line(vb, u, p[0], [(vector_insertion(ez, *zu), p[3]), (vector_insertion(ew, gw, 0.0), p[2])]),
           fermion_line(vb, u, p[0], [(vector_insertion(ew, gw, 0.0), p[2]), (vector_insertion(ez, *zd), p[3])])]
    q = p[0] + p[1]
    W = vector_prop(q, ffv_current(vb, u, gw, 0.0), par.mW, par.wW)
    out.append(-1j * par.g * par.cw * mdot(vvv_out(W, q, ew, -p[2], -p[3], 1.0), ez))
    return [x / 1j for x in out]


def udx_wpz(P, par=SMParams()):
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W):
        M = sum(udx_wpz_amplitudes(P, h, par))
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# h h > h h  (the SSSS contact vertex and the s-, t- and u-channel Higgs exchange)
# --------------------------------------------------------------------------
def hh_hh(P, par=SMParams()):
    """h(0) h(1) > h(2) h(3) from the Feynman rules of Sect. 4.2 (SSS and SSSS): the contact vertex
    -i 3 mH^2/v^2 and the three exchange diagrams, each (-i 3 mH^2/v)^2 times the scalar propagator
    i/(q^2 - mH^2 + i mH wH).  No spins or colours to sum."""
    p = [P[:, k] for k in range(4)]
    v = par.vev
    g3 = -3.0 * par.mH ** 2 / v
    g4 = -3.0 * par.mH ** 2 / v ** 2
    iM = 1j * g4 + 0.0 * p[0][:, 0]
    for q in (p[0] + p[1], p[0] - p[2], p[0] - p[3]):
        iM = iM + (1j * g3) * scalar_prop(q, par.mH, par.wH) * (1j * g3)
    return np.abs(iM / 1j) ** 2


# --------------------------------------------------------------------------
# u u~ > W+ W- gamma  (quark-line emissions, W-line emissions, the WWAA and WWAZ quartic vertices)
# --------------------------------------------------------------------------
def vvvv(gg, V1, V2, V3, V4):
    """The four-vector function of Sect. 4.2 (VVVV): gg [(V1.V4)(V2.V3) - (V1.V3)(V2.V4)], the
    Lagrangian of four distinct vectors evaluated on the four wavefunctions."""
    return gg * (mdot(V1, V4) * mdot(V2, V3) - mdot(V1, V3) * mdot(V2, V4))


def ww33(gg, Wm, V2, Wp, V4):
    """The electroweak quartic W- W3 W+ W3 vertex as the sum of its two channels (Sect. 4.2 VVVV,
    the W W W3 W3 identification): Gamma(gg; W-, V2, W+, V4) + Gamma(gg; W-, V4, W+, V2), with the
    vectors named by their outgoing quantum numbers and gg = g^2 times the W3 projections of the two
    neutral bosons (sw^2 for two photons, sw cw for a photon and a Z, cw^2 for two Z).  Its factor
    in i M is i times this value."""
    return vvvv(gg, Wm, V2, Wp, V4) + vvvv(gg, Wm, V4, Wp, V2)


def uux_wpwma_amplitudes(P, hel, par=SMParams(), eps_override=None, widths=True):
    """The fifteen diagrams of u(p0) u~(p1) > W+(p2) W-(p3) gamma(p4) for fixed helicities, returned
    as M values in five groups:
      line   the photon on the u, d or u segment of the t-channel quark line (3),
      wline  the photon from the W+ or the W- of the t-channel graph (2),
      isr    the photon from the quark line before or after the s-channel photon or Z that turns
             into W+ W- (4),
      wv     the s-channel photon or Z into W+* W- or W+ W-* with the photon from the W (4),
      quart  the s-channel photon or Z into W+ W- gamma through the quartic vertex (2).
    The WWV vertex is the one of uux_wpwm_amplitudes; the quartic one is ww33.  eps_override
    replaces the photon's polarisation vector (the Ward identity); widths=False sets the W and Z
    widths to zero."""
    p = [P[:, k] for k in range(5)]
    gw = par.g / np.sqrt(2.0)
    wW = par.wW if widths else 0.0
    wZ = par.wZ if widths else 0.0
    u = u_spinor(p[0], hel[0])
    vb = bar(v_spinor(p[1], hel[1]))
    ep = polarisation(p[2], hel[2], mass=par.mW).conj()
    em = polarisation(p[3], hel[3], mass=par.mW).conj()
    ea = polarisation(p[4], hel[4]).conj() if eps_override is None else eps_override
    Wp_ins = vector_insertion(ep, gw, 0.0)
    Wm_ins = vector_insertion(em, gw, 0.0)
    Au = vector_insertion(ea, *(2 * (_a_coupling("u", par),)))
    Ad = vector_insertion(ea, *(2 * (_a_coupling("d", par),)))
    out = {}
    out["line"] = [fermion_line(vb, u, p[0], [(Au, p[4]), (Wp_ins, p[2]), (Wm_ins, p[3])]),
                   fermion_line(vb, u, p[0], [(Wp_ins, p[2]), (Ad, p[4]), (Wm_ins, p[3])]),
                   fermion_line(vb, u, p[0], [(Wp_ins, p[2]), (Wm_ins, p[3]), (Au, p[4])])]
    # off-shell W+* -> W+ gamma and W-* -> W- gamma, propagated (the WWA vertex, coupling e)
    Pp = p[2] + p[4]
    Pm = p[3] + p[4]
    Wps = vector_prop(Pp, -1j * par.e * vvv_out(ep, -p[2], ea, -p[4], Pp, 1.0), par.mW, wW)
    Wms = vector_prop(Pm, -1j * par.e * vvv_out(ea, -p[4], em, -p[3], Pm, 1.0), par.mW, wW)
    out["wline"] = [fermion_line(vb, u, p[0], [(vector_insertion(Wps, gw, 0.0), Pp), (Wm_ins, p[3])]),
                    fermion_line(vb, u, p[0], [(Wp_ins, p[2]), (vector_insertion(Wms, gw, 0.0), Pm)])]
    q = p[0] + p[1]
    Q = p[2] + p[3]
    ga = _a_coupling("u", par)
    out["isr"], out["wv"], out["quart"] = [], [], []
    for gv, (gl, gr), mV, wV, g4 in ((par.e, (ga, ga), 0.0, 0.0, par.g ** 2 * par.sw2),
                                     (par.g * par.cw, _z_couplings("u", par), par.mZ, wZ,
                                      par.g ** 2 * par.sw * par.cw)):
        # photon from the quark line, then V* (momentum p2 + p3) into W+ W-
        X = -1j * gv * vvv_out(em, -p[3], ep, -p[2], Q, 1.0)
        Vins = vector_insertion(vector_prop(Q, X, mV, wV), gl, gr)
        out["isr"] += [fermion_line(vb, u, p[0], [(Au, p[4]), (Vins, Q)]),
                       fermion_line(vb, u, p[0], [(Vins, Q), (Au, p[4])])]
        V = vector_prop(q, ffv_current(vb, u, gl, gr), mV, wV)
        out["wv"] += [-1j * gv * mdot(vvv_out(em, -p[3], Wps, -Pp, q, 1.0), V),
                      -1j * gv * mdot(vvv_out(Wms, -Pm, ep, -p[2], q, 1.0), V)]
        out["quart"] += [1j * ww33(g4, em, ea, ep, V)]
    return {k: [x / 1j for x in v] for k, v in out.items()}


def uux_wpwma(P, par=SMParams()):
    tot = 0.0
    for h in itertools.product(HEL_F, HEL_F, HEL_W, HEL_W, HEL_V):
        M = sum(sum(v) for v in uux_wpwma_amplitudes(P, h, par).values())
        tot = tot + colour.colour_sum([M], [_DELTA3])
    return tot / 36.0


# --------------------------------------------------------------------------
# n gluons: colour-ordered Berends-Giele recursion + brute-force colour matrix
# --------------------------------------------------------------------------
_SQ2 = np.sqrt(2.0)


def _v3_ordered(J1, k1, J2, k2, g):
    """Colour-ordered three-gluon vertex with legs (1, 2, X) in cyclic order,
    all momenta outgoing, legs 1 and 2 contracted; returns the vector of X.

    V3 = (i g / sqrt2) [ g^{nu rho}(k1-k2)^mu + g^{rho mu}(k2-kX)^nu + g^{mu nu}(kX-k1)^rho ].
    """
    kX = -(k1 + k2)
    return (1j * g / _SQ2) * (mdot(J1, J2)[..., None] * (k1 - k2)
                               + J2 * mdot(k2 - kX, J1)[..., None]
                               + J1 * mdot(kX - k1, J2)[..., None])


def _v4_ordered(J1, J2, J3, g):
    """Colour-ordered four-gluon vertex, legs (1,2,3,X) in cyclic order:
    i g^2 g^{13} g^{2X} - (i g^2/2)(g^{12} g^{3X} + g^{1X} g^{23})."""
    return (1j * g * g) * (mdot(J1, J3)[..., None] * J2
                          - 0.5 * (mdot(J1, J2)[..., None] * J3 + mdot(J2, J3)[..., None] * J1))


def gluon_partial_amplitudes(K, E, g):
    """All colour-ordered amplitudes A(1, sigma_2..sigma_n) for one helicity.

    K: [n, ..., 4] outgoing momenta (incoming legs carry -p); E: [n, ..., 4]
    external wavefunctions.  Leg 0 is the root; the recursion runs over
    ordered tuples of the other legs and every ordered tuple's current is
    built from its consecutive splittings (Berends-Giele).  Returns
    (orders, A[len(orders), ...]) with A the colour-ordered "i M".
    """
    n = K.shape[0]
    cur = {}
    mom = {}

    def current(S):
        if S in cur:
            return cur[S]
        if len(S) == 1:
            cur[S] = E[S[0]]
            mom[S] = K[S[0]]
            return cur[S]
        amp = amputated(S)
        P = mom[S]
        cur[S] = -1j * amp / mdot(P, P)[..., None]
        return cur[S]

    def amputated(S):
        L = len(S)
        P = sum(K[s] for s in S)
        mom[S] = P
        out = 0.0
        for i in range(1, L):
            S1, S2 = S[:i], S[i:]
            J1, J2 = current(S1), current(S2)
            out = out + _v3_ordered(J1, mom[S1], J2, mom[S2], g)
        for i in range(1, L - 1):
            for j in range(i + 1, L):
                S1, S2, S3 = S[:i], S[i:j], S[j:]
                out = out + _v4_ordered(current(S1), current(S2), current(S3), g)
        return out

    orders = [(0,) + q for q in itertools.permutations(range(1, n))]
    A = []
    for o in orders:
        A.append(mdot(amputated(o[1:]), E[0]))
    return orders, np.stack(A, axis=0)


def gluons(P, par=SMParams(), per_helicity=False, eps_override=None, colour_matrix=None, n_in=2):
    """g g > g ... g: sum over all helicities of sum_{sigma,tau} A_sigma C A_tau^*.

    Full amplitude: i M = sum_sigma Tr(T^{a1} T^{a_sigma2} ...) A(1, sigma),
    T^a = sqrt2 t^a, so the colour sum is A^T C A^* with the brute-force C
    of oracle.colour.gluon_trace_matrix.  Averaged over 4 * 8 * 8.
    """
    N, n, _ = P.shape
    g = par.gs
    if colour_matrix is None:
        orders, C = colour.gluon_trace_matrix(n)
    else:
        orders, C = colour_matrix
    K = np.stack([(-P[:, k] if k < n_in else P[:, k]) for k in range(n)], axis=0)
    tot = 0.0
    ph = {}
    for h in itertools.product(HEL_V, repeat=n):
        E = []
        for k in range(n):
            eps = polarisation(P[:, k], h[k])
            E.append(eps if k < n_in else eps.conj())
        if eps_override:
            for leg, vec in eps_override.items():
                E[leg] = vec.astype(complex)
        E = np.stack(E, axis=0)
        o2, A = gluon_partial_amplitudes(K, E, g)
        assert o2 == orders
        m2 = np.real(np.einsum("sn,st,tn->n", A, C, A.conj()))
        ph[h] = m2
        tot = tot + m2
    avg = tot / (4.0 * 64.0)
    return (avg, ph) if per_helicity else avg


PROCESSES = {
    "u u~ > e+ e-": uux_epem,
    "u d~ > e+ ve": udx_epve,
    "u d~ > e+ ve g": udx_epveg,
    "u d~ > w+ g g": udx_wpgg,
    "u u~ > z g g": uux_zgg,
    "u s > d c h g": us_dchg,
    "u u~ > g g": uux_gg,
    "u d~ > e+ ve g g": udx_epvegg,
    "g g > t t~": gg_ttx,
    "g g > t t~ > b e+ ve b~ e- ve~": gg_ttx_dilep,
    "u s > d c h h": us_dchh,
    "u u > u u": uu_uu,
    "u u~ > z z": uux_zz,
    "u u~ > z h": uux_zh,
    "u d~ > w+ h": udx_wph,
    "u d~ > w+ g": udx_wpg,
    "u u~ > z g": uux_zg,
    "u u~ > z a": uux_za,
    "u u~ > a a": uux_aa,
    "u g > w+ d": ug_wpd,
    "u u~ > z z g": uux_zzg,
    "u u~ > z h g": uux_zhg,
    "u d~ > w+ h g": udx_wphg,
    "u d~ > w+ a": udx_wpa,
    "u d~ > w+ z g": udx_wpzg,
    "u u~ > w+ w- g": uux_wpwmg,
    "g g > w+ d u~": gg_wpdux,
    "g g > z u u~": gg_zuux,
    "u u~ > w+ w- a": uux_wpwma,
    "g g > t t~ h": gg_ttxh,
    "u u~ > t t~": uux_ttx,
    "u u~ > t t~ g": uux_ttxg,
    "u s > d c h": us_dch,
    "u s > d c h h h": us_dchhh,
    "u d > u d h": ud_udh,
    "u d > u d h h": ud_udhh,
    "u d > u d h h h": ud_udhhh,
    "u u > u u h": uu_uuh_n,
    "u u > u u h h": uu_uuhh,
    "u u > u u h h h": uu_uuhhh,
    "u d~ > w+ g g g": udx_wpggg,
    "u u~ > z g g g": uux_zggg,
    "g g > t t~ h g": gg_ttxhg,
    "g g > t t~ g g": gg_ttxgg,
    "u s > d c h g g": us_dchgg,
    "u u~ > z z g g": uux_zzgg,
    "u d~ > w+ h g g": udx_wphgg,
    "u d~ > w+ h g g g": udx_wphggg,
    "u u~ > w+ w- g g": uux_wpwmgg,
    "u d~ > w+ z g g": udx_wpzgg,
    "g g > t t~ g": gg_ttxg,
    "h h > h h": hh_hh,
    "u u~ > w+ w-": uux_wpwm,
    "u d~ > w+ z": udx_wpz,
    "g g > g g": gluons,
    "g g > g g g": gluons,
    "g g > g g g g": gluons,
}


def me(process, P, par=SMParams()):
    """|M|^2_avg for a process name of PROCESSES."""
    return PROCESSES[process](P, par=par)
