"""CUDA code generation for a compiled Program (the MG2CUDA role, Sect. 5).

For each process the generator writes one translation unit holding a
straight-line per-event evaluator templated on the amplitude precision R
(double: FP64 path; float: mixed path) and the launch wrappers the runtime
dispatches to.  Per event it emits, in order:

  1. the momenta (FP64) read from structure-of-arrays memory,
  2. every internal line's momentum and propagator denominator, once per
     event (FP64; the mixed path converts the reciprocal to complex FP32),
  3. the external wavefunctions for every helicity some live amplitude needs,
  4. every sub-current variant once (helicity recycling: shared by all
     diagrams and helicities that use it),
  5. the diagram amplitudes accumulated into colour components
     J_h,k = sum_d c_dk A_d (exact coefficients folded into literals),
  6. the colour sum |M_h|^2 = (J^T C J)/den with the integer matrix in the
     code, the helicity sum and the initial-state average.

Programs longer than HEL_LOOP_FLOPS (V + 3 jets, t t~ g, t t~ H g, W+ W- gamma) are emitted in the
helicity-loop form instead: one copy of steps 3-6 inside a loop over the live
helicity combinations, read from a table at run time (no recycling across
helicities, but a program n_live times shorter to compile and to hold).
Internal lines that carry the same external legs and particle share one
momentum and denominator.  All-gluon processes use the colour-ordered block
kernel (gluon_process.cu) instead.
"""
from fractions import Fraction

from .model import COMPLEX_COUPLINGS, PARTICLES, couplings
from .program import _ext_chirality, _is_column, _PAIRINGS

_TAG = {frozenset("u"): "me::kUp", frozenset("l"): "me::kLo", frozenset("ul"): "me::kAll"}


def _tag(h):
    return _TAG[frozenset(h)]


def _flip(h):
    return frozenset({"u": "l", "l": "u"}[x] for x in h)


def _hname(h):
    return {-1: "m", 0: "z", 1: "p", "r": "r"}[h]


# the variant of every node in the helicity-loop form: helicities known at run time only
RT = ("rt",)

# straight-line programs above this many FP32 flops per event are emitted in the helicity-loop form
# (g g > t t~ g, 94k: 2.3 times faster in the loop form; u u~ > w+ w- a, 73k: 3 % faster)
HEL_LOOP_FLOPS = 50000


def _vname(nid, var):
    if var == RT:
        return f"w{nid}"
    return f"w{nid}_" + "".join(_hname(h) for h in var) if var else f"w{nid}"


def hel_codes(prog):
    """Live helicity combinations packed 2 bits per leg (h + 1), leg 0 in the lowest bits."""
    assert prog.n_ext <= 16
    return [sum((h + 1) << (2 * k) for k, h in enumerate(hs)) for hs in prog.live]


def _ident(name):
    """C identifier for a coupling name (e.g. GA_e- -> GA_em)."""
    return name.replace("-", "m").replace("+", "p").replace("~", "x").replace(".", "_")


def _lit(x):
    """A floating literal typed as R."""
    v = float(x)
    return f"R({v!r})"


class _Emitter:
    def __init__(self, prog, tag, mode="fp64", hel_loop=False, interleave=False):
        self.p = prog
        self.tag = tag
        self.hel_loop = hel_loop  # one copy of the program in a loop over the live helicities
        self.interleave = interleave  # straight-line form: each amplitude right after its new sub-currents
        self.mode = mode          # "fp64": FP64 momenta and amplitudes; "mixed": double-float momenta, FP32
        self.lines = []
        self.flops32 = 0      # amplitude-precision flops per event
        self.flops64 = 0      # FP64 flops per event (momenta, invariants)
        self.cpl_names = set()
        self.mx_masses = {}       # mixed path: mass parameter -> width parameter of its resonant lines
        self.half = {}            # spinor variable -> set of halves ("u", "l") that can be non-zero
        self.pv = set()           # massless external vectors carried as me::PV (zero time, real z component)

    def emit(self, s):
        self.lines.append(s)

    def cpl(self, name):
        assert name not in COMPLEX_COUPLINGS, name
        self.cpl_names.add(name)
        return f"c_{_ident(name)}"

    def cplx(self, name):
        """A coupling of COMPLEX_COUPLINGS as a cx<R> expression (parameters name.re, name.im)."""
        self.cpl_names.add(name + ".re")
        self.cpl_names.add(name + ".im")
        return f"me::mk((R)c_{_ident(name)}_re, (R)c_{_ident(name)}_im)"

    def gmul(self, name, expr):
        """coupling * expr, a complex product for the couplings of COMPLEX_COUPLINGS."""
        if name in COMPLEX_COUPLINGS:
            self.flops32 += 4
            return f"({self.cplx(name)} * ({expr}))"
        return f"((R){self.cpl(name)} * ({expr}))"

    def ffs_args(self, v, scalar):
        """Coupling arguments of an FFS vertex and its scalar operand: a complex (gL = gR) coupling is
        moved onto the scalar (S g (P_L + P_R) = (g S) (P_L + P_R))."""
        gl, gr = v.couplings
        if gl in COMPLEX_COUPLINGS or gr in COMPLEX_COUPLINGS:
            assert gl == gr, "complex FFS couplings need gL = gR"
            return "(R)1, (R)1, true, true", self.gmul(gl, scalar)
        has_l, has_r = gl != "ZERO", gr != "ZERO"
        return (f"(R){self.cpl(gl) if has_l else '0.0'}, (R){self.cpl(gr) if has_r else '0.0'}, "
                f"{str(has_l).lower()}, {str(has_r).lower()}"), scalar

    # ------------------------------------------------------------------
    def generate(self):
        p = self.p
        n = p.n_ext
        E = self.emit
        nodes = p.nodes
        mixed = self.mode == "mixed"
        E("  // momenta: " + ("double-float (hi, lo) pairs" if mixed else "FP64"))
        for k in range(n):
            E(f"  const {'me::df' if mixed else 'double'}* p{k} = pm[{k}];")
        used_nodes = sorted(p.node_variants)
        E("  // external momenta in amplitude precision: r = physical, k = flowing into the vertex")
        for nid in used_nodes:
            nd = nodes[nid]
            if nd.external:
                k = nd.leg
                E(f"  const me::P4<R> r{nid} = {'me::p4f' if mixed else 'me::p4<R>'}(p{k});")
                if p.legs[k].incoming:
                    E(f"  const me::P4<R> k{nid} = r{nid};")
                else:
                    E(f"  const me::P4<R> k{nid} = me::neg(r{nid});")
        E("  // internal lines: momentum (into the parent vertex) and reciprocal propagator denominator.")
        if mixed:
            E("  // Massive (resonant) lines form q^2 - m^2 in double-float arithmetic from the double-float")
            E("  // momenta (no FP64 instructions); massless lines use FP32.")
        else:
            E("  // Massive (resonant) lines form q^2 - m^2 in FP64 from the FP64 momenta.")
        # lines of different diagrams that carry the same external legs and propagate the same
        # particle share one momentum and one denominator (the first such line's)
        line_of = {}
        for nid in used_nodes:
            nd = nodes[nid]
            if nd.external:
                continue
            kids = nd.children
            part = PARTICLES[nd.ptype]
            key = (frozenset(nd.legs), part.mass, part.width)
            if key in line_of:
                first = line_of[key]
                E(f"  const me::P4<R> k{nid} = k{first};")
                E(f"  const {'R' if part.massless else 'me::cx<R>'} inv{nid} = inv{first};")
                continue
            line_of[key] = nid
            if not (mixed and not part.massless):
                E(f"  const me::P4<R> k{nid} = " + " + ".join(f"k{c}" for c in kids) + ";")
                self.flops32 += 4 * (len(kids) - 1)
            if part.massless:
                E(f"  const R inv{nid} = R(1) / me::msq(k{nid});  // real: massless line")
                self.flops32 += 8
            else:
                m = self.cpl(part.mass)
                w = self.cpl(part.width) if part.width != "0" else None
                legs = sorted(nd.legs)
                terms = []
                for l in legs:
                    sgn = "+" if p.legs[l].incoming else "-"
                    terms.append((sgn, l))
                comps = []
                for mu in range(4):
                    e = ""
                    for j, (sgn, l) in enumerate(terms):
                        if j == 0:
                            e += ("" if sgn == "+" else "-") + f"p{l}[{mu}]"
                        else:
                            e += f" {sgn} p{l}[{mu}]"
                    comps.append(e)
                wexpr = f"{m} * {w}" if w else "0.0"
                if mixed:
                    dcomps = []
                    for mu in range(4):
                        e = ""
                        for j, (sgn, l) in enumerate(terms):
                            if j == 0:
                                e += ("" if sgn == "+" else "-") + f"p{l}[{mu}]"
                            else:
                                e += f" {sgn} p{l}[{mu}]"
                        dcomps.append(e)
                    E(f"  const me::df Q{nid}[4] = {{{', '.join(dcomps)}}};")
                    # the line's FP32 momentum is the rounding of its double-float sum: FP32 sums of the
                    # rounded external momenta lose the digits that cancel between incoming and outgoing
                    # legs, and near-collinear decay products turn that loss into errors of 1e-3 in |M|^2
                    E(f"  const me::P4<R> k{nid} = me::p4f(Q{nid});")
                    self.flops32 += 4
                    E(f"  const me::df q2_{nid} = ((me::sqr(Q{nid}[0]) - me::sqr(Q{nid}[1])) - me::sqr(Q{nid}[2])) - "
                      f"me::sqr(Q{nid}[3]);")
                    # m^2 (double-float) and m Gamma (FP32) come converted from the host (ParamsMx)
                    mname = _ident(part.mass)
                    self.mx_masses[mname] = _ident(part.width) if w else None
                    E(f"  const me::cx<R> inv{nid} = inv_den_f(me::to_float(q2_{nid} - prm.sq_{mname}), prm.mw_{mname});")
                    self.flops32 += 20 * (len(legs) - 1) * 4 + 4 * 8 + 3 * 20 + 20
                else:
                    E(f"  const double Q{nid}[4] = {{{', '.join(comps)}}};")
                    E(f"  const double q2_{nid} = Q{nid}[0] * Q{nid}[0] - Q{nid}[1] * Q{nid}[1] - Q{nid}[2] * Q{nid}[2] - "
                      f"Q{nid}[3] * Q{nid}[3];")
                    E(f"  const me::cx<R> inv{nid} = inv_den<R>(q2_{nid} - {m} * {m}, {wexpr});")
                    self.flops64 += 4 * (len(legs) - 1) + 7 + 3
        # Wavefunctions and sub-currents are emitted on demand, helicity by helicity: each
        # helicity's amplitudes are preceded by the variants they use that are not emitted yet,
        # and followed by its colour sum, so a variant lives only from its first to its last use
        # (shorter live ranges, fewer registers held across the program).
        emitted = set()

        def need(nid, var):
            if (nid, var) in emitted:
                return
            nd = nodes[nid]
            if not nd.external:
                for c in nd.children:
                    need(c, self.child_vars(nid, var, c))
            self.node_code(nid, var)
            emitted.add((nid, var))

        K = p.n_colour
        C = p.cmat_num
        if self.hel_loop:
            self._hel_loop_body(need, emitted)
            return
        E("  // per helicity: the wavefunctions and sub-currents it needs first, its diagram amplitudes")
        E("  // into colour components, then its colour sum (J^T C J)/den; helicity sum, average")
        E("  R tot = R(0);")
        for hi, terms in enumerate(p.amp_terms):
            if self.interleave:
                for k in range(K):
                    E(f"  me::cx<R> J{hi}_{k} = me::mk(R(0), R(0));")
                for aid, chvars in terms:
                    for c, cv in zip(p.amps[aid].children, chvars):
                        need(c, cv)
                    self.amp_code(aid, chvars, hi)
            else:
                for aid, chvars in terms:
                    for c, cv in zip(p.amps[aid].children, chvars):
                        need(c, cv)
                for k in range(K):
                    E(f"  me::cx<R> J{hi}_{k} = me::mk(R(0), R(0));")
                for aid, chvars in terms:
                    self.amp_code(aid, chvars, hi)
            E("  {")
            E("    R s = R(0);")
            for k in range(K):
                if C[k][k]:
                    E(f"    s += {_lit(C[k][k])} * me::abs2(J{hi}_{k});")
                    self.flops32 += 4
                for l in range(k + 1, K):
                    if C[k][l]:
                        E(f"    s += {_lit(2 * C[k][l])} * (J{hi}_{k}.re * J{hi}_{l}.re + J{hi}_{k}.im * J{hi}_{l}.im);")
                        self.flops32 += 5
            E("    tot += s;")
            E("  }")
        if self.mode == "mixed":
            E(f"  return tot * {float(p.average / p.cmat_den)!r}f;")
        else:
            E(f"  return (double)tot * {float(p.average / p.cmat_den)!r};")

    def _colour_sum(self, hi):
        p = self.p
        E = self.emit
        C = p.cmat_num
        E("  {")
        E("    R s = R(0);")
        for k in range(p.n_colour):
            if C[k][k]:
                E(f"    s += {_lit(C[k][k])} * me::abs2(J{hi}_{k});")
                self.flops32 += 4
            for l in range(k + 1, p.n_colour):
                if C[k][l]:
                    E(f"    s += {_lit(2 * C[k][l])} * (J{hi}_{k}.re * J{hi}_{l}.re + J{hi}_{k}.im * J{hi}_{l}.im);")
                    self.flops32 += 5
        E("    tot += s;")
        E("  }")

    def fermion_groups(self):
        """Live combinations grouped by the helicities of the massless external fermions: one loop
        body per group, with those helicities (so the spinor halves) fixed at compile time."""
        p = self.p
        fl = [k for k, leg in enumerate(p.legs) if PARTICLES[leg.particle].is_fermion
              and PARTICLES[leg.particle].massless]
        groups = {}
        for i, hs in enumerate(p.live):
            groups.setdefault(tuple(hs[k] for k in fl), []).append(i)
        return fl, list(groups.items())

    def _hel_loop_body(self, need, emitted):
        """The helicity-loop form: one copy of every wavefunction, sub-current and amplitude per group of
        live combinations that share the massless fermions' helicities (fixed in the code, so the zero
        spinor halves stay known), with the other helicities read from the group's table (hel_code_g)
        at run time, in a loop over the group.  No helicity recycling across the loop, so more flops
        per helicity, but the program is many times shorter (the paper's remedy for amplitude functions
        too long to compile or to keep in registers, Sect. 5.3)."""
        p = self.p
        E = self.emit
        fl, groups = self.fermion_groups()
        E("  R tot = R(0);")
        f0 = self.flops32
        total = 0
        for gi, (key, idxs) in enumerate(groups):
            fixed = dict(zip(fl, key))
            E(f"  {{  // massless fermion helicities {key}: the other legs' from hel_code_g{gi}, 2 bits per leg (h + 1)")
            E("#pragma unroll 1")
            E(f"  for (int ih = 0; ih < {len(idxs)}; ++ih) {{")
            E(f"  const uint32_t hc = hel_code_g{gi}(ih);")
            for k in range(p.n_ext):
                if k not in fixed:
                    E(f"  const int hl{k} = (int)((hc >> {2 * k}) & 3u) - 1;")
            emitted.clear()

            def var_of(nid):
                return tuple(fixed.get(l, "r") for l in sorted(p.nodes[nid].legs))
            aids = sorted({aid for hi in idxs for aid, _ in p.amp_terms[hi]})
            g0 = self.flops32
            for k in range(p.n_colour):
                E(f"  me::cx<R> J_{k} = me::mk(R(0), R(0));")
            # each amplitude right after the sub-currents it needs first: a sub-current lives from
            # its first to its last use instead of across the whole body
            for aid in aids:
                for c in p.amps[aid].children:
                    need(c, var_of(c))
                self.amp_code(aid, [var_of(c) for c in p.amps[aid].children], "")
            self._colour_sum("")
            E("  }")
            E("  }")
            total += (self.flops32 - g0) * len(idxs)
            self.flops32 = g0
        self.flops32 = f0 + total
        if self.mode == "mixed":
            E(f"  return tot * {float(p.average / p.cmat_den)!r}f;")
        else:
            E(f"  return (double)tot * {float(p.average / p.cmat_den)!r};")

    # ------------------------------------------------------------------
    def child_vars(self, nid, var, child):
        if var == RT:
            return RT
        nd = self.p.nodes[nid]
        legs = sorted(nd.legs)
        hmap = dict(zip(legs, var))
        cl = sorted(self.p.nodes[child].legs)
        return tuple(hmap[l] for l in cl)

    def ext_code(self, nid, var):
        p = self.p
        nd = p.nodes[nid]
        leg = p.legs[nd.leg]
        part = PARTICLES[leg.particle]
        rt = var == RT or var[0] == "r"
        h = f"hl{nd.leg}" if rt else var[0]
        name = _vname(nid, var)
        inc = "true" if leg.incoming else "false"
        if part.is_fermion and not part.massless:
            m = self.cpl(part.mass)
            fn = "ext_column_massive" if _is_column(nd.ptype) else "ext_row_massive"
            self.emit(f"  const me::W4<R> {name} = me::{fn}<R>(r{nid}, {h}, {inc}, (R){m});")
            self.half[name] = frozenset("ul")
            self.flops32 += 40
        elif part.is_fermion:
            if rt:  # the chirality is known at run time only: both halves
                up, lo = frozenset("ul"), frozenset("ul")
            else:
                chi = _ext_chirality(leg, h)
                up, lo = frozenset("u" if chi == "L" else "l"), frozenset("l" if chi == "L" else "u")
            if _is_column(nd.ptype):
                self.emit(f"  const me::W4<R> {name} = me::ext_column_massless<R>(r{nid}, {h}, {inc});")
                self.half[name] = up
            else:
                self.emit(f"  const me::W4<R> {name} = me::ext_row_massless<R>(r{nid}, {h}, {inc});")
                self.half[name] = lo
            self.flops32 += 12
        elif part.is_vector and part.massless:
            self.emit(f"  const me::PV<R> {name} = me::ext_pol<R>(r{nid}, {h}, {inc});")
            self.pv.add(name)
            self.flops32 += 25
        elif part.is_vector:
            self.emit(f"  const me::W4<R> {name} = me::ext_vector<R>(r{nid}, {h}, {inc}, (R){self.cpl(part.mass)});")
            self.flops32 += 25
        else:
            self.emit(f"  const me::cx<R> {name} = me::mk(R(1), R(0));")

    def node_code(self, nid, var):
        p = self.p
        nd = p.nodes[nid]
        if nd.external:
            self.ext_code(nid, var)
            return
        v = nd.vertex
        kids = [(c, s, _vname(c, self.child_vars(nid, var, c))) for c, s in zip(nd.children, nd.slots)]
        name = _vname(nid, var)
        part = PARTICLES[nd.ptype]
        E = self.emit
        if v.kind == "FFV":
            gl, gr = v.couplings
            has_l, has_r = gl != "ZERO", gr != "ZERO"
            gls = self.cpl(gl) if has_l else "0.0"
            grs = self.cpl(gr) if has_r else "0.0"
            nch = int(has_l) + int(has_r)
            cargs = f"(R){gls}, (R){grs}, {str(has_l).lower()}, {str(has_r).lower()}"
            if part.is_fermion:
                fk = [k for k in kids if k[1] in (0, 1)][0]
                vk = [k for k in kids if k[1] == 2][0]
                m = "R(0)" if part.massless else f"(R){self.cpl(part.mass)}"
                hin = self.half[fk[2]]
                if _is_column(nd.ptype):
                    hx = set()
                    if "u" in hin and has_l:
                        hx.add("l")
                    if "l" in hin and has_r:
                        hx.add("u")
                    hx = frozenset(hx)
                    E(f"  const me::W4<R> {name} = me::prop_col<R, {_tag(hx)}>(me::ffv_col<R, {_tag(hin)}>("
                      f"{fk[2]}, {vk[2]}, {cargs}), k{nid}, {m}, inv{nid});")
                else:
                    hx = set()
                    if "l" in hin and has_l:
                        hx.add("u")
                    if "u" in hin and has_r:
                        hx.add("l")
                    hx = frozenset(hx)
                    E(f"  const me::W4<R> {name} = me::prop_row<R, {_tag(hx)}>(me::ffv_row<R, {_tag(hin)}>("
                      f"{fk[2]}, {vk[2]}, {cargs}), me::neg(k{nid}), {m}, inv{nid});")
                self.half[name] = _flip(hx) if part.massless else frozenset("ul")
                # per non-zero half: vertex 40 (sigma matrix 8, two components of 16; 28 with a PV
                # vector); propagator 24 with the real reciprocal of a massless line, 32 with a complex
                # one, plus the mass term
                vtx = 28 if vk[2] in self.pv else 40
                self.flops32 += (vtx + (24 if part.massless else 32)) * len(hx) + 2 + (32 if not part.massless else 0)
            else:
                rk = [k for k in kids if k[1] == 0][0]
                ck = [k for k in kids if k[1] == 1][0]
                massive = not part.massless and nid not in p.conserved
                mc2 = f"inv_mc2_{part.mass}" if massive else "me::mk(R(0), R(0))"
                if massive:
                    self.cpl(part.mass)
                    self.cpl(part.width)
                hr, hc = self.half[rk[2]], self.half[ck[2]]
                E(f"  const me::W4<R> {name} = me::prop_vec<R>(me::ffv_current<R, {_tag(hr)}, {_tag(hc)}>("
                  f"{rk[2]}, {ck[2]}, {cargs}), k{nid}, inv{nid}, {str(massive).lower()}, {mc2});")
                nterm = int(has_l and "l" in hr and "u" in hc) + int(has_r and "u" in hr and "l" in hc)
                self.flops32 += 48 * nterm + (60 if massive else 8)
        elif v.kind == "FFS":
            gl, gr = v.couplings
            has_l, has_r = gl != "ZERO", gr != "ZERO"
            if part.is_fermion:
                fk = [k for k in kids if k[1] in (0, 1)][0]
                sk = [k for k in kids if k[1] == 2][0]
                cargs, sval = self.ffs_args(v, sk[2])
                m = "R(0)" if part.massless else f"(R){self.cpl(part.mass)}"
                hin = self.half[fk[2]]
                # S (gL P_L + gR P_R) keeps the halves: gL acts on the upper, gR on the lower one
                hx = set()
                if "u" in hin and has_l:
                    hx.add("u")
                if "l" in hin and has_r:
                    hx.add("l")
                hx = frozenset(hx)
                if _is_column(nd.ptype):
                    E(f"  const me::W4<R> {name} = me::prop_col<R, {_tag(hx)}>(me::ffs_col<R, {_tag(hin)}>("
                      f"{fk[2]}, {sval}, {cargs}), k{nid}, {m}, inv{nid});")
                else:
                    E(f"  const me::W4<R> {name} = me::prop_row<R, {_tag(hx)}>(me::ffs_row<R, {_tag(hin)}>("
                      f"{fk[2]}, {sval}, {cargs}), me::neg(k{nid}), {m}, inv{nid});")
                self.half[name] = _flip(hx) if part.massless else frozenset("ul")
                self.flops32 += (14 + 24 + (32 if not part.massless else 0)) * len(hx) + 2
            else:
                rk = [k for k in kids if k[1] == 0][0]
                ck = [k for k in kids if k[1] == 1][0]
                hr, hc = self.half[rk[2]], self.half[ck[2]]
                cargs, one = self.ffs_args(v, "R(1)")
                E(f"  const me::cx<R> {name} = {one} * me::ffs_scalar<R, {_tag(hr)}, {_tag(hc)}>({rk[2]}, {ck[2]}, "
                  f"{cargs}) * inv{nid};")
                self.flops32 += 34
        elif v.kind == "VVV":
            g = self.cpl(v.couplings[0])
            # inputs in cyclic order after the output slot: the antisymmetric Lorentz structure
            # then equals the vertex's (slot 0, 1, 2) form
            by_slot = {k[1]: k for k in kids}
            o = nd.out_slot
            a, b = by_slot[(o + 1) % 3], by_slot[(o + 2) % 3]
            # a massive line keeps the k k / m^2 term unless its current is conserved
            massive = not part.massless and nid not in p.conserved
            mc2 = f"inv_mc2_{part.mass}" if massive else "me::mk(R(0), R(0))"
            if massive:
                self.cpl(part.mass)
                self.cpl(part.width)
            E(f"  const me::W4<R> {name} = me::prop_vec<R>(me::vvv_current<R>({a[2]}, k{a[0]}, {b[2]}, k{b[0]}, "
              f"(R){g}), k{nid}, inv{nid}, {str(massive).lower()}, {mc2});")
            self.flops32 += self._vvv_current_flops(a[2], b[2]) + (60 if massive else 8)
        elif v.kind == "VVVV" and v.colour != "ff":
            # electroweak quartic: C [T_a + T_b - 2 T_pair], T_j the current of pairing j
            g = self.cpl(v.couplings[0])
            slot = {s: nm for _, s, nm in kids}
            o = nd.out_slot
            t = [self._v4_term(o, list(_PAIRINGS[j]), slot) for j in range(3)]
            ta, tb = [t[j] for j in range(3) if j != v.pair]
            massive = not part.massless and nid not in p.conserved
            mc2 = f"inv_mc2_{part.mass}" if massive else "me::mk(R(0), R(0))"
            if massive:
                self.cpl(part.mass)
                self.cpl(part.width)
            E(f"  const me::W4<R> {name} = me::prop_vec<R>(me::w4_quartic<R>({ta}, {tb}, {t[v.pair]}, (R){g}), "
              f"k{nid}, inv{nid}, {str(massive).lower()}, {mc2});")
            self.flops32 += 3 * 54 + 40 + (60 if massive else 8)
        elif v.kind == "VVVV":
            g = self.cpl(v.couplings[0])
            slot = {s: nm for _, s, nm in kids}
            o = nd.out_slot
            (x, y), (z, w) = _PAIRINGS[nd.struct]
            # L = g_xz g_yw - g_xw g_yz; current for the open slot o
            t1 = self._v4_term(o, [(x, z), (y, w)], slot)
            t2 = self._v4_term(o, [(x, w), (y, z)], slot)
            E(f"  const me::W4<R> {name} = me::prop_vec<R>(me::w4_sub<R>({t1}, {t2}, (R){g}), k{nid}, inv{nid}, "
              f"false, me::mk(R(0), R(0)));")
            self.flops32 += 2 * 54 + 16 + 8
        elif v.kind in ("VVS", "VVSS"):
            vs = [k for k in kids if PARTICLES[v.fields[k[1]]].is_vector]
            ss = [k for k in kids if PARTICLES[v.fields[k[1]]].is_scalar]
            sprod = " * ".join(k[2] for k in ss) if ss else None
            if part.is_vector:
                s_expr = self.gmul(v.couplings[0], sprod)
                massive = not part.massless
                mc2 = f"inv_mc2_{part.mass}" if massive else "me::mk(R(0), R(0))"
                if massive:
                    self.cpl(part.mass)
                    self.cpl(part.width)
                E(f"  const me::W4<R> {name} = me::prop_vec<R>(me::w4_scale<R>({vs[0][2]}, {s_expr}), k{nid}, "
                  f"inv{nid}, {str(massive).lower()}, {mc2});")
                self.flops32 += 24 + (60 if massive else 8) + 6 * len(ss)
            else:
                d = f"me::mdot<R>({vs[0][2]}, {vs[1][2]})"
                extra = f" * {sprod}" if sprod else ""
                E(f"  const me::cx<R> {name} = {self.gmul(v.couplings[0], d)}{extra} * inv{nid};")
                self.flops32 += 30 + 12 + 6 * len(ss)
        elif v.kind in ("SSS", "SSSS"):
            prod = " * ".join(k[2] for k in kids)
            E(f"  const me::cx<R> {name} = {self.gmul(v.couplings[0], prod)} * inv{nid};")
            self.flops32 += 8 + 6 * len(kids)
        else:
            raise NotImplementedError(v.kind)

    def _vvv_current_flops(self, v1, v2):
        """vvv_current: 154 flops for two W4 vectors; a PV operand saves 30 (its zero time and real z
        components in V1.V2, in its momentum contraction and in the output combination), two save 51."""
        npv = int(v1 in self.pv) + int(v2 in self.pv)
        return 150 - (0, 30, 51)[npv]

    def _v4_term(self, o, pairs, slot):
        """Current of sum over pairs structure g_{ab} g_{cd} with slot o open."""
        (a, b), (c, d) = pairs
        if o in (a, b):
            partner = b if o == a else a
            return f"me::v4_term<R>({slot[partner]}, {slot[c]}, {slot[d]})"
        partner = d if o == c else c
        return f"me::v4_term<R>({slot[partner]}, {slot[a]}, {slot[b]})"

    def amp_code(self, aid, chvars, hi):
        p = self.p
        a = p.amps[aid]
        v = a.vertex
        kids = [(c, s, _vname(c, cv)) for c, s, cv in zip(a.children, a.slots, chvars)]
        slot = {s: nm for _, s, nm in kids}
        E = self.emit
        if v.kind == "FFV":
            gl, gr = v.couplings
            has_l, has_r = gl != "ZERO", gr != "ZERO"
            gls = self.cpl(gl) if has_l else "0.0"
            grs = self.cpl(gr) if has_r else "0.0"
            hr, hc = self.half[slot[0]], self.half[slot[1]]
            expr = (f"me::ffv_amp<R, {_tag(hr)}, {_tag(hc)}>({slot[0]}, {slot[1]}, {slot[2]}, (R){gls}, (R){grs}, "
                    f"{str(has_l).lower()}, {str(has_r).lower()})")
            nterm = int(has_l and "u" in hc and "l" in hr) + int(has_r and "l" in hc and "u" in hr)
            self.flops32 += (28 if slot[2] in self.pv else 40) * nterm + 16 * nterm
        elif v.kind == "FFS":
            hr, hc = self.half[slot[0]], self.half[slot[1]]
            cargs, sval = self.ffs_args(v, slot[2])
            expr = f"(me::ffs_scalar<R, {_tag(hr)}, {_tag(hc)}>({slot[0]}, {slot[1]}, {cargs}) * {sval})"
            self.flops32 += 34 + 6
        elif v.kind == "VVV":
            g = self.cpl(v.couplings[0])
            k0 = [c for c, s, _ in kids if s == 0][0]
            k1 = [c for c, s, _ in kids if s == 1][0]
            expr = f"me::vvv_amp<R>({slot[0]}, k{k0}, {slot[1]}, k{k1}, {slot[2]}, (R){g})"
            self.flops32 += self._vvv_current_flops(slot[0], slot[1]) + (18 if slot[2] in self.pv else 30)
        elif v.kind == "VVVV" and v.colour != "ff":
            g = self.cpl(v.couplings[0])
            prods = [f"me::mdot<R>({slot[x]}, {slot[y]}) * me::mdot<R>({slot[z]}, {slot[w]})"
                     for (x, y), (z, w) in _PAIRINGS]
            pa, pb = [prods[j] for j in range(3) if j != v.pair]
            expr = f"(R){g} * ({pa} + {pb} - R(2) * ({prods[v.pair]}))"
            self.flops32 += 6 * 30 + 3 * 6 + 12
        elif v.kind == "VVVV":
            g = self.cpl(v.couplings[0])
            (x, y), (z, w) = _PAIRINGS[a.struct]
            expr = (f"(R){g} * (me::mdot<R>({slot[x]}, {slot[z]}) * me::mdot<R>({slot[y]}, {slot[w]}) - "
                    f"me::mdot<R>({slot[x]}, {slot[w]}) * me::mdot<R>({slot[y]}, {slot[z]}))")
            self.flops32 += 4 * 30 + 16
        elif v.kind in ("VVS", "VVSS"):
            vs = [nm for _, s, nm in kids if PARTICLES[v.fields[s]].is_vector]
            ss = [nm for _, s, nm in kids if PARTICLES[v.fields[s]].is_scalar]
            expr = self.gmul(v.couplings[0], f"me::mdot<R>({vs[0]}, {vs[1]})") + "".join(f" * {s}" for s in ss)
            self.flops32 += 32 + 6 * len(ss)
        elif v.kind in ("SSS", "SSSS"):
            prod = " * ".join(slot[s] for s in range(len(v.fields)))
            expr = self.gmul(v.couplings[0], prod)
            self.flops32 += 2 + 6 * len(v.fields)
        else:
            raise NotImplementedError(v.kind)
        E(f"  {{ const me::cx<R> a = {expr};")
        for k in range(p.n_colour):
            c = p.coeffs.get((aid, k))
            if c is None or c.is_zero():
                continue
            cr, ci = float(c.re), float(c.im)
            if ci == 0:
                E(f"    J{hi}_{k}.re += {_lit(cr)} * a.re; J{hi}_{k}.im += {_lit(cr)} * a.im;")
                self.flops32 += 4
            elif cr == 0:
                E(f"    J{hi}_{k}.re -= {_lit(ci)} * a.im; J{hi}_{k}.im += {_lit(ci)} * a.re;")
                self.flops32 += 4
            else:
                E(f"    J{hi}_{k} = J{hi}_{k} + me::mk({_lit(cr)} * a.re - {_lit(ci)} * a.im, "
                  f"{_lit(cr)} * a.im + {_lit(ci)} * a.re);")
                self.flops32 += 8
        E("  }")


def process_symbol(name):
    out = []
    for ch in name:
        out.append(ch if ch.isalnum() else "_")
    return "p_" + "".join(out).strip("_")


def generate_source(prog, tag, hel_loop=None, interleave=False):
    """CUDA source for one process: the FP64 and mixed evaluators in a traits struct.

    hel_loop: True for the helicity-loop form, False for the straight-line form, None to take the
    loop form when the straight-line mixed program exceeds HEL_LOOP_FLOPS."""
    if hel_loop is None:
        probe = _Emitter(prog, tag, "mixed")
        probe.generate()
        hel_loop = probe.flops32 > HEL_LOOP_FLOPS
    em64 = _Emitter(prog, tag, "fp64", hel_loop, interleave)
    em64.generate()
    emmx = _Emitter(prog, tag, "mixed", hel_loop, interleave)
    emmx.generate()
    hel_fn = ""
    if hel_loop:
        codes = hel_codes(prog)
        _, groups = emmx.fermion_groups()
        for gi, (key, idxs) in enumerate(groups):
            cases = " ".join(f"case {i}: return {codes[c]}u;" for i, c in enumerate(idxs))
            hel_fn += f"""
  // live helicity combinations with massless fermion helicities {key}, 2 bits per leg (h + 1)
  static __host__ __device__ __forceinline__ uint32_t hel_code_g{gi}(int ih) {{
    switch (ih) {{ {cases} default: return 0u; }}
  }}
"""
    cpl = sorted(em64.cpl_names | emmx.cpl_names)
    masses_for_mc2 = sorted({n for n in cpl if n.startswith("M")})
    params = "\n".join(f"    double {_ident(n)};" for n in cpl) or "    double unused;"
    unpack = "\n".join(f"    const double c_{_ident(n)} = prm.{_ident(n)};" for n in cpl)
    mc2 = []
    for mname in masses_for_mc2:
        wname = "W" + mname[1:]
        if wname in cpl:
            mc2.append(f"    const me::cx<R> inv_mc2_{mname} = inv_den<R>(c_{mname} * c_{mname}, "
                       f"-c_{mname} * c_{wname});")
    mc2 = "\n".join(mc2)
    # mixed path: every parameter as FP32, and per mass m^2 (double-float), m Gamma and
    # 1/(m^2 - i m Gamma), converted once per launch on the host; in the kernel they are
    # constant-bank operands (no conversion, no register held across the point loop)
    mx_masses = sorted(set(masses_for_mc2) | set(emmx.mx_masses))
    mx_fields = [f"    float {_ident(n)};" for n in cpl]
    mx_init = [f"    q.{_ident(n)} = (float)p.{_ident(n)};" for n in cpl]
    for mname in mx_masses:
        wname = "W" + mname[1:]
        wexpr = f"p.{mname} * p.{wname}" if wname in cpl else "0.0"
        mx_fields += [f"    me::df sq_{mname};", f"    float mw_{mname};", f"    me::cx<float> imc2_{mname};"]
        mx_init += [f"    q.sq_{mname} = me::from_double(p.{mname} * p.{mname});",
                    f"    q.mw_{mname} = (float)({wexpr});",
                    f"    q.imc2_{mname} = inv_den<float>(p.{mname} * p.{mname}, -({wexpr}));"]
    if not mx_fields:
        mx_fields = ["    float unused;"]
    mx_fields = "\n".join(mx_fields)
    mx_init = "\n".join(mx_init)
    unpack_mx = "\n".join(f"    const float c_{_ident(n)} = prm.{_ident(n)};" for n in cpl)
    mc2_mx = "\n".join(f"    const me::cx<R> inv_mc2_{m} = prm.imc2_{m};" for m in masses_for_mc2
                        if ("W" + m[1:]) in cpl)
    body64 = "\n".join("  " + ln for ln in em64.lines)
    bodymx = "\n".join("  " + ln for ln in emmx.lines)
    n = prog.n_ext
    src = f"""// Generated by paper_1305_0708_gb300.compiler for: {prog.name}
// diagrams: {len(prog.amps)}, live helicities: {len(prog.live)} of {_ncomb(prog)}, colour basis: {prog.n_colour}
#include "process_common.cuh"

namespace me {{
namespace {tag} {{

struct Traits {{
  static constexpr int NEXT = {n};
  struct Params {{
{params}
  }};
  struct ParamsMx {{
{mx_fields}
  }};
  static ParamsMx mixed_params(const Params& p) {{
    ParamsMx q;
{mx_init}
    return q;
  }}
{hel_fn}
  // FP64 path: FP64 momenta, invariants and amplitudes
  static __host__ __device__ __forceinline__ double eval64(const double (&pm)[{n}][4], const Params& prm) {{
    using R = double;
{unpack}
{mc2}
{body64}
  }}

  // mixed path: double-float momenta and resonant invariants, FP32 amplitudes and result
  static __host__ __device__ __forceinline__ float evalmx(const me::df (&pm)[{n}][4], const ParamsMx& prm) {{
    using R = float;
{unpack_mx}
{mc2_mx}
{bodymx}
  }}
}};

}}  // namespace {tag}
}}  // namespace me

ME_DEFINE_PROCESS({tag}, {n}, {len(cpl) if cpl else 1})
"""
    info = {"flops_amp": emmx.flops32, "flops_fp64": em64.flops64 + em64.flops32, "params": cpl,
            "hel_loop": bool(hel_loop)}
    return src, info


def _ncomb(prog):
    n = 1
    for l in prog.legs:
        n *= len(l.hels)
    return n


def param_values(info, par):
    c = couplings(par)
    return [c[n] for n in info["params"]]
