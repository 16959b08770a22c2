"""Process compiler: diagrams -> straight-line helicity program + exact colour matrix.

compile_process(name) returns a Program holding
  * the external legs (particle, incoming, mass parameter, helicity states),
  * the live helicity combinations (structural zeros from massless chirality
    dropped, analytic zeros kept),
  * every sub-current ("node") with the helicity variants some live
    amplitude needs -- a wavefunction is computed once per variant of the
    legs it depends on, and shared by all diagrams and helicities using it,
  * every diagram amplitude with, per live helicity, its child variants,
  * the colour decomposition J_k = sum_d c_dk A_d with exact complex
    rational c_dk (phases of i from vertices and propagators and the
    fermion-permutation sign folded in), and
  * the exact colour matrix C_kl, stored as integers over a common
    denominator (Sect. 5.4 of the paper stores the decomposed colour matrix
    in constant memory; here it is folded into the code or a tensor-core
    operand).

Phases: every vertex and propagator factor i^n is tracked symbolically so the
device functions compute only real-coupling ("stripped") expressions.
"""
import itertools
import math
from dataclasses import dataclass, field
from fractions import Fraction

from . import colour as col
from .diagrams import generate, parse
from .model import PARTICLES

# own phase (power of i) of a current: vertex factor + propagator
_PROP_PHASE = {"F": 1, "V": 3, "S": 1}
_VERTEX_PHASE = {"FFV": 1, "FFS": 1, "VVV": 0, "VVVV": 3, "VVS": 1, "VVSS": 1, "SSS": 1, "SSSS": 1}


def _kind_of(ptype):
    p = PARTICLES[ptype]
    return "F" if p.is_fermion else ("V" if p.is_vector else "S")


def _is_column(ptype):
    """A fermion line bringing fermion number into its vertex (u-type spinor)."""
    return PARTICLES[ptype].is_fermion and PARTICLES[ptype].pdg > 0


def helicity_states(pname):
    p = PARTICLES[pname]
    if p.is_fermion:
        return (-1, 1)
    if p.is_vector:
        return (-1, 1) if p.massless else (-1, 0, 1)
    return (0,)


@dataclass
class Leg:
    particle: str
    incoming: bool
    mass: str
    hels: tuple
    colour: int


@dataclass
class Program:
    name: str
    legs: list
    nodes: list
    amps: list
    live: list                      # live helicity combos (tuples over legs)
    node_variants: dict             # node id -> sorted list of variant tuples (helicities of node.legs)
    amp_terms: list                 # per live combo: list of (amp id, [child variant tuples])
    coeffs: dict                    # (amp id, basis k) -> CQ (phase and sign folded)
    basis: list
    cmat_num: list                  # integer colour matrix C * den
    cmat_den: int
    average: Fraction               # 1/(spin states x colour states) of the initial legs
    phases: dict = field(default_factory=dict)
    conserved: set = field(default_factory=set)   # vector lines whose k k / m^2 term vanishes
    flops: dict = field(default_factory=dict)

    @property
    def n_ext(self):
        return len(self.legs)

    @property
    def n_colour(self):
        return len(self.basis)


# ---------------------------------------------------------------------------
# structural zeros: chirality of massless fermion lines
# ---------------------------------------------------------------------------
def _ext_chirality(leg, h):
    """Chirality (L/R) of the column spinor underlying a massless external fermion."""
    column = _is_column(leg.particle if leg.incoming else PARTICLES[leg.particle].anti)
    if column:
        left = (h == -1) if leg.incoming else (h == 1)     # u(p,h) incoming, v(p,h) outgoing
    else:
        left = (h == -1) if not leg.incoming else (h == 1)  # ubar outgoing, vbar incoming
    return "L" if left else "R"


def _ffv_allowed(vertex, coup_zero):
    gl, gr = vertex.couplings
    allowed = set()
    if not coup_zero(gl):
        allowed.add("L")
    if not coup_zero(gr):
        allowed.add("R")
    return allowed


def _chir_ok(chi, X):
    return chi == "M" or chi == X


class _Analysis:
    def __init__(self, proc, legs, nodes, amps):
        self.proc, self.legs, self.nodes, self.amps = proc, legs, nodes, amps
        self.cache = {}

    @staticmethod
    def coup_zero(name):
        return name == "ZERO"

    def node_state(self, nid, hmap):
        """None (structural zero), 'L'/'R'/'M' for fermions, True otherwise."""
        nd = self.nodes[nid]
        key = (nid, tuple(hmap[l] for l in sorted(nd.legs)))
        if key in self.cache:
            return self.cache[key]
        if nd.external:
            leg = self.legs[nd.leg]
            if PARTICLES[leg.particle].is_fermion:
                res = "M" if not PARTICLES[leg.particle].massless else _ext_chirality(leg, hmap[nd.leg])
            else:
                res = True
        else:
            ch = [self.node_state(c, hmap) for c in nd.children]
            if any(c is None for c in ch):
                res = None
            elif nd.vertex.kind == "FFS":
                # a scalar vertex flips chirality; no pruning through it (both chiralities kept)
                res = "M" if PARTICLES[nd.ptype].is_fermion else True
            elif nd.vertex.kind == "FFV":
                allowed = _ffv_allowed(nd.vertex, self.coup_zero)
                ferm = [c for c, s in zip(ch, nd.slots) if s in (0, 1)]
                if len(ferm) == 2:
                    res = True if any(_chir_ok(ferm[0], X) and _chir_ok(ferm[1], X) for X in allowed) else None
                else:
                    ok = [X for X in allowed if _chir_ok(ferm[0], X)]
                    if not ok:
                        res = None
                    elif PARTICLES[nd.ptype].massless and len(ok) == 1:
                        res = ok[0]
                    else:
                        res = "M"
            else:
                res = True
        self.cache[key] = res
        return res

    def amp_nonzero(self, a, hmap):
        ch = [self.node_state(c, hmap) for c in a.children]
        if any(c is None for c in ch):
            return False
        if a.vertex.kind == "FFV":
            allowed = _ffv_allowed(a.vertex, self.coup_zero)
            ferm = [c for c, s in zip(ch, a.slots) if s in (0, 1)]
            return any(_chir_ok(ferm[0], X) and _chir_ok(ferm[1], X) for X in allowed)
        return True


# ---------------------------------------------------------------------------
# colour and fermion sign
# ---------------------------------------------------------------------------
def _label(nodes, legs, nid):
    nd = nodes[nid]
    if nd.external:
        c = legs[nd.leg].colour
        return ("q", nd.leg) if abs(c) == 3 else (("g", nd.leg) if c == 8 else None)
    p = PARTICLES[nd.ptype]
    return ("i", nid) if abs(p.colour) == 3 else (("a", nid) if p.colour == 8 else None)


_PAIRINGS = [((0, 1), (2, 3)), ((0, 2), (1, 3)), ((0, 3), (1, 2))]


def _vertex_colour(vertex, slot_labels, struct, elabel):
    c = vertex.colour
    if c == "none":
        return {(): col.CQ(1)}
    if c == "delta":
        return col.delta(slot_labels[0], slot_labels[1])
    if c == "T":
        return col.t_string(slot_labels[0], [slot_labels[2]], slot_labels[1])
    if c == "f":
        return col.f_abc(*slot_labels[:3])
    if c == "ff":
        (x, y), (z, w) = _PAIRINGS[struct]
        L = slot_labels
        return col.mul(col.f_abc(L[x], L[y], elabel), col.f_abc(L[z], L[w], elabel))
    raise ValueError(c)


def _node_colour(nodes, legs, nid, cache, internal):
    if nid in cache:
        return cache[nid]
    nd = nodes[nid]
    if nd.external:
        res = {(): col.CQ(1)}
    else:
        labels = [None] * len(nd.vertex.fields)
        for c, s in zip(nd.children, nd.slots):
            labels[s] = _label(nodes, legs, c)
        labels[nd.out_slot] = _label(nodes, legs, nid)
        elabel = ("e", nid)
        internal.add(elabel)
        res = _vertex_colour(nd.vertex, labels, nd.struct, elabel)
        for c in nd.children:
            res = col.mul(res, _node_colour(nodes, legs, c, cache, internal))
            if not nodes[c].external:
                lab = _label(nodes, legs, c)
                if lab is not None:
                    internal.add(lab)
        res = col.contract(res, internal)
    cache[nid] = res
    return res


def _amp_colour(nodes, legs, a, cache, internal):
    labels = [None] * len(a.vertex.fields)
    for c, s in zip(a.children, a.slots):
        labels[s] = _label(nodes, legs, c)
    elabel = ("e", "amp", a.id)
    internal.add(elabel)
    res = _vertex_colour(a.vertex, labels, a.struct, elabel)
    for c in a.children:
        res = col.mul(res, _node_colour(nodes, legs, c, cache, internal))
        if not nodes[c].external:
            lab = _label(nodes, legs, c)
            if lab is not None:
                internal.add(lab)
    return col.contract(res, internal)


def _fermion_leaf(nodes, nid):
    """External leg at the end of the fermion line a fermion node belongs to."""
    nd = nodes[nid]
    if nd.external:
        return nd.leg
    for c, s in zip(nd.children, nd.slots):
        if s in (0, 1):
            return _fermion_leaf(nodes, c)
    raise AssertionError


def _fermion_sign(nodes, a):
    pairs = []

    def visit(nid):
        nd = nodes[nid]
        if nd.external:
            return
        if nd.vertex.kind in ("FFV", "FFS") and not PARTICLES[nd.ptype].is_fermion:
            row = [c for c, s in zip(nd.children, nd.slots) if s == 0][0]
            colm = [c for c, s in zip(nd.children, nd.slots) if s == 1][0]
            pairs.append((_fermion_leaf(nodes, row), _fermion_leaf(nodes, colm)))
        for c in nd.children:
            visit(c)

    for c in a.children:
        visit(c)
    if a.vertex.kind in ("FFV", "FFS"):
        row = [c for c, s in zip(a.children, a.slots) if s == 0][0]
        colm = [c for c, s in zip(a.children, a.slots) if s == 1][0]
        pairs.append((_fermion_leaf(nodes, row), _fermion_leaf(nodes, colm)))
    seq = [x for p in sorted(pairs) for x in p]
    inv = sum(1 for i in range(len(seq)) for j in range(i + 1, len(seq)) if seq[i] > seq[j])
    return -1 if inv % 2 else 1


def _vphase(v):
    return v.phase if v.phase >= 0 else _VERTEX_PHASE[v.kind]


def _phase(nodes, nid, cache):
    if nid in cache:
        return cache[nid]
    nd = nodes[nid]
    if nd.external:
        ph = 0
    else:
        ph = _vphase(nd.vertex) + _PROP_PHASE[_kind_of(nd.ptype)]
        ph += sum(_phase(nodes, c, cache) for c in nd.children)
    cache[nid] = ph % 4
    return cache[nid]


_IPOW = [col.CQ(1), col.CQ(0, 1), col.CQ(-1), col.CQ(0, -1)]


# ---------------------------------------------------------------------------
def compile_process(name):
    proc = parse(name)
    legs = []
    for p, inc in zip(proc.particles, proc.incoming):
        P = PARTICLES[p]
        legs.append(Leg(p, inc, P.mass, helicity_states(p), P.colour))
    nodes, amps = generate(proc)
    if not amps:
        raise ValueError(f"no tree diagrams for {name!r}")

    # helicities: structural zeros
    an = _Analysis(proc, legs, nodes, amps)
    live = []
    amp_live = {}
    for h in itertools.product(*[l.hels for l in legs]):
        hmap = dict(enumerate(h))
        nz = [a.id for a in amps if an.amp_nonzero(a, hmap)]
        if nz:
            live.append(h)
            amp_live[h] = nz

    # node variants needed
    need = {}

    def mark(nid, h):
        nd = nodes[nid]
        var = tuple(h[l] for l in sorted(nd.legs))
        s = need.setdefault(nid, set())
        if var in s:
            return
        s.add(var)
        for c in nd.children:
            mark(c, h)

    amp_terms = []
    for h in live:
        terms = []
        for aid in amp_live[h]:
            a = amps[aid]
            for c in a.children:
                mark(c, h)
            terms.append((aid, [tuple(h[l] for l in sorted(nodes[c].legs)) for c in a.children]))
        amp_terms.append(terms)
    node_variants = {nid: sorted(v) for nid, v in need.items()}

    # colour decomposition with phases and fermion signs
    cache, internal = {}, set()
    pcache = {}
    amp_col = []
    basis_set = {}
    for a in amps:
        expr = _amp_colour(nodes, legs, a, cache, internal)
        ph = (_vphase(a.vertex) + sum(_phase(nodes, c, pcache) for c in a.children) + 3) % 4
        sgn = _fermion_sign(nodes, a)
        fac = _IPOW[ph] * sgn
        expr = {k: v * fac for k, v in expr.items()}
        amp_col.append(expr)
        for k in expr:
            basis_set.setdefault(k, len(basis_set))
    basis = sorted(basis_set, key=repr)
    bindex = {k: i for i, k in enumerate(basis)}
    coeffs = {}
    for a, expr in zip(amps, amp_col):
        for k, v in expr.items():
            coeffs[(a.id, bindex[k])] = v
    C = col.colour_matrix(basis)
    for row in C:
        for x in row:
            assert x.im == 0, "colour matrix must be real"
    den = 1
    for row in C:
        for x in row:
            den = den * x.re.denominator // math.gcd(den, x.re.denominator)
    cnum = [[int(x.re * den) for x in row] for row in C]

    # average over initial helicities and colours
    avg = Fraction(1)
    for l in legs:
        if l.incoming:
            avg /= len(l.hels)
            avg /= abs(l.colour)
    # vector lines whose k^mu k^nu / m^2 propagator term gives exactly zero: the current they carry, or
    # the current they are contracted with at every place they are used, comes from two external
    # massless fermions (k.J = 0 by the Dirac equation).  Computing such a term anyway adds only
    # rounding, amplified in FP32 by the size of k.J of the other end.
    def _massless_pair(vertex_kind, children):
        return vertex_kind == "FFV" and all(nodes[c].external and PARTICLES[nodes[c].ptype].massless
                                            for c in children if PARTICLES[nodes[c].ptype].is_fermion)
    uses = {}
    for nd in nodes:
        if not nd.external:
            for c in nd.children:
                uses.setdefault(c, []).append((nd.vertex.kind, [x for x in nd.children if x != c]))
    for a in amps:
        for c in a.children:
            uses.setdefault(c, []).append((a.vertex.kind, [x for x in a.children if x != c], "amp"))
    conserved = set()
    for nd in nodes:
        if nd.external or PARTICLES[nd.ptype].is_fermion:
            continue
        if _massless_pair(nd.vertex.kind, nd.children):
            conserved.add(nd.id)
        elif PARTICLES[nd.ptype].is_vector and nd.id in uses and all(
                len(u) == 3 and _massless_pair(u[0], u[1]) for u in uses[nd.id]):
            conserved.add(nd.id)
    prog = Program(name, legs, nodes, amps, live, node_variants, amp_terms, coeffs, basis, cnum, den, avg,
                   phases={nid: _phase(nodes, nid, pcache) for nid in range(len(nodes))}, conserved=conserved)
    return prog
