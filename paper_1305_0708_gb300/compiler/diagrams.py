"""Tree-diagram enumeration from the Feynman rules (the converter's role, Sect. 5).

A process "a b > c d ..." is read as external legs in string order, incoming
first.  Every leg is given the particle type it brings *into* the vertex it
attaches to (incoming legs: the particle; outgoing legs: its antiparticle),
and all momenta are counted flowing into vertices (incoming legs +p,
outgoing legs -p).  Diagrams are built by dynamic programming over subsets
of the legs other than the root (the last leg): a current for a subset S is
one distinct sub-tree, with the particle type it carries into its parent
vertex; the amplitudes join currents that partition all non-root legs with
the root at one vertex.  Distinct sub-trees are kept apart (no summation),
so every diagram keeps its own colour factor and shares its sub-currents
with the others, as the paper's generated code does (Sect. 5.5).

Decay chains "a b > (t > b (w+ > e+ ve)) ..." keep only the diagrams that
contain each named resonance on the internal line that carries exactly its
decay products.
"""
import itertools
import re
from dataclasses import dataclass, field

from .model import PARTICLES, VERTICES, ALIASES


@dataclass
class Node:
    id: int
    legs: frozenset
    ptype: str                 # particle type flowing into the parent vertex
    leg: int = -1              # external leg index (external nodes)
    vertex: object = None      # model.Vertex (internal nodes)
    slots: tuple = ()          # vertex slot of each child, in child order
    children: tuple = ()       # child node ids
    out_slot: int = -1         # vertex slot of the line towards the parent
    struct: int = -1           # VVVV colour/Lorentz pairing (0, 1, 2)

    @property
    def external(self):
        return self.leg >= 0


@dataclass
class Amplitude:
    id: int
    vertex: object
    slots: tuple
    children: tuple
    struct: int = -1


@dataclass
class Process:
    name: str
    particles: list            # particle name per leg
    incoming: list             # bool per leg
    resonances: list = field(default_factory=list)   # (particle, frozenset(legs))


def parse(process):
    """Parse 'a b > c (t > x y) ...' into a Process."""
    s = process.strip()
    lhs, rhs = s.split(">", 1)
    ins = lhs.split()
    tokens = re.findall(r"\(|\)|>|[^\s()>]+", rhs)
    outs = []
    res = []

    def parse_list(pos, stop):
        legs = []
        while pos < len(tokens) and tokens[pos] != stop:
            t = tokens[pos]
            if t == "(":
                name = tokens[pos + 1]
                assert tokens[pos + 2] == ">", "decay syntax is (X > a b ...)"
                sub, pos = parse_list(pos + 3, ")")
                res.append((ALIASES.get(name, name), frozenset(sub)))
                legs += sub
                pos += 1
            else:
                name = ALIASES.get(t, t)
                if name not in PARTICLES:
                    raise ValueError(f"unknown particle {t!r}")
                outs.append(name)
                legs.append(len(ins) + len(outs) - 1)
                pos += 1
        return legs, pos

    parse_list(0, None)
    for p in ins:
        if ALIASES.get(p, p) not in PARTICLES:
            raise ValueError(f"unknown particle {p!r}")
    ins = [ALIASES.get(p, p) for p in ins]
    return Process(process, ins + outs, [True] * len(ins) + [False] * len(outs), res)


def _vertex_matches(types):
    """Vertices whose fields contain the multiset `types` (children), with the slot
    assignments and the remaining slot(s).  One assignment per distinct result."""
    out = []
    k = len(types)
    for v in VERTICES:
        if len(v.fields) != k + 1 and len(v.fields) != k:
            continue
        seen = set()
        for perm in itertools.permutations(range(len(v.fields)), k):
            if all(v.fields[perm[i]] == types[i] for i in range(k)):
                rest = [s for s in range(len(v.fields)) if s not in perm]
                key = tuple(sorted(v.fields[s] for s in rest))
                if key in seen:
                    continue
                seen.add(key)
                out.append((v, perm, rest))
    return out


def _splits(mask, parts):
    """Unordered partitions of a bitmask into `parts` non-empty submasks."""
    bits = [b for b in range(mask.bit_length()) if mask >> b & 1]
    if parts == 2:
        low = 1 << bits[0]
        rest = mask ^ low
        sub = rest
        while True:
            s1 = low | sub
            s2 = mask ^ s1
            if s2:
                yield (s1, s2)
            if sub == 0:
                break
            sub = (sub - 1) & rest
    elif parts == 3:
        for s1, rem in _splits(mask, 2):
            if bin(rem).count("1") >= 2:
                for s2, s3 in _splits(rem, 2):
                    yield (s1, s2, s3)


def generate(proc):
    """Return (nodes, amplitudes) for a Process."""
    n = len(proc.particles)
    root = n - 1
    etype = [p if inc else PARTICLES[p].anti for p, inc in zip(proc.particles, proc.incoming)]
    nodes = []
    by_mask = {}
    for leg in range(n - 1):
        nd = Node(len(nodes), frozenset([leg]), etype[leg], leg=leg)
        nodes.append(nd)
        by_mask[1 << leg] = [nd.id]
    full = (1 << (n - 1)) - 1
    masks = sorted(range(1, full + 1), key=lambda m: bin(m).count("1"))
    for mask in masks:
        if bin(mask).count("1") < 2 or mask == full:
            continue
        cur = []
        for parts in (2, 3):
            for split in _splits(mask, parts):
                for combo in itertools.product(*[by_mask.get(s, []) for s in split]):
                    types = [nodes[c].ptype for c in combo]
                    for v, perm, rest in _vertex_matches(types):
                        if len(rest) != 1:
                            continue
                        out = rest[0]
                        ptype = PARTICLES[v.fields[out]].anti
                        structs = [0, 1, 2] if v.colour == "ff" else [-1]
                        for st in structs:
                            nd = Node(len(nodes), frozenset().union(*[nodes[c].legs for c in combo]), ptype,
                                      vertex=v, slots=tuple(perm), children=tuple(combo), out_slot=out, struct=st)
                            nodes.append(nd)
                            cur.append(nd.id)
        by_mask[mask] = cur
    rnode = Node(len(nodes), frozenset([root]), etype[root], leg=root)
    nodes.append(rnode)
    amps = []
    for parts in (2, 3):
        for split in _splits(full, parts):
            for combo in itertools.product(*[by_mask.get(s, []) for s in split]):
                combo = tuple(combo) + (rnode.id,)
                types = [nodes[c].ptype for c in combo]
                for v, perm, rest in _vertex_matches(types):
                    if rest:
                        continue
                    structs = [0, 1, 2] if v.colour == "ff" else [-1]
                    for st in structs:
                        amps.append(Amplitude(len(amps), v, tuple(perm), combo, st))
    nodes, amps = _prune(nodes, amps, proc)
    return nodes, amps


def _uses(nodes, nid, acc):
    acc.add(nid)
    for c in nodes[nid].children:
        _uses(nodes, c, acc)
    return acc


def _prune(nodes, amps, proc):
    """Apply the decay-chain filter and drop nodes no amplitude uses."""
    n = len(proc.particles)
    all_legs = frozenset(range(n))
    if proc.resonances:
        keep = []
        for a in amps:
            used = set()
            for c in a.children:
                _uses(nodes, c, used)
            ok = True
            for part, legs in proc.resonances:
                found = False
                for u in used:
                    nd = nodes[u]
                    if nd.external:
                        continue
                    if nd.legs == legs and nd.ptype == PARTICLES[part].anti:
                        found = True
                    if nd.legs == all_legs - legs and nd.ptype == part:
                        found = True
                ok = ok and found
            if ok:
                keep.append(a)
        amps = [Amplitude(i, a.vertex, a.slots, a.children, a.struct) for i, a in enumerate(keep)]
    used = set()
    for a in amps:
        for c in a.children:
            _uses(nodes, c, used)
    remap = {}
    out = []
    for nd in nodes:
        if nd.id in used:
            remap[nd.id] = len(out)
            out.append(nd)
    for nd in out:
        nd.id = remap[nd.id]
        nd.children = tuple(remap[c] for c in nd.children)
    for a in amps:
        a.children = tuple(remap[c] for c in a.children)
    return out, amps
