"""Colour-ordered program for all-gluon processes g g > g ... g.

For many gluons the straight-line diagram program grows too large for one
thread (six gluons: 510 diagram terms, 64 helicities, 120 colour components).
The same tree sum is organised by colour ordering instead: with the colour
basis of single traces Tr(t^{a_0} t^{a_s1} ... t^{a_s(n-1)}) (the basis the
colour algebra of this package produces for gluon trees), the coefficient of
each trace is the colour-ordered amplitude A(0, s), the sum of the planar
diagrams of that ordering.  The colour-ordered Feynman rules follow from the
Feynman rules of Sect. 4.2 (Eqs. 27-36) by the same trace algebra
(colour.py), with t normalisation Tr(t^a t^b) = delta/2:

  three-gluon, legs (1, 2, 3) in cyclic order, momenta outgoing:
      2 i g V^{mu nu rho}(k1, k2, k3),  V = g^{mu nu}(k1-k2)^rho + cyclic
  four-gluon, legs (1, 2, 3, 4):  2 i g^2 [2 g_13 g_24 - g_12 g_34 - g_14 g_23]
  internal line: -i g_{mu nu} / P^2 times 1/2, the weight with which
      sum_e t^e_ij t^e_kl joins two traces (Tr(t^a t^b) = delta/2)

so every vertex-line pair carries the real factor 1 (sub-current
J = (g V3 + g^2 V4 terms) / P^2), the root vertex the factor 2, and the global
phase of A is i for every ordering.  Sub-currents J(S) of ordered tuples S of
the non-root legs are built from their consecutive splittings; the amplitude
of ordering s contracts the root's polarisation with the amputated current of
the full tuple s.  This module emits the recursion tables and the exact
colour matrix; the kernel (csrc/gluon.cuh) runs them.
"""
import itertools
import math

from . import colour as col


def tables(n):
    """Recursion tables for n gluons (legs 0..n-1, root 0, incoming legs 0 and 1).

    Returns dict with:
      n_ext, currents: list of (tuple, v3 terms [(a, b)], v4 terms [(a, b, c)]) in phase order
        (index 0..n-2 are the single external legs 1..n-1),
      phases: list of (start, count) per size 2..n-2,
      amps: list of (tuple, v3 terms, v4 terms) for the (n-1)! orderings of legs 1..n-1,
      cnum, den: exact colour matrix C = cnum / den over the orderings (0, s), t normalisation.
    """
    legs = list(range(1, n))
    index = {}
    currents = []
    for l in legs:
        index[(l,)] = len(currents)
        currents.append(((l,), [], []))
    phases = []
    for size in range(2, n - 1):
        start = len(currents)
        for tup in itertools.permutations(legs, size):
            index[tup] = len(currents)
            currents.append((tup, _v3_terms(tup, index), _v4_terms(tup, index)))
        phases.append((start, len(currents) - start))
    amps = []
    for tup in itertools.permutations(legs, n - 1):
        amps.append((tup, _v3_terms(tup, index), _v4_terms(tup, index)))
    # exact colour matrix over the traces Tr(t^0 t^s1 ...), s in the order of `amps`
    basis = [(("t", (("g", 0),) + tuple(("g", l) for l in tup)),) for tup, _, _ in amps]
    C = col.colour_matrix(basis)
    den = 1
    for row in C:
        for x in row:
            assert x.im == 0
            den = den * x.re.denominator // math.gcd(den, x.re.denominator)
    cnum = [[int(x.re * den) for x in row] for row in C]
    return dict(n_ext=n, currents=currents, phases=phases, amps=amps, cnum=cnum, den=den, index=index)


def _v3_terms(tup, index):
    return [(index[tup[:i]], index[tup[i:]]) for i in range(1, len(tup))]


def _v4_terms(tup, index):
    out = []
    L = len(tup)
    for i in range(1, L - 1):
        for j in range(i + 1, L):
            out.append((index[tup[:i]], index[tup[i:j]], index[tup[j:]]))
    return out


def header(n):
    """C++ header with the recursion tables and colour matrix for n gluons."""
    t = tables(n)
    cur = t["currents"]
    amps = t["amps"]
    lines = [f"// Generated by paper_1305_0708_gb300.compiler.gluon for {n} gluons.", "#pragma once",
             "#include <cstdint>", "namespace me {", "namespace gluon {", f"struct Tables{n} {{",
             f"  static constexpr int NG = {n};",
             f"  static constexpr int NCUR = {len(cur)};",
             f"  static constexpr int NAMP = {len(amps)};",
             f"  static constexpr int NPHASE = {len(t['phases'])};",
             f"  static constexpr int DEN = {t['den']};"]

    def flat(entries):
        # per entry: leg mask, n_v3, n_v4, offset; term list of int16 child indices
        meta, terms = [], []
        for tup, v3, v4 in entries:
            mask = sum(1 << l for l in tup)
            meta.append((mask, len(v3), len(v4), len(terms)))
            for a, b in v3:
                terms += [a, b]
            for a, b, c in v4:
                terms += [a, b, c]
        return meta, terms

    cm, ct = flat(cur)
    am, at = flat(amps)
    # per tuple size S (currents of one phase, or the amplitudes for S = n-1): the distinct
    # currents of the vertex terms of an entry s -- prefixes s[:t] and suffixes s[t:]
    # (t = 1..S-1), then middles s[i:j] (1 <= i < j <= S-1); the three-gluon terms are
    # (s[:t], s[t:]) and the four-gluon terms (s[:i], s[i:j], s[j:]).  Stored slot-major,
    # pqm[slot * COUNT + entry], so that a warp reads consecutive entries.
    start, count, off, pqm = [0] * n, [0] * n, [0] * n, []
    by_size = {sz: (st, ct_) for sz, (st, ct_) in zip(range(2, n - 1), t["phases"])}
    by_size[n - 1] = (0, len(amps))
    index = t["index"]
    for sz in range(2, n):
        st, cnt = by_size[sz]
        ents = amps if sz == n - 1 else cur[st:st + cnt]
        npre = sz - 1
        pairs = [(i, j) for i in range(1, npre + 1) for j in range(i + 1, npre + 1)]
        rows = []
        for tup, v3, v4 in ents:
            assert len(tup) == sz and len(v3) == npre and len(v4) == len(pairs)
            rows.append([index[tup[:k]] for k in range(1, npre + 1)] + [index[tup[k:]] for k in range(1, npre + 1)] +
                        [index[tup[i:j]] for i, j in pairs])
        start[sz], count[sz], off[sz] = st, cnt, len(pqm)
        for j in range(len(rows[0])):
            pqm += [r[j] for r in rows]
    lines.append(f"  static constexpr int START[{n}] = {{{', '.join(map(str, start))}}};")
    lines.append(f"  static constexpr int COUNT[{n}] = {{{', '.join(map(str, count))}}};")
    lines.append(f"  static constexpr int PQM_OFF[{n}] = {{{', '.join(map(str, off))}}};")
    lines.append("};")
    lines.append(f"__device__ const int16_t kPQM{n}[{len(pqm)}] = {{" + ", ".join(map(str, pqm)) + "};")
    lines.append(f"__device__ const int32_t kCurMeta{n}[{len(cm) * 4}] = {{" +
                 ", ".join(str(x) for m in cm for x in m) + "};")
    lines.append(f"__device__ const int16_t kCurTerms{n}[{max(len(ct), 1)}] = {{" +
                 (", ".join(str(x) for x in ct) or "0") + "};")
    lines.append(f"__device__ const int32_t kAmpMeta{n}[{len(am) * 4}] = {{" +
                 ", ".join(str(x) for m in am for x in m) + "};")
    lines.append(f"__device__ const int16_t kAmpTerms{n}[{len(at)}] = {{" + ", ".join(str(x) for x in at) + "};")
    lines.append(f"__device__ const int32_t kPhase{n}[{max(2 * len(t['phases']), 2)}] = {{" +
                 (", ".join(str(x) for p in t["phases"] for x in p) or "0, 0") + "};")
    cn = t["cnum"]
    diag = cn[0][0]
    assert all(cn[i][i] == diag for i in range(len(cn))), "trace colour matrix has a constant diagonal"
    assert all(cn[i][j] == cn[j][i] for i in range(len(cn)) for j in range(i)), "colour matrix is symmetric"
    off = max(abs(cn[i][j]) for i in range(len(cn)) for j in range(len(cn)) if i != j)
    lines.append(f"constexpr float kColourDiag{n} = {float(diag)!r}f;  // off-diagonal max |C| = {off}")
    lines.append(f"constexpr bool kColourOffFitsHalf{n} = {'true' if off <= 2048 else 'false'};")
    lines.append(f"__device__ const float kColour{n}[{len(cn) * len(cn)}] = {{" +
                 ", ".join(f"{float(x)!r}f" for row in cn for x in row) + "};")
    # host copies for host-side checks
    lines.append(f"static const int16_t kPQM{n}_h[{len(pqm)}] = {{" + ", ".join(map(str, pqm)) + "};")
    lines.append(f"static const int32_t kCurMeta{n}_h[{len(cm) * 4}] = {{" +
                 ", ".join(str(x) for m in cm for x in m) + "};")
    lines.append(f"static const int16_t kCurTerms{n}_h[{max(len(ct), 1)}] = {{" +
                 (", ".join(str(x) for x in ct) or "0") + "};")
    lines.append(f"static const int32_t kAmpMeta{n}_h[{len(am) * 4}] = {{" +
                 ", ".join(str(x) for m in am for x in m) + "};")
    lines.append(f"static const int16_t kAmpTerms{n}_h[{len(at)}] = {{" + ", ".join(str(x) for x in at) + "};")
    lines.append(f"static const int32_t kPhase{n}_h[{max(2 * len(t['phases']), 2)}] = {{" +
                 (", ".join(str(x) for p in t["phases"] for x in p) or "0, 0") + "};")
    lines.append(f"static const float kColour{n}_h[{len(cn) * len(cn)}] = {{" +
                 ", ".join(f"{float(x)!r}f" for row in cn for x in row) + "};")
    lines.append("}  // namespace gluon")
    lines.append("}  // namespace me")
    return "\n".join(lines) + "\n", t
