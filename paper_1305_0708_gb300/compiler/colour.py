"""Exact SU(N) colour algebra for tree diagrams (the colour decomposition step).

The paper leaves colour summation to MadGraph (Sect. 2) and stores the
decomposed colour matrix as "independent colour factors" (Sect. 5.4).  Here
every diagram's colour factor is reduced exactly, with rational complex
coefficients, to a basis of products of open strings (t^a1 ... t^ak)_{i j}
and traces Tr(t^a1 ... t^ak) over external indices; the colour matrix
C_kl = sum_colours B_k B_l^* is reduced the same way.

Rules (t normalisation Tr(t^a t^b) = delta^{ab}/2):
  f^{abc}              = -2i [Tr(t^a t^b t^c) - Tr(t^b t^a t^c)]
  t^e_ij t^e_kl        = 1/2 (delta_il delta_kj - delta_ij delta_kl / N)
  Tr() = N, Tr(t^a) = 0, strings joined over contracted quark indices.
"""
from fractions import Fraction
import itertools

NC = 3


class CQ:
    """Complex rational number."""
    __slots__ = ("re", "im")

    def __init__(self, re=0, im=0):
        self.re = Fraction(re)
        self.im = Fraction(im)

    def __add__(self, o):
        return CQ(self.re + o.re, self.im + o.im)

    def __mul__(self, o):
        if isinstance(o, CQ):
            return CQ(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)
        o = Fraction(o)
        return CQ(self.re * o, self.im * o)

    __rmul__ = __mul__

    def __neg__(self):
        return CQ(-self.re, -self.im)

    def conj(self):
        return CQ(self.re, -self.im)

    def is_zero(self):
        return self.re == 0 and self.im == 0

    def __eq__(self, o):
        return isinstance(o, CQ) and self.re == o.re and self.im == o.im

    def __hash__(self):
        return hash((self.re, self.im))

    def __repr__(self):
        return f"({self.re}{'+' if self.im >= 0 else ''}{self.im}i)"

    def as_complex(self):
        return complex(float(self.re), float(self.im))


# A chain is ("s", row, labels, col) for (t^l1 ... t^lk)_{row,col} or ("t", labels).
# An expression is a dict {tuple(sorted chains): CQ}.

def _canon_trace(labels):
    if not labels:
        return ("t", ())
    k = min(range(len(labels)), key=lambda i: labels[i:] + labels[:i])
    return ("t", tuple(labels[k:] + labels[:k]))


def _key(chains):
    return tuple(sorted(chains, key=repr))


def expr_from(chains, coeff=CQ(1)):
    return {_key(chains): coeff}


def mul(a, b):
    out = {}
    for ka, ca in a.items():
        for kb, cb in b.items():
            k = _key(list(ka) + list(kb))
            out[k] = out.get(k, CQ()) + ca * cb
    return {k: v for k, v in out.items() if not v.is_zero()}


def add(a, b, scale=CQ(1)):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, CQ()) + v * scale
    return {k: v for k, v in out.items() if not v.is_zero()}


def f_abc(a, b, c):
    """f^{abc} as traces."""
    return {
        _key([_canon_trace((a, b, c))]): CQ(0, -2),
        _key([_canon_trace((b, a, c))]): CQ(0, 2),
    } if _canon_trace((a, b, c)) != _canon_trace((b, a, c)) else {}


def t_string(row, labels, col):
    return expr_from([("s", row, tuple(labels), col)])


def delta(row, col):
    return expr_from([("s", row, (), col)])


def _simplify_term(chains, coeff, internal):
    """Fully contract the internal indices of one product of chains; returns an expression."""
    work = [(list(chains), coeff)]
    done = {}
    while work:
        ch, c = work.pop()
        ch = list(ch)
        # 1. join strings over contracted fundamental indices, close traces
        changed = True
        while changed:
            changed = False
            for i, x in enumerate(ch):
                if x[0] != "s":
                    continue
                if x[1] == x[3] and x[1] in internal:
                    ch[i] = _canon_trace(x[2]) if x[2] else ("t", ())
                    changed = True
                    break
                for j, y in enumerate(ch):
                    if i != j and y[0] == "s" and x[3] == y[1] and x[3] in internal:
                        new = ("s", x[1], x[2] + y[2], y[3])
                        ch = [z for k, z in enumerate(ch) if k not in (i, j)] + [new]
                        changed = True
                        break
                if changed:
                    break
        # 2. traces: Tr() = N, Tr(t) = 0
        zero = False
        rest = []
        for x in ch:
            if x[0] == "t":
                if len(x[1]) == 0:
                    c = c * NC
                    continue
                if len(x[1]) == 1:
                    zero = True
                    break
                rest.append(_canon_trace(x[1]))
            else:
                rest.append(x)
        if zero:
            continue
        ch = rest
        # 3. find a repeated internal adjoint label
        occ = {}
        for ci, x in enumerate(ch):
            labels = x[2] if x[0] == "s" else x[1]
            for li, lab in enumerate(labels):
                if lab in internal:
                    occ.setdefault(lab, []).append((ci, li))
        rep = next((lab for lab, v in occ.items() if len(v) == 2), None)
        if rep is None:
            k = _key(ch)
            done[k] = done.get(k, CQ()) + c
            continue
        (c1, l1), (c2, l2) = occ[rep]
        half = c * Fraction(1, 2)
        mhalfN = c * Fraction(-1, 2 * NC)
        others = [x for k, x in enumerate(ch) if k not in (c1, c2)]
        X = ch[c1]
        if c1 == c2:
            lab = X[2] if X[0] == "s" else X[1]
            i, j = sorted((l1, l2))
            A, B, C = lab[:i], lab[i + 1:j], lab[j + 1:]
            if X[0] == "s":
                # (A t B t C) = 1/2 [Tr(B) (A C) - 1/N (A B C)]
                work.append((others + [("s", X[1], A + C, X[3]), ("t", B)], half))
                work.append((others + [("s", X[1], A + B + C, X[3])], mhalfN))
            else:
                # Tr(A t B t C) = Tr(C A t B t) = 1/2 [Tr(CA) Tr(B) - 1/N Tr(CAB)]
                work.append((others + [("t", C + A), ("t", B)], half))
                work.append((others + [("t", C + A + B)], mhalfN))
            continue
        Y = ch[c2]

        def split(Z, li):
            lab = Z[2] if Z[0] == "s" else Z[1]
            return lab[:li], lab[li + 1:]

        A, B = split(X, l1)
        Cc, D = split(Y, l2)
        if X[0] == "s" and Y[0] == "s":
            # (A t B)_{r1 c1} (C t D)_{r2 c2} = 1/2 [(A D)_{r1 c2} (C B)_{r2 c1} - 1/N (AB)(CD)]
            work.append((others + [("s", X[1], A + D, Y[3]), ("s", Y[1], Cc + B, X[3])], half))
            work.append((others + [("s", X[1], A + B, X[3]), ("s", Y[1], Cc + D, Y[3])], mhalfN))
        elif X[0] == "t" and Y[0] == "t":
            # Tr(Xp t) Tr(Yp t) = 1/2 [Tr(Xp Yp) - 1/N Tr(Xp) Tr(Yp)], Xp = B A
            Xp, Yp = B + A, D + Cc
            work.append((others + [("t", Xp + Yp)], half))
            work.append((others + [("t", Xp), ("t", Yp)], mhalfN))
        else:
            if X[0] == "t":
                X, Y = Y, X
                A, B, Cc, D = Cc, D, A, B
            # (A t B)_{rc} Tr(Cc t D) = (A t B)_{rc} Tr(D Cc t) = 1/2 [(A (D Cc) B) - 1/N (A B) Tr(D Cc)]
            Zp = D + Cc
            work.append((others + [("s", X[1], A + Zp + B, X[3])], half))
            work.append((others + [("s", X[1], A + B, X[3]), ("t", Zp)], mhalfN))
    return {k: v for k, v in done.items() if not v.is_zero()}


def contract(expr, internal):
    """Contract all indices in `internal` (a set of labels) in every term."""
    out = {}
    for chains, c in expr.items():
        out = add(out, _simplify_term(chains, c, internal))
    return out


def conj_chain(x):
    if x[0] == "s":
        return ("s", x[3], tuple(reversed(x[2])), x[1])
    return _canon_trace(tuple(reversed(x[1])))


def colour_matrix(basis):
    """Exact C_kl = sum over external colours of B_k B_l^* for a list of basis keys."""
    n = len(basis)
    C = [[None] * n for _ in range(n)]
    cache = {}
    for k in range(n):
        for l in range(k, n):
            chains = list(basis[k]) + [conj_chain(x) for x in basis[l]]
            labels = set()
            for x in chains:
                if x[0] == "s":
                    labels.update([x[1], x[3]])
                    labels.update(x[2])
                else:
                    labels.update(x[1])
            key = _relabel_key(chains)
            if key not in cache:
                res = _simplify_term(key, CQ(1), set(_all_labels(key)))
                val = CQ()
                for kk, cc in res.items():
                    assert kk == (), f"uncontracted colour: {kk}"
                    val = val + cc
                cache[key] = val
            C[k][l] = cache[key]
            C[l][k] = cache[key].conj()
    return C


def _all_labels(chains):
    out = []
    for x in chains:
        if x[0] == "s":
            out += [x[1], x[3]] + list(x[2])
        else:
            out += list(x[1])
    return out


def _relabel_key(chains):
    """Rename labels in order of first appearance so equivalent products share a cache entry."""
    names = {}
    for lab in _all_labels(chains):
        if lab not in names:
            names[lab] = ("x", len(names))
    out = []
    for x in chains:
        if x[0] == "s":
            out.append(("s", names[x[1]], tuple(names[a] for a in x[2]), names[x[3]]))
        else:
            out.append(_canon_trace(tuple(names[a] for a in x[1])))
    return tuple(out)
