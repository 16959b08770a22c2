"""Host-side checks of the process compiler against the oracle's plain definitions."""
import itertools

import numpy as np
import pytest

from oracle import colour as ocol, processes as opr
from paper_1305_0708_gb300.compiler.program import compile_process

CASES = {
    "u u~ > e+ e-": (2, 4, 1),
    "u d~ > e+ ve g g": (8, 4, 2),
    "g g > (t > b (w+ > e+ ve)) (t~ > b~ (w- > e- ve~))": (3, 4, 2),
    "u s > d c h h": (4, 1, 1),
    "u u~ > g g": (3, 8, 2),
    "g g > g g": (6, 16, 6),
    # diagram terms (the four-gluon vertex counts once per colour structure), live helicities, colour
    # dimension, each counted by hand from the Feynman rules
    "u u~ > w+ w-": (3, 18, 1),          # t-channel d; s-channel photon and Z
    "u d~ > w+ z": (3, 9, 1),            # Z from u, Z from d; s-channel W
    "u d~ > w+ a": (3, 6, 1),            # photon from u, from d~, from the s-channel W
    "u u~ > z a": (2, 12, 1),
    "u u~ > a a": (2, 8, 1),
    "u u~ > z z": (2, 18, 1),
    "u u~ > z h": (1, 6, 1),
    "u d~ > w+ h": (1, 3, 1),
    "u d~ > w+ g": (2, 6, 1),
    "u g > w+ d": (2, 6, 1),
    "u u~ > z g": (2, 12, 1),
    "u u~ > z z g": (6, 36, 1),          # 3! orders of Z, Z, g along the quark line
    "u u~ > z h g": (2, 12, 1),          # the gluon before or after the s-channel Z
    "u d~ > w+ h g": (2, 6, 1),          # the gluon before or after the s-channel W
    "u d~ > w+ z g": (8, 18, 1),         # 3 + 3 along the two t-channel lines, 2 beside the s-channel W
    "u u~ > w+ w- g": (7, 36, 1),        # 3 along the t-channel line, 2 beside each s-channel photon and Z
    "g g > w+ d u~": (8, 12, 2),         # 3! orders of g, g, W along the quark line, 2 with the s-channel gluon
    "g g > z u u~": (8, 24, 2),          # the same graphs; both quark chiralities couple to the Z
    "u u~ > w+ w- a": (15, 36, 1),       # 3 + 2 + 4 + 4 + 2 (line, W lines, ISR, W emission, quartic)
    "g g > t t~": (3, 16, 2),
    "u u~ > t t~": (3, 8, 2),            # s-channel g, photon, Z; opposite light-quark helicities
    "u u~ > t t~ g": (13, 16, 4),        # (2 + 2) emissions x (g, photon, Z) + the three-gluon vertex
    "g g > t t~ h": (8, 16, 2),          # the Higgs on every top line of the three g g > t t~ graphs
    "g g > t t~ g": (18, 32, 6),         # 6 + 6 + 3 + one four-gluon graph with three colour structures
    "u u > u u": (6, 6, 2),              # g, photon, Z in the t and u channels; chirality-conserving helicities
    "h h > h h": (4, 1, 1),              # contact plus s, t, u exchange
    "u s > d c h": (1, 1, 1),            # W+ W- fusion; all four quarks left-handed
}


@pytest.mark.parametrize("name", list(CASES))
def test_diagram_helicity_colour_counts(name):
    prog = compile_process(name)
    nd, nh, nc = CASES[name]
    assert len(prog.amps) == nd
    assert len(prog.live) == nh
    assert prog.n_colour == nc


def _cmat(prog):
    return np.array(prog.cmat_num, dtype=float) / prog.cmat_den


def test_quark_gluon_colour_matrix_matches_brute_force():
    """(t^a t^b)_{ij}, (t^b t^a)_{ij}: the oracle's explicit-generator sum gives [[16/3,-2/3],[-2/3,16/3]]."""
    prog = compile_process("u d~ > e+ ve g g")
    C = _cmat(prog)
    cab = opr._colour_string([0, 1], 2)
    cba = opr._colour_string([1, 0], 2)
    M = np.array([c.ravel() for c in (cab, cba)])
    K = (M @ M.conj().T).real
    assert np.allclose(np.sort(C.ravel()), np.sort(K.ravel()))


@pytest.mark.parametrize("n", [4, 5])
def test_gluon_colour_matrix_matches_brute_force(n):
    """Trace basis with t normalisation: C_compiler = C_oracle / 2^n (T = sqrt2 t)."""
    name = "g g > " + " ".join(["g"] * (n - 2))
    prog = compile_process(name)
    C = _cmat(prog)
    orders, Co = ocol.gluon_trace_matrix(n)
    # map compiler basis (single traces over legs 0..n-1, canonical rotation) to the oracle orderings
    perm = []
    for key in prog.basis:
        assert len(key) == 1 and key[0][0] == "t"
        labels = [lab[1] for lab in key[0][1]]
        k = labels.index(0)
        perm.append(orders.index(tuple(labels[k:] + labels[:k])))
    sub = Co.real[np.ix_(perm, perm)] / 2 ** n
    assert np.allclose(C, sub, atol=1e-10)


@pytest.mark.parametrize("name,fn", [("u d~ > e+ ve g g", opr.udx_epvegg),
                                     ("g g > (t > b (w+ > e+ ve)) (t~ > b~ (w- > e- ve~))", opr.gg_ttx_dilep),
                                     ("u u~ > e+ e-", opr.uux_epem)])
def test_pruned_helicities_are_exact_zeros(name, fn):
    """Every helicity combination the compiler drops vanishes in the oracle.

    The oracle builds massless spinors from sqrt(E -+ |p|) with E and |p| from the
    momentum components, so a dropped chirality leaks at the rounding level
    (|M_h|^2 below 1e-13 of the total) instead of being an exact zero."""
    from oracle import phasespace as ps
    prog = compile_process(name)
    live = set(prog.live)
    n = prog.n_ext
    if n == 4:
        P, _ = ps.two_to_two_massless(500.0, ps.uniforms(0, np.arange(8), np.zeros(8), 4))
    elif n == 6:
        pf, _ = ps.rambo_massless(1000.0, 4, ps.uniforms(0, np.arange(8), np.zeros(8), 16))
        P = np.zeros((8, 6, 4))
        P[:, 0], P[:, 1] = ps.incoming(1000.0, 8)
        P[:, 2:] = pf
    else:
        from oracle.sm import SMParams
        Q, _, ok, _ = ps.ttbar_dilepton(ps.uniforms(0, np.arange(32), np.zeros(32), 16), SMParams(), (400, 2000))
        P = Q[ok][:8]
    _, ph = fn(P, per_helicity=True)
    tot = sum(ph.values())
    for h, v in ph.items():
        if h not in live:
            assert np.all(v <= 1e-13 * tot), h
    assert sum(1 for h in ph if h in live and np.any(ph[h] > 1e-12 * tot)) > 0


def test_every_compiled_process_has_a_pinned_oracle_and_a_parity_workload():
    """Each process string compiled into the library has an oracle function, and each workload or
    variant that the GPU parity tests and the bench run names a compiled process with an oracle."""
    from paper_1305_0708_gb300 import build
    from paper_1305_0708_gb300.workloads import VARIANTS, WORKLOADS
    compiled = set()
    for name, aliases in build.PROCESSES:
        compiled.add(name)
        compiled.update(aliases)
        assert name in opr.PROCESSES or any(a in opr.PROCESSES for a in aliases), name
    for n, _ in build.GLUON_PROCESSES:
        assert "g g > " + " ".join(["g"] * (n - 2)) in opr.PROCESSES
    for key, w in {**WORKLOADS, **VARIANTS}.items():
        proc = w["process"]
        assert proc in compiled or proc.startswith("g g > g g g"), key
