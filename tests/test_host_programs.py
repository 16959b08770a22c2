"""The generated helicity programs, compiled for the host CPU, against the oracle.

The code generator's FP64 and mixed-precision evaluators are host-and-device functions.  Compiled
into a small host program (tests/host/host_eval.cu) they run here without a GPU, so the process
compiler, the HEGET-style device functions and the double-float arithmetic are checked on the
CPU.  The same tolerances as the GPU parity tests apply, on inputs made on shell and balanced to
FP64 rounding: FP64 within 1e-12 relative plus the oracle's own spread under rounding-level input
perturbations (median below 1e-12), mixed median <= 1e-5 and max <= 1e-3.  Needs nvcc.
"""
import math
import os
import re
import shutil
import struct
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import phasespace as ps, processes as opr
from oracle.sm import SMParams
from kinematics import conditioning, consistent

PAR = SMParams()
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1305_0708_gb300", "csrc")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc")

# process -> (oracle, sqrt(s), final-state masses, legs with pT > 20 and |eta| < 2.5)
CASES = {
    "u u~ > w+ w- a": (opr.uux_wpwma, 500.0, (80.4, 80.4, 0.0), (4,)),
    "g g > t t~ h": (opr.gg_ttxh, 1000.0, (175.0, 175.0, 125.0), ()),
    "g g > t t~ g": (opr.gg_ttxg, 1000.0, (175.0, 175.0, 0.0), (4,)),
    "u u~ > z z g": (opr.uux_zzg, 500.0, (91.1876, 91.1876, 0.0), (4,)),
    "u s > d c h h": (opr.us_dchh, 1000.0, (0.0, 0.0, 125.0, 125.0), ()),
    "u s > d c h": (opr.us_dch, 1000.0, (0.0, 0.0, 125.0), ()),
    "u u~ > w+ w-": (opr.uux_wpwm, 500.0, (80.4, 80.4), ()),
    "u d~ > w+ z": (opr.udx_wpz, 500.0, (80.4, 91.1876), ()),
    "u d~ > w+ a": (opr.udx_wpa, 500.0, (80.4, 0.0), (3,)),
    "u u~ > z a": (opr.uux_za, 500.0, (91.1876, 0.0), (3,)),
    "u u~ > a a": (opr.uux_aa, 500.0, (0.0, 0.0), (2, 3)),
    "u u~ > z z": (opr.uux_zz, 500.0, (91.1876, 91.1876), ()),
    "u u~ > z h": (opr.uux_zh, 500.0, (91.1876, 125.0), ()),
    "u d~ > w+ h": (opr.udx_wph, 500.0, (80.4, 125.0), ()),
    "u d~ > w+ g": (opr.udx_wpg, 500.0, (80.4, 0.0), (3,)),
    "u u~ > z g": (opr.uux_zg, 500.0, (91.1876, 0.0), (3,)),
    "g g > t t~": (opr.gg_ttx, 800.0, (175.0, 175.0), ()),
    "u u > u u": (opr.uu_uu, 500.0, (0.0, 0.0), (2, 3)),
    "u g > w+ d": (opr.ug_wpd, 500.0, (80.4, 0.0), (3,)),
    "u u~ > z h g": (opr.uux_zhg, 600.0, (91.1876, 125.0, 0.0), (4,)),
    "u d~ > w+ h g": (opr.udx_wphg, 600.0, (80.4, 125.0, 0.0), (4,)),
    "u d~ > w+ z g": (opr.udx_wpzg, 600.0, (80.4, 91.1876, 0.0), (4,)),
    "u u~ > w+ w- g": (opr.uux_wpwmg, 600.0, (80.4, 80.4, 0.0), (4,)),
    "g g > w+ d u~": (opr.gg_wpdux, 600.0, (80.4, 0.0, 0.0), (3, 4)),
    "g g > z u u~": (opr.gg_zuux, 600.0, (91.1876, 0.0, 0.0), (3, 4)),
    "u u~ > t t~": (opr.uux_ttx, 800.0, (175.0, 175.0), ()),
    "u u~ > t t~ g": (opr.uux_ttxg, 1000.0, (175.0, 175.0, 0.0), (4,)),
    "u d~ > w+ g g": (opr.udx_wpgg, 600.0, (80.4, 0.0, 0.0), (3, 4)),
    "u u~ > z g g": (opr.uux_zgg, 600.0, (91.1876, 0.0, 0.0), (3, 4)),
    "u s > d c h g": (opr.us_dchg, 1000.0, (0.0, 0.0, 125.0, 0.0), (5,)),
    "u s > d c h h h": (opr.us_dchhh, 1500.0, (0.0, 0.0, 125.0, 125.0, 125.0), ()),
    "u d > u d h": (opr.ud_udh, 1000.0, (0.0, 0.0, 125.0), ()),
    "u d > u d h h": (opr.ud_udhh, 1000.0, (0.0, 0.0, 125.0, 125.0), ()),
    "u d > u d h h h": (opr.ud_udhhh, 1500.0, (0.0, 0.0, 125.0, 125.0, 125.0), ()),
    "u d~ > w+ g g g": (opr.udx_wpggg, 800.0, (80.4, 0.0, 0.0, 0.0), (3, 4, 5)),
    "u u~ > z g g g": (opr.uux_zggg, 800.0, (91.1876, 0.0, 0.0, 0.0), (3, 4, 5)),
    "g g > t t~ h g": (opr.gg_ttxhg, 1500.0, (175.0, 175.0, 125.0, 0.0), (5,)),
    "u s > d c h g g": (opr.us_dchgg, 1000.0, (0.0, 0.0, 125.0, 0.0, 0.0), (2, 3, 5, 6)),
    "u u~ > z z g g": (opr.uux_zzgg, 600.0, (91.1876, 91.1876, 0.0, 0.0), (4, 5)),
    "u d~ > w+ h g g": (opr.udx_wphgg, 700.0, (80.4, 125.0, 0.0, 0.0), (4, 5)),
    "u u > u u h h": (opr.uu_uuhh, 1000.0, (0.0, 0.0, 125.0, 125.0), ()),
    "u u > u u h h h": (opr.uu_uuhhh, 1500.0, (0.0, 0.0, 125.0, 125.0, 125.0), ()),
    "u u~ > w+ w- g g": (opr.uux_wpwmgg, 700.0, (80.4, 80.4, 0.0, 0.0), (4, 5)),
    "u d~ > w+ z g g": (opr.udx_wpzgg, 700.0, (80.4, 91.1876, 0.0, 0.0), (4, 5)),
    "u d~ > w+ h g g g": (opr.udx_wphggg, 900.0, (80.4, 125.0, 0.0, 0.0, 0.0), (4, 5, 6)),
}

# the complex-mass option (Sect. 7.11): processes whose couplings it makes complex
CMS_CASES = ["u s > d c h h", "u s > d c h h h", "u d > u d h h h", "g g > t t~ h", "u u~ > z h"]


def _nvcc():
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _points(sqrt_s, masses, cut_legs, n, seed):
    u = ps.uniforms(seed, np.arange(n), np.zeros(n), 4 * len(masses))
    pf, _ = ps.rambo_massive(sqrt_s, list(masses), u)
    P = np.zeros((n, len(masses) + 2, 4))
    P[:, 0], P[:, 1] = ps.incoming(sqrt_s, n)
    P[:, 2:] = pf
    keep = np.ones(n, dtype=bool)
    for leg in cut_legs:
        pt = np.hypot(P[:, leg, 1], P[:, leg, 2])
        eta = np.arcsinh(P[:, leg, 3] / np.maximum(pt, 1e-300))
        keep &= (pt > 20.0) & (np.abs(eta) < 2.5)
    return P[keep]


def _tolerance(fn, P, ref):
    """1e-12 relative plus 32 times the oracle's spread under 2^-52 input perturbations (the inputs
    are on shell and balanced to rounding, kinematics.consistent)."""
    return 1e-12 * np.abs(ref) + 32 * conditioning(fn, P, ref, PAR, draws=3)


def _build(name, workdir, hel_loop=None):
    from paper_1305_0708_gb300.compiler.codegen import generate_source, process_symbol
    from paper_1305_0708_gb300.compiler.program import compile_process
    tag = process_symbol(name) + ("_loop" if hel_loop else "")
    src, _ = generate_source(compile_process(name), tag, hel_loop=hel_loop)
    cut = src.rindex("ME_DEFINE_PROCESS(")           # kernels and registration stay out of the host build
    unit = os.path.join(workdir, tag + ".cuh")
    with open(unit, "w") as f:
        f.write(src[:cut] + src[src.index("\n", cut):])
    fields = re.findall(r"double (\w+);", src[src.index("struct Params {"):src.index("struct ParamsMx")])
    exe = os.path.join(workdir, tag)
    n_ext = int(re.search(r"static constexpr int NEXT = (\d+);", src).group(1))
    cmd = [_nvcc(), "-O1", "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", CSRC, "-I", workdir, "-I", os.path.join(ROOT, "include"), f'-DGEN_UNIT="{unit}"', f"-DTAG={tag}",
           f"-DNEXT_H={n_ext}", os.path.join(HERE, "host", "host_eval.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe, fields


def _params(fields, complex_mass=0):
    """The parameter block of a unit: its fields (C identifiers of the coupling names) in order."""
    from paper_1305_0708_gb300.compiler.codegen import _ident
    from paper_1305_0708_gb300.compiler.model import DEFAULT_PARAMS, couplings
    c = {_ident(k): v for k, v in couplings(dict(DEFAULT_PARAMS, complex_mass=complex_mass)).items()}
    return [c[x] for x in fields]


@pytest.fixture(scope="module")
def programs():
    from paper_1305_0708_gb300.compiler import dftables
    with tempfile.TemporaryDirectory() as d:
        with open(os.path.join(d, "dfloat_tables.h"), "w") as f:
            f.write(dftables.header())
        with ThreadPoolExecutor(max_workers=min(6, os.cpu_count() or 1)) as ex:
            built = dict(zip(CASES, ex.map(lambda n: _build(n, d), CASES)))
        yield d, built


def _run(exe, params, P, workdir):
    inp = os.path.join(workdir, os.path.basename(exe) + ".in")
    out = os.path.join(workdir, os.path.basename(exe) + ".out")
    with open(inp, "wb") as f:
        f.write(struct.pack("ii", P.shape[0], len(params)))
        f.write(np.asarray(params, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(P, dtype=np.float64).tobytes())
    subprocess.run([exe, inp, out], check=True)
    return np.fromfile(out).reshape(-1, 2)


@pytest.mark.parametrize("name", list(CASES))
def test_host_program_matches_oracle(programs, name):
    d, built = programs
    fn, rs, masses, cut_legs = CASES[name]
    P = consistent(_points(rs, masses, cut_legs, 300, seed=7), (0.0, 0.0) + tuple(masses))
    assert P.shape[0] > 200
    exe, fields = built[name]
    got = _run(exe, _params(fields), P, d)
    ref = fn(P, PAR)
    assert np.all(np.abs(got[:, 0] - ref) <= _tolerance(fn, P, ref)), np.max(np.abs(got[:, 0] - ref) / _tolerance(fn, P, ref))
    assert np.median(np.abs(got[:, 0] / ref - 1)) <= 1e-12
    rel = np.abs(got[:, 1] / ref - 1)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())
    assert math.isfinite(float(got.sum()))


# processes checked in the helicity-loop form as well (massive fermions and vectors, massless
# polarisation vectors, the four-gluon and electroweak quartic vertices, complex couplings)
LOOP_CASES = ["g g > t t~ g", "u u~ > w+ w- a", "u d~ > w+ g g", "u s > d c h h", "g g > t t~ h", "u u > u u"]


@pytest.fixture(scope="module")
def loop_programs():
    from paper_1305_0708_gb300.compiler import dftables
    with tempfile.TemporaryDirectory() as d:
        with open(os.path.join(d, "dfloat_tables.h"), "w") as f:
            f.write(dftables.header())
        with ThreadPoolExecutor(max_workers=min(6, os.cpu_count() or 1)) as ex:
            built = dict(zip(LOOP_CASES, ex.map(lambda n: _build(n, d, hel_loop=True), LOOP_CASES)))
        yield d, built


@pytest.mark.parametrize("name", LOOP_CASES)
def test_helicity_loop_form_matches_oracle(loop_programs, name):
    """The helicity-loop form of the generated program (one copy of the diagrams, helicities from
    the live table at run time) at the tolerances of the straight-line form."""
    d, built = loop_programs
    fn, rs, masses, cut_legs = CASES[name]
    P = consistent(_points(rs, masses, cut_legs, 200, seed=9), (0.0, 0.0) + tuple(masses))
    exe, fields = built[name]
    got = _run(exe, _params(fields), P, d)
    ref = fn(P, PAR)
    assert np.all(np.abs(got[:, 0] - ref) <= _tolerance(fn, P, ref)), np.max(np.abs(got[:, 0] - ref) / _tolerance(fn, P, ref))
    assert np.median(np.abs(got[:, 0] / ref - 1)) <= 1e-12
    rel = np.abs(got[:, 1] / ref - 1)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())


@pytest.mark.parametrize("name", CMS_CASES)
def test_host_program_complex_mass_option(programs, name):
    """The same programs with the complex-mass parameter block (complex V V H, H H H, H H H H and
    t t H couplings, the W tied to the Z) against the oracle's complex-mass card; the same
    tolerances."""
    d, built = programs
    fn, rs, masses, cut_legs = CASES[name]
    cms = PAR.with_cms()
    P = consistent(_points(rs, masses, cut_legs, 200, seed=8), (0.0, 0.0) + tuple(masses))
    exe, fields = built[name]
    got = _run(exe, _params(fields, complex_mass=1), P, d)
    ref = fn(P, cms)
    tol = 1e-12 * np.abs(ref) + 32 * conditioning(fn, P, ref, cms, draws=3)
    assert np.all(np.abs(got[:, 0] - ref) <= tol), np.max(np.abs(got[:, 0] - ref) / tol)
    assert np.median(np.abs(got[:, 0] / ref - 1)) <= 1e-12
    rel = np.abs(got[:, 1] / ref - 1)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())
    # the option changes the result (not a no-op)
    assert np.median(np.abs(ref / fn(P, PAR) - 1)) > 1e-4


# points of the full-size workloads (seed, event) where FP32 amplitudes lost most: near-collinear
# b~ ve~ (or b ve) pairs from the top decays, a far off-shell W with both gluons backward
HARD_POINTS = {
    "udx_epvegg": [757858, 528462, 831301],
    "gg_ttx_dilep": [806363, 96860, 902978, 226505],
}


@pytest.mark.parametrize("key", list(HARD_POINTS))
def test_mixed_path_at_the_hardest_full_size_points(key):
    """The mixed program at the points of the 2^20-point workloads where it was worst (errors of
    1.2e-3 to 1.4e-3 before the resonant lines' FP32 momenta were taken from their double-float
    sums and the vanishing k k / m^2 terms dropped): within the 1e-3 bound against the oracle, and
    the FP64 program within 1e-12 plus the rounding-level spread."""
    from oracle import xsec as oxs
    from paper_1305_0708_gb300.workloads import WORKLOADS
    w = WORKLOADS[key]
    kin = {"udx_epvegg": {"kind": "rambo", "sqrt_s": 1000.0, "n_final": 4,
                          "cuts": {"legs": [2, 4, 5], "pt_min": 20.0, "eta_max": 2.5, "dr_min": 0.4}},
           "gg_ttx_dilep": {"kind": "ttbar", "sqrt_s_range": (400.0, 2000.0)}}[key]
    P, _, _, _ = oxs.generate(kin, PAR, w["seed"], np.array(HARD_POINTS[key]))
    fn = {"udx_epvegg": opr.udx_epvegg, "gg_ttx_dilep": opr.gg_ttx_dilep}[key]
    ref = fn(P, PAR)
    with tempfile.TemporaryDirectory() as d:
        from paper_1305_0708_gb300.compiler import dftables
        with open(os.path.join(d, "dfloat_tables.h"), "w") as f:
            f.write(dftables.header())
        exe, fields = _build(w["process"], d)
        got = _run(exe, _params(fields), P, d)
    assert np.all(np.abs(got[:, 0] - ref) <= _tolerance(fn, P, ref))
    rel = np.abs(got[:, 1] / ref - 1)
    assert rel.max() <= 1e-3, rel
