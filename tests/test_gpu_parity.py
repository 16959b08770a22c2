"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle, on the same seeded inputs.

Inputs given to me_eval are on shell and balanced to FP64 rounding (kinematics.consistent), so that
every evaluator reads the same masses and momenta whichever legs it takes them from.

Tolerances
  FP64 path   |gpu - oracle| <= 1e-12 |oracle| + 32 * kappa, where kappa is the
              oracle's own spread when its input momenta are perturbed at the
              rounding level (2^-52 relative): points near a resonance or with a
              large gauge cancellation are conditioned so that no FP64 program
              can agree better than that.  The median relative difference must
              still be below 1e-12.
  mixed path  relative difference: median <= 1e-5, max <= 1e-3.
  phase space draws per point (integer) bit-exact; momenta and weights
              within 1e-12 relative (FP64 with different rounding order).

With ME_PARITY_REPORT set to a file name, each comparison appends one JSON line (process, path,
median and max relative difference; FP64: the largest difference as a fraction of its tolerance and
the largest kappa relative to |M|^2).
"""
import json
import os

import numpy as np
import pytest

from kinematics import conditioning, consistent

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_1305_0708_gb300 import binding
    binding.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


from oracle import processes as opr, xsec as oxs  # noqa: E402
from oracle.sm import SMParams  # noqa: E402
from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args  # noqa: E402

PAR = SMParams()
ORACLE = {"uux_epem": opr.uux_epem, "udx_epvegg": opr.udx_epvegg, "gg_ttx_dilep": opr.gg_ttx_dilep,
          "us_dchh": opr.us_dchh, "gg_gggg": opr.gluons}


def oracle_kin(w):
    if w["kind"] == "two_body":
        k = {"kind": "2to2", "sqrt_s": w["sqrt_s"]}
    elif w["kind"] == "rambo":
        nf = len(opr_legs(w)) - 2
        k = {"kind": "rambo", "sqrt_s": w["sqrt_s"], "n_final": nf}
        if "masses" in w:
            k["masses"] = list(w["masses"][2:])
    elif w["kind"] == "rambo_bw":
        k = {"kind": "rambo_bw", "sqrt_s": w["sqrt_s"], "n_final": len(opr_legs(w)) - 2,
             "res_mass": w["res_mass"], "res_width": w["res_width"]}
    elif w["kind"] == "ypt":
        k = {"kind": "ypt", "sqrt_s": w["sqrt_s"], "n_final": len(opr_legs(w)) - 2, "objects": w["objects"]}
    else:
        k = {"kind": "ttbar", "sqrt_s_range": w["sqrt_s_range"]}
    if w.get("leg_class"):
        from paper_1305_0708_gb300.workloads import PAPER_CUTS
        k["paper_cuts"] = {"leg_class": list(w["leg_class"]), "thresholds": dict(PAPER_CUTS)}
    if w.get("cuts"):
        c = w["cuts"]
        k["cuts"] = {"legs": list(c["legs"]), "pt_min": c["pt_min"], "eta_max": c["eta_max"], "dr_min": c["dr_min"]}
    return k


def opr_legs(w):
    from paper_1305_0708_gb300.compiler.diagrams import parse
    return parse(w["process"]).particles


def soa(P):
    return torch.from_numpy(np.ascontiguousarray(P.transpose(1, 2, 0))).cuda()


def from_soa(t, n_ext, n):
    return t.cpu().numpy().reshape(n_ext, 4, n).transpose(2, 0, 1)


def fp64_tolerance(fn, P, ref):
    return 1e-12 * np.abs(ref) + 32 * conditioning(fn, P, ref, PAR)


def report(process, prec, got, ref, kappa=None):
    path = os.environ.get("ME_PARITY_REPORT")
    if not path:
        return
    rel = np.abs(got / ref - 1)
    rec = {"process": process, "path": "fp64" if prec == 0 else "mixed", "points": int(len(ref)),
           "median": float(np.median(rel)), "max": float(rel.max())}
    if kappa is not None:
        # the largest difference as a fraction of the point's FP64 tolerance 1e-12 |ref| + 32 kappa
        rec["max_diff_over_tolerance"] = float(np.max(np.abs(got - ref) / (1e-12 * np.abs(ref) + 32 * kappa)))
        rec["max_kappa_rel"] = float(np.max(kappa / np.abs(ref)))
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def masses_of(w, n_ext):
    return tuple(w.get("masses", (0.0,) * n_ext))


def eval_gpu(B, process, P, prec, params=None):
    n = P.shape[0]
    h = B.me_create(process, params, prec)
    out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    B.me_eval(h, soa(P), n, out)
    torch.cuda.synchronize()
    B.me_destroy(h)
    return out.cpu().numpy()


@pytest.mark.parametrize("key", list(WORKLOADS))
def test_me_eval_parity(B, key):
    """me_eval on oracle-generated points (several tiles and a ragged tail)."""
    w = WORKLOADS[key]
    n = {"gg_ttx_dilep": 400, "gg_gggg": 200}.get(key, 1000)
    P, _, _, _ = oxs.generate(oracle_kin(w), PAR, 99, np.arange(n))
    P = consistent(P, masses_of(w, P.shape[1]))
    ref = ORACLE[key](P, PAR)
    g64 = eval_gpu(B, w["process"], P, B.ME_FP64)
    tol = fp64_tolerance(ORACLE[key], P, ref)
    report(w["process"], 0, g64, ref, (tol - 1e-12 * np.abs(ref)) / 32)
    assert np.all(np.abs(g64 - ref) <= tol), np.max(np.abs(g64 - ref) / tol)
    assert np.median(np.abs(g64 / ref - 1)) < 1e-12
    g32 = eval_gpu(B, w["process"], P, B.ME_MIXED)
    report(w["process"], 1, g32, ref)
    rel = np.abs(g32 / ref - 1)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", list(WORKLOADS))
def test_generate_parity(B, key, prec):
    """On-device Philox + generator + cuts + redraws against the oracle's own generator
    (FP64 generator for the FP64 path; double-float RAMBO for the mixed path)."""
    w = WORKLOADS[key]
    n_ext = len(opr_legs(w))
    n, off = 3000, 12345
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    mom = torch.empty(n_ext * 4 * n, dtype=torch.float64, device="cuda")
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    sh = torch.empty(n, dtype=torch.float64, device="cuda")
    tries = torch.empty(n, dtype=torch.int32, device="cuda")
    B.me_generate(h, w["seed"], off, n, kin, mom, wt, sh, tries)
    torch.cuda.synchronize()
    B.me_destroy(h)
    P, W, S, T = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(off, off + n))
    assert np.array_equal(tries.cpu().numpy(), T)
    scale = w.get("sqrt_s", 2000.0)
    assert np.abs(from_soa(mom, n_ext, n) - P).max() <= 1e-12 * scale * 4
    assert np.allclose(wt.cpu().numpy(), W, rtol=1e-12, atol=0)
    assert np.allclose(sh.cpu().numpy(), S, rtol=1e-13, atol=0)


@pytest.mark.parametrize("key", ["uux_epem", "udx_epvegg"])
def test_xsec_step_parity(B, key):
    """Weights summed on the device against the oracle's accumulate on its own points."""
    w = WORKLOADS[key]
    n = 2000
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, B.ME_FP64)
    acc = B.xsec_step(h, w["seed"], 0, n, kin)
    acc = B.xsec_step(h, w["seed"], n, n, kin, acc=acc)
    B.me_destroy(h)
    P, W, S, T = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(2 * n))
    sw, sw2, nacc, ntry = oxs.accumulate(ORACLE[key](P, PAR), W, S, T, w["s_ident"])
    assert acc.n_acc == nacc == 2 * n
    assert acc.n_try == ntry
    assert acc.sum_w == pytest.approx(sw, rel=1e-11)
    assert acc.sum_w2 == pytest.approx(sw2, rel=1e-11)
    s_gpu = B.me_xsec_estimate(acc)
    s_or = oxs.estimate(sw, sw2, ntry)
    assert s_gpu[0] == pytest.approx(s_or[0], rel=1e-11) and s_gpu[1] == pytest.approx(s_or[1], rel=1e-8)


def test_five_gluons_parity(B):
    """g g > g g g through the colour-ordered block kernel, both paths."""
    from oracle import phasespace as ps
    n = 300
    u = ps.uniforms(11, np.arange(n), np.zeros(n), 12)
    pf, _ = ps.rambo_massless(1000.0, 3, u)
    P = np.zeros((n, 5, 4))
    P[:, 0], P[:, 1] = ps.incoming(1000.0, n)
    P[:, 2:] = pf
    P = consistent(P, (0.0,) * 5)
    ref = opr.gluons(P, par=PAR)
    g64 = eval_gpu(B, "g g > g g g", P, B.ME_FP64)
    tol = fp64_tolerance(opr.gluons, P, ref)
    report("g g > g g g", 0, g64, ref, (tol - 1e-12 * np.abs(ref)) / 32)
    assert np.all(np.abs(g64 - ref) <= tol)
    assert np.median(np.abs(g64 / ref - 1)) < 1e-12
    g32 = eval_gpu(B, "g g > g g g", P, B.ME_MIXED)
    report("g g > g g g", 1, g32, ref)
    rel = np.abs(g32 / ref - 1)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3


def test_edge_cases(B):
    w = WORKLOADS["udx_epvegg"]
    kin = B.make_kin(**kin_args(w))
    for prec in (B.ME_FP64, B.ME_MIXED):
        h = B.me_create(w["process"], None, prec)
        B.me_eval(h, None, 0, None)                        # empty batch: no-op
        acc = B.xsec_step(h, 1, 0, 0, kin)
        assert acc.n_acc == 0 and acc.n_try == 0
        for n in (1, 31, 129):                             # single point, ragged tails
            me2 = torch.empty(n, dtype=torch.float64, device="cuda")
            mom = torch.empty(24 * n, dtype=torch.float64, device="cuda")
            B.xsec_step(h, 1, 2 ** 40 + 7, n, kin, me2_out=me2, momenta_out=mom)
            P = from_soa(mom, 6, n)
            ref = opr.udx_epvegg(np.ascontiguousarray(P), PAR)
            tol = 1e-10 if prec == B.ME_FP64 else 1e-3
            assert np.allclose(me2.cpu().numpy(), ref, rtol=tol, atol=0)
        with pytest.raises(B.MeError):
            B.me_eval(h, None, 4, None)
        bad = B.make_kin(**dict(kin_args(w), cut_legs=(0, 4)))
        with pytest.raises(B.MeError):
            B.xsec_step(h, 1, 0, 10, bad)
        B.me_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", list(WORKLOADS))
def test_full_size_sampled(B, key, prec):
    """Every workload's full-size step (2^20 points; 65,536 for u u~ > e+ e-, 2^18 for six gluons and
    u s > d c h h) in the launch shape the benchmark uses, both paths: points sampled over the whole
    launch (first and last included) recomputed one by one by the oracle on the momenta the device
    produced, the device momenta against the oracle's generator, and (FP64 path) the total number of
    draws of every point against the oracle's generator."""
    w = WORKLOADS[key]
    n = w["n"]
    n_ext = len(opr_legs(w))
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    me2 = torch.empty(n, dtype=torch.float64, device="cuda")
    mom = torch.empty(n_ext * 4 * n, dtype=torch.float64, device="cuda")
    acc = B.xsec_step(h, w["seed"], 0, n, kin, me2_out=me2, momenta_out=mom)
    B.me_destroy(h)
    k = 24 if key == "gg_gggg" else 256
    idx = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(5).choice(n, k - 2, replace=False)]))
    Pg = mom.view(n_ext, 4, n)[:, :, torch.from_numpy(idx).cuda()].cpu().numpy().transpose(2, 0, 1).copy()
    P, _, _, _ = oxs.generate(oracle_kin(w), PAR, w["seed"], idx)
    assert np.abs(Pg - P).max() <= 4e-12 * w.get("sqrt_s", 2000.0)
    ref = ORACLE[key](Pg, PAR)
    got = me2.cpu().numpy()[idx]
    if prec == 0:
        tol = fp64_tolerance(ORACLE[key], Pg, ref)
        report(w["process"] + " (full-size step)", 0, got, ref, (tol - 1e-12 * np.abs(ref)) / 32)
        assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
        assert np.median(np.abs(got / ref - 1)) < 1e-12
        # total number of draws over all points: the oracle's generator alone (no |M|^2)
        _, _, _, Tall = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(n))
        assert acc.n_try == int(Tall.sum())
    else:
        report(w["process"] + " (full-size step)", 1, got, ref)
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())


# events of the full-size workloads where the mixed path was worst (seed of the workload)
HARD_POINTS = {"udx_epvegg": [757858, 528462, 831301], "gg_ttx_dilep": [806363, 96860, 902978, 226505]}


@pytest.mark.parametrize("key", list(HARD_POINTS))
def test_mixed_path_at_the_hardest_full_size_points(B, key):
    """me_eval at the points of the 2^20-point workloads where FP32 amplitudes lost most
    (near-collinear decay products of the tops; a far off-shell W with both gluons backward):
    mixed within 1e-3 of the oracle, FP64 within its tolerance."""
    w = WORKLOADS[key]
    P, _, _, _ = oxs.generate(oracle_kin(w), PAR, w["seed"], np.array(HARD_POINTS[key]))
    ref = ORACLE[key](P, PAR)
    g64 = eval_gpu(B, w["process"], P, B.ME_FP64)
    assert np.all(np.abs(g64 - ref) <= fp64_tolerance(ORACLE[key], P, ref))
    rel = np.abs(eval_gpu(B, w["process"], P, B.ME_MIXED) / ref - 1)
    assert rel.max() <= 1e-3, rel


@pytest.mark.parametrize("prec", [0, 1])
def test_resonance_generator_parity(B, prec):
    """The resonance-mapped generator (App. A.2) on the device against the oracle's: draws, momenta
    and weights; the FP64 path's Monte Carlo sums against the oracle's.  Mixed-path weights: the
    double-float massive rescaling divides by the resonance's massless RAMBO energy, which carries
    2^-48 of sqrt(s) (FP64: 2^-53), hence 5e-11 instead of 1e-12."""
    from paper_1305_0708_gb300.workloads import VARIANTS
    w = VARIANTS["udx_epvegg_bw"]
    n, off = 3000, 777
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    mom = torch.empty(24 * n, dtype=torch.float64, device="cuda")
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    sh = torch.empty(n, dtype=torch.float64, device="cuda")
    tries = torch.empty(n, dtype=torch.int32, device="cuda")
    B.me_generate(h, w["seed"], off, n, kin, mom, wt, sh, tries)
    me2 = torch.empty(n, dtype=torch.float64, device="cuda")
    acc = B.xsec_step(h, w["seed"], off, n, kin, None, None, me2)
    torch.cuda.synchronize()
    B.me_destroy(h)
    P, W, S, T = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(off, off + n))
    assert np.array_equal(tries.cpu().numpy(), T)
    assert np.abs(from_soa(mom, 6, n) - P).max() <= 4e-12 * w["sqrt_s"]
    assert np.allclose(wt.cpu().numpy(), W, rtol=1e-12 if prec == 0 else 5e-11, atol=0)
    ref = ORACLE["udx_epvegg"](P, PAR)
    sw, sw2, nacc, ntry = oxs.accumulate(ref, W, S, T, w["s_ident"])
    assert acc.n_try == ntry
    if prec == 0:
        assert acc.sum_w == pytest.approx(sw, rel=1e-11) and acc.sum_w2 == pytest.approx(sw2, rel=1e-11)
    else:
        rel = np.abs(me2.cpu().numpy() / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
        assert acc.sum_w == pytest.approx(sw, rel=1e-5)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", ["uux_wpwm", "udx_wpz"])
def test_ew_boson_pair_parity(B, key, prec):
    """u u~ > W+ W- and u d~ > W+ Z (electroweak triple-gauge vertices, massive external vectors):
    me_eval on the oracle's massive-RAMBO points and the Monte Carlo sums of xsec_step against the
    oracle's generate and accumulate."""
    import itertools
    from paper_1305_0708_gb300.workloads import VARIANTS
    w = VARIANTS[key]
    fn = {"uux_wpwm": opr.uux_wpwm, "udx_wpz": opr.udx_wpz}[key]
    amps = {"uux_wpwm": opr.uux_wpwm_amplitudes, "udx_wpz": opr.udx_wpz_amplitudes}[key]
    n = 1500
    P0, W, S, T = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(n))
    P = consistent(P0, masses_of(w, P0.shape[1]))
    ref = fn(P, PAR)
    got = eval_gpu(B, w["process"], P, prec)
    if prec == 0:
        # the diagrams cancel (gauge cancellation: their summed magnitudes squared are ~10^3 times
        # |M|^2), so FP64 rounding of the individual diagrams bounds the agreement: 64 roundings of
        # that scale beside the input-conditioning term
        scale = 0.0
        for h in itertools.product((-1, 1), (-1, 1), (-1, 0, 1), (-1, 0, 1)):
            scale = scale + sum(np.abs(a) for a in amps(P, h, PAR)) ** 2
        scale = scale * 3.0 / 36.0
        tol = fp64_tolerance(fn, P, ref) + 64 * 2.0 ** -52 * scale
        report(w["process"], 0, got, ref, (tol - 1e-12 * np.abs(ref)) / 32)
        assert np.all(np.abs(got - ref) <= tol)
        assert np.median(np.abs(got / ref - 1)) <= 1e-12
    else:
        report(w["process"], 1, got, ref)
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    acc = B.xsec_step(h, w["seed"], 0, n, kin)
    B.me_destroy(h)
    # the Monte Carlo sums: the oracle on its own generated points, as the device generates them
    sw, sw2, nacc, ntry = oxs.accumulate(fn(P0, PAR), W, S, T, w["s_ident"])
    assert acc.n_acc == nacc == n and acc.n_try == ntry
    tol = 1e-11 if prec == 0 else 1e-5
    assert acc.sum_w == pytest.approx(sw, rel=tol) and acc.sum_w2 == pytest.approx(sw2, rel=2 * tol)


@pytest.mark.parametrize("prec", [0, 1])
def test_identical_quarks_parity(B, prec):
    """u u > u u: gluon, photon and Z exchange in the t and u channels, whose relative minus sign the
    compiler's fermion-permutation sign must supply; me_eval on the oracle's two-body points at
    |cos theta| < 0.95 (away from the forward poles)."""
    n = 2000
    P, _, _, _ = oxs.generate({"kind": "2to2", "sqrt_s": 400.0}, PAR, 21, np.arange(n))
    P = consistent(P[np.abs(P[:, 2, 3] / P[:, 2, 0]) < 0.95], (0.0,) * 4)
    ref = opr.uu_uu(P, PAR)
    got = eval_gpu(B, "u u > u u", P, prec)
    if prec == 0:
        tol = fp64_tolerance(opr.uu_uu, P, ref)
        report("u u > u u", 0, got, ref, (tol - 1e-12 * np.abs(ref)) / 32)
        assert np.all(np.abs(got - ref) <= tol)
        assert np.median(np.abs(got / ref - 1)) <= 1e-12
    else:
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", ["uux_zz", "uux_zh", "udx_wph", "uux_wpwma", "gg_ttx", "gg_ttxh", "udx_wpg",
                                 "uux_zg", "ug_wpd", "uux_zzg", "gg_ttxg", "uux_zhg", "udx_wpzg",
                                 "uux_wpwmg", "gg_wpdux", "gg_zuux", "udx_wphg",
                                 "uux_ttx", "uux_ttxg", "us_dch", "udx_wpa",
                                 "uux_za", "uux_aa", "udx_wpgg", "uux_zgg", "us_dchg",
                                 "us_dchhh", "ud_udh", "ud_udhh", "ud_udhhh", "udx_wpggg", "uux_zggg", "gg_ttxhg", "us_dchgg", "uux_zzgg", "udx_wphgg", "uu_uuhh", "uu_uuhhh", "uux_wpwmgg", "udx_wpzgg", "udx_wphggg"])
def test_massive_final_state_parity(B, key, prec):
    """u u~ > Z Z (identical massive vectors, identical-particle factor 1/2), u u~ > Z H (ZZH vertex,
    external scalar), u d~ > W+ H (WWH vertex), u u~ > W+ W- gamma (the electroweak quartic
    vertices, VVV currents into massive W lines, photon pT and rapidity cuts), g g > t t~ (massive
    external spinors), u u~ > t t~ and u u~ > t t~ g (gluon, photon and Z exchange), g g > t t~ H (the FFS Yukawa vertex), u d~ > W+ g, u u~ > Z g, u g > W+ d and
    u u~ > Z Z g, u u~ > Z H g, u d~ > W+ H g, u d~ > W+ Z g, u u~ > W+ W- g (bosons plus one jet, jet cuts), g g > W+ d u~
    and g g > Z u u~ (V plus two jets from two gluons), u s > d c H (W+ W- fusion), u d~ > W+ gamma, u u~ > Z gamma, u u~ > gamma gamma and g g > t t~ g (the
    four-gluon vertex beside a top line), u s > d c H H H and u d > u d + 1, 2, 3 Higgs (weak-boson fusion,
    Sect. 2.10), u d~ > W+ g g g and u u~ > Z g g g (V plus three jets) and g g > t t~ H g (H t t~ plus a
    jet) and u u~ > Z Z g g (V V plus two jets), helicity-loop programs, u s > d c H g g (WBF H plus two
    jets), u d~ > W+ H g g and W+ H g g g (H V plus two and three jets), u u~ > W+ W- g g and u d~ > W+ Z g g (V V plus two jets) and u u > u u H H (H)
    (Z Z fusion, identical quarks): me_eval on the oracle's massive-RAMBO points and the Monte Carlo sums
    against the oracle."""
    from paper_1305_0708_gb300.workloads import VARIANTS
    w = VARIANTS[key]
    fn = {"uux_zz": opr.uux_zz, "uux_zh": opr.uux_zh, "udx_wph": opr.udx_wph, "uux_wpwma": opr.uux_wpwma,
          "gg_ttx": opr.gg_ttx, "gg_ttxh": opr.gg_ttxh, "udx_wpg": opr.udx_wpg, "uux_zg": opr.uux_zg,
          "ug_wpd": opr.ug_wpd, "uux_zzg": opr.uux_zzg, "gg_ttxg": opr.gg_ttxg, "uux_zhg": opr.uux_zhg,
          "udx_wpzg": opr.udx_wpzg, "uux_wpwmg": opr.uux_wpwmg, "gg_wpdux": opr.gg_wpdux,
          "gg_zuux": opr.gg_zuux, "udx_wphg": opr.udx_wphg,
          "uux_ttx": opr.uux_ttx, "uux_ttxg": opr.uux_ttxg, "us_dch": opr.us_dch, "udx_wpa": opr.udx_wpa,
          "uux_za": opr.uux_za, "uux_aa": opr.uux_aa, "udx_wpgg": opr.udx_wpgg, "uux_zgg": opr.uux_zgg,
          "us_dchg": opr.us_dchg, "us_dchhh": opr.us_dchhh, "ud_udh": opr.ud_udh, "ud_udhh": opr.ud_udhh,
          "ud_udhhh": opr.ud_udhhh, "udx_wpggg": opr.udx_wpggg, "uux_zggg": opr.uux_zggg,
          "gg_ttxhg": opr.gg_ttxhg, "us_dchgg": opr.us_dchgg, "uux_zzgg": opr.uux_zzgg,
          "udx_wphgg": opr.udx_wphgg, "uu_uuhh": opr.uu_uuhh, "uu_uuhhh": opr.uu_uuhhh,
          "uux_wpwmgg": opr.uux_wpwmgg, "udx_wpzgg": opr.udx_wpzgg, "udx_wphggg": opr.udx_wphggg}[key]
    n = {"udx_wpggg": 300, "uux_zggg": 300, "gg_ttxhg": 300, "uux_zzgg": 300, "uux_wpwmgg": 300,
         "udx_wpzgg": 300, "udx_wphggg": 300}.get(key, 1500)
    P0, W, S, T = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(n))
    P = consistent(P0, masses_of(w, P0.shape[1]))
    ref = fn(P, PAR)
    got = eval_gpu(B, w["process"], P, prec)
    if prec == 0:
        tol = fp64_tolerance(fn, P, ref)
        report(w["process"], 0, got, ref, (tol - 1e-12 * np.abs(ref)) / 32)
        assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
        assert np.median(np.abs(got / ref - 1)) <= 1e-12
    else:
        report(w["process"], 1, got, ref)
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    acc = B.xsec_step(h, w["seed"], 0, n, kin)
    B.me_destroy(h)
    # the Monte Carlo sums: the oracle on its own generated points, as the device generates them
    sw, sw2, nacc, ntry = oxs.accumulate(fn(P0, PAR), W, S, T, w["s_ident"])
    assert acc.n_acc == nacc == n and acc.n_try == ntry
    # mixed: a weighted sum's relative error is at most the largest per-point one, so the sums take
    # 1e-5 or twice the largest per-point error seen above, whichever is larger (a few dominant
    # weights among the 300 points of V + 3 jets put the sum of w^2 near that point's error)
    tol = 1e-11 if prec == 0 else max(1e-5, 2 * float(rel.max()))
    assert acc.sum_w == pytest.approx(sw, rel=tol) and acc.sum_w2 == pytest.approx(sw2, rel=2 * tol)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", ["us_dchh", "us_dchhh", "ud_udhhh", "gg_ttxh", "uux_zh"])
def test_complex_mass_option_parity(B, key, prec):
    """The complex-mass option of Sect. 7.11 (me_params.complex_mass = 1: complex V V H, H H H, H H H H
    and t t H couplings, the W tied to the Z) against the oracle's complex-mass card: me_eval per point
    and the Monte Carlo sums, at the tolerances of the fixed-width runs."""
    from paper_1305_0708_gb300.workloads import VARIANTS, WORKLOADS
    w = {**WORKLOADS, **VARIANTS}[key]
    fn = {"us_dchh": opr.us_dchh, "us_dchhh": opr.us_dchhh, "ud_udhhh": opr.ud_udhhh, "gg_ttxh": opr.gg_ttxh,
          "uux_zh": opr.uux_zh}[key]
    cms = PAR.with_cms()
    prm = B.make_params(complex_mass=1)
    n = 1200
    P0, W, S, T = oxs.generate(oracle_kin(w), cms, w["seed"], np.arange(n))
    P = consistent(P0, masses_of(w, P0.shape[1]))
    ref = fn(P, cms)
    got = eval_gpu(B, w["process"], P, prec, prm)
    if prec == 0:
        tol = 1e-12 * np.abs(ref) + 32 * conditioning(fn, P, ref, cms)
        report(w["process"] + " (complex mass)", 0, got, ref, (tol - 1e-12 * np.abs(ref)) / 32)
        assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
        assert np.median(np.abs(got / ref - 1)) <= 1e-12
    else:
        report(w["process"] + " (complex mass)", 1, got, ref)
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], prm, prec)
    acc = B.xsec_step(h, w["seed"], 0, n, kin)
    B.me_destroy(h)
    sw, sw2, nacc, ntry = oxs.accumulate(fn(P0, cms), W, S, T, w["s_ident"])
    assert acc.n_acc == nacc == n and acc.n_try == ntry
    tol = 1e-11 if prec == 0 else 1e-5
    assert acc.sum_w == pytest.approx(sw, rel=tol) and acc.sum_w2 == pytest.approx(sw2, rel=2 * tol)


@pytest.mark.parametrize("prec", [0, 1])
def test_scalar_quartic_parity(B, prec):
    """h h > h h (the SSSS contact vertex beside s-, t- and u-channel Higgs exchange through SSS):
    me_eval on massive incoming and outgoing Higgs bosons from threshold to 3 TeV, against the
    oracle (no generator takes massive beams, so there is no Monte Carlo leg)."""
    import math
    n = 700
    rng = np.random.default_rng(51)
    rs = rng.uniform(255.0, 3000.0, n)
    c = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2 * np.pi, n)
    m = PAR.mH
    P = np.zeros((n, 4, 4))
    pin = np.sqrt(rs * rs / 4 - m * m)
    P[:, 0] = np.stack([rs / 2, 0 * rs, 0 * rs, pin], axis=1)
    P[:, 1] = np.stack([rs / 2, 0 * rs, 0 * rs, -pin], axis=1)
    nv = np.stack([np.sqrt(1 - c * c) * np.cos(phi), np.sqrt(1 - c * c) * np.sin(phi), c], axis=1)
    P[:, 2, 0] = P[:, 3, 0] = rs / 2
    P[:, 2, 1:] = pin[:, None] * nv
    P[:, 3, 1:] = -pin[:, None] * nv
    ref = opr.hh_hh(P, PAR)
    got = eval_gpu(B, "h h > h h", P, prec)
    if prec == 0:
        tol = fp64_tolerance(opr.hh_hh, P, ref)
        report("h h > h h", 0, got, ref, (tol - 1e-12 * np.abs(ref)) / 32)
        assert np.all(np.abs(got - ref) <= tol)
        assert np.median(np.abs(got / ref - 1)) <= 1e-12
    else:
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
    assert math.isfinite(float(got.sum()))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", ["udx_epvegg_ypt", "gg_gggg_ypt"])
def test_paper_parametrisation_parity(B, key, prec):
    """The paper's y, pT, phi parametrisation (Eq. 13, App. A.1, Eq. 17, App. A.2) with its cuts
    (Eqs. 8-11) on the device against the oracle's: draws per point bit-exact, momenta within
    4e-12 sqrt(s), weights within 1e-12 (the generator runs in FP64 on both paths); the Monte Carlo
    sums against the oracle's accumulate."""
    from paper_1305_0708_gb300.workloads import PAPER_PS
    w = PAPER_PS[key]
    n_ext = len(opr_legs(w))
    n, off = 600 if key == "gg_gggg_ypt" else 2000, 4242
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    mom = torch.empty(n_ext * 4 * n, dtype=torch.float64, device="cuda")
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    sh = torch.empty(n, dtype=torch.float64, device="cuda")
    tries = torch.empty(n, dtype=torch.int32, device="cuda")
    B.me_generate(h, w["seed"], off, n, kin, mom, wt, sh, tries)
    me2 = torch.empty(n, dtype=torch.float64, device="cuda")
    mom2 = torch.empty(n_ext * 4 * n, dtype=torch.float64, device="cuda")
    acc = B.xsec_step(h, w["seed"], off, n, kin, None, None, me2, mom2)
    torch.cuda.synchronize()
    with pytest.raises(B.MeError):  # the fused allocation-free step does not compile this generator
        B.xsec_step_noalloc(h, w["seed"], off, n, kin)
    B.me_destroy(h)
    P, W, S, T = oxs.generate(oracle_kin(w), PAR, w["seed"], np.arange(off, off + n))
    assert np.array_equal(tries.cpu().numpy(), T)
    assert np.abs(from_soa(mom, n_ext, n) - P).max() <= 4e-12 * w["sqrt_s"]
    assert np.abs(from_soa(mom2, n_ext, n) - P).max() <= 4e-12 * w["sqrt_s"]
    assert np.allclose(wt.cpu().numpy(), W, rtol=1e-12, atol=0)
    fn = ORACLE["udx_epvegg" if key == "udx_epvegg_ypt" else "gg_gggg"]
    sw, sw2, nacc, ntry = oxs.accumulate(fn(P, PAR), W, S, T, w["s_ident"])
    assert acc.n_acc == nacc == n and acc.n_try == ntry
    if prec == 0:
        # point by point on these points made consistent to rounding (the generated ones conserve
        # momentum to ~1e-14 of sqrt(s) only), then the sums
        Pc = consistent(P, (0.0,) * n_ext)
        ref = fn(Pc, PAR)
        got = eval_gpu(B, w["process"], Pc, 0)
        assert np.all(np.abs(got - ref) <= fp64_tolerance(fn, Pc, ref))
        assert acc.sum_w == pytest.approx(sw, rel=1e-11) and acc.sum_w2 == pytest.approx(sw2, rel=1e-11)
    else:
        Pg = from_soa(mom2, n_ext, n).copy()
        rel = np.abs(me2.cpu().numpy() / fn(Pg, PAR) - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
        # a sum of a few hundred heavy-tailed weights carries the relative error of its largest
        # terms (six gluons: up to ~2e-5 per point there)
        assert acc.sum_w == pytest.approx(sw, rel=1e-4)
