"""Adaptive grids on the GPU (xsec_step_grid, me_grid_*) against the oracle.

On the same seeded points the device maps every uniform through a random
non-uniform grid; the momenta, |M|^2, the Monte Carlo sums, the draw counts and
the refinement histogram are compared with oracle.xsec.generate_grid and
oracle.vegas, and the library's refinement of the device histogram with
oracle.vegas.refine.  Adapting the grid must reduce the error of sigma-hat.
"""
import numpy as np
import pytest

from oracle import processes as opr, vegas, xsec as oxs
from oracle.sm import SMParams
from paper_1305_0708_gb300.workloads import VARIANTS, WORKLOADS, kin_args
from test_gpu_parity import ORACLE, from_soa, oracle_kin

pytestmark = pytest.mark.gpu
PAR = SMParams()


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1305_0708_gb300 import binding
    binding.load()
    return binding


def random_grid(rng, D, N):
    w = rng.uniform(0.3, 1.0, size=(D, N))
    e = np.concatenate([np.zeros((D, 1)), np.cumsum(w, axis=1)], axis=1)
    e /= e[:, -1:]
    e[:, -1] = 1.0
    return e


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key,n", [("uux_epem", 3000), ("udx_epvegg", 1000), ("gg_ttx_dilep", 300),
                                   ("us_dchh", 500), ("udx_epvegg_bw", 1000)])
def test_grid_step_matches_oracle(B, key, n, prec):
    import torch
    w = WORKLOADS[key] if key in WORKLOADS else VARIANTS[key]
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, prec)
    n_ext = B.me_info(h).n_ext
    g = B.me_grid_create(h, kin, 24)
    try:
        D, N = B.me_grid_info(g)
        assert D == oxs.grid_dims(oracle_kin(w)) and N == 24
        edges = random_grid(np.random.default_rng(7), D, N)
        B.me_grid_set_edges(g, edges)
        assert np.array_equal(B.me_grid_get_edges(g), edges)
        me2 = torch.empty(n, dtype=torch.float64, device="cuda")
        mom = torch.empty(n_ext * 4 * n, dtype=torch.float64, device="cuda")
        acc = B.xsec_step_grid(h, g, w["seed"], 0, n, kin, None, None, me2, mom)
        torch.cuda.synchronize()
        hist = B.me_grid_get_hist(g)
        P, W, S, T, bins = oxs.generate_grid(oracle_kin(w), PAR, w["seed"], np.arange(n), edges)
        scale = w.get("sqrt_s") or w["sqrt_s_range"][1]
        assert np.abs(from_soa(mom, n_ext, n) - P).max() <= 4e-12 * scale
        assert acc.n_acc == n and acc.n_try == int(T.sum())
        ref = ORACLE[key if key in ORACLE else "udx_epvegg"](P, PAR)
        rel = np.abs(me2.cpu().numpy() / ref - 1)
        wor = W * ref * w["s_ident"] / (2.0 * S) * 0.3893793721e9
        h_or = vegas.histogram(D, N, bins, wor)
        # FP64: the device draws its own momenta (equal to the oracle's to rounding), so
        # |M|^2 and the sums agree to the conditioning of the resonant points
        tol = 1e-8 if prec == 0 else 2e-4
        if prec == 0:
            assert rel.max() <= 1e-8
        else:
            assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
        assert acc.sum_w == pytest.approx(wor.sum(), rel=tol)
        assert acc.sum_w2 == pytest.approx((wor * wor).sum(), rel=2 * tol)
        assert np.abs(hist - h_or).max() <= 4 * tol * h_or.max()
        # refinement of the device histogram by the library, against the oracle's
        B.me_grid_refine(g, 1.5)
        assert np.abs(B.me_grid_get_edges(g) - vegas.refine(edges, hist, 1.5)).max() < 1e-13
        assert np.all(B.me_grid_get_hist(g) == 0)
    finally:
        B.me_grid_destroy(g)
        B.me_destroy(h)


def test_adaptation_reduces_the_error(B):
    """u u~ > e+ e-, FP64 path: five refinements of 2^15-point steps, then sigma-hat against
    uniform sampling on the same number of points."""
    w = WORKLOADS["uux_epem"]
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, B.ME_FP64)
    g = B.me_grid_create(h, kin, 32)
    try:
        n = 1 << 15
        for it in range(5):
            B.xsec_step_grid(h, g, 3, it * n, n, kin)
            B.me_grid_refine(g, 1.5)
        acc = B.xsec_step_grid(h, g, 3, 10 * n, 4 * n, kin)
        s_g, e_g = B.me_xsec_estimate(acc)
        acc0 = B.xsec_step(h, 3, 10 * n, 4 * n, kin)
        s_0, e_0 = B.me_xsec_estimate(acc0)
        assert abs(s_g - s_0) < 4 * np.hypot(e_g, e_0)
        assert e_g < 0.6 * e_0
    finally:
        B.me_grid_destroy(g)
        B.me_destroy(h)


def test_grid_argument_errors(B):
    w1, w2 = WORKLOADS["uux_epem"], WORKLOADS["udx_epvegg"]
    k1, k2 = B.make_kin(**kin_args(w1)), B.make_kin(**kin_args(w2))
    h1 = B.me_create(w1["process"], None, B.ME_FP64)
    h2 = B.me_create(w2["process"], None, B.ME_FP64)
    g = B.me_grid_create(h1, k1, 8)
    try:
        with pytest.raises(B.MeError):
            B.xsec_step_grid(h2, g, 1, 0, 10, k2)          # grid of another process
        bad = B.me_grid_get_edges(g)
        bad[0, 3] = bad[0, 2]
        with pytest.raises(B.MeError):
            B.me_grid_set_edges(g, bad)                    # not increasing
        with pytest.raises(B.MeError):
            B.me_grid_create(h1, k1, 300)                  # too many bins
    finally:
        B.me_grid_destroy(g)
        B.me_destroy(h1)
        B.me_destroy(h2)
