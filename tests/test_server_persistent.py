"""Request server results against the FP64 oracle, and the persistent lanes (include/me_server.h).

- Sampled points of requests served alone and in a mix, in both scheduling modes, recomputed one by
  one by the oracle on the momenta the server returned (Eq. 4 is the quantity served).
- Persistent mode: results equal xsec_step's, are bit-identical alone and in a mix, and the lanes'
  kernels ran as captured graphs.
- A persistent kernel whose feeder stalls (host-side failure injection: the scheduler publishes no
  work and never closes the queue) gives up after its wait limit; the request fails with
  ME_ERR_TIMEOUT and the device stays usable.
"""
import numpy as np
import pytest

from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args

pytestmark = pytest.mark.gpu


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


def kin(B, key):
    return B.make_kin(**kin_args(WORKLOADS[key]))


def n_ext(key):
    from paper_1305_0708_gb300.compiler.diagrams import parse
    return len(parse(WORKLOADS[key]["process"]).particles)


def check_against_oracle(key, prec, me2, mom, n, k=96):
    """k points of a request recomputed by the oracle on the returned momenta."""
    from oracle.sm import SMParams
    from test_gpu_parity import ORACLE, fp64_tolerance
    par = SMParams()
    idx = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(n).choice(n, k - 2, replace=False)]))
    P = mom.reshape(n_ext(key), 4, n)[:, :, idx].transpose(2, 0, 1).copy()
    ref = ORACLE[key](P, par)
    got = me2[idx]
    if prec == 0:
        assert np.all(np.abs(got - ref) <= fp64_tolerance(ORACLE[key], P, ref))
    else:
        rel = np.abs(got / ref - 1)
        assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3, (np.median(rel), rel.max())


@pytest.mark.parametrize("persistent", [0, 1])
def test_server_results_against_the_oracle_alone_and_in_a_mix(B, persistent):
    s = B.me_server_create(n_slots=4, persistent=persistent)
    try:
        cases = [("udx_epvegg", B.ME_MIXED, 30000), ("us_dchh", B.ME_FP64, 20000), ("gg_ttx_dilep", B.ME_MIXED, 20000)]
        out = {}
        for alone in (True, False):
            tickets = []
            if not alone:  # other requests around them
                for i, k in enumerate(("uux_epem", "udx_epvegg", "gg_ttx_dilep", "us_dchh")):
                    tickets.append(B.me_server_submit(s, WORKLOADS[k]["process"], B.ME_MIXED, 50 + i, 0, 25000,
                                                      kin(B, k)))
            mine = []
            for i, (key, prec, n) in enumerate(cases):
                me2, mom = np.empty(n), np.empty(n_ext(key) * 4 * n)
                t = B.me_server_submit(s, WORKLOADS[key]["process"], prec, 9 + i, 1000, n, kin(B, key),
                                       want_me2=True, want_momenta=True)
                mine.append((key, prec, n, t, me2, mom))
            for key, prec, n, t, me2, mom in mine:
                res = B.me_server_wait(s, t, 300.0, me2, mom)
                assert res.status == 0
                check_against_oracle(key, prec, me2, mom, n)
                out.setdefault((key, prec), []).append((me2.copy(), res.acc.sum_w, res.acc.n_try))
            for t in tickets:
                assert B.me_server_wait(s, t, 300.0).status == 0
        for v in out.values():
            assert np.array_equal(v[0][0], v[1][0]) and v[0][1] == v[1][1] and v[0][2] == v[1][2]
    finally:
        B.me_server_destroy(s)


def test_persistent_lanes_agree_with_xsec_step_and_run_as_graphs(B):
    import torch
    s = B.me_server_create(n_slots=4, persistent=1)
    try:
        for key, prec, n in (("udx_epvegg", B.ME_MIXED, 70001), ("gg_ttx_dilep", B.ME_FP64, 9000),
                             ("uux_epem", B.ME_MIXED, 1)):
            w = WORKLOADS[key]
            tile = B.me_server_warm(s, w["process"], prec, kin(B, key))
            assert tile % 128 == 0 and tile >= 256
            me2 = np.empty(n)
            t = B.me_server_submit(s, w["process"], prec, 21, 333, n, kin(B, key), want_me2=True)
            res = B.me_server_wait(s, t, 300.0, me2)
            assert res.status == 0 and res.chunk == tile
            h = B.me_create(w["process"], None, prec)
            ref = torch.empty(n, dtype=torch.float64, device="cuda")
            acc = B.xsec_step(h, 21, 333, n, kin(B, key), None, None, ref)
            torch.cuda.synchronize()
            B.me_destroy(h)
            assert np.allclose(me2, ref.cpu().numpy(), rtol=1e-12, atol=0)
            assert res.acc.n_acc == n and res.acc.n_try == acc.n_try
            assert res.acc.sum_w == pytest.approx(acc.sum_w, rel=1e-12)
            assert res.acc.sum_w2 == pytest.approx(acc.sum_w2, rel=1e-12)
        st = B.me_server_get_stats(s)
        assert st.lane_launches >= 1 and st.lane_items >= 1 and st.lane_timeouts == 0
        assert st.graph_launches >= st.lane_launches  # the lanes' kernels started as captured graphs
        assert st.completed == st.submitted and st.active == 0
    finally:
        B.me_server_destroy(s)


def test_persistent_kernel_wait_limit_fails_the_request_not_the_device(B):
    import torch
    s = B.me_server_create(n_slots=2, persistent=1, spin_limit_us=20000, inject_feeder_stall=1)
    try:
        key = "udx_epvegg"
        B.me_server_warm(s, WORKLOADS[key]["process"], B.ME_MIXED, kin(B, key))
        t = B.me_server_submit(s, WORKLOADS[key]["process"], B.ME_MIXED, 1, 0, 5000, kin(B, key))
        with pytest.raises(B.MeError) as ei:
            B.me_server_wait(s, t, 120.0)
        assert ei.value.status == -5  # ME_ERR_TIMEOUT
        st = B.me_server_get_stats(s)
        assert st.lane_timeouts == 1 and st.completed == 1
    finally:
        B.me_server_destroy(s)
    # the context is still usable
    w = WORKLOADS[key]
    h = B.me_create(w["process"], None, B.ME_MIXED)
    acc = B.xsec_step(h, 1, 0, 5000, kin(B, key))
    torch.cuda.synchronize()
    B.me_destroy(h)
    assert acc.n_acc == 5000 and acc.sum_w > 0
