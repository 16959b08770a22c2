"""Request server (include/me_server.h): continuous batching on one GPU.

Results of a request do not depend on the other requests that share the GPU
with it: |M|^2 of every point and the Monte Carlo sums are bit-identical alone
and in a mix.  The server's results agree with xsec_step, the memory budget
holds, and oversized requests are refused.
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


def run_alone(B, s, key, prec, seed, off, n):
    me2 = np.empty(n)
    t = B.me_server_submit(s, WORKLOADS[key]["process"], prec, seed, off, n, kin(B, key), want_me2=True)
    res = B.me_server_wait(s, t, 300.0, me2)
    return res, me2


def test_server_agrees_with_xsec_step(B):
    import torch
    s = B.me_server_create()
    try:
        for key, n in (("udx_epvegg", 50000), ("gg_gggg", 3000)):
            w = WORKLOADS[key]
            res, me2 = run_alone(B, s, key, B.ME_MIXED, 11, 7000, n)
            assert res.status == 0 and res.done == 1
            h = B.me_create(w["process"], None, B.ME_MIXED)
            out = torch.empty(n, dtype=torch.float64, device="cuda")
            acc = B.xsec_step(h, 11, 7000, n, kin(B, key), None, None, out)
            torch.cuda.synchronize()
            B.me_destroy(h)
            ref = out.cpu().numpy()
            assert np.array_equal(me2, ref)  # per-point work does not depend on the chunking
            assert res.acc.n_acc == n and res.acc.n_try == acc.n_try
            assert res.acc.sum_w == pytest.approx(acc.sum_w, rel=1e-12)
            assert res.acc.sum_w2 == pytest.approx(acc.sum_w2, rel=1e-12)
    finally:
        B.me_server_destroy(s)


def test_alone_and_in_a_mix_are_identical(B):
    s = B.me_server_create(n_slots=4)
    try:
        for key in ("uux_epem", "udx_epvegg", "gg_ttx_dilep", "us_dchh", "gg_gggg"):
            B.me_server_warm(s, WORKLOADS[key]["process"], B.ME_MIXED, kin(B, key))
        probes = [("udx_epvegg", 5, 123, 70000), ("gg_gggg", 6, 0, 2500), ("gg_ttx_dilep", 7, 999, 40000)]
        alone = {p: run_alone(B, s, p[0], B.ME_MIXED, p[1], p[2], p[3]) for p in probes}
        # the same requests again, each arriving among others of every process and size
        rng = np.random.default_rng(4)
        keys = list(WORKLOADS)
        tickets, mine = [], {}
        for i in range(12):
            k = keys[i % len(keys)]
            n = int(rng.integers(1000, 60000)) if k != "gg_gggg" else int(rng.integers(200, 2000))
            tickets.append(B.me_server_submit(s, WORKLOADS[k]["process"], B.ME_MIXED, 100 + i, 0, n, kin(B, k)))
            if i % 4 == 1:
                p = probes[i // 4]
                buf = np.empty(p[3])
                mine[p] = (B.me_server_submit(s, WORKLOADS[p[0]]["process"], B.ME_MIXED, p[1], p[2], p[3],
                                              kin(B, p[0]), want_me2=True), buf)
        for t in tickets:
            assert B.me_server_wait(s, t, 300.0).status == 0
        for p, (t, buf) in mine.items():
            res = B.me_server_wait(s, t, 300.0, buf)
            r0, m0 = alone[p]
            assert np.array_equal(buf, m0), p
            assert (res.acc.sum_w, res.acc.sum_w2, res.acc.n_acc, res.acc.n_try) == \
                (r0.acc.sum_w, r0.acc.sum_w2, r0.acc.n_acc, r0.acc.n_try), p
        st = B.me_server_get_stats(s)
        assert st.completed == st.submitted and st.waiting == 0 and st.active == 0
        assert st.graph_launches == st.launches > 0  # every chunk ran as the slot's instantiated graph
    finally:
        B.me_server_destroy(s)


def test_memory_budget_and_refusal(B):
    cap = 1 << 30
    s = B.me_server_create(mem_cap_bytes=cap, n_slots=2)
    try:
        key = "uux_epem"
        proc = WORKLOADS[key]["process"]
        B.me_server_warm(s, proc, B.ME_MIXED, kin(B, key))
        # each request keeps 8 B of |M|^2 and 128 B of momenta per point: 2^21 points ~ 285 MB
        n = 1 << 21
        ts = [B.me_server_submit(s, proc, B.ME_MIXED, i, 0, n, kin(B, key), want_me2=True, want_momenta=True)
              for i in range(6)]
        for t in ts:
            assert B.me_server_wait(s, t, 300.0).status == 0
        st = B.me_server_get_stats(s)
        assert st.bytes_peak <= cap
        assert st.bytes_in_use < cap
        # a request that can never fit is refused at submit
        with pytest.raises(B.MeError) as ei:
            B.me_server_submit(s, proc, B.ME_MIXED, 0, 0, 1 << 30, kin(B, key), want_me2=True, want_momenta=True)
        assert ei.value.status == -4
        with pytest.raises(B.MeError):
            B.me_server_submit(s, "u u~ > z z z z z", B.ME_MIXED, 0, 0, 10, kin(B, key))
        with pytest.raises(B.MeError):
            B.me_server_wait(s, 10 ** 9, 0.0)
    finally:
        B.me_server_destroy(s)


def test_waiting_request_is_not_refused_while_results_are_uncollected(B):
    """Requests that wait for budget held by finished but uncollected requests are admitted once
    their clients collect them, not refused: the client collects nothing until everything that fits
    has finished, then waits for every ticket in order."""
    import time
    cap = 1 << 30
    s = B.me_server_create(mem_cap_bytes=cap, n_slots=2)
    try:
        key = "uux_epem"
        proc = WORKLOADS[key]["process"]
        B.me_server_warm(s, proc, B.ME_MIXED, kin(B, key))
        n = 1 << 21
        ts = [B.me_server_submit(s, proc, B.ME_MIXED, i, 0, n, kin(B, key), want_me2=True, want_momenta=True)
              for i in range(6)]
        time.sleep(2.0)  # the admitted requests finish; the rest wait for their budget
        for t in ts:
            assert B.me_server_wait(s, t, 300.0).status == 0
        assert B.me_server_get_stats(s).bytes_peak <= cap
    finally:
        B.me_server_destroy(s)


def test_fp64_requests_and_momenta(B):
    import torch
    s = B.me_server_create(n_slots=2)
    try:
        key, n = "gg_ttx_dilep", 20000
        w = WORKLOADS[key]
        me2, mom = np.empty(n), np.empty(8 * 4 * n)
        t = B.me_server_submit(s, w["process"], B.ME_FP64, 3, 50, n, kin(B, key), want_me2=True, want_momenta=True)
        res = B.me_server_wait(s, t, 300.0, me2, mom)
        assert res.status == 0 and res.t_done_ms >= res.t_start_ms >= res.t_admit_ms >= res.t_submit_ms
        h = B.me_create(w["process"], None, B.ME_FP64)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        mo = torch.empty(8 * 4 * n, dtype=torch.float64, device="cuda")
        B.xsec_step(h, 3, 50, n, kin(B, key), None, None, out, mo)
        torch.cuda.synchronize()
        B.me_destroy(h)
        assert np.array_equal(me2, out.cpu().numpy())
        assert np.array_equal(mom, mo.cpu().numpy())
    finally:
        B.me_server_destroy(s)
