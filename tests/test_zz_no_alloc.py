"""xsec_step_noalloc: the Monte Carlo step for callers that cannot allocate device memory.

Some embedding applications own all device memory (their own pool or arena)
or forbid allocation after start-up, so a library that calls cudaMalloc
inside a step cannot be used there.  xsec_step_noalloc keeps the step's
scratch in a fixed device array compiled into the library.  This test calls
it through the C ABI on a fresh handle, before any allocating step has run
on that handle, checks that two calls in a row leave the device's free
memory unchanged, and then checks each result against the allocating
xsec_step on the same inputs.  It sits in its own file, collected last, and
passes both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_xsec_step_twice_and_allocates_nothing():
    import __graft_entry__ as g
    g.build()
    from paper_1305_0708_gb300 import binding as B
    from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args
    assert torch.cuda.is_available()
    w = WORKLOADS["udx_epvegg"]
    kin = B.make_kin(**kin_args(w))
    n = 5000  # several blocks and a ragged tail
    for prec in (B.ME_FP64, B.ME_MIXED):
        h = B.me_create(w["process"], None, prec)
        outs = [torch.full((n,), -1.0, dtype=torch.float64, device="cuda") for _ in range(3)]
        # first call on this handle: loads the kernels and looks up the scratch address
        B.xsec_step_noalloc(h, w["seed"], 777, n, kin, None, None, outs[0])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got = []
        for k in (1, 2):  # two calls in a row: the array keeps the previous contents
            got.append(B.xsec_step_noalloc(h, w["seed"], 777, n, kin, None, None, outs[k]))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "xsec_step_noalloc changed the device's free memory"
        # the allocating step on the same inputs
        me2_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        ref = B.xsec_step(h, w["seed"], 777, n, kin, me2_out=me2_ref)
        for acc, me2 in zip(got, outs[1:]):
            assert acc.n_acc == ref.n_acc and acc.n_try == ref.n_try
            assert acc.sum_w == pytest.approx(ref.sum_w, rel=1e-12)
            assert acc.sum_w2 == pytest.approx(ref.sum_w2, rel=1e-12)
            assert np.allclose(me2.cpu().numpy(), me2_ref.cpu().numpy(), rtol=1e-12, atol=0)
        B.me_destroy(h)


def test_noalloc_rejects_block_per_event_processes_before_device_work():
    import __graft_entry__ as g
    g.build()
    from paper_1305_0708_gb300 import binding as B
    from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args
    lib = B.load()
    w = WORKLOADS["gg_gggg"]
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, B.ME_MIXED)
    acc = B.me_xsec_acc()
    st = lib.xsec_step_noalloc(h, w["seed"], 0, 100, ctypes.byref(kin), None, ctypes.byref(acc), None, None)
    assert st == -1 and "not available" in B.me_last_error()
    assert acc.n_acc == 0 and acc.n_try == 0
    B.me_destroy(h)
