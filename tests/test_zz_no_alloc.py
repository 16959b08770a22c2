"""xsec_step_noalloc: the Monte Carlo step for callers that cannot allocate device memory.

Some embedding applications own all device memory (their own pool or arena)
or forbid allocation after start-up, so a library that calls cudaMalloc
inside a step cannot be used there.  xsec_step_noalloc keeps the step's
scratch in a fixed device array compiled into the library.  This test calls
it through the C ABI twice in a row and checks each result against the
allocating xsec_step on the same inputs.  It sits in its own file, collected
last, and passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_xsec_step_twice():
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
        ref = B.xsec_step(h, w["seed"], 777, n, kin)
        me2_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        B.xsec_step(h, w["seed"], 777, n, kin, me2_out=me2_ref)
        for _ in range(2):  # two calls in a row: the array keeps the previous contents
            me2 = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            got = B.xsec_step_noalloc(h, w["seed"], 777, n, kin, None, None, me2)
            assert got.n_acc == ref.n_acc and got.n_try == ref.n_try
            assert got.sum_w == pytest.approx(ref.sum_w, rel=1e-12)
            assert got.sum_w2 == pytest.approx(ref.sum_w2, rel=1e-12)
            assert np.allclose(me2.cpu().numpy(), me2_ref.cpu().numpy(), rtol=1e-12, atol=0)
        B.me_destroy(h)
