"""me_eval_host (|M|^2 for host buffers) against me_eval on device buffers.

Both host paths -- page-locked mapped memory read by the kernel directly, and
pageable memory staged through the handle's two device buffers in chunks of
2^17 points -- must give |M|^2 bit-identical to me_eval on the same momenta, on
both precisions, for sizes that span several chunks with a ragged tail.  The
momenta are the device generator's own points (their parity with the oracle is
tested in test_gpu_parity).
"""
import numpy as np
import pytest

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


def _points(B, key, n):
    from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args
    w = WORKLOADS[key]
    h = B.me_create(w["process"], None, B.ME_FP64)
    n_ext = B.me_info(h).n_ext
    mom = torch.empty(n_ext * 4 * n, dtype=torch.float64, device="cuda")
    B.me_generate(h, w["seed"], 5, n, B.make_kin(**kin_args(w)), mom)
    torch.cuda.synchronize()
    B.me_destroy(h)
    return w["process"], mom


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key,n", [("udx_epvegg", 3 * (1 << 17) + 4321), ("uux_epem", 1000), ("gg_ttx_dilep", 1 << 17)])
def test_host_paths_equal_device_path(B, key, n, prec):
    proc, mom = _points(B, key, n)
    h = B.me_create(proc, None, prec)
    try:
        ref = torch.empty(n, dtype=torch.float64, device="cuda")
        B.me_eval(h, mom, n, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        # page-locked (mapped) host memory
        mom_p = mom.cpu().pin_memory()
        out_p = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
        B.me_eval_host(h, mom_p, n, out_p)
        assert np.array_equal(out_p.numpy(), ref)
        # pageable host memory: the staged chunk pipeline
        mom_n = np.ascontiguousarray(mom.cpu().numpy())
        out_n = np.full(n, -1.0)
        B.me_eval_host(h, mom_n.ctypes.data, n, out_n.ctypes.data)
        assert np.array_equal(out_n, ref)
        # a second call reuses the staging buffers
        out_n[:] = -1.0
        B.me_eval_host(h, mom_n.ctypes.data, n, out_n.ctypes.data)
        assert np.array_equal(out_n, ref)
    finally:
        B.me_destroy(h)


def test_host_entry_argument_errors(B):
    h = B.me_create("u u~ > e+ e-", None, B.ME_MIXED)
    try:
        d = torch.zeros(16, dtype=torch.float64, device="cuda")
        o = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(B.MeError):
            B.me_eval_host(h, d, 1, o)            # device buffers belong to me_eval
        with pytest.raises(B.MeError):
            B.me_eval_host(h, None, 1, None)
        with pytest.raises(B.MeError):
            B.me_eval_host(h, np.zeros(16).ctypes.data, -1, np.zeros(1).ctypes.data)
        B.me_eval_host(h, np.zeros(16).ctypes.data, 0, np.zeros(1).ctypes.data)  # n = 0: no-op
    finally:
        B.me_destroy(h)


@pytest.mark.parametrize("key,n,steps", [("udx_epvegg", 50000, 3), ("gg_ttx_dilep", (1 << 20) + 4097, 1)])
def test_async_steps_equal_synchronous_steps(B, key, n, steps):
    """xsec_step_async adds each step's fixed-order sums on the device: after the same steps the
    device accumulator equals the host accumulator of xsec_step exactly."""
    from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args
    w = WORKLOADS[key]
    kin = B.make_kin(**kin_args(w))
    h = B.me_create(w["process"], None, B.ME_MIXED)
    try:
        acc = B.me_xsec_acc()
        for s in range(steps):
            B.xsec_step(h, w["seed"], s * n, n, kin, None, acc)
        acc_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
        for s in range(steps):
            B.xsec_step_async(h, w["seed"], s * n, n, kin, acc_dev)
        torch.cuda.synchronize()
        a = acc_dev.cpu().numpy()
        assert a[0] == acc.sum_w and a[1] == acc.sum_w2 and a[2] == acc.n_try and a[3] == 0.0
        with pytest.raises(B.MeError):
            B.xsec_step_async(h, w["seed"], 0, 10, kin, np.zeros(4).ctypes.data)  # host accumulator
    finally:
        B.me_destroy(h)
