"""The C-ABI library builds, loads and exports every entry point of include/*.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1305_0708_gb300 import binding
    return binding.load()


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(?:me_status|void|int32_t|const char \*)\s*\*?\s*(\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"me_create", "me_eval", "xsec_step", "me_generate", "me_info", "me_destroy", "me_server_create",
            "me_server_submit", "me_server_wait"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1305_0708_gb300 import binding
    assert set(binding.EXPORTS) == set(declared_functions())
    for n in binding.EXPORTS:
        assert callable(getattr(binding, n))


def test_registry_lists_the_workload_processes(lib):
    from paper_1305_0708_gb300 import binding
    from paper_1305_0708_gb300.workloads import WORKLOADS
    names = [binding.me_process_name(i) for i in range(binding.me_n_processes())]
    for w in WORKLOADS.values():
        assert w["process"] in names
    assert binding.me_process_name(-1) is None
    assert binding.me_process_name(len(names)) is None


def test_argument_errors_before_device_work(lib):
    from paper_1305_0708_gb300 import binding
    h = ctypes.c_void_p()
    assert lib.me_create(None, None, 0, ctypes.byref(h)) == -1
    assert lib.me_create(b"u d~ > e+ ve g g", None, 7, ctypes.byref(h)) == -1
    assert lib.me_create(b"u u~ > z z z z z", None, 0, ctypes.byref(h)) == -2
    assert "not compiled" in binding.me_last_error()
    assert lib.me_eval(None, None, 4, None, None) == -1
    assert lib.me_eval_host(None, None, 4, None, None) == -1
    assert lib.xsec_step_async(None, 0, 0, 1, None, None, None) == -1
    assert lib.me_info(None, None) == -1


def test_xsec_estimate_arithmetic(lib):
    from paper_1305_0708_gb300 import binding
    acc = binding.me_xsec_acc(sum_w=10.0, sum_w2=30.0, n_acc=5, n_try=10)
    s, e = binding.me_xsec_estimate(acc)
    assert s == pytest.approx(1.0)
    assert e == pytest.approx(((30.0 / 10 - 1.0) / 9) ** 0.5)
    with pytest.raises(binding.MeError):
        binding.me_xsec_estimate(binding.me_xsec_acc())


def test_server_struct_layouts_match_the_header(lib, tmp_path):
    """ctypes mirrors of the server structs have the C sizes (host compiler, no GPU)."""
    import shutil
    import subprocess
    from paper_1305_0708_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "me_server.h"\nint main(void){printf("%zu %zu %zu %zu %zu",'
                   'sizeof(me_kin), sizeof(me_request), sizeof(me_request_result), sizeof(me_server_stats),'
                   'sizeof(me_server_config));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(t) for t in (B.me_kin, B.me_request, B.me_request_result, B.me_server_stats,
                                       B.me_server_config)]
    assert got == want


def test_server_argument_errors_without_device_work(lib):
    from paper_1305_0708_gb300 import binding as B
    s = ctypes.c_void_p()
    assert lib.me_server_create(None, None) == -1
    cfg = B.me_server_config(0, 17, 0)
    assert lib.me_server_create(ctypes.byref(cfg), ctypes.byref(s)) == -1
    assert "n_slots" in B.me_last_error()
    t = ctypes.c_int64()
    assert lib.me_server_submit(None, None, ctypes.byref(t)) == -1
    assert lib.me_server_wait(None, 1, 0.0, None, None, None) == -1


def test_library_vegas_refinement_matches_the_oracle(lib):
    """The library's host refinement of an adaptive grid against oracle.vegas.refine (no GPU)."""
    import numpy as np
    from oracle import vegas
    from paper_1305_0708_gb300 import binding as B
    rng = np.random.default_rng(11)
    for D, N, alpha in ((1, 8, 1.0), (3, 16, 1.5), (15, 50, 0.7)):
        w = rng.uniform(0.2, 1.0, size=(D, N))
        e = np.concatenate([np.zeros((D, 1)), np.cumsum(w, axis=1)], axis=1)
        e /= e[:, -1:]
        h = rng.random((D, N)) ** 3
        h[0, : N // 3] = 0.0
        if D > 2:
            h[2] = 0.0
        got = B.me_vegas_refine_edges(e, h, alpha)
        ref = vegas.refine(e, h, alpha)
        assert np.abs(got - ref).max() < 1e-13
    with pytest.raises(B.MeError):
        B.me_vegas_refine_edges(e, h, -1.0)
