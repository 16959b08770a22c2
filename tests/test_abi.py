"""The C-ABI library builds, loads and exports every entry point of include/me.h (no GPU needed)."""
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
    src = open(os.path.join(ROOT, "include", "me.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:me_status|void|int32_t|const char \*)\s*\*?\s*(\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"me_create", "me_eval", "xsec_step", "me_generate", "me_info", "me_destroy"} <= set(names)
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
    assert lib.me_info(None, None) == -1


def test_xsec_estimate_arithmetic(lib):
    from paper_1305_0708_gb300 import binding
    acc = binding.me_xsec_acc(sum_w=10.0, sum_w2=30.0, n_acc=5, n_try=10)
    s, e = binding.me_xsec_estimate(acc)
    assert s == pytest.approx(1.0)
    assert e == pytest.approx(((30.0 / 10 - 1.0) / 9) ** 0.5)
    with pytest.raises(binding.MeError):
        binding.me_xsec_estimate(binding.me_xsec_acc())
