"""Thin ctypes binding of the C ABI (include/me.h, include/me_server.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device buffers
may be given as torch CUDA tensors (their data pointer is passed) or raw
integer addresses; streams as torch.cuda.Stream, a raw handle or None.
Nothing here computes: every step runs in the library's kernels.  If the
library is missing the import fails loudly; there is no fallback.
"""
import ctypes
import os

from . import build as _build

_LIB = None


class MeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"me status {status}: {msg}")
        self.status = status


class me_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("alpha", "sw2", "mZ", "wZ", "mW", "wW", "alpha_s", "mt", "wt", "mH", "wH")] + [
        ("complex_mass", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class me_kin(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("max_attempts", ctypes.c_int32), ("sqrt_s", ctypes.c_double),
                ("sqrt_s_min", ctypes.c_double), ("sqrt_s_max", ctypes.c_double), ("mass", ctypes.c_double * 16),
                ("n_cut_legs", ctypes.c_int32), ("cut_legs", ctypes.c_int32 * 8), ("pt_min", ctypes.c_double),
                ("eta_max", ctypes.c_double), ("dr_min", ctypes.c_double), ("s_ident", ctypes.c_double),
                ("res_mass", ctypes.c_double), ("res_width", ctypes.c_double),
                ("n_obj", ctypes.c_int32), ("cut_mode", ctypes.c_int32), ("obj_legs", (ctypes.c_int32 * 2) * 8),
                ("leg_class", ctypes.c_int32 * 16), ("obj_mass", ctypes.c_double * 8),
                ("obj_res_mass", ctypes.c_double * 8), ("obj_res_width", ctypes.c_double * 8),
                ("obj_y_max", ctypes.c_double * 8), ("obj_pt_min", ctypes.c_double * 8),
                ("obj_pt_max", ctypes.c_double * 8), ("jet_pt", ctypes.c_double), ("jet_eta", ctypes.c_double),
                ("jet_ptij", ctypes.c_double), ("b_pt", ctypes.c_double), ("b_eta", ctypes.c_double),
                ("lep_pt", ctypes.c_double), ("lep_eta", ctypes.c_double)]


class me_xsec_acc(ctypes.Structure):
    _fields_ = [("sum_w", ctypes.c_double), ("sum_w2", ctypes.c_double), ("n_acc", ctypes.c_int64),
                ("n_try", ctypes.c_int64)]


class me_info_t(ctypes.Structure):
    _fields_ = [("n_ext", ctypes.c_int32), ("n_hel", ctypes.c_int32), ("n_hel_live", ctypes.c_int32),
                ("n_colour", ctypes.c_int32), ("n_diagrams", ctypes.c_int32), ("pdg", ctypes.c_int32 * 16),
                ("flops_amp", ctypes.c_double), ("flops_fp64", ctypes.c_double),
                ("flops_colour", ctypes.c_double)]


class me_server_config(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_uint64), ("n_slots", ctypes.c_int32), ("max_requests", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("spin_limit_us", ctypes.c_int32),
                ("inject_feeder_stall", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class me_request(ctypes.Structure):
    _fields_ = [("process", ctypes.c_char_p), ("precision", ctypes.c_int32), ("want_me2", ctypes.c_int32),
                ("want_momenta", ctypes.c_int32), ("pad_", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("counter_offset", ctypes.c_uint64), ("n", ctypes.c_int64), ("kin", me_kin)]


class me_request_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("acc", me_xsec_acc),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("chunk", ctypes.c_int64)]


class me_server_stats(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64),
                ("bytes_peak", ctypes.c_uint64), ("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("waiting", ctypes.c_int64), ("active", ctypes.c_int64),
                ("points_done", ctypes.c_int64), ("launches", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("lane_launches", ctypes.c_int64), ("lane_items", ctypes.c_int64), ("lane_timeouts", ctypes.c_int64)]


ME_FP64, ME_MIXED = 0, 1
ME_PS_TWO_BODY, ME_PS_RAMBO, ME_PS_TTBAR, ME_PS_RAMBO_BW, ME_PS_YPT = 0, 1, 2, 3, 4

EXPORTS = ["me_create", "me_eval", "me_eval_host", "me_generate", "xsec_step", "xsec_step_async", "xsec_step_noalloc", "me_step_timing",
           "me_xsec_estimate", "me_info", "me_n_processes", "me_process_name", "me_destroy", "me_last_error",
           "me_server_create", "me_server_warm", "me_server_submit", "me_server_poll", "me_server_wait",
           "me_server_get_stats", "me_server_destroy", "me_grid_create", "me_grid_info", "me_grid_get_edges",
           "me_grid_set_edges", "me_grid_get_hist", "me_grid_clear_hist", "me_grid_refine", "xsec_step_grid",
           "me_grid_destroy", "me_vegas_refine_edges"]


def lib_path():
    return _build.LIB


def load(path=None):
    """Load libme.so (built by build.build()); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libme.so not built at {path}: run paper_1305_0708_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
    L.me_create.argtypes = [ctypes.c_char_p, ctypes.POINTER(me_params), i32, ctypes.POINTER(vp)]
    L.me_eval.argtypes = [vp, vp, i64, vp, vp]
    L.me_eval_host.argtypes = [vp, vp, i64, vp, vp]
    L.me_generate.argtypes = [vp, u64, u64, i64, ctypes.POINTER(me_kin), vp, vp, vp, vp, vp]
    L.xsec_step.argtypes = [vp, u64, u64, i64, ctypes.POINTER(me_kin), vp, ctypes.POINTER(me_xsec_acc), vp, vp]
    L.xsec_step_async.argtypes = [vp, u64, u64, i64, ctypes.POINTER(me_kin), vp, vp]
    L.xsec_step_noalloc.argtypes = [vp, u64, u64, i64, ctypes.POINTER(me_kin), vp, ctypes.POINTER(me_xsec_acc),
                                    vp, vp]
    L.me_step_timing.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.me_xsec_estimate.argtypes = [ctypes.POINTER(me_xsec_acc), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
    L.me_info.argtypes = [vp, ctypes.POINTER(me_info_t)]
    L.me_n_processes.restype = i32
    L.me_process_name.argtypes = [i32]
    L.me_process_name.restype = ctypes.c_char_p
    L.me_destroy.argtypes = [vp]
    L.me_destroy.restype = None
    L.me_last_error.restype = ctypes.c_char_p
    L.me_server_create.argtypes = [ctypes.POINTER(me_server_config), ctypes.POINTER(vp)]
    L.me_server_warm.argtypes = [vp, ctypes.c_char_p, i32, ctypes.POINTER(me_kin), ctypes.POINTER(i64)]
    L.me_server_submit.argtypes = [vp, ctypes.POINTER(me_request), ctypes.POINTER(i64)]
    L.me_server_poll.argtypes = [vp, i64, ctypes.POINTER(me_request_result)]
    L.me_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(me_request_result), vp, vp]
    L.me_server_get_stats.argtypes = [vp, ctypes.POINTER(me_server_stats)]
    L.me_server_destroy.argtypes = [vp]
    L.me_server_destroy.restype = None
    dp = ctypes.POINTER(ctypes.c_double)
    L.me_grid_create.argtypes = [vp, ctypes.POINTER(me_kin), i32, ctypes.POINTER(vp)]
    L.me_grid_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.me_grid_get_edges.argtypes = [vp, vp]
    L.me_grid_set_edges.argtypes = [vp, vp]
    L.me_grid_get_hist.argtypes = [vp, vp]
    L.me_grid_clear_hist.argtypes = [vp]
    L.me_grid_refine.argtypes = [vp, ctypes.c_double]
    L.xsec_step_grid.argtypes = [vp, vp, u64, u64, i64, ctypes.POINTER(me_kin), vp, ctypes.POINTER(me_xsec_acc),
                                 vp, vp]
    L.me_grid_destroy.argtypes = [vp]
    L.me_grid_destroy.restype = None
    L.me_vegas_refine_edges.argtypes = [vp, vp, i32, i32, ctypes.c_double, vp]
    for fn in ("me_create", "me_eval", "me_eval_host", "me_generate", "xsec_step", "xsec_step_async", "xsec_step_noalloc", "me_step_timing",
               "me_xsec_estimate", "me_info", "me_server_create", "me_server_warm", "me_server_submit",
               "me_server_poll", "me_server_wait", "me_server_get_stats", "me_grid_create", "me_grid_info",
               "me_grid_get_edges", "me_grid_set_edges", "me_grid_get_hist", "me_grid_clear_hist",
               "me_grid_refine", "xsec_step_grid", "me_vegas_refine_edges"):
        getattr(L, fn).restype = ctypes.c_int
    _LIB = L
    return L


def _check(st):
    if st != 0:
        raise MeError(st, _LIB.me_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_params(**kw):
    p = me_params(alpha=1 / 128, sw2=0.2312, mZ=91.1876, wZ=2.4952, mW=80.4, wW=2.085, alpha_s=0.118, mt=175.0,
                  wt=1.5, mH=125.0, wH=0.0, complex_mass=0, reserved_=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_kin(kind, sqrt_s=0.0, sqrt_s_range=(0.0, 0.0), masses=(), cut_legs=(), pt_min=0.0, eta_max=0.0,
             dr_min=0.0, s_ident=1.0, max_attempts=0, res_mass=0.0, res_width=0.0, objects=(), leg_class=None,
             paper_cuts=None):
    """me_kin.  objects (ME_PS_YPT): dicts with legs ((k,) or (k1, k2) for a resonance), mass or
    res_mass/res_width, y_max, pt_min, pt_max.  leg_class (per leg, 0..3) selects the paper's cuts
    (cut_mode 1) with the thresholds of paper_cuts (keys jet_pt, jet_eta, jet_ptij, b_pt, b_eta,
    lep_pt, lep_eta)."""
    k = me_kin()
    k.n_obj = len(objects)
    for j, o in enumerate(objects):
        legs = tuple(o["legs"])
        k.obj_legs[j][0] = legs[0]
        k.obj_legs[j][1] = legs[1] if len(legs) == 2 else -1
        k.obj_mass[j] = o.get("mass", 0.0)
        k.obj_res_mass[j] = o.get("res_mass", 0.0)
        k.obj_res_width[j] = o.get("res_width", 0.0)
        k.obj_y_max[j], k.obj_pt_min[j], k.obj_pt_max[j] = o["y_max"], o["pt_min"], o["pt_max"]
    for j in range(len(objects), 8):
        k.obj_legs[j][0] = k.obj_legs[j][1] = -1
    if leg_class is not None:
        k.cut_mode = 1
        for i, c in enumerate(leg_class):
            k.leg_class[i] = c
        for key, v in (paper_cuts or {}).items():
            setattr(k, key, v)
    k.kind = kind
    k.max_attempts = max_attempts
    k.sqrt_s = sqrt_s
    k.sqrt_s_min, k.sqrt_s_max = sqrt_s_range
    for i, m in enumerate(masses):
        k.mass[i] = m
    k.n_cut_legs = len(cut_legs)
    for i, l in enumerate(cut_legs):
        k.cut_legs[i] = l
    k.pt_min, k.eta_max, k.dr_min, k.s_ident = pt_min, eta_max, dr_min, s_ident
    k.res_mass, k.res_width = res_mass, res_width
    return k


def me_create(process, params=None, prec=ME_FP64):
    L = load()
    h = ctypes.c_void_p()
    _check(L.me_create(process.encode(), ctypes.byref(params) if params is not None else None, prec,
                       ctypes.byref(h)))
    return h.value


def me_eval(h, momenta, n, out, stream=None):
    _check(load().me_eval(h, _ptr(momenta), n, _ptr(out), _stream(stream)))


def me_eval_host(h, momenta, n, out, stream=None):
    """|M|^2 for host buffers (CPU tensors or addresses); returns when out is filled."""
    _check(load().me_eval_host(h, _ptr(momenta), n, _ptr(out), _stream(stream)))


def me_generate(h, seed, counter_offset, n, kin, momenta=None, weight=None, shat=None, tries=None, stream=None):
    _check(load().me_generate(h, seed, counter_offset, n, ctypes.byref(kin), _ptr(momenta), _ptr(weight),
                              _ptr(shat), _ptr(tries), _stream(stream)))


def xsec_step(h, seed, counter_offset, n_accept, kin, stream=None, acc=None, me2_out=None, momenta_out=None):
    acc = acc if acc is not None else me_xsec_acc()
    _check(load().xsec_step(h, seed, counter_offset, n_accept, ctypes.byref(kin), _stream(stream),
                            ctypes.byref(acc), _ptr(me2_out), _ptr(momenta_out)))
    return acc


def xsec_step_async(h, seed, counter_offset, n_accept, kin, acc_dev, stream=None):
    """xsec_step adding its sums to acc_dev (device, 4 doubles) without a host synchronisation."""
    _check(load().xsec_step_async(h, seed, counter_offset, n_accept, ctypes.byref(kin), _stream(stream),
                                  _ptr(acc_dev)))


def xsec_step_noalloc(h, seed, counter_offset, n_accept, kin, stream=None, acc=None, me2_out=None,
                      momenta_out=None):
    """xsec_step without device allocations (scratch in a static device array; see include/me.h)."""
    acc = acc if acc is not None else me_xsec_acc()
    _check(load().xsec_step_noalloc(h, seed, counter_offset, n_accept, ctypes.byref(kin), _stream(stream),
                                    ctypes.byref(acc), _ptr(me2_out), _ptr(momenta_out)))
    return acc


def me_step_timing(h, enable):
    """Returns (ms_ps, ms_me) accumulated since the previous call; enable turns recording on/off."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().me_step_timing(h, int(enable), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def me_xsec_estimate(acc):
    s, e = ctypes.c_double(), ctypes.c_double()
    _check(load().me_xsec_estimate(ctypes.byref(acc), ctypes.byref(s), ctypes.byref(e)))
    return s.value, e.value


def me_info(h):
    info = me_info_t()
    _check(load().me_info(h, ctypes.byref(info)))
    return info


def me_n_processes():
    return load().me_n_processes()


def me_process_name(i):
    r = load().me_process_name(i)
    return r.decode() if r else None


def me_destroy(h):
    load().me_destroy(h)


def me_last_error():
    return load().me_last_error().decode()


# ---------------------------------------------------------------------------
# request server (include/me_server.h)
# ---------------------------------------------------------------------------
def me_server_create(mem_cap_bytes=0, n_slots=0, max_requests=0, persistent=0, spin_limit_us=0,
                     inject_feeder_stall=0):
    L = load()
    cfg = me_server_config(mem_cap_bytes, n_slots, max_requests, persistent, spin_limit_us, inject_feeder_stall, 0)
    s = ctypes.c_void_p()
    _check(L.me_server_create(ctypes.byref(cfg), ctypes.byref(s)))
    return s.value


def me_server_warm(s, process, precision, kin):
    c = ctypes.c_int64()
    _check(load().me_server_warm(s, process.encode(), precision, ctypes.byref(kin), ctypes.byref(c)))
    return c.value


def me_server_submit(s, process, precision, seed, counter_offset, n, kin, want_me2=False, want_momenta=False):
    r = me_request(process.encode(), precision, int(want_me2), int(want_momenta), 0, seed, counter_offset, n, kin)
    t = ctypes.c_int64()
    _check(load().me_server_submit(s, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def me_server_poll(s, ticket):
    res = me_request_result()
    _check(load().me_server_poll(s, ticket, ctypes.byref(res)))
    return res


def me_server_wait(s, ticket, timeout_s=-1.0, me2_host=None, momenta_host=None):
    """Waits for a request; me2_host / momenta_host: host buffers (numpy arrays or addresses) or None."""
    res = me_request_result()

    def hp(a):
        if a is None:
            return None
        return a if isinstance(a, int) else a.ctypes.data
    st = load().me_server_wait(s, ticket, timeout_s, ctypes.byref(res), hp(me2_host), hp(momenta_host))
    if st != 0:
        raise MeError(st, _LIB.me_last_error().decode())
    return res


def me_server_get_stats(s):
    st = me_server_stats()
    _check(load().me_server_get_stats(s, ctypes.byref(st)))
    return st


def me_server_destroy(s):
    load().me_server_destroy(s)


# ---------------------------------------------------------------------------
# adaptive grids (include/me.h, me_grid_*)
# ---------------------------------------------------------------------------
def me_grid_create(h, kin, n_bins):
    g = ctypes.c_void_p()
    _check(load().me_grid_create(h, ctypes.byref(kin), n_bins, ctypes.byref(g)))
    return g.value


def me_grid_info(g):
    d, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().me_grid_info(g, ctypes.byref(d), ctypes.byref(b)))
    return d.value, b.value


def me_grid_get_edges(g):
    import numpy as np
    d, b = me_grid_info(g)
    out = np.empty((d, b + 1))
    _check(load().me_grid_get_edges(g, out.ctypes.data))
    return out


def me_grid_set_edges(g, edges):
    import numpy as np
    e = np.ascontiguousarray(edges, dtype=np.float64)
    _check(load().me_grid_set_edges(g, e.ctypes.data))


def me_grid_get_hist(g):
    import numpy as np
    d, b = me_grid_info(g)
    out = np.empty((d, b))
    _check(load().me_grid_get_hist(g, out.ctypes.data))
    return out


def me_grid_clear_hist(g):
    _check(load().me_grid_clear_hist(g))


def me_grid_refine(g, alpha=1.5):
    _check(load().me_grid_refine(g, alpha))


def xsec_step_grid(h, g, seed, counter_offset, n_accept, kin, stream=None, acc=None, me2_out=None,
                   momenta_out=None):
    acc = acc if acc is not None else me_xsec_acc()
    _check(load().xsec_step_grid(h, g, seed, counter_offset, n_accept, ctypes.byref(kin), _stream(stream),
                                 ctypes.byref(acc), _ptr(me2_out), _ptr(momenta_out)))
    return acc


def me_grid_destroy(g):
    load().me_grid_destroy(g)


def me_vegas_refine_edges(edges, hist, alpha=1.5):
    """Host-only refinement of edges [D, N+1] from hist [D, N] (no device)."""
    import numpy as np
    e = np.ascontiguousarray(edges, dtype=np.float64)
    h = np.ascontiguousarray(hist, dtype=np.float64)
    out = np.empty_like(e)
    _check(load().me_vegas_refine_edges(e.ctypes.data, h.ctypes.data, e.shape[0], e.shape[1] - 1, alpha,
                                        out.ctypes.data))
    return out
