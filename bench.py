"""Benchmark: |M|^2 evaluations per second of one Monte Carlo step on GB300.

A step is one pass of the whole hot path over one batch of 2^20 accepted
points of u d~ > e+ ve g g at sqrt(s) = 1 TeV (RAMBO, pT > 20 GeV,
|eta| < 2.5, Delta R > 0.4, seed 1): Philox draws, phase space, cuts and
redraws, invariants, wavefunctions, the diagram program, colour sum,
helicity sum, weights and the deterministic Monte Carlo reduction, through
xsec_step of the C ABI, in the mixed precision (FP32 amplitudes, FP64
momenta, resonant invariants and accumulation).  The FP64 path is timed
beside it for context.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload KEY]

Output: the last line of stdout is one compact JSON record (rate, FP64 rate, the relative error
of both paths against the FP64 CPU oracle on points sampled over one full-size step, roofline,
CPU baseline, end-to-end rate, clocks); the full record (per-kernel figures, every process's
rates and errors, the serving mix, the adaptive grids) goes to --detail (bench_detail.json).

With N > 1 (torchrun, one process per GPU) each rank runs its own 2^20 points
(disjoint Philox counters): weak scaling, no data-path collective.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 operations per accepted point of the mixed-path kernels as executed: FADD + FMUL + 2 FFMA
# thread instructions of one ncu capture per workload, divided by the points of that launch
# (profiles/ holds the captures; k_ps includes every draw of a point).  The code generator's own
# count of the |M|^2 program (me_info flops_amp) counts the program as written, before the compiler
# removes the repeated subexpressions of the helicity variants; it is the fallback where no
# capture exists.
EXECUTED_FLOPS_PER_POINT = {
    ("udx_epvegg", "k_ps"): 3916.3,
    ("udx_epvegg", "k_me"): 3039.0,
    ("gg_ttx_dilep", "k_ps"): 7003.3,
    ("gg_ttx_dilep", "k_me"): 6758.0,
    ("us_dchh", "k_ps"): 5216.0,
    ("us_dchh", "k_me"): 1793.8,
    ("uux_epem", "k_ps"): 18.0,
    ("uux_epem", "k_me"): 1091.0,
    ("gg_gggg", "k_ps"): 4249.2,
    ("gg_gggg", "k_me"): 10968317.3,
    ("uux_wpwm", "k_ps"): 3200.0,
    ("uux_wpwm", "k_me"): 3691.7,
    ("udx_epvegg_bw", "k_ps"): 6256.0,
    ("udx_epvegg_bw", "k_me"): 3039.0,
    ("udx_wpz", "k_ps"): 3224.0,
    ("udx_wpz", "k_me"): 2346.6,
}

# DRAM bytes per point of the mixed-path kernels (dram__bytes_read.sum + dram__bytes_write.sum of one
# ncu capture, divided by the points of that launch; profiles/ holds the captures).  A launch's
# traffic is this times its points: the kernels stream their points, so traffic grows in proportion.
TRAFFIC_PER_POINT = {("udx_epvegg", "k_ps"): (4.913152e6 + 229.596928e6) / 2 ** 20,
                     ("udx_epvegg", "k_me"): (214.00448e6 + 3.760384e6) / 2 ** 20,
                     ("gg_gggg", "k_me"): (3.488256e6 + 0.070912e6) / 16384}

# Warp instructions issued per accepted point (smsp__inst_executed.sum of the same ncu captures,
# divided by the points of the launch).  The phase-space kernel mixes integer (Philox), FP32 and
# control instructions and is bound by instruction issue, so its roofline is also stated against
# the issue rate.
WARP_INSTRUCTIONS_PER_POINT = {("udx_epvegg", "k_ps"): 174954989.0 / 2 ** 20,
                               ("udx_epvegg", "k_me"): 94714880.0 / 2 ** 20}

SM_COUNT = 152
FP32_LANES_PER_SM = 128
SCHEDULERS_PER_SM = 4
SM_MAX_MHZ = 2070.0


def issue_roofline(workload, kernel, ms, points, mhz=SM_MAX_MHZ):
    """Issue-rate view of a kernel's roofline: warp instructions per second against the SMs' issue
    ceiling (152 SMs x 4 schedulers x one warp instruction per cycle x clock), or None without a
    capture for this workload and kernel."""
    per_point = WARP_INSTRUCTIONS_PER_POINT.get((workload, kernel))
    if per_point is None or ms <= 0:
        return None
    achieved = per_point * points / (ms * 1e-3) / 1e9
    peak = SM_COUNT * SCHEDULERS_PER_SM * mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp instructions/s", "frac": achieved / peak,
            "instructions_per_point": per_point,
            "source": "smsp__inst_executed.sum of the ncu capture; peak 152 SMs x 4 schedulers x 1 per cycle "
                      "x 2070 MHz"}


def fp32_alu_peak_tflops(mhz=SM_MAX_MHZ):
    """FP32 CUDA-core peak: SMs x FP32 lanes x 2 flop (FMA) x clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def tensor_peak_tflops():
    """Measured dense bf16 tensor peak of this GPU type (burst), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        mhz.sort()
        return {"sm_mhz": mhz[len(mhz) // 2] if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Philox counter ranges of the ranks: rank r draws its points from counters
# [r * RANK_STRIDE, r * RANK_STRIDE + steps * points), disjoint for < 2^40 points per rank
RANK_STRIDE = 1 << 40


def rank_offset(rank):
    return rank * RANK_STRIDE


def job_rate(step_ms, points_per_rank, world, dist=None, device=None):
    """Whole-job rate: every rank's points over the slowest rank's step time (max over ranks)."""
    import torch
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return points_per_rank * world / (t_max * 1e-3), t_max


def merge_acc(acc, world, dist=None, device=None):
    """Monte Carlo sums of all ranks (each rank's xsec_step accumulator), summed."""
    import torch
    v = torch.tensor([acc.sum_w, acc.sum_w2, float(acc.n_acc), float(acc.n_try)], dtype=torch.float64,
                     device=device)
    if world > 1:
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return {"sum_w": float(v[0]), "sum_w2": float(v[1]), "n_acc": int(v[2]), "n_try": int(v[3])}


def oracle_kin(w):
    from paper_1305_0708_gb300.compiler.diagrams import parse
    n_ext = len(parse(w["process"]).particles)
    if w["kind"] == "two_body":
        k = {"kind": "2to2", "sqrt_s": w["sqrt_s"]}
    elif w["kind"] == "rambo":
        k = {"kind": "rambo", "sqrt_s": w["sqrt_s"], "n_final": n_ext - 2}
        if "masses" in w:
            k["masses"] = list(w["masses"][2:])
    elif w["kind"] == "rambo_bw":
        k = {"kind": "rambo_bw", "sqrt_s": w["sqrt_s"], "n_final": n_ext - 2, "res_mass": w["res_mass"],
             "res_width": w["res_width"]}
    elif w["kind"] == "ypt":
        k = {"kind": "ypt", "sqrt_s": w["sqrt_s"], "n_final": n_ext - 2, "objects": w["objects"]}
    else:
        k = {"kind": "ttbar", "sqrt_s_range": w["sqrt_s_range"]}
    if w.get("leg_class"):
        from paper_1305_0708_gb300.workloads import PAPER_CUTS
        k["paper_cuts"] = {"leg_class": list(w["leg_class"]), "thresholds": dict(PAPER_CUTS)}
    if w.get("cuts"):
        c = w["cuts"]
        k["cuts"] = {"legs": list(c["legs"]), "pt_min": c["pt_min"], "eta_max": c["eta_max"], "dr_min": c["dr_min"]}
    return k


def oracle_me_fn(process):
    """The oracle's |M|^2 function of a compiled process string (the decay-chain tt~ process under
    either of its names)."""
    from oracle import processes as opr
    alias = {"g g > (t > b (w+ > e+ ve)) (t~ > b~ (w- > e- ve~))": "g g > t t~ > b e+ ve b~ e- ve~"}
    return opr.PROCESSES[alias.get(process, process)]


def oracle_step(w, events):
    """The oracle's whole step on a sample of events: generate, |M|^2, accumulate."""
    from oracle import xsec as oxs
    from oracle.sm import SMParams
    fn = oracle_me_fn(w["process"])
    par = SMParams()
    P, W, S, T = oxs.generate(oracle_kin(w), par, w["seed"], events)
    return oxs.accumulate(fn(P, par), W, S, T, w["s_ident"])


def _pool_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    import oracle.processes  # noqa: F401  (imports paid before the clock)


def _pool_step(job):
    w, events = job
    return oracle_step(w, events)


def oracle_pool(cores):
    """Process pool for the oracle on the host cores, started with spawn (safe beside CUDA)."""
    import multiprocessing
    return multiprocessing.get_context("spawn").Pool(cores, initializer=_pool_init)


def oracle_step_cores(pool, cores, w, events):
    """The oracle's step on a sample split by points over the pool's processes; sums summed."""
    import numpy as np
    parts = [e for e in np.array_split(events, cores) if len(e)]
    res = pool.map(_pool_step, [(w, e) for e in parts])
    return tuple(sum(r[k] for r in res) for k in range(4))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, w, rank, world):
    """FP64 CPU oracle on the host cores: bounded samples per step."""
    import numpy as np
    if rank != 0:
        return
    cores = host_cores()
    sample = args.ref_sample * cores
    pool = oracle_pool(cores)
    oracle_step_cores(pool, cores, w, np.arange(8 * cores))  # warm caches and imports
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle_step_cores(pool, cores, w, np.arange(s * sample, (s + 1) * sample))
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    pool.close()
    pool.join()
    per_step = sum(times) / len(times)
    value = sample / per_step
    line = {"metric": "|M|^2 evals/s", "value": value, "unit": "evals/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "describe": w["describe"], "points_per_step": sample,
                       "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} accepted points per step of the same workload (numpy FP64, "
                                       f"split over {cores} single-threaded processes)"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def per_process_table(B, torch, dev, stream, flush, offset0, warmup, steps):
    """Every workload and variant: mixed and FP64 xsec_step rates on the full point count, the mixed
    |M|^2 kernel's CUDA-core fraction, and the mixed path's relative error against the FP64
    GPU path on the FP64 path's own momenta (median and max over the accepted points)."""
    from paper_1305_0708_gb300.workloads import PAPER_PS, VARIANTS, WORKLOADS, kin_args
    peak = fp32_alu_peak_tflops()
    table = {}
    for key, w in list(WORKLOADS.items()) + list(VARIANTS.items()) + list(PAPER_PS.items()):
        try:
            n = w["n"]
            kin = B.make_kin(**kin_args(w))
            row = {"points": n}
            prm = B.make_params(**w["params"]) if "params" in w else None
            for prec, name in ((B.ME_MIXED, "mixed"), (B.ME_FP64, "fp64")):
                h = B.me_create(w["process"], prm, prec)
                slow = prec == B.ME_FP64 and key == "gg_gggg"
                nw, ns = (1, 2) if slow else (warmup, steps)
                acc_dev = torch.zeros(4, dtype=torch.float64, device=dev)
                for s_ in range(nw):
                    B.xsec_step_async(h, w["seed"], offset0 + s_ * n, n, kin, acc_dev, stream)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ns)]
                for s_ in range(ns):
                    flush.zero_()
                    ev[s_][0].record(stream)
                    B.xsec_step_async(h, w["seed"], offset0 + (nw + s_) * n, n, kin, acc_dev, stream)
                    ev[s_][1].record(stream)
                torch.cuda.synchronize(dev)
                ms = sum(a.elapsed_time(b) for a, b in ev) / ns
                sums = acc_dev.cpu().tolist()  # (sum w, sum w^2, draws, exhausted) over nw + ns steps
                npts = (nw + ns) * n
                mean = sums[0] / sums[2]
                err = math.sqrt(max(sums[1] / sums[2] - mean * mean, 0.0) / max(sums[2] - 1, 1))
                # per-kernel device time on further steps of the same work
                nt = 1 if slow else ns
                B.me_step_timing(h, 1)
                for s_ in range(nt):
                    flush.zero_()
                    B.xsec_step(h, w["seed"], offset0 + (nw + ns + s_) * n, n, kin, stream, B.me_xsec_acc())
                t_ps, t_me = B.me_step_timing(h, 0)
                ns_t = nt
                info = B.me_info(h)
                fl = (EXECUTED_FLOPS_PER_POINT.get((key, "k_me"), info.flops_amp) if prec == B.ME_MIXED
                      else info.flops_fp64)
                row[name] = {"evals_per_s": n / (ms * 1e-3), "ms_per_step": ms, "k_me_ms": t_me / ns_t,
                             "k_me_tflops": fl * n / (t_me / ns_t * 1e-3) / 1e12,
                             "sigma_pb": mean, "error_pb": err, "points": npts, "draws_per_point": sums[2] / npts}
                if prec == B.ME_MIXED:
                    row[name]["k_me_frac_fp32_peak"] = row[name]["k_me_tflops"] / peak
                else:
                    # FP64 momenta and |M|^2 of one step, then the mixed me_eval on the same momenta
                    mom = torch.empty(info.n_ext * 4 * n, dtype=torch.float64, device=dev)
                    m64 = torch.empty(n, dtype=torch.float64, device=dev)
                    B.xsec_step(h, w["seed"], offset0, n, kin, stream, B.me_xsec_acc(), m64, mom)
                    hm = B.me_create(w["process"], prm, B.ME_MIXED)
                    mmx = torch.empty(n, dtype=torch.float64, device=dev)
                    B.me_eval(hm, mom, n, mmx, stream)
                    torch.cuda.synchronize(dev)
                    B.me_destroy(hm)
                    ok = m64 > 0
                    rel = ((mmx[ok] - m64[ok]).abs() / m64[ok]).double()
                    row["mixed_rel_err"] = {"median": float(rel.median().item()), "max": float(rel.max().item()),
                                            "p99_99": float(torch.quantile(rel.float().cpu(), 0.9999).item()),
                                            "frac_above_1e-3": float((rel > 1e-3).double().mean().item()),
                                            "sum_me2": float(((mmx[ok].sum() - m64[ok].sum()) / m64[ok].sum()).abs()),
                                            "points": int(ok.sum().item())}
                    # conditioning of the points above 1e-3: how far the FP64 program itself moves when
                    # its input momenta are rounded to FP32 (what any FP32-wavefunction evaluation sees)
                    bad = torch.nonzero(ok & ((mmx - m64).abs() > 1e-3 * m64.abs())).flatten()[:64]
                    if bad.numel():
                        nb = int(bad.numel())
                        mb = mom.view(info.n_ext * 4, n)[:, bad].float().double().contiguous()
                        o64 = torch.empty(nb, dtype=torch.float64, device=dev)
                        B.me_eval(h, mb, nb, o64, stream)
                        torch.cuda.synchronize(dev)
                        shift = ((o64 - m64[bad]).abs() / m64[bad]).cpu().tolist()
                        err = ((mmx[bad] - m64[bad]).abs() / m64[bad]).cpu().tolist()
                        row["mixed_rel_err"]["above_1e-3"] = [{"mixed_err": e_, "fp64_shift_at_fp32_inputs": s_}
                                                             for e_, s_ in zip(err, shift)]
                B.me_destroy(h)
            row["mixed_over_fp64"] = row["mixed"]["evals_per_s"] / row["fp64"]["evals_per_s"]
            table[key] = row
        except Exception as exc:  # an auxiliary row that fails is recorded, not fatal to the headline line
            table[key] = {"points": w["n"], "error": f"{type(exc).__name__}: {exc}"[:300]}
    return table


def make_stream(rate, count, seed=4):
    """Poisson request stream: arrival times (s), process keys, batch sizes, momentum seeds."""
    import numpy as np
    from paper_1305_0708_gb300.workloads import WORKLOADS
    rng = np.random.default_rng([seed, int(rate)])
    keys = list(WORKLOADS)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    procs = [keys[i] for i in rng.integers(0, len(keys), size=count)]
    sizes = np.exp(rng.uniform(np.log(1e3), np.log(1e6), size=count)).astype(np.int64)
    seeds = rng.integers(0, 2 ** 62, size=count)
    return [(float(a), k, int(n), int(sd)) for a, k, n, sd in zip(t, procs, sizes, seeds)]


def pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def serve_stream(B, srv, kins, rate, count):
    """One Poisson stream through a running server: sustained rate and latency percentiles."""
    from paper_1305_0708_gb300.workloads import WORKLOADS
    reqs = make_stream(rate, count)
    t0 = time.perf_counter()
    tickets = []
    for arr, k, n, sd in reqs:
        dt = t0 + arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append((B.me_server_submit(srv, WORKLOADS[k]["process"], B.ME_MIXED, sd, 0, n, kins[k]), n))
    res, failed = [], {}
    for t, _ in tickets:
        try:
            res.append(B.me_server_wait(srv, t, 600.0))
        except B.MeError as exc:  # recorded, not fatal: the line states how many failed and why
            failed[str(exc.status)] = failed.get(str(exc.status), 0) + 1
    if not res:
        return {"requests": count, "failed": failed}
    lat = [r.t_done_ms - r.t_submit_ms for r in res]
    span = (max(r.t_done_ms for r in res) - min(r.t_submit_ms for r in res)) * 1e-3
    pts = sum(n for _, n in tickets)
    return {"requests": count, "points": pts, "offered_evals_per_s": pts / reqs[-1][0], "evals_per_s": pts / span,
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat)}, "failed": failed}


def one_launch_per_request(B, kins, rate, count, prec, budget_s):
    """The plain path: one synchronous xsec_step per request in arrival order, stopped after budget_s."""
    from paper_1305_0708_gb300.workloads import WORKLOADS
    reqs = make_stream(rate, count)
    hs = {k: B.me_create(w["process"], None, prec) for k, w in WORKLOADS.items()}
    for k in hs:  # load kernels once, outside the clock
        B.xsec_step(hs[k], 1, 0, 1000, kins[k])
    lat, pts, done = [], 0, 0
    t0 = time.perf_counter()
    for arr, k, n, sd in reqs:
        if time.perf_counter() - t0 > budget_s:
            break
        dt = t0 + arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        B.xsec_step(hs[k], sd, 0, n, kins[k])
        lat.append((time.perf_counter() - t0 - arr) * 1e3)
        pts += n
        done += 1
    wall = time.perf_counter() - t0
    for h in hs.values():
        B.me_destroy(h)
    return {"rate": rate, "requests": count, "completed_within_budget": done, "budget_s": budget_s,
            "precision": "fp64" if prec == B.ME_FP64 else "mixed", "evals_per_s": pts / wall,
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat) if lat else None}}


def serving_mix(B, rates=((10, 48), (100, 128), (1000, 256)), baseline_budget_s=30.0):
    """Request server under Poisson streams (mixed precision, continuous batching), in both
    scheduling modes: chunk graphs on 4 slots, and persistent lanes (the all-gluon requests keep
    chunk launches there).  Against them, the plain one-launch-per-request path in the server's
    precision at every rate, and in FP64 at the lowest rate."""
    from paper_1305_0708_gb300.workloads import WORKLOADS, kin_args
    kins = {k: B.make_kin(**kin_args(w)) for k, w in WORKLOADS.items()}
    out = {}
    for mode, persistent in (("chunk_graphs", 0), ("persistent_lanes", 1)):
        srv = B.me_server_create(persistent=persistent)
        tuned = {k: B.me_server_warm(srv, w["process"], B.ME_MIXED, kins[k]) for k, w in WORKLOADS.items()}
        o = {"server": {"n_slots": 4, "mem_cap_gib": 40, "precision": "mixed", "persistent": persistent,
                        "points_per_chunk_or_tile": tuned}, "rates": {}}
        try:
            for rate, count in rates:
                o["rates"][str(rate)] = serve_stream(B, srv, kins, rate, count)
            st = B.me_server_get_stats(srv)
            o["server"].update(bytes_peak=st.bytes_peak, launches=st.launches, graph_launches=st.graph_launches,
                               lane_launches=st.lane_launches, lane_items=st.lane_items,
                               lane_timeouts=st.lane_timeouts)
        finally:
            B.me_server_destroy(srv)
        out[mode] = o
    out["one_launch_per_request_mixed"] = {str(r): one_launch_per_request(B, kins, r, c, B.ME_MIXED, baseline_budget_s)
                                           for r, c in rates}
    out["one_launch_per_request_fp64"] = one_launch_per_request(B, kins, rates[0][0], rates[0][1], B.ME_FP64,
                                                                baseline_budget_s)
    return out


def vegas_leg(B, torch, dev, stream, keys=("uux_epem", "gg_ttx_dilep", "udx_epvegg", "udx_epvegg_bw"), rounds=5, n_round=1 << 18, n_final=1 << 20):
    """Adaptive grids: `rounds` refinements of n_round-point grid steps, then sigma-hat on n_final
    points with the adapted grid against uniform sampling on the same points (mixed precision)."""
    from paper_1305_0708_gb300.workloads import VARIANTS, WORKLOADS, kin_args
    out = {}
    for key in keys:
        w = WORKLOADS[key] if key in WORKLOADS else VARIANTS[key]
        kin = B.make_kin(**kin_args(w))
        h = B.me_create(w["process"], None, B.ME_MIXED)
        g = B.me_grid_create(h, kin, 64)
        t0 = time.perf_counter()
        for r in range(rounds):
            B.xsec_step_grid(h, g, w["seed"], r * n_round, n_round, kin, stream)
            B.me_grid_refine(g, 1.5)
        t_adapt = time.perf_counter() - t0
        off = 1 << 36
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        acc = B.xsec_step_grid(h, g, w["seed"], off, n_final, kin, stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_g = ev0.elapsed_time(ev1)
        ev0.record(stream)
        acc0 = B.xsec_step(h, w["seed"], off, n_final, kin, stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_0 = ev0.elapsed_time(ev1)
        (s_g, e_g), (s_0, e_0) = B.me_xsec_estimate(acc), B.me_xsec_estimate(acc0)
        out[key] = {"sigma_pb_adapted": s_g, "error_pb_adapted": e_g, "sigma_pb_uniform": s_0,
                    "error_pb_uniform": e_0, "error_ratio": e_g / e_0, "points": n_final,
                    "rounds": rounds, "points_per_round": n_round, "bins": 64, "adapt_s": t_adapt,
                    "step_ms_adapted": ms_g, "step_ms_uniform": ms_0}
        B.me_grid_destroy(g)
        B.me_destroy(h)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="udx_epvegg")
    ap.add_argument("--ref-sample", type=int, default=1000)
    ap.add_argument("--cpu-sample", type=int, default=1000)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the per-process table")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-mix leg")
    ap.add_argument("--no-vegas", action="store_true", help="skip the adaptive-grid leg")
    ap.add_argument("--par-sample", type=int, default=512,
                    help="points of one full-size step compared with the oracle (0: skip)")
    ap.add_argument("--detail", default="bench_detail.json",
                    help="file for the full record (per-kernel figures, per-process table, serving, grids)")
    ap.add_argument("--points", type=int, default=0,
                    help="points per step instead of the workload's own count (small cases for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

    from paper_1305_0708_gb300.workloads import VARIANTS, WORKLOADS, kin_args
    w = WORKLOADS[args.workload] if args.workload in WORKLOADS else VARIANTS[args.workload]
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    import __graft_entry__ as g
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    g.build() if rank == 0 or world == 1 else None
    if world > 1:
        dist.barrier()
    from paper_1305_0708_gb300 import binding as B
    B.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.points if args.points > 0 else w["n"]
    kin = B.make_kin(**kin_args(w))
    stream = torch.cuda.current_stream(dev)
    offset0 = rank_offset(rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def time_steps(h, steps, warmup):
        """Steps queued back to back with xsec_step_async (sums accumulated on the device, read
        once at the end); each step bracketed by CUDA events on the launch stream, the L2 flush
        between steps outside the brackets."""
        acc_dev = torch.zeros(4, dtype=torch.float64, device=dev)
        for s in range(warmup):
            B.xsec_step_async(h, w["seed"], offset0 + s * n, n, kin, acc_dev, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        t0 = time.perf_counter()
        for s in range(steps):
            flush.zero_()
            ev[s][0].record(stream)
            B.xsec_step_async(h, w["seed"], offset0 + (warmup + s) * n, n, kin, acc_dev, stream)
            ev[s][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in ev]
        a = acc_dev.cpu().tolist()
        if a[3] != 0:
            raise RuntimeError("a point exhausted its phase-space redraws")
        acc = B.me_xsec_acc(sum_w=a[0], sum_w2=a[1], n_acc=(warmup + steps) * n, n_try=int(round(a[2])))
        return ms, wall, acc

    clocks = Clocks()
    h32 = B.me_create(w["process"], None, B.ME_MIXED)
    info = B.me_info(h32)
    clocks.start()
    ms32, wall32, acc32 = time_steps(h32, args.steps, args.warmup)
    clk = clocks.stop(local)
    step_ms = sum(ms32) / len(ms32)
    value, step_ms = job_rate(step_ms, n, world, dist, dev)
    mc = merge_acc(acc32, world, dist, dev)

    # per-kernel device time of the step (CUDA events recorded by the library on the launch
    # stream around k_ps and k_me), taken on extra steps of the same work after the timed region
    B.me_step_timing(h32, 1)
    acc_t = B.me_xsec_acc()
    n_kt = max(3, args.steps // 2)
    for s_ in range(n_kt):
        flush.zero_()
        B.xsec_step(h32, w["seed"], offset0 + (args.warmup + args.steps + s_) * n, n, kin, stream, acc_t)
    t_ps, t_me = B.me_step_timing(h32, 0)
    ps_ms, me_ms = t_ps / n_kt, t_me / n_kt
    tries_per_point = acc_t.n_try / acc_t.n_acc
    me_flops = EXECUTED_FLOPS_PER_POINT.get((args.workload, "k_me"))
    ps_flops = EXECUTED_FLOPS_PER_POINT.get((args.workload, "k_ps"))
    flops_event = me_flops if me_flops is not None else info.flops_amp
    peak = fp32_alu_peak_tflops()
    me_tflops = flops_event * n / (me_ms * 1e-3) / 1e12
    ps_tflops = (ps_flops or 0.0) * n / (ps_ms * 1e-3) / 1e12
    kernels = {
        "k_me": {"ms": me_ms, "achieved_tflops": me_tflops, "frac": me_tflops / peak,
                 "flops_per_point": flops_event, "flops_model": info.flops_amp,
                 "flops_source": "executed (ncu FP32 op counters)" if me_flops is not None else "code generator count",
                 "what": "|M|^2, weights, block sums (FP32 amplitudes; CUDA-core flops)"},
        "k_ps": {"ms": ps_ms, "achieved_tflops": ps_tflops, "frac": ps_tflops / peak,
                 "flops_per_point": ps_flops, "draws_per_point": tries_per_point,
                 "flops_source": "executed (ncu FP32 op counters)" if ps_flops is not None else "none",
                 "what": "Philox + double-float RAMBO + cuts + redraw queue"},
    }
    if info.flops_colour > 0:
        # colour quadratic form on the tensor cores (FP16 hi/lo operands, FP32 accumulation):
        # algorithmic flops against the measured dense bf16 peak (FP16 runs at the same rate)
        tpk = tensor_peak_tflops()
        col_tflops = info.flops_colour * n / (me_ms * 1e-3) / 1e12
        kernels["k_me"]["tensor"] = {"flops_per_point": info.flops_colour, "achieved_tflops": col_tflops,
                                     "peak": tpk, "frac": col_tflops / tpk,
                                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured",
                                     "what": "colour sum x.C.x, mma.sync m16n8k16 f16, hi/lo split"}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    achieved = kernels[dom]["achieved_tflops"]
    tpp = TRAFFIC_PER_POINT.get((args.workload, dom))
    traffic = tpp * n if tpp is not None else None

    # FP64 path for context
    fp64 = None
    if not args.no_fp64:
        h64 = B.me_create(w["process"], None, B.ME_FP64)
        ms64, _, _ = time_steps(h64, max(3, args.steps // 4), 3)
        s64 = sum(ms64) / len(ms64)
        fp64 = {"value": n / (s64 * 1e-3), "unit": "evals/s", "ms_per_step": s64}
        B.me_destroy(h64)

    # end to end through the public API with host buffers: me_eval_host on page-locked host
    # momenta and |M|^2 (the momenta cross to the device and |M|^2 back inside the call)
    mom_dev = torch.empty(info.n_ext * 4 * n, dtype=torch.float64, device=dev)
    me2_dev = torch.empty(n, dtype=torch.float64, device=dev)
    B.xsec_step(h32, w["seed"], offset0, n, kin, stream, B.me_xsec_acc(), me2_dev, mom_dev)
    mom_host = mom_dev.cpu().pin_memory()
    out_host = torch.empty(n, dtype=torch.float64).pin_memory()
    for _ in range(3):
        B.me_eval_host(h32, mom_host, n, out_host, stream)
    barrier()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        B.me_eval_host(h32, mom_host, n, out_host, stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = sorted(e2e_ms)[len(e2e_ms) // 2]
    # the CPU-GPU link alone: the same momenta as one page-locked copy-engine transfer
    lk = []
    for _ in range(5):
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        mom_dev.copy_(mom_host, non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize(dev)
        lk.append(l0.elapsed_time(l1))
    link_gbs = mom_host.numel() * 8 / (sorted(lk)[len(lk) // 2] * 1e-3) / 1e9
    e2e_gbs = mom_host.numel() * 8 / (e2e_step * 1e-3) / 1e9
    e2e = {"value": n * world / (e2e_step * 1e-3), "unit": "evals/s",
           "h2d_bytes_per_step": int(mom_host.numel() * 8), "d2h_bytes_per_step": int(n * 8),
           "h2d_gbs": e2e_gbs, "link_copy_gbs": link_gbs, "frac_of_link": e2e_gbs / link_gbs,
           "path": "me_eval_host on page-locked host momenta and |M|^2 (the kernel reads and writes the mapped "
                   "host memory over the CPU-GPU link)"}
    # kernel-only me_eval time (momenta resident)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evals = []
    for _ in range(5):
        flush.zero_()
        ev0.record(stream)
        B.me_eval(h32, mom_dev, n, me2_dev, stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        evals.append(ev0.elapsed_time(ev1))
    me_eval_ms = sorted(evals)[len(evals) // 2]
    B.me_destroy(h32)

    serving = None
    if not args.no_serving and world == 1:
        serving = serving_mix(B)

    vegas = None
    if not args.no_vegas and world == 1:
        vegas = vegas_leg(B, torch, dev, stream)

    table = None
    if not args.no_table:
        table = per_process_table(B, torch, dev, stream, flush, offset0, 2, 3)

    # sampled points of one full-size step in the timed launch shape, both precisions, for the
    # oracle comparison in the cpu_baseline leg: |M|^2 and the momenta of n_par points spread
    # over the whole launch (first and last point included)
    samples = {}
    if rank == 0 and world == 1 and args.par_sample > 0:
        idx = torch.from_numpy(np.unique(np.linspace(0, n - 1, args.par_sample).astype(np.int64))).to(dev)
        for prec, name in ((B.ME_MIXED, "mixed"), (B.ME_FP64, "fp64")):
            hp = B.me_create(w["process"], None, prec)
            mom_s = torch.empty(info.n_ext * 4 * n, dtype=torch.float64, device=dev)
            me2_s = torch.empty(n, dtype=torch.float64, device=dev)
            B.xsec_step(hp, w["seed"], offset0 + (1 << 32), n, kin, stream, B.me_xsec_acc(), me2_s, mom_s)
            torch.cuda.synchronize(dev)
            P = mom_s.view(info.n_ext, 4, n)[:, :, idx].permute(2, 0, 1).contiguous().cpu().numpy()
            samples[name] = (me2_s[idx].cpu().numpy(), P)
            B.me_destroy(hp)
            del mom_s, me2_s

    cpu = None
    parity = None
    if rank == 0 and world == 1:
        # the oracle on the sampled points of both paths: relative error of |M|^2 per point
        if samples:
            from oracle.sm import SMParams
            fn = oracle_me_fn(w["process"])
            parity = {"points": int(len(samples["fp64"][0])), "spread_over": n}
            for name, (got, P) in samples.items():
                ref = fn(np.ascontiguousarray(P), SMParams())
                ok = ref > 0
                rel = np.abs(got[ok] / ref[ok] - 1.0)
                parity[name] = {"median": float(np.median(rel)), "max": float(rel.max())}
        # one core, then every host core (the sample split by points over single-threaded processes)
        events = np.arange(args.cpu_sample)
        oracle_step(w, np.arange(32))
        t0 = time.perf_counter()
        oracle_step(w, events)
        v1 = args.cpu_sample / (time.perf_counter() - t0)
        cores = host_cores()
        pool = oracle_pool(cores)
        oracle_step_cores(pool, cores, w, np.arange(4 * cores))
        n_all = args.cpu_sample * cores
        t0 = time.perf_counter()
        oracle_step_cores(pool, cores, w, np.arange(10 ** 7, 10 ** 7 + n_all))
        vall = n_all / (time.perf_counter() - t0)
        pool.close()
        pool.join()
        cpu = {"value": vall, "unit": "evals/s", "cores": cores, "kind": "oracle", "value_1core": v1,
               "sample": f"{n_all} accepted points of the same workload (generate, |M|^2, weights), numpy FP64 "
                         f"split over {cores} single-threaded processes; value_1core: {args.cpu_sample} points "
                         f"on one core"}

    if rank == 0:
        # the full record (per-kernel figures, the per-process table, the serving mix, the adaptive
        # grids) goes to a side file; stdout ends with one compact headline line
        detail = {"kernels": kernels, "me_eval_ms": me_eval_ms, "per_process": table, "serving": serving,
                  "vegas": vegas, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "wall_s_timed": wall32,
                  "mc": {"sigma_pb": mc["sum_w"] / mc["n_try"], "n_try": mc["n_try"], "n_acc": mc["n_acc"],
                         "ranks": world}}
        if args.detail:
            d = os.path.dirname(os.path.abspath(args.detail))
            os.makedirs(d, exist_ok=True)
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1)
        iss = issue_roofline(args.workload, dom, kernels[dom]["ms"], n)
        line = {
            "metric": "|M|^2 evals/s", "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (on-device Philox phase space)",
            "config": {"workload": args.workload, "points_per_step_per_gpu": n, "precision": "mixed",
                       "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
            "fp64_path": None if fp64 is None else {"value": fp64["value"], "ms_per_step": fp64["ms_per_step"]},
            "rel_err_vs_oracle": parity,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                         "issue_frac": None if iss is None else iss["frac"]},
            "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
            "gpu_launches": 3 * args.steps,
            "clocks": {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "detail_file": args.detail or None,
        }
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
