"""Build the sm_103a matrix-element library in-tree.

Steps: run the process compiler on every process of PROCESSES, write one
CUDA unit per process plus the registry, compile all units in parallel with
nvcc for sm_103a, and link libme.so under paper_1305_0708_gb300/_build/.
Rebuilds only what changed (content hashes).
"""
import concurrent.futures as cf
import hashlib
import json
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libme.so")

# (canonical name, aliases)
PROCESSES = [
    ("u u~ > e+ e-", []),
    ("u d~ > e+ ve g g", []),
    ("g g > (t > b (w+ > e+ ve)) (t~ > b~ (w- > e- ve~))", ["g g > t t~ > b e+ ve b~ e- ve~"]),
    ("u s > d c h h", []),
    ("u s > d c h", []),
    ("u d~ > e+ ve", []),
    ("u u~ > g g", []),
    ("g g > g g", []),
    ("u u~ > w+ w-", []),
    ("u d~ > w+ z", []),
    ("u d~ > w+ a", []),
    ("u u~ > z a", []),
    ("u u~ > a a", []),
    ("u u > u u", []),
    ("u u~ > z z", []),
    ("u u~ > z h", []),
    ("u d~ > w+ h", []),
    ("u u~ > w+ w- a", []),
    ("g g > t t~", []),
    ("u u~ > t t~", []),
    ("u u~ > t t~ g", []),
    ("g g > t t~ h", []),
    ("h h > h h", []),
    ("u d~ > w+ g", []),
    ("u u~ > z g", []),
    ("u g > w+ d", []),
    ("u u~ > z z g", []),
    ("g g > t t~ g", []),
    ("u u~ > z h g", []),
    ("u d~ > w+ h g", []),
    ("u d~ > w+ z g", []),
    ("u u~ > w+ w- g", []),
    ("g g > w+ d u~", []),
    ("g g > z u u~", []),
    ("u d~ > w+ g g", []),
    ("u u~ > z g g", []),
    ("u s > d c h g", []),
    ("u s > d c h h h", []),
    ("u d > u d h", []),
    ("u d > u d h h", []),
    ("u d > u d h h h", []),
    ("u d~ > w+ g g g", []),
    ("u u~ > z g g g", []),
    ("g g > t t~ h g", []),
    ("u s > d c h g g", []),
    ("u u~ > z z g g", []),
    ("u d~ > w+ h g g", []),
    ("u u > u u h h", []),
    ("u u > u u h h h", []),
    ("u u~ > w+ w- g g", []),
    ("u d~ > w+ z g g", []),
    ("u d~ > w+ h g g g", []),
]

# all-gluon processes run by the colour-ordered block kernel (gluon_process.cu, one unit per count)
GLUON_PROCESSES = [(5, "g g > g g g"), (6, "g g > g g g g")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-I", INCLUDE, "-I", CSRC, "-I", GEN]
STATIC_SOURCES = ["me_runtime.cu", "me_server.cu", "me_grid.cu"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _hash(*parts):
    h = hashlib.sha256()
    for p in parts:
        h.update(p.encode() if isinstance(p, str) else p)
    return h.hexdigest()[:16]


def _hel_loop_choice(prog):
    """None (the code generator's threshold on program length), or the form forced for every process
    whose straight-line program exceeds ME_HEL_LOOP_FLOPS FP32 flops per event when that is set (to
    compare the two forms on the same process)."""
    limit = os.environ.get("ME_HEL_LOOP_FLOPS")
    if not limit:
        return None
    from paper_1305_0708_gb300.compiler.codegen import _Emitter
    probe = _Emitter(prog, "probe", "mixed")
    probe.generate()
    return probe.flops32 > float(limit)


def generate_units():
    """Run the process compiler; returns [(tag, path, meta)]."""
    sys.path.insert(0, ROOT)
    from paper_1305_0708_gb300.compiler.program import compile_process
    from paper_1305_0708_gb300.compiler.codegen import generate_source, process_symbol
    from paper_1305_0708_gb300.compiler.model import PARTICLES
    os.makedirs(GEN, exist_ok=True)
    units = []
    for name, aliases in PROCESSES:
        tag = process_symbol(name)
        prog = compile_process(name)
        # ME_INTERLEAVE=1 emits the straight-line programs in the helicity loop's order (each
        # amplitude after its new sub-currents), to compare the two orders on the same processes
        src, info = generate_source(prog, tag, hel_loop=_hel_loop_choice(prog),
                                    interleave=os.environ.get("ME_INTERLEAVE") == "1")
        path = os.path.join(GEN, tag + ".cu")
        if not os.path.exists(path) or open(path).read() != src:
            with open(path, "w") as f:
                f.write(src)
        ncomb = 1
        for l in prog.legs:
            ncomb *= len(l.hels)
        meta = dict(name=name, aliases=aliases, tag=tag, n_ext=prog.n_ext, params=info["params"],
                    n_hel=ncomb, n_hel_live=len(prog.live), n_colour=prog.n_colour, n_diagrams=len(prog.amps),
                    flops_amp=info["flops_amp"], flops_fp64=info["flops_fp64"], flops_colour=0.0,
                    pdg=[PARTICLES[l.particle].pdg for l in prog.legs])
        units.append((tag, path, meta))
    # all-gluon units: recursion tables, colour matrix, registry entries
    from paper_1305_0708_gb300.compiler import gluon as gl
    from paper_1305_0708_gb300.compiler.diagrams import generate, parse
    for ng, name in GLUON_PROCESSES:
        hsrc, tab = gl.header(ng)
        hpath = os.path.join(GEN, f"gluon_tables{ng}.h")
        if not os.path.exists(hpath) or open(hpath).read() != hsrc:
            with open(hpath, "w") as f:
                f.write(hsrc)
        f3, f4 = 158.0, 194.0
        cur = sum(len(v3) * f3 + len(v4) * f4 + 8 for _, v3, v4 in tab["currents"][ng - 1:])
        amp = sum(len(v3) * f3 + len(v4) * f4 + 28 for _, v3, v4 in tab["amps"])
        colour_fl = 8.0 * len(tab["amps"]) ** 2
        nh = 2 ** (ng - 1)
        _, amps = generate(parse(name))
        meta = dict(name=name, aliases=[], tag=f"gluon{ng}", n_ext=ng, params=["GS"], n_hel=2 ** ng,
                    n_hel_live=2 ** ng, n_colour=len(tab["amps"]), n_diagrams=len(amps), flops_amp=nh * (cur + amp),
                    flops_fp64=nh * (cur + amp + colour_fl), flops_colour=nh * colour_fl, pdg=[21] * ng, gluon=ng)
        units.append((f"gluon{ng}", None, meta))
    # double-float tables
    from paper_1305_0708_gb300.compiler import dftables
    tpath = os.path.join(GEN, "dfloat_tables.h")
    tsrc = dftables.header()
    if not os.path.exists(tpath) or open(tpath).read() != tsrc:
        with open(tpath, "w") as f:
            f.write(tsrc)
    # registry
    lines = ['#include "me_internal.h"', "namespace me {"]
    entries = []
    for tag, _, m in units:
        lines.append(f'extern "C" void me_register_{tag}(ProcessDesc* d);')
    for tag, _, m in units:
        pn = ", ".join(f'"{p}"' for p in m["params"]) or '"ZERO"'
        lines.append(f"static const char* const params_{tag}[] = {{{pn}}};")
        lines.append(f"static const int pdg_{tag}[] = {{{', '.join(str(x) for x in m['pdg'])}}};")
        for nm in [m["name"]] + m["aliases"]:
            entries.append((tag, nm, m))
    lines.append(f"static ProcessDesc table[{len(entries)}];")
    lines.append("static bool ready = false;")
    lines.append("static void init() {")
    for i, (tag, nm, m) in enumerate(entries):
        np_ = max(len(m["params"]), 1)
        lines.append(f'  table[{i}].name = "{nm}"; table[{i}].n_params = {np_}; table[{i}].param_names = params_{tag};')
        lines.append(f"  table[{i}].n_hel = {m['n_hel']}; table[{i}].n_hel_live = {m['n_hel_live']}; "
                     f"table[{i}].n_colour = {m['n_colour']}; table[{i}].n_diagrams = {m['n_diagrams']};")
        lines.append(f"  table[{i}].flops_amp = {float(m['flops_amp'])!r}; table[{i}].flops_fp64 = {float(m['flops_fp64'])!r}; "
                     f"table[{i}].flops_colour = {float(m['flops_colour'])!r}; "
                     f"table[{i}].pdg = pdg_{tag};")
        lines.append(f"  me_register_{tag}(&table[{i}]);")
    lines.append("  ready = true;")
    lines.append("}")
    lines.append(f"int registry_size() {{ return {len(entries)}; }}")
    lines.append("ProcessDesc* registry_entry(int i) { if (!ready) init(); return &table[i]; }")
    lines.append("}  // namespace me")
    reg = "\n".join(lines) + "\n"
    rpath = os.path.join(GEN, "registry.cu")
    if not os.path.exists(rpath) or open(rpath).read() != reg:
        with open(rpath, "w") as f:
            f.write(reg)
    with open(os.path.join(BUILD, "processes.json"), "w") as f:
        json.dump([m for _, _, m in units], f, indent=1)
    return units, rpath


def _headers_hash():
    parts = []
    for d in (CSRC, INCLUDE, GEN):
        for fn in sorted(os.listdir(d)):
            if fn.endswith((".cuh", ".h")):
                parts.append(open(os.path.join(d, fn), "rb").read())
    return _hash(*parts)


def _compile(src, obj, hh, verbose, extra=()):
    stamp = obj + ".hash"
    h = _hash(open(src, "rb").read(), hh, " ".join(NVCC_FLAGS), " ".join(extra))
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == h:
        return obj, False
    cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-6000:]}")
    with open(stamp, "w") as f:
        f.write(h)
    return obj, True


def build(verbose=False, jobs=None):
    """Generate, compile and link; returns the path of libme.so."""
    units, rpath = generate_units()
    os.makedirs(os.path.join(BUILD, "obj"), exist_ok=True)
    hh = _headers_hash()
    jobs_list = [(os.path.join(CSRC, s), os.path.basename(s) + ".o", ()) for s in STATIC_SOURCES]
    for tag, path, m in units:
        if m.get("gluon"):
            jobs_list.append((os.path.join(CSRC, "gluon_process.cu"), f"{tag}.o", (f"-DNGLUON={m['gluon']}",)))
        else:
            jobs_list.append((path, os.path.basename(path) + ".o", ()))
    jobs_list.append((rpath, "registry.cu.o", ()))
    objs = []
    jobs = jobs or min(len(jobs_list), os.cpu_count() or 4)
    changed = False
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, s, os.path.join(BUILD, "obj", o), hh, verbose, extra) for s, o, extra in jobs_list]
        for f in futs:
            o, ch = f.result()
            objs.append(o)
            changed |= ch
    if changed or not os.path.exists(LIB):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
