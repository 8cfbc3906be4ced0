#!/usr/bin/env python
"""Benchmark of the hot path: one complex-Langevin step followed by gauge-
cooling sweeps on a 32^4 lattice (SU(3) Wilson + clover theta-term,
beta = 6.2, theta = 1.0, Haar-random SU(3) start), measured in
site-updates/s (one site through one CL step and all of that step's cooling
sweeps).

Prints ONE JSON line (rank 0).  The headline `value` is the FP64 form; the
FP32-storage form (FP32 links, FP64 exponentials / re-projection /
reductions) runs on the same seeded noise and is reported under
"forms".  Per-kernel durations come from CUDA events recorded by the library
around each launch on the lattice's stream; `roofline` is for the kernel
that dominates the step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 (torchrun): every rank advances its own lattice (independent chains,
no data-path collective); value = all ranks' site-updates / max rank time.
--impl reference times the FP64 CPU oracle (the reference implementation of
this method) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(L=(32, 32, 32, 32), beta=6.2, theta=1.0, seed=1, eps=0.005, sweeps=10, alpha=1.0)
WORKLOAD_NAME = ("32^4 SU(3) Wilson + clover theta, beta 6.2, theta 1.0, Haar hot start; "
                 "1 CL step (eps 0.005) + 10 gauge-cooling sweeps (alpha_ad = alpha / D_1, alpha 1)")
METRIC = "CL+cooling site-updates/s"
UNIT = "site-updates/s"
# Bytes that must move per site-update (links read + written once per CL step
# and once per fused cooling sweep, plus f): FP64 13,952 B, FP32 links 7,616 B.
ALG_BYTES = {"fp64": 1152 + 10 * 1280, "fp32": 576 + 10 * 704}
CPU_SAMPLE_L = (8, 8, 8, 8)


# Floating-point operations per site of each kernel of the step, counted
# from the kernel source (FMA = 2 flops; the transcendental calls of the
# Box-Muller noise are not counted).  Building blocks: 3x3 complex product
# 198, product-accumulate 216, adjugate 126, Hermitian-times-general 162.
# ncu's executed-instruction counters agree within 1 % on these sources
# (profiles/ncu_fp64_counts_24x4.md).  "pipe" is the unit the kernel loads:
# the FP64 pipe in the FP64 form; in the FP32-storage form only the
# exponentials, the re-projection and the cooling Omega stay on it.
MUL, MULACC, ADJ, HERM = 198, 216, 126, 162


# FP64 flops per unit that the FP32-storage form's FP64 work executes
# (2 x DFMA + DMUL + DADD thread instructions from ncu, 24^4, divided by the
# links or sites; profiles/ncu_fp32_update_cooling_24x4.md).  Its series stop
# at the FP32-storage tolerance, whose term count follows each argument's
# norm, so the analytic model above does not apply to them.
FP32_STORAGE_FP64_FLOPS = {"update": 4 * 663, "cool_omega": 163, "cool_grad_omega": 160}


def flop_model(prec, theta_on=True, n_taylor=15):
    expm = MUL + 6 + 72 + 36 + 16 * n_taylor + 9 * (6 + 8) + 6  # Cayley-Hamilton + Horner
    det_root = 64 + 19                                           # det + three-term cube-root series
    if theta_on:
        force = 6 * (12 * MUL + ADJ + 9 * MULACC + 162)          # per-plaquette drift, 6 planes
    else:
        force = 6 * (4 * MUL + 36)
    m = {
        "force": force,
        "clover": 4 * ADJ + 6 * (3 * MUL + ADJ + 18) + (6 * (3 * (MUL + MULACC) + 54) if theta_on else 0),
        "cool_grad": 914,
        "cool_omega": 209,
        "cool_apply": 4 * 2 * HERM,
        "cool_grad_omega": 914 + 209,
    }
    if prec == "fp64":
        m["update"] = 4 * (12 * 18 + 32 + 38 + expm + MUL + det_root + 54)
        pipe = {k: "fp64" for k in m}
    else:
        pipe = {k: "fp32" for k in m}
        for k, v in FP32_STORAGE_FP64_FLOPS.items():  # FP64 part only
            m[k] = v
            pipe[k] = "fp64"
    return m, pipe


def fp64_peak_tflops(sm_max_mhz):
    # 152 SMs x 2 FP64 FMA per SM per clock (4 flops) x clock: 1.259 TFLOP/s at 2070 MHz.
    return 152 * 4 * sm_max_mhz * 1e6 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh)
    except Exception:
        return {}


# The sources of the kernels the bench launches (their launch shapes included);
# the host runtime, the server and the chain kernel do not change them.
KERNEL_SOURCES = ("bm_tables.cuh", "df64.cuh", "expm.cuh", "k_update.cuh", "k_update_df64.cu", "k_update_f32.cu",
                  "k_update_f64.cu",
                  "kernels.cu", "launch.h",
                  "lattice.cuh", "philox.cuh", "su3.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1311_1056_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(kernel, prec, V=None, path=None):
    """Per-launch DRAM bytes of a roofline family from a committed ncu summary
    (profiles/dram_traffic.json), if taken on the current sources.  The
    capture runs a smaller lattice (capture_sites); every kernel's traffic
    grows with the sites it processes, so the bytes are scaled to V."""
    p = path or os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        e = d[prec][kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        b = e["bytes_per_launch"]
        cap = d.get("capture_sites")
        return b * (V / cap) if (V and cap) else b
    except Exception:
        return None


# Kernels of each roofline family, per form (a family's bytes per launch sum
# over its kernels: the split force runs a then b once per step).
TRAFFIC_FAMILIES = {
    "fp64": {"force": ("k_plaq_force_a<double>", "k_plaq_force_b<double>"),
             "update": ("k_update_gather<double, 0>",), "cool_apply": ("k_cool_apply_tiles<double>",),
             "cool_grad": ("k_cool_grad<double>",), "cool_omega": ("k_cool_omega<double>",),
             "cool_grad_omega": ("k_cool_grad_omega<double>",)},
    "fp32": {"force": ("k_plaq_force_ab<float>",), "update": ("k_update_gather<float, 0>",),
             "cool_apply": ("k_cool_apply_tiles<float>",), "cool_grad": ("k_cool_grad<float>",),
             "cool_omega": ("k_cool_omega<float>",), "cool_grad_omega": ("k_cool_grad_omega<float>",)},
    "df64": {"force": ("k_plaq_force_a_df", "k_plaq_force_b_df"),
             "update": ("k_update_gather<df64, 0>",), "cool_apply": ("k_cool_apply_df",),
             "cool_grad": ("k_cool_grad_df",), "cool_omega": ("k_cool_omega<df64>",)},
}


def ingest_ncu(path, out_json=None, capture_sites=None):
    """Reads ncu launch lists (--csv, metrics gpu__time_duration.sum and
    dram__bytes_{read,write}.sum, --kernel-name-base demangled; one path or a
    list), prints the per-kernel summary as a markdown table and writes the
    per-launch DRAM bytes of each roofline family to profiles/dram_traffic.json,
    stamped with the current kernel-source hash and, when given, the sites of
    the captured lattice (dram_traffic scales to the bench's lattice)."""
    import csv
    import re
    paths = [path] if isinstance(path, str) else list(path)
    rows = []
    for k, pth in enumerate(paths):
        part = list(csv.reader(line for line in open(pth) if line.startswith('"')))
        hdr = part[0]
        col = {h: i for i, h in enumerate(hdr)}
        for r in part[1:]:
            r = list(r)
            r[col["ID"]] = "%d:%s" % (k, r[col["ID"]])  # launch IDs restart in every file
            rows.append(r)
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1e-6, "nsecond": 1e-6, "us": 1e-3,
             "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3}
    launches = {}
    for r in rows:
        name = r[col["Kernel Name"]]
        name = name.split("(clgc::Geo")[0] if "(clgc::Geo" in name else name.split("(")[0]
        name = re.sub(r"^void ", "", name)
        for ns in ("(anonymous namespace)::", "<unnamed>::", "unnamed>::", "clgc::"):
            name = name.replace(ns, "")
        name = name.strip()
        d = launches.setdefault(r[col["ID"]], {"name": name})
        d[r[col["Metric Name"]]] = float(r[col["Metric Value"]].replace(",", "")) * scale[r[col["Metric Unit"]]]
    agg = {}
    for d in launches.values():
        a = agg.setdefault(d["name"], {"n": 0, "ms": 0.0, "rd": 0.0, "wr": 0.0})
        a["n"] += 1
        a["ms"] += d.get("gpu__time_duration.sum", 0.0)
        a["rd"] += d.get("dram__bytes_read.sum", 0.0)
        a["wr"] += d.get("dram__bytes_write.sum", 0.0)
    tot = sum(a["ms"] for a in agg.values())
    print("%d launches, %.1f ms of kernel time" % (len(launches), tot))
    print("| kernel | launches | total ms | share | ms / launch | DRAM read GB / launch | DRAM write GB / launch |")
    print("|---|---:|---:|---:|---:|---:|---:|")
    for n, a in sorted(agg.items(), key=lambda kv: -kv[1]["ms"]):
        print("| %s | %d | %.2f | %.1f %% | %.3f | %.3f | %.3f |" % (
            n, a["n"], a["ms"], 100 * a["ms"] / tot, a["ms"] / a["n"], a["rd"] / a["n"] / 1e9, a["wr"] / a["n"] / 1e9))
    h = kernel_source_hash()
    out = {"source_hash": h}
    if capture_sites:
        out["capture_sites"] = capture_sites
    for form, fams in TRAFFIC_FAMILIES.items():
        for fam, kernels in fams.items():
            if all(k in agg for k in kernels):
                b = sum((agg[k]["rd"] + agg[k]["wr"]) / agg[k]["n"] for k in kernels)
                out.setdefault(form, {})[fam] = {"bytes_per_launch": b, "source_hash": h}
    with open(out_json or os.path.join(ROOT, "profiles", "dram_traffic.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    return agg, out


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(seconds=10.0, L=CPU_SAMPLE_L):
    """The FP64 oracle on a bounded sample of the workload: an 8^4 lattice with
    the same parameters, one site-update (CL step + 10 sweeps) per repetition."""
    import oracle as O
    w = WORKLOAD
    U = O.hot_start(L, w["seed"])
    cp = O.cool_params(w["eps"], w["alpha"], O.D1, forced_sweeps=w["sweeps"])
    V = 1
    for v in L:
        V *= v
    reps, t0, step = 0, time.perf_counter(), 0
    while True:
        U = O.cl_step(L, U, w["beta"], w["theta"], w["eps"], w["seed"], step)
        U, _ = O.cool(L, U, cp)
        reps += 1
        step += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": V * reps / el, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d^4 lattice (%d sites), %d site-update(s) of the same workload "
                      "(1 CL step + %d sweeps), %.1f s" % (L[0], V, reps, w["sweeps"], el)}


def rank_max(x, device="cpu"):
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(sites_per_rank, ms_max, world):
    """Whole-job site-updates/s: every rank advances its own lattice (weak
    scaling), the job takes as long as the slowest rank."""
    return world * sites_per_rank / (ms_max * 1e-3)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_form(cl, torch, prec_name, args, rank, stream):
    w = WORKLOAD
    prec = {"fp64": cl.CL_FP64, "fp32": cl.CL_FP32_STORAGE, "df64": cl.CL_DF64}[prec_name]
    L = tuple(args.L) if args.L else w["L"]
    V = L[0] * L[1] * L[2] * L[3]
    lat = cl.Lattice(L, beta=w["beta"], theta=w["theta"], prec=prec, seed=w["seed"] + rank,
                     start=cl.CL_START_HOT, stream=stream.cuda_stream)
    cp = cl.make_cool(w["eps"], w["alpha"], cl.CL_D1, forced_sweeps=w["sweeps"])

    def one_step():
        cl.cl_step(lat.h, w["eps"], 1)
        cl.cl_cool(lat.h, cp, want_report=False)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    cl.cl_set_timing(lat.h, 1)
    n0 = lat.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if args.world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = lat.launches() - n0
    phases = cl.cl_get_timing(lat.h)
    cl.cl_set_timing(lat.h, 0)
    obs = lat.observables()
    return lat, V, ms, launches, phases, obs, one_step


def e2e_measure(cl, torch, lat, V, one_step, steps):
    """Through the public API with host buffers: each step copies the links in
    from pinned host memory, runs the step and reads the links back."""
    import numpy as np
    n = V * 4 * 18
    hin = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hout = torch.empty(n, dtype=torch.float64, pin_memory=True)
    a_in = hin.numpy().view(np.complex128).reshape(V, 4, 3, 3)
    a_out = hout.numpy().view(np.complex128).reshape(V, 4, 3, 3)
    cl.cl_get_links(lat.h, V, a_in)
    # one untimed round trip first (touches the output buffer and the staging buffer)
    cl.cl_set_links(lat.h, a_in)
    one_step()
    cl.cl_get_links(lat.h, V, a_out)
    torch.cuda.synchronize()
    t_set = t_step = t_get = 0.0
    t0 = time.perf_counter()
    for _ in range(steps):
        ta = time.perf_counter()
        cl.cl_set_links(lat.h, a_in)  # returns once the copy and the layout conversion are done
        tb = time.perf_counter()
        one_step()
        tc = time.perf_counter()
        cl.cl_get_links(lat.h, V, a_out)  # waits for the step, then converts and copies back
        td = time.perf_counter()
        t_set += tb - ta
        t_step += tc - tb
        t_get += td - tc
    el = (time.perf_counter() - t0) / steps
    return {"value": V / el, "unit": UNIT, "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
            "ms_per_step": el * 1e3,
            "host_ms_per_step": {"set_links": round(t_set / steps * 1e3, 3),
                                 "enqueue_step": round(t_step / steps * 1e3, 3),
                                 "step_and_get_links": round(t_get / steps * 1e3, 3)}}


# FP32 instructions per site that the DF64 kernels execute, from ncu's
# executed-instruction counters on one launch at 24^4
# (smsp__sass_thread_inst_executed_op_{ffma,fadd,fmul}_pred_on.sum divided by
# the 331,776 sites; profiles/ncu_df64_fp32_ops_24x4.md).  These kernels load
# the FP32 pipe, so their roofline is that pipe: flops (FFMA = 2) against the
# FP32 peak, and FP32-pipe instructions against the pipe's issue rate (the
# error-free transformations are mostly FADDs, one flop per issue slot).
DF64_FP32_OPS_PER_SITE = {
    "force": {"ffma": 43740, "fadd": 126684, "fmul": 14580},
    "cool_grad": {"ffma": 1323, "fadd": 4211, "fmul": 513},
    "cool_apply": {"ffma": 2160, "fadd": 5472, "fmul": 720},
}


def fp32_peak_tflops(sm_max_mhz):
    # 152 SMs x 128 FP32 FMA per SM per clock (256 flops) x clock: 80.5 TFLOP/s at 2070 MHz.
    return 152 * 128 * 2 * sm_max_mhz * 1e6 / 1e12


def roofline_of(prec_name, V, phases, sm_max_mhz, theta_on=True):
    """Roofline of the kernel that dominates the step (a single-kernel phase),
    against the peak of the pipe that kernel loads."""
    fm, pipe = flop_model("fp64" if prec_name == "df64" else prec_name, theta_on)
    single = {k: v for k, v in phases.items() if k in ("force", "update", "cool_grad", "cool_omega",
                                                       "cool_apply", "cool_grad_omega")}
    dom = max(single, key=lambda k: single[k][0])
    ms_tot, n = phases[dom]
    per = ms_tot / max(n, 1)
    if prec_name == "df64":
        # double-float arithmetic runs on the FP32 pipe: its executed FP32
        # operations (ncu counts) against the FP32 peak
        ops = DF64_FP32_OPS_PER_SITE.get(dom)
        peak = fp32_peak_tflops(sm_max_mhz)
        src = ("executed FP32 operations of the double-float kernels (ncu, 24^4, FFMA = 2 flops) against "
               "152 SMs x 128 FP32 FMA/clk x %d MHz (FP32 is not in MEASURED_PEAKS.json)" % sm_max_mhz)
        if not ops:
            return {"kernel": dom, "bound": "alu", "pipe": "fp32", "achieved": None, "peak": round(peak, 4),
                    "unit": "TFLOP/s", "frac": None, "traffic": dram_traffic(dom, prec_name, V),
                    "avg_launch_ms": round(per, 4), "launches": n, "peak_source": src}
        flops = (2 * ops["ffma"] + ops["fadd"] + ops["fmul"]) * V
        inst = (ops["ffma"] + ops["fadd"] + ops["fmul"]) * V
        ach = flops / (per * 1e-3) / 1e12
        inst_rate = inst / (per * 1e-3) / 1e12
        inst_peak = peak / 2
        return {"kernel": dom, "bound": "alu", "pipe": "fp32", "achieved": round(ach, 4),
                "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                "fp32_pipe_inst_per_s": round(inst_rate * 1e12, 1), "fp32_pipe_inst_frac": round(inst_rate / inst_peak, 4),
                "traffic": dram_traffic(dom, prec_name, V), "flops_per_launch": flops,
                "avg_launch_ms": round(per, 4), "launches": n, "peak_source": src}
    flops = fm[dom] * V
    if pipe[dom] == "fp64":
        peak = fp64_peak_tflops(sm_max_mhz)
        src = "152 SMs x 2 FP64 FMA/clk x %d MHz (FP64 is not in MEASURED_PEAKS.json)" % sm_max_mhz
    else:
        peak = fp32_peak_tflops(sm_max_mhz)
        src = "152 SMs x 128 FP32 FMA/clk x %d MHz" % sm_max_mhz
    ach = flops / (per * 1e-3) / 1e12
    return {"kernel": dom, "bound": "alu", "pipe": pipe[dom], "achieved": round(ach, 4),
            "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(ach / peak, 4),
            "traffic": dram_traffic(dom, prec_name, V), "flops_per_launch": flops,
            "avg_launch_ms": round(per, 4), "launches": n, "peak_source": src}


def native(args):
    import torch
    from paper_1311_1056_gb300 import build, cl

    ws, rank, local = dist_setup()
    args.world = ws
    if ws > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    cl.load()
    stream = torch.cuda.Stream()
    peaks = measured_peaks()
    sampler = ClockSampler(local)
    sampler.start()
    lat, V, ms, launches, phases, obs, one_step = run_form(cl, torch, "fp64", args, rank, stream)
    clocks = sampler.stop()
    ms_max = rank_max(ms, "cuda")
    value = job_value(V, ms_max, ws)
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "lattice": list(args.L or WORKLOAD["L"]),
                   "beta": WORKLOAD["beta"], "theta": WORKLOAD["theta"], "eps": WORKLOAD["eps"],
                   "cooling": "alpha_ad = alpha / D_1 (normalised unitarity norm), alpha 1, "
                              "10 sweeps per step (fixed count)",
                   "precision": "fp64 links and arithmetic",
                   "l2": "no flush: the link fields (604 MB fp64 / 302 MB fp32) exceed the 129 MB L2",
                   "parallelism": "replicas x%d (independent chains)" % ws},
        "gpu_launches": launches,
        "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in phases.items()},
        "roofline": roofline_of("fp64", V, phases, sm_max),
        "hbm": {"alg_bytes_per_site_update": ALG_BYTES["fp64"],
                "achieved_gbs": round(ALG_BYTES["fp64"] * value / ws / 1e9, 2),
                "peak_gbs": peaks.get("hbm_gbs"),
                "frac": round(ALG_BYTES["fp64"] * value / ws / 1e9 / peaks["hbm_gbs"], 5)
                if peaks.get("hbm_gbs") else None},
        "observables_after": {k: obs[k] for k in ("plaq_re", "un", "q_re", "q_im")},
        "clocks": clocks,
    }
    result["e2e"] = e2e_measure(cl, torch, lat, V, one_step, max(2, min(args.steps, 5)))
    result["e2e"]["value"] = job_value(V, rank_max(result["e2e"]["ms_per_step"], "cuda"), ws)
    lat.close()
    if not args.no_fp32:
        lat32, V32, ms32, l32, ph32, obs32, _ = run_form(cl, torch, "fp32", args, rank, stream)
        lat32.close()
        ms32 = rank_max(ms32, "cuda")
        result["forms"] = {"fp32_storage": {
            "value": job_value(V32, ms32, ws), "ms_per_step": ms32, "gpu_launches": l32,
            "dtype": "f32 links + f64 exp/reprojection/reductions",
            "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in ph32.items()},
            "roofline": roofline_of("fp32", V32, ph32, sm_max),
            "hbm_frac": round(ALG_BYTES["fp32"] * V32 / (ms32 * 1e-3) / 1e9 / peaks["hbm_gbs"], 5)
            if peaks.get("hbm_gbs") else None,
            "observables_after": {k: obs32[k] for k in ("plaq_re", "un", "q_re", "q_im")}}}
    if not args.no_df64:
        latd, Vd, msd, ld, phd, obsd, _ = run_form(cl, torch, "df64", args, rank, stream)
        latd.close()
        msd = rank_max(msd, "cuda")
        result.setdefault("forms", {})["df64"] = {
            "value": job_value(Vd, msd, ws), "ms_per_step": msd, "gpu_launches": ld,
            "dtype": "df64 links (hi + lo floats); link algebra, noise, exponentials and re-projection "
                     "in double-float on the FP32 pipe; f64 final sums of the reductions",
            "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in phd.items()},
            "roofline": roofline_of("df64", Vd, phd, sm_max),
            "observables_after": {k: obsd[k] for k in ("plaq_re", "un", "q_re", "q_im")},
            "abs_diff_vs_fp64_after": {k: abs(obsd[k] - obs[k]) for k in ("plaq_re", "un", "q_re", "q_im")}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


def reference(args):
    """The oracle arm; under torchrun only rank 0 runs it, the others return."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return None
    import oracle as O
    w = WORKLOAD
    L = CPU_SAMPLE_L
    V = L[0] * L[1] * L[2] * L[3]
    U = O.hot_start(L, w["seed"])
    cp = O.cool_params(w["eps"], w["alpha"], O.D1, forced_sweeps=w["sweeps"])
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        U = O.cl_step(L, U, w["beta"], w["theta"], w["eps"], w["seed"], i)
        U, _ = O.cool(L, U, cp)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = V / (ms * 1e-3)
    sample = "%d^4 lattice (%d sites) per step, same parameters as the workload" % (L[0], V)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "lattice": list(WORKLOAD["L"]), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------- batched ensemble
# Cooling: alpha_ad = alpha / D_2 with alpha = 0.1 (with alpha = 1 the step
# eps alpha / <|f|> passes the stability bound of the gradient flow once <|f|>
# drops below ~0.3 and the field explodes), 0..10 sweeps, no sweep within 1e-6
# of SU(3), stop below 1 % relative progress.  k_ref: the adaptive Langevin
# step size (eps_n = eps min(1, k_ref / K_max)); typical K_max of these
# lattices is 17-19, and without it chains at beta 5.6, theta 2 run away.
BATCH = dict(eps=0.005, alpha=0.1, n_min=0, n_max=10, tol_rel=0.01, d_floor=1e-6, k_ref=12.0)
BATCH_NAME = ("ensemble of independent chains, L^4 with L uniform in {8, 12, 16}, beta ~ U[5.6, 6.2], "
              "theta in {0, 0.5, 1, 1.5, 2}, cold start; each CL step (eps 0.005) followed by adaptive "
              "cooling (alpha_ad = 0.1 / D_2, 0..10 sweeps, stop below 1 % relative progress or within "
              "1e-6 of SU(3)), adaptive step size k_ref 12")


def _log(msg):
    print("[bench %.1fs] %s" % (time.perf_counter() - _T0, msg), file=sys.stderr, flush=True)


_T0 = time.perf_counter()


def _run_chains(cl, torch, chains, prec, n_steps, batched, tune, fused=False):
    """Advance every chain by n_steps; returns (seconds, observables, reports,
    launches, tuned blocks).  batched: one graph launch per step for all chains
    (each chain on its own stream, or with fused one launch per kernel family
    over all chains); otherwise one chain after the other with eager calls."""
    cp = cl.make_cool(BATCH["eps"], BATCH["alpha"], cl.CL_D2_MEANABS, n_min=BATCH["n_min"],
                      n_max=BATCH["n_max"], tol_rel=BATCH["tol_rel"], d_floor=BATCH["d_floor"])
    lats = [cl.Lattice(c["L"], beta=c["beta"], theta=c["theta"], prec=prec, seed=c["seed"],
                       start=cl.CL_START_COLD, own_stream=True) for c in chains]
    for lat in lats:
        lat.set_adaptive_step(BATCH["k_ref"])
    tuned = {}
    if tune:
        for c, lat in zip(chains, lats):
            blocks, _ = lat.autotune(BATCH["eps"], cp, reps=3, use_cache=True)
            tuned["%d^4 theta%s0" % (c["L"][0], "!=" if c["theta"] else "=")] = blocks
    n0 = sum(l.launches() for l in lats)
    torch.cuda.synchronize()
    _log("  %d lattices ready" % len(lats))
    if batched:
        b = cl.Batch(lats, BATCH["eps"], [cp] * len(lats), fused=fused)
        torch.cuda.synchronize()
        _log("  batch graph captured")
        t0 = time.perf_counter()
        b.run(n_steps)
        b.synchronize()
        sec = time.perf_counter() - t0
        b.close()
    else:
        t0 = time.perf_counter()
        for lat in lats:
            for _ in range(n_steps):
                lat.step(BATCH["eps"], 1)
                cl.cl_cool(lat.h, cp, want_report=False)
            lat.synchronize()
        sec = time.perf_counter() - t0
    launches = sum(l.launches() for l in lats) - n0
    obs = [l.observables() for l in lats]
    reps = [l.last_cool_report() for l in lats]
    for l in lats:
        l.close()
    return sec, obs, reps, launches, tuned


def batch_mode(args):
    # more hardware work queues than the default 8, so that the chains'
    # streams do not serialise behind one another (read at CUDA init)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch
    from paper_1311_1056_gb300 import build, cl, workloads

    build.build()
    cl.load()
    chains = workloads.ensemble(args.chains, seed=0)
    n_steps = args.batch_steps
    total = sum(workloads.sites(c) for c in chains) * n_steps
    # warm-up (module load, graph upload, clocks): a short batched run of 4 chains
    _run_chains(cl, torch, chains[:4], cl.CL_FP32_STORAGE, 3, True, False)
    sampler = ClockSampler(0)
    sampler.start()
    arms = {}
    for name, prec, batched, fused in (("batched_fp32", cl.CL_FP32_STORAGE, True, False),
                                       ("fused_fp32", cl.CL_FP32_STORAGE, True, True),
                                       ("batched_fp64", cl.CL_FP64, True, False),
                                       ("fused_fp64", cl.CL_FP64, True, True),
                                       ("batched_df64", cl.CL_DF64, True, False),
                                       ("alone_fp32", cl.CL_FP32_STORAGE, False, False),
                                       ("alone_fp64", cl.CL_FP64, False, False)):
        if args.batch_arms and name not in args.batch_arms:
            continue
        _log("arm %s" % name)
        arms[name] = _run_chains(cl, torch, chains, prec, n_steps, batched, batched and not fused, fused)
        _log("arm %s: %.2f s" % (name, arms[name][0]))
    clocks = sampler.stop()
    ref_obs = arms["alone_fp64"][1] if "alone_fp64" in arms else None

    def obs_err(obs):
        if ref_obs is None:
            return None
        out = {}
        for k in ("plaq_re", "plaq_im", "un", "q_re", "q_im"):
            d = [abs(a[k] - b[k]) for a, b in zip(obs, ref_obs) if np.isfinite(a[k]) and np.isfinite(b[k])]
            out[k] = {"max": float(max(d)) if d else None, "median": float(np.median(d)) if d else None}
        return out

    res = {}
    for name, (sec, obs, reps, launches, tuned) in arms.items():
        res[name] = {"value": total / sec, "seconds": round(sec, 4), "gpu_launches": launches,
                     "nonfinite_chains": sum(1 for o in obs if not np.isfinite(o["un"])),
                     "mean_sweeps_last_step": float(np.mean([r["sweeps"] for r in reps])),
                     "abs_err_vs_alone_fp64": obs_err(obs)}
        if tuned:
            res[name]["autotuned_blocks"] = tuned
    def ratio(a, b):
        return res[a]["value"] / res[b]["value"] if a in res and b in res else None

    best = max((k for k in ("batched_fp32", "fused_fp32") if k in res), key=lambda k: res[k]["value"], default=None)
    line = {
        "metric": "batched CL+cooling site-updates/s", "unit": UNIT,
        "value": res[best]["value"] if best else None, "best_fp32_arm": best, "higher_is_better": True,
        "n_gpus": 1, "dtype": "f32 links, f64 exp/reductions", "data": "synthetic",
        "config": {"workload": BATCH_NAME, "chains": len(chains), "steps": n_steps,
                   "sites_per_step": total // n_steps,
                   "sizes": {str(L): sum(1 for c in chains if c["L"][0] == L) for L in workloads.ENSEMBLE_SIZES}},
        "speedup_vs_alone_fp64": ratio(best, "alone_fp64") if best else None,
        "fused_vs_graph_fp32": ratio("fused_fp32", "batched_fp32"),
        "fused_vs_graph_fp64": ratio("fused_fp64", "batched_fp64"),
        "df64_speedup_vs_alone_fp64": ratio("batched_df64", "alone_fp64"),
        "arms": res, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- serving
SERVE_NAME = ("request trace: Poisson arrivals, L^4 with L = round(exp U[ln 4, ln 24]), beta ~ U[5.6, 6.2], "
              "theta ~ U[0, 2], 100..2000 CL steps (eps 0.005) each followed by adaptive cooling "
              "(alpha_ad = 0.1 / D_2, 0..10 sweeps), adaptive step size k_ref 12; HBM budget 150 GB")


# A request whose unitarity norm climbs past this after a chunk has run away
# (the norm stays within 1e-3 of 1 on healthy chains and goes to inf within
# tens of steps once past ~1.01): the server stops it there.
SERVE_RUNAWAY_UN = 1.1


def _serve_once(cl, trace, prec, slots, graphs, tune):
    cp = cl.make_cool(BATCH["eps"], BATCH["alpha"], cl.CL_D2_MEANABS, n_min=BATCH["n_min"],
                      n_max=BATCH["n_max"], tol_rel=BATCH["tol_rel"], d_floor=BATCH["d_floor"])
    reqs = [cl.make_request(r["L"], r["beta"], r["theta"], BATCH["eps"], r["steps"], seed=r["seed"],
                            start=cl.CL_START_COLD, tag=r["id"]) for r in trace]
    arrivals = [r["t"] - trace[0]["t"] for r in trace]
    cfg = cl.make_server_config(hbm_budget_bytes=150e9, max_slots=slots, prec=prec, chunk_steps=8,
                                use_graphs=graphs, cool=cp, blocks_from_autotune=tune, k_ref=BATCH["k_ref"],
                                runaway_un=SERVE_RUNAWAY_UN)
    with cl.Server(cfg) as srv:
        res = srv.run_trace(reqs, arrivals)
        st = srv.stats()
    return {r["tag"]: r for r in res}, st


def serve_mode(args):
    import numpy as np
    from paper_1311_1056_gb300 import build, cl, workloads

    build.build()
    cl.load()
    trace = workloads.trace(args.requests, rate=args.rate, seed=0)
    work = sum(workloads.sites(r) * r["steps"] for r in trace)
    # warm-up: a few small requests through both configurations
    warm = workloads.trace(4, rate=1000.0, seed=1, steps=(20, 20), l_range=(4, 8))
    _serve_once(cl, warm, cl.CL_FP32_STORAGE, args.slots, True, True)
    if not args.no_serve_df64:
        _serve_once(cl, warm, cl.CL_DF64, args.slots, True, True)
    _serve_once(cl, warm, cl.CL_FP64, 1, False, False)
    sampler = ClockSampler(0)
    sampler.start()
    arms = {}
    _log("serve: served_fp32")
    arms["served_fp32"] = _serve_once(cl, trace, cl.CL_FP32_STORAGE, args.slots, True, True)
    if not args.no_serve_df64:
        _log("serve: served_df64")
        arms["served_df64"] = _serve_once(cl, trace, cl.CL_DF64, args.slots, True, True)
    _log("serve: one_at_a_time_fp64")
    arms["one_at_a_time_fp64"] = _serve_once(cl, trace, cl.CL_FP64, 1, False, False)
    _log("serve: done")
    clocks = sampler.stop()
    ref = arms["one_at_a_time_fp64"][0]
    out = {}
    for name, (res, st) in arms.items():
        lat = np.array([res[r["id"]]["t_done"] - res[r["id"]]["t_submit"] for r in trace])
        span = max(v["t_done"] for v in res.values()) - min(v["t_submit"] for v in res.values())
        errs = {}
        both = [i for i in res if res[i]["status"] == cl.CL_OK and ref[i]["status"] == cl.CL_OK]
        for k in ("plaq_re", "un", "q_re"):
            d = np.array([abs(res[i]["obs"][k] - ref[i]["obs"][k]) for i in both])
            errs[k] = {"max": float(d.max()) if d.size else None,
                       "median": float(np.median(d)) if d.size else None}
        sites = {r["id"]: workloads.sites(r) for r in trace}
        done_work = sum(sites[i] * res[i]["n_steps"] for i in res)  # site-steps actually run
        out[name] = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                     "mean_s": float(lat.mean()), "makespan_s": span, "value": done_work / span,
                     "requests_per_s": len(trace) / span, "peak_active": st["peak_active"],
                     "peak_bytes": st["peak_bytes"],
                     "runaway": sum(1 for v in res.values() if v["status"] == cl.CL_ERR_RUNAWAY),
                     "nonfinite": sum(1 for v in res.values() if v["status"] == cl.CL_ERR_NONFINITE),
                     "steps_run": int(sum(v["n_steps"] for v in res.values())),
                     "abs_err_vs_one_at_a_time_fp64": errs}
    a, b = out["served_fp32"], out["one_at_a_time_fp64"]
    line = {"metric": "served CL+cooling site-updates/s; p50/p99 latency", "unit": UNIT,
            "value": a["value"], "higher_is_better": True, "n_gpus": 1,
            "dtype": "f32 links, f64 exp/reductions", "data": "synthetic",
            "config": {"workload": SERVE_NAME, "requests": len(trace), "rate_per_s": args.rate,
                       "slots": args.slots, "chunk_steps": 8, "site_steps": work},
            "p50_s": a["p50_s"], "p99_s": a["p99_s"],
            "vs_one_at_a_time_fp64": {"throughput_x": a["value"] / b["value"], "p50_x": b["p50_s"] / a["p50_s"],
                                      "p99_x": b["p99_s"] / a["p99_s"]},
            "arms": out, "clocks": clocks}
    if "served_df64" in out:  # the same serving at FP64-grade accuracy (double-float links)
        c = out["served_df64"]
        line["served_df64_vs_one_at_a_time_fp64"] = {"throughput_x": c["value"] / b["value"],
                                                     "p50_x": b["p50_s"] / c["p50_s"],
                                                     "p99_x": b["p99_s"] / c["p99_s"]}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- studies
def cooling_study_mode(args):
    """NEXT-2: D_0 / D_1 / D_2 decay of the distance under cooling alone."""
    from paper_1311_1056_gb300 import build, cl, studies

    build.build()
    cl.load()
    out = {"metric": "gauge-cooling decay d(sweeps), D_0 / D_1 / D_2", "chains": {}, "su3_8x4": {}}
    for n in (1, 10, 100, 1000):
        for mode, alpha in (("D0", 1.0), ("D1", 1.0), ("D2", 1.0), ("D2", 0.1)):
            d = studies.chain_cooling(n, mode, alpha=alpha, eps=0.01, sweeps=args.sweeps)
            out["chains"]["N=%d %s alpha=%g" % (n, mode, alpha)] = studies.summarize(d[:, 0])
            _log("chain N=%d %s alpha=%g done" % (n, mode, alpha))
    for mode, alpha in (("D0", 1.0), ("D1", 1.0), ("D2", 1.0), ("D2", 0.1)):
        d = studies.lattice_cooling((8, 8, 8, 8), mode, alpha=alpha, eps=0.01, sweeps=min(args.sweeps, 1000))
        out["su3_8x4"]["%s alpha=%g" % (mode, alpha)] = studies.summarize(d)
        _log("SU(3) %s alpha=%g done" % (mode, alpha))
    print(json.dumps(out), flush=True)


def theta_scan_mode(args):
    """NEXT-4: plaquette and Q_L against theta_L^2 on 6^4 (Sec. 5)."""
    import numpy as np
    from paper_1311_1056_gb300 import build, cl, studies

    build.build()
    cl.load()
    t0 = time.perf_counter()
    res = studies.theta_scan(n_steps=args.scan_steps)
    sec = time.perf_counter() - t0
    rows = []
    for r in res:
        p, q = r["plaq"], r["q"]
        keep = slice(len(p) // 4, None)  # drop the first quarter (thermalisation)
        fin = np.isfinite(p[keep]).all()

        def mean_err(x):
            x = x[keep]
            nb = 10
            b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
            return complex(x.mean()), float(np.abs(b - b.mean()).std() / np.sqrt(nb))
        pm, pe = mean_err(p)
        qm, qe = mean_err(q)
        rows.append({"beta": r["beta"], "theta2": r["theta2"], "finite": bool(fin),
                     "langevin_time": round(r["langevin_time"], 3),
                     "plaq": [round(pm.real, 6), round(pm.imag, 6)], "plaq_err": round(pe, 6),
                     "Q": [round(qm.real, 4), round(qm.imag, 4)], "Q_err": round(qe, 4),
                     "un_final": float(r["un"][-1])})
    print(json.dumps({"metric": "theta scan, 6^4 SU(3), CL + adaptive cooling", "steps": args.scan_steps,
                      "seconds": round(sec, 2), "rows": rows}), flush=True)


def precision_mode(args):
    """The FP32-storage and DF64 forms against the FP64 form, every observable."""
    from paper_1311_1056_gb300 import build, cl, studies

    build.build()
    cl.load()
    L = tuple(args.L) if args.L else WORKLOAD["L"]
    tab = studies.precision_table(L=L, checkpoints=(1, 10, 100))
    tab_df = studies.precision_table(L=L, checkpoints=(1, 10, 100), prec=cl.CL_DF64)
    print(json.dumps({"metric": "FP32-storage error vs FP64 on identical noise", "workload": WORKLOAD_NAME,
                      "lattice": list(L), "table": {str(k): v for k, v in tab.items()},
                      "df64_table": {str(k): v for k, v in tab_df.items()}}), flush=True)


# 16^4 long runs (the theta-scan config): FP64, FP32 storage and DF64
# ensembles of independent chains (disjoint Philox seeds per form), compared
# in distribution after thermalisation.
# Without the adaptive step size most theta = 2 chains (and some theta = 1
# chains) run away within 1000 steps at eps 0.005; with k_ref = 12 (the
# batch and serving workloads' value) every chain stays finite.
LONGRUN = dict(L=(16, 16, 16, 16), beta=6.0, thetas=(0.0, 0.5, 1.0, 2.0), eps=0.005, every=10, k_ref=12.0)
LONGRUN_NAME = ("16^4 SU(3) Wilson + clover theta, beta 6.0, theta in {0, 0.5, 1, 2}, cold start; CL steps at "
                "eps 0.005 with the adaptive step size (k_ref 12) and adaptive cooling (alpha_ad = 0.1 / D_2, "
                "0..10 sweeps, stop below 1 % relative progress or within 1e-6 of SU(3)); observables every 10 "
                "steps")


def longrun_mode(args):
    import numpy as np
    from paper_1311_1056_gb300 import build, cl, studies

    build.build()
    cl.load()
    w = LONGRUN
    L = tuple(args.L) if args.L else w["L"]
    forms = (("fp64", cl.CL_FP64, 0), ("fp32_storage", cl.CL_FP32_STORAGE, 100), ("df64", cl.CL_DF64, 200))
    floors = {"fp32_storage": 1e-6, "df64": 1e-12}
    sampler = ClockSampler(0)
    sampler.start()
    out = {}
    for theta in w["thetas"]:
        row = {}
        stats = {}
        for name, prec, off in forms:
            seeds = [7000 + off + i for i in range(args.longrun_chains)]
            t0 = time.perf_counter()
            ser = studies.longrun(L, w["beta"], theta, prec, seeds, args.longrun_steps, every=w["every"],
                                  eps=w["eps"], k_ref=w["k_ref"])
            sec = time.perf_counter() - t0
            st = studies.chain_means(ser)
            stats[name] = st
            row[name] = {"mean": dict(zip(studies.SERIES_KEYS, st["mean"].tolist())),
                         "err": dict(zip(studies.SERIES_KEYS, st["err"].tolist())),
                         "chains": st["chains"], "nonfinite_chains": st["dropped"], "seconds": round(sec, 2),
                         "seeds": seeds}
            if name == "fp64":
                row[name]["first_chain_series"] = {k: ser[0, :, j].tolist()
                                                   for j, k in enumerate(studies.SERIES_KEYS)}
            _log("longrun theta %.1f %s: %.1f s" % (theta, name, sec))
        for name in ("fp32_storage", "df64"):
            if stats[name]["chains"] < 2 or stats["fp64"]["chains"] < 2:
                row["z_%s_vs_fp64" % name] = None  # too few finite chains for an error bar
                continue
            z = studies.compare_means(stats[name], stats["fp64"], floors[name])
            row["z_%s_vs_fp64" % name] = dict(zip(studies.SERIES_KEYS, np.round(z, 3).tolist()))
        out["%g" % theta] = row
    clocks = sampler.stop()
    zs = [v for row in out.values() for key in row if key.startswith("z_") and row[key] for v in row[key].values()]
    runaway = sum(row[f]["nonfinite_chains"] for row in out.values() for f in ("fp64", "fp32_storage", "df64"))
    print(json.dumps({"metric": "long-run observables per arithmetic form (ensemble means, 3 sigma bar)",
                      "workload": LONGRUN_NAME, "lattice": list(L), "steps": args.longrun_steps,
                      "chains_per_form": args.longrun_chains, "thermalisation_dropped": 0.2,
                      "max_z": max(zs) if zs else None, "runaway_chains": runaway, "thetas": out,
                      "clocks": clocks}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--L", type=int, nargs=4, default=None, help="override the lattice (testing)")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-df64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--mode", choices=["step", "batch", "serve", "cooling-study", "theta-scan", "precision",
                                       "longrun"],
                    default="step",
                    help="step: the 32^4 single-chain step (default); batch: the chain ensemble; "
                         "serve: the request trace; cooling-study, theta-scan: the studies of Sec. 4-5; "
                         "longrun: 16^4 ensembles of the three arithmetic forms compared in distribution")
    ap.add_argument("--longrun-chains", type=int, default=4)
    ap.add_argument("--longrun-steps", type=int, default=1000)
    ap.add_argument("--sweeps", type=int, default=3000)
    ap.add_argument("--scan-steps", type=int, default=20000)
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--chains", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--batch-arms", nargs="*", default=None, help="batch: run only these arms")
    ap.add_argument("--no-serve-df64", action="store_true", help="serve: skip the double-float arm")
    ap.add_argument("--ingest-ncu", metavar="CSV", nargs="+", default=None,
                    help="summarise ncu launch lists with DRAM bytes and update profiles/dram_traffic.json")
    ap.add_argument("--ingest-sites", type=int, default=None,
                    help="--ingest-ncu: sites of the captured lattice (the bench scales the bytes to its own)")
    args = ap.parse_args()
    if args.ingest_ncu:
        return ingest_ncu(args.ingest_ncu, capture_sites=args.ingest_sites)
    if args.mode == "batch":
        return batch_mode(args)
    if args.mode == "serve":
        return serve_mode(args)
    if args.mode == "cooling-study":
        return cooling_study_mode(args)
    if args.mode == "theta-scan":
        return theta_scan_mode(args)
    if args.mode == "precision":
        return precision_mode(args)
    if args.mode == "longrun":
        return longrun_mode(args)
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        reference(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
