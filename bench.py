#!/usr/bin/env python3
"""Benchmark of the arrested-Newton-flow step on one GB300 (or N replicas).

Default workload: the B=4 cubic rational map on a 128^3 lattice (h = 0.1,
m = 1), FP32 field/velocity/force arithmetic with FP64 energy, baryon-number
and virial sums.  One bench step is one flow iteration over the lattice
(fused step kernel + the speculative-arrest fix-up check).  The metric is
interior site-updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload on its own GPU
(independent problems, no data-path collective): value = all ranks' site
updates / the slowest rank's time.  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "Gsite-updates/s of arrested Newton flow, FP32/batched vs FP64 at 1e-5 rel. energy"
UNIT = "Gsite-updates/s"
BYTES_PER_SITE_F32 = 64   # read phi, v; write phi', v' (16 B each)
BYTES_PER_SITE_F64 = 128
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0     # GB/s, used only when the measured peaks file is absent
# FP operations per site-update (FMA = 2): the formulas evaluated plainly, once
# per site, as the FP64 tile kernel first did (ncu op counts dadd + dmul +
# 2 dfma of one launch on a 64^3 lattice, divided by its 60^3 interior sites;
# the hand tallies of the formulas give 590 and 860: the rest is the square
# root and division sequences and the sums).  The kernels now cancel terms
# and share minors, and execute fewer; these counts stay the definition.
FLOPS_PER_SITE = 621      # the standard model
FLOPS_PER_SITE_EXT = 888  # with the Section 7.8 potentials and sextic term
FLOPS_PER_SITE_POT = 638  # potentials only (the standard count + their 17-operation tally)
# FP64 operations (FMA = 2) the diagnostic kernels execute, from ncu op
# counts (dadd + dmul + 2 dfma) on the 128^3 field; each formula is evaluated
# once per site and pass, so these are their arithmetic:
OBS_FP64_FLOPS_PER_SITE = 1032          # Section 5 observables: 124 + 908 per interior site
RENDER_VOLUME_FP64_FLOPS_PER_SITE = 183  # volume record + normalisation, per lattice site
GRAPH_CHUNK = 250         # iterations per captured CUDA graph


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def alu_peaks(sk):
    """Measured FMA throughput of this GPU (TFLOP/s): packed FP32 pairs, FP64."""
    return {"fp32_tflops": round(sk.measure_fma_peak(sk.PEAK_FP32), 2),
            "fp64_tflops": round(sk.measure_fma_peak(sk.PEAK_FP64), 4),
            "method": "skyrme_measure_fma_peak: 8 independent FMA chains per thread, "
                      "8 CTAs of 256 threads per SM, best of 3 timed launches"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_indices(n: int, rank: int, ws: int):
    """Contiguous, balanced share of n independent items for one rank."""
    lo = n * rank // ws
    hi = n * (rank + 1) // ws
    return list(range(lo, hi))


def reduce_over_ranks(local_ms: float, local_units: float, ws: int):
    """(slowest rank's time, all ranks' units): the whole-job numbers."""
    if ws <= 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if (
        dist.get_backend() == "nccl") else torch.device("cpu")
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def lattice_of(sk, wl, prec):
    return sk.Lattice(wl.n, wl.h, wl.m, prec, m_y=wl.m_y, m_z=wl.m_z, m_w=wl.m_w, c6=wl.c6)


def oracle_mass(oracle, wl):
    """The oracle's model argument: the pion mass, or the extension model."""
    return oracle.Model(wl.m, wl.m_y, wl.m_z, wl.m_w, wl.c6) if wl.extended else wl.m


def flops_per_site(wl):
    if not wl.extended:
        return FLOPS_PER_SITE
    return FLOPS_PER_SITE_EXT if wl.c6 != 0.0 else FLOPS_PER_SITE_POT


def step_kernel_key(wl, prec):
    """Name of the step kernel a workload runs on (the traffic record key):
    the FP32 streaming kernel for the standard model and the potentials, the
    tile kernels for FP64 and for the sextic term."""
    if prec == 32 and wl.streaming:
        return f"step_f32_{wl.name}"
    return f"step_tile_f{prec}_{wl.name}" if wl.extended else f"step_f64_{wl.name}"


def launches_per_step(wl, prec):
    """Kernel launches of one ARRESTED iteration: the FP32 streaming step
    corrects its own arrest mispredictions; the tile kernels (FP64, the
    sextic term) are followed by a fix-up check launch."""
    return 1 if (prec == 32 and wl.streaming) else 2


def l2_note(wl):
    mb = 4 * (16 if wl.precision == 32 else 32) * int(np.prod(wl.n)) / 1e6
    rel = "larger than" if mb > 129 else "smaller than"
    return f"inputs {rel} L2: 4 field/velocity buffers of {mb / 4:.1f} MB = {mb:.0f} MB vs 129 MB"


def workload_config(wl):
    return {
        "workload": wl.name,
        "lattice": list(wl.n),
        "h": wl.h,
        "m": wl.m,
        **({"m_y": wl.m_y, "m_z": wl.m_z, "m_w": wl.m_w, "c6": wl.c6} if wl.extended else {}),
        "dt": wl.dt,
        "dt_configured": wl.dt_configured,
        "seed": wl.description,
        "interior_sites": wl.interior_sites,
        "precision": "fp32 field/velocity/force, fp64 energy/B/virial sums and arrest test"
                     if wl.precision == 32 else "fp64 throughout",
        "l2": l2_note(wl),
        "parallelism": "replicas (one lattice per GPU)",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid_hint: str | None):
        self.uuid = (uuid_hint or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[1].lower()]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------ our kernels
def source_code_only(text: str) -> str:
    """C/CUDA source without its comments and with whitespace runs collapsed
    (the sources hashed here hold no comment markers inside string literals)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_fingerprint(kernel_key: str):
    """Hash of the code of a step kernel's sources: the FP32 streaming
    kernel (keys step_f32_*) or the tile kernels (every other key), with
    their shared header; comments and layout do not count."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2604_25876_gb300", "csrc")
    src = "flow_f32.cu" if kernel_key.startswith("step_f32_") else "flow_generic.cu"
    for name in (src, "skyrme_device.cuh"):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(source_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str, per_launch_sites: int):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel_key)
    except Exception:
        return None
    if not rec or rec.get("fingerprint") != kernel_fingerprint(kernel_key):
        return None
    scale = per_launch_sites / float(rec["sites"])
    return float(rec["dram_bytes_per_launch"]) * scale


def run_ours(args, ws, rank, local):
    import torch

    import paper_2604_25876_gb300 as sk

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sk.load()
    wl = workloads.ALL[args.workload]()
    prec = wl.precision
    lat = lattice_of(sk, wl, prec)
    st = sk.State(lat, dev)
    seed = sk.Seed.from_spec(wl.seed)
    sk.init_field(lat, seed, st)
    torch.cuda.synchronize(dev)  # the seed is written on the current stream; the flow runs on another
    stream = torch.cuda.current_stream(dev)
    K, W = args.steps, args.warmup
    sites = wl.interior_sites

    # the timed iterations replay CUDA graphs of CHUNK iterations each
    stream = torch.cuda.Stream(dev)
    chunk = min(K, GRAPH_CHUNK)
    graphs = [sk.FlowGraph(lat, st, wl.dt, chunk, sk.ARRESTED, stream)]
    if K % chunk:
        graphs.append(sk.FlowGraph(lat, st, wl.dt, K % chunk, sk.ARRESTED, stream))
    plan = [graphs[0]] * (K // chunk) + graphs[1:]
    warm = sk.FlowGraph(lat, st, wl.dt, W, sk.ARRESTED, stream)

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in plan]
    # the W warm-up iterations run as a graph right before the timed ones, so
    # that the timed region starts on a GPU that was just busy, not after the
    # clock sampler's idle start-up
    warm.launch(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for (a, b), gr in zip(ev, plan):
        a.record(stream)
        gr.launch(stream)
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    iter_ms = [a.elapsed_time(b) / gr.nsteps for (a, b), gr in zip(ev, plan)]
    # the same K-step region timed again (each repeat continues the flow):
    # the spread of single passes, next to the one pass the line reports
    repeats = []
    for _ in range(max(0, args.repeats)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        for gr in plan:
            gr.launch(stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        repeats.append(sites * K / (a.elapsed_time(b) * 1e-3) / 1e9)
    for gr in graphs + [warm]:
        gr.close()
    rep = sk.read_report(lat, st)
    if rep["status"] != 0:
        raise RuntimeError(f"device status {rep['status']}")

    total_ms, all_units = reduce_over_ranks(total_ms, float(sites) * K, ws)
    value = all_units / (total_ms * 1e-3) / 1e9

    # roofline of the dominant kernel: algorithmic bytes per launch over the
    # mean duration of one iteration (step launch + fix-up check)
    hbm, peak_kind = peaks()
    alu = alu_peaks(sk)
    mean_iter = statistics.fmean(iter_ms)
    # the roofline is the slower of the HBM and ALU bounds (site-updates/s)
    bytes_site = BYTES_PER_SITE_F32 * (1 if prec == 32 else 2)
    alu_tflops = alu["fp32_tflops"] if prec == 32 else alu["fp64_tflops"]
    fps = flops_per_site(wl)
    key = step_kernel_key(wl, prec)
    hbm_bound = hbm * 1e9 / bytes_site / 1e9
    alu_bound = alu_tflops * 1e12 / fps / 1e9
    traffic = recorded_traffic(key, sites)
    bounds = {"hbm_bound_gsites": round(hbm_bound, 2), "alu_bound_gsites": round(alu_bound, 3),
              "alu_peaks": alu, "algorithmic_flops_per_site": fps,
              "algorithmic_bytes_per_site": bytes_site, "kernel": key}
    if hbm_bound <= alu_bound:
        achieved = bytes_site * sites / (mean_iter * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved / hbm, 4),
                    "traffic": traffic,
                    **target_note(achieved / hbm, traffic, mean_iter, hbm, bytes_site * sites),
                    "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                    if peak_kind == "measured" else "fallback 6.8 TB/s",
                    "duration": "mean per iteration (every launch of an iteration) from CUDA "
                                "events around each graph replay", **bounds}
    else:
        tfl = fps * sites / (mean_iter * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": round(tfl, 4), "peak": alu_tflops,
                    "unit": "TFLOP/s", "frac": round(tfl / alu_tflops, 4),
                    "traffic": traffic,
                    "peak_source": "measured FP%d FMA throughput (skyrme_measure_fma_peak)" % prec,
                    "duration": "mean per iteration (every launch of an iteration) from CUDA "
                                "events around each graph replay", **bounds}

    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": K,
           "warmup": W, "ms_per_step": round(total_ms / K, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == 32 else "f64",
           "data": "synthetic",
           "config": workload_config(wl), "roofline": roofline,
           "gpu_launches": launches_per_step(wl, prec) * K, "graph_chunk": chunk, "clocks": clk,
           "repeats": spread(repeats, f"{len(repeats)} more passes of the same {K} graph-replayed "
                                      "iterations, each continuing the flow"),
           "flow": {"steps_done": rep["steps"], "arrests": rep["arrests"],
                    "fixups": rep["fixups"], "E": rep["E"], "B": rep["B"],
                    "virial": rep["virial"], "delta": rep["delta"],
                    **({"E6": rep["E6"]} if wl.extended else {})}}

    if not args.no_extras and prec == 32 and not wl.extended:
        out["batched"] = run_batched(sk, torch, dev, ws, rank)
    if rank == 0 and not args.no_extras and args.workload == "b4_cubic_128":
        # the sizes the 70% target is judged on: inputs far larger than L2
        out["c3_256"] = run_size_leg(sk, torch, dev, workloads.b8_cluster_256(), hbm, iters=50,
                                     fp64=True)
        out["c5_512"] = run_size_leg(sk, torch, dev, workloads.b32_cluster_512(), hbm, iters=20,
                                     fp64=False)
        out["slabs_256"] = run_slab_leg(sk, torch, dev, workloads.b8_cluster_256(), iters=40)
    if rank == 0 and not args.no_extras:
        out["e2e"] = run_e2e(sk, torch, dev, wl, K)
        if prec == 32:
            # as many iterations as the FP32 flow ran (warm-up, timed pass and
            # repeats), so that the two energies are of the same iteration
            out["fp64_gpu"] = run_fp64_compare(sk, torch, dev, wl, rep["steps"], rep, alu["fp64_tflops"])
        if not wl.extended:
            out["diagnostics"] = run_diagnostics(sk, torch, dev, wl, alu["fp64_tflops"])
            if prec == 32:
                out["variants"] = run_variants(sk, torch, dev, wl, hbm)
        out["cpu_baseline"] = run_cpu_baseline(wl, args.cpu_seconds)
    return out


ROOFLINE_TARGET = 0.70  # fraction of the roofline the FP32 and batched flows aim at


def target_note(frac, traffic, iter_ms, hbm, alg_bytes):
    """Whether the roofline target is met, and the DRAM bytes the kernel
    actually moved (ncu) as a bandwidth: below the algorithmic bytes the
    working set is partly served by L2 and HBM is not what binds."""
    note = {"target_frac": ROOFLINE_TARGET, "target_met": bool(frac >= ROOFLINE_TARGET)}
    if traffic:
        dram = traffic / (iter_ms * 1e-3) / 1e9
        note["dram_gbs_measured_traffic"] = round(dram, 1)
        note["dram_frac_measured_traffic"] = round(dram / hbm, 4)
        note["traffic_over_algorithmic"] = round(traffic / alg_bytes, 3)
    return note


def spread(values, what):
    if not values:
        return {"n": 0}
    return {"n": len(values), "median": round(statistics.median(values), 4),
            "min": round(min(values), 4), "max": round(max(values), 4), "unit": UNIT,
            "what": what}


def run_size_leg(sk, torch, dev, wl, hbm, iters, repeats=5, fp64=False):
    """One FP32 workload at full size: `repeats` timed graph launches of
    `iters` iterations each (median, min, max), the HBM roofline of the
    median with the recorded DRAM traffic, and optionally the FP64 GPU flow
    over the same iterations for the FP32 energy error."""
    lat = lattice_of(sk, wl, 32)
    st = sk.State(lat, dev)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    g = sk.FlowGraph(lat, st, wl.dt, iters, sk.ARRESTED)
    g.launch()  # warm-up
    g.stream.synchronize()
    vals = []
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        g.launch()
        b.record(g.stream)
        g.stream.synchronize()
        vals.append(wl.interior_sites * iters / (a.elapsed_time(b) * 1e-3) / 1e9)
    g.close()
    rep = sk.read_report(lat, st)
    sites = wl.interior_sites
    med = statistics.median(vals)
    iter_ms = sites / (med * 1e9) * 1e3
    key = step_kernel_key(wl, 32)
    traffic = recorded_traffic(key, sites)
    achieved = BYTES_PER_SITE_F32 * med
    out = {"workload": wl.name, "lattice": list(wl.n), "interior_sites": sites,
           "dt": wl.dt, "value": round(med, 4), "unit": UNIT,
           "repeats": spread(vals, f"{repeats} graph launches of {iters} iterations"),
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                        "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
                        "kernel": key,
                        **target_note(achieved / hbm, traffic, iter_ms, hbm,
                                      BYTES_PER_SITE_F32 * sites)},
           "steps_done": rep["steps"], "arrests": rep["arrests"], "E": rep["E"], "B": rep["B"],
           "status": int(rep["status"]), "l2": l2_note(wl)}
    del st
    torch.cuda.empty_cache()
    if fp64:
        lat64 = lattice_of(sk, wl, 64)
        st64 = sk.State(lat64, dev)
        sk.init_field(lat64, sk.Seed.from_spec(wl.seed), st64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize(dev)
        a.record(stream)
        r64 = sk.flow_step(lat64, wl.dt, rep["steps"], sk.ARRESTED, st64, report=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        out["fp64_gpu"] = {"value": round(sites * rep["steps"] / (ms * 1e-3) / 1e9, 4),
                           "unit": UNIT, "steps": r64["steps"], "E_fp64": r64["E"]}
        out["fp32_energy_rel_err"] = abs(rep["E"] - r64["E"]) / abs(r64["E"])
        del st64
        torch.cuda.empty_cache()
    return out


def run_slab_leg(sk, torch, dev, wl, iters, nslabs=2):
    """The x-slab decomposition on one GPU: the lattice in `nslabs` slab
    states whose records are combined and halos copied on the device every
    iteration, against the whole-lattice flow of the same iterations.  The
    difference is the cost of the decomposition's extra launches and copies
    (on several GPUs the copies become NCCL transfers)."""
    from paper_2604_25876_gb300.slab import LocalSlabFlow
    lat = lattice_of(sk, wl, 32)
    st = sk.State(lat, dev)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    seed = st.field().clone()
    flow = LocalSlabFlow(lat, nslabs, dev)
    flow.load(seed)
    torch.cuda.synchronize(dev)  # loaded on the current stream; the flow runs on another
    stream = torch.cuda.Stream(dev)
    how = "CUDA graph of the slab iterations (torch.cuda.graph)"
    graph = None
    with torch.cuda.stream(stream):
        flow.flow(wl.dt, 2, sk.ARRESTED)  # warm-up, outside any capture
    stream.synchronize()
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
            flow.flow(wl.dt, iters, sk.ARRESTED)
        flow_steps = lambda: graph.replay()
    except Exception as e:  # measured without a graph instead
        graph = None
        how = f"direct launches (graph capture failed: {type(e).__name__})"
        flow.load(seed)

        def flow_steps():
            with torch.cuda.stream(stream):
                flow.flow(wl.dt, iters, sk.ARRESTED)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        flow_steps()  # a graph replays on the current stream
        b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    reps = [s.st.report() for s in flow.slabs]
    # the whole-lattice flow over the same iterations
    g = sk.FlowGraph(lat, st, wl.dt, iters, sk.ARRESTED)
    g.launch()
    g.stream.synchronize()
    a.record(g.stream)
    g.launch()
    b.record(g.stream)
    g.stream.synchronize()
    ms_whole = a.elapsed_time(b)
    g.close()
    sites = wl.interior_sites
    return {"workload": wl.name, "slabs": nslabs, "iterations": iters, "how": how,
            "value": round(sites * iters / (ms * 1e-3) / 1e9, 4), "unit": UNIT,
            "whole_lattice_value": round(sites * iters / (ms_whole * 1e-3) / 1e9, 4),
            "overhead": round(ms / ms_whole - 1.0, 4),
            "slab_reports_agree": len({(r["E"], r["arrests"], r["steps"]) for r in reps}) == 1,
            "status": sorted({int(r["status"]) for r in reps})}


def run_batched(sk, torch, dev, ws, rank, steps=200, count=64):
    """The batched workload: `count` (64) smoothed-noise lattices with sides
    drawn from {64,...,128}, sharded over the ranks, one persistent launch per
    iteration replayed from a CUDA graph after the autotuner has chosen the
    tile."""
    wls = workloads.batched_noise(count=count, steps=steps)
    mine = [wls[i] for i in shard_indices(len(wls), rank, ws)]
    lats, states = [], []
    for w in mine:
        lat = sk.Lattice(w.n, w.h, w.m, 32)
        st = sk.State(lat, dev)
        sk.init_field(lat, sk.Seed.from_spec(w.seed), st)
        lats.append(lat)
        states.append(st)
    torch.cuda.synchronize(dev)  # seeds written before the tuning and flow on another stream
    batch = sk.Batch(lats, states, [w.dt for w in mine])
    stream = torch.cuda.Stream(dev)
    tile, tune_ms = batch.autotune(trials=3, stream=stream)
    chunk = min(steps, 100)
    graph = sk.FlowGraph(nsteps=chunk, batch=batch, stream=stream)
    graph.launch()
    stream.synchronize()
    reps = steps // chunk
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(reps):
        graph.launch()
    b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b)
    sites = sum(w.interior_sites for w in mine)
    ms_all, units = reduce_over_ranks(ms, float(sites) * reps * chunk, ws)
    info = batch.tile()
    rr = batch.reports()
    graph.close()
    batch.close()
    hbm, _ = peaks()
    gs = units / (ms_all * 1e-3) / 1e9
    return {"value": round(gs, 4), "unit": UNIT, "instances": len(wls),
            "interior_sites": sum(w.interior_sites for w in wls), "steps": reps * chunk,
            "tile": [info["ty"], info["tz"]], "grid": info["grid"],
            "split": "plane-balanced" if info.get("balanced") else "even by centres",
            "autotune_ms_per_step": round(tune_ms, 4),
            "roofline": {"bound": "hbm", "achieved": round(gs * BYTES_PER_SITE_F32, 1),
                         "peak": hbm, "unit": "GB/s",
                         "frac": round(gs * BYTES_PER_SITE_F32 / hbm, 4)},
            "arrests": int(sum(r["arrests"] for r in rr)),
            "fixups": int(sum(r["fixups"] for r in rr)),
            "status": sorted(set(int(r["status"]) for r in rr))}


def run_e2e(sk, torch, dev, wl, K):
    """The same metric through the C ABI's host-buffer call (skyrme_flow_host):
    upload the seed field from pinned host memory, K flow iterations, the
    report and the final field downloaded; all inside the timed region."""
    lat = lattice_of(sk, wl, wl.precision)
    st = sk.State(lat, dev)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    host_in = torch.empty(st.phi[0].shape, dtype=lat.dtype, pin_memory=True)
    host_in.copy_(st.phi[0])
    host_out = torch.empty_like(host_in, pin_memory=True)
    stream = torch.cuda.current_stream(dev)

    def job():
        """One job through skyrme_flow_host: every byte of its input and
        output crosses the host link inside the timed region."""
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        t_wall = time.perf_counter()
        a.record(stream)
        sk.flow_host(lat, wl.dt, K, sk.ARRESTED, st, host_in, host_out, report=True, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b), time.perf_counter() - t_wall

    job()  # warm-up: the first call of a lattice encodes its tensor maps and kernel attributes
    runs = [job() for _ in range(3)]
    ms, wall = sorted(runs)[1]
    bytes_field = host_in.numel() * host_in.element_size()
    return {"value": round(wl.interior_sites * K / (ms * 1e-3) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": bytes_field / K,
            "d2h_bytes_per_step": (bytes_field + 128) / K,
            "wall_s": round(wall, 4),
            "jobs_ms": [round(r[0], 4) for r in runs],
            "what": f"the median of 3 jobs (after one untimed) of {K} iterations each through "
                    "skyrme_flow_host with pinned host buffers: seed upload, flow, report and field "
                    "download"}


def run_fp64_compare(sk, torch, dev, wl, nsteps, rep32, fp64_tflops):
    """FP64 GPU flow of the same workload for the same iterations (validated
    against the FP64 oracle by the parity tests): its throughput, its ALU
    roofline and the FP32 energy error relative to it."""
    lat = lattice_of(sk, wl, 64)
    st = sk.State(lat, dev)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rep = sk.flow_step(lat, wl.dt, nsteps, sk.ARRESTED, st, report=True)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    gs = wl.interior_sites * nsteps / (ms * 1e-3) / 1e9
    tfl = gs * flops_per_site(wl) / 1e3
    return {"value": round(gs, 4), "unit": UNIT, "steps": nsteps,
            "roofline": {"bound": "alu", "achieved": round(tfl, 4),
                         "peak": fp64_tflops, "unit": "TFLOP/s",
                         "frac": round(tfl / fp64_tflops, 4),
                         "peak_source": "measured FP64 FMA throughput (skyrme_measure_fma_peak)",
                         "algorithmic_flops_per_site": flops_per_site(wl)},
            "E_fp64": rep["E"],
            "fp32_energy_rel_err": abs(rep32["E"] - rep["E"]) / abs(rep["E"])
            if rep32["steps"] == rep["steps"] else None}


# The run-to-tolerance leg relaxes the whole workload in FP32 and in FP64;
# it runs on lattices of at most this many interior sites (the 128^3
# workloads), with these iteration caps, so that the bench stays short.
UNTIL_MAX_SITES = 2_100_000
UNTIL_MAX_STEPS = {32: 40000, 64: 8000}


def run_variants(sk, torch, dev, wl, hbm, tol=1e-3, chunk=250, iters=1000):
    """The other flow modes and the run-to-tolerance driver (Section 3,
    Section 7.9): Newton and gradient flow throughput from graph replays of
    the same step kernel, and the time to relax the workload's seed to
    max |F| <= tol in one launch of a WHILE-node graph, in FP32 and in FP64
    (128^3-class lattices only, with an iteration cap)."""
    if wl.interior_sites > UNTIL_MAX_SITES:
        return {"skipped": f"run only on lattices of at most {UNTIL_MAX_SITES} interior sites "
                           "(the FP64 relaxation of a larger one takes minutes)"}
    out = {}
    for name, mode, bps in (("newton", sk.NEWTON, BYTES_PER_SITE_F32),
                            ("gradient", sk.GRADIENT, BYTES_PER_SITE_F32 // 2)):
        lat = lattice_of(sk, wl, 32)
        st = sk.State(lat, dev)
        sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
        g = sk.FlowGraph(lat, st, wl.dt, chunk, mode)
        g.launch()  # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        for _ in range(iters // chunk):
            g.launch()
        b.record(g.stream)
        g.stream.synchronize()
        g.close()
        ms = a.elapsed_time(b) / (iters // chunk * chunk)
        rep = sk.read_report(lat, st)
        gbs = bps * wl.interior_sites / (ms * 1e-3) / 1e9
        out[name] = {"value": round(wl.interior_sites / (ms * 1e-3) / 1e9, 4), "unit": UNIT,
                     "steps": iters // chunk * chunk, "status": int(rep["status"]),
                     "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm,
                                  "unit": "GB/s", "frac": round(gbs / hbm, 4),
                                  "algorithmic_bytes_per_site": bps}}
    until = {"tol": tol, "chunk": chunk}
    for prec in (32, 64):
        lat = lattice_of(sk, wl, prec)
        st = sk.State(lat, dev)
        sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
        g = sk.FlowGraph(lat, st, wl.dt, chunk, sk.ARRESTED, until=(tol, UNTIL_MAX_STEPS[prec]))
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        g.launch()
        b.record(g.stream)
        g.stream.synchronize()
        g.close()
        ms = a.elapsed_time(b)
        rep = sk.read_report(lat, st)
        r = {"steps": rep["steps"], "ms": round(ms, 3), "E": rep["E"], "delta": rep["delta"],
             "converged": bool(rep["delta"] <= tol), "status": int(rep["status"]),
             "gsites": round(wl.interior_sites * rep["steps"] / (ms * 1e-3) / 1e9, 4)}
        if prec == 32 and rep["steps"] % chunk == 0:
            # the same iterations from the same seed as plain graph replays:
            # the cost of the device-side stop test
            sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
            g = sk.FlowGraph(lat, st, wl.dt, chunk, sk.ARRESTED)
            torch.cuda.synchronize(dev)
            a.record(g.stream)
            for _ in range(rep["steps"] // chunk):
                g.launch()
            b.record(g.stream)
            g.stream.synchronize()
            g.close()
            r["plain_graphs_ms"] = round(a.elapsed_time(b), 3)
            r["until_overhead"] = round(ms / a.elapsed_time(b) - 1.0, 4)
        until["fp%d" % prec] = r
    until["energy_rel_diff"] = abs(until["fp32"]["E"] - until["fp64"]["E"]) / abs(until["fp64"]["E"])
    until["time_ratio_fp64_over_fp32"] = round(until["fp64"]["ms"] / until["fp32"]["ms"], 2)
    out["until"] = until
    return out


def run_diagnostics(sk, torch, dev, wl, fp64_tflops, reps=5):
    """Timings of the Section 5 observables and the Section 6.2 volume render
    of the workload's field after 200 flow iterations (standard model)."""
    lat = lattice_of(sk, wl, wl.precision)
    st = sk.State(lat, dev)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    sk.flow_step(lat, wl.dt, 200, sk.ARRESTED, st, report=False)
    sites, nall = wl.interior_sites, int(np.prod(wl.n))
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    obs_ms = timed(lambda: sk.observables(lat, st))
    vol = torch.empty(tuple(wl.n) + (4,), dtype=torch.float64, device=dev)
    vol_ms = timed(lambda: sk.render_volume(lat, st, out=vol))
    c, s_ = math.cos(0.6), math.sin(0.6)
    rp = sk.render_params(1024, 768, view=[[c, 0, s_], [0, 1, 0], [-s_, 0, c]], step=0.005)
    ray_ms = timed(lambda: sk.render_rays(vol, rp))
    def fp64_roofline(flops, ms, per):
        tfl = flops / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": round(tfl, 4), "peak": fp64_tflops,
                "unit": "TFLOP/s", "frac": round(tfl / fp64_tflops, 4), "fp64_flops_per": per,
                "peak_source": "measured FP64 FMA throughput (skyrme_measure_fma_peak)"}

    obs = {"ms": round(obs_ms, 4), "gsites": round(sites / (obs_ms * 1e-3) / 1e9, 4),
           "what": "skyrme_observables: two FP64 passes over the interior, host read-back",
           "roofline": fp64_roofline(OBS_FP64_FLOPS_PER_SITE * sites, obs_ms,
                                     f"{OBS_FP64_FLOPS_PER_SITE} per interior site")}
    return {"observables": obs,
            "render_volume": {"ms": round(vol_ms, 4),
                              "roofline": fp64_roofline(RENDER_VOLUME_FP64_FLOPS_PER_SITE * nall,
                                                        vol_ms,
                                                        f"{RENDER_VOLUME_FP64_FLOPS_PER_SITE} per "
                                                        "lattice site")},
            "render_rays": {"ms": round(ray_ms, 4), "pixels": 1024 * 768, "step": 0.005,
                            "mpixels_per_s": round(1024 * 768 / (ray_ms * 1e-3) / 1e6, 2)}}


def run_cpu_baseline(wl, seconds):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the workload (the first iterations of the same lattice and seed)."""
    import oracle
    oracle.build()
    n = wl.n
    if wl.seed.kind == "rational_map":
        phi = oracle.seed_rational_map(n, wl.h, wl.seed.B, wl.seed.profile_scale)
    else:
        phi = oracle.seed_product(n, wl.h, wl.seed.positions, wl.seed.quaternions,
                                  wl.seed.profile_scale, wl.seed.symmetrise)
    st = oracle.new_state(phi)
    m = oracle_mass(oracle, wl)
    t = time.perf_counter()
    oracle.flow(st, wl.h, m, wl.dt, 1)
    one = time.perf_counter() - t
    steps = max(1, int(seconds / max(one, 1e-6)))
    t = time.perf_counter()
    oracle.flow(st, wl.h, m, wl.dt, steps)
    el = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(wl.interior_sites * steps / el / 1e9, 6), "unit": UNIT,
            "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 oracle iterations of the full {n[0]}^3 workload "
                      f"({el:.1f} s, after one untimed iteration)",
            "single_core": single_core_oracle(wl)}


def single_core_oracle(wl, timed_steps=2):
    """The same oracle on one host core (OMP_NUM_THREADS=1 in a child
    process): one untimed and `timed_steps` timed iterations of the workload."""
    code = (
        "import json, sys, time; sys.path.insert(0, %r)\n"
        "import oracle, workloads\n"
        "wl = workloads.ALL[%r]()\n"
        "phi = oracle.seed_rational_map(wl.n, wl.h, wl.seed.B, wl.seed.profile_scale)\n"
        "st = oracle.new_state(phi)\n"
        "oracle.flow(st, wl.h, wl.m, wl.dt, 1)\n"
        "t = time.perf_counter(); oracle.flow(st, wl.h, wl.m, wl.dt, %d)\n"
        "print(json.dumps({'s': time.perf_counter() - t}))\n") % (ROOT, wl.name, timed_steps)
    if wl.seed.kind != "rational_map":
        return {"skipped": "single-core figure taken on the rational-map workloads"}
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=120)
        el = json.loads(r.stdout.strip().splitlines()[-1])["s"]
    except Exception as e:
        return {"skipped": f"single-core run failed: {type(e).__name__}"}
    return {"value": round(wl.interior_sites * timed_steps / el / 1e9, 6), "unit": UNIT,
            "cores": 1, "sample": f"{timed_steps} FP64 oracle iterations of the full "
                                  f"{wl.n[0]}^3 workload ({el:.1f} s) with OMP_NUM_THREADS=1"}


# ------------------------------------------------------------ reference arm
def run_reference(args):
    import oracle
    oracle.build()
    wl = workloads.b4_cubic_128()
    K, W = args.steps, args.warmup
    phi = oracle.seed_rational_map(wl.n, wl.h, wl.seed.B, wl.seed.profile_scale)
    st = oracle.new_state(phi)
    t = time.perf_counter()
    oracle.flow(st, wl.h, wl.m, wl.dt, 1)
    one = time.perf_counter() - t
    # bounded sample: each reference step covers a slab of the lattice so that
    # the whole run stays within about two minutes
    budget = 120.0
    frac = min(1.0, budget / max((K + W) * one, 1e-9))
    nx = max(5, int(round(wl.n[0] * frac)))
    slab = (nx, wl.n[1], wl.n[2])
    sphi = np.ascontiguousarray(phi[:nx])
    oracle.apply_vacuum_boundary(sphi)
    sst = oracle.new_state(sphi)
    oracle.flow(sst, wl.h, wl.m, wl.dt, W)
    t = time.perf_counter()
    oracle.flow(sst, wl.h, wl.m, wl.dt, K)
    el = time.perf_counter() - t
    sites = (nx - 4) * (wl.n[1] - 4) * (wl.n[2] - 4)
    value = sites * K / el / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{K} FP64 oracle iterations on a {slab[0]}x{slab[1]}x{slab[2]} slab of the "
              f"{wl.n[0]}^3 workload")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": K, "warmup": W,
            "ms_per_step": round(el * 1e3 / K, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(workloads.ALL), default="b4_cubic_128",
                    help="the 128^3 B=4 workload (default) is the one the metric is quoted on")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--repeats", type=int, default=5,
                    help="extra passes of the K timed iterations, reported as a spread")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e, FP64 and CPU-baseline legs")
    ap.add_argument("--batched-only", type=int, default=0, metavar="COUNT",
                    help="run only the batched leg, on COUNT lattices for --steps iterations "
                         "(a smaller batch for profiling); prints its record")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    ws, rank, local = dist_env()

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.batched_only > 0:
        import torch

        import paper_2604_25876_gb300 as sk
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        sk.load()
        out = run_batched(sk, torch, dev, ws, rank, steps=max(100, args.steps // 100 * 100),
                          count=args.batched_only)
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
