#!/usr/bin/env python3
"""Benchmark of the contraction-tree executor; prints one JSON line.

Workloads (``--workload``):

  circuit7x7  (default) one amplitude of a 7x7-qubit, 14-cycle random circuit,
              Hyper-Greedy tree sliced to W_s <= 28 (2^24 slices of up to 2^28
              complex entries per tensor); one step = a bounded sample of
              consecutive slices (``--slices``, default 2); the time per
              amplitude is extrapolated over all slices (as the paper does for
              its starred rows).  The oracle checks the GPU on sub-slices of
              the same tree sliced further, to W_s <= 20.
  ising100    Ising partition function of a random 3-regular graph,
              N = 100, beta = 0.3, J = +-1, greedy tree sliced to W_s <= 24,
              float32 leaves.  One step = one full contraction (all slices).
  circuit4x4  one amplitude of a 4x4-qubit, 8-cycle random circuit, greedy
              tree, no slicing (complex64 leaves).
  circuit5x5  one amplitude of a 5x5-qubit, 10-cycle random circuit (the
              smaller circuit that is checked in full), greedy tree.
  grad5x4     loss = mean over 64 bitstrings of ln|c_x|^2 of a 5x4-qubit,
              12-cycle circuit and its gradient with respect to the (theta, phi)
              of all 93 fSim gates, through the autograd Function (forward tree
              and reverse sweep on the GPU); one step = loss + gradient.
  node        one large complex node alone (two random tensors, M x K and
              K x N by --node-bits, default 15,13,10 = the largest node of
              the 7x7x14 slice), open M x N output: the tensor-core kernel
              measured on its own; sampled outputs checked in FP64.
  batch       1024 amplitudes of a 6x6-qubit, 12-cycle circuit (one shared
              tree, blocks of copies per launch sequence) plus 256 Ising
              networks with N even in [40, 160] in one batch (networks wider
              than 24 sliced to W_s <= 24 inside it); per-network completion
              latency p50 / p99.

Throughput = algorithmic FLOPs (8 C complex, 2 C real per slice, Eq.
vertexcon) over device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode tf32_split]
  python bench.py --impl reference ...   (the FP64 oracle on host cores)

Under torchrun each rank contracts its own network (seed = rank) or its own
slice range: weak scaling, no collective on the data path; the timing is the
max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contraction FLOP/s & % roofline per tree; s/amplitude; rel. error vs FP64 oracle"
WORKLOAD_NAMES = {
    "ising100": "ising_rr3_n100_beta0.3_greedy_ws24",
    "ising100_hyper": "ising_rr3_n100_beta0.3_hyperedge_form_greedy_ws24",
    "circuit4x4": "circuit_4x4_8cyc_greedy_amplitude",
    "circuit5x5": "circuit_5x5_10cyc_greedy_amplitude",
    "circuit7x7": "circuit_7x7_14cyc_hypergreedy_ws28_slice_sample",
    "batch": "batch_6x6_12cyc_amplitudes_plus_256_ising",
    "grad5x4": "grad_5x4_12cyc_fsim_params_64_bitstrings",
    "node": "single_complex_node",
    "sample": "sample_5x4_12cyc_open6_fidelity_mixture",
}
MODES = ["fp32", "tf32_split", "fp16_split", "bf16_split", "tf32_3m"]
# accuracy each mode is held to (relative, against the FP64 oracle run on the
# same leaf values the GPU reads)
MODE_TOL = {"fp32": 1e-5, "tf32_split": 1e-5, "fp16_split": 1e-5, "bf16_split": 1e-4, "tf32_3m": 1e-2}
L2_FLUSH_BYTES = 512 << 20
# FP32 FMA peak of one GB300: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz.
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# nominal dense tensor rates per GPU (TF32 : BF16 = 1.1 : 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
# real products executed per algorithmic product on the tensor cores
MODE_PASSES = {"tf32_split": 3, "bf16_split": 3, "fp16_split": 3, "tf32_3m": 1}
# modes whose tensor-core operands are 16-bit (kind::f16: the BF16 rate)
HALF_MODES = ("bf16_split", "fp16_split")


# DRAM bytes of the dominant launch step (the largest node's operand pack and
# tensor-core GEMM) per launch, summed over those kernels from one ncu capture
# of the default command (dram__bytes_read.sum + dram__bytes_write.sum); valid
# while the tensor-core kernel file is the one that was measured (SHA-256).
TRAFFIC = {
    ("circuit7x7", "fp16_split"): {
        "bytes": 4.798e9,  # node 1067 (M 2^15, N 2^13, K 2^10): k_pack 0.687 GB + k_umma2 4.111 GB
        "tn_tc_sha256": "7f0fb9ae8d577b371196cf51913ecf66e4ed26f029f36fc16842673446233a8f",
        "profile": "profiles/launches_circuit7x7_fp16split.md",
    },
}


def measured_traffic(workload, mode):
    import hashlib
    t = TRAFFIC.get((workload, mode))
    if t is None:
        return None, None
    src = os.path.join(ROOT, "paper_2002_01935_gb300", "csrc", "tn_tc.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if sha != t["tn_tc_sha256"]:
        return None, "kernel changed since the capture"
    return t["bytes"], t["profile"]


def tc_peak(mode, peaks):
    """Dense tensor peak of the mode's operand type: measured BF16 for the
    16-bit formats, measured BF16 x 1.1/2.25 (nominal TF32 : BF16) for TF32."""
    if mode in HALF_MODES:
        return peaks["bf16_tflops"], f"{peaks['source']} bf16 (fp16 and bf16 share the rate)"
    return peaks["bf16_tflops"] * TF32_OVER_BF16, f"{peaks['source']} bf16 x 1.1/2.25 (nominal TF32:BF16)"


def gpu_leaves(net):
    """The network as the GPU reads it (leaves rounded to complex64 /
    float32, widened back): the oracle's parity reference is computed on
    these values, so the comparison measures the executor's arithmetic and
    not the rounding of the inputs."""
    return net.as_stored()


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def wl_ising(seed: int, n: int = 100, target: float = 24.0, hyper: bool = False, simplified: bool = False):
    from paper_2002_01935_gb300 import inputs, planner, simplify
    net = inputs.random_ising_hyper(n, seed) if hyper else inputs.random_ising(n, seed)
    if simplified:
        net, _ = simplify.simplify(net)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    info = planner.tree_info(net.labels, net.dims, pairs, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target) if info.W > target else []
    info = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
    return {"net": net, "pairs": pairs, "sliced": sliced, "info": info,
            "slice_begin": 0, "slice_count": int(info.d_sliced), "oracle": "full",
            "config": {"n_vertices": n, "beta": 0.3, "J": "+-1", "graph_seed": seed,
                       "form": "hyperedge (one label per spin)" if hyper else "COPY tensor per vertex",
                       "simplified": net.meta.get("simplified"),
                       "tree": "greedy (alpha=1, tau=0)", "target_W_s": target}}


def wl_circuit(rows: int, cols: int, cycles: int, seed: int, simplified: bool = False):
    from paper_2002_01935_gb300 import inputs, planner, simplify
    circ = inputs.random_circuit(rows, cols, cycles, seed=seed)
    bits = inputs.random_bitstrings(rows * cols, 1, seed=1000 + seed)[0]
    net = inputs.circuit_network(circ, bits)
    if simplified:
        net, _ = simplify.simplify(net)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    info = planner.tree_info(net.labels, net.dims, pairs, net.open)
    return {"net": net, "pairs": pairs, "sliced": [], "info": info, "slice_begin": 0,
            "slice_count": 1, "oracle": "full",
            "config": {"qubits": rows * cols, "grid": f"{rows}x{cols}", "cycles": cycles,
                       "circuit_seed": seed, "bitstring_seed": 1000 + seed,
                       "simplified": net.meta.get("simplified"),
                       "tree": "greedy (alpha=1, tau=0)"}}


def wl_circuit7x7(rank: int, slices: int, trials: int = 16, target: float = 28.0):
    from paper_2002_01935_gb300 import inputs, planner
    circ = inputs.random_circuit(7, 7, 14, seed=0)
    bits = inputs.random_bitstrings(49, 1, seed=1000)[0]
    net = inputs.circuit_network(circ, bits)
    t0 = time.perf_counter()
    pairs, sliced, info = planner.hyper_greedy(net.labels, net.dims, net.open, trials=trials,
                                               seed=0, target_width=target)
    t_plan = time.perf_counter() - t0
    count = min(slices, int(info.d_sliced))
    return {"net": net, "pairs": pairs, "sliced": sliced, "info": info,
            "slice_begin": rank * count, "slice_count": count, "oracle": "subslice",
            "config": {"qubits": 49, "grid": "7x7", "cycles": 14, "circuit_seed": 0,
                       "bitstring_seed": 1000, "target_W_s": target,
                       "tree": f"Hyper-Greedy, {trials} seeded trials scored by C_s at W_s <= {target:g}",
                       "planning_s": round(t_plan, 2),
                       "slice_sample": f"slices [{rank * count}, {rank * count + count}) of "
                                       f"{int(info.d_sliced)}; time per amplitude extrapolated"}}


def node_figures(net, pairs, info, elem_bytes: int):
    """Algorithmic FLOPs and bytes of every node for one slice:
    FLOPs = (2 real | 8 complex) * 2^vc (Eq. vertexcon), bytes = (|A|+|B|+|C|) * elem."""
    n = net.n_tensors
    per = 8.0 if net.is_complex else 2.0
    out = []
    for k, (a, b) in enumerate(pairs):
        sz = lambda s: float(math.prod(net.dims[l] for l in s))
        sa, sb, sc = info.sets[a], info.sets[b], info.sets[n + k]
        out.append({"flops": per * 2.0 ** info.vc[k],
                    "bytes": (sz(sa) + sz(sb) + sz(sc)) * elem_bytes})
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            # the timed region starts once sampling runs (first row written)
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.06)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# --------------------------------------------------------------------------
# oracle legs (host cores, FP64, as it stands)
# --------------------------------------------------------------------------

def oracle_full(net, pairs, sliced, info, budget_s: float = 12.0, max_runs: int = 40):
    """Time full oracle contractions (all slices) of the network as the GPU
    reads it (leaves rounded to its storage type); also returns the value
    for the leaves before that rounding (context: the inputs' own rounding)."""
    from oracle import tree
    gnet = gpu_leaves(net)
    times = []
    val = None
    t_all = time.perf_counter()
    while len(times) < max_runs and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        m, e = tree.contract_net(gnet, pairs, sliced)
        times.append(time.perf_counter() - t0)
        val = (m, e)
    t = statistics.mean(times)
    flops = info.flops(net.is_complex)
    val_wide = tree.contract_net(net, pairs, sliced)
    return {"value": flops / t / 1e12, "unit": "TFLOP/s", "cores": tree.max_threads(),
            "kind": "oracle", "s_per_network": t,
            "sample": f"{len(times)} full contractions of the same network (all slices)"}, val, val_wide


def subslicing(net, pairs, target: float = 20.0):
    """The tree's slicing refined to W_s <= target (sub-slices the oracle
    finishes in about a second each)."""
    from paper_2002_01935_gb300 import planner
    sl2 = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target)
    return sl2, planner.tree_info(net.labels, net.dims, pairs, net.open, sl2)


def oracle_subslices(net, pairs, target: float = 20.0, budget_s: float = 10.0, max_slices: int = 64):
    """Time the oracle on consecutive sub-slices of the same tree sliced
    further, to W_s <= target: a bounded sample of the same contraction, on
    the leaf values the GPU reads.  Returns the timing, the sub-slicing, the
    per-sub-slice values and their sums, on those leaves and on the leaves
    before rounding to the GPU's storage type (same sub-slices)."""
    from oracle import tree
    sl2, i2 = subslicing(net, pairs, target)
    gnet = gpu_leaves(net)
    k, t_sum = 0, 0.0
    vals = []
    t_all = time.perf_counter()
    while k < max_slices and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        m, e = tree.contract_net(gnet, pairs, sl2, slice_begin=k, slice_count=1)
        t_sum += time.perf_counter() - t0
        vals.append((complex(m), int(e)))
        k += 1
    e_max = max(e for _, e in vals)
    ref = sum(m * 2.0 ** (e - e_max) for m, e in vals)
    mw, ew = tree.contract_net(net, pairs, sl2, slice_begin=0, slice_count=k)
    per = 8.0 if net.is_complex else 2.0
    return ({"value": per * i2.C * k / t_sum / 1e12, "unit": "TFLOP/s", "cores": tree.max_threads(),
             "kind": "oracle", "s_per_subslice": t_sum / k,
             "sample": f"{k} consecutive sub-slices of the same tree sliced to W_s <= {target:g} "
                       f"(C per sub-slice {i2.C:.3e})"},
            {"sliced": sl2, "count": k, "vals": vals, "ref": (ref, e_max),
             "ref_wide": (complex(mw), int(ew))})


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import __graft_entry__  # noqa: F401  (path setup)
    from oracle import build as obuild
    from oracle import tree
    obuild.build()
    if args.workload not in ("ising100", "ising100_hyper", "circuit4x4", "circuit5x5", "circuit7x7"):
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the FP64 oracle needs hours per step on the {args.workload} workload"}))
        return 0
    simp = bool(getattr(args, "simplify", False))
    w = (wl_ising(0, simplified=simp) if args.workload == "ising100" else
         wl_ising(0, hyper=True) if args.workload == "ising100_hyper" else
         wl_circuit(4, 4, 8, 0, simplified=simp) if args.workload == "circuit4x4" else
         wl_circuit(5, 5, 10, 0, simplified=simp) if args.workload == "circuit5x5" else
         wl_circuit7x7(0, args.slices))
    net, pairs, sliced, info = w["net"], w["pairs"], w["sliced"], w["info"]
    gnet = gpu_leaves(net)
    per = 8.0 if net.is_complex else 2.0
    if args.workload == "circuit7x7":
        # one step = one sub-slice of the W_s <= 28 slicing refined to
        # W_s <= 20 (a W_s <= 28 slice takes the oracle hours): a bounded
        # sample of the same contraction, consecutive sub-slices
        sl2, i2 = subslicing(net, pairs)
        run = lambda k: tree.contract_net(gnet, pairs, sl2, slice_begin=k, slice_count=1)
        flops_unit = per * i2.C
        sample = (f"one sub-slice per step: consecutive sub-slices of the same tree with its "
                  f"slicing refined to W_s <= 20 (C per sub-slice {i2.C:.3e})")
    else:
        run = lambda k: tree.contract_net(gnet, pairs, sliced)
        flops_unit = info.flops(net.is_complex)
        sample = f"{args.steps} full contractions"
    k = 0
    for _ in range(1 if args.warmup > 0 else 0):
        run(k)
        k += 1
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run(k)
        times.append(time.perf_counter() - t0)
        k += 1
    t = statistics.mean(times)
    val = flops_unit / t / 1e12
    cfg = dict(workload=WORKLOAD_NAMES[args.workload] + ("_simplified" if simp else ""),
               W_s=info.W, C=info.C, d_sliced=info.d_sliced, **w["config"])
    line = {"metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": cfg,
            "s_per_network": per * info.C * info.d_sliced / (val * 1e12),
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": tree.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if net.is_complex:
        line["s_per_amplitude"] = line["s_per_network"]
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# helpers on the GPU side
# --------------------------------------------------------------------------

def scalar_value(m, e, cplx):
    """(mantissa tensor, exponent tensor) -> (python scalar mantissa, int exponent)."""
    return (complex(m.cpu()) if cplx else float(m.cpu())), int(e.cpu())


def rel_error(got, got_e, ref, ref_e, cplx):
    if cplx:
        return abs(got * 2.0 ** (got_e - ref_e) - ref) / abs(ref)
    return abs(math.expm1(math.log(abs(got)) + (got_e - ref_e) * math.log(2) - math.log(abs(ref))))


def roofline(steps, dom, dom_ms, nodes, mode, ms_per_step, peaks):
    dnodes = steps[dom]["nodes"]
    dn = {"flops": sum(nodes[k]["flops"] for k in dnodes),
          "bytes": sum(nodes[k]["bytes"] for k in dnodes)}
    dmean = statistics.mean(dom_ms) / 1e3
    st = steps[dom]
    t_hbm = dn["bytes"] / (peaks["hbm_gbs"] * 1e9)
    if st["kind"] == 2:
        pk, pk_src = tc_peak(mode, peaks)
        passes = MODE_PASSES.get(mode, 1)
        t_alu = dn["flops"] * passes / (pk * 1e12)
        pipe = {"bound": "tensor", "peak": pk, "peak_source": pk_src,
                "executed_flops": dn["flops"] * passes}
    else:
        t_alu = dn["flops"] / (FP32_SIMT_TFLOPS * 1e12)
        pipe = {"bound": "alu", "peak": FP32_SIMT_TFLOPS,
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz"}
    if t_hbm >= t_alu:
        roof = {"bound": "hbm", "achieved": dn["bytes"] / dmean / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "peak_source": peaks["source"]}
    else:
        roof = {"bound": pipe["bound"], "achieved": dn["flops"] / dmean / 1e12, "peak": pipe["peak"],
                "unit": "TFLOP/s", "peak_source": pipe["peak_source"]}
        if "executed_flops" in pipe:
            roof["executed_frac"] = pipe["executed_flops"] / dmean / 1e12 / pipe["peak"]
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    cfg_names = {0: "generic", 1: "tile64x64", 2: "tile16x256", 3: "tile4x1024", 4: "tile256x16", 6: "tile128x64",
                 5: "dot"}
    kname = {0: "k_generic", 1: "k_tile", 2: "k_tc (tcgen05)"}[st["kind"]]
    roof["kernel"] = (f"step {dom} of {len(steps)}: " +
                      (f"k_wave over {len(dnodes)} nodes" if st["wave"] else
                       f"node {dnodes[0]}, {kname}" +
                       (f" {cfg_names.get(st['cfg'], '')}" if st["kind"] == 1 else "")))
    roof["algorithmic"] = {"flops": dn["flops"], "bytes": dn["bytes"]}
    roof["share_of_step"] = dmean * 1e3 / ms_per_step
    return roof


def tree_roofline(steps, nodes, mode, ms_per_step, slices_per_step, peaks, step_ms):
    """Per-tree roofline: the sum over nodes of max(executed FLOPs / pipe
    peak, algorithmic bytes / HBM bandwidth) -- the pipe being the tensor
    cores for tensor-core nodes, FP32 SIMT for the rest -- over the measured
    time; nodes whose bound is under 2 us are latency-bound, and the steps
    that hold only such nodes are reported with their share of the time."""
    t_roof = 0.0
    tiny, tiny_steps_ms = 0, 0.0
    for k, st in enumerate(steps):
        all_tiny = True
        for j in st["nodes"]:
            nd = nodes[j]
            t_hbm = nd["bytes"] / (peaks["hbm_gbs"] * 1e9)
            if st["kind"] == 2:
                t_alu = nd["flops"] * MODE_PASSES.get(mode, 1) / (tc_peak(mode, peaks)[0] * 1e12)
            else:
                t_alu = nd["flops"] / (FP32_SIMT_TFLOPS * 1e12)
            t = max(t_hbm, t_alu)
            t_roof += t
            if t < 2e-6:
                tiny += 1
            else:
                all_tiny = False
        if all_tiny and k < len(step_ms):
            tiny_steps_ms += step_ms[k]
    t_ms = t_roof * slices_per_step * 1e3
    return {"t_roof_ms": t_ms, "measured_ms": ms_per_step, "frac": t_ms / ms_per_step,
            "peaks": "measured HBM and bf16 (FP16 = bf16; TF32 = bf16 x 1.1/2.25), derived FP32 SIMT",
            "latency_bound_nodes": tiny, "nodes": sum(len(s["nodes"]) for s in steps),
            "latency_bound_step_ms": tiny_steps_ms * slices_per_step,
            "latency_bound_time_frac": tiny_steps_ms * slices_per_step / ms_per_step}


def device_events(torch, stream, n):
    # torch creates the CUDA event lazily: record once so .cuda_event is valid
    evl = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    for ev in evl:
        ev.record(stream)
    return evl


# --------------------------------------------------------------------------
# single-network workloads
# --------------------------------------------------------------------------

def run_network(args, torch, dist, rank, world, local):
    import numpy as np
    from paper_2002_01935_gb300 import binding

    if args.workload == "ising100":
        w = wl_ising(rank, target=args.target_ws, simplified=args.simplify)
    elif args.workload == "ising100_hyper":
        w = wl_ising(rank, hyper=True)
    elif args.workload == "circuit4x4":
        w = wl_circuit(4, 4, 8, rank, simplified=args.simplify)
    elif args.workload == "circuit5x5":
        w = wl_circuit(5, 5, 10, rank, simplified=args.simplify)
    else:
        w = wl_circuit7x7(rank, args.slices)
    net, pairs, sliced, info = w["net"], w["pairs"], w["sliced"], w["info"]
    sb, sc = w["slice_begin"], w["slice_count"]
    mode = args.mode
    cplx = net.is_complex
    dt = torch.complex64 if cplx else torch.float32
    elem = 8 if cplx else 4
    leaves = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, leaves, complex_=cplx)
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        ch = tnw.autotune(pairs, sliced, mode, reps=10)
        tuned = {"seconds": round(time.perf_counter() - t0, 3),
                 "tensor_core": ch.count(8) + ch.count(9) + ch.count(10), "tensor_core_128col": ch.count(9),
                 "tensor_core_planar": ch.count(10),
                 "tile_shapes": {n: ch.count(v) for v, n in
                                 ((1, "64x64"), (2, "16x256"), (3, "4x1024"), (4, "256x16"), (6, "128x64"))
                                 if ch.count(v)}}
    plan = tnw.plan_info(pairs, sliced, mode)
    per = 8.0 if cplx else 2.0
    flops_step = per * info.C * sc
    nodes = node_figures(net, pairs, info, elem)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def call(md=mode, **kw):
        return tnw.contract(pairs, sliced, md, slice_begin=sb, slice_count=sc, persistent=args.persistent, **kw)

    steps = tnw.plan_steps(pairs, sliced, mode)
    if args.persistent:
        # the persistent plan is one dataflow launch over every node
        steps = [{"wave": True, "kind": 1, "cfg": 0, "nodes": list(range(len(pairs))), "launches": 1}]
    n_steps = len(steps)
    for _ in range(args.warmup):
        m, e = call()

    # one per-step profile pass to find the dominant launch step
    evs = device_events(torch, stream, n_steps + 1)
    flush.zero_()
    call(prof_events=evs, prof_first=0)
    torch.cuda.synchronize()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(n_steps)]
    dom = int(np.argmax(step_ms))

    # timed region: K steps, each bracketed by events; L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # every 4th timed step also records events around the dominant launch step
    # (the roofline's live duration); the hooks cost a little device time
    hooked = [i for i in range(args.steps) if i % 4 == 3] or [args.steps - 1]
    dom_ev = {i: device_events(torch, stream, 2) for i in hooked}
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    torch.cuda.nvtx.range_push("timed")  # ncu --nvtx --nvtx-include timed/ profiles just this
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        if i in dom_ev:
            m, e = call(prof_events=dom_ev[i], prof_first=dom)
        else:
            m, e = call()
        ends[i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    call_ms = [s.elapsed_time(t) for s, t in zip(starts, ends)]
    dom_ms = [a.elapsed_time(b) for a, b in dom_ev.values()]
    total_ms = sum(call_ms)
    if dist:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = flops_step * world * args.steps / (total_ms / 1e3) / 1e12
    result, result_exp = scalar_value(m, e, cplx)
    peaks = load_peaks()
    roof = roofline(steps, dom, dom_ms, nodes, mode, ms_per_step, peaks)
    if not args.persistent:
        roof["traffic"], roof["traffic_source"] = measured_traffic(args.workload, mode)

    # end to end through the C-ABI with host buffers (copies inside the call)
    e2e = None
    if rank == 0:
        hl = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().pin_memory()
              for t in net.tensors]
        htn = binding.TensorNetwork(net.labels, net.dims, net.open, hl, complex_=cplx)
        if not args.no_autotune:
            htn.autotune(pairs, sliced, mode, reps=10)
        odt = torch.complex128 if cplx else torch.float64
        hout = torch.empty(tnw.out_shape, dtype=odt).pin_memory()
        hexp = torch.empty((), dtype=torch.int64).pin_memory()
        for _ in range(args.warmup):
            htn.contract(pairs, sliced, mode, out=hout, out_exp=hexp, slice_begin=sb, slice_count=sc,
                         persistent=args.persistent)
        t_e2e = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            htn.contract(pairs, sliced, mode, out=hout, out_exp=hexp, slice_begin=sb, slice_count=sc,
                         persistent=args.persistent)
            t_e2e += time.perf_counter() - t0
        h2d = sum(int(t.numel()) * elem for t in hl)
        d2h = hout.numel() * hout.element_size() + 8
        e2e = {"value": flops_step * args.steps / t_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": t_e2e / args.steps * 1e3}
        htn.close()

    # the oracle on the host cores: timing and the reference value, computed
    # on the leaf values the GPU reads (parity), and on the leaves before
    # their rounding to complex64 / float32 (context: the inputs' rounding)
    cpu, rel_err, rel_err_wide, ref = None, None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if w["oracle"] == "full":
            cpu, (om, oe), (wm, we) = oracle_full(net, pairs, sliced, info)
            ref = {"ref": (complex(om) if cplx else float(om), int(oe)),
                   "ref_wide": (complex(wm) if cplx else float(wm), int(we)),
                   "sliced": sliced, "begin": 0, "count": sc}
            got = (result, result_exp)
        else:
            cpu, sub = oracle_subslices(net, pairs)
            ref = {"ref": sub["ref"], "ref_wide": sub["ref_wide"], "sliced": sub["sliced"],
                   "begin": 0, "count": sub["count"], "vals": sub["vals"]}
            got = scalar_value(*tnw.contract(pairs, sub["sliced"], mode, slice_begin=0,
                                             slice_count=sub["count"]), cplx)
            cpu["rel_err_sample"] = ("GPU vs oracle on the same sub-slices (the slice sample "
                                     "itself is beyond the oracle's reach)")
        rel_err = rel_error(got[0], got[1], ref["ref"][0], ref["ref"][1], cplx)
        rel_err_wide = rel_error(got[0], got[1], ref["ref_wide"][0], ref["ref_wide"][1], cplx)

    # every precision mode on the same work (device buffers), with its error
    modes_cmp = None
    if rank == 0 and not args.no_modes:
        modes_cmp = {}
        reps = min(args.steps, 5) if args.workload == "circuit7x7" else args.steps
        for md in MODES:
            if not args.no_autotune:
                tnw.autotune(pairs, sliced, md, reps=10)
            for _ in range(2):
                call(md)
            es, ee2 = device_events(torch, stream, reps), device_events(torch, stream, reps)
            for i in range(reps):
                flush.zero_()
                es[i].record(stream)
                mm_, ee_ = call(md)
                ee2[i].record(stream)
            torch.cuda.synchronize()
            tms = sum(a.elapsed_time(b2) for a, b2 in zip(es, ee2)) / reps
            entry = {"ms_per_step": tms, "tflops": flops_step / (tms / 1e3) / 1e12,
                     "tol": MODE_TOL[md]}
            if ref is not None:
                gm, ge = scalar_value(*tnw.contract(pairs, ref["sliced"], md, slice_begin=ref["begin"],
                                                    slice_count=ref["count"]), cplx)
                entry["rel_err"] = rel_error(gm, ge, ref["ref"][0], ref["ref"][1], cplx)
                entry["within_tol"] = entry["rel_err"] <= MODE_TOL[md]
                entry["rel_err_c128_leaves"] = rel_error(gm, ge, ref["ref_wide"][0], ref["ref_wide"][1], cplx)
                if "vals" in ref:
                    # every sub-slice on its own, against the oracle's value of it
                    errs = []
                    for j, (vm, ve) in enumerate(ref["vals"]):
                        sm_, se_ = scalar_value(*tnw.contract(pairs, ref["sliced"], md, slice_begin=j,
                                                              slice_count=1), cplx)
                        errs.append(rel_error(sm_, se_, vm, ve, cplx))
                    entry["subslice_rel_err_max"] = max(errs)
                    entry["subslice_rel_err_median"] = statistics.median(errs)
            modes_cmp[md] = entry

    groups = 1 if args.persistent else sc
    # our kernels per call: call setup (leaf maxima + control block) and the
    # result copy; per slice group the steps' launches and the accumulation
    # (which also advances the slice counter when it is one block)
    n_out = math.prod(net.dims[l] for l in net.open)
    launches_per_call = 2 + groups * (1 + (n_out > 256) + sum(s.get("launches", 1) for s in steps))
    cfg = {"workload": WORKLOAD_NAMES[args.workload] + ("_simplified" if args.simplify else ""),
           "mode": mode, "W_s": info.W, "C": info.C,
           "d_sliced": info.d_sliced, "slices_per_step": sc,
           "flops_per_step": flops_step, "nodes": len(pairs),
           "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
           "plan_kernels": {"generic": plan["n_generic"], "tiled": plan["n_tiled"],
                            "tensor_core": plan["n_tensor_core"]},
           "launch_steps": n_steps, "wave_steps": sum(1 for s in steps if s["wave"]),
           "workspace_bytes": plan["ws_bytes"], "autotune": tuned,
           "persistent": bool(args.persistent)}
    cfg.update(w["config"])
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64" if cplx else "f32", "data": "synthetic", "config": cfg,
        "s_per_network": ms_per_step / 1e3 * (info.d_sliced / sc),
        "rel_err_vs_oracle": rel_err,
        "rel_err_vs_oracle_c128_leaves": rel_err_wide,
        "rel_err_definition": ("|got - oracle| / |oracle|, the oracle (FP64) run on the leaf values "
                               "the GPU reads; *_c128_leaves: against the leaves before their rounding "
                               "to the GPU's storage type"),
        "roofline": roof,
        "tree_roofline": tree_roofline(steps, nodes, mode, ms_per_step, sc, peaks, step_ms),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_call * args.steps,
        "modes": modes_cmp,
        "step_profile": [{"step": k, "kind": ["generic", "tile", "tcgen05"][s["kind"]],
                          "wave": s["wave"], "nodes": len(s["nodes"]), "ms": round(step_ms[k], 4)}
                         for k, s in enumerate(steps)],
        "clocks": clocks,
    }
    if cplx:
        line["s_per_amplitude"] = line["s_per_network"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    tnw.close()
    return 0


# --------------------------------------------------------------------------
# batch workload: amplitudes of one circuit + many Ising networks
# --------------------------------------------------------------------------

def run_batch(args, torch, dist, rank, world, local):
    """Config 4: 1024 distinct amplitudes of one 6x6-qubit, 12-cycle circuit
    (one shared Hyper-Greedy tree) plus 256 Ising networks with N even,
    uniform in [40, 160].  The Ising networks run as one batch: those whose
    greedy width is at most 24 in the merged forest (one captured launch
    sequence), wider ones sliced to W_s <= 24 (config 1's rule) as sliced
    members of the same batch.  The amplitudes run in blocks of copies, each
    block one launch sequence of tn_contract_instances (every node launch
    covers the block).  One step = all of it; per-network latency from the
    step's start (Ising: the batch's completion timestamps; amplitudes: the
    completion of their block)."""
    import numpy as np
    from paper_2002_01935_gb300 import binding, inputs, planner

    mode = args.mode
    t0 = time.perf_counter()
    circ = inputs.random_circuit(6, 6, 12, seed=0)
    n_amp = min(args.amplitudes, 1024)
    bits = inputs.random_bitstrings(36, 1024, seed=1000 + rank)[:n_amp]
    amp_nets = [inputs.circuit_network(circ, b) for b in bits[:1]]
    a_pairs, _, a_info = planner.hyper_greedy(amp_nets[0].labels, amp_nets[0].dims, amp_nets[0].open,
                                              trials=32, seed=0, target_width=None)
    rng = np.random.default_rng(4242 + rank)
    ising_n = [int(x) for x in rng.choice(np.arange(40, args.ising_max_n + 1, 2), size=args.ising)]
    ising_nets = [inputs.random_ising(n, seed=7000 + 1000 * rank + j) for j, n in enumerate(ising_n)]
    ising_trees, ising_sliced, ising_info = [], [], []
    for nt in ising_nets:
        pr = planner.greedy_tree(nt.labels, nt.dims, nt.open)
        inf = planner.tree_info(nt.labels, nt.dims, pr, nt.open)
        sl = planner.slice_greedy(nt.labels, nt.dims, pr, nt.open, 24.0) if inf.W > 24 else []
        ising_trees.append(pr)
        ising_sliced.append(sl)
        ising_info.append(planner.tree_info(nt.labels, nt.dims, pr, nt.open, sl))
    t_plan = time.perf_counter() - t0
    flops_ising = [2.0 * i.C * i.d_sliced for i in ising_info]
    flops_amp = 8.0 * a_info.C * n_amp
    flops_step = flops_amp + sum(flops_ising)

    # Ising leaves in one flat device buffer (one host->device copy for e2e)
    sizes = [int(np.prod(np.shape(t))) for nt in ising_nets for t in nt.tensors]
    i_dev = torch.zeros(sum(-(-x // 4) * 4 for x in sizes), dtype=torch.float32, device="cuda")
    i_host = torch.zeros(i_dev.numel(), dtype=torch.float32).pin_memory()
    handles, keep, pos = [], [], 0
    for nt in ising_nets:
        ts = []
        for t in nt.tensors:
            a = np.array(t, order="C")
            i_host[pos:pos + a.size] = torch.from_numpy(a.reshape(-1)).float()
            ts.append(i_dev[pos:pos + a.size].view(a.shape))
            pos += -(-a.size // 4) * 4
        keep.append(ts)
    i_dev.copy_(i_host)
    for nt, ts in zip(ising_nets, keep):
        handles.append(binding.TensorNetwork(nt.labels, nt.dims, nt.open, ts, complex_=False))
    if not args.no_autotune:
        for h, tr, sl in zip(handles, ising_trees, ising_sliced):
            if not sl:
                h.autotune(tr, [], mode, reps=2)
    batch = binding.Batch(handles, ising_trees, mode, sliced=ising_sliced)

    # amplitudes: shared leaves once, the output states of all bitstrings
    # stacked [n_amp, 2] per qubit; a block reads rows [b0, b0 + B)
    net0 = amp_nets[0]
    n = net0.n_tensors
    first_out = n - 36
    a_leaves = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda() for t in net0.tensors]
    outs_host = torch.zeros((36, n_amp, 2), dtype=torch.complex64).pin_memory()
    for q in range(36):
        outs_host[q, torch.arange(n_amp), torch.from_numpy(bits[:, q].astype(np.int64))] = 1.0
    outs_dev = outs_host.cuda()
    atn = binding.TensorNetwork(net0.labels, net0.dims, net0.open, a_leaves, complex_=True)
    ws1 = atn.plan_info(a_pairs, [], mode)["ws_bytes"]
    B = int(max(1, min(args.amp_block, n_amp, (48 << 30) // max(ws1, 1))))
    strides = [0] * first_out + [2] * 36
    blocks = [(b0, min(B, n_amp - b0)) for b0 in range(0, n_amp, B)]

    def run_amplitudes(evs=None):
        res = []
        for j, (b0, cnt) in enumerate(blocks):
            leaves = list(a_leaves)
            for q in range(36):
                leaves[first_out + q] = outs_dev[q, b0:b0 + cnt]
            atn.set_tensors(leaves)
            res.append(atn.contract_instances(a_pairs, mode, cnt, strides))
            if evs is not None:
                evs[j].record(stream)
        return res

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # warm-up: the Ising batch W times; the amplitude blocks once (a
    # minute of work: the first pass builds every plan and graph, later
    # passes repeat it unchanged)
    for _ in range(args.warmup):
        batch.contract()
    run_amplitudes()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    blk_ev = [device_events(torch, stream, len(blocks)) for _ in range(args.steps)]
    lats = []
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        out, ex, lat = batch.contract()
        amp_res = run_amplitudes(blk_ev[i])
        ends[i].record(stream)
        lats.append(lat)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    total_ms = sum(s.elapsed_time(t) for s, t in zip(starts, ends))
    if dist:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = flops_step * world * args.steps / (total_ms / 1e3) / 1e12
    li = np.stack([x.cpu().numpy() for x in lats]).astype(np.float64).ravel() / 1e6  # ms
    la = np.array([starts[i].elapsed_time(blk_ev[i][j]) for i in range(args.steps)
                   for j, (b0, cnt) in enumerate(blocks) for _ in range(cnt)])
    pct = lambda x, q: float(np.percentile(x, q)) if x.size else None
    out, ex = out.cpu().numpy(), ex.cpu().numpy()
    amp_m = torch.cat([r[0] for r in amp_res]).cpu().numpy()
    amp_e = torch.cat([r[1] for r in amp_res]).cpu().numpy()

    # e2e: every leaf copied from pinned host memory per step, results read back
    e2e = None
    if rank == 0:
        h2d = int(pos) * 4 + int(outs_host.numel()) * 8
        t_e2e = 0.0
        for i in range(2):  # one untimed pass, one timed
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            i_dev.copy_(i_host, non_blocking=True)
            outs_dev.copy_(outs_host, non_blocking=True)
            o2, x2, _ = batch.contract()
            r2 = run_amplitudes()
            o2h, x2h = o2.cpu(), x2.cpu()
            rh = [(a.cpu(), b_.cpu()) for a, b_ in r2]
            if i >= 1:
                t_e2e += time.perf_counter() - t1
        e2e = {"value": flops_step / t_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(o2h.numel() * 8 + x2h.numel() * 8 + n_amp * 24),
               "ms_per_step": t_e2e * 1e3,
               "path": "Ising leaves and the amplitudes' output states copied host->device, "
                       "the batch call and the amplitude blocks, results read back"}

    # the oracle: a sample of the Ising networks (same sliced trees, on the
    # leaf values the GPU reads) and sub-slices of one amplitude
    cpu, rel = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import tree
        errs, t_or, fl_or, k = [], 0.0, 0.0, 0
        t_all = time.perf_counter()
        order = sorted(range(len(ising_nets)), key=lambda j: flops_ising[j])
        for j in order:
            if time.perf_counter() - t_all > 10.0:
                break
            t1 = time.perf_counter()
            om, oe = tree.contract_net(gpu_leaves(ising_nets[j]), ising_trees[j], ising_sliced[j])
            t_or += time.perf_counter() - t1
            fl_or += flops_ising[j]
            errs.append(rel_error(float(out[j, 0]), int(ex[j]), float(om), int(oe), False))
            k += 1
        cpu = {"value": fl_or / t_or / 1e12, "unit": "TFLOP/s", "cores": tree.max_threads(),
               "kind": "oracle", "sample": f"the {k} smallest of the {len(ising_nets)} Ising networks, full"}
        rel = {"ising_max": max(errs) if errs else None, "ising_checked": k}
        a0 = binding.TensorNetwork(net0.labels, net0.dims, net0.open, a_leaves, complex_=True)
        sub, so = oracle_subslices(net0, a_pairs, budget_s=6.0)
        gm, ge = scalar_value(*a0.contract(a_pairs, so["sliced"], mode, slice_begin=0,
                                           slice_count=so["count"]), True)
        rel["amplitude_subslices"] = rel_error(gm, ge, so["ref"][0], so["ref"][1], True)
        rel["amplitude_sample"] = sub["sample"]
        # block copy 0 is bitstring 0: against the single-network call
        sm_, se_ = scalar_value(*a0.contract(a_pairs, [], mode), True)
        a0.close()
        rel["amplitude_block_vs_single_call"] = rel_error(
            complex(amp_m[0, 0], amp_m[0, 1]), int(amp_e[0]), sm_, se_, True)

    n_sl = sum(1 for sl in ising_sliced if sl)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES["batch"], "mode": mode,
                   "amplitudes": n_amp, "amplitude_block": B, "amplitude_blocks": len(blocks),
                   "circuit": "6x6, 12 cycles",
                   "amplitude_tree": f"Hyper-Greedy 32 trials, W {a_info.W:g}, C {a_info.C:.3e}",
                   "ising_networks": len(ising_nets),
                   "ising_N": f"even, uniform in [40, {args.ising_max_n}]",
                   "ising_sliced": f"{n_sl} networks with greedy width > 24 sliced to W_s <= 24",
                   "ising_flops": sum(flops_ising), "amplitude_flops": flops_amp,
                   "flops_per_step": flops_step, "planning_s": round(t_plan, 2),
                   "warmup": f"the Ising batch {args.warmup} times, the amplitude blocks once",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "s_per_amplitude": ms_per_step / 1e3 / max(n_amp, 1),
        "latency_ms": {"amplitude_p50": pct(la, 50), "amplitude_p99": pct(la, 99),
                       "ising_p50": pct(li, 50), "ising_p99": pct(li, 99),
                       "all_p50": pct(np.concatenate([la, li]), 50),
                       "all_p99": pct(np.concatenate([la, li]), 99)},
        "rel_err_vs_oracle": rel,
        "roofline": None,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": None,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    atn.close()
    for h in handles:
        h.close()
    return 0


def fsim_batch(torch, theta, phi):
    """fSim(theta, phi) for vectors of angles: [n, 2, 2, 2, 2] complex64 (the
    circuit model that produces the leaves, not part of the contraction)."""
    n = theta.shape[0]
    c, s = torch.cos(theta).to(torch.complex128), torch.sin(theta).to(torch.complex128)
    g = torch.zeros((n, 4, 4), dtype=torch.complex128, device=theta.device)
    g[:, 0, 0] = 1
    g[:, 1, 1] = c
    g[:, 2, 2] = c
    g[:, 1, 2] = -1j * s
    g[:, 2, 1] = -1j * s
    g[:, 3, 3] = torch.exp(-1j * phi.to(torch.complex128))
    return g.to(torch.complex64).reshape(n, 2, 2, 2, 2)


def run_grad(args, torch, dist, rank, world, local):
    import numpy as np
    from paper_2002_01935_gb300 import autograd, binding, inputs, planner, shard

    mode = args.mode
    R, C, T = 5, 4, 12
    circ = inputs.random_circuit(R, C, T, seed=0)
    bits = inputs.random_bitstrings(R * C, 64, seed=1000 + rank)
    fs = circ.fsim_gates()
    nets = [inputs.circuit_network(circ, b) for b in bits]
    net0 = nets[0]
    pairs = planner.greedy_tree(net0.labels, net0.dims, net0.open)
    info = planner.tree_info(net0.labels, net0.dims, pairs, net0.open)
    n = net0.n_tensors
    first_out = n - R * C  # output states are the last leaves
    base = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda() for t in net0.tensors]
    outs = [[torch.from_numpy(np.array(nt.tensors[v], order="C")).to(torch.complex64).cuda()
             for v in range(first_out, n)] for nt in nets]
    leaf_of = [net0.meta["gate_leaf"][g] for g in fs]
    theta = torch.tensor([circ.gates[g].params[0] for g in fs], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    phi = torch.tensor([circ.gates[g].params[1] for g in fs], dtype=torch.float64, device="cuda",
                       requires_grad=True)
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, base, complex_=True)
    if not args.no_autotune:
        tnw.autotune(pairs, [], mode, reps=3)

    # One gradient step through the batched autograd Function: the fSim
    # leaves from the parameters (torch), the 64 amplitudes in one launch
    # sequence (instances), L = mean log|A_x|^2 (torch), and its backward: one
    # reverse sweep per bitstring with the adjoint on the device, the fSim
    # leaves' gradients summed over the bitstrings in the library, then torch
    # from those leaves to (theta, phi).
    nb = len(bits)
    outs_all = torch.stack([torch.stack(o) for o in outs])          # [B, R*C, 2]
    batch = {first_out + q: outs_all[:, q].contiguous() for q in range(R * C)}

    def step():
        theta.grad = None
        phi.grad = None
        G = fsim_batch(torch, theta, phi)
        leaves = list(base)
        for i, v in enumerate(leaf_of):
            leaves[v] = G[i]
        vals = autograd.contract_batch(tnw, pairs, mode, leaves[:first_out] + [None] * (R * C), batch)
        loss = torch.mean(torch.log(torch.abs(vals) ** 2))
        loss.backward()
        if dist:  # data parallel over bitstrings: the parameter gradients summed over the ranks
            shard.combine_grads([theta.grad, phi.grad])
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    clk.start()
    times = []
    stream = torch.cuda.current_stream()
    # the backward runs on autograd's own thread, outside a thread-scoped
    # NVTX range: the profiler start/stop marks the timed region for
    # ncu --profile-from-start off
    torch.cuda.nvtx.range_push("timed")
    torch.cuda.profiler.start()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        loss = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
    torch.cuda.profiler.stop()
    torch.cuda.nvtx.range_pop()
    clocks = clk.stop()
    total = sum(times)
    if dist:
        tt = torch.tensor([total], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total = float(tt.item())
    ms_per_step = total / args.steps * 1e3
    # algorithmic work: forward 8 C, reverse sweep 2 x 8 C per bitstring
    flops_step = 24.0 * info.C * len(bits)
    value = flops_step * world / (ms_per_step / 1e3) / 1e12

    # parity sample: leaf derivatives of bitstring 0 against the oracle's
    # environments (the exact derivative), and the oracle's time for them
    cpu, rel = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import gradient, tree
        G = fsim_batch(torch, theta.detach(), phi.detach())
        lv = list(base)
        for i, v in enumerate(leaf_of):
            lv[v] = G[i]
        lv = lv[:first_out] + outs[0]
        tnw.set_tensors(lv)
        grads = tnw.grad(pairs, [], mode, np.array(1.0 + 0j))
        host = [t.detach().cpu().numpy().astype(np.complex128) for t in lv]
        sample = [leaf_of[0], leaf_of[len(leaf_of) // 2], leaf_of[-1]]
        errs, t_or = [], 0.0
        tf = lambda l, d, o: planner.greedy_tree(l, d, o)
        for v in sample:
            t1 = time.perf_counter()
            env = gradient.environment(host, net0.labels, net0.dims, v, tf)
            t_or += time.perf_counter() - t1
            got = np.conj(grads[v].detach().cpu().numpy().astype(np.complex128))
            errs.append(float(np.linalg.norm(got - env) / np.linalg.norm(env)))
        t1 = time.perf_counter()
        tree.contract(host, net0.labels, net0.dims, net0.open, pairs)
        t_fwd = time.perf_counter() - t1
        cpu = {"value": 8.0 * info.C / t_fwd / 1e12, "unit": "TFLOP/s", "cores": tree.max_threads(),
               "kind": "oracle", "s_per_gradient_step_extrapolated": 64 * (t_fwd + (n - 1) * t_or / len(sample)),
               "sample": "one forward contraction and the environments of 3 fSim leaves of bitstring 0"}
        rel = {"leaf_gradient_max": max(errs), "leaves_checked": len(sample)}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES["grad5x4"], "mode": mode, "qubits": R * C, "cycles": T,
                   "parameters": 2 * len(fs), "bitstrings": len(bits), "W": info.W, "C": info.C,
                   "flops_per_step": flops_step, "tree": "greedy (alpha=1, tau=0)",
                   "flops_convention": "24 C per bitstring: forward 8 C + reverse sweep 16 C"},
        "loss": float(loss.detach().cpu()),
        "s_per_gradient_step": ms_per_step / 1e3,
        "rel_err_vs_oracle": rel,
        "roofline": None,
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": None,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    tnw.close()
    return 0


def run_sample(args, torch, dist, rank, world, local):
    """Bitstring samples of a 5x4, 12-cycle circuit (Sec. 5's sampling
    procedure): 14 fixed qubits drawn uniformly, the 2^6 amplitudes over
    the other 6 qubits from one open-output contraction on the GPU, x_f drawn
    from them.  value = contraction FLOP/s; s_per_sample beside it."""
    import numpy as np
    from oracle import tree as otree
    from paper_2002_01935_gb300 import inputs, planner, sampling

    R, C, T = 5, 4, 12
    circ = inputs.random_circuit(R, C, T, seed=rank)
    open_q = list(range(R * C - 6, R * C))
    prov = sampling.OpenAmplitudes(circ, open_q, mode=args.mode)
    net0 = inputs.circuit_network(circ, [0] * (R * C), open_qubits=open_q)
    info = planner.tree_info(net0.labels, net0.dims, prov.pairs, net0.open)
    sampling.sample(R * C, open_q, prov, args.warmup, seed=99)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    clk.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s = sampling.sample(R * C, open_q, prov, args.steps, fidelity=1.0, seed=1000 + rank)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    total = ev0.elapsed_time(ev1) / 1e3
    if dist:
        tt = torch.tensor([total], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total = float(tt.item())
    flops = 8.0 * info.C * args.steps
    rel, cpu = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        x_u = [s[0][0][q] for q in prov.fixed]
        got = prov(x_u)
        bits = [0] * (R * C)
        for q, b in zip(prov.fixed, x_u):
            bits[q] = b
        t0 = time.perf_counter()
        m, e = otree.contract_net(inputs.circuit_network(circ, bits, open_qubits=open_q), prov.pairs)
        t_or = time.perf_counter() - t0
        ref = np.asarray(m) * 2.0 ** e
        rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        cpu = {"value": 8.0 * info.C / t_or / 1e12, "unit": "TFLOP/s", "cores": otree.max_threads(),
               "kind": "oracle", "s_per_contraction": t_or,
               "sample": "one open-output contraction (2^6 amplitudes) of the first sample's x_u"}
    prov.close()
    line = {
        "metric": METRIC, "value": flops * world / total / 1e12, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "mode": args.mode, "qubits": R * C,
                   "cycles": T, "open_qubits": open_q, "amplitudes_per_contraction": 64,
                   "fidelity": 1.0, "W": info.W, "C": info.C, "tree": "greedy (alpha=1, tau=0)",
                   "step": "one sample: uniform x_u, one contraction, x_f drawn on the host"},
        "s_per_sample": total / args.steps,
        "rel_err_vs_oracle": rel,
        "roofline": None, "cpu_baseline": cpu, "e2e": None, "gpu_launches": None, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_node(args, torch, dist, rank, world, local):
    import numpy as np
    from paper_2002_01935_gb300 import binding, inputs

    mb, nb, kb = (int(x) for x in args.node_bits.split(","))
    mode = args.mode
    rng = np.random.default_rng(11 + rank)
    ml = list(range(mb))
    nl = list(range(mb, mb + nb))
    kl = list(range(mb + nb, mb + nb + kb))
    dims = {l: 2 for l in ml + nl + kl}
    # K labels interleaved with M / N labels, as in a contraction tree
    la = kl[::2] + ml + kl[1::2]
    lb = nl[:3] + kl + nl[3:]
    f = lambda s: (rng.standard_normal(s) + 1j * rng.standard_normal(s)).astype(np.complex64)
    ta, tb = f([2] * len(la)), f([2] * len(lb))
    net = inputs.Network([ta, tb], [la, lb], dims, ml + nl)
    pairs = [(0, 1)]
    leaves = [torch.from_numpy(t).cuda() for t in (ta, tb)]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, leaves, complex_=True)
    plan = tnw.plan_info(pairs, [], mode)
    steps = tnw.plan_steps(pairs, [], mode)
    flops = 8.0 * 2.0 ** (mb + nb + kb)
    stream = torch.cuda.current_stream()
    out = torch.empty([2] * (mb + nb), dtype=torch.complex128, device="cuda")
    ex = torch.empty((), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        tnw.contract(pairs, [], mode, out=out, out_exp=ex)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    node_ev = [device_events(torch, stream, 2) for _ in range(args.steps)]
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        tnw.contract(pairs, [], mode, out=out, out_exp=ex, prof_events=node_ev[i], prof_first=0)
        ends[i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_step = sum(s.elapsed_time(t) for s, t in zip(starts, ends)) / args.steps
    ms_node = statistics.mean(a.elapsed_time(b) for a, b in node_ev)
    peaks = load_peaks()
    tc = steps[0]["kind"] == 2
    passes = MODE_PASSES.get(mode, 1) if tc else 1
    if mode == "tf32_3m" and tc:
        passes = 0.75  # three real products per complex one instead of four
    peak = tc_peak(mode, peaks)[0] if tc else FP32_SIMT_TFLOPS
    achieved = flops / (ms_node / 1e3) / 1e12
    roof = {"bound": "tensor" if tc else "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "executed_frac": achieved * passes / peak, "traffic": None,
            "peak_source": tc_peak(mode, peaks)[1] if tc
            else "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz",
            "kernel": f"node ({mb}, {nb}, {kb}) bits, {'pack + tcgen05 GEMM' if tc else 'k_tile'}",
            "share_of_step": ms_node / ms_step}
    # sampled outputs against the definition, in FP64
    res = out.cpu().numpy().reshape(2 ** mb, 2 ** nb) * 2.0 ** int(ex.cpu())
    A = ta.astype(np.complex128).transpose([la.index(l) for l in ml + kl]).reshape(2 ** mb, 2 ** kb)
    B = tb.astype(np.complex128).transpose([lb.index(l) for l in kl + nl]).reshape(2 ** kb, 2 ** nb)
    ii = rng.integers(0, 2 ** mb, 64)
    jj = rng.integers(0, 2 ** nb, 64)
    ref = np.einsum("sk,ks->s", A[ii], B[:, jj])
    scale = np.einsum("sk,ks->s", np.abs(A[ii]), np.abs(B[:, jj]))
    err = float(np.max(np.abs(res[ii, jj] - ref) / scale))
    line = {
        "metric": METRIC, "value": flops / (ms_step / 1e3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES["node"], "mode": mode, "bits_m_n_k": [mb, nb, kb],
                   "plan_kernels": {"tensor_core": plan["n_tensor_core"], "tiled": plan["n_tiled"]},
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "step": "the node, its FP64 output accumulation and the copy to the caller's tensor"},
        "node_ms": ms_node,
        "rel_err_vs_fp64_sample": err,
        "rel_err_definition": "64 sampled outputs, |got - exact| / (sum over k of |A||B|)",
        "roofline": roof, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    tnw.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 400 for the sub-millisecond workloads, so that the "
                         "timed region spans several clock samples; 20 for circuit7x7 and for "
                         "--impl reference; 5 otherwise)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="circuit7x7", choices=list(WORKLOAD_NAMES))
    ap.add_argument("--mode", default="fp16_split", choices=MODES)
    ap.add_argument("--slices", type=int, default=2, help="circuit7x7: slices per step")
    ap.add_argument("--amplitudes", type=int, default=1024, help="batch: amplitudes per step")
    ap.add_argument("--amp-block", type=int, default=32, help="batch: amplitudes per instances launch")
    ap.add_argument("--ising", type=int, default=256, help="batch: Ising networks per step")
    ap.add_argument("--node-bits", default="15,13,10", help="node: M,N,K label bits")
    ap.add_argument("--ising-max-n", type=int, default=160,
                    help="batch: largest Ising N (even N uniform in [40, this])")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--simplify", action="store_true",
                    help="structure simplifications (Sec. 3.7) of the network before planning "
                         "(ising100, circuit4x4, circuit5x5; not the configs' plain method)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the per-mode comparison")
    ap.add_argument("--no-autotune", action="store_true", help="keep the planner's kernel choices")
    ap.add_argument("--target-ws", type=float, default=24.0,
                    help="ising100: slice the greedy tree to this width (config 1: 24)")
    ap.add_argument("--persistent", action="store_true",
                    help="network workloads: every node of every slice in one persistent launch")
    args = ap.parse_args()
    if args.steps is None:
        short = args.workload in ("ising100", "ising100_hyper", "circuit4x4", "circuit5x5")
        args.steps = (20 if args.impl == "reference" or args.workload == "circuit7x7"
                      else (400 if short else (1 if args.workload == "batch" else 5)))
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "batch":
        rc = run_batch(args, torch, dist, rank, world, local)
    elif args.workload == "grad5x4":
        rc = run_grad(args, torch, dist, rank, world, local)
    elif args.workload == "node":
        rc = run_node(args, torch, dist, rank, world, local)
    elif args.workload == "sample":
        rc = run_sample(args, torch, dist, rank, world, local)
    else:
        rc = run_network(args, torch, dist, rank, world, local)
    if dist:
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
