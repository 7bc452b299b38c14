#!/usr/bin/env python3
"""Benchmark of the contraction-tree executor; prints one JSON line.

Workload (default): the Ising partition function of a random 3-regular
graph with N = 100 vertices, beta = 0.3, J = +-1 (one COPY tensor per
vertex, one Boltzmann matrix per edge), greedy tree sliced to W_s <= 24,
float32 on the GPU.  One step = one full contraction of the network (all
slices) through the C-ABI.  Throughput = algorithmic FLOPs 2 C_s per
network (real; 8 C_s complex) over device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fp32]
  python bench.py --impl reference ...   (the FP64 oracle on host cores)

Under torchrun each rank contracts its own network (seed = rank): weak
scaling, no collective on the data path; the timing is the max over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contraction FLOP/s & % roofline per tree; s/amplitude; rel. error vs FP64 oracle"
WORKLOAD = "ising_rr3_n100_beta0.3_greedy_ws24"
L2_FLUSH_BYTES = 512 << 20
# FP32 FMA peak of one GB300: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz.
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# nominal dense tensor rates per GPU (TF32 : BF16 = 1.1 : 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
# real products executed per algorithmic product on the tensor cores
MODE_PASSES = {"tf32_split": 3, "bf16_split": 3, "tf32_3m": 1}


def build_workload(seed: int, n: int = 100, target: float = 24.0):
    from paper_2002_01935_gb300 import inputs, planner
    net = inputs.random_ising(n, seed)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    info = planner.tree_info(net.labels, net.dims, pairs, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target) if info.W > target else []
    info = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
    return net, pairs, sliced, info


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
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
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


def oracle_baseline(net, pairs, sliced, info, budget_s: float = 12.0, max_runs: int = 40):
    """Time the FP64 oracle, as it stands, on the host cores."""
    from oracle import tree
    times = []
    val = None
    t_all = time.perf_counter()
    while len(times) < max_runs and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        m, e = tree.contract_net(net, pairs, sliced)
        times.append(time.perf_counter() - t0)
        val = (m, e)
    t = statistics.mean(times)
    flops = info.flops(net.is_complex)
    return {"value": flops / t / 1e12, "unit": "TFLOP/s", "cores": tree.max_threads(),
            "kind": "oracle", "s_per_network": t,
            "sample": f"{len(times)} full contractions of the same network (all slices)"}, val


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import __graft_entry__  # noqa: F401  (path setup)
    from oracle import build as obuild
    obuild.build()
    net, pairs, sliced, info = build_workload(0)
    # each step: one full oracle contraction, bounded to a few minutes in all
    from oracle import tree
    for _ in range(max(args.warmup, 0) and 1):
        tree.contract_net(net, pairs, sliced)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        tree.contract_net(net, pairs, sliced)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    val = info.flops(net.is_complex) / t / 1e12
    line = {"metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n_vertices": 100, "beta": 0.3, "W_s": info.W,
                       "C": info.C, "d_sliced": info.d_sliced},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": tree.max_threads(),
                             "kind": "oracle", "sample": f"{args.steps} full contractions"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--mode", default="fp32")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-modes", action="store_true",
                    help="also time every precision mode (device buffers) and report the error")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import numpy as np
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
    from paper_2002_01935_gb300 import binding

    net, pairs, sliced, info = build_workload(rank)
    cplx = net.is_complex
    dt = torch.complex64 if cplx else torch.float32
    elem = 8 if cplx else 4
    leaves = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, leaves, complex_=cplx)
    plan = tnw.plan_info(pairs, sliced, args.mode)
    flops_step = info.flops(cplx)
    nodes = node_figures(net, pairs, info, elem)
    n_nodes = len(pairs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # warm-up, then one per-step profile pass to find the dominant launch
    steps = tnw.plan_steps(pairs, sliced, args.mode)
    n_steps = len(steps)
    for _ in range(args.warmup):
        m, e = tnw.contract(pairs, sliced, args.mode)

    def events(n):
        # torch creates the CUDA event lazily: record once so .cuda_event is valid
        evl = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for ev in evl:
            ev.record(stream)
        return evl

    evs = events(n_steps + 1)
    flush.zero_()
    tnw.contract(pairs, sliced, args.mode, prof_events=evs, prof_first=0)
    torch.cuda.synchronize()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(n_steps)]
    dom = int(np.argmax(step_ms))

    # timed region: K steps, each bracketed by events; L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    dom_ev = [events(2) for _ in range(args.steps)]
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        m, e = tnw.contract(pairs, sliced, args.mode, prof_events=dom_ev[i], prof_first=dom)
        ends[i].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    call_ms = [s.elapsed_time(t) for s, t in zip(starts, ends)]
    dom_ms = [a.elapsed_time(b) for a, b in dom_ev]
    total_ms = sum(call_ms)
    if dist:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = flops_step * world * args.steps / (total_ms / 1e3) / 1e12
    result = complex(m.cpu()) if cplx else float(m.cpu())
    result_exp = int(e.cpu())

    # roofline of the dominant launch step
    peaks = load_peaks()
    dnodes = steps[dom]["nodes"]
    dn = {"flops": sum(nodes[k]["flops"] for k in dnodes),
          "bytes": sum(nodes[k]["bytes"] for k in dnodes)}
    dmean = statistics.mean(dom_ms) / 1e3
    st = steps[dom]
    t_hbm = dn["bytes"] / (peaks["hbm_gbs"] * 1e9)
    if st["kind"] == 2:
        tc_peak = peaks["bf16_tflops"] * (1.0 if args.mode == "bf16_split" else TF32_OVER_BF16)
        passes = MODE_PASSES.get(args.mode, 1)
        t_alu = dn["flops"] * passes / (tc_peak * 1e12)
        pipe = {"bound": "tensor", "peak": tc_peak,
                "peak_source": f"{peaks['source']} bf16 x " +
                               ("1" if args.mode == "bf16_split" else "1.1/2.25 (nominal TF32:BF16)"),
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
    cfg_names = {0: "generic", 1: "tile64x64", 2: "tile16x256", 3: "tile4x1024", 4: "tile256x16",
                 5: "dot"}
    kname = {0: "k_generic", 1: "k_tile", 2: "k_tc (tcgen05)"}[st["kind"]]
    roof["kernel"] = (f"step {dom} of {n_steps}: " +
                      (f"k_wave over {len(dnodes)} nodes" if st["wave"] else
                       f"node {dnodes[0]}, {kname}" +
                       (f" {cfg_names.get(st['cfg'], '')}" if st["kind"] == 1 else "")))
    roof["algorithmic"] = {"flops": dn["flops"], "bytes": dn["bytes"]}
    roof["share_of_step"] = dmean * 1e3 / ms_per_step

    # end to end through the C-ABI with host buffers (copies inside the call)
    e2e = None
    if rank == 0:
        hl = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().pin_memory()
              for t in net.tensors]
        htn = binding.TensorNetwork(net.labels, net.dims, net.open, hl, complex_=cplx)
        odt = torch.complex128 if cplx else torch.float64
        hout = torch.empty(tnw.out_shape, dtype=odt).pin_memory()
        hexp = torch.empty((), dtype=torch.int64).pin_memory()
        for _ in range(args.warmup):
            htn.contract(pairs, sliced, args.mode, out=hout, out_exp=hexp)
        t_e2e = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            htn.contract(pairs, sliced, args.mode, out=hout, out_exp=hexp)
            t_e2e += time.perf_counter() - t0
        h2d = sum(int(t.numel()) * elem for t in hl)
        d2h = hout.numel() * hout.element_size() + 8
        e2e = {"value": flops_step * args.steps / t_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": t_e2e / args.steps * 1e3}
        htn.close()

    cpu = None
    rel_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, (om, oe) = oracle_baseline(net, pairs, sliced, info)
        if cplx:
            ref = complex(om)
            rel_err = abs(result * 2.0 ** (result_exp - oe) - ref) / abs(ref)
        else:
            rel_err = abs(math.expm1(math.log(abs(result)) + (result_exp - oe) * math.log(2)
                                     - math.log(abs(float(om)))))

    modes_cmp = None
    if args.compare_modes and rank == 0:
        modes_cmp = {}
        ref_ln = None
        if cpu is not None:
            ref_ln = math.log(abs(float(om))) + oe * math.log(2) if not cplx else None
        for md in ["fp32", "tf32_split", "bf16_split", "tf32_3m"]:
            for _ in range(3):
                mm_, ee_ = tnw.contract(pairs, sliced, md)
            es, ee2 = events(args.steps), events(args.steps)
            for i in range(args.steps):
                flush.zero_()
                es[i].record(stream)
                mm_, ee_ = tnw.contract(pairs, sliced, md)
                ee2[i].record(stream)
            torch.cuda.synchronize()
            tms = sum(a.elapsed_time(b2) for a, b2 in zip(es, ee2)) / args.steps
            entry = {"ms_per_network": tms, "tflops": flops_step / (tms / 1e3) / 1e12}
            if cpu is not None:
                if cplx:
                    ref = complex(om)
                    entry["rel_err"] = abs(complex(mm_.cpu()) * 2.0 ** (int(ee_.cpu()) - oe) - ref) / abs(ref)
                else:
                    entry["rel_err"] = abs(math.expm1(math.log(abs(float(mm_.cpu()))) +
                                                      int(ee_.cpu()) * math.log(2) - ref_ln))
            modes_cmp[md] = entry

    launches_per_step = sum(1 + (1 if (s["cfg"] in (1, 2, 3, 4, 5) and not s["wave"]) else 0)
                            for s in steps) * info.d_sliced + 2 * info.d_sliced + 3
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_vertices": 100, "beta": 0.3, "J": "+-1",
                   "mode": args.mode, "W_s": info.W, "C": info.C, "d_sliced": info.d_sliced,
                   "flops_per_network": flops_step, "nodes": n_nodes,
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "tree": "greedy (alpha=1, tau=0)",
                   "plan_kernels": {"generic": plan["n_generic"], "tiled": plan["n_tiled"],
                                    "tensor_core": plan["n_tensor_core"]},
                   "launch_steps": n_steps,
                   "wave_steps": sum(1 for s in steps if s["wave"])},
        "s_per_network": ms_per_step / 1e3,
        "rel_err_vs_oracle": rel_err,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "modes": modes_cmp,
        "step_profile": [{"step": k, "kind": ["generic", "tile", "tcgen05"][s["kind"]],
                          "wave": s["wave"], "nodes": len(s["nodes"]), "ms": round(step_ms[k], 4)}
                         for k, s in enumerate(steps)],
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    tnw.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
