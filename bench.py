"""Throughput benchmark: amplitudes/s of the sliced QAOA tensor-network
contraction on the 80-qubit, p = 1, 16-cut workload (65536 slices per
amplitude, 8 bit strings per step, one graph and plan).

One step = one pass of the whole hot path over one batch: the gate tensors
of 8 bit strings built in FP64, all 8 x 65536 slices contracted, the slice
sums (FP64, compensated) and the normalisation -- one replay of the plan's
CUDA graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                  [--impl ours|reference]

Prints ONE JSON line on rank 0.  --impl reference times the CPU oracle (the
paper's scheme on the host cores: worker threads over slice ranges, master
sum) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="qaoa80_p1_k16", n=80, p=1, k=16, seed=3, bitstrings=8)
METRIC = "amplitudes/sec, n=80 QAOA p=1, 16 cut edges (65536 slices)"

# FP32 pipe instructions per real multiply-add of each arithmetic (the
# double-float MAC with lazy normalisation: 1 FMUL + 3 FFMA for the product,
# one TwoSum (6) into the high word, 2 FADD into the low word = 12, plus one
# TwoSum per part and output; emulated TF32 / split forms: conversions +
# products on the FP32 pipe).  Only used for the issue share reported beside
# the roofline fraction, never to scale the peak.
INSTR_PER_MAC = {"fp32": 1, "fp32x2": 12, "tf32": 3, "tf32x3": 9, "bf16x3": 13, "bf16x6": 22}


def pipe_peak(prec: str, peaks: dict) -> float:
    """Measured peak (TFLOP/s, 2 flops per multiply-add) of the pipe that runs
    the arithmetic: the FP64 pipe for complex128, the FP32 pipe otherwise (the
    higher of its scalar and packed-pair multiply-add rates: the generated
    double-float executor issues packed pairs)."""
    if prec == "fp64":
        return peaks["fp64_tflops"]
    return max(peaks["fp32_tflops"], peaks.get("fp32x2_tflops") or 0.0)


def measure_pipe_peaks(local_rank: int) -> dict:
    """qtn_pipe_peaks (FP32 and FP64 multiply-add chains over the whole GPU,
    best of 5, CUDA events) with the SM clock sampled while it runs."""
    from paper_2010_14962_gb300 import qtn

    with ClockSampler(local_rank) as clk:
        time.sleep(0.2)
        pk = qtn.pipe_peaks(5)
        try:
            pk["fp32x2_tflops"] = qtn.pipe_peak_fp32x2(5)
        except qtn.QTNError:
            pk["fp32x2_tflops"] = None
        time.sleep(0.2)
    pk["clocks"] = clk.summary()
    pk["how"] = ("qtn_pipe_peaks / qtn_pipe_peak_fp32x2: 8 independent FMA chains per thread (scalar FP32, FP64, "
                 "packed fma.rn.f32x2 pairs), 4 x SMs x resident blocks of 256 threads, best of 5 launches timed "
                 "with CUDA events; 2 flops per multiply-add")
    return pk


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# What the benchmark's executor (the kernel generated per plan) is generated from: the program compiler, the
# generator and the arithmetic it embeds.
KERNEL_SOURCES = ("program.hpp", "program.cpp", "jit.cpp", "arith.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_14962_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(prec: str):
    """DRAM bytes per executor launch from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    e = t.get(prec)
    if not e or e.get("kernel_sources_sha256_16") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def step_classes(prog: dict, elem_bytes: int) -> list:
    """Per merge class (K = 2^kb summed entries) of a program: steps, share of
    the executed multiply-adds, and flop per byte of shared-memory traffic
    with every operand and result moved once (the root's outputs are summed,
    not stored); every class is on chip, so the ALU roof bounds it."""
    cls = {}
    for st in prog["steps"]:
        ma, nb, kb, bb = st["ma"], st["nb"], st["kb"], st["bb"]
        macs = 2 ** (ma + nb + kb + bb)
        moved = 2 ** (ma + kb + bb) + 2 ** (kb + nb + bb) + (0 if st["flags"] & 4 else 2 ** (ma + nb + bb))
        c = cls.setdefault(2 ** kb, [0, 0, 0])
        c[0] += 1
        c[1] += macs
        c[2] += moved * elem_bytes
    total = sum(c[1] for c in cls.values())
    return [{"K": k, "steps": c[0], "mac_share": c[1] / total, "flop_per_byte": 8 * c[1] / c[2]}
            for k, c in sorted(cls.items())]


def setup_workload(rank: int, form: str = "gates"):
    from paper_2010_14962_gb300 import instances as I
    from paper_2010_14962_gb300 import qtn

    w = WORKLOAD
    inst = I.qaoa_instance(w["n"], w["p"], w["seed"])
    net = qtn.Network(w["n"], inst.edges, inst.gamma, inst.beta, form=form)
    plan = qtn.Plan(net, k=w["k"])
    xs = I.bitstrings(w["n"], w["bitstrings"], w["seed"] + 1000 * rank)
    return inst, net, plan, xs


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2010_14962_gb300 import qtn

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    inst, net, plan, xs = setup_workload(rank, args.form)
    nx = xs.shape[0]
    cost = plan.cost()
    pipe_peaks = measure_pipe_peaks(local_rank)
    sweep = None
    if args.precision == "auto":
        sweep, args.precision = precision_sweep(plan, inst, xs, torch, rank == 0 and not args.no_oracle_refs)
    flops_per_amp = (2 ** cost["k"]) * 8 * cost["macs_per_slice"]
    stream = torch.cuda.current_stream()
    d_x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    d_out = torch.zeros((nx, 2), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    if args.executor:
        plan.select_executor(args.executor, args.precision, nx)

    def step():
        plan.contract_amplitudes_device(d_x, d_out, args.precision, stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    # The executor the autotuner picked (first call above) and the work it
    # executes per amplitude: 2^(outer classes) items x MACs per item.
    desc = plan.describe()
    prec_id = qtn.PRECISIONS[args.precision]
    tuned = [t for t in desc["tuned"] if t["prec"] == prec_id and t["nx"] == nx][0]
    prog = desc["programs"][tuned["executor"]]
    exec_macs_per_amp = (2 ** len(prog["outer_class"])) * prog["macs_per_item"]
    exec_flops_per_amp = 8 * exec_macs_per_amp

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        # Timed region: K steps, each a replay of the plan's CUDA graph, L2
        # flushed between steps (outside the step's events).
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            starts[i].record(stream)
            step()
            ends[i].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
        # Executor kernel time: the same K steps launched directly with CUDA
        # events around the executor on the launching stream.
        plan.set_kernel_timing(True)
        for i in range(args.steps):
            step()
            stream.synchronize()
            kernel_ms.append(plan.kernel_ms())
            flush.zero_()
        plan.set_kernel_timing(False)
        torch.cuda.synchronize()
        time.sleep(0.3)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    amps = nx * args.steps * world
    value = amps / (total_ms / 1e3)

    # End to end through the public host API: pinned host x in, host results out.
    plans = [plan] * nx
    xl = np.ascontiguousarray(xs, dtype=np.uint8)  # one row per bit string
    for _ in range(2):
        qtn.contract_batch(plans, xl, args.precision)
    e2e_steps = max(3, min(args.steps, 50))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        qtn.contract_batch(plans, xl, args.precision)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = nx * e2e_steps * world / e2e_s

    clocks = clk.summary()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak = pipe_peak(args.precision, pipe_peaks)
    avg_kernel_s = statistics.mean(kernel_ms) / 1e3
    achieved = exec_flops_per_amp * nx / avg_kernel_s / 1e12
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "amplitudes/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "c64", "fp64": "c128", "fp32x2": "c64x2 (double-float)"}.get(args.precision, "c64"),
        "data": "synthetic: seeded random 3-regular graph, gamma/beta ~ U[0,pi), seeded bit strings",
        "config": {"workload": WORKLOAD["name"], "n": WORKLOAD["n"], "p": WORKLOAD["p"], "cuts": WORKLOAD["k"],
                   "slices_per_amplitude": 2 ** cost["k"], "bitstrings_per_step": nx, "precision": args.precision,
                   "executor": tuned["executor"], "autotune_ms": tuned["ms"], "plan_width": cost["width"],
                   "cut_classes": max(desc["cut_class"]) + 1 if desc["cut_class"] else 0,
                   "inner_classes": len(prog["inner_class"]),
                   "macs_per_slice_unshared": cost["macs_per_slice"],
                   "executed_macs_per_amplitude": exec_macs_per_amp,
                   "executed_tflops": exec_flops_per_amp * value / 1e12,
                   "effective_tflops_per_slice_method": flops_per_amp * value / 1e12,
                   "slices_per_s": value * 2 ** cost["k"], "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"weak: {nx} bit strings per GPU, slices across CTAs/threads"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(args.precision),
                     "kernel": {"lane": "lane_exec_kernel", "level": "level_exec_kernel",
                                "level-jit": "qtn_level_jit (generated for this plan)"}.get(prog["executor"],
                                                                                             "block_exec_kernel"),
                     "peak_source": ("measured %s multiply-add peak of this GPU (qtn_pipe_peaks%s, median SM clock "
                                     "%s MHz)" % ("FP64" if args.precision == "fp64" else
                                                  "FP32 (higher of scalar and packed-pair)",
                                                  "" if args.precision == "fp64" else " / qtn_pipe_peak_fp32x2",
                                                  pipe_peaks["clocks"].get("sm_mhz"))),
                     "achieved_def": ("executed algorithmic flops per launch (8 x complex multiply-adds of the "
                                      "executor's program) / executor kernel time (CUDA events on its stream)"),
                     "pipe_issue_frac": (achieved * INSTR_PER_MAC[args.precision] / peak
                                         if args.precision in INSTR_PER_MAC else None),
                     "pipe_issue_def": ("share of the FP32 pipe's lane operations the arithmetic's own "
                                        "operations fill (model: %s per real multiply-add)"
                                        % INSTR_PER_MAC.get(args.precision)),
                     "measured_peaks_tflops": {"fp32": pipe_peaks["fp32_tflops"], "fp64": pipe_peaks["fp64_tflops"],
                                               "fp32x2": pipe_peaks.get("fp32x2_tflops")},
                     "attainable": ({"tflops": peak / INSTR_PER_MAC[args.precision],
                                     "frac": achieved * INSTR_PER_MAC[args.precision] / peak,
                                     "def": ("every step class of this program is on chip (shared memory), so the "
                                             "attainable rate is the FP32 pipe's at %s FP32 operations per real "
                                             "multiply-add of the arithmetic" % INSTR_PER_MAC[args.precision])}
                                    if args.precision in INSTR_PER_MAC else
                                    {"tflops": peak, "frac": achieved / peak,
                                     "def": "FP64 pipe, one FMA per real multiply-add"}),
                     "kernel_ms_avg": avg_kernel_s * 1e3,
                     "step_classes": step_classes(prog, 8 if args.precision in ("fp32", "tf32", "bf16x3", "tf32x3",
                                                                                "bf16x6") else 16)},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "amplitudes/s", "h2d_bytes_per_step": int(nx * WORKLOAD["n"]),
                "d2h_bytes_per_step": int(nx * 16), "api": "qtn_contract_batch (host x in, host amplitudes out)"},
        "gpu_launches": (3 + (1 if prog.get("prologue") else 0)) * args.steps,
        "wall_s_timed_region": wall,
    }
    if sweep is not None:
        out["precision_sweep"] = sweep
        out["config"]["precision_rule"] = sweep["rule"]
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


SWEEP = ["fp64", "fp32", "fp32x2", "tf32", "bf16x3", "tf32x3", "bf16x6"]
ANGLE_DRAWS = 4      # the workload's own (gamma, beta) and three more seeded draws
ORACLE_REF_CUTS = 8  # the oracle's own cut set for the reference values (fast, exact)


def angle_draws(inst):
    """(gamma, beta) of each draw: the workload's own angles first."""
    from paper_2010_14962_gb300 import instances as I

    draws = [(np.asarray(inst.gamma, float), np.asarray(inst.beta, float))]
    for d in range(1, ANGLE_DRAWS):
        draws.append(I.angles(inst.p, 7000 + d))
    return draws


def oracle_refs(inst, xs, draws):
    """The oracle's amplitudes (its own 8-cut plan, all host cores) for every
    (draw, bit string) pair, draw-major."""
    from oracle import oracle as O

    cuts, _ = O.choose_cuts(inst.n, inst.edges, inst.p, ORACLE_REF_CUTS)
    return np.array([O.tn_amplitude(inst.n, inst.edges, g, b, x, cuts=cuts, threads=os.cpu_count() or 1).value
                     for g, b in draws for x in xs])


def precision_sweep(plan, inst, xs, torch, with_oracle: bool):
    """Throughput of every arithmetic on the workload (its own angles, 8 bit
    strings) and its accuracy over ANGLE_DRAWS seeded (gamma, beta) draws on
    the same graph and plan (8 bit strings each, one sweep launch); returns
    (table, chosen precision).  The chosen form is the fastest whose worst
    relative error over all draws is within 1e-6 (against the oracle when its
    values are computed, else against the FP64 GPU form)."""
    nx = xs.shape[0]
    d_x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    draws = angle_draws(inst)
    nd = len(draws)
    d_xs = torch.from_numpy(np.ascontiguousarray(np.tile(xs, (nd, 1)))).cuda()
    d_g = torch.from_numpy(np.ascontiguousarray(np.repeat(np.stack([g for g, _ in draws]), nx, axis=0))).cuda()
    d_b = torch.from_numpy(np.ascontiguousarray(np.repeat(np.stack([b for _, b in draws]), nx, axis=0))).cuda()
    stream = torch.cuda.current_stream()
    refs = oracle_refs(inst, xs, draws) if with_oracle else None
    table, vals = {}, {}
    for prec in SWEEP:
        d_out = torch.zeros((nx, 2), dtype=torch.float64, device="cuda")
        plan.contract_amplitudes_device(d_x, d_out, prec, stream)  # autotunes
        for _ in range(3):
            plan.contract_amplitudes_device(d_x, d_out, prec, stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        a.record(stream)
        for _ in range(reps):
            plan.contract_amplitudes_device(d_x, d_out, prec, stream)
        b.record(stream)
        torch.cuda.synchronize()
        d_all = torch.zeros((nd * nx, 2), dtype=torch.float64, device="cuda")
        plan.contract_sweep_device(d_xs, d_g, d_b, d_all, prec, stream)
        torch.cuda.synchronize()
        o = d_all.cpu().numpy()
        vals[prec] = o[:, 0] + 1j * o[:, 1]
        tuned = [t for t in plan.describe()["tuned"] if t["prec"] == plan_prec_id(prec) and t["nx"] == nx]
        table[prec] = {"amplitudes_per_s": nx * reps / (a.elapsed_time(b) / 1e3),
                       "executor": tuned[0]["executor"] if tuned else None,
                       "emulated_tensor_core_numerics": prec in ("tf32", "bf16x3", "tf32x3", "bf16x6")}
    f64 = vals["fp64"]
    for prec in SWEEP:
        e = np.abs(vals[prec] - f64) / np.abs(f64)
        table[prec]["max_rel_err_vs_fp64_gpu"] = float(np.max(e))
        table[prec]["max_rel_err_vs_fp64_gpu_per_draw"] = [float(np.max(e[d * nx:(d + 1) * nx])) for d in range(nd)]
        if refs is not None:
            e = np.abs(vals[prec] - refs) / np.abs(refs)
            table[prec]["max_rel_err_vs_oracle"] = float(np.max(e))
            table[prec]["max_rel_err_vs_oracle_per_draw"] = [float(np.max(e[d * nx:(d + 1) * nx]))
                                                             for d in range(nd)]
    key = "max_rel_err_vs_oracle" if refs is not None else "max_rel_err_vs_fp64_gpu"
    ok = [p for p in SWEEP if table[p][key] <= 1e-6]
    chosen = max(ok, key=lambda p: table[p]["amplitudes_per_s"])
    table["chosen"] = chosen
    table["rule"] = (f"fastest arithmetic whose worst relative error over {nd} (gamma, beta) draws x {nx} bit "
                     f"strings is <= 1e-6 ({key})")
    table["draws"] = [{"gamma": [float(v) for v in g], "beta": [float(v) for v in b]} for g, b in draws]
    table["speedup_vs_fp64_gpu"] = table[chosen]["amplitudes_per_s"] / table["fp64"]["amplitudes_per_s"]
    return table, chosen


def plan_prec_id(prec):
    from paper_2010_14962_gb300 import qtn

    return qtn.PRECISIONS[prec]


def cpu_baseline(seconds: float, bundle=None):
    """The oracle (as it stands) on a bounded sample of the workload's slices,
    all host cores, scaled to amplitudes/s.  The oracle cuts 16 wire segments
    of its own choosing (oracle.choose_cuts), so nothing here depends on the
    product library."""
    from oracle import oracle as O

    inst, xs, cuts = bundle or setup_workload_cpu()
    cores = os.cpu_count() or 1
    S = 2 ** len(cuts)
    chunk = 64 * cores
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < S:
        hi = min(S, done + chunk)
        O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, xs[0], cuts=cuts, slices=(done, hi),
                       threads=cores)
        done = hi
    dt = time.perf_counter() - t0
    # One core as well (the paper's single-core comparison), on a shorter sample.
    one, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < max(1.0, seconds / 4) and one < S:
        hi = min(S, one + 64)
        O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, xs[0], cuts=cuts, slices=(one, hi), threads=1)
        one = hi
    dt1 = time.perf_counter() - t1
    return {"value": (done / S) / dt, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} of {S} slices of one amplitude ({WORKLOAD['name']}, the oracle's own "
                      f"{len(cuts)}-cut plan), {dt:.1f} s",
            "one_core": {"value": (one / S) / dt1, "sample": f"{one} of {S} slices, {dt1:.1f} s"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    bundle = setup_workload_cpu()
    for _ in range(args.warmup):
        cpu_baseline(0.2, bundle)
    vals = []
    t0 = time.perf_counter()
    per_step = max(0.5, min(10.0, 60.0 / max(args.steps, 1)))
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(per_step, bundle)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / max(args.steps, 1) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": {"workload": WORKLOAD["name"], "n": WORKLOAD["n"], "p": WORKLOAD["p"],
                                           "cuts": WORKLOAD["k"]},
           "cpu_baseline": {"value": value, "unit": "amplitudes/s", "cores": last["cores"], "kind": "oracle",
                            "sample": last["sample"] + " per step"},
           "e2e": {"value": value, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


UNEVEN = dict(name="uneven64", jobs=64, n_range=(30, 100), p_choices=(1, 2), k_range=(6, 18), seed=4)
UNEVEN_METRIC = "amplitudes/sec, 64 uneven QAOA jobs (n 30-100, p in {1,2}, own cut set each), one launch sequence"


def setup_uneven(rank: int, jobs: int = 0):
    import concurrent.futures as cf

    from paper_2010_14962_gb300 import instances as I
    from paper_2010_14962_gb300 import qtn

    w = {k: v for k, v in UNEVEN.items() if k != "name"}
    if jobs:
        w["jobs"] = jobs
    spec = I.uneven_jobs(**w)

    def one(jd):
        j, d = jd
        inst = I.qaoa_instance(d["n"], d["p"], d["seed"])
        plan = qtn.plan_job(d["n"], d["p"], inst.edges, inst.gamma, inst.beta, d["k"])
        return inst, plan, I.bitstrings(d["n"], 1, 700 + j + 1000 * rank)[0]

    with cf.ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        jobs = list(ex.map(one, enumerate(spec)))
    return spec, jobs


def uneven_cpu_baseline(seconds: float, jobs):
    """The oracle on a bounded sample of the batch: jobs in a seeded random
    order, each contracted over slice ranges (doubling in size) for at most a
    quarter of ``seconds``; the value is the amplitudes' worth of slices done
    (fraction of each job's 2^k slices, summed) per second, all host cores.
    Depth-2 jobs on more than 40 qubits are left out: the oracle contracts
    the gate network, whose slices there hold 2^30 and more entries."""
    from oracle import oracle as O

    cores = os.cpu_count() or 1
    order = np.random.default_rng(11).permutation(len(jobs))
    per_job = seconds / 4.0
    done_frac = 0.0
    used = []
    t0 = time.perf_counter()
    for j in order:
        if time.perf_counter() - t0 >= seconds:
            break
        inst, plan, x = jobs[j]
        if inst.p == 2 and inst.n > 40:
            continue
        cuts, _ = O.choose_cuts(inst.n, inst.edges, inst.p, plan.k)  # the oracle's own plan
        S = 2 ** len(cuts)
        lo, chunk, tj = 0, 1, time.perf_counter()
        while lo < S and time.perf_counter() - tj < per_job:
            hi = min(S, lo + chunk)
            O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, slices=(lo, hi), threads=cores)
            lo, chunk = hi, chunk * 2
        done_frac += lo / S
        used.append((int(j), round(lo / S, 4)))
    dt = time.perf_counter() - t0
    return {"value": done_frac / dt, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
            "sample": f"slice ranges of {len(used)} of {len(jobs)} jobs (job, fraction of its slices): {used}, "
                      f"{dt:.1f} s"}


def run_uneven(args, rank, world, local_rank):
    import torch

    from paper_2010_14962_gb300 import qtn

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    spec, jobs = setup_uneven(rank, args.jobs)
    pipe_peaks = measure_pipe_peaks(local_rank)
    plans = [j[1] for j in jobs]
    xs = [j[2] for j in jobs]
    nj = len(jobs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(prec):
        # Device time of the whole call (on-chip jobs' launch sequence and the
        # wide jobs after it), CUDA events on the stream.
        ev0.record(stream)
        out = qtn.contract_batch(plans, xs, prec, stream)
        ev1.record(stream)
        ev1.synchronize()
        return out, ev0.elapsed_time(ev1)

    ref = step("fp64")[0]
    sweep = {}
    for prec in (["fp64", "fp32", "fp32x2"] if args.precision == "auto" else [args.precision]):
        for _ in range(2):
            step(prec)
        ms = []
        for _ in range(5):
            got, m = step(prec)
            ms.append(m)
            flush.zero_()
        err = float(np.max(np.abs(got - ref) / np.abs(ref)))
        sweep[prec] = {"amplitudes_per_s": nj / (statistics.median(ms) / 1e3), "max_rel_err_vs_fp64": err}
    if args.precision == "auto":
        ok = [p for p, v in sweep.items() if v["max_rel_err_vs_fp64"] <= 1e-6]
        args.precision = max(ok, key=lambda p: sweep[p]["amplitudes_per_s"])
    prec = args.precision
    for _ in range(args.warmup):
        step(prec)
        flush.zero_()
    torch.cuda.synchronize()
    dev_ms = []
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dev_ms.append(step(prec)[1])
            flush.zero_()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
        time.sleep(0.3)
    total_ms = float(sum(dev_ms))
    if dist:
        t = torch.tensor([total_ms, wall], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, wall = float(t[0].item()), float(t[1].item())
    value = nj * args.steps * world / (total_ms / 1e3)
    e2e_value = nj * args.steps * world / wall
    clocks = clk.summary()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    exec_flops = 0.0
    ran = qtn.batch_last_programs()  # the program each job ran in the last call
    for pl, name in zip(plans, ran):
        prog = pl.describe()["programs"][name]
        exec_flops += 8.0 * ((2 ** len(prog["outer_class"])) * prog["macs_per_item"] + prog["macs_prologue"])
    method_flops = sum((2 ** c["k"]) * 8 * c["macs_per_slice"] for c in (pl.cost() for pl in plans))
    peak = pipe_peak(prec, pipe_peaks)
    avg_s = statistics.mean(dev_ms) / 1e3
    achieved = exec_flops / avg_s / 1e12
    ks = [pl.k for pl in plans]
    out = {
        "metric": UNEVEN_METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "c64", "fp64": "c128", "fp32x2": "c64x2 (double-float)"}.get(prec, "c64"),
        "data": "synthetic: seeded random 3-regular graphs, gamma/beta ~ U[0,pi), seeded bit strings",
        "config": {"workload": UNEVEN["name"] if nj == UNEVEN["jobs"] else f"uneven{nj}", "jobs": nj, "n": [min(d["n"] for d in spec), max(d["n"] for d in spec)],
                   "p1_jobs": sum(d["p"] == 1 for d in spec), "p2_jobs": sum(d["p"] == 2 for d in spec),
                   "graphical_model_jobs": sum(pl.network.form == "gm" for pl in plans),
                   "wide_executor_jobs": sum(name.startswith("wide") for name in ran),
                   "programs_run": ran,
                   "cuts": [min(ks), max(ks)], "precision": prec,
                   "executed_flops_per_step": exec_flops, "method_flops_per_step": method_flops,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "one launch sequence per step: all jobs' chunks on one persistent grid"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "kernel": "whole batch call (multi-job launch sequence of the on-chip jobs, wide executors)",
                     "peak_source": ("measured %s FMA peak of this GPU (qtn_pipe_peaks)"
                                     % ("FP64" if prec == "fp64" else "FP32")),
                     "pipe_issue_frac": achieved * INSTR_PER_MAC[prec] / peak if prec in INSTR_PER_MAC else None,
                     "kernel_ms_avg": avg_s * 1e3},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "amplitudes/s", "h2d_bytes_per_step": int(sum(d["n"] for d in spec)),
                "d2h_bytes_per_step": int(nj * 16), "api": "qtn_contract_batch (host x in, host amplitudes out)"},
        "gpu_launches": None,
        "precision_sweep": sweep,
        "wall_s_timed_region": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = uneven_cpu_baseline(args.cpu_seconds, jobs)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


DEEP = dict(name="qaoa20_p3_k2", n=20, p=3, k=2, seed=11, bitstrings=8)
DEEP_METRIC = "amplitudes/sec, n=20 QAOA p=3, 2 cut edges (per-slice tensors of rank 23: wide executor)"
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate of GB300


def run_deep(args, rank, world, local_rank):
    """The wide executor on a deep circuit whose per-slice tensors exceed
    shared memory: every arithmetic (FP64, FP32X2, FP32, and TF32X3 / TF32
    with their dense merges on the tensor cores) against the state vector;
    the fastest form within 1e-6 is the line's value.  The tensor-core
    kernel's rate comes from the autotuner's CUDA-event timings of the
    merges it won."""
    import torch

    from oracle import oracle as O
    from paper_2010_14962_gb300 import instances as I
    from paper_2010_14962_gb300 import qtn

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    w = DEEP
    inst = I.qaoa_instance(w["n"], w["p"], w["seed"])
    plan = qtn.Plan(qtn.Network(w["n"], inst.edges, inst.gamma, inst.beta), k=w["k"])
    xs = I.bitstrings(w["n"], w["bitstrings"], w["seed"])
    nx = len(xs)
    sv = O.statevector(w["n"], inst.edges, inst.gamma, inst.beta)
    refs = np.array([sv[O.bits_to_int(x)] for x in xs])
    pipe_peaks = measure_pipe_peaks(local_rank)
    peaks_file = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks_file = json.load(f)
    except OSError:
        pass
    tf32_peak = peaks_file.get("bf16_tflops", 1900.0) * TF32_PER_BF16
    stream = torch.cuda.current_stream()
    d_x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    table = {}
    precs = ("fp64", "fp32x2", "fp32", "tf32x3", "tf32") if args.precision == "auto" else (args.precision,)
    for prec in precs:
        d_out = torch.zeros((nx, 2), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            plan.contract_amplitudes_device(d_x, d_out, prec, stream)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        for i in range(args.steps):
            ev[2 * i].record(stream)
            plan.contract_amplitudes_device(d_x, d_out, prec, stream)
            ev[2 * i + 1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        ms = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)) / args.steps
        o = d_out.cpu().numpy()
        got = o[:, 0] + 1j * o[:, 1]
        desc = plan.describe()
        tuned = [t for t in desc["tuned"] if t["prec"] == qtn.PRECISIONS[prec] and t["nx"] == nx][0]
        prog = desc["programs"][tuned["executor"]]
        entry = {"amplitudes_per_s": nx / (ms / 1e3), "ms_per_step": ms, "executor": tuned["executor"],
                 "max_rel_err_vs_statevector": float(np.max(np.abs(got - refs) / np.abs(refs)))}
        states = [st for st in prog.get("wide_states", []) if st["prec"] == qtn.PRECISIONS[prec] and st["nx"] == nx]
        if states:
            st = states[0]
            kinds = {}
            for kname in st["step_kernels"]:
                kinds[kname] = kinds.get(kname, 0) + 1
            entry["step_kernels"] = kinds
            # Merges won by the tensor cores: their algorithmic flops over their
            # timed duration (the tuning launches, group items each).
            tc_flops = tc_ms = 0.0
            tot_ms = 0.0
            for s_desc, k_name, tms in zip(prog["steps"], st["step_kernels"], st["step_ms"]):
                if not tms:
                    continue
                t_best = tms.get(k_name)
                if t_best is None:
                    continue
                tot_ms += t_best
                if k_name == "tcgen05":
                    tc_ms += t_best
                    tc_flops += 8.0 * 2 ** (s_desc["ma"] + s_desc["nb"] + s_desc["kb"] + s_desc["bb"]) * st["group"]
            if tc_ms > 0:
                products = 3 if prec == "tf32x3" else 1
                ach = tc_flops / (tc_ms / 1e3) / 1e12
                entry["tensor_core_merges"] = {
                    "achieved_tflops": ach, "pipe_tflops": ach * products, "peak_tflops": tf32_peak,
                    "frac_of_peak": ach * products / tf32_peak, "time_share_of_timed_steps": tc_ms / tot_ms,
                    "peak_source": "measured bf16 cuBLAS burst (MEASURED_PEAKS.json) x nominal TF32/BF16 ratio 1.1/2.25",
                    "pipe_def": f"{products} TF32 products per complex multiply-add term"}
        table[prec] = entry
    ok = [p for p in table if table[p]["max_rel_err_vs_statevector"] <= 1e-6] or list(table)
    chosen = max(ok, key=lambda p: table[p]["amplitudes_per_s"])
    best = table[chosen]
    cost = plan.cost()
    # End to end through the host API: host x in, host amplitude out.
    t0 = time.perf_counter()
    e2e_n = 0
    while time.perf_counter() - t0 < 1.0 or e2e_n < nx:
        plan.contract_amplitude(xs[e2e_n % nx], chosen)
        e2e_n += 1
    e2e = e2e_n / (time.perf_counter() - t0)
    out = {
        "metric": DEEP_METRIC, "value": best["amplitudes_per_s"], "unit": "amplitudes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "c64", "fp64": "c128", "fp32x2": "c64x2 (double-float)"}.get(chosen, "c64"),
        "data": "synthetic: seeded random 3-regular graph, gamma/beta ~ U[0,pi), seeded bit strings",
        "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "cuts": w["k"], "bitstrings_per_step": nx,
                   "width": cost["width"], "log2_flops_per_amplitude": cost["log2_flops"], "precision": chosen,
                   "l2": "flushed between timed steps (256 MB write)",
                   "precision_rule": "fastest arithmetic within 1e-6 of the state vector on every bit string"},
        "precision_sweep": table,
        "measured_peaks_tflops": {"fp32": pipe_peaks["fp32_tflops"], "fp64": pipe_peaks["fp64_tflops"],
                                  "tf32_tensor": tf32_peak},
        "e2e": {"value": e2e, "unit": "amplitudes/s", "h2d_bytes_per_step": w["n"], "d2h_bytes_per_step": 16,
                "api": "qtn_contract_amplitude (host x in, host amplitude out), one bit string per call"},
    }
    print(json.dumps(out), flush=True)


LEARNED = dict(name="learned120", n=120, p=1, k=22, seed=5, bitstrings=8, train=200000, holdout=10000,
               train_n=(40, 120), train_k=(8, 24), epochs=40)


def run_learned(args, rank, world, local_rank):
    """The learned planner at n = 120: the surrogate is trained on the device
    on exact-counter labels, then Algorithm 1 guided by it and Algorithm 1 with
    the exact counter search 22 cuts under the same evaluation budget, counted
    in exact-counter evaluations (a surrogate evaluation costs the measured
    ratio of feature to exact-count host time); both plans are contracted
    (FP32X2) on the same bit strings."""
    import torch

    from paper_2010_14962_gb300 import instances as I
    from paper_2010_14962_gb300 import qtn

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    w = LEARNED
    threads = min(32, os.cpu_count() or 1)
    t0 = time.perf_counter()
    X, Y = qtn.surrogate_dataset(w["train"] + w["holdout"], w["train_n"][0], w["train_n"][1], 1, 1, w["train_k"][0],
                                 w["train_k"][1], seed=11, threads=threads)
    t_data = time.perf_counter() - t0
    m = qtn.MLP(qtn.SURROGATE_FEATURES, 256, qtn.SURROGATE_TARGETS, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = m.fit(X[: w["train"]], Y[: w["train"]], epochs=w["epochs"], batch=512, lr=1e-3, seed=2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    P = m.predict(X[w["train"]:])
    Yv = Y[w["train"]:]
    rank_of = lambda v: np.argsort(np.argsort(v))
    spearman = float(np.corrcoef(rank_of(P[:, 0]), rank_of(Yv[:, 0]))[0, 1])
    mae = float(np.mean(np.abs(P[:, 0] - Yv[:, 0])))

    inst = I.qaoa_instance(w["n"], w["p"], w["seed"])
    net = qtn.Network(w["n"], inst.edges, inst.gamma, inst.beta)
    # Host cost of one surrogate evaluation (features) against one exact count.
    _, n_idx = net.info()
    rng = np.random.default_rng(0)
    sets = [rng.choice(n_idx, w["k"], replace=False).astype(np.int32) for _ in range(200)]
    t0 = time.perf_counter()
    for c in sets:
        qtn.surrogate_features(net, c)
    t_feat = (time.perf_counter() - t0) / len(sets)
    t0 = time.perf_counter()
    for c in sets:
        qtn.surrogate_labels(net, c)
    t_exact = (time.perf_counter() - t0) / len(sets)
    eval_cost = t_feat / t_exact
    searches = {}
    nets = {w["seed"]: net}
    for g in (6, 7):
        gi = I.qaoa_instance(w["n"], w["p"], g)
        nets[g] = qtn.Network(w["n"], gi.edges, gi.gamma, gi.beta)
    runs = [(f"graph{g}_random_start_seed{sd}", g, False, sd) for g in nets for sd in (1, 2, 3)]
    runs.append(("greedy_seeded", w["seed"], True, 1))
    for label, g, seed_greedy, seed in runs:
        net_g = nets[g]
        t0 = time.perf_counter()
        cuts_s, best_s, n_exact, n_sur, _ = qtn.search_cuts_surrogate(net_g, w["k"], m, T=10, N=256, top=4, seed=seed,
                                                                       seed_greedy=seed_greedy)
        t_s = time.perf_counter() - t0
        budget = n_exact + eval_cost * n_sur
        t0 = time.perf_counter()
        cuts_e, _, n_ga = qtn.search_cuts(net_g, w["k"], "ga_flops", seed=seed, ga_T=max(1, int(budget // 11) - 1),
                                          ga_N=11, seed_greedy=seed_greedy)
        t_e = time.perf_counter() - t0
        best_e = float(qtn.surrogate_labels(net_g, cuts_e)[0])
        searches[label] = dict(
            budget_exact_evals=budget,
            surrogate=dict(log2_flops=float(best_s), surrogate_evals=n_sur, exact_evals=n_exact, search_s=t_s,
                           cuts=[int(c) for c in cuts_s]),
            exact=dict(log2_flops=best_e, exact_evals=n_ga, search_s=t_e, cuts=[int(c) for c in cuts_e]))
    gains = [searches[k]["exact"]["log2_flops"] - searches[k]["surrogate"]["log2_flops"]
             for k in searches if "random_start" in k]
    pick = searches["greedy_seeded"]
    plans = {"surrogate": qtn.Plan(net, cuts=pick["surrogate"]["cuts"], max_slice_bytes=150e9),
             "exact": qtn.Plan(net, cuts=pick["exact"]["cuts"], max_slice_bytes=150e9)}
    xs = I.bitstrings(w["n"], w["bitstrings"], w["seed"])
    d_x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    results, vals = {}, {}
    for name, plan in plans.items():
        d_out = torch.zeros((len(xs), 2), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            plan.contract_amplitudes_device(d_x, d_out, "fp32x2", stream)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        for i in range(args.steps):
            ev[2 * i].record(stream)
            plan.contract_amplitudes_device(d_x, d_out, "fp32x2", stream)
            ev[2 * i + 1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        ms = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps))
        o = d_out.cpu().numpy()
        vals[name] = o[:, 0] + 1j * o[:, 1]
        c = plan.cost()
        results[name] = dict(amplitudes_per_s=len(xs) * args.steps / (ms / 1e3), log2_flops=c["log2_flops"],
                             log2_peak_bytes=c["log2_peak_bytes"], width=c["width"])
    agree = float(np.max(np.abs(vals["surrogate"] - vals["exact"]) / np.abs(vals["exact"])))
    out = {
        "metric": "amplitudes/sec, n=120 QAOA p=1, 22 cuts from the surrogate-guided search",
        "value": results["surrogate"]["amplitudes_per_s"], "unit": "amplitudes/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64x2 (double-float)", "data": "synthetic: seeded random 3-regular graphs",
        "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "cuts": w["k"], "bitstrings_per_step": len(xs),
                   "surrogate": {"train_pairs": w["train"], "holdout_pairs": w["holdout"], "epochs": w["epochs"],
                                 "layers": 3, "width": 256, "dataset_s": t_data, "train_s": t_train,
                                 "loss_first_last": [float(losses[0]), float(losses[-1])],
                                 "holdout_spearman_log2_flops": spearman, "holdout_mae_log2_flops": mae},
                   "search_budget": "equal, in exact-counter evaluations; a surrogate evaluation counts as "
                                    "feature_s / exact_count_s (measured on the host)",
                   "feature_s": t_feat, "exact_count_s": t_exact, "surrogate_eval_cost": eval_cost,
                   "searches": searches,
                   "random_start_mean_gain_log2_flops": float(np.mean(gains)),
                   "random_start_gains_log2_flops": [float(x) for x in gains],
                   "contracted": results, "max_rel_diff_between_plans": agree,
                   "memory_cap_bytes": 150e9},
    }
    print(json.dumps(out), flush=True)


def setup_workload_cpu():
    """The workload's instance, bit strings and the oracle's own 16-cut set:
    inputs from the instance generator only, so the reference arm never loads
    the product library."""
    from oracle import oracle as O
    from paper_2010_14962_gb300 import instances as I

    w = WORKLOAD
    inst = I.qaoa_instance(w["n"], w["p"], w["seed"])
    xs = I.bitstrings(w["n"], w["bitstrings"], w["seed"])
    cuts, _ = O.choose_cuts(w["n"], inst.edges, w["p"], 16)
    return inst, xs, cuts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="auto", choices=["auto"] + SWEEP,
                    help="auto: sweep every arithmetic and time the fastest within 1e-6 of the FP64 GPU form")
    ap.add_argument("--no-oracle-refs", action="store_true", help="sweep without the oracle's reference values")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--executor", default=None, help="force an executor (default: autotuned)")
    ap.add_argument("--workload", default="qaoa80_p1_k16",
                    choices=["qaoa80_p1_k16", "uneven64", "learned120", "qaoa20_p3_k2"],
                    help="uneven64: 64 independent jobs of different plans in one launch sequence")
    ap.add_argument("--jobs", type=int, default=0, help="uneven64: take the first N jobs (default all 64)")
    ap.add_argument("--form", default="gates", choices=["gates", "gm"],
                    help="network form of the n=80 workload: the paper's gate network (16 cuts) or the "
                         "graphical model with shared diagonal-gate indices (8 cuts)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.form == "gm":
        global METRIC
        WORKLOAD.update(name="qaoa80_p1_gm_k8", k=8, form="gm")
        METRIC = "amplitudes/sec, n=80 QAOA p=1, graphical-model network, 8 cut variables (256 slices)"
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "uneven64":
        run_uneven(args, rank, world, local_rank)
    elif args.workload == "learned120":
        run_learned(args, rank, world, local_rank)
    elif args.workload == "qaoa20_p3_k2":
        run_deep(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
