#!/usr/bin/env python
"""Q2X benchmark: element-moments/s of the Q2X step on GB300.

Workload: the SH-perturbed level-7 icosphere (327,680 flat triangles,
163,842 vertices), linear per-vertex density U[-1,1], uniform depth-5 octree
over [-1.125, 1.125]^3, p = 12, single + double layer in one pass, FP64
coefficients out.  A step is one Q2X call over the whole mesh; the metric
counts (p+1)^2 moments per element per output layer.  The FP32-mixed path is
measured on the same workload and reported beside it, each with its error
against the FP64 oracle on the CPU-baseline sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch with torch.distributed.run: the workload is replicated N
times, the leaf list cut into N contiguous cost-balanced ranges and each rank
runs its range (weak scaling; no collective on the data path, the step time is
the max over ranks).
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

import workloads as W  # noqa: E402

METRIC = "Q2X element-moments/s (elems*(p+1)^2), FP32-mixed vs FP64 at stated rel. error"
UNIT = "element-moments/s"
LEVEL, DEPTH, P = 7, 5, 12
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the FP64
# element kernel on this workload, from the ncu capture summarised in the
# profile named below (set to None whenever the kernel changes)
TRAFFIC_FP64 = 9732864 + 39978752
TRAFFIC_SOURCE = "ncu --set full, profiles/q2x_elem_kernel_sphere-L7-linear-p12.md (bytes per launch)"
# FP64 flops the same capture counted as executed per launch: 2 x DFMA + DADD + DMUL
# thread instructions (168.70 + 79.73 + 11.38 per elapsed cycle over 6.674 M cycles)
EXECUTED_FLOPS_FP64 = (2 * 168.701704 + 79.728916 + 11.382976) * 6673646.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default="sphere-L7-linear",
                    choices=["sphere-L7-linear", "icosphere-L3", "sphere-L9-const", "mixed-ball",
                             "sphere-L8-adjoint", "upward", "far-field", "galerkin", "biot-savart", "leaf-reduce",
                             "near-field"],
                    help="workload; the default is the headline configuration, the others are the "
                         "precision, ragged-batch and adjoint configurations")
    return ap.parse_args()


def workload():
    return W.cfg_sphere_linear(level=LEVEL, depth=DEPTH, p=P)


def workload_name(prob):
    return "sphere-L%d-linear-depth%d: %d triangles, %d vertices, %d leaves, p=%d, single+double layer" % (
        LEVEL, DEPTH, prob["idx"].shape[1], prob["vxyz"].shape[1], prob["leaf_c"].shape[1], P)


def moments_per_step(prob, layers=2):
    return layers * prob["idx"].shape[1] * (P + 1) ** 2


# ------------------------------------------------------------ oracle (CPU)

def sample_leaves(prob, target_elems):
    """Leaves taken in a fixed seeded order until target_elems elements."""
    off = prob["leaf_off"]
    nl = off.shape[0] - 1
    order = np.random.default_rng(99).permutation(nl)
    pick, tot = [], 0
    for L in order:
        pick.append(int(L))
        tot += int(off[L + 1] - off[L])
        if tot >= target_elems:
            break
    return np.array(sorted(pick))


def sub_problem(prob, leaves):
    off = prob["leaf_off"]
    idx = np.concatenate([prob["idx"][:, off[L]:off[L + 1]] for L in leaves], axis=1)
    sizes = np.array([off[L + 1] - off[L] for L in leaves])
    sub_off = np.zeros(len(leaves) + 1, dtype=np.int64)
    np.cumsum(sizes, out=sub_off[1:])
    return dict(vxyz=prob["vxyz"], idx=np.ascontiguousarray(idx), sigma=prob["sigma"], leaf_off=sub_off,
                leaf_c=np.ascontiguousarray(prob["leaf_c"][:, leaves]), leaf_rho=prob["leaf_rho"][leaves],
                p=prob["p"])


def oracle_run(orc, sub, nthreads=0):
    s = orc.moments("triangle", sub["vxyz"], sub["idx"], sub["sigma"], P, leaf_off=sub["leaf_off"],
                    leaf_c=sub["leaf_c"], layer=0, density=1, nthreads=nthreads)
    d = orc.moments("triangle", sub["vxyz"], sub["idx"], sub["sigma"], P, leaf_off=sub["leaf_off"],
                    leaf_c=sub["leaf_c"], layer=1, density=1, nthreads=nthreads)
    return s, d


def calibrate_sample(orc, prob, seconds):
    """Number of elements whose oracle run takes about `seconds`."""
    probe = sub_problem(prob, sample_leaves(prob, 2000))
    t0 = time.perf_counter()
    oracle_run(orc, probe)
    dt = time.perf_counter() - t0
    per = dt / max(1, probe["idx"].shape[1])
    return max(200, int(seconds / per))


def norm_err(test, ref, rho, layer):
    """max over leaves of max|dM^| / max|M^_ref| with M^_n^m = M_n^m
    sqrt((n+|m|)!(n-|m|)!) / rho^n (double layer: / (n rho^{n-1}))."""
    worst = 0.0
    for L in range(ref.shape[0]):
        s = np.zeros((P + 1) ** 2)
        for n in range(P + 1):
            for m in range(-n, n + 1):
                f = math.sqrt(math.factorial(n + abs(m)) * math.factorial(n - abs(m)))
                s[n * n + n + m] = f / rho[L] ** n if layer == 0 else f / (max(n, 1) * rho[L] ** max(n - 1, 0))
        den = np.max(np.abs(ref[L] * s))
        num = np.max(np.abs((test[L] - ref[L]) * s))
        worst = max(worst, num / den if den > 0 else num)
    return worst


# ------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.uuid = uuid
        self.path = os.path.join(tempfile.gettempdir(), "q2x_clocks_%d.csv" % os.getpid())

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as orc
    prob = workload()
    cores = orc.max_threads()
    n = calibrate_sample(orc, prob, max(1.0, args.cpu_seconds / 3))
    sub = sub_problem(prob, sample_leaves(prob, n))
    ne = sub["idx"].shape[1]
    for _ in range(args.warmup):
        oracle_run(orc, sub)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_run(orc, sub)
    dt = (time.perf_counter() - t0) / args.steps
    val = 2 * ne * (P + 1) ** 2 / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(prob), "sample_elements": ne},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d of %d triangles (whole leaves), single+double layer, FP64 Gauss "
                                       "quadrature, OpenMP" % (ne, prob["idx"].shape[1])},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ our arm

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.config != "sphere-L7-linear":
        import bench_configs
        return bench_configs.run(args)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2107_10942_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.q2x import problem_to_device
    from paper_2107_10942_gb300.roofline import PEAK_FP32_FLOPS, PEAK_FP64_FLOPS, element_flops

    full = workload()
    prob = full
    if world > 1:
        # weak scaling: `world` copies of the workload, leaves cut into
        # contiguous cost-balanced ranges, one range per rank, no collective
        from paper_2107_10942_gb300 import shard as S
        rep = S.replicate_problem(full, world)
        bounds = S.partition_leaves(S.leaf_costs(rep["leaf_off"], rep["leaf_p"], "triangle", "linear", 2), world)
        prob = S.shard_problem(rep, bounds[rank], bounds[rank + 1])
        del rep
    d = problem_to_device(prob, dev)
    n_elem = prob["idx"].shape[1]
    nc = (P + 1) ** 2
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    outs = {}

    def step(plan, cs, cd):
        plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                       density="linear", single=True, double=True, coef_single=cs, coef_double=cd)

    def timed(prec):
        plan = q.Plan(P, precision=prec)
        cs = torch.empty((prob["leaf_c"].shape[1], nc), dtype=torch.float64, device=dev)
        cd = torch.empty_like(cs)
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step(plan, cs, cd)
        plan.sync()
        # the step (checks, element kernel, fix-up) as one CUDA graph, timed over K replays
        g = plan.capture(lambda: step(plan, cs, cd))
        for _ in range(args.warmup):
            flush.fill_(1.0)
            g.replay()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))  # L2 flush between timed steps (outside the events)
            evs[k][0].record(stream)
            g.replay()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        plan.sync()
        launches = g.kernels * args.steps
        ms_steps = [a.elapsed_time(b) for a, b in evs]
        # the element kernel's own duration: the same steps launched directly, with the
        # plan's CUDA events around that kernel (untimed for the step figure)
        plan.set_kernel_timing(True)
        plan.kernel_timing()
        for k in range(args.steps):
            flush.fill_(float(k))
            step(plan, cs, cd)
        kms, kn = plan.kernel_timing()
        plan.set_kernel_timing(False)
        plan.sync()
        ms = sum(ms_steps) / len(ms_steps)
        if dist:
            t = torch.tensor([ms], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        outs[prec] = (cs.cpu().numpy(), cd.cpu().numpy())
        return dict(ms=ms, kernel_ms=kms / max(kn, 1), launches=launches, plan=plan)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = ClockSampler(uuid) if rank == 0 else None
    if clk:
        clk.start()
    r64 = timed("fp64")
    clocks = clk.stop() if clk else None
    r32 = timed("fp32")

    # ---- end to end through the public API with host buffers
    host = {k: torch.from_numpy(np.ascontiguousarray(prob[k])).pin_memory()
            for k in ("vxyz", "idx", "sigma", "leaf_off", "leaf_c", "leaf_rho")}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    out_s = torch.empty((prob["leaf_c"].shape[1], nc), dtype=torch.float64).pin_memory()
    out_d = torch.empty_like(out_s).pin_memory()
    d2h = 2 * out_s.numel() * 8
    plan = q.Plan(P, precision="fp64")

    def e2e_step():
        g = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        cs, cd = plan.triangles(g["vxyz"], g["idx"], g["sigma"], g["leaf_off"], g["leaf_c"], g["leaf_rho"], None,
                                density="linear", single=True, double=True)
        out_s.copy_(cs, non_blocking=True)
        out_d.copy_(cd, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    plan.sync()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
        dist.barrier()

    per_step = moments_per_step(prob)
    total_moments = per_step
    if dist:
        t = torch.tensor([per_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_moments = float(t.item())
    value = total_moments / (r64["ms"] * 1e-3)
    flops_elem = element_flops("triangle", "linear", ("single", "double"), P)
    achieved64 = flops_elem * n_elem / (r64["kernel_ms"] * 1e-3)
    achieved32 = flops_elem * n_elem / (r32["kernel_ms"] * 1e-3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- CPU baseline: the oracle on a bounded sample, and the GPU errors on it
    cpu = None
    errs = {}
    if not args.no_cpu_baseline and world == 1:
        import oracle as orc
        n = calibrate_sample(orc, prob, args.cpu_seconds)
        leaves = sample_leaves(prob, n)
        sub = sub_problem(prob, leaves)
        t0 = time.perf_counter()
        ref_s, ref_d = oracle_run(orc, sub)
        dt = time.perf_counter() - t0
        ne = sub["idx"].shape[1]
        cpu = {"value": 2 * ne * nc / dt, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
               "sample": "%d of %d triangles (%d whole leaves), single+double layer, FP64 Gauss quadrature "
                         "(%d nodes/direction), OpenMP; %.1f s" % (ne, n_elem, len(leaves), (P + 5) // 2, dt)}
        # the same oracle on one core, on a sample sized for about a quarter of that time
        leaves1 = sample_leaves(prob, max(200, int(ne * min(1.0, 0.25 / max(orc.max_threads(), 1)))))
        sub1 = sub_problem(prob, leaves1)
        t0 = time.perf_counter()
        oracle_run(orc, sub1, nthreads=1)
        dt1 = time.perf_counter() - t0
        ne1 = sub1["idx"].shape[1]
        cpu["single_core"] = {"value": 2 * ne1 * nc / dt1, "unit": UNIT, "cores": 1,
                              "sample": "%d triangles (%d whole leaves), %.1f s" % (ne1, len(leaves1), dt1)}
        for prec in ("fp64", "fp32"):
            cs, cd = outs[prec]
            errs[prec] = {"single": norm_err(cs[leaves], ref_s, prob["leaf_rho"][leaves], 0),
                          "double": norm_err(cd[leaves], ref_d, prob["leaf_rho"][leaves], 1)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(full) + (" per rank" if world > 1 else ""), "precision": "fp64",
                   "density": "linear", "layers": ["single", "double"], "p": P, "n_elem": n_elem,
                   "moments_per_step": total_moments, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "leaf-sharded dp%d (no collective)" % world if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved64 / 1e12, "peak": PEAK_FP64_FLOPS / 1e12,
                     "unit": "TFLOP/s", "frac": achieved64 / PEAK_FP64_FLOPS, "traffic": TRAFFIC_FP64,
                     "traffic_source": TRAFFIC_SOURCE,
                     "kernel": "q2x_elem_kernel<double,12,TRI,LINEAR>", "kernel_ms": r64["kernel_ms"],
                     "flops_per_launch": flops_elem * n_elem,
                     "executed": {"flops_per_launch": EXECUTED_FLOPS_FP64,
                                  "frac": EXECUTED_FLOPS_FP64 / (r64["kernel_ms"] * 1e-3) / PEAK_FP64_FLOPS,
                                  "source": "ncu DFMA/DADD/DMUL counts, " + TRAFFIC_SOURCE},
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz (recipe FP64 1.25 TF)"},
        "fp32_mixed": {"value": total_moments / (r32["ms"] * 1e-3), "ms_per_step": r32["ms"],
                       "speedup_vs_fp64": r64["ms"] / r32["ms"],
                       "roofline": {"bound": "alu", "achieved": achieved32 / 1e12, "peak": PEAK_FP32_FLOPS / 1e12,
                                    "unit": "TFLOP/s", "frac": achieved32 / PEAK_FP32_FLOPS,
                                    "kernel": "q2x_elem_kernel<float,12,TRI,LINEAR>", "kernel_ms": r32["kernel_ms"],
                                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"}},
        "errors_vs_oracle": errs or None,
        "cpu_baseline": cpu,
        "e2e": {"value": total_moments / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": r64["launches"],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
