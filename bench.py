#!/usr/bin/env python
"""Q2X benchmark: element-moments/s of the Q2X step on GB300.

Headline workload (the precision configuration): the SH-perturbed level-9
icosphere (5,242,880 flat triangles, 2,621,442 vertices), constant density
U[-1,1] per triangle, uniform depth-7 octree over [-1.125, 1.125]^3 (59,805
non-empty leaves), p = 16, single layer, FP64 coefficients out.  A step is one
Q2X call over the whole mesh; the metric counts (p+1)^2 moments per element
and output layer.  `value` is the plain FP64 path; the FP32-mixed path runs
on the same workload and is reported beside it, each with its normalised
coefficient error against the FP64 oracle on sampled leaves, and with the
far-field potential error of both coefficient sets at stated targets (the
speedup at equal accuracy).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config sphere-L9-const|sphere-L7-linear|...]

`--config sphere-L7-linear` runs the level-7 workload (327,680 triangles,
linear per-vertex density, depth 5, p = 12, single + double layer) through
the same path; the other configurations live in bench_configs.py.

For N > 1 launch with torch.distributed.run: the workload is replicated N
times, the leaf list cut into N contiguous cost-balanced ranges and each rank
runs its range (weak scaling; no collective on the data path, the step time is
the max over ranks).
"""
from __future__ import annotations

import argparse
import datetime
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
L2_FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "sphere-L9-const": dict(level=9, depth=7, p=16, density="const", layers=("single",),
                            gen=lambda: W.cfg_sphere_const(level=9, depth=7, p=16)),
    "sphere-L7-linear": dict(level=7, depth=5, p=12, density="linear", layers=("single", "double"),
                             gen=lambda: W.cfg_sphere_linear(level=7, depth=5, p=12)),
}
DEFAULT_WORKLOAD = "sphere-L9-const"

# Per-launch DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) and
# executed flops of the dominant kernel of each arm (the element kernel; for
# the FP32-mixed single layer, the leaf-tile kernel), from one ncu capture of
# the current kernel on each workload (empty: not captured since the kernel
# last changed).  The leaf-tile kernel's executed count includes the idle
# lanes of rounds that a leaf fills only partly.
# Executed flops: FP64 2 x DFMA + DADD + DMUL thread instructions; FP32
# 4 x FFMA2 + 2 x FFMA + 2 x FADD2 + 2 x FMUL2 + FADD + FMUL (per-opcode thread counts:
# the packed instructions are not in the FFMA/FADD class counters).
KERNEL_COUNTERS = {
    ("sphere-L9-const", "fp64"): dict(traffic=218932480 + 111733248, executed_flops=29402290440),
    ("sphere-L9-const", "fp32"): dict(traffic=177844224 + 104552192, executed_flops=47011848132),
    ("sphere-L7-linear", "fp64"): dict(traffic=9516288 + 23808, executed_flops=2644445248),
    ("sphere-L7-linear", "fp32"): dict(traffic=9379072 + 512, executed_flops=3266600364),
}
COUNTER_SOURCE = "ncu --set full capture of one launch of this kernel on this workload"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default=DEFAULT_WORKLOAD,
                    choices=list(WORKLOADS) + ["icosphere-L3", "mixed-ball", "sphere-L8-adjoint", "upward",
                                               "far-field", "galerkin", "biot-savart", "leaf-reduce", "near-field"],
                    help="workload; the default is the headline (precision) configuration")
    return ap.parse_args()


def workload_name(wl, prob):
    return "%s-depth%d: %d triangles, %d vertices, %d leaves, p=%d, %s layer%s, %s density" % (
        "sphere-L%d-%s" % (wl["level"], wl["density"]), wl["depth"], prob["idx"].shape[1], prob["vxyz"].shape[1],
        prob["leaf_c"].shape[1], wl["p"], "+".join(wl["layers"]), "s" if len(wl["layers"]) > 1 else "",
        "linear per-vertex" if wl["density"] == "linear" else "constant")


# ------------------------------------------------------------ oracle (CPU)

def sample_leaves(prob, target_elems, seed=99):
    """Leaves taken in a fixed seeded order until target_elems elements."""
    off = prob["leaf_off"]
    nl = off.shape[0] - 1
    order = np.random.default_rng(seed).permutation(nl)
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
    if prob.get("density") == "linear":
        sigma = prob["sigma"]
    else:
        sigma = np.concatenate([prob["sigma"][off[L]:off[L + 1]] for L in leaves])
    return dict(vxyz=prob["vxyz"], idx=np.ascontiguousarray(idx), sigma=sigma, leaf_off=sub_off,
                leaf_c=np.ascontiguousarray(prob["leaf_c"][:, leaves]), leaf_rho=prob["leaf_rho"][leaves],
                p=prob["p"], density=prob.get("density", "const"))


def oracle_run(orc, wl, sub, nthreads=0):
    dens = 1 if wl["density"] == "linear" else 0
    return [orc.moments("triangle", sub["vxyz"], sub["idx"], sub["sigma"], wl["p"], leaf_off=sub["leaf_off"],
                        leaf_c=sub["leaf_c"], layer=0 if ly == "single" else 1, density=dens, nthreads=nthreads)
            for ly in wl["layers"]]


def calibrate_sample(orc, wl, prob, seconds):
    """Number of elements whose oracle run takes about `seconds`."""
    probe = sub_problem(prob, sample_leaves(prob, 2000))
    t0 = time.perf_counter()
    oracle_run(orc, wl, probe)
    dt = time.perf_counter() - t0
    per = dt / max(1, probe["idx"].shape[1])
    return max(200, int(seconds / per))


def norm_err(test, ref, rho, layer, p):
    """max over leaves of max|dM^| / max|M^_ref| with M^_n^m = M_n^m
    sqrt((n+|m|)!(n-|m|)!) / rho^n (double layer: / (n rho^{n-1}))."""
    worst = 0.0
    for L in range(ref.shape[0]):
        s = np.zeros((p + 1) ** 2)
        for n in range(p + 1):
            for m in range(-n, n + 1):
                f = math.sqrt(math.factorial(n + abs(m)) * math.factorial(n - abs(m)))
                s[n * n + n + m] = f / rho[L] ** n if layer == 0 else f / (max(n, 1) * rho[L] ** max(n - 1, 0))
        den = np.max(np.abs(ref[L] * s))
        num = np.max(np.abs((test[L] - ref[L]) * s))
        worst = max(worst, num / den if den > 0 else num)
    return worst


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms, query only) with timestamps, so that
    each timed window gets the clocks seen inside it."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid=None):
        self.proc = None
        self.uuid = uuid
        self.path = os.path.join(tempfile.gettempdir(), "q2x_clocks_%d.csv" % os.getpid())
        self.windows = []
        self.samples = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def window(self, name, t0, t1):
        self.windows.append((name, t0, t1))

    def stop(self):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        out = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, smax, pw = float(parts[2]), float(parts[3]), float(parts[4])
            except ValueError:
                continue
            reasons = [nm for nm, v in zip(self.REASONS, parts[6:10]) if v.lower() == "active"]
            out.append((ts, sm, smax, pw, reasons))
        self.samples = out

    def summary(self, names=None):
        """Clocks over the windows named (all windows if None)."""
        if self.samples is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        wins = [w for w in self.windows if names is None or w[0] in names]
        sel = [s for s in self.samples if any(t0 - 0.1 <= s[0] <= t1 + 0.1 for _, t0, t1 in wins)]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = sorted({r for s in sel for r in s[4]})
        return {"sm_mhz": statistics.median(s[1] for s in sel), "sm_max_mhz": max(s[2] for s in sel),
                "reasons": reasons, "samples": len(sel), "power_w_max": max(s[3] for s in sel)}

    def per_window(self):
        return {name: self.summary([name]) for name, _, _ in self.windows}


# ------------------------------------------------------------ ALU peaks

def measure_alu_peaks(dev, seconds=1.0, clk=None):
    """FMA rate of the device's FP64 and FP32 pipes from the library's FMA-chain
    probe (q2x_alu_peak_probe): a short calibration launch, then one launch
    sized to about `seconds`, timed with CUDA events on the launching stream."""
    import torch
    from paper_2107_10942_gb300.q2x import alu_peak_probe
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for kind in ("dfma", "ffma", "ffma2"):
        iters = 1024 if kind == "dfma" else 16384
        while True:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            alu_peak_probe(kind, iters, sink, stream)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            if ms > 20.0 or iters > (1 << 36):
                break
            iters *= 4
        iters = max(16, int(iters * seconds * 1e3 / ms))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        a.record(stream)
        flops = alu_peak_probe(kind, iters, sink, stream)
        b.record(stream)
        b.synchronize()
        t1 = time.time()
        ms = a.elapsed_time(b)
        if clk:
            clk.window("peak_" + kind, t0, t1)
        res[kind] = {"tflops": flops / (ms * 1e-3) / 1e12, "ms": ms}
    return res


# ------------------------------------------------------------ equal accuracy

def equal_accuracy(orc, prob, wl, coef64, coef32, n_leaves=24, n_dir=16, dists=(1.5, 2.0, 3.0)):
    """Far-field potential error of the FP64 and FP32-mixed leaf coefficients.

    For n_leaves sampled leaves and targets at distance d = f * h (h the leaf
    side, f in dists) from the leaf centre in n_dir seeded directions: the
    series sum F_n^m S_n^m(r - c) (Eq. (bas3)) of each coefficient set,
    against the leaf's exact potential (1/4pi) sum_e int sigma / |r - y| by
    the oracle's direct quadrature.  Error per leaf = max |phi - phi_exact| /
    max |phi_exact| over its targets; reported is the maximum over leaves.
    For the FP64 set the error of every truncation degree p' <= p is also
    formed (its first (p'+1)^2 coefficients), so the smallest FP64 degree at
    least as accurate as FP32-mixed at degree p is known."""
    p = wl["p"]
    off = prob["leaf_off"]
    h = 2.25 / (1 << wl["depth"])
    rng = np.random.default_rng(41)
    nl = off.shape[0] - 1
    cand = np.nonzero(np.diff(off) >= 8)[0]
    leaves = np.sort(rng.choice(cand, size=min(n_leaves, len(cand)), replace=False))
    dens = 1 if wl["density"] == "linear" else 0
    out = {}
    for f in dists:
        e32 = 0.0
        e64 = np.zeros(p + 1)
        for L in leaves:
            c = prob["leaf_c"][:, L]
            dirs = rng.normal(size=(n_dir, 3))
            tgt = c[None, :] + f * h * dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
            idx = np.ascontiguousarray(prob["idx"][:, off[L]:off[L + 1]])
            sig = prob["sigma"] if dens else prob["sigma"][off[L]:off[L + 1]]
            exact = orc.potential("triangle", prob["vxyz"], idx, sig, tgt, density=dens, nq=12)
            scale = np.max(np.abs(exact))
            phi32, _ = orc.farfield(coef32[L], c, tgt, p)
            e32 = max(e32, float(np.max(np.abs(phi32 - exact)) / scale))
            for pp in range(p + 1):
                phi64, _ = orc.farfield(coef64[L][:(pp + 1) ** 2], c, tgt, pp)
                e64[pp] = max(e64[pp], float(np.max(np.abs(phi64 - exact)) / scale))
        p_eq = next((pp for pp in range(p + 1) if e64[pp] <= e32), p)
        out[f] = {"d_over_h": f, "err_fp32_mixed": e32, "err_fp64": float(e64[p]), "fp64_degree_equal": int(p_eq),
                  "err_fp64_at_that_degree": float(e64[p_eq]), "err_fp64_by_degree": [float(x) for x in e64]}
    return leaves, h, out


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as orc
    wl = WORKLOADS[args.config]
    prob = wl["gen"]()
    cores = orc.max_threads()
    n = calibrate_sample(orc, wl, prob, max(1.0, args.cpu_seconds / 3))
    sub = sub_problem(prob, sample_leaves(prob, n))
    ne = sub["idx"].shape[1]
    nc = (wl["p"] + 1) ** 2
    for _ in range(args.warmup):
        oracle_run(orc, wl, sub)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_run(orc, wl, sub)
    dt = (time.perf_counter() - t0) / args.steps
    val = len(wl["layers"]) * ne * nc / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(wl, prob), "sample_elements": ne},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d of %d triangles (whole leaves), %s layer, FP64 Gauss quadrature, "
                                       "OpenMP" % (ne, prob["idx"].shape[1], "+".join(wl["layers"]))},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ our arm

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.config not in WORKLOADS:
            args.config = DEFAULT_WORKLOAD
        return run_reference(args, rank, world)
    if args.config not in WORKLOADS:
        import bench_configs
        return bench_configs.run(args)
    wl = WORKLOADS[args.config]
    P = wl["p"]
    layers = wl["layers"]
    single, double = "single" in layers, "double" in layers

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
    from paper_2107_10942_gb300.roofline import element_flops

    full = wl["gen"]()
    prob = full
    if world > 1:
        # weak scaling: `world` copies of the workload, leaves cut into
        # contiguous cost-balanced ranges, one range per rank, no collective
        from paper_2107_10942_gb300 import shard as S
        rep = S.replicate_problem(full, world)
        bounds = S.partition_leaves(S.leaf_costs(rep["leaf_off"], rep["leaf_p"], "triangle", wl["density"],
                                                 len(layers)), world)
        prob = S.shard_problem(rep, bounds[rank], bounds[rank + 1])
        del rep
    d = problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")}, dev)
    n_elem = prob["idx"].shape[1]
    n_leaves = prob["leaf_c"].shape[1]
    nc = (P + 1) ** 2
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    outs = {}

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = ClockSampler(uuid) if rank == 0 else None
    if clk:
        clk.start()

    peaks = measure_alu_peaks(dev, 1.0, clk)
    peak64 = peaks["dfma"]["tflops"] * 1e12
    peak32 = max(peaks["ffma"]["tflops"], peaks["ffma2"]["tflops"]) * 1e12

    def step(plan, cs, cd):
        plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                       density=wl["density"], single=single, double=double, coef_single=cs, coef_double=cd)

    def timed(prec, p_eff=P, min_seconds=0.0, keep=True):
        """K graph replays of the step (L2 flushed between them); repeated in
        rounds of K until min_seconds of device time, so that short steps
        still span clock samples.  Then the element kernel's own duration
        from the same steps launched directly with the plan's events."""
        plan = q.Plan(p_eff, precision=prec)
        ncp = (p_eff + 1) ** 2
        cs = torch.empty((n_leaves, ncp), dtype=torch.float64, device=dev) if single else None
        cd = torch.empty((n_leaves, ncp), dtype=torch.float64, device=dev) if double else None
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step(plan, cs, cd)
        plan.sync()
        g = plan.capture(lambda: step(plan, cs, cd))
        for _ in range(args.warmup):
            flush.fill_(1.0)
            g.replay()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ms_steps = []
        t0 = time.time()
        rounds = 0
        while True:
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for k in range(args.steps):
                flush.fill_(float(k))  # L2 flush between timed steps (outside the events)
                evs[k][0].record(stream)
                g.replay()
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            ms_steps += [a.elapsed_time(b) for a, b in evs]
            rounds += 1
            if sum(ms_steps) >= min_seconds * 1e3:
                break
        t1 = time.time()
        if dist:
            dist.barrier()
        plan.sync()
        if clk:
            clk.window("%s_p%d" % (prec, p_eff), t0, t1)
        launches = g.kernels * args.steps
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
        if keep:
            outs[prec] = (cs.cpu().numpy() if single else None, cd.cpu().numpy() if double else None)
        return dict(ms=ms, kernel_ms=kms / max(kn, 1), launches=launches, steps=len(ms_steps), rounds=rounds)

    r64 = timed("fp64")
    r32 = timed("fp32", min_seconds=1.0)

    # ---- end to end through the public API with host buffers
    keys = ("vxyz", "idx", "sigma", "leaf_off", "leaf_c", "leaf_rho")
    host = {k: torch.from_numpy(np.ascontiguousarray(prob[k])).pin_memory() for k in keys}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    # A streaming pipeline, as a serving loop runs it: step k's host-to-device
    # copy, compute and device-to-host copy go on three streams, with the
    # device inputs and outputs double-buffered, so that the copies of steps
    # k + 1 and k - 1 overlap the compute of step k.  Every step still copies
    # its inputs in and its coefficients out inside the timed region.
    out_h = [[torch.empty((n_leaves, nc), dtype=torch.float64).pin_memory() for _ in layers] for _ in range(2)]
    d2h = sum(o.numel() * 8 for o in out_h[0])
    s_h2d, s_cmp, s_d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    plan = q.Plan(P, precision="fp64", stream=s_cmp)
    dbuf = [{k: torch.empty(v.shape, dtype=v.dtype, device=dev) for k, v in host.items()} for _ in range(2)]
    obuf = [[torch.empty((n_leaves, nc), dtype=torch.float64, device=dev) for _ in layers] for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]    # inputs of buffer b copied
    ev_cmp = [torch.cuda.Event() for _ in range(2)]   # compute on buffer b done
    ev_out = [torch.cuda.Event() for _ in range(2)]   # outputs of buffer b copied out
    used = [False, False]

    def e2e_step(k):
        b = k & 1
        if used[b]:
            s_h2d.wait_event(ev_cmp[b])  # step k - 2 has read these inputs
        with torch.cuda.stream(s_h2d):
            for key, v in host.items():
                dbuf[b][key].copy_(v, non_blocking=True)
            ev_in[b].record(s_h2d)
        s_cmp.wait_event(ev_in[b])
        if used[b]:
            s_cmp.wait_event(ev_out[b])  # step k - 2's outputs have been copied out
        g = dbuf[b]
        outs = {"coef_single": obuf[b][0]} if single else {}
        if double:
            outs["coef_double"] = obuf[b][1 if single else 0]
        cs, cd = plan.triangles(g["vxyz"], g["idx"], g["sigma"], g["leaf_off"], g["leaf_c"], g["leaf_rho"], None,
                                density=wl["density"], single=single, double=double, **outs)
        ev_cmp[b].record(s_cmp)
        s_d2h.wait_event(ev_cmp[b])
        with torch.cuda.stream(s_d2h):
            for o, c in zip(out_h[b], [c for c in (cs, cd) if c is not None]):
                o.copy_(c, non_blocking=True)
            ev_out[b].record(s_d2h)
        used[b] = True

    for k in range(args.warmup):
        e2e_step(k)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(s_cmp)
    s_h2d.wait_event(e0)
    s_d2h.wait_event(e0)
    for k in range(args.steps):
        e2e_step(args.warmup + k)
    for b in range(2):
        if used[b]:
            s_cmp.wait_event(ev_out[b])
    e1.record(s_cmp)
    torch.cuda.synchronize()
    t1 = time.time()
    if clk:
        clk.window("e2e", t0, t1)
    plan.sync()
    del plan
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
        dist.barrier()

    per_step = len(layers) * n_elem * nc
    total_moments = per_step
    if dist:
        t = torch.tensor([per_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_moments = float(t.item())
    value = total_moments / (r64["ms"] * 1e-3)
    flops_elem = element_flops("triangle", wl["density"], layers, P, point="order")  # FP64 kernel
    flops_elem32 = element_flops("triangle", wl["density"], layers, P)  # FP32 kernels: stencil on every level

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- CPU baseline: the oracle on a bounded sample, the GPU errors on it,
    # and the far-field accuracy of both coefficient sets
    cpu = None
    errs = {}
    eq = None
    if not args.no_cpu_baseline and world == 1:
        import oracle as orc
        n = calibrate_sample(orc, wl, prob, args.cpu_seconds)
        leaves = sample_leaves(prob, n)
        sub = sub_problem(prob, leaves)
        t0 = time.perf_counter()
        refs = oracle_run(orc, wl, sub)
        dt = time.perf_counter() - t0
        ne = sub["idx"].shape[1]
        cpu = {"value": len(layers) * ne * nc / dt, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
               "sample": "%d of %d triangles (%d whole leaves, seeded), %s layer, FP64 Gauss quadrature "
                         "(%d nodes/direction), OpenMP; %.1f s" % (ne, n_elem, len(leaves), "+".join(layers),
                                                                  (P + 5) // 2, dt)}
        # the same oracle on one core, on a sample sized for about a quarter of that time
        leaves1 = sample_leaves(prob, max(200, int(ne * min(1.0, 0.25 / max(orc.max_threads(), 1)))))
        sub1 = sub_problem(prob, leaves1)
        t0 = time.perf_counter()
        oracle_run(orc, wl, sub1, nthreads=1)
        dt1 = time.perf_counter() - t0
        ne1 = sub1["idx"].shape[1]
        cpu["single_core"] = {"value": len(layers) * ne1 * nc / dt1, "unit": UNIT, "cores": 1,
                              "sample": "%d triangles (%d whole leaves), %.1f s" % (ne1, len(leaves1), dt1)}
        for prec in ("fp64", "fp32"):
            errs[prec] = {}
            for li, ly in enumerate(layers):
                got = outs[prec][0 if ly == "single" else 1]
                errs[prec][ly] = norm_err(got[leaves], refs[li], prob["leaf_rho"][leaves], 0 if ly == "single" else 1,
                                          P)
        errs["sampled_leaves"] = int(len(leaves))
        errs["sampled_elements"] = int(ne)
        if single:
            eq_leaves, h, by_d = equal_accuracy(orc, prob, wl, outs["fp64"][0], outs["fp32"][0])
            # the FP64 degree that matches FP32-mixed at each distance, timed
            times = {}
            for f, rec in by_d.items():
                pe = rec["fp64_degree_equal"]
                if pe not in times:
                    times[pe] = r64["ms"] if pe == P else timed("fp64", p_eff=pe, keep=False)["ms"]
                rec["ms_fp64_at_that_degree"] = times[pe]
                rec["speedup_fp32_mixed_at_equal_accuracy"] = times[pe] / r32["ms"]
            eq = {"targets": "%d sampled leaves (>= 8 elements), 16 seeded directions at each distance d = f h from "
                             "the leaf centre (h = %.5f the leaf side); error = max |phi - phi_exact| / max "
                             "|phi_exact| over a leaf's targets, max over leaves; phi = series of Eq. (bas3) of the "
                             "leaf coefficients, phi_exact = oracle quadrature of the leaf's elements"
                             % (len(eq_leaves), h),
                  "by_distance": [by_d[f] for f in sorted(by_d)],
                  "speedup": min(rec["speedup_fp32_mixed_at_equal_accuracy"] for rec in by_d.values()),
                  "speedup_note": "minimum over the distances of t_fp64(p') / t_fp32_mixed(p), p' the smallest "
                                  "FP64 degree whose potential error is at most FP32-mixed's at p"}

    if clk:
        clk.stop()
    timed_windows = [w[0] for w in clk.windows] if clk else []
    clocks = clk.summary(timed_windows) if clk else None
    if clocks is not None:
        clocks["windows"] = clk.per_window()

    k64 = KERNEL_COUNTERS.get((args.config, "fp64"), {})
    k32 = KERNEL_COUNTERS.get((args.config, "fp32"), {})
    achieved64 = flops_elem * n_elem / (r64["kernel_ms"] * 1e-3)
    achieved32 = flops_elem32 * n_elem / (r32["kernel_ms"] * 1e-3)

    def executed(kc, kernel_ms, peak):
        if not kc.get("executed_flops"):
            return None
        return {"flops_per_launch": kc["executed_flops"],
                "frac": kc["executed_flops"] / (kernel_ms * 1e-3) / peak, "source": COUNTER_SOURCE}

    dname = "TRI,%s,%s" % (wl["density"].upper(), "+".join(layers))
    peak_src = ("measured in this run: q2x_alu_peak_probe, %s, %.2f s of 8 independent FMA chains per thread on "
                "every SM, CUDA events")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(wl, full) + (" per rank" if world > 1 else ""), "precision": "fp64",
                   "density": wl["density"], "layers": list(layers), "p": P, "n_elem": n_elem,
                   "moments_per_step": total_moments, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "leaf-sharded dp%d (no collective)" % world if world > 1 else "single GPU",
                   "step": "one CUDA-graph replay: leaf-offset check, element kernel, fix-up of split leaves"},
        "roofline": {"bound": "alu", "achieved": achieved64 / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                     "frac": achieved64 / peak64, "traffic": k64.get("traffic"),
                     "traffic_source": COUNTER_SOURCE if k64.get("traffic") else "not captured for this kernel",
                     "kernel": "q2x_elem_kernel<double,%d,%s>" % (P, dname), "kernel_ms": r64["kernel_ms"],
                     "flops_per_element": flops_elem, "flops_per_launch": flops_elem * n_elem,
                     "algorithmic_bytes_per_launch": None,
                     "executed": executed(k64, r64["kernel_ms"], peak64),
                     "peak_source": peak_src % ("DFMA", peaks["dfma"]["ms"] * 1e-3),
                     "peak_fp64_fallback": "recipe: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz = 1.26 TFLOP/s"},
        "fp32_mixed": {"value": total_moments / (r32["ms"] * 1e-3), "ms_per_step": r32["ms"],
                       "steps": r32["steps"], "speedup_vs_fp64": r64["ms"] / r32["ms"],
                       "roofline": {"bound": "alu", "achieved": achieved32 / 1e12, "peak": peak32 / 1e12,
                                    "unit": "TFLOP/s", "frac": achieved32 / peak32, "traffic": k32.get("traffic"),
                                    "kernel": ("q2x_batch_group_kernel<float,%d,%s> (leaf tiles)" % (P, dname)
                                               if tuple(layers) == ("single",) else
                                               "q2x_elem_kernel<float,%d,%s>" % (P, dname)),
                                    "kernel_ms": r32["kernel_ms"],
                                    "flops_per_element": flops_elem32, "flops_per_launch": flops_elem32 * n_elem,
                                    "executed": executed(k32, r32["kernel_ms"], peak32),
                                    "peak_source": peak_src % ("FFMA and packed FFMA2, the larger",
                                                               peaks["ffma"]["ms"] * 1e-3)}},
        "alu_peaks_measured": peaks,
        "speedup_at_equal_accuracy": eq,
        "errors_vs_oracle": errs or None,
        "cpu_baseline": cpu,
        "e2e": {"value": total_moments / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "pipeline": "each step copies its inputs from pinned host memory and its coefficients back; "
                            "the copies of neighbouring steps overlap this step's compute (three streams, "
                            "double-buffered device inputs and outputs)"},
        "gpu_launches": r64["launches"],
        "clocks": clocks,
    }
    # algorithmic bytes per launch: indices, densities, vertex coordinates read
    # once, leaf data, and the coefficients written
    alg_bytes = (prob["idx"].nbytes + prob["sigma"].nbytes + prob["vxyz"].nbytes + prob["leaf_off"].nbytes
                 + prob["leaf_c"].nbytes + prob["leaf_rho"].nbytes + len(layers) * n_leaves * nc * 8)
    line["roofline"]["algorithmic_bytes_per_launch"] = alg_bytes
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
