"""Measurements of the non-headline workloads (run through `bench.py --config`):

  icosphere-L3      1280 triangles of the level-3 icosphere, one expansion
                    about the origin, p = 10, FP64 (latency-bound)
  mixed-ball        2M filament segments + 4M sphere triangles + 1M tetrahedra
                    in the unit ball, adaptive octree (<= 2000 per leaf),
                    p_leaf ~ U{8..20}: one CUDA-graph replay of the batch (FP32)
  sphere-L8-adjoint 1M triangles of the perturbed level-8 sphere, depth 6,
                    p = 12: FP32-mixed forward + adjoint (FP64 accumulation)

Each prints one JSON line in the format of bench.py's (metric counted per
output layer as elements x (p+1)^2, or sum over leaves of elements x
(p_leaf+1)^2 for the ragged batch).  Errors against the FP64 oracle are
measured on a few sampled leaves."""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

import workloads as W
from bench import METRIC, UNIT, ClockSampler, L2_FLUSH_BYTES

LINES = []
# filled by run(): measured FP64 / FP32 FMA peaks (flop/s) of this device
PEAKS = {}
PEAK_SOURCE = "measured in this run (q2x_alu_peak_probe, FMA chains on every SM, CUDA events)"


def _norm_err(test, ref, rho, p, layer=0):
    worst = 0.0
    for L in range(ref.shape[0]):
        s = np.zeros((p + 1) ** 2)
        for n in range(p + 1):
            for m in range(-n, n + 1):
                f = math.sqrt(math.factorial(n + abs(m)) * math.factorial(n - abs(m)))
                s[n * n + n + m] = f / rho[L] ** n
        den = np.max(np.abs(ref[L] * s))
        worst = max(worst, np.max(np.abs((test[L] - ref[L]) * s)) / den if den > 0 else 0.0)
    return worst


CLOCKS = {}


def _time(fn, steps, warmup, flush, stream):
    for _ in range(warmup):
        flush.fill_(1.0)
        fn()
    torch.cuda.synchronize()
    clk = ClockSampler()
    clk.start()
    ms = []
    t0 = time.time()
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ms.append((a, b))
    torch.cuda.synchronize()
    clk.window("timed", t0, time.time())
    clk.stop()
    CLOCKS.update(clk.summary())
    return sum(x.elapsed_time(y) for x, y in ms) / steps


def _emit(line):
    line["clocks"] = dict(CLOCKS)
    line["config"]["l2"] = "flushed between timed steps (256 MiB write)"
    print(json.dumps(line), flush=True)


def run_mixed_ball(args, dev):
    import paper_2107_10942_gb300 as q
    m = W.cfg_mixed_ball()
    kinds = {}
    names = {"segment": "segments", "triangle": "triangles", "tetra": "tetra"}
    for k, dd in m["kinds"].items():
        kinds[names[k]] = {key: torch.from_numpy(v).to(dev) for key, v in dd.items()}
    lc, lr, lp = (torch.from_numpy(m[k]).to(dev) for k in ("leaf_c", "leaf_rho", "leaf_p"))
    plan = q.Plan(m["p"], precision="fp32")
    tile = q.q2x.autotuned_tile(plan, "mixed-ball-%d" % m["leaf_c"].shape[1],
                                __import__("os").path.join(__import__("tempfile").gettempdir(), "q2x_autotune.json"),
                                candidates=(128, 256, 512, 1024, 2048), reps=3, leaf_c=lc, leaf_rho=lr, leaf_p=lp,
                                **kinds)
    b = q.q2x.Batch(plan, lc, lr, lp, tile_elems=tile, **kinds)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ms = _time(b.run, args.steps, args.warmup, flush, stream)
    got = b.coef.cpu().numpy()
    plan.sync()
    lpn = m["leaf_p"].astype(np.int64)
    n_per_leaf = sum(np.diff(dd["leaf_off"]) for dd in m["kinds"].values())
    per_step = int(np.sum(n_per_leaf * (lpn + 1) ** 2))
    # oracle on 8 sampled leaves of 8..400 elements (bounded oracle time)
    import oracle as orc
    cand = np.nonzero((n_per_leaf >= 8) & (n_per_leaf <= 400))[0]
    pick = np.sort(np.random.default_rng(4).choice(cand, size=min(8, len(cand)), replace=False))
    t0 = time.perf_counter()
    ref = np.zeros((len(pick), (m["p"] + 1) ** 2))
    for i, L in enumerate(pick):
        for k, dd in m["kinds"].items():
            o = dd["leaf_off"]
            if o[L + 1] > o[L]:
                idx = np.ascontiguousarray(dd["idx"][:, o[L]:o[L + 1]])
                ref[i] += orc.moments(k, dd["vxyz"], idx, dd["sigma"][o[L]:o[L + 1]], m["p"],
                                      leaf_off=np.array([0, idx.shape[1]]), leaf_c=m["leaf_c"][:, L:L + 1],
                                      leaf_p=m["leaf_p"][L:L + 1])[0]
    dt = time.perf_counter() - t0
    err = _norm_err(got[pick], ref, m["leaf_rho"][pick], m["p"])
    info = b.info()
    from paper_2107_10942_gb300.roofline import element_flops
    kind_flops = {"segment": ("segment", "const"), "triangle": ("triangle", "const"), "tetra": ("tetra", "const")}
    flops = 0.0
    for k, dd in m["kinds"].items():
        cnt = np.diff(dd["leaf_off"])
        per_p = {pp: element_flops(kind_flops[k][0], kind_flops[k][1], ("single",), int(pp))
                 for pp in np.unique(lpn)}
        flops += float(sum(cnt[lpn == pp].sum() * f for pp, f in per_p.items()))
    _emit({"metric": METRIC, "value": per_step / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32-mixed",
           "data": "synthetic",
           "config": {"workload": "mixed-ball: %d segments + %d triangles + %d tetrahedra, %d adaptive leaves, "
                                  "p_leaf in 8..20" % tuple([m["kinds"][k]["idx"].shape[1] for k in
                                                              ("segment", "triangle", "tetra")] +
                                                             [m["leaf_c"].shape[1]]),
                      "tiles": info["tiles"], "tile_elems": info["tile_elems"],
                      "launch": "one CUDA-graph replay (counter reset, one persistent kernel per (kind, degree "
                                "bin) group of tiles on four parallel branches, combine)"},
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": PEAKS["fp32"] / 1e12,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / PEAKS["fp32"],
                        "note": "whole graph replay (reset + persistent kernel + combine) as the duration"},
           "errors_vs_oracle": {"fp32": err, "sampled_leaves": len(pick)},
           "cpu_baseline": {"value": float(np.sum(n_per_leaf[pick] * (lpn[pick] + 1) ** 2)) / dt, "unit": UNIT,
                            "kind": "oracle", "cores": orc.max_threads(), "sample": "8 leaves"}})


def run_adjoint(args, dev):
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.q2x import problem_to_device
    prob = W.cfg_sphere_adjoint(level=8, n_tri=1_000_000, depth=6, p=12)
    d = problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")}, dev)
    p = 12
    n_elem = prob["idx"].shape[1]
    plan = q.Plan(p, precision="fp32")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    vx = d["vxyz"].clone().requires_grad_(True)
    sg = d["sigma"].clone().requires_grad_(True)

    def step():
        coef = q.q2x.triangles_single(vx, sg, plan, d["idx"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)
        loss = torch.sum(coef * d["G"])
        return torch.autograd.grad(loss, (vx, sg))

    ms = _time(step, args.steps, args.warmup, flush, stream)
    gv32, gs32 = (t.cpu().numpy() for t in step())
    plan64 = q.Plan(p, precision="fp64")
    gv64, gs64 = plan64.triangles_single_vjp(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["G"],
                                             d["leaf_rho"], None)
    gv64, gs64 = gv64.cpu().numpy(), gs64.cpu().numpy()
    rel_v = float(np.max(np.abs(gv32 - gv64)) / np.max(np.abs(gv64)))
    rel_s = float(np.max(np.abs(gs32 - gs64)) / np.max(np.abs(gs64)))
    per_step = n_elem * (p + 1) ** 2
    from paper_2107_10942_gb300.roofline import element_flops, vjp_flops
    flops = float(element_flops("triangle", "const", ("single",), p) + vjp_flops(p)) * n_elem
    _emit({"metric": METRIC + " (forward + adjoint)", "value": per_step / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "dtype": "f32-mixed forward, f32 per element + f64 accumulation backward", "data": "synthetic",
           "config": {"workload": "sphere-L8-adjoint: %d triangles, depth 6, p=12, single layer, "
                                  "loss = sum(G * coef), G ~ N(0,1)" % n_elem},
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": PEAKS["fp32"] / 1e12,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / PEAKS["fp32"],
                        "flops_per_element": flops / n_elem,
                        "note": "whole step (forward kernel + adjoint kernels + autograd glue) against the FP32 peak"},
           "errors_vs_fp64_adjoint": {"grad_vertices": rel_v, "grad_sigma": rel_s}})


def run_icosphere_l3(args, dev):
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.q2x import problem_to_device
    import oracle as orc
    prob = W.cfg_icosphere_l3(p=10)
    d = to_dev(prob, dev)
    p = 10
    n_elem = prob["idx"].shape[1]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    plan = q.Plan(p, precision="fp64")
    coef = torch.empty((1, (p + 1) ** 2), dtype=torch.float64, device=dev)
    fn = lambda: plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                                coef_single=coef)
    # the step (check, element kernel, fix-up) as one CUDA graph, so that host
    # launch gaps do not enter the device time of this small problem
    g = plan.capture(fn)
    ms = _time(g.replay, args.steps, args.warmup, flush, stream)
    plan.set_kernel_timing(True)
    plan.kernel_timing()
    _time(fn, args.steps, 0, flush, stream)
    kms, kn = plan.kernel_timing()
    plan.set_kernel_timing(False)
    got = coef.cpu().numpy()
    plan.sync()
    t0 = time.perf_counter()
    reps = 0
    while True:
        ref = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], p, leaf_off=prob["leaf_off"],
                          leaf_c=prob["leaf_c"])
        reps += 1
        if time.perf_counter() - t0 > 2.0:
            break
    dt = (time.perf_counter() - t0) / reps
    per_step = n_elem * (p + 1) ** 2
    _emit({"metric": METRIC, "value": per_step / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "icosphere-L3: %d triangles, one expansion about the origin, p=10, single layer, "
                                  "constant density" % n_elem,
                      "step": "one CUDA-graph replay (check, element kernel, fix-up)", "kernel_ms": kms / max(kn, 1),
                      "note": "latency-bound: 40 warps of 32 triangles, one per SM sub-partition; each runs its "
                              "round's FP64 chain alone on its sub-partition's FP64 pipe (about 2,000 FP64 "
                              "instructions of 64 pipe cycles each), so the kernel cannot take less than about "
                              "0.06 ms however many SMs are idle"},
           "errors_vs_oracle": {"fp64": _norm_err(got, ref, prob["leaf_rho"], p)},
           "cpu_baseline": {"value": per_step / dt, "unit": UNIT, "kind": "oracle", "cores": orc.max_threads(),
                            "sample": "the whole workload, %d repetitions" % reps}})


def translate_macs(p):
    """complex multiply-adds of one translation of degree p (COEFF formula)"""
    t = 0
    for n in range(p + 1):
        for m in range(n + 1):
            for k in range(n + 1):
                nn = n - k
                t += max(0, min(k, nn - m) - max(-k, -nn - m) + 1)
    return t


def run_upward(args, dev):
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.upward import Upward
    import oracle as orc
    p, depth = 12, 5
    prob = W.cfg_sphere_linear(level=7, depth=depth, p=p)
    d = to_dev(prob, dev)
    plan = q.Plan(p, precision="fp64")
    leaf, _ = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                             density="linear")
    up = Upward(plan, d["leaf_c"], -1.125, 2.25, depth)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    # the pass as one CUDA graph (five levels, ten kernels, one host launch)
    up.capture(leaf)
    ms = _time(up.replay, args.steps, args.warmup, flush, stream)
    outs = up.replay()
    root = outs[-1].cpu().numpy()
    plan.sync()
    n_tr = sum(int(lv["dst_off"][-1]) for lv in up.levels)
    flops = 8.0 * translate_macs(p) * n_tr
    # the root against quadrature of the whole sphere about the cube centre
    t0 = time.perf_counter()
    ref = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], p,
                      leaf_off=np.array([0, prob["idx"].shape[1]]), leaf_c=np.zeros((3, 1)), density=1)
    dt = time.perf_counter() - t0
    rho = np.max(np.linalg.norm(prob["vxyz"], axis=0))
    err = _norm_err(root, ref, np.array([rho]), p)
    _emit({"metric": "M2M translations/s (upward pass of the leaf coefficients)", "value": n_tr / (ms * 1e-3),
           "unit": "translations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "upward pass of the level-7 sphere's depth-5 leaves (%d leaves, %d translations, "
                                  "5 levels, one CUDA graph replay), p=12, FP64" % (prob["leaf_c"].shape[1], n_tr)},
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": PEAKS["fp64"] / 1e12,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / PEAKS["fp64"],
                        "flops_per_translation": 8 * translate_macs(p)},
           "errors_vs_oracle": {"root_vs_quadrature": err},
           "cpu_baseline": {"value": None, "note": "oracle quadrature of the root expansion over all %d triangles: "
                            "%.2f s" % (prob["idx"].shape[1], dt), "kind": "oracle", "cores": orc.max_threads()}})


# FP64 flops per evaluation ncu counted as executed at p = 12:
# (2 x 104.19 + 13.57 + 137.94) per elapsed cycle x 2.858 M cycles / 1,048,576
EVAL_EXECUTED_FLOPS = (2 * 104.187417 + 13.573713 + 137.938271) * 2858268.0 / 1048576


def eval_flops(p):
    """Flops of one far-field evaluation (q2x_evaluate): per (n, m >= 0)
    term a three-term step (3 multiplies, 1 FMA) and two FMAs = 9 flops; per
    order m the update of T_m^m and the column's complex product (about 16)."""
    return 9 * (p + 1) * (p + 2) // 2 + 16 * (p + 1)


def run_farfield(args, dev):
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.upward import Upward
    import oracle as orc
    p, depth, n_tgt = 12, 5, 1 << 20
    prob = W.cfg_sphere_linear(level=7, depth=depth, p=p)
    d = to_dev(prob, dev)
    plan = q.Plan(p, precision="fp64")
    leaf, _ = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                             density="linear")
    root = Upward(plan, d["leaf_c"], -1.125, 2.25, depth).run(leaf)[-1]
    rng = np.random.default_rng(17)
    tg = rng.normal(size=(3, n_tgt))
    tg = 3.0 * tg / np.linalg.norm(tg, axis=0)
    tgt = torch.from_numpy(tg).to(dev)
    centre = torch.zeros((3, 1), dtype=torch.float64, device=dev)
    out = torch.empty(n_tgt, dtype=torch.float64, device=dev)
    off = torch.arange(n_tgt + 1, dtype=torch.int64, device=dev)
    idx = torch.zeros(n_tgt, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ms = _time(lambda: plan.evaluate(root, centre, tgt, off, idx, out=out), args.steps, args.warmup, flush, stream)
    got = out.cpu().numpy()
    rc = root.cpu().numpy()[0]
    plan.sync()
    pick = rng.choice(n_tgt, 64, replace=False)
    ref = orc.farfield(rc, np.zeros(3), tg[:, pick].T, p)[0]
    err = float(np.max(np.abs(got[pick] - ref)) / np.max(np.abs(ref)))
    flops = float(eval_flops(p)) * n_tgt
    _emit({"metric": "far-field evaluations/s (one p=12 expansion per target)", "value": n_tgt / (ms * 1e-3),
           "unit": "evaluations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "root expansion of the level-7 sphere (p=12, from Q2X + upward pass) at %d targets "
                                  "on the radius-3 sphere" % n_tgt},
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": PEAKS["fp64"] / 1e12,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / PEAKS["fp64"],
                        "flops_per_evaluation": eval_flops(p),
                        "executed": {"flops_per_evaluation": EVAL_EXECUTED_FLOPS,
                                     "frac": EVAL_EXECUTED_FLOPS * n_tgt / (ms * 1e-3) / PEAKS["fp64"],
                                     "source": "ncu DFMA/DADD/DMUL counts of one capture of this "
                                               "kernel on this workload"}},
           "errors_vs_oracle": {"series": err, "sampled_targets": 64}})


def run_galerkin(args, dev):
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.roofline import element_flops
    import oracle as orc
    p, depth = 12, 5
    prob = W.cfg_sphere_linear(level=7, depth=depth, p=p)
    d = to_dev(prob, dev)
    nl = prob["leaf_c"].shape[1]
    n_elem = prob["idx"].shape[1]
    w = torch.from_numpy(np.random.default_rng(21).standard_normal((nl, (p + 1) ** 2))).to(dev)
    ones = torch.ones(n_elem, dtype=torch.float64, device=dev)
    out = torch.empty(n_elem, dtype=torch.float64, device=dev)
    plan = q.Plan(p, norm="moment", precision="fp64")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    run = lambda: plan.galerkin_triangles(d["vxyz"], d["idx"], w, d["leaf_off"], d["leaf_c"], d["leaf_rho"],
                                          sigma=ones, layer=0, out=out)
    ms = _time(run, args.steps, args.warmup, flush, stream)
    got = out.cpu().numpy()
    plan.sync()
    # sampled elements against the oracle's per-element moments contracted with w
    rng = np.random.default_rng(22)
    el = np.sort(rng.choice(n_elem, 200, replace=False))
    leaf_of = np.repeat(np.arange(nl), np.diff(prob["leaf_off"]))
    P = orc.moments("triangle", prob["vxyz"], np.ascontiguousarray(prob["idx"][:, el]), np.ones(len(el)), p,
                    leaf_off=None, leaf_c=np.ascontiguousarray(prob["leaf_c"][:, leaf_of[el]]), norm=1)
    wn = w.cpu().numpy()
    ref = np.sum(P * wn[leaf_of[el]], axis=1)
    err = float(np.max(np.abs(got[el] - ref) / np.sum(np.abs(P * wn[leaf_of[el]]), axis=1)))
    flops = (element_flops("triangle", "const", ("single",), p, point="order") + (p + 1) ** 2) * n_elem
    _emit({"metric": "Galerkin element integrals/s (local expansion over each receiving triangle)",
           "value": n_elem / (ms * 1e-3), "unit": "elements/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "the level-7 sphere's %d triangles against random local expansions of its %d "
                                  "depth-5 leaves, p=12, single layer" % (n_elem, nl)},
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": PEAKS["fp64"] / 1e12,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / PEAKS["fp64"]},
           "errors_vs_oracle": {"relative_to_sum_of_terms": err, "sampled_elements": 200}})


def run_biot_savart(args, dev):
    import paper_2107_10942_gb300 as q
    from paper_2107_10942_gb300.roofline import level_flops, point_level_order_flops
    from paper_2107_10942_gb300.upward import Upward
    p = 12
    m = W.cfg_mixed_ball()
    sg = m["kinds"]["segment"]
    vx, idx = sg["vxyz"], sg["idx"]
    # vortex-filament currents: strength sigma along each segment's direction
    tang = vx[:, idx[1]] - vx[:, idx[0]]
    cur = sg["sigma"] * tang / np.linalg.norm(tang, axis=0)
    n_elem = idx.shape[1]
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(vxyz=vx, idx=idx, cur=cur, leaf_off=sg["leaf_off"], leaf_c=m["leaf_c"], leaf_rho=m["leaf_rho"]).items()}
    plan = q.Plan(p, precision="fp64")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ms_q2x = _time(lambda: plan.segments_vector(d["vxyz"], d["idx"], d["cur"], d["leaf_off"], d["leaf_c"],
                                                d["leaf_rho"]), args.steps, args.warmup, flush, stream)
    c3 = plan.segments_vector(d["vxyz"], d["idx"], d["cur"], d["leaf_off"], d["leaf_c"], d["leaf_rho"])
    up = Upward(plan, m["leaf_c"], -1.0, 2.0, m["leaf_depth"])
    root3 = torch.stack([up.run(c3[k].contiguous())[-1] for k in range(3)]).contiguous()
    n_tgt = 1 << 18
    tg = np.random.default_rng(5).normal(size=(3, n_tgt))
    tgt = torch.from_numpy(2.0 * tg / np.linalg.norm(tg, axis=0)).to(dev)
    centre = torch.zeros((3, 1), dtype=torch.float64, device=dev)
    off = torch.arange(n_tgt + 1, dtype=torch.int64, device=dev)
    eidx = torch.zeros(n_tgt, dtype=torch.int64, device=dev)
    H = torch.empty((3, n_tgt), dtype=torch.float64, device=dev)
    ms_curl = _time(lambda: plan.evaluate_curl(root3, centre, tgt, off, eidx, out=H), args.steps, args.warmup,
                    flush, stream)
    plan.sync()
    per_step = 3 * n_elem * (p + 1) ** 2
    # one recursion (the segment chain's two levels) and three weighted sums (one FMA per column each)
    flops = (point_level_order_flops(p) + level_flops(p) + 3 * 2 * (p + 1) ** 2) * n_elem
    _emit({"metric": "vector line-density Q2X element-moments/s (three components, Eq. st3)",
           "value": per_step / (ms_q2x * 1e-3), "unit": "element-moments/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_q2x, "higher_is_better": True, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "the mixed ball's %d filament segments with vortex currents along them, %d "
                                  "adaptive leaves, p=12 (one recursion pass for the three components)" % (n_elem,
                                                                                           m["leaf_c"].shape[1])},
           "roofline": {"bound": "alu", "achieved": flops / (ms_q2x * 1e-3) / 1e12,
                        "peak": PEAKS["fp64"] / 1e12, "unit": "TFLOP/s",
                        "frac": flops / (ms_q2x * 1e-3) / PEAKS["fp64"]},
           "curl_evaluation": {"targets": n_tgt, "ms": ms_curl, "value": n_tgt / (ms_curl * 1e-3),
                               "unit": "H evaluations/s (root expansion, p=12, radius 2)"}})


def measured_hbm_gbs():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def run_leaf_reduce(args, dev):
    import paper_2107_10942_gb300 as q
    p = 12
    prob = W.cfg_sphere_linear(level=7, depth=5, p=p)
    n_elem, nl = prob["idx"].shape[1], prob["leaf_c"].shape[1]
    np_ = (p + 1) ** 2
    gen = torch.Generator(device=dev).manual_seed(3)
    elem = torch.randn((n_elem, np_), dtype=torch.float64, device=dev, generator=gen)
    off = torch.from_numpy(prob["leaf_off"]).to(dev)
    out = torch.empty((nl, np_), dtype=torch.float64, device=dev)
    plan = q.Plan(p, precision="fp64")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ms = _time(lambda: plan.leaf_reduce(elem, p, off, coef=out), args.steps, args.warmup, flush, stream)
    plan.sync()
    # exact check on sampled leaves (same order of summation as a plain loop)
    e_np = elem.cpu().numpy()
    o_np = out.cpu().numpy()
    rng = np.random.default_rng(4)
    err = 0.0
    for L in rng.choice(nl, 20, replace=False):
        ref = np.zeros(np_)
        for e in range(prob["leaf_off"][L], prob["leaf_off"][L + 1]):
            ref += e_np[e]
        err = max(err, float(np.max(np.abs(o_np[L] - ref))))
    bytes_ = 8.0 * np_ * (n_elem + nl)
    peak, src = measured_hbm_gbs()
    gbs = bytes_ / (ms * 1e-3) / 1e9
    _emit({"metric": "segmented leaf reduce (q2x_leaf_reduce) bandwidth", "value": gbs, "unit": "GB/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "%d per-element rows of (p+1)^2 = %d FP64 into the level-7 sphere's %d leaves"
                                  % (n_elem, np_, nl)},
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "peak_source": src, "bytes_per_launch": bytes_,
                        "traffic": 444732928 + 6349568,
                        "traffic_source": "ncu dram__bytes_read/write of one capture of this kernel on this "
                                          "workload"},
           "errors_vs_oracle": {"max_abs_vs_sequential_sum": err, "sampled_leaves": 20}})


# FP64 operations per (target, triangle) pair as the near-field kernel
# evaluates the closed form from a precomputed face frame: frame coordinates
# and height (about 20), three vertex distances (9), three edges of about 17
# (edge coordinates, the log's argument), the solid angle's denominator (13),
# the sums (2), and each of the 3 sqrt, 3 divisions, 3 log1p and 1 atan2
# counted as one
NEARFIELD_OPS_PER_PAIR = 20 + 9 + 3 * 17 + 13 + 2 + 3 + 3 + 3 + 1
# FP64 flops per pair ncu counted as executed (2 x DFMA + DADD + DMUL thread
# instructions, library sequences of sqrt, division, log1p and atan2 included):
# (2 x 92.31 + 33.24 + 37.07) per elapsed cycle x 59.66 M cycles / 39.54 M pairs
NEARFIELD_EXECUTED_FLOPS_PER_PAIR = (2 * 92.309745 + 33.237194 + 37.074234) * 59656234.0 / 39541618


def run_nearfield(args, dev):
    import paper_2107_10942_gb300 as q
    from oracle import nearfield as onf
    p = 12
    prob = W.cfg_sphere_linear(level=7, depth=5, p=p)
    vx, idx, off = prob["vxyz"], prob["idx"], prob["leaf_off"]
    n_elem, nl = idx.shape[1], prob["leaf_c"].shape[1]
    sig = prob["sigma"][idx].mean(axis=0)  # a constant density per triangle
    tgt = np.ascontiguousarray(vx[:, idx].mean(axis=1))  # collocation points: the centroids
    cnt = np.diff(off)
    leaf_of = np.repeat(np.arange(nl), cnt)
    tgt_off = np.concatenate([[0], np.cumsum(cnt[leaf_of])]).astype(np.int64)
    # target t lists every triangle of its own leaf
    first = off[leaf_of]
    rep = np.repeat(np.arange(n_elem), cnt[leaf_of])
    elem_idx = (first[rep] + (np.arange(tgt_off[-1]) - tgt_off[rep])).astype(np.int64)
    pairs = int(tgt_off[-1])
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
         for k, v in dict(vxyz=vx, idx=idx, sigma=sig, tgt=tgt, tgt_off=tgt_off, elem_idx=elem_idx).items()}
    out = torch.empty(n_elem, dtype=torch.float64, device=dev)
    plan = q.Plan(p, precision="fp64")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    run = lambda: plan.nearfield("triangle", d["vxyz"], d["idx"], d["sigma"], d["tgt"], d["tgt_off"], d["elem_idx"],
                                 out=out)
    ms = _time(run, args.steps, args.warmup, flush, stream)
    got = out.cpu().numpy()
    plan.sync()
    rng = np.random.default_rng(31)
    pick = rng.choice(n_elem, 12, replace=False)
    lists = [range(off[leaf_of[t]], off[leaf_of[t] + 1]) for t in pick]
    ref = onf.potentials("triangle", vx, idx, sig, tgt[:, pick], lists)
    err = float(np.max(np.abs(got[pick] - ref)) / np.max(np.abs(ref)))
    ops = NEARFIELD_OPS_PER_PAIR * pairs
    _emit({"metric": "near-field element potentials/s (exact triangle integrals, Sec. 4.1)",
           "value": pairs / (ms * 1e-3), "unit": "target-element pairs/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "collocation at the centroids of the level-7 sphere's %d triangles, each against "
                                  "every triangle of its depth-5 leaf: %d pairs, single layer" % (n_elem, pairs)},
           "roofline": {"bound": "alu", "achieved": ops / (ms * 1e-3) / 1e12, "peak": PEAKS["fp64"] / 1e12,
                        "unit": "TFLOP/s", "frac": ops / (ms * 1e-3) / PEAKS["fp64"],
                        "ops_per_pair": NEARFIELD_OPS_PER_PAIR,
                        "note": "sqrt, division, log and atan2 count as one operation each: a lower bound",
                        "executed": {"flops_per_pair": NEARFIELD_EXECUTED_FLOPS_PER_PAIR,
                                     "frac": NEARFIELD_EXECUTED_FLOPS_PER_PAIR * pairs / (ms * 1e-3)
                                     / PEAKS["fp64"],
                                     "source": "ncu DFMA/DADD/DMUL counts of one capture of this "
                                               "kernel on this workload"}},
           "errors_vs_oracle": {"graded_quadrature": err, "sampled_targets": len(pick)}})


def to_dev(prob, dev):
    from paper_2107_10942_gb300.q2x import problem_to_device
    return problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")}, dev)


def run(args):
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2107_10942_gb300 import build
    build.build()
    # ALU peaks of this device, measured in this run (the roofline denominators)
    from bench import measure_alu_peaks
    pk = measure_alu_peaks(dev, 0.5)
    PEAKS["fp64"] = pk["dfma"]["tflops"] * 1e12
    PEAKS["fp32"] = max(pk["ffma"]["tflops"], pk["ffma2"]["tflops"]) * 1e12
    PEAKS["measured"] = pk
    {"icosphere-L3": run_icosphere_l3, "upward": run_upward,
     "far-field": run_farfield, "galerkin": run_galerkin, "biot-savart": run_biot_savart,
     "leaf-reduce": run_leaf_reduce, "near-field": run_nearfield, "mixed-ball": run_mixed_ball,
     "sphere-L8-adjoint": run_adjoint}[args.config](args, dev)
