"""Benchmark of the solid-angle labeling hot path on GB300.

One step = one zef_label_points call over the whole workload (binning, exact
bounding-box and hull culling, FP32 cap-tree kernel, FP64 re-evaluation,
priority resolve), inputs resident in HBM.  Default workload: the full-scale
synthetic head -- 24 compartments (scalp, skull, CSF, grey and white matter
surfaces plus 19 subcortical structures, 1,526,588 triangles) against the
56,197,120 tet centroids of a 1 mm lattice over a 224 mm cube.  The
three-layer head on a 2 mm lattice (5 M centroids) and the 20 deep
structures on a 1 mm lattice (20.5 M centroids, one persistent batched launch
with autotuned tiles) are measured after it as secondary keys.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on bounded samples of the same workload instead.  Under torchrun (N > 1) the
points of the one workload are split into contiguous equal-work ranges of
their Morton order, one range per rank; `--replicas` makes every rank label
the whole workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point×triangle solid-angle pairs/s on 1 GB300, FP32+rescue vs FP64; labels=oracle"
# Algorithmic FP32 work of one point x triangle pair of the Van Oosterom-Strackee
# formula as written (FMA = 2 flops): R_k 9, three norms 18 (incl. sqrt), triple
# product 14, denominator 23, atan2 20 (division, degree-7 minimax, reflections),
# accumulation 1.
FLOPS_PER_PAIR = 85
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0
L2_NOTE = "flushed between steps (256 MB device write inside the timed region)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--extra-configs", default="1,2,ary",
                    help="secondary workloads measured after the headline (comma list, '' for none)")
    ap.add_argument("--points", type=int, default=0, help="limit points (0 = full workload)")
    ap.add_argument("--omega-points", type=int, default=200_000,
                    help="sample size of the FP32-sum accuracy check (0 = skip)")
    ap.add_argument("--fp64-points", type=int, default=100_000,
                    help="points of the FP32+rescue vs plain-FP64 comparison")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample points (0 = auto)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timing")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-refine", action="store_true", help="skip the refine-and-relabel measurement")
    ap.add_argument("--no-compare", action="store_true", help="skip the tile-coherence-off comparison step")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: every rank labels the whole workload (weak scaling by replicas)")
    ap.add_argument("--shape", default="", help="threads,ppt override")
    ap.add_argument("--kernel", type=int, default=0,
                    help="FP32 kernel form (0 cap trees, 1 strips with grouped products, 2 strips per triangle)")
    return ap.parse_args()


def workload(cfg, limit: int):
    import zef_synth as zs
    if cfg not in (0, 1, 2, 4, "ary"):
        raise SystemExit("bench workloads: configs 0, 1, 2, 4 and ary")
    w = zs.ary_spheres() if cfg == "ary" else zs.make_config(cfg)
    if limit and w.points.shape[0] > limit:
        # a centred window of the lattice order: the middle z-layers, where
        # every compartment's bounding box is crossed
        c = w.points.shape[0] // 2
        w.points = np.ascontiguousarray(w.points[c - limit // 2: c - limit // 2 + limit])
    return w


def config_dict(w, n_points):
    return {"workload": w.name, "points": int(n_points), "triangles": int(w.total_tris),
            "compartments": len(w.surfaces), "l2": L2_NOTE}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "sm_min_mhz": float(min(sm)) if sm else None,
                "power_w_median": float(np.median(pw)) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle arm
def cpu_oracle_rate(w, sample: int, seed: int = 3):
    """Oracle pairs/s on a seeded sample of the workload (all host cores)."""
    import oracle
    import zef_synth as zs
    oracle.build()
    idx = zs.sample_rows(w.points, sample, seed=seed)
    pts = w.points[idx]
    t0 = time.perf_counter()
    oracle.label_points(pts, w.surfaces, w.priority)
    dt = time.perf_counter() - t0
    pairs = len(pts) * w.total_tris
    return pairs / dt, dt, len(pts), oracle.max_threads()


def auto_sample(w, target_s: float):
    """Size the oracle sample for about target_s seconds of CPU work."""
    probe = max(64, int(2e8 / w.total_tris))
    rate, dt, n, _ = cpu_oracle_rate(w, probe, seed=1)
    return int(max(64, min(len(w.points), rate * target_s / w.total_tris)))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.config, args.points)
    sample = args.cpu_sample or auto_sample(w, 5.0)
    times = []
    cores = 0
    for k in range(args.warmup + args.steps):
        rate, dt, n, cores = cpu_oracle_rate(w, sample, seed=100 + k)
        if k >= args.warmup:
            times.append(dt)
    T = float(np.sum(times))
    value = sample * w.total_tris * args.steps / T
    ms_step = 1e3 * T / args.steps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, w.points.shape[0]),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} seeded points of the workload per step (a new seed each "
                                       f"step), all {w.total_tris} triangles each, no culling"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def make_context(zef, w, device):
    ctx = zef.Context(device)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(w.priority)
    return ctx


def timed_steps(torch, ctx, pts, labels, opts, steps, warmup, flush, stream, barrier, sampler=None):
    """W untimed calls, then K calls bracketed by a barrier + synchronize on
    both sides, an L2 flush before each, CUDA events on the context's stream
    (torch's current stream).  Returns the timing dict."""
    st = None
    for _ in range(max(3, warmup)):
        _, _, st = ctx.label_points(pts, labels=labels, opts=opts, stats=True)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(1.0)      # let nvidia-smi attach before the timed region
    ms_label, ms_rescue, launches = [], [], 0
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    e0.record(stream)
    for k in range(steps):
        flush.fill_(1)
        ev[k].record(stream)
        _, _, s2 = ctx.label_points(pts, labels=labels, opts=opts, stats=True)
        ms_label.append(s2["ms_label"])
        ms_rescue.append(s2["ms_rescue"])
        launches += s2["kernel_launches"]
    ev[steps].record(stream)
    e1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    return {"ms": e0.elapsed_time(e1), "step_ms": [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)],
            "ms_label": float(np.mean(ms_label)), "ms_rescue": float(np.mean(ms_rescue)),
            "launches": launches, "stats": st, "clocks": clocks}


def fp32_peak_tflops(torch, dev):
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms, sms * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12


def roofline(st, ms_label, peak, sms, clocks=None, traffic=None):
    fp32_pairs = st["pairs_evaluated"] - st["pairs_rescued"]
    achieved = fp32_pairs * FLOPS_PER_PAIR / (ms_label * 1e-3) / 1e12
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
         "traffic": traffic, "kernel": f"k_label32<{st['block_threads']}, {st['points_per_thread']}, 2>",
         "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {MAX_SM_MHZ:.0f} MHz (max clock), computed",
         "flops_per_pair": FLOPS_PER_PAIR, "fp32_pairs_per_launch": fp32_pairs,
         "ms_per_launch": ms_label}
    if clocks and clocks.get("sm_mhz"):
        r["frac_at_sampled_clock"] = achieved / (sms * 256 * clocks["sm_mhz"] * 1e6 / 1e12)
    try:   # the median SM clock of the driver's sustained GEMM loop (power-capped), for reference
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["clocks_under_load"]["sm_mhz_median"])
        r["frac_at_measured_under_load_clock"] = achieved / (sms * 256 * mhz * 1e6 / 1e12)
        r["measured_under_load_mhz"] = mhz
    except Exception:
        pass
    return r


def traffic_record(cfg, st, kernel):
    """DRAM bytes of one launch of the label kernel from an ncu capture, used
    only while the kernel source and the launch shape are the captured ones."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return None
    try:
        recs = json.load(open(tpath)).get(f"config{cfg}") or []
        if isinstance(recs, dict):
            recs = [recs]
        src = os.path.join(ROOT, "paper_2203_10000_gb300", "csrc", "zef_label.cu")
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        variant = 2 if kernel == 0 else kernel - 1
        shape = f"k_label32<{st['block_threads']},{st['points_per_thread']},{variant}>"
        for rec in recs:
            if rec["source_sha256_prefix"] == sha and rec["kernel"] == shape:
                return rec["bytes_per_launch"]
    except Exception:
        return None
    return None


def secondary(zef, torch, dev, cfg, flush, stream, barrier, peak, sms, kernel):
    """A secondary workload: 3 warm-up + 5 timed calls."""
    w = workload(cfg, 0)
    ctx = make_context(zef, w, dev.index)
    pts = torch.from_numpy(np.ascontiguousarray(w.points)).to(dev)
    labels = torch.empty(pts.shape[0], dtype=torch.int32, device=dev)
    r = timed_steps(torch, ctx, pts, labels, zef.make_opts(kernel=kernel), 5, 3, flush, stream, barrier)
    st = r["stats"]
    ms = r["ms"] / 5
    out = {"workload": w.name, "points": int(w.points.shape[0]), "triangles": int(w.total_tris),
           "compartments": len(w.surfaces), "ms_per_step": ms,
           "nominal_pairs_per_s": st["pairs_nominal"] / (ms * 1e-3),
           "evaluated_pairs_per_s": st["pairs_evaluated"] / (ms * 1e-3),
           "points_per_s": w.points.shape[0] / (ms * 1e-3),
           "ms_label_kernel": r["ms_label"], "ms_rescue": r["ms_rescue"],
           "uncertain_pairs_per_step": st["uncertain_pairs"],
           "autotuned_shape": [st["block_threads"], st["points_per_thread"]],
           "roofline_frac": roofline(st, r["ms_label"], peak, sms)["frac"],
           "step_ms": [round(x, 3) for x in r["step_ms"]]}
    ctx.close()
    del pts, labels
    torch.cuda.empty_cache()
    return out


def refine_measure(zef, torch, dev):
    """Refine-and-relabel workload: the three-layer head plus 8 deep
    compartments on a 4 mm lattice (51^3 nodes), 3 levels as one CUDA graph.
    The second call reuses the captured graph; its device time is reported
    with the per-level counts."""
    import zef_synth as zs
    w = zs.config3()
    ctx = make_context(zef, w, dev.index)
    ncap, tcap = 6_000_000, 16_000_000
    nodes = torch.zeros((ncap, 3), dtype=torch.float32, device=dev)
    tets = torch.zeros((tcap, 4), dtype=torch.int32, device=dev)
    labels = torch.zeros(ncap, dtype=torch.int32, device=dev)
    n0, m0 = w.nodes.shape[0], w.tets.shape[0]
    src_n = torch.from_numpy(w.nodes).to(dev)
    src_t = torch.from_numpy(w.tets).to(dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return res, e0.elapsed_time(e1)

    out = None
    for rep in range(2):
        nodes[:n0].copy_(src_n)
        tets[:m0].copy_(src_t)
        (n1, m1, per), ms = timed(lambda: ctx.refine_and_relabel(nodes, tets, labels, n0, m0, 3))
        out = {"workload": w.name, "initial_nodes": n0, "initial_tets": m0, "levels": per,
               "ms_total_incl_initial_labeling": ms, "final_nodes": n1, "final_tets": m1}
    # the same three levels closed into a conforming mesh (Fig. 2 c-e)
    ncap_c, tcap_c = 8_000_000, 26_000_000
    nodes_c = torch.zeros((ncap_c, 3), dtype=torch.float32, device=dev)
    tets_c = torch.zeros((tcap_c, 4), dtype=torch.int32, device=dev)
    labels_c = torch.zeros(ncap_c, dtype=torch.int32, device=dev)
    for rep in range(2):
        nodes_c[:n0].copy_(src_n)
        tets_c[:m0].copy_(src_t)
        (cn1, cm1, cper), ms = timed(lambda: ctx.refine_and_relabel(nodes_c, tets_c, labels_c, n0, m0, 3,
                                                                    conforming=True))
    out["conforming"] = {"levels": cper, "ms_total_incl_initial_labeling": ms,
                         "final_nodes": cn1, "final_tets": cm1}
    del nodes_c, tets_c, labels_c
    # element labels (four-nodes rule) of the refined mesh, then the recursive
    # boundary re-labeling after every node moved by up to 0.2 mm (seeded)
    rn, rt, rl = nodes[:n1], tets[:m1], labels[:n1].clone()
    elem = torch.empty(m1, dtype=torch.int32, device=dev)
    for rep in range(2):
        _, ms = timed(lambda: ctx.label_elements(rn, rt, elem_labels=elem, stats=False))
    out["elements"] = {"nodes": n1, "tets": m1, "ms": ms, "node_pairs_nominal": n1 * w.total_tris,
                       "note": "node inside bits of every compartment (no priority early exit), AND per tet"}
    g = torch.Generator(device=dev)
    g.manual_seed(41)
    moved = (rn + (torch.rand(rn.shape, generator=g, device=dev) - 0.5) * 0.4).contiguous()
    for rep in range(2):
        lab = rl.clone()
        (passes, conv), ms = timed(lambda: ctx.relabel_boundary(moved, rt, lab, 64))
    out["relabel_boundary"] = {"nodes": n1, "tets": m1, "displacement_mm": 0.2, "ms": ms,
                               "passes": len(passes), "converged": conv,
                               "evaluated": sum(e for e, _ in passes), "changed": sum(c for _, c in passes),
                               "per_pass": passes}
    # post-processing on the refined mesh: Taubin smoothing (lambda = mu = 0.4,
    # 10 iterations) and one inflation towards the brain surface (zeta = 0.05)
    xs = rn.clone()
    for rep in range(2):
        xs.copy_(rn)
        its, ms = timed(lambda: ctx.taubin_smooth(xs, rt, 0.4, 0.4, 0.0, 10))
    out["taubin_smooth"] = {"nodes": n1, "tets": m1, "iterations": its, "ms": ms,
                            "note": "includes building the unique-edge adjacency"}
    # the tissue boundaries of the element labels, the paper's stop rule xi = 0.1
    for rep in range(2):
        xs.copy_(rn)
        (sits, nfaces), ms = timed(lambda: ctx.taubin_smooth_surface(xs, rt, elem, 0.4, 0.4, 0.1, 100))
    out["taubin_smooth_surface"] = {"nodes": n1, "tets": m1, "boundary_faces": nfaces, "iterations": sits,
                                    "xi": 0.1, "ms": ms,
                                    "note": "includes finding the boundary faces and their edge adjacency"}
    brain = [s_.id for s_ in w.surfaces if s_.name == "brain"][0]
    for rep in range(2):
        xs.copy_(rn)
        mv, ms = timed(lambda: ctx.inflate(xs, rt, brain, 0.05))
    out["inflate"] = {"nodes": n1, "tets": m1, "compartment": "brain", "moved_nodes": mv, "ms": ms,
                      "note": "includes labeling every node and the adjacency"}
    ctx.close()
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2203_10000_gb300 import zef

    w = workload(args.config, args.points)
    N = int(w.points.shape[0])
    sharded = ws > 1 and not args.replicas
    order = cuts = None
    if sharded:
        # one workload split into contiguous equal-work ranges of its Morton
        # order; each rank labels only its range
        from paper_2203_10000_gb300.shard import equal_work_ranges
        order, cuts, est = equal_work_ranges(w.points, w.surfaces, ws)
        pts_h = np.ascontiguousarray(w.points[order[cuts[rank]:cuts[rank + 1]]])
    else:
        pts_h = np.ascontiguousarray(w.points)
    n_local = int(pts_h.shape[0])
    ctx = make_context(zef, w, local)
    pts = torch.from_numpy(pts_h).to(dev)
    labels = torch.empty(n_local, dtype=torch.int32, device=dev)
    opts = zef.make_opts(kernel=args.kernel)
    if args.shape:
        t, p = (int(x) for x in args.shape.split(","))
        opts = zef.make_opts(block_threads=t, points_per_thread=p, kernel=args.kernel)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    flush.fill_(0)            # load the fill kernel before the timed region
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    r = timed_steps(torch, ctx, pts, labels, opts, args.steps, args.warmup, flush, stream, barrier,
                    sampler=ClockSampler(local))
    st = r["stats"]
    ms = r["ms"]
    if ws > 1:
        from paper_2203_10000_gb300.shard import max_over_ranks
        ms = max_over_ranks(ms, device=dev)
    ms_step = ms / args.steps
    tt = w.total_tris
    # headline: every point x triangle pair of the workload is decided each
    # step (pairs outside a closed surface's box or hull exactly, by culling;
    # pairs of coherent tiles by an exact representative), so the rate is
    # N x sum(T) / step time -- the basis of nodes x triangles / labeling
    # time and of the oracle, which culls nothing.  Evaluated pairs/s and
    # labelled points/s are reported beside it.
    job_points = N * (ws if (ws > 1 and not sharded) else 1)
    nominal_job = job_points * tt
    value = nominal_job / (ms_step * 1e-3)
    sms, peak = fp32_peak_tflops(torch, dev)
    rl = roofline(st, r["ms_label"], peak, sms, r["clocks"],
                  traffic_record(args.config, st, args.kernel) if not sharded else None)

    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(w, N),
            "value_basis": "nominal pairs: points x total triangles per step / step time",
            "pairs_nominal_per_step": nominal_job,
            "pairs_evaluated_per_step_rank0": st["pairs_evaluated"],
            "evaluated_pairs_per_s_rank0": st["pairs_evaluated"] / (ms_step * 1e-3),
            "points_per_s": job_points / (ms_step * 1e-3),
            "uncertain_pairs_per_step_rank0": st["uncertain_pairs"],
            "rescued_pairs_per_step_rank0": st["pairs_rescued"],
            "coherent_pairs_per_step_rank0": st["coherent_pairs"],
            "representative_pairs_per_step_rank0": st["representative_pairs"],
            "lane_walk_items_per_step_rank0": st["lane_walk_items"],
            "ms_label_kernel": r["ms_label"], "ms_rescue": r["ms_rescue"],
            "autotuned_shape": [st["block_threads"], st["points_per_thread"]],
            "step_ms": [round(x, 3) for x in r["step_ms"]],
            "roofline": rl, "gpu_launches": r["launches"],
            "gpu_launches_note": "the library's own kernels in the timed region (its per-call count summed "
                                 "over the steps); the L2 flush is torch's fill kernel",
            "clocks": r["clocks"]}
    if ws > 1:
        line["sharding"] = ("one workload, contiguous equal-work ranges of the Morton order "
                            f"(rank 0 holds {n_local} of {N} points)") if sharded else \
            "replicas: every rank labels the whole workload"

    # end to end through the C ABI with host buffers: every step copies the
    # points from pinned host memory to the device and the labels back into
    # pinned host memory (copies inside the timed region).  The headline
    # e2e is the pipelined entry point (zef_label_points_async: each step's
    # copies on their own streams, overlapping the neighbouring steps'
    # labeling); the synchronous single call is reported beside it.
    if not args.no_e2e:
        pts_pin = torch.from_numpy(pts_h).pin_memory()
        lab_pin = [torch.empty(n_local, dtype=torch.int32).pin_memory() for _ in range(2)]
        ke = max(1, args.steps)
        ctx.label_points(pts_pin, labels=lab_pin[0], opts=opts, stats=False)
        e2e_clk = ClockSampler(local)
        e2e_clk.start()
        time.sleep(1.0)
        singles = []
        for _ in range(ke):
            barrier()
            t0 = time.perf_counter()
            ctx.label_points(pts_pin, labels=lab_pin[0], opts=opts, stats=False)
            barrier()
            singles.append(time.perf_counter() - t0)
        t_single = float(np.median(singles))
        same_single = bool(np.array_equal(lab_pin[0].numpy(), labels.cpu().numpy()))
        for k in range(2):                   # warm-up: the two staging slots
            lab_pin[k].fill_(-7)
            ctx.label_points_async(pts_pin, lab_pin[k], opts=opts)
        ctx.synchronize()
        reps = []
        for _ in range(5):                   # five runs of K calls; the median is reported
            barrier()
            t0 = time.perf_counter()
            for k in range(ke):
                ctx.label_points_async(pts_pin, lab_pin[k % 2], opts=opts)
            ctx.synchronize()
            barrier()
            reps.append((time.perf_counter() - t0) / ke)
        te = float(np.median(reps))
        # the host link itself at this moment (the GPUs' hosts are shared)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        pts.copy_(pts_pin, non_blocking=True)
        ev[1].record(stream)
        lab_pin[0].copy_(labels, non_blocking=True)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        link = {"h2d_gbs": pts_pin.numel() * 4 / (ev[0].elapsed_time(ev[1]) * 1e6),
                "d2h_gbs": labels.numel() * 4 / (ev[1].elapsed_time(ev[2]) * 1e6)}
        e2e_clocks = e2e_clk.stop()
        if ws > 1:
            from paper_2203_10000_gb300.shard import max_over_ranks
            te = max_over_ranks(te, device=dev)
            t_single = max_over_ranks(t_single, device=dev)
        ref_lab = labels.cpu().numpy()
        line["e2e"] = {"value": nominal_job / te, "unit": "pairs/s", "h2d_bytes_per_step": int(n_local * 12),
                       "d2h_bytes_per_step": int(n_local * 4), "ms_per_step": te * 1e3, "steps": ke,
                       "api": "zef_label_points_async, K calls then zef_synchronize (median of 5 runs)",
                       "host_memory": "pinned", "timer": "host clock around K calls, synchronized",
                       "labels_equal_device_run": bool(all(np.array_equal(lab_pin[k].numpy(), ref_lab)
                                                           for k in range(min(2, ke)))),
                       "runs_ms_per_step": [round(x * 1e3, 3) for x in reps],
                       "host_link": link,
                       "clocks": e2e_clocks,
                       "single_call": {"api": "zef_label_points (synchronous), median of K calls",
                                       "ms_per_step": t_single * 1e3,
                                       "calls_ms": [round(x * 1e3, 3) for x in singles],
                                       "value": nominal_job / t_single,
                                       "labels_equal_device_run": same_single}}
        del pts_pin, lab_pin

    # accuracy of the FP32 sums themselves: on a seeded sample, every pair
    # with an FP32 sum of its own (ZEF_OMEGA_RAW, no FP64 re-evaluation)
    # against 4 pi k, k the winding number of the default call (certified
    # or re-evaluated in FP64; the exact Omega of a closed surface off the
    # surface is 4 pi k)
    if args.omega_points > 0 and rank == 0:
        ns = min(n_local, args.omega_points)
        idx = np.sort(np.random.default_rng(11).choice(n_local, ns, replace=False))
        sub = pts[torch.from_numpy(idx).to(dev)].contiguous()
        _, om_def, _ = ctx.label_points(sub, want_omega=True, opts=zef.make_opts(kernel=args.kernel), stats=False)
        _, om_raw, _ = ctx.label_points(sub, want_omega=True, stats=False,
                                        opts=zef.make_opts(kernel=args.kernel, omega_raw=True,
                                                           precision=zef.ZEF_FP32_ONLY))
        four_pi = 4.0 * np.pi
        od = om_def.double().cpu().numpy()
        orw = om_raw.double().cpu().numpy()
        fin = np.isfinite(od) & np.isfinite(orw)
        k = np.rint(od[fin] / four_pi)
        raw = orw[fin]
        own = raw != (k * four_pi).astype(np.float32).astype(np.float64)   # pairs with a sum of their own
        err = np.abs(raw[own] - four_pi * k[own])
        line["omega_fp32"] = {
            "points": int(ns), "pairs": int(fin.sum()), "pairs_with_fp32_sum": int(own.sum()),
            "max_abs_err_sr": float(err.max()) if err.size else 0.0,
            "p9999_abs_err_sr": float(np.quantile(err, 0.9999)) if err.size else 0.0,
            "above_1e-5": int((err > 1e-5).sum()),
            "basis": "|Omega32 - 4 pi k| per (point, compartment) pair, ZEF_FP32_ONLY + ZEF_OMEGA_RAW; k from "
                     "the default call; seeded uniform sample of the workload"}

    # FP32 + rescue vs the plain FP64 kernel on the same subset
    if args.fp64_points > 0 and rank == 0:
        nsub = min(n_local, args.fp64_points)
        c0 = n_local // 2 - nsub // 2
        sub = pts[c0:c0 + nsub].contiguous()
        lab_sub = torch.empty(nsub, dtype=torch.int32, device=dev)
        _, _, s32 = ctx.label_points(sub, labels=lab_sub, opts=opts, stats=True)
        l32 = lab_sub.clone()
        _, _, s64 = ctx.label_points(sub, labels=lab_sub, opts=zef.make_opts(precision=zef.ZEF_FP64_PLAIN),
                                     stats=True)
        same = bool(torch.equal(l32, lab_sub))
        line["fp64_plain"] = {"points": nsub, "ms_fp32_rescue": s32["ms_total"], "ms_fp64_plain": s64["ms_total"],
                              "speedup": s64["ms_total"] / s32["ms_total"], "labels_equal": same,
                              "fp64_pairs_per_s": s64["pairs_evaluated"] / (s64["ms_total"] * 1e-3)}

    # measured FMA throughput of this GPU (cross-check of the FP32 peak; the
    # FP64 rate sets the cost of the re-evaluation and of the plain FP64 kernel)
    if rank == 0:
        f32 = ctx.fma_rate(fp64=False)
        f64 = ctx.fma_rate(fp64=True)
        line["fma_microbench"] = {"fp32_tflops": f32, "fp64_tflops": f64, "fp32_frac_of_peak": f32 / peak}

    if sharded:
        # the labels of the one workload, gathered once after the timed region
        from paper_2203_10000_gb300.shard import gather_sharded
        full = gather_sharded(labels, order, cuts)
        line["gathered_labels"] = {"points": int(full.numel()), "nonnegative": bool((full >= 0).all().item())}

    if rank == 0 and not args.no_compare:
        # the same step with every point evaluated (tile coherence off)
        opts_nc = zef.make_opts(kernel=args.kernel, coherence=False)
        if args.shape:
            t_, p_ = (int(x) for x in args.shape.split(","))
            opts_nc = zef.make_opts(block_threads=t_, points_per_thread=p_, kernel=args.kernel, coherence=False)
        ctx.label_points(pts, labels=labels, opts=opts_nc, stats=True)
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        _, _, snc = ctx.label_points(pts, labels=labels, opts=opts_nc, stats=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        msnc = c0.elapsed_time(c1)
        line["no_tile_coherence"] = {"ms_per_step": msnc, "value": st["pairs_nominal"] / (msnc * 1e-3),
                                     "pairs_evaluated_per_step": snc["pairs_evaluated"],
                                     "evaluated_pairs_per_s": snc["pairs_evaluated"] / (msnc * 1e-3),
                                     "ms_label_kernel": snc["ms_label"]}
    ctx.close()
    del pts, labels
    torch.cuda.empty_cache()

    if rank == 0:
        for tok in [c.strip() for c in args.extra_configs.split(",") if c.strip()]:
            cfg = int(tok) if tok.isdigit() else tok
            if cfg == args.config:
                continue
            line[f"config{cfg}" if tok.isdigit() else cfg] = secondary(zef, torch, dev, cfg, flush, stream, lambda: torch.cuda.synchronize(dev),
                                             peak, sms, args.kernel)

    if rank == 0 and not args.no_refine:
        line["refine"] = refine_measure(zef, torch, dev)

    if rank == 0 and not args.no_cpu:
        sample = args.cpu_sample or auto_sample(w, 12.0)
        rate, dt, n, cores = cpu_oracle_rate(w, sample)
        line["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n} seeded points of the workload x all {w.total_tris} triangles "
                                          f"({dt:.1f} s, no culling)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
