#!/usr/bin/env python
"""Benchmark: per-Gaussian visibility precompute on one GB300.

A step is one whole precompute of the visibility table: LBVH build over the
Gaussians plus the trace of every ray cast from every Gaussian along each of
K Fibonacci directions (Sec. 4.1-4.2), inputs already resident in HBM.
Default workload: the 2M-Gaussian object-scale scene (flattened Gaussians on
2 spheres, a torus, a box and a ground plane; opacity Beta(5,1)) x 128
directions = 256M rays per step.

Printed (rank 0, one JSON line): traced rays/s of the whole precompute, ms
per precompute, the roofline of the trace kernel (algorithmic bytes of node
boxes and Gaussians fetched per ray over the measured HBM peak), the
end-to-end rate through the C ABI from pinned host buffers, the FP64 oracle's
rate on the host cores (a bounded sample), and SM clocks sampled during the
timed region.

`--impl reference` times the FP64 brute-force oracle (the reference for this
method) on the host cores on bounded samples of the same workload.
With `--gpus N` (torchrun) every rank runs an independent replica: the
precompute has no exchange step, so there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, n, seed, K)
    "object_2m_k128": ("object", 2_000_000, 2, 128),
    "object_300k_k128": ("object", 300_000, 2, 128),
    "uniform_4k_k32": ("uniform", 4096, 1, 32),
    # 16 uniform scenes (log-uniform sizes, ~8M Gaussians), 128 directions +
    # 512 env-map shadow rays per Gaussian, one graph-captured launch
    "batch16_k128_env512": ("batch", 8_000_000, 300, 128),
    # the same composition with object-scale scenes (flattened Gaussians on surfaces)
    "batch16_objects_k128_env512": ("batch_objects", 8_000_000, 300, 128),
    # one composed scene: 16 instances of 4 object-scale objects (125k each)
    # under seeded rigid maps, two-level BVH, true inter-object occlusion
    "composed16_objects_k128": ("composed", 2_000_000, 60, 128),
}
KERNEL_NAMES = ["auto", "per-ray binary", "packet binary", "packet 4-wide", "per-ray 4-wide",
                "per-ray 4-wide, lane refill", "warp per ray"]
ENV_SAMPLES = 512
METRIC = "traced rays/s & ms per 2M-Gaussian visibility precompute; surrogate speedup at MAE"
TRACE_SOURCES = ["paper_2311_16043_gb300/csrc/rt_trace.cu", "paper_2311_16043_gb300/csrc/rt_trace_core.cuh"]
# input check, bounds, morton, 4 x (hist, 3-kernel scan, scatter), perm,
# prep, karras, refit, and the 4-wide collapse: one launch per level, 63 levels
BUILD_KERNELS_PER_STEP = 27 + 63


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="object_2m_k128")
    ap.add_argument("--kernel", type=int, default=0, choices=range(7),
                    help="0 auto, 1 per-ray binary, 2 packet binary, 3 packet 4-wide, 4 per-ray 4-wide, "
                         "5 per-ray 4-wide with lane refill, 6 warp per ray")
    ap.add_argument("--order-block", type=int, default=0)
    ap.add_argument("--cpu-rays", type=int, default=2048, help="oracle sample for cpu_baseline")
    ap.add_argument("--cpu-lbvh-rays", type=int, default=1 << 20, help="sample for the CPU BVH tracer baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-pbr", action="store_true")
    ap.add_argument("--no-refit", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 16-scene batch section of the default line")
    ap.add_argument("--surrogate-steps", type=int, default=2000)
    ap.add_argument("--band", type=float, default=0.3)
    ap.add_argument("--pos-weight", type=float, default=4.0,
                    help="surrogate loss weight on the lit term (visibility decoded as 1 / (1 + w e^-z))")
    ap.add_argument("--gaussians", type=int, default=0,
                    help="override the workload's Gaussian count (a small case of the same kernels, for "
                         "profiling); the JSON line reports the count used")
    args = ap.parse_args()
    if args.gaussians > 0:
        gen, _, seed, K = WORKLOADS[args.workload]
        WORKLOADS[args.workload] = (gen, args.gaussians, seed, K)
    return args


def make_scene(name):
    import scenes
    gen, n, seed, K = WORKLOADS[name]
    if gen == "composed":  # the reference arm samples rays of one object
        return scenes.object_scene(n // 16, seed), scenes.fibonacci_sphere(K)
    if gen.startswith("batch"):
        # sizes log-uniform in [50k, 2M] for the 8M-Gaussian workload; a smaller
        # total (--gaussians) scales the range with it
        f = n / 8_000_000
        sizes = scenes.batch_scene_sizes(16, n, seed, lo=max(1000, int(50_000 * f)), hi=max(1000, int(2_000_000 * f)))
        gen_scenes = scenes.batch_scenes if gen == "batch" else scenes.batch_object_scenes
        return gen_scenes(sizes, seed_base=seed), scenes.fibonacci_sphere(K)
    sc = scenes.object_scene(n, seed) if gen == "object" else scenes.uniform_scene(n, seed)
    return sc, scenes.fibonacci_sphere(K)


def workload_config(name, extra=None):
    gen, n, seed, K = WORKLOADS[name]
    if gen.startswith("batch"):
        kind = "uniform" if gen == "batch" else "object-scale"
        cfg = {"workload": name, "scenes": 16, "gaussians": n, "directions": K, "env_samples": ENV_SAMPLES,
               "rays_per_step": None, "scene": f"16 {kind} scenes, log-uniform sizes in [50k, 2M]",
               "seed": seed, "step": "one replay of the graph-captured persistent launch over all scenes",
               "l2": "outputs > L2 (T tables ~20 GB)"}
        if extra:
            cfg.update(extra)
        return cfg
    if gen == "composed":
        cfg = {"workload": name, "gaussians": n, "directions": K,
               "scene": "16 instances of 4 object-scale objects (125k Gaussians each), seeded rigid maps",
               "seed": seed, "step": "top-level rebuild + trace of every Gaussian of every instance",
               "l2": "outputs > L2 (T table 1024 MB) and a 512 MB L2 flush between steps"}
        if extra:
            cfg.update(extra)
        return cfg
    cfg = {"workload": name, "gaussians": n, "directions": K, "rays_per_step": n * K,
           "scene": "object-scale: 2 spheres, torus, box, ground plane" if gen == "object"
           else "uniform cube", "seed": seed,
           "step": "LBVH build + trace of every (Gaussian, direction) ray",
           "l2": "inputs+outputs > L2 (T table %.0f MB) and a 512 MB L2 flush between steps" % (n * K * 4 / 1e6)}
    if extra:
        cfg.update(extra)
    return cfg


def reduce_max(x: float, world: int, device=None) -> float:
    """Maximum of x over the ranks (the replicas' slowest time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: int, ms_max: float, world: int) -> float:
    """Whole-job throughput: every replica's units over the slowest time."""
    return world * units_per_rank / (ms_max / 1000.0)


def oracle_rate(sc, dirs, m, seed=99):
    """Rays/s of the FP64 brute-force oracle on a seeded sample of m rays."""
    import oracle
    import scenes
    oracle.build()
    n, K = sc["mean"].shape[0], dirs.shape[0]
    ids = scenes.sample_ray_ids(n * K, m, seed)
    o, d, s = oracle.dir_rays(sc["mean"], dirs, ids)
    t0 = time.perf_counter()
    oracle.trace(sc, o, d, s)
    dt = time.perf_counter() - t0
    return m / dt, dt


def lbvh_rate(sc, dirs, m, seed=98):
    """Rays/s of the oracle's FP64 CPU BVH tracer (the brute-force T through
    the LBVH twin) on a seeded sample of m rays: a fairer CPU baseline than
    brute force.  The tree build is timed apart."""
    import oracle
    import scenes
    oracle.build()
    n, K = sc["mean"].shape[0], dirs.shape[0]
    ids = scenes.sample_ray_ids(n * K, m, seed)
    t0 = time.perf_counter()
    B = oracle.BvhTracer(sc)
    t1 = time.perf_counter()
    out = B.trace_dirs(dirs, ids)
    t2 = time.perf_counter()
    B.close()
    return {"value": m / (t2 - t1), "unit": "rays/s", "cores": os.cpu_count(), "kind": "oracle CPU BVH tracer",
            "build_s": t1 - t0, "sample": f"{m} seeded rays of the {n * K}, {t2 - t1:.1f} s",
            "per_ray": {"box_tests": float(out["counts"][0]) / m, "gaussian_tests": float(out["counts"][1]) / m}}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def trace_traffic():
    """DRAM bytes per launch of the trace kernel from the committed ncu summary,
    if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "k_trace_dram_object2m_k128.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256()
    for p in TRACE_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    if kv.get("kernel_sha256") != h.hexdigest()[:16]:
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_surrogate(args, rt, torch, d, dirs, T, prm, dev):
    """Learned visibility: train the MLP on the tracer's table (weighted BCE,
    weight `--pos-weight` on the lit term), then infer on held-out rays —
    the Fibonacci set under a seeded random rotation — in batches of 1M-64M
    rays sampled over the whole scene (one ray id per equal stratum of the
    256M), with and without tracer fallback.  Per batch: MAE against the
    traced T next to the MAE of predicting 0, the best constant (the batch's
    median T) and the batch's mean T; MAE on the lit rays (T > 0.05); rays/s
    against the tracer on the same rays and at its full-set rate."""
    import scenes
    n, K = T.shape
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], prm)
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs)
    s = rt.rt_surrogate_create(rt.mlp_cfg(batch=262144, lr=1e-3, pos_weight=args.pos_weight), seed=5)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    curve = rt.rt_surrogate_train(s, bvh, rs, T.view(-1), steps=args.surrogate_steps, seed=5)
    ev[1].record()
    torch.cuda.synchronize()
    train_ms = ev[0].elapsed_time(ev[1])
    train_flop = 3 * 118528 * args.surrogate_steps * 262144
    held = torch.from_numpy(scenes.rotated_fibonacci(K, 51)).to(dev)
    rs_h = rt.rayspec(rt.RT_RAYS_DIRS, dirs=held)
    Th = torch.empty(n * K, dtype=torch.float32, device=dev)
    rt.rt_trace_visibility(bvh, rs_h, Th)
    ev[0].record()
    rt.rt_trace_visibility(bvh, rs_h, Th)
    ev[1].record()
    torch.cuda.synchronize()
    tracer_rate = n * K / (ev[0].elapsed_time(ev[1]) / 1000.0)
    pk, _ = peaks()
    out = {"train_steps": args.surrogate_steps, "train_batch": 262144, "pos_weight": args.pos_weight,
           "train_ms": train_ms, "train_samples": args.surrogate_steps * 262144,
           "train_tflops": train_flop / (train_ms / 1000.0) / 1e12,
           "train_frac_of_sustained_bf16": train_flop / (train_ms / 1000.0) / 1e12
           / pk.get("bf16_tflops_sustained", pk["bf16_tflops"]),
           "loss_first": float(curve[:10].mean()), "loss_last": float(curve[-10:].mean()), "band": args.band,
           "heldout": "rotated Fibonacci set (seed 51); batches: one ray id per equal stratum of all n*K ids",
           "tracer_rays_per_s_heldout_full": tracer_rate, "batches": []}
    nfb = torch.zeros(1, dtype=torch.int64, device=dev)
    for j, B in enumerate((1 << 20, 1 << 22, 1 << 24, 1 << 26)):
        if B > n * K:
            break
        ids = torch.from_numpy(scenes.stratified_ray_ids(n * K, B, 51 + j)).to(dev)
        rsb = rt.rayspec(rt.RT_RAYS_DIRS, dirs=held, ray_ids=ids)
        ref = Th[ids]
        lit = ref > 0.05
        med = float(ref.median())
        out_b = {"rays": B, "mean_T": float(ref.mean()), "lit_fraction_T_gt_0.05": float(lit.float().mean()),
                 "mae_predict_zero": float(ref.abs().mean()),
                 "mae_best_constant": float((ref - med).abs().mean()), "best_constant": med,
                 "mae_predict_mean": float((ref - ref.mean()).abs().mean()),
                 "mae_predict_zero_lit": float(ref[lit].abs().mean()) if bool(lit.any()) else None}
        for band, key in ((0.0, "surrogate_only"), (args.band, "with_fallback")):
            q = torch.empty(B, dtype=torch.float32, device=dev)
            rt.rt_surrogate_infer(s, bvh, rsb, band=band, T_out=q, n_fallback=nfb)
            ev[0].record()
            rt.rt_surrogate_infer(s, bvh, rsb, band=band, T_out=q, n_fallback=nfb)
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1])
            mae = float((q - ref).abs().mean())
            out_b[key] = {"ms": ms, "rays_per_s": B / (ms / 1000.0), "mae": mae,
                          "mae_lit": float((q - ref)[lit].abs().mean()) if bool(lit.any()) else None,
                          "mae_over_predict_zero": mae / max(out_b["mae_predict_zero"], 1e-30),
                          "fallback_fraction": float(nfb.item()) / B}
        tq = torch.empty(B, dtype=torch.float32, device=dev)
        rt.rt_trace_visibility(bvh, rsb, tq)
        ev[0].record()
        rt.rt_trace_visibility(bvh, rsb, tq)
        ev[1].record()
        torch.cuda.synchronize()
        out_b["tracer_same_rays"] = {"ms": ev[0].elapsed_time(ev[1]),
                                     "rays_per_s": B / (ev[0].elapsed_time(ev[1]) / 1000.0)}
        out_b["speedup_vs_tracer_same_rays"] = (out_b["with_fallback"]["rays_per_s"]
                                                / out_b["tracer_same_rays"]["rays_per_s"])
        out_b["speedup_vs_tracer_full_rate"] = out_b["with_fallback"]["rays_per_s"] / tracer_rate
        # training charged to the batch: spread over the scene's whole ray table
        # (the precompute the surrogate stands in for), or all on this batch
        tracer_ms = 1000.0 * B / tracer_rate
        fb_ms = out_b["with_fallback"]["ms"]
        out_b["speedup_incl_training_amortised"] = tracer_ms / (fb_ms + train_ms * B / (n * K))
        out_b["speedup_incl_training_not_amortised"] = tracer_ms / (fb_ms + train_ms)
        out["batches"].append(out_b)
    s.destroy()
    bvh.destroy()
    out["other_scenes"] = [surrogate_other_scene(rt, torch, dev, *c, pos_weight=args.pos_weight, band=args.band)
                           for c in (("uniform_4k_k32", "uniform", 4096, 1, 32),
                                     ("uniform_300k_k64", "uniform", 300_000, 3, 64))]
    return out


def surrogate_other_scene(rt, torch, dev, name, gen, n, seed, K, pos_weight, band, steps=2000):
    """The surrogate on a second scene: trained (the same recipe) on its
    Fibonacci table, evaluated on every ray of the rotated set, next to the
    trivial predictors.  uniform_4k_k32 is the sparse config-1 scene (no
    T = 0 rays); uniform_300k_k64 the same distributions at 300k Gaussians
    (optically dense)."""
    import scenes
    sc = scenes.uniform_scene(n, seed) if gen == "uniform" else scenes.object_scene(n, seed)
    d = {k: torch.from_numpy(v).to(dev) for k, v in sc.items()}
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=torch.from_numpy(scenes.fibonacci_sphere(K)).to(dev))
    T = rt.rt_trace_visibility(bvh, rs)
    rs_h = rt.rayspec(rt.RT_RAYS_DIRS, dirs=torch.from_numpy(scenes.rotated_fibonacci(K, 51)).to(dev))
    Th = rt.rt_trace_visibility(bvh, rs_h, opts=rt.trace_opts(kernel=rt.RT_KERNEL_WARP_RAY))
    s = rt.rt_surrogate_create(rt.mlp_cfg(batch=262144, lr=1e-3, pos_weight=pos_weight), seed=5)
    rt.rt_surrogate_train(s, bvh, rs, T.view(-1), steps=steps, seed=5)
    p = rt.rt_surrogate_infer(s, bvh, rs_h, band=0.0)
    nfb = torch.zeros(1, dtype=torch.int64, device=dev)
    q = rt.rt_surrogate_infer(s, bvh, rs_h, band=band, n_fallback=nfb)
    torch.cuda.synchronize()
    med = float(Th.median())
    out = {"scene": name, "gaussians": n, "directions": K, "rays": n * K, "mean_T": float(Th.mean()),
           "zero_fraction": float((Th == 0).float().mean()), "mae_predict_zero": float(Th.abs().mean()),
           "mae_best_constant": min(float(Th.abs().mean()), float((Th - med).abs().mean())),
           "mae_predict_mean": float((Th - Th.mean()).abs().mean()),
           "mae_surrogate_only": float((p - Th).abs().mean()), "mae_with_fallback": float((q - Th).abs().mean()),
           "fallback_fraction": float(nfb.item()) / (n * K)}
    s.destroy()
    bvh.destroy()
    return out


def run_pbr(rt, torch, d, sc, dev):
    """Hemisphere workload of Sec. 3.3 / 4.2 on the bench scene: N_s = 64
    Fibonacci directions about each Gaussian's normal (its shortest axis):
    visibility table, the per-Gaussian PBR colour of Eq. 10 from that table,
    the fused trace + shade (no table), and fused ambient occlusion."""
    import scenes
    n, K = sc["mean"].shape[0], 64
    nrm = torch.from_numpy(scenes.shortest_axis_normals(sc["scale"], sc["quat"])).to(dev)
    hemi = torch.from_numpy(scenes.fibonacci_hemisphere(K)).to(dev)
    mat = scenes.pbr_material(n, 6)
    env = torch.from_numpy(scenes.light_envmap(6)).to(dev)
    inp = rt.pbr_inputs(torch.from_numpy(mat["albedo"]).to(dev), torch.from_numpy(mat["roughness"]).to(dev),
                        env, (1.0, 3.0, 2.5), sh=torch.from_numpy(mat["sh"]).to(dev))
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params())
    rs = rt.rayspec(rt.RT_RAYS_HEMI, dirs=hemi, normals=nrm)
    V = torch.empty(n * K, dtype=torch.float32, device=dev)
    rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    ao = torch.empty(n, dtype=torch.float32, device=dev)

    def timed(f, reps):
        f()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            f()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    t_ms = timed(lambda: rt.rt_trace_visibility(bvh, rs, V), 2)
    s_ms = timed(lambda: rt.rt_pbr_shade(bvh, rs, inp, V=V, rgb=rgb), 10)
    f_ms = timed(lambda: rt.rt_pbr_shade(bvh, rs, inp, rgb=rgb), 2)
    a_ms = timed(lambda: rt.rt_trace_ao(bvh, rs, ao), 2)
    # bytes the shading kernel must move: the table, the per-Gaussian inputs
    # (normal 12, albedo 12, roughness 4, SH 108, mean 16, rank 4) and the colour
    shade_bytes = 4 * n * K + n * (12 + 12 + 4 + 108 + 16 + 4 + 12)
    out = {"gaussians": n, "directions": K, "rays": n * K, "mean_visibility": float(V.mean()),
           "trace_table_ms": t_ms, "trace_rays_per_s": n * K / (t_ms / 1000.0),
           "shade_from_table_ms": s_ms, "shade_terms_per_s": n * K / (s_ms / 1000.0),
           "shade_bytes_per_launch": shade_bytes, "shade_gbs": shade_bytes / (s_ms / 1000.0) / 1e9,
           "table_plus_shade_ms": t_ms + s_ms, "fused_trace_shade_ms": f_ms,
           "fused_gaussians_per_s": n / (f_ms / 1000.0), "fused_ao_ms": a_ms,
           "mean_ao": float(ao.mean()), "rgb_max": float(rgb.max())}
    bvh.destroy()
    return out


def run_refit(rt, torch, d, sc, dirs, opts, dev):
    """Refit-only rebuild on the bench scene: refit time against a full build,
    and the trace after the means move by N(0, 1 mm) — refit (stale Morton
    order) against a fresh build of the moved scene."""
    def timed(f, reps):
        f()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            f()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    prm = rt.params()
    n, K = sc["mean"].shape[0], dirs.shape[0]
    T = torch.empty(n * K, dtype=torch.float32, device=dev)
    holder = []

    def build():
        if holder:
            holder.pop().destroy()
        holder.append(rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], prm))

    build_ms = timed(build, 10)
    bvh = holder.pop()
    refit_ms = timed(lambda: rt.rt_bvh_refit(bvh, d["mean"], d["scale"], d["quat"], d["opacity"]), 10)
    moved = (d["mean"] + 1e-3 * torch.randn(d["mean"].shape, generator=torch.Generator(device=dev).manual_seed(7),
                                             device=dev)).contiguous()
    rt.rt_bvh_refit(bvh, moved, d["scale"], d["quat"], d["opacity"])
    t_refit = timed(lambda: rt.rt_trace_visibility_dirs(bvh, dirs, T, opts), 1)
    fresh = rt.rt_build_bvh(moved, d["scale"], d["quat"], d["opacity"], prm)
    t_fresh = timed(lambda: rt.rt_trace_visibility_dirs(fresh, dirs, T, opts), 1)
    fresh.destroy()
    bvh.destroy()
    return {"build_ms": build_ms, "refit_ms": refit_ms, "motion": "means + N(0, 1e-3^2)",
            "trace_ms_after_refit": t_refit, "trace_ms_after_fresh_build": t_fresh}


def run_adjoint(rt, torch, dev):
    """Differentiation workload: L = sum_r w_r T_r over the rays of the first
    1,024 Gaussians of a 4,096-Gaussian uniform scene x 16 directions, and
    over all 4,096 x 32; forward + hand-written adjoint, with the hit log
    replayed and with re-traversal, and with the hit log and deterministic
    (fixed-point) accumulation; hit-log memory."""
    import scenes
    out = []
    for n_sub, K in ((1024, 16), (4096, 32)):
        sc = {k: v[:n_sub].copy() for k, v in scenes.uniform_scene(4096, 4).items()}
        d = {k: torch.from_numpy(v).to(dev) for k, v in sc.items()}
        dirs = torch.from_numpy(scenes.fibonacci_sphere(K)).to(dev)
        R = n_sub * K
        w = torch.from_numpy(scenes.loss_weights(R, 41)).to(dev)
        prm = rt.params(t_min=0.0)
        bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], prm)
        bvh_det = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params(t_min=0.0,
                                                                                             deterministic=True))
        rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs)
        cap = 64
        ids = torch.empty((R, cap), dtype=torch.int32, device=dev)
        cnt = torch.empty(R, dtype=torch.int32, device=dev)
        res = {"gaussians": n_sub, "directions": K, "rays": R}
        for mode in ("log", "recompute", "log_deterministic"):
            def run():
                tree = bvh_det if mode == "log_deterministic" else bvh
                use_log = mode != "recompute"
                o = rt.trace_opts(hit_ids=ids, hit_count=cnt) if use_log else None
                T = rt.rt_trace_visibility(tree, rs, opts=o)
                return T, rt.rt_trace_visibility_backward(tree, rs, d["mean"], d["scale"], d["quat"], d["opacity"], T,
                                                          w, ids if use_log else None, cnt if use_log else None)
            for _ in range(3):
                run()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(10):
                run()
            ev[1].record()
            torch.cuda.synchronize()
            res[f"{mode}_ms_fwd_bwd"] = ev[0].elapsed_time(ev[1]) / 10
        hits = int(cnt.to(torch.int64).sum())
        res["hits"] = hits
        res["hit_log_bytes_compact"] = 4 * hits + 8 * R
        res["hit_log_bytes_fixed_capacity"] = 4 * cap * R + 4 * R
        res["max_hits_per_ray"] = int(cnt.max())
        out.append(res)
        bvh.destroy()
        bvh_det.destroy()
    return out


def batch_setup(name, torch, rt, dev, autotune=True):
    """Every scene's BVH, the DIRS and ENV jobs over them and the batch (one
    graph-captured persistent launch over all jobs)."""
    import scenes
    scs, dirs_np = make_scene(name)
    env = scenes.envmap(399)
    E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
    dirs = torch.from_numpy(dirs_np).to(dev)
    jobs, bvhs, build_ms, specs = [], [], 0.0, []
    for s_idx, sc in enumerate(scs):
        d = {k: torch.from_numpy(v).to(dev) for k, v in sc.items()}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params())
        e1.record()
        torch.cuda.synchronize()
        build_ms += e0.elapsed_time(e1)
        bvhs.append((bvh, d))
        for kind, mk in (("dirs", lambda ids=None: rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs, ray_ids=ids)),
                         ("env", lambda ids=None, s_idx=s_idx: rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=ENV_SAMPLES,
                                                                          seed=399 + s_idx, ray_ids=ids))):
            rs = mk()
            jobs.append((bvh, rs, torch.empty(rt.rt_rayspec_count(bvh, rs), dtype=torch.float32, device=dev)))
            specs.append((kind, mk))
    t0 = time.perf_counter()
    batch = rt.rt_batch_create(jobs, autotune=autotune)
    create_s = time.perf_counter() - t0
    return {"E": E, "dirs": dirs, "jobs": jobs, "bvhs": bvhs, "specs": specs, "batch": batch,
            "build_ms": build_ms, "create_s": create_s}


def batch_ray_stats(B, torch, rt, dev, sample=1 << 16):
    """Outside the timed region: per ray kind, the early-exit fraction over
    every output, and per-ray work (child-box tests, Gaussian tests, accepted
    hits) counted on `sample` seeded rays of each job with the per-ray 4-wide
    traversal, which does each ray's minimal work; the work estimate of the
    whole batch in the bench's byte model (28 B per box test, 40 B per
    Gaussian test, 16 B per ray) from those per-job averages."""
    import scenes
    stats, alg_bytes = {}, 0.0
    for kind in ("dirs", "env"):
        rays = zeros = box = gauss = hits = sampled = 0
        for (bvh, _, T), (k2, mk) in zip(B["jobs"], B["specs"]):
            if k2 != kind:
                continue
            rays += T.numel()
            zeros += int((T == 0).sum())
            ids = torch.from_numpy(scenes.sample_ray_ids(T.numel(), min(sample, T.numel()), 5)).to(dev)
            cnt = torch.zeros(4, dtype=torch.int64, device=dev)
            rt.rt_trace_visibility(bvh, mk(ids), opts=rt.trace_opts(kernel=rt.RT_KERNEL_RAY_WIDE, counters=cnt))
            c = [int(x) for x in cnt.cpu()]
            m = ids.numel()
            alg_bytes += T.numel() * (28.0 * c[0] / m + 40.0 * c[1] / m + 16.0)
            box, gauss, hits, sampled = box + c[0], gauss + c[1], hits + c[2], sampled + m
        stats[kind] = {"rays": rays, "early_exit_fraction": zeros / max(rays, 1),
                       "box_tests_per_ray": box / max(sampled, 1), "gaussian_tests_per_ray": gauss / max(sampled, 1),
                       "accepted_hits_per_ray": hits / max(sampled, 1)}
    return stats, alg_bytes


def batch_destroy(B):
    B["batch"].destroy()
    for bvh, _ in B["bvhs"]:
        bvh.destroy()
    B["E"].destroy()


def run_batch_section(args, torch, rt, dev):
    """The batch workload inside the default bench line: one warm-up replay
    and one timed replay of the object-scale 16-scene batch, with the
    roofline of its one persistent launch."""
    name = "batch16_objects_k128_env512"
    B = batch_setup(name, torch, rt, dev)
    info = B["batch"].info()
    B["batch"].run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0.record()
    B["batch"].run()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats, alg = batch_ray_stats(B, torch, rt, dev)
    pk, pk_kind = peaks()
    R = info["n_rays"]
    out = {"workload": name, "rays": R, "ms": ms, "rays_per_s": R / (ms / 1000.0), "warmup": 1, "steps": 1,
           "scene_sizes": [b.n for b, _ in B["bvhs"]], "build_ms_all_scenes": B["build_ms"],
           "batch_create_s": B["create_s"], "strategy_per_job": info["kernel"], "ray_stats": stats,
           "roofline": {"bound": "hbm", "achieved": alg / (ms / 1000.0) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": alg / (ms / 1000.0) / 1e9 / pk["hbm_gbs"], "peak_kind": pk_kind,
                        "algorithmic_bytes_per_launch": alg, "kernel": "k_trace_batch (one persistent launch)",
                        "bytes_model": "28 B per child-box test + 40 B per Gaussian test + 16 B per ray; per-ray "
                                       "counts from 2^16 sampled rays per job (per-ray 4-wide traversal)"},
           "clocks": clk}
    batch_destroy(B)
    return out


def run_batch(args, rank, world, local, torch, dist, rt):
    """Batched multi-scene workload: every scene's BVH is built, then one
    graph-captured persistent launch traces all scenes' direction and
    env-map rays; a step is one replay of that graph."""
    dev = torch.device("cuda", local)
    B = batch_setup(args.workload, torch, rt, dev)
    batch = B["batch"]
    info = batch.info()
    R = info["n_rays"]
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for i in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    m = reduce_max(statistics.mean(ms), world, dev)
    stats, alg = batch_ray_stats(B, torch, rt, dev)
    pk, pk_kind = peaks()
    if rank == 0:
        achieved = alg / (statistics.mean(ms) / 1000.0) / 1e9
        line = {"metric": METRIC, "value": replica_rate(R, m, world), "unit": "rays/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": m, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.workload, {
                    "rays_per_step": R, "work_items": info["n_items"], "build_ms_all_scenes": B["build_ms"],
                    "batch_create_s": B["create_s"], "strategy_per_job": info["kernel"],
                    "order_block_per_job": info["order_block"],
                    "scene_sizes": [b.n for b, _ in B["bvhs"]], "ray_stats": stats}),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                             "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_kind": pk_kind,
                             "algorithmic_bytes_per_launch": alg, "kernel": "k_trace_batch (one persistent launch)",
                             "bytes_model": "28 B per child-box test + 40 B per Gaussian test + 16 B per ray; "
                                            "per-ray counts from 2^16 sampled rays per job"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    batch_destroy(B)


def run_composed(args, rank, world, local, torch, dist, rt):
    """Composed scene (Sec. 4.3): a step rebuilds the top level for the
    instances' maps (host) and traces every Gaussian of every instance along
    128 directions through all instances."""
    import scenes
    dev = torch.device("cuda", local)
    objs, pick, xf = scenes.composed_objects(per_obj=WORKLOADS[args.workload][1] // 16)
    bvhs = []
    for sc in objs:
        d = {k: torch.from_numpy(v).to(dev) for k, v in sc.items()}
        bvhs.append(rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params()))
    dirs = torch.from_numpy(scenes.fibonacci_sphere(WORKLOADS[args.workload][3])).to(dev)
    scene = rt.rt_scene_create([bvhs[i] for i in pick], xf)
    R = scene.n_total * dirs.shape[0]
    T = torch.empty((scene.n_total, dirs.shape[0]), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        rt.rt_scene_update(scene, xf)
        rt.rt_scene_trace_dirs(scene, dirs, T)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    m = reduce_max(statistics.mean(ms), world, dev)
    if rank == 0:
        line = {"metric": METRIC, "value": replica_rate(R, m, world), "unit": "rays/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": m, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.workload, {"rays_per_step": R, "instances": len(pick),
                                                          "objects": len(objs), "mean_T": float(T.mean())}),
                "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    scene.destroy()


def run_reference(args, rank, world):
    if rank != 0:
        return
    sc, dirs = make_scene(args.workload)
    if isinstance(sc, list):  # batched scenes: sample rays of the largest scene
        sc = max(sc, key=lambda x: x["mean"].shape[0])
    n, K = sc["mean"].shape[0], dirs.shape[0]
    # at least 64 rays per host core (the oracle hands out rays in chunks of
    # 64), else ~4e8 ray-Gaussian tests per step
    m = max(64 * (os.cpu_count() or 1), min(args.cpu_rays, int(4e8 // max(n, 1))))
    rates = []
    for i in range(args.warmup + args.steps):
        r, dt = oracle_rate(sc, dirs, m, seed=1000 + i)
        if i >= args.warmup:
            rates.append((r, dt))
    value = statistics.mean(r for r, _ in rates)
    ms = 1000.0 * n * K / value
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, {"parallelism": "host cores (OpenMP)"}),
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{m} seeded rays per step of the {n * K} (brute force, every ray vs every Gaussian)"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2311_16043_gb300 import rt

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if WORKLOADS[args.workload][0].startswith("batch"):
        run_batch(args, rank, world, local, torch, dist, rt)
        return
    if WORKLOADS[args.workload][0] == "composed":
        run_composed(args, rank, world, local, torch, dist, rt)
        return

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    rt.lib()
    sc, dirs_np = make_scene(args.workload)
    n, K = sc["mean"].shape[0], dirs_np.shape[0]
    R = n * K
    dev = torch.device("cuda", local)
    d = {k: torch.from_numpy(v).to(dev) for k, v in sc.items()}
    dirs = torch.from_numpy(dirs_np).to(dev)
    T = torch.empty((n, K), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prm = rt.params()
    opts = rt.trace_opts(kernel=args.kernel, order_block=args.order_block)

    def step(ev=None):
        if ev:
            ev[0].record()
        bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], prm)
        if ev:
            ev[1].record()
        rt.rt_trace_visibility_dirs(bvh, dirs, T, opts)
        if ev:
            ev[2].record()
        bvh.destroy()

    for _ in range(args.warmup):
        step()
    barrier()
    # per-ray work of this trace, counted once (outside the timed region)
    cnt = torch.zeros(4, dtype=torch.int64, device=dev)
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], prm)
    rt.rt_trace_visibility_dirs(bvh, dirs, T, rt.trace_opts(kernel=args.kernel, order_block=args.order_block,
                                                              counters=cnt))
    torch.cuda.synchronize()
    bvh.destroy()
    box_tests, gauss_tests, hits, rays_cnt = (int(x) for x in cnt.cpu())
    assert rays_cnt == R, (rays_cnt, R)
    alg_bytes = 28 * box_tests + 40 * gauss_tests + 16 * R

    clocks = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        step(evs[i])
    barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    trace_ms = [e[1].elapsed_time(e[2]) for e in evs]
    ms = reduce_max(statistics.mean(step_ms), world, dev)
    value = replica_rate(R, ms, world)

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(v).pin_memory() for k, v in sc.items()}
        hdirs = torch.from_numpy(dirs_np).pin_memory()
        hT = torch.empty((n, K), dtype=torch.float32).pin_memory()
        h2d = sum(v.numel() * 4 for v in host.values()) + hdirs.numel() * 4
        d2h = hT.numel() * 4
        e_ms = []
        e_clocks = ClockSampler(local)
        for i in range(args.warmup + args.steps):
            if i == args.warmup:
                e_clocks.start()
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            # one C-ABI call: copies in, build, trace, copy of T out
            rt.rt_visibility_dirs_host(host["mean"], host["scale"], host["quat"], host["opacity"], hdirs, hT,
                                       prm, opts)
            e1.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                e_ms.append(e0.elapsed_time(e1))
        e_clk = e_clocks.stop()
        # this machine's host link, for reading the gap between e2e and value:
        # one plain copy of the T table to the same page-locked buffer, right
        # after the last step's copy (a warm link)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        hT.copy_(T, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        d2h_probe_ms = c0.elapsed_time(c1)
        # the same steps as the call, one at a time through the binding, each
        # timed on the stream (after one more L2 flush): if e2e exceeds their
        # sum, the difference is in the call itself (its allocations)
        flush.fill_(-1.0)
        pe = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        pe[0].record()
        dd = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        ddirs = hdirs.to(dev, non_blocking=True)
        pe[1].record()
        pbvh = rt.rt_build_bvh(dd["mean"], dd["scale"], dd["quat"], dd["opacity"], prm)
        pe[2].record()
        rt.rt_trace_visibility_dirs(pbvh, ddirs, T, opts)
        pe[3].record()
        hT.copy_(T, non_blocking=True)
        pe[4].record()
        torch.cuda.synchronize()
        pbvh.destroy()
        phases = {"h2d_ms": pe[0].elapsed_time(pe[1]), "build_ms": pe[1].elapsed_time(pe[2]),
                  "trace_ms": pe[2].elapsed_time(pe[3]), "d2h_ms": pe[3].elapsed_time(pe[4])}
        phases["sum_ms"] = sum(phases.values())
        # the same copy again, back to back (the host link's rate varies from
        # moment to moment on a shared machine)
        c0.record()
        hT.copy_(T, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        phases["d2h_repeat_ms"] = c0.elapsed_time(c1)
        em = reduce_max(statistics.mean(e_ms), world, dev)
        e2e = {"value": replica_rate(R, em, world), "unit": "rays/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": em, "ms_each": e_ms,
               "call": "rt_visibility_dirs_host (C ABI) from page-locked host buffers", "clocks": e_clk,
               "d2h_copy_probe": {"ms": d2h_probe_ms, "gbs": d2h / d2h_probe_ms / 1e6},
               "phases_through_binding": phases}

    surrogate = None
    if not args.no_surrogate and rank == 0:
        surrogate = run_surrogate(args, rt, torch, d, dirs, T, prm, dev)
    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = run_adjoint(rt, torch, dev)
    pbr = None
    if not args.no_pbr and rank == 0:
        pbr = run_pbr(rt, torch, d, sc, dev)
    refit = None
    if not args.no_refit and rank == 0:
        refit = run_refit(rt, torch, d, sc, dirs, opts, dev)
    batch_sec = None
    if not args.no_batch and rank == 0:
        del T
        torch.cuda.empty_cache()
        batch_sec = run_batch_section(args, torch, rt, dev)

    pk, pk_kind = peaks()
    tr_ms = statistics.mean(trace_ms)
    achieved = alg_bytes / (tr_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": trace_traffic(),
                "kernel": "k_trace (visibility trace)", "peak_kind": pk_kind,
                "algorithmic_bytes_per_launch": alg_bytes,
                "per_ray": {"box_tests": box_tests / R, "gaussian_tests": gauss_tests / R,
                            "accepted_hits": hits / R},
                "bytes_model": "28 B per child-box test + 40 B per Gaussian test + 16 B per ray"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        m = max(32, min(args.cpu_rays, int(4e9 // max(n, 1))))
        rate, dt = oracle_rate(sc, dirs_np, m)
        cpu = {"value": rate, "unit": "rays/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{m} seeded rays of the {R} (FP64 brute force, every ray vs all {n} Gaussians), {dt:.1f} s"}
        cpu["lbvh_tracer"] = lbvh_rate(sc, dirs_np, args.cpu_lbvh_rays)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.workload, {
                    "parallelism": "replicas" if world > 1 else "single GPU",
                    "build_ms": statistics.mean(build_ms), "trace_ms": tr_ms,
                    "kernel": KERNEL_NAMES[args.kernel]}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": (BUILD_KERNELS_PER_STEP + 1) * args.steps,
                "clocks": clk, "surrogate": surrogate, "adjoint": adjoint, "pbr": pbr, "refit": refit,
                "batch": batch_sec}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
