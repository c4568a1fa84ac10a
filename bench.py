"""Benchmark: Diffusing Winding Gradients orientation on one GB300.

Workload (default): the 100,000-point torus (R = 1, r = 0.3, Gaussian noise
0.5 % of the bounding-box diagonal, area weights 4 pi^2 R r / N), plain kernel,
exact all-pairs FP32 with compensated sums, octree depth 8, k = 10, tol 0.1 deg,
random initial normals (seed 1), up to 30 iterations.

One step = one full orientation (dwg_orient): every iteration evaluates w and
grad w at all N points (N^2 interactions) and w at all Q octree-leaf corners
(Q*N interactions), extracts the w_bar level set, scatters face gradients to
the 10 nearest points, updates the normals and tests convergence, all inside
one CUDA graph launch.

Metric: GWN+grad interactions per second (performed kernel evaluations),
whole job over all ranks; also seconds to converged normals.  Multi-GPU runs
are independent replicas (weak scaling): the method's per-cloud loop has an
exchange step only when one cloud is split, which this benchmark does not do.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# FP32 operations per interaction in the minimal formulation of each kernel
# (sub x3, fma x3 for rho^2, mul+fma x2 for <m,d>, then the kernel's own):
#   w only, plain 12 | w and grad, plain 20 | w only, screened 17 | w and grad, screened 29
FP32_OPS = {("w", 0): 12, ("wg", 0): 20, ("w", 1): 17, ("wg", 1): 29}
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", type=int, default=0, help="0 plain, 1 screened (lambda 10)")
    ap.add_argument("--depth", type=int, default=None)
    ap.add_argument("--workload", default="torus-100k",
                    choices=["torus-100k", "metaballs-1m", "batch-64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--one-step", action="store_true",
                    help="run one iteration of the workload and exit (for profiler captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    if args.workload == "metaballs-1m":
        W = synth.workload_metaballs1m()
        W["path"] = 2     # Barnes-Hut
    else:
        W = synth.workload_torus100k()
        W["path"] = 1     # exact all-pairs
        W["theta"] = 0.5
    if args.depth:
        W["depth"] = args.depth
    W["kernel"] = args.kernel
    W["lambda"] = 10.0 if args.kernel == 1 else 0.0
    return W


def profiled_traffic(kernel_file):
    """dram bytes per launch recorded in a committed ncu summary (or None)."""
    try:
        for line in open(os.path.join(ROOT, "profiles", kernel_file)):
            if line.startswith("dram_bytes_per_launch:"):
                return int(line.split(":")[1])
    except OSError:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(torch, buf):
    buf.add_(1.0)  # writes 256 MiB, larger than the 129 MB L2


def run_ours(args, rank, world, local):
    import torch
    from paper_2405_13839_gb300 import dwg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = workload(args)
    p_host = W["points"]
    n = len(p_host)
    stream = torch.cuda.current_stream(dev)
    p_dev = torch.from_numpy(p_host).to(dev)
    a_dev = torch.from_numpy(W["weights"]).to(dev)
    h = dwg.dwg_create(p_dev)
    dwg.dwg_set_stream(h, stream.cuda_stream)
    dwg.dwg_set_weights(h, a_dev)
    dwg.dwg_set_params(h, W["kernel"], W["eps"], W["lambda"], W["max_iters"], W["tol"])
    dwg.dwg_set_update(h, W["depth"], 10, dwg.DWG_UPDATE_LEVELSET)
    dwg.dwg_set_tree(h, W["path"], W["theta"])
    dwg.dwg_set_init(h, dwg.DWG_INIT_RANDOM, 1)
    out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        dwg.dwg_orient(h, out)
    torch.cuda.synchronize()
    st = dwg.dwg_get_stats(h)
    iters = st["iters"]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    inter = 0.0
    it_list = []
    for k in range(args.steps):
        flush_l2(torch, flush)
        ev[k][0].record(stream)
        rc, it = dwg.dwg_orient(h, out)
        ev[k][1].record(stream)
        s = dwg.dwg_get_stats(h)
        inter += s["interactions"]
        it_list.append(it)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(ms) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dev_s, inter], dtype=torch.float64)
        tt = t.clone()
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dev_s = float(tmax[0])
        inter = float(tt[1])
    value = inter / dev_s

    # per-kernel device times of one iteration (same kernels and launch shapes)
    dwg.dwg_set_init(h, dwg.DWG_INIT_RANDOM, 1)
    prof = []
    for _ in range(3):
        prof.append(dwg.dwg_profile_step(h))
    kms = {k: statistics.median(p[k] for p in prof) for k in prof[0]}
    st = dwg.dwg_get_stats(h)
    nc = st["n_corners"]
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fmax = (peaks.get("sm_max_mhz") or 2070.0) * 1e6
    lanes = sm_count * FP32_LANES_PER_SM * fmax
    kind = W["kernel"]
    # dominant kernel: w at the leaf corners
    dom = "eval_corners" if kms.get("eval_corners", 0) >= kms["eval_points"] else "eval_points"
    if dom == "eval_corners":
        work = float(nc) * n
        ops = FP32_OPS[("w", kind)]
    else:
        work = float(n) * n
        ops = FP32_OPS[("wg", kind)]
    achieved = work / (kms[dom] / 1e3)
    peak = lanes / ops
    iter_ms = sum(kms.values())
    traffic = profiled_traffic("eval_corners_torus100k.md") if (
        dom == "eval_corners" and W["kernel"] == 0 and W["depth"] == 8) else None
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Ginteractions/s", "frac": achieved / peak, "traffic": traffic,
            "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x {fmax/1e6:.0f} MHz"
                          f" / {ops} FP32 ops per interaction",
            "kernel_ms": {k: round(v, 4) for k, v in kms.items()},
            "share": {k: round(v / iter_ms, 4) for k, v in kms.items()}}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        ph = torch.from_numpy(p_host).pin_memory()
        ah = torch.from_numpy(W["weights"]).pin_memory()
        oh = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        e2e_t = []
        e2e_inter = 0.0
        for k in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            h2 = dwg.dwg_create(ph)
            dwg.dwg_set_weights(h2, ah)
            dwg.dwg_set_params(h2, W["kernel"], W["eps"], W["lambda"], W["max_iters"], W["tol"])
            dwg.dwg_set_update(h2, W["depth"], 10, dwg.DWG_UPDATE_LEVELSET)
            dwg.dwg_set_tree(h2, W["path"], W["theta"])
            dwg.dwg_set_init(h2, dwg.DWG_INIT_RANDOM, 1)
            dwg.dwg_orient(h2, oh)
            e2e_inter += dwg.dwg_get_stats(h2)["interactions"]
            dwg.dwg_destroy(h2)
            e2e_t.append(time.perf_counter() - t1)
        e2e = {"value": e2e_inter / sum(e2e_t), "unit": "interactions/s",
               "s_per_orient": statistics.median(e2e_t),
               "h2d_bytes_per_step": int(ph.numel() * 4 + ah.numel() * 4),
               "d2h_bytes_per_step": int(oh.numel() * 4 + 4)}
    dwg.dwg_destroy(h)
    launches_per_step = 3 + 9 * statistics.mean(it_list)  # reset, random init, pack + 9 per iteration
    return dict(value=value, dev_s=dev_s, ms=ms, iters=it_list, st=st, roof=roof, clocks=ck,
                e2e=e2e, wall=wall, launches=int(round(launches_per_step * args.steps)), W=W,
                nc=nc)


def cpu_baseline(W, nc_hint, budget_s=12.0):
    """The oracle timed on a bounded sample: w and grad w at sampled points and
    w at sampled octree corners, against all N sources (FP64, all host cores)."""
    import oracle
    oracle.build()
    p, a = W["points"], W["weights"]
    n = len(p)
    n0 = synth.random_unit_normals(n, seed=1)
    L = oracle.octree_leaves(p, W["depth"])
    K = oracle.corner_keys(L, W["depth"])
    C = oracle.corner_positions(K, W["depth"], oracle.cube(p, W["depth"]))
    rng_pts = (synth.uniform(5, 1, 4096) * n).astype(np.int64)
    rng_cor = (synth.uniform(5, 2, 4096) * len(C)).astype(np.int64)
    kern, lam, eps = W["kernel"], W["lambda"], W["eps"]
    # probe, then size the sample to about budget_s seconds
    t = time.perf_counter()
    oracle.gwn(p, n0, a, p[rng_pts[:64]], kernel=kern, eps=eps, lam=lam)
    probe = time.perf_counter() - t
    m = int(max(64, min(4096, 64 * budget_s / 2 / max(probe, 1e-6))))
    t = time.perf_counter()
    oracle.gwn(p, n0, a, p[rng_pts[:m]], kernel=kern, eps=eps, lam=lam)
    tg = time.perf_counter() - t
    t = time.perf_counter()
    oracle.gwn(p, n0, a, C[rng_cor[:m]], kernel=kern, eps=eps, lam=lam, grad=False)
    tw = time.perf_counter() - t
    per_q_g = tg / m
    per_q_w = tw / m
    rate = (2 * m * n) / (tg + tw)
    # extrapolated time of one iteration of the full workload
    it_s = n * per_q_g + len(C) * per_q_w
    return {"value": rate, "unit": "interactions/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"w+grad at {m} sampled points and w at {m} sampled octree corners, "
                      f"each against all {n} sources (FP64, OpenMP)",
            "extrapolated_s_per_iteration": it_s, "corners": int(len(C))}


def one_step(args):
    """One iteration of the workload: the launch shapes of a bench step."""
    import torch
    from paper_2405_13839_gb300 import dwg
    W = workload(args)
    h = dwg.dwg_create(W["points"])
    dwg.dwg_set_weights(h, W["weights"])
    dwg.dwg_set_params(h, W["kernel"], W["eps"], W["lambda"], W["max_iters"], W["tol"])
    dwg.dwg_set_update(h, W["depth"], 10, dwg.DWG_UPDATE_LEVELSET)
    dwg.dwg_set_tree(h, W["path"], W["theta"])
    dwg.dwg_set_init(h, dwg.DWG_INIT_RANDOM, 1)
    iso, stat = dwg.dwg_step(h)
    torch.cuda.synchronize()
    dwg.dwg_destroy(h)
    print(json.dumps({"one_step": W["name"], "iso": iso, "stat": stat}))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.one_step:
        one_step(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        if rank != 0:
            return
        W = workload(args)
        n = len(W["points"])
        for _ in range(args.warmup):
            cpu_baseline(W, None, budget_s=1.0)
        vals = []
        t0 = time.perf_counter()
        last = None
        for _ in range(args.steps):
            last = cpu_baseline(W, None, budget_s=8.0)
            vals.append(last["value"])
        wall = time.perf_counter() - t0
        v = statistics.median(vals)
        line = {"impl": "reference", "metric": "GWN+grad interactions/s", "value": v,
                "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": W["name"], "points": n, "kernel": "plain" if W["kernel"] == 0 else "screened",
                           "path": "all-pairs", "depth": W["depth"]},
                "cpu_baseline": {k: last[k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": "interactions/s"},
                "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    r = run_ours(args, rank, world, local)
    if rank != 0:
        return
    W = r["W"]
    n = len(W["points"])
    cpu = None
    if world == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline(W, r["nc"])
        except Exception as e:  # the oracle is a reported baseline only
            cpu = {"error": str(e)}
    ms_per_step = 1e3 * r["dev_s"] / args.steps
    line = {
        "metric": "GWN+grad interactions/s", "value": r["value"], "unit": "interactions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": W["name"], "points": n, "corners": r["nc"],
                   "kernel": "plain" if W["kernel"] == 0 else "screened lambda=10",
                   "path": "all-pairs exact, compensated FP32", "depth": W["depth"], "knn": 10,
                   "tol_deg": W["tol"], "init": "random seed 1", "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MiB write) before every step"},
        "s_to_converged_normals": ms_per_step / 1e3,
        "iterations": r["iters"][0],
        "interactions_per_step": r["value"] * r["dev_s"] / args.steps / world,
        "roofline": r["roof"], "cpu_baseline": cpu, "clocks": r["clocks"], "e2e": r["e2e"],
        "gpu_launches": r["launches"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
