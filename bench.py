#!/usr/bin/env python
"""Converged null vectors per second at relative residual 1e-8.

Workload (default): graph Laplacian with n = 1,000,000 nodes, 500 disjoint
components (power-law sizes, minimum 50), each the union of 4 random Hamiltonian
cycles (mean degree 8), unit weights, FP64 CSR; B = A + eps D (SPD form), block
size d = 1, restart length 120, lock tolerance 1e-10, plain FP64 GPU path.

One step = one ns_solve (Lanczos with locking + FP64 refinement + re-
orthonormalization) on the matrix already resident in HBM.  A step counts only
if the nullity is 500 and max_j ||A x_j|| / ||A||_2 <= 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|mixed] [--d 1|4]
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged null vecs/s at rel. residual 1e-8"
UNIT = "null_vecs/s"
HBM_GBS = 6783.5          # measured copy bandwidth of the GB300s
FP64_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 4 FP64 flop/clk (1.25 TF nominal) x 2.07 GHz


def peaks():
    p = {"hbm_gbs": HBM_GBS, "src": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        p["hbm_gbs"] = float(j["hbm_gbs"])
        p["src"] = "measured"
    except Exception:
        pass
    return p


def workload_params(args):
    return dict(n=args.n, ncomp=args.components, seed=0x2407046340 + 1, solver_seed=1001, d=args.d, restart=120,
                tol=1e-10, precision=args.precision)


def describe(p, A):
    return {"workload": f"graph Laplacian n={p['n']:,} ({p['ncomp']} components, power-law sizes, mean degree 8), "
                        f"SPD form A+eps*D, {p['precision'].upper()} path, d={p['d']}, restart {p['restart']}",
            "n": p["n"], "nnz": int(A.nnz), "components": p["ncomp"], "d": p["d"], "restart_len": p["restart"],
            "tol": p["tol"], "eps": 1e-3, "precision": p["precision"],
            "l2": "inputs larger than L2 (Lanczos basis %.2f GB, locked set up to %.2f GB, matrix %.2f GB)"
                  % (p["n"] * (p["restart"] + p["d"]) * 8 * 2 / 1e9, p["n"] * p["ncomp"] * 8 / 1e9,
                     A.nnz * 12 / 1e9)}


# ---------------------------------------------------------------- clocks -----

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- CPU oracle leg --

ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from workloads import laplacian_cycle_components
from oracle import lanczos_nullspace
w = laplacian_cycle_components({seed}, {n}, {k}, 8, "powerlaw", 50)
A = w.A.to_scipy()
t = time.perf_counter()
r = lanczos_nullspace(A, "spd", {d}, {restart}, tol={tol}, seed={sseed})
dt = time.perf_counter() - t
res = float(np.linalg.norm(A @ r.X) / r.normA) if r.N else 0.0
print(json.dumps(dict(N=int(r.N), expect={k}, seconds=dt, matvecs=int(r.stats["matvecs"]), residual=res)))
"""


def run_oracle_sample(p, n, k):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, seed=p["seed"], n=n, k=k, d=p["d"], restart=p["restart"],
                                 tol=p["tol"], sseed=p["solver_seed"])
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(p, n=60_000, k=30):
    r = run_oracle_sample(p, n, k)
    return {"value": r["N"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"same generator at n={n:,}, {k} components (nullity {r['N']}, expected {k}), "
                      f"single-threaded FP64 oracle, {r['seconds']:.1f} s, {r['matvecs']} matvecs, "
                      f"residual {r['residual']:.1e}"}


# ------------------------------------------------------------- reference ----

def bench_reference(args, rank):
    if rank != 0:
        return
    p = workload_params(args)
    n, k = 30_000, 15
    times, Ns = [], []
    for i in range(args.warmup + args.steps):
        r = run_oracle_sample(p, n, k)
        if i >= args.warmup:
            times.append(r["seconds"])
            Ns.append(r["N"])
    tot = sum(times)
    val = sum(Ns) / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": describe(p, _FakeA(9 * p["n"]))["workload"],
                                            "oracle_sample": f"n={n:,}, {k} components"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"same generator at n={n:,}, {k} components, single-threaded FP64 oracle"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class _FakeA:
    def __init__(self, nnz):
        self.nnz = nnz


# -------------------------------------------------------------------- ours --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--d", type=int, default=1)
    ap.add_argument("--profile-every", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=1_000_000, help="nodes (a smaller case is for profiling only)")
    ap.add_argument("--components", type=int, default=500)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        bench_reference(args, rank)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2407_04634_gb300 import nullspace as ns
    from workloads import laplacian_cycle_components

    p = workload_params(args)
    w = laplacian_cycle_components(p["seed"], p["n"], p["ncomp"], 8, "powerlaw", 50)
    A = w.A
    h = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, p["solver_seed"], "spd")
    stream = torch.cuda.current_stream()

    def one_step(profile=0):
        r = h.solve(p["d"], p["restart"], p["tol"], check=False, precision=p["precision"], profile=profile)
        return r

    def valid(r):
        return (r.status == ns.NS_OK and r.nullity == p["ncomp"] and r.stats.get("refine_resid_max", 1) <= 1e-8)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [one_step(profile=args.profile_every) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = h.profile()  # kernel classes of the last timed step
    units = sum(r.nullity for r in results if valid(r))
    all_valid = all(valid(r) for r in results)
    t_max = ms
    if dist:
        tt = torch.tensor([ms, float(units)], device="cuda", dtype=torch.float64)
        tmax = tt.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        t_max, units = float(tmax[0]), float(tt[1])
    value = units / (t_max / 1e3)
    launches = sum(r.stats.get("kernel_launches", 0) for r in results)

    # roofline of the dominant kernel class and of the B-apply (SpMM) class
    pk = peaks()
    dom = max(prof, key=lambda c: c["ms_total_est"])

    def roof(c):
        if c["name"] == "b_apply":
            ach = c["bytes_per_launch"] / (c["ms_per_launch"] / 1e3) / 1e9
            return {"kernel": c["name"], "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_src": pk["src"],
                    "bytes_per_launch": c["bytes_per_launch"], "ms_per_launch": c["ms_per_launch"],
                    "launches": c["launches"], "sampled": c["sampled"]}
        if p["precision"] == "fp64":
            ach = c["flops_per_launch"] / (c["ms_per_launch"] / 1e3) / 1e12
            return {"kernel": c["name"], "bound": "alu", "achieved": ach, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_TFLOPS, "traffic": None,
                    "peak_src": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz",
                    "flops_per_launch": c["flops_per_launch"], "ms_per_launch": c["ms_per_launch"],
                    "launches": c["launches"], "sampled": c["sampled"]}
        ach = c["bytes_per_launch"] / (c["ms_per_launch"] / 1e3) / 1e9
        return {"kernel": c["name"], "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_src": pk["src"],
                "bytes_per_launch": c["bytes_per_launch"], "ms_per_launch": c["ms_per_launch"],
                "launches": c["launches"], "sampled": c["sampled"]}

    roofline = roof(dom)
    spmm = roof(next(c for c in prof if c["name"] == "b_apply"))

    # end-to-end through the public API: pinned host CSR -> ns_create -> ns_solve -> basis to pinned host
    rp = torch.from_numpy(A.rowptr).pin_memory()
    ci = torch.from_numpy(A.colind).pin_memory()
    va = torch.from_numpy(A.vals).pin_memory()
    out = torch.empty((p["ncomp"], p["n"]), dtype=torch.float64).pin_memory()
    h2d = rp.numel() * 8 + ci.numel() * 4 + va.numel() * 8
    d2h = out.numel() * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_units = 0
    for _ in range(args.e2e_steps):
        he = ns.Handle(rp.numpy(), ci.numpy(), va.numpy(), A.m, A.n, p["solver_seed"], "spd")
        r = he.solve(p["d"], p["restart"], p["tol"], check=False, precision=p["precision"])
        if valid(r):
            he.lib.ns_basis(he.h, ns.C.c_void_p(out.data_ptr()), p["n"], 0)
            e2e_units += r.nullity
        he.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "steps": args.e2e_steps}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_baseline(p)
        except Exception as e:  # reported, not hidden
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    last = results[-1].stats
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if p["precision"] == "fp64" else "f32+f64",
            "data": "synthetic", "config": describe(p, A), "valid": all_valid,
            "gpu_launches": int(launches), "clocks": clk, "roofline": roofline, "spmm_roofline": spmm,
            "e2e": e2e, "cpu_baseline": cpu,
            "solve": {k: last.get(k) for k in ("nullity", "matvecs", "restarts", "reorth_X", "reorth_Z",
                                               "lock_events", "refine_iters_max", "refine_resid_max",
                                               "orth_before", "orth_after", "t_lanczos_ms", "t_refine_ms")},
            "kernel_classes": [{k: c[k] for k in ("name", "launches", "sampled", "ms_per_launch", "ms_total_est")}
                               for c in prof]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
