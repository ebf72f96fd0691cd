#!/usr/bin/env python
"""Converged null vectors per second at relative residual 1e-8.

Workload (default): graph Laplacian with n = 1,000,000 nodes, 500 disjoint
components (power-law sizes, minimum 50), each the union of 4 random Hamiltonian
cycles (mean degree 8), unit weights, FP64 CSR; B = A + eps D (SPD form), block
size d = 1, restart length 120, lock tolerance 1e-10, plain FP64 GPU path.

Other workloads: --workload incidence (8e6 x 2e6 incidence matrix, nullity 1000,
d = 4, restart 160, mixed path) and --workload copies (3e6 x 2e6 matrix with 300
planted column copies, d = 2, restart 150, mixed path).

One step = one ns_solve (Lanczos with locking + FP64 refinement + re-
orthonormalization) on the matrix already resident in HBM.  A step counts only
if the nullity equals the planted one and max_j ||A x_j|| / ||A||_2 <= 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload laplacian|incidence|copies] [--precision fp64|mixed] [--d D]
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
HBM_GBS = 6800.0          # fallback copy bandwidth when MEASURED_PEAKS.json is absent
FP64_TFLOPS_DERIVED = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 4 FP64 flop/clk x 2.07 GHz (fallback only)


def alu_peaks(ns, local):
    """FP64 and FP32 FMA throughput measured on this device (ns_fma_peak), in TFLOP/s,
    with the median SM clock sampled while it ran (so a rate can be rescaled to the
    clock of another timed region: the FMA rate is proportional to the SM clock)."""
    out = {}
    for prec in ("fp64", "mixed"):
        clocks = ClockSampler(local)
        clocks.start()
        try:
            vals = [ns.fma_peak(prec) for _ in range(3)]
            val, src = max(vals), "measured: ns_fma_peak (8 FMA chains x 256 threads x 8 CTAs per SM), best of 3"
        except Exception as e:  # reported, not hidden
            val, src = (FP64_TFLOPS_DERIVED if prec == "fp64" else None), f"derived (measurement failed: {e})"
        clk = clocks.stop()
        out[prec] = (val, src, clk.get("sm_mhz"))
    return out


def at_clock(peak, peak_mhz, mhz):
    """A pipe's peak measured at peak_mhz, rescaled to the SM clock mhz of a timed region."""
    if peak is None or not peak_mhz or not mhz:
        return peak
    return peak * mhz / peak_mhz


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


WORKLOADS = {
    # configuration 2 (the default): graph Laplacian, SPD form, plain FP64 path
    "laplacian": dict(cfg=2, mode="spd", d=1, restart=120, precision="fp64", cpu_scale=0.06, ref_scale=0.03),
    # configuration 3: +-1 edge-vertex incidence matrix, normal form, precision form
    "incidence": dict(cfg=3, mode="normal", d=4, restart=160, precision="mixed", cpu_scale=0.02, ref_scale=0.01),
    # configuration 4: rectangular N(0,1) matrix with planted sign-flipped column copies
    "copies": dict(cfg=4, mode="normal", d=2, restart=150, precision="mixed", cpu_scale=0.01, ref_scale=0.005),
    # configuration 5: 4,096 independent Laplacians in one persistent launch (batched form)
    "batched": dict(cfg=5, mode="spd", d=1, restart=40, precision="mixed", cpu_scale=0.01, ref_scale=0.005,
                    tol=1e-5),
    # not a benchmark configuration: 500 2-D grid Laplacians (sides 15-30, ~2.6e5 nodes),
    # badly conditioned, solved with the outer IC(0) preconditioner (Sec. 4.4.2)
    "grid": dict(cfg=6, mode="spd", d=1, restart=120, precision="fp64", cpu_scale=0.02, ref_scale=0.01,
                 precond=1),
}


def ncu_traffic_ratio(cls):
    """DRAM bytes / algorithmic bytes of a kernel class from the committed ncu capture,
    or None when the kernel sources changed since the capture (or no capture exists)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            j = json.load(f)
        h = hashlib.sha256(b"".join(open(os.path.join(ROOT, x), "rb").read() for x in j["source_files"])).hexdigest()
        if h != j["source_sha256"] or cls not in j["classes"]:
            return None
        return float(j["classes"][cls]["ratio"])
    except Exception:
        return None


def workload_params(args):
    wl = WORKLOADS[args.workload]
    return dict(name=args.workload, cfg=wl["cfg"], mode=wl["mode"], scale=args.scale,
                d=args.d or wl["d"], restart=wl["restart"], tol=wl.get("tol", 1e-10),
                precision=args.precision or wl["precision"], solver_seed=1000 + wl["cfg"] - 1,
                cpu_scale=wl["cpu_scale"], ref_scale=wl["ref_scale"],
                precond=args.precond if args.precond is not None else wl.get("precond", 0))


def build_workload(p):
    from workloads import make_config
    w, _ = make_config(p["cfg"], p["scale"])
    return w


def describe(p, w):
    A = w.A
    kind = {"laplacian": "graph Laplacian (power-law component sizes, mean degree 8), SPD form A+eps*D",
            "incidence": "oriented edge-vertex incidence matrix (mean degree 8, uniform component sizes), "
                         "normal form A^T A+eps*D",
            "copies": "rectangular sparse N(0,1) matrix, 12 nnz/row, planted sign-flipped column copies, "
                      "normal form A^T A+eps*D",
            "grid": "graph Laplacian of 2-D grid components (sides 15-30), SPD form"}[p["name"]]
    if p.get("precond"):
        kind += ", outer IC(0) preconditioning B_R = L^-1 A~ L^-T + eps*D (diagcomp 0.1)"
    vec = 4 if p["precision"] == "mixed" else 8
    return {"workload": f"{kind}; m={A.m:,} n={A.n:,} nnz={A.nnz:,}, nullity {w.nullity}; "
                        f"{p['precision'].upper()} path, d={p['d']}, restart {p['restart']}, tol {p['tol']:g}",
            "m": int(A.m), "n": int(A.n), "nnz": int(A.nnz), "nullity": int(w.nullity), "d": p["d"],
            "restart_len": p["restart"], "tol": p["tol"], "eps": 1e-3, "precision": p["precision"],
            "mode": p["mode"], "precond": int(p.get("precond", 0)),
            "l2": "inputs larger than L2 (Lanczos basis %.2f GB, locked set up to %.2f GB, matrix %.2f GB)"
                  % (A.n * (p["restart"] + p["d"]) * vec * 2 / 1e9, A.n * w.nullity * vec / 1e9,
                     A.nnz * (4 + vec) / 1e9)}


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
from workloads import make_config
from oracle import lanczos_nullspace
w, _ = make_config({cfg}, {scale})
A = w.A.to_scipy()
t = time.perf_counter()
r = lanczos_nullspace(A, {mode!r}, {d}, {restart}, tol={tol}, seed={sseed}, precond={precond})
dt = time.perf_counter() - t
res = float(np.linalg.norm(A @ r.X) / r.normA) if r.N else 0.0
print(json.dumps(dict(N=int(r.N), expect=int(w.nullity), n=int(A.shape[1]), seconds=dt,
                      matvecs=int(r.stats["matvecs"]), residual=res)))
"""


def rank_slice(count: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced slice [lo, hi) of `count` independent instances for `rank`."""
    return rank * count // world, (rank + 1) * count // world


def reduce_over_ranks(ms: float, units: float, dist, device) -> tuple[float, float]:
    """(max over ranks of the timed milliseconds, sum over ranks of the converged units)."""
    if dist is None:
        return ms, units
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def run_oracle_sample(p, scale):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    snippet = BATCH_ORACLE_SNIPPET if p["cfg"] == 5 else ORACLE_SNIPPET
    code = snippet.format(root=ROOT, cfg=p["cfg"], scale=scale, mode=p["mode"], d=p["d"],
                          restart=p["restart"], tol=p["tol"], sseed=p["solver_seed"],
                          precond=0.1 if p.get("precond") else None)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


BATCH_ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from workloads import make_config
from oracle import lanczos_nullspace
ws, _ = make_config(5, {scale})
N = E = n = mv = 0
res = 0.0
t = time.perf_counter()
for i, w in enumerate(ws):
    A = w.A.to_scipy()
    r = lanczos_nullspace(A, "spd", 1, {restart}, tol={tol}, seed={sseed} + i)
    N += int(r.N); E += int(w.nullity); n += int(A.shape[1]); mv += int(r.stats["matvecs"])
    if r.N:
        res = max(res, float(np.linalg.norm(A @ r.X) / r.normA))
dt = time.perf_counter() - t
print(json.dumps(dict(N=N, expect=E, n=n, seconds=dt, matvecs=mv, residual=res, instances=len(ws))))
"""


def cpu_baseline(p):
    r = run_oracle_sample(p, p["cpu_scale"])
    if p["cfg"] == 5:
        return {"value": r["N"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the first {r['instances']} of the 4,096 instances (sum n={r['n']:,}, nullity "
                          f"{r['N']}, expected {r['expect']}), single-threaded FP64 oracle, {r['seconds']:.1f} s, "
                          f"{r['matvecs']} matvecs, residual {r['residual']:.1e}"}
    return {"value": r["N"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"same generator scaled by {p['cpu_scale']} (n={r['n']:,}, nullity {r['N']}, "
                      f"expected {r['expect']}), single-threaded FP64 oracle, {r['seconds']:.1f} s, "
                      f"{r['matvecs']} matvecs, residual {r['residual']:.1e}"}


# ------------------------------------------------------------- reference ----

def bench_reference(args, rank):
    if rank != 0:
        return
    p = workload_params(args)
    times, Ns, last = [], [], None
    for i in range(args.warmup + args.steps):
        r = run_oracle_sample(p, p["ref_scale"])
        last = r
        if i >= args.warmup:
            times.append(r["seconds"])
            Ns.append(r["N"])
    tot = sum(times)
    val = sum(Ns) / tot
    if p["cfg"] == 5:
        sample = (f"the first {last['instances']} of the 4,096 instances (sum n={last['n']:,}, nullity "
                  f"{last['N']}), single-threaded FP64 oracle, one solve per instance")
    else:
        sample = (f"same generator scaled by {p['ref_scale']} (n={last['n']:,}, nullity {last['N']}), "
                  f"single-threaded FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{p['name']} (configuration {p['cfg']}), oracle sample",
                                            "oracle_sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def closed_form_sine(w, X):
    """Largest principal-angle sine between the computed basis X (n x N, CUDA tensor) and
    the workload's known null space: component indicators (Laplacians, incidence
    matrices) or (e_src + e_copy)/sqrt(2) (planted column copies).  Computed on the
    device after the timed region: ||(I - U U^T) X||_2 from the N x N Gram matrix."""
    import numpy as np
    import torch
    if w.labels is not None:
        lab = torch.as_tensor(np.asarray(w.labels), device=X.device, dtype=torch.long)
        k = int(lab.max()) + 1
        sums = torch.zeros((k, X.shape[1]), dtype=X.dtype, device=X.device).index_add_(0, lab, X)
        cnt = torch.bincount(lab, minlength=k).to(X.dtype)
        PX = (sums / cnt[:, None])[lab]
    elif w.copy_pairs is not None:
        pr = torch.as_tensor(np.asarray(w.copy_pairs), device=X.device, dtype=torch.long)
        PX = torch.zeros_like(X)
        avg = 0.5 * (X[pr[:, 0]] + X[pr[:, 1]])
        PX[pr[:, 0]] = avg
        PX[pr[:, 1]] = avg
    else:
        return None
    R = X - PX
    G = R.T @ R
    return float(np.sqrt(max(np.linalg.eigvalsh(G.double().cpu().numpy())[-1], 0.0)))


def device_csr(A, device="cuda"):
    """scipy CSR -> torch sparse CSR (FP64) on the device (for the independent checks)."""
    import numpy as np
    import torch
    A = A.tocsr()
    return torch.sparse_csr_tensor(torch.as_tensor(A.indptr.astype(np.int64), device=device),
                                   torch.as_tensor(A.indices.astype(np.int64), device=device),
                                   torch.as_tensor(A.data.astype(np.float64), device=device),
                                   size=A.shape, dtype=torch.float64)


def norm2_power(Ad, AdT, iters=150):
    """||A||_2 by power iteration on A^T A (a lower bound: residual ratios are over-, never
    under-estimated).  AdT is None for a symmetric A."""
    import torch
    g = torch.Generator(device=Ad.device).manual_seed(0)
    x = torch.randn((Ad.shape[1], 1), dtype=torch.float64, device=Ad.device, generator=g)
    x /= torch.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = Ad @ x
        y = (AdT @ y) if AdT is not None else (Ad @ y)
        lam = float(torch.linalg.norm(y))
        x = y / lam
    return lam ** 0.5


def residual_ratio(Ad, X, normA, chunk=64):
    """||A X||_F / ||A||_2 for a device basis X (n x N), in column chunks."""
    import torch
    tot = 0.0
    for c0 in range(0, X.shape[1], chunk):
        R = Ad @ X[:, c0:c0 + chunk].contiguous()
        tot += float(torch.sum(R * R))
    return tot ** 0.5 / normA


def d_sweep(ns, h, w, p, args, local):
    """Block size at a fixed Krylov dimension (Sec. 5.3.1, Table tabCH): for each d in
    1, 2, 4, 8 one timed solve (CUDA events on the current stream; d = 1 after one
    untimed warm-up solve) at restart length dim K = the workload's restart length
    rounded down to a multiple of 8; reports B applications (counted per column, as
    the table does), restarts, the solve time and the nullity, and which d the rule
    d = dim K / 16 picks.  Solves with d > 1 stop at 3 x the B applications of d = 1."""
    import torch
    R = 8 * (p["restart"] // 8)
    precision = args.precision or p["precision"]
    stream = torch.cuda.current_stream()
    rows = []
    cap = 0  # B applications allowed per solve: 3 x those of d = 1 (a stalled d is reported, not waited out)
    for d in (1, 2, 4, 8):
        def one():
            return h.solve(d, R, p["tol"], check=False, precision=precision, precond=p["precond"], max_matvec=cap)
        if d == 1:
            one()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = one()
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ok = r.status == ns.NS_OK and r.nullity == w.nullity and r.stats.get("refine_resid_max", 1) <= 1e-8
        if d == 1:
            cap = 3 * int(r.stats.get("matvecs", 0))
        rows.append({"d": d, "status": ns.STATUS.get(r.status, r.status), "matvec_cap": cap if d > 1 else None,
                     "matvecs": r.stats.get("matvecs"), "restarts": r.stats.get("restarts"),
                     "ms": e0.elapsed_time(e1), "nullity": r.nullity, "valid": ok,
                     "t_lanczos_ms": r.stats.get("t_lanczos_ms"), "sm_mhz": clk.get("sm_mhz"),
                     "reasons": clk.get("reasons")})
    # the library's choice for d = 0 (one cycle is enough to read it back)
    rule = h.solve(0, R, p["tol"], check=False, precision=precision, precond=p["precond"],
                   max_matvec=1).stats.get("d")
    print(json.dumps({"sweep": "block size d at fixed dim K", "dim_K": R, "precision": precision,
                      "rule_d": rule, "rows": rows,
                      "config": describe(p, w)}), flush=True)


def large_block(ns, h, w, p, args, local):
    """Small-block (perturbed, the workload's d) against the large-block variant of
    Sec. 5.3.2 (eps = 0, d = 8 >= N; Table tabCHLB) on a workload with nullity <= 8: one
    untimed and one timed solve each (CUDA events on the current stream)."""
    import torch
    if w.nullity > 8:
        raise SystemExit("--large-block needs a nullity <= 8 (the kernels' largest block); use a small --scale")
    precision = args.precision or p["precision"]
    stream = torch.cuda.current_stream()
    rows = []
    for name, d, R, eps in (("small-block", p["d"], p["restart"], 1e-3), ("large-block", 8, 64, 0.0)):
        def one():
            return h.solve(d, R, p["tol"], check=False, precision=precision, eps=eps)
        one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = one()
        e1.record(stream)
        torch.cuda.synchronize()
        rows.append({"variant": name, "d": d, "restart_len": R, "eps": eps, "status": ns.STATUS.get(r.status),
                     "nullity": r.nullity, "matvecs": r.stats.get("matvecs"), "restarts": r.stats.get("restarts"),
                     "ms": e0.elapsed_time(e1), "refine_resid_max": r.stats.get("refine_resid_max")})
    print(json.dumps({"comparison": "small-block vs large-block (Sec. 5.3.2)", "precision": precision,
                      "rows": rows, "config": describe(p, w)}), flush=True)


def kernel_probe(ns, h, w, p):
    """A handful of hot-kernel launches on the workload's inputs (for ncu captures):
    three B-applies in each precision and every SpMM schedule, the thick-restart
    product with every kernel (n x min(restart, 128) times half as many Ritz vectors),
    and CGS2 projections of 2- and 8-wide panels against 256 vectors in FP64 pairs,
    FP64 and FP32."""
    import numpy as np
    rng = np.random.default_rng(0)
    n = w.A.n
    out = {}
    X = rng.standard_normal((n, p["d"]))
    for prec in ("fp64", "mixed"):
        t = time.perf_counter()
        for _ in range(3):
            h.apply_B(X, 1e-3, prec)
        out[f"apply_B_{prec}_s"] = (time.perf_counter() - t) / 3
        for sched in (128, 64, 1, 2, 4, 8):  # every SpMM schedule (sliced ELLPACK, TMA-staged, lanes per row)
            try:
                h.apply_B(X, 1e-3, prec, sched)
            except ns.NullspaceError:  # no sliced-ELLPACK copy for this matrix
                pass
    # thick-restart product Z V_Z(:, keep) at the workload's restart length, every kernel
    R = p["restart"] - p["restart"] % 16 if p["restart"] > 128 else p["restart"]
    R = min(R, 128)
    Zr = rng.standard_normal((n, R)) / np.sqrt(n)
    Vr, _ = np.linalg.qr(rng.standard_normal((R, R)))
    keep = np.arange(R // 2, dtype=np.int32)
    for prec, gemm in (("fp64", "tc_exact"), ("mixed", "tc3"), ("mixed", "tc2"), ("fp64", "cuda_cores"),
                       ("mixed", "cuda_cores")):
        t = time.perf_counter()
        ns.restart_product(Zr, Vr, keep, 0, 1, prec, gemm)
        out[f"restart_{prec}_{gemm}_s"] = time.perf_counter() - t
    del Zr
    V, _ = np.linalg.qr(rng.standard_normal((n, 256)))
    for w in (2, 8):  # the merged [Q_j | Q_j+1] panel at d = 1 and d = 4
        W = rng.standard_normal((n, w))
        for prec in ("fp64_pairs", "fp64", "mixed"):
            t = time.perf_counter()
            ns.project(V, W, prec)
            out[f"project_w{w}_{prec}_s"] = time.perf_counter() - t
    print(json.dumps({"kernel_probe": p["name"], **out}), flush=True)


# ----------------------------------------------------------------- batched --

def bench_batched(args, world, rank, local):
    """Configuration 5: 4,096 Laplacians (n log-uniform in [200, 20000], 1-8 cycle-union
    components each) in one persistent launch per step, replayed from a CUDA graph.
    Ranks take disjoint slices of the instance list (weak scaling, no collective)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2407_04634_gb300 import nullspace as ns
    from workloads import make_config
    from oracle import norm2_A  # validity check of sampled outputs, outside the timed region

    p = workload_params(args)
    ws_all, _ = make_config(5, args.scale)
    lo, hi = rank_slice(len(ws_all), world, rank)
    ws = ws_all[lo:hi]  # contiguous slice: global instance i keeps the key solver_seed + i
    seed = p["solver_seed"] + lo
    n = np.array([w.A.n for w in ws], dtype=np.int64)
    rp = np.concatenate([w.A.rowptr for w in ws])
    ci = np.concatenate([w.A.colind for w in ws])
    va = np.concatenate([w.A.vals for w in ws]).astype(np.float32)  # FP32 CSR, as given (vals_is_fp32)
    nnz = np.array([w.A.nnz for w in ws], dtype=np.int64)
    expect = np.array([w.nullity for w in ws])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = ns.Batch.from_arrays(n, rp, ci, va, seed)

        def step(**kw):
            st = b.solve(p["restart"], p["tol"], check=False, eps=1e-3, batch_block=args.batch_block, **kw)
            N, S, I = b.results()
            return st, N, S, I

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        outs = [step() for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    bst = b.stats()

    def valid(o):
        st, N, S, _ = o
        return st == ns.NS_OK and (S == 0).all() and (N == expect).all()

    units = float(sum(int(o[1].sum()) for o in outs if valid(o)))
    all_valid = all(valid(o) for o in outs)
    # sampled residual check of the last step (outside the timed region)
    worst = 0.0
    for k in range(0, len(ws), max(1, len(ws) // 24)):
        X = b.basis(k)
        A = ws[k].A.to_scipy()
        if X.shape[1]:
            worst = max(worst, float(np.linalg.norm(A @ X) / norm2_A(A, "spd")))
    all_valid = all_valid and worst <= 1e-8
    t_max, units = reduce_over_ranks(ms, units, dist, "cuda")
    value = units / (t_max / 1e3) if all_valid else 0.0

    # roofline of the persistent kernel: algorithmic bytes of the B applications
    I = outs[-1][3]
    mv = I[:, 0].astype(np.float64)
    bytes_step = float((mv * (8.0 * nnz + 28.0 * n)).sum())
    ms_kernel = bst["t_solve_ms"]
    ach = bytes_step / (ms_kernel / 1e3) / 1e9
    pk = peaks()
    roofline = {"kernel": "k_batched", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_src": pk["src"],
                "bytes_per_launch": bytes_step, "ms_per_launch": ms_kernel,
                "note": "bytes = sum_i matvecs_i (8 nnz_i + 28 n_i); each CTA's instance is largely L2-resident, "
                        "so the kernel is bound by CTA-wide reductions, not HBM"}

    # end-to-end: pinned host CSR -> ns_batch_create -> ns_batch_solve -> every basis to pinned host
    rp_p = torch.from_numpy(rp).pin_memory()
    ci_p = torch.from_numpy(ci).pin_memory()
    va_p = torch.from_numpy(va).pin_memory()
    out = torch.empty(int((n * expect).sum()), dtype=torch.float64).pin_memory()
    h2d = rp.nbytes + ci.nbytes + va.nbytes + n.nbytes
    d2h = out.numel() * 8 + len(ws) * (4 + 4 + 40)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_units = 0
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            be = ns.Batch.from_arrays(n, rp_p.numpy(), ci_p.numpy(), va_p.numpy(), seed)
            st = be.solve(p["restart"], p["tol"], check=False, eps=1e-3, batch_block=args.batch_block)
            N, S, _ = be.results()
            if st == ns.NS_OK and (N == expect).all():
                be.basis_packed(out.numpy())  # every basis, one device-to-host transfer
                e2e_units += int(N.sum())
            be.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "steps": args.e2e_steps}

    # the same instances through the single-instance FP64 path, one ns_solve each (a sample)
    every = max(1, len(ws) // max(1, args.loop_sample))
    loop_t, loop_N, loop_ok = 0.0, 0, True
    picked = list(range(0, len(ws), every)) if args.loop_sample > 0 else []
    with torch.cuda.stream(stream):
        for k in picked:
            A = ws[k].A
            hk = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, seed + k, "spd")
            hk.solve(1, p["restart"], p["tol"], check=False, precision="fp64")  # warm-up of this handle
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = hk.solve(1, p["restart"], p["tol"], check=False, precision="fp64")
            e1.record(stream)
            torch.cuda.synchronize()
            loop_t += e0.elapsed_time(e1) / 1e3
            loop_ok = loop_ok and r.status == ns.NS_OK and r.nullity == ws[k].nullity
            loop_N += r.nullity
            hk.close()
    loop = {"value": loop_N / loop_t if loop_t > 0 else None, "unit": UNIT, "valid": bool(loop_ok),
            "sample": f"{len(picked)} of the {len(ws)} instances (every {every}th), "
                      f"one FP64 ns_solve each (d=1, restart {p['restart']}, tol {p['tol']:g}), "
                      f"CUDA-event time of the solve, warm handle"}

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
    mats = 8 * int(nnz.sum()) + 12 * int(n.sum())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{len(ws_all):,} independent graph Laplacians, n log-uniform in [200, 20000], "
                                   f"1-8 components of 3 random Hamiltonian cycles each (mean degree 6), "
                                   f"sum n={int(sum(w.A.n for w in ws_all)):,}, sum nnz="
                                   f"{int(sum(w.A.nnz for w in ws_all)):,}, total nullity "
                                   f"{int(sum(w.nullity for w in ws_all))}; batched persistent launch "
                                   f"(graph replay), d=1, restart {p['restart']}, tol {p['tol']:g}",
                       "instances": len(ws_all), "d": 1, "restart_len": p["restart"], "tol": p["tol"],
                       "eps": 1e-3, "precision": "mixed", "mode": "spd",
                       "l2": "inputs larger than L2 (matrices %.2f GB on the device)" % (mats / 1e9)},
            "valid": bool(all_valid), "residual_max_sampled": worst,
            "gpu_launches": int(bst["kernel_launches"]) * args.steps, "clocks": clk, "roofline": roofline,
            "e2e": e2e, "cpu_baseline": cpu, "loop_fp64": loop,
            "batched_vs_loop_fp64": (value / loop["value"]) if loop["value"] else None,
            "batch": {k: bst[k] for k in ("lanes", "block", "grid", "blocks_per_sm", "graph", "t_solve_ms", "t_tune_ms",
                                          "matvecs_total", "matvecs_max", "total_nullity", "failed")},
            "phase_share": {k: float(I[:, 5 + j].sum() / max(1, I[:, 4].sum()))
                            for j, k in enumerate(ns.BATCH_ISTATS[5:11])},
            "jacobi_sweeps_per_restart": {"fp32": float(I[:, 11].sum() / max(1, I[:, 1].sum())),
                                          "fp64": float(I[:, 12].sum() / max(1, I[:, 1].sum()))}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# -------------------------------------------------------------------- ours --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="laplacian", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"])
    ap.add_argument("--d", type=int, default=None)
    ap.add_argument("--profile-every", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision sub-record")
    ap.add_argument("--fp64-products", type=int, default=0, choices=[0, 1],
                    help="FP64 path's Gram-Schmidt products: 0 compensated FP32 pairs (default), 1 FP64 FMA")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (< 1 is for profiling only)")
    ap.add_argument("--kernel-probe", action="store_true", help="launch a few hot kernels, no bench line")
    ap.add_argument("--precond", type=int, default=None, choices=[0, 1],
                    help="SPD workloads: outer IC(0) preconditioning (default: on for grid, off otherwise)")
    ap.add_argument("--large-block", action="store_true",
                    help="small-block vs the unperturbed large-block variant (nullity <= 8), one line, no bench line")
    ap.add_argument("--d-sweep", action="store_true",
                    help="block sizes 1, 2, 4, 8 at a fixed dim K (Sec. 5.3.1), one line, no bench line")
    ap.add_argument("--loop-sample", type=int, default=32,
                    help="batched workload: instances solved one by one with the FP64 path for comparison")
    ap.add_argument("--batch-block", type=int, default=0, choices=[0, 128, 256],
                    help="threads per CTA of the batched kernel (0 = library default)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        bench_reference(args, rank)
        return
    if args.workload == "batched":
        bench_batched(args, world, rank, local)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2407_04634_gb300 import nullspace as ns
    p = workload_params(args)
    w = build_workload(p)
    A = w.A
    # configuration 4's values are FP32 numbers and go in as FP32 (vals_is_fp32)
    vals_in = A.vals.astype(np.float32) if p["cfg"] == 4 else A.vals
    h = ns.Handle(A.rowptr, A.colind, vals_in, A.m, A.n, p["solver_seed"], p["mode"])
    stream = torch.cuda.current_stream()
    if args.kernel_probe:
        kernel_probe(ns, h, w, p)
        return
    if args.d_sweep:
        d_sweep(ns, h, w, p, args, local)
        return
    if args.large_block:
        large_block(ns, h, w, p, args, local)
        return

    alu = alu_peaks(ns, local)
    fp64_peak_raw, fp64_src, fp64_mhz = alu["fp64"]

    def valid(r):
        return (r.status == ns.NS_OK and r.nullity == w.nullity and r.stats.get("refine_resid_max", 1) <= 1e-8)

    def timed_solves(precision):
        """W untimed warm-up solves, then K solves bracketed by barrier + synchronize
        and CUDA events on the library stream; returns (ms max over ranks, units, results,
        profile of the last solve, clocks)."""
        def one_step(profile=0):
            return h.solve(p["d"], p["restart"], p["tol"], check=False, precision=precision, profile=profile,
                           precond=p["precond"],
                           fp64_products=args.fp64_products)
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
        t_max, units = reduce_over_ranks(ms, float(units), dist, "cuda")
        return t_max, units, results, prof, clk

    pk = peaks()

    def roof(c, precision, clk):
        if not c["sampled"] or c["ms_per_launch"] <= 0:
            return {"kernel": c["name"], "bound": None, "achieved": None, "peak": None, "unit": None,
                    "frac": None, "traffic": None, "note": "not sampled (run with --profile-every > 0)"}
        key = c["name"] if c["name"] != "b_apply" else ("b_apply_fp64" if precision == "fp64" else "b_apply_mixed")
        if key == "cgs2_project" and precision != "fp64":
            key = "cgs2_project_mixed"
        ratio = ncu_traffic_ratio(key)
        traffic = None if ratio is None else ratio * c["bytes_per_launch"]
        base = {"kernel": c["name"], "traffic": traffic, "bytes_per_launch": c["bytes_per_launch"],
                "flops_per_launch": c["flops_per_launch"], "ms_per_launch": c["ms_per_launch"],
                "launches": c["launches"], "sampled": c["sampled"]}
        fp64_pipe = {"projected_eig"} | ({"cgs2_project"} if args.fp64_products == 1 else set())
        if precision == "fp64" and c["name"] in fp64_pipe and c["flops_per_launch"] > 0:
            # kernel classes that run on the FP64 pipe (above its ridge point): the projected
            # eigenproblem, and the Gram-Schmidt products when FP64 FMA is selected; the
            # default FP64 products run in compensated FP32 pairs and are bound by HBM
            ach = c["flops_per_launch"] / (c["ms_per_launch"] / 1e3) / 1e12
            fp64_peak = at_clock(fp64_peak_raw, fp64_mhz, clk.get("sm_mhz"))
            return {**base, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak,
                    "peak_src": f"{fp64_src}; {fp64_peak_raw:.4f} TFLOP/s at {fp64_mhz} MHz, rescaled to the "
                                f"timed region's {clk.get('sm_mhz')} MHz"}
        ach = c["bytes_per_launch"] / (c["ms_per_launch"] / 1e3) / 1e9
        return {**base, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "peak_src": pk["src"]}

    # independent checks of a basis (outside the timed region): closed-form sine, and the
    # residual ||A X||_F / ||A||_2 recomputed with PyTorch's sparse product and a
    # power-iteration ||A||_2 (not the library's own refinement statistics)
    As = A.to_scipy()
    Ad = AdT = None
    normA_ind = None

    def basis_checks(r):
        nonlocal Ad, AdT, normA_ind
        if r.nullity != w.nullity or w.nullity == 0:
            return None, None
        if Ad is None:
            Ad = device_csr(As)
            AdT = device_csr(As.T.tocsr()) if p["mode"] == "normal" else None
            normA_ind = norm2_power(Ad, AdT)
        Xd = torch.empty((w.nullity, A.n), dtype=torch.float64, device="cuda")
        h.basis(out=Xd)
        sine = closed_form_sine(w, Xd.T)
        res = residual_ratio(Ad, Xd.T, normA_ind)
        del Xd
        torch.cuda.empty_cache()
        return sine, res

    t_max, units, results, prof, clk = timed_solves(p["precision"])
    value = units / (t_max / 1e3)
    all_valid = all(valid(r) for r in results)
    launches = sum(r.stats.get("kernel_launches", 0) for r in results)
    dom = max(prof, key=lambda c: (c["ms_total_est"], c["launches"]))
    roofline = roof(dom, p["precision"], clk)
    spmm = roof(next(c for c in prof if c["name"] == "b_apply"), p["precision"], clk)
    sine, res_ind = basis_checks(results[-1])
    all_valid = all_valid and res_ind is not None and res_ind <= 1e-8

    # the metric's comparison: the mixed-precision path on the same resident matrix, the
    # same number of warm-up and timed solves
    mixed = None
    if p["precision"] == "fp64" and not args.no_mixed:
        mt, mu, mres, mprof, mclk = timed_solves("mixed")
        msine, mres_ind = basis_checks(mres[-1])
        mvalid = all(valid(r) for r in mres) and mres_ind is not None and mres_ind <= 1e-8
        mdom = max(mprof, key=lambda c: (c["ms_total_est"], c["launches"]))
        mlast = mres[-1].stats
        mixed = {"value": mu / (mt / 1e3), "unit": UNIT, "ms_per_step": mt / args.steps, "steps": args.steps,
                 "warmup": args.warmup, "valid": bool(mvalid), "dtype": "f32+f64",
                 "vs_fp64": (mu / (mt / 1e3)) / value if value > 0 else None,
                 "basis_check": {"sine_vs_closed_form": msine, "residual_independent": mres_ind,
                                 "residual_library": mlast.get("refine_resid_max")},
                 "roofline": roof(mdom, "mixed", mclk), "spmm_roofline": roof(
                     next(c for c in mprof if c["name"] == "b_apply"), "mixed", mclk),
                 "clocks": mclk, "gpu_launches": int(sum(r.stats.get("kernel_launches", 0) for r in mres)),
                 "solve": {k: mlast.get(k) for k in ("nullity", "matvecs", "restarts", "reorth_X", "reorth_Z",
                                                     "lock_events", "refine_iters_max", "t_lanczos_ms",
                                                     "t_refine_ms")},
                 "kernel_classes": [{k: c[k] for k in ("name", "launches", "sampled", "ms_per_launch",
                                                       "ms_total_est")} for c in mprof]}
        launches += mixed["gpu_launches"]

    # end-to-end through the public API: pinned host CSR -> ns_create -> ns_solve -> basis to pinned host
    rp = torch.from_numpy(A.rowptr).pin_memory()
    ci = torch.from_numpy(A.colind).pin_memory()
    va = torch.from_numpy(vals_in).pin_memory()
    out = torch.empty((w.nullity, A.n), dtype=torch.float64).pin_memory()
    h2d = rp.numel() * 8 + ci.numel() * 4 + va.numel() * va.element_size()
    d2h = out.numel() * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_units = 0
    for _ in range(args.e2e_steps):
        he = ns.Handle(rp.numpy(), ci.numpy(), va.numpy(), A.m, A.n, p["solver_seed"], p["mode"])
        r = he.solve(p["d"], p["restart"], p["tol"], check=False, precision=p["precision"], precond=p["precond"])
        if valid(r):
            he.lib.ns_basis(he.h, ns.C.c_void_p(out.data_ptr()), A.n, 0)
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
            "data": "synthetic", "config": describe(p, w), "valid": all_valid,
            "gpu_launches": int(launches), "clocks": clk, "roofline": roofline, "spmm_roofline": spmm,
            "e2e": e2e, "cpu_baseline": cpu, "mixed": mixed,
            "alu_peaks_tflops": {k: {"value": v[0], "src": v[1], "sm_mhz": v[2]} for k, v in alu.items()},
            "basis_check": {"sine_vs_closed_form": sine, "residual_independent": res_ind,
                            "residual_library": last.get("refine_resid_max"), "normA_power_iteration": normA_ind,
                            "bars": "sine <= 1e-6 (FP64) / 1e-5 (mixed), residual <= 1e-8"},
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
