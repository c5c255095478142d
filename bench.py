"""Benchmark of the GB300 Schur-complement Stokes path.

One step = create_geometry (mask -> face flags, components) followed, for Uzawa and for
SIMPLE, by schur_solve (Algorithm 1 to tol 1e-8, inner tolerances 1e-12), velocity
recovery and the permeability read-back: two Schur solves per step on the workload
"spheres128" (128^3 periodic overlapping spheres, radii U[4,8), porosity 0.40, seed 0,
f = e_x, FP64).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = Schur solves per second on the device-resident mask;
e2e = the same with the mask in host memory (its H2D copy and the permeability D2H
inside the timed region).  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload and scales it to whole solves with the oracle's own
iteration counts.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Schur solves/s & stencil HBM GB/s, SIMPLE vs Uzawa, FP64 vs mixed; p50/p99"
UNIT = "solves/s"
WORKLOAD = dict(name="spheres128", n=128, r_min=4.0, r_max=8.0, porosity=0.40, seed=0,
                force=(1.0, 0.0, 0.0), tol=1e-8, tol_inner=1e-12)
DESC = ("spheres128: 128^3 periodic overlapping solid spheres, radii U[4,8), porosity "
        "0.40, seed 0 (+rank), f = e_x, FP64; Uzawa and SIMPLE Schur-CG to 1e-8 "
        "(unpreconditioned), inner Jacobi-PCG to 1e-12")
W_BYTES = 8
# algorithmic bytes per unknown (face kernels) or per fluid cell (cell kernels), FP64
ALG_BYTES = {
    "cgA_dir": lambda nu, npf, d: (3 * W_BYTES + 1) * nu,
    "cgA_matvec": lambda nu, npf, d: (2 * W_BYTES + 1) * nu,
    "cgA_update": lambda nu, npf, d: (6 * W_BYTES + 1) * nu,
    "cgS_dir": lambda nu, npf, d: 4 * W_BYTES * npf,
    "cgS_matvec": lambda nu, npf, d: (2 * W_BYTES + 1 + d) * npf,
    "cgS_update": lambda nu, npf, d: 7 * W_BYTES * npf,
}


def make_mask(rank: int = 0):
    from paper_2307_05266_gb300 import synth
    w = WORKLOAD
    return synth.sphere_packing(w["n"], w["r_min"], w["r_max"], w["porosity"], w["seed"] + rank)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------
def oracle_iteration_counts():
    counts = {}
    for pc in ("uzawa", "simple"):
        path = os.path.join(ROOT, "tests", "golden", f"oracle_spheres128_{pc}.json")
        if os.path.exists(path):
            with open(path) as f:
                counts[pc] = json.load(f)
    return counts


def oracle_sample(n_inner: int = 10) -> dict:
    """Time the oracle on a bounded sample of the workload: assembly, n_inner inner A
    iterations and n_inner inner SIMPLE iterations; scale to two whole solves with the
    oracle's recorded iteration counts."""
    import numpy as np

    from oracle import mac, stokes
    mask = make_mask(0)
    t0 = time.perf_counter()
    prob = stokes.StokesProblem(mask)
    t_asm = time.perf_counter() - t0
    b = mac.force(prob.geo, WORKLOAD["force"])
    t0 = time.perf_counter()
    prob.solve_A(b, 1e-300, n_inner)
    t_a = (time.perf_counter() - t0) / n_inner
    r = prob.B @ prob.solve_A(b, 1e-300, 2).x
    t0 = time.perf_counter()
    prob.solve_simple(r, 1e-300, n_inner)
    t_s = (time.perf_counter() - t0) / n_inner
    counts = oracle_iteration_counts()
    t_step = t_asm
    used = {}
    for pc in ("uzawa", "simple"):
        c = counts.get(pc)
        if c is None:
            return dict(ok=False, why=f"no recorded oracle iteration counts for {pc}",
                        t_assemble=t_asm, t_inner_A=t_a, t_inner_S=t_s)
        ia = c["inner_iters_A"] + c["recovery_iters"]
        t_step += ia * t_a + c["inner_iters_S"] * t_s
        used[pc] = dict(outer=c["outer_iters"], inner_A=ia, inner_S=c["inner_iters_S"])
    sample_s = t_asm + (n_inner + 2) * t_a + n_inner * t_s
    return dict(ok=True, value=2.0 / t_step, t_step=t_step, t_assemble=t_asm, t_inner_A=t_a,
                t_inner_S=t_s, counts=used, sample_seconds=sample_s)


def run_oracle_subprocess(threads: int = 1) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads), CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"],
                         capture_output=True, text=True, env=env, timeout=900)
    for line in out.stdout.splitlines()[::-1]:
        line = line.strip()
        if line.startswith("{"):
            return json.loads(line)
    return dict(ok=False, why="oracle sample failed: " + out.stderr[-300:])


def sample_text(s: dict) -> str:
    return (f"128^3 spheres workload: oracle assembly ({s['t_assemble']:.2f} s) + 10 inner A "
            f"({s['t_inner_A'] * 1e3:.1f} ms/it) and 10 inner SIMPLE ({s['t_inner_S'] * 1e3:.1f} "
            f"ms/it) FP64 CG iterations, scaled to 2 whole solves with the oracle's recorded "
            f"iteration counts {s['counts']}")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    samples = []
    s = None
    for i in range(args.warmup + args.steps):
        s = run_oracle_subprocess(1)
        if not s.get("ok"):
            print(json.dumps({"impl": "reference", "unavailable": s.get("why", "oracle failed")}))
            return 0
        if i >= args.warmup:
            samples.append(s)
    t_step = statistics.median([x["t_step"] for x in samples])
    value = 2.0 / t_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": DESC, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample_text(s)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2307_05266_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local < len(ids):
            dev_index = ids[local]
    binding.load()
    w = WORKLOAD
    mask_np = make_mask(rank)
    mask_dev = torch.from_numpy(mask_np).cuda()
    porosity = float(mask_np.mean())
    stream = torch.cuda.current_stream()
    precs = (("uzawa", binding.UZAWA), ("simple", binding.SIMPLE))

    def step(mask, rec):
        g = binding.Geometry(mask)
        g.set_force(w["force"])
        launches = 2  # flags + S-hat diagonal
        for name, pc in precs:
            t0 = time.perf_counter()
            st = g.solve(precond=pc, tol=w["tol"], tol_inner_A=w["tol_inner"],
                         tol_inner_S=w["tol_inner"])
            rs = g.recover_velocity()
            k = g.permeability(0)
            t1 = time.perf_counter()
            launches += st.kernel_launches + rs.kernel_launches
            if rec is not None:
                rec.setdefault(name, []).append(dict(
                    ms=(t1 - t0) * 1e3, outer=st.outer_iters, inner_A=st.inner_iters_A,
                    inner_S=st.inner_iters_S, recovery=rs.inner_iters_A, k=k,
                    rel_res=st.rel_res))
        info = g.info
        g.close()
        return launches, info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(mask_dev, None)
    rec = {}
    launches = 0
    barrier()
    with ClockSampler(str(dev_index)) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            n, info = step(mask_dev, rec)
            launches += n
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    solves = 2 * args.steps * world
    value = solves / (ms_max / 1e3)

    # end to end: host mask in, permeabilities out
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(mask_np, None)
    e1.record(stream)
    barrier()
    t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = solves / (float(t.item()) / 1e3)

    # per-kernel timing: CUDA events around single launches on the bench stream, L2
    # flushed (a 512 MiB write) before every launch
    g = binding.Geometry(mask_dev)
    g.set_force(w["force"])
    g.solve(precond=binding.SIMPLE, tol=w["tol"], tol_inner_A=w["tol_inner"],
            tol_inner_S=w["tol_inner"])
    info = g.info
    nu = int(sum(info.n_unknown[a] for a in range(info.ndim)))
    npf = int(info.n_fluid)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    kern = {}
    for name in binding.KERNELS:
        times = []
        for _ in range(12):
            flush.zero_()
            times.append(g.time_kernel(name))
        avg = statistics.mean(times[2:])
        alg = ALG_BYTES[name](nu, npf, info.ndim)
        kern[name] = {"ms": avg, "alg_bytes": alg, "alg_GBps": alg / (avg / 1e3) / 1e9}
    g.close()
    peak, peak_kind = load_peaks()
    # dominant kernel: largest share of one inner A iteration
    dom = max(("cgA_dir", "cgA_matvec", "cgA_update"), key=lambda k: kern[k]["ms"])
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["alg_GBps"], "peak": peak,
            "unit": "GB/s", "frac": kern[dom]["alg_GBps"] / peak, "traffic": None,
            "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind ==
            "measured" else "fallback",
            "timing": "CUDA events around single launches on the bench stream after the "
                      "timed region, L2 flushed before each launch, mean of 10"}

    per = {}
    for name, rows in rec.items():
        per[name] = {"ms_median": statistics.median(r["ms"] for r in rows),
                     "outer": rows[-1]["outer"], "inner_A": rows[-1]["inner_A"],
                     "inner_S": rows[-1]["inner_S"], "recovery": rows[-1]["recovery"],
                     "k": rows[-1]["k"], "rel_res": rows[-1]["rel_res"]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = run_oracle_subprocess(1) if world == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": DESC, "grid": w["n"], "porosity": porosity,
                   "n_unknown": nu, "n_fluid": npf,
                   "step": "create_geometry + (solve + recover + permeability) x {Uzawa, SIMPLE}",
                   "l2": "inputs larger than L2: solver working set "
                         f"{info.device_bytes / 1e9:.2f} GB vs 0.13 GB L2",
                   "parallelism": f"replicas x{world}"},
        "per_precond": per,
        "kernels": kern,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(mask_np.nbytes),
                "d2h_bytes_per_step": 16},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if cpu is not None and cpu.get("ok"):
        line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": 1,
                                "kind": "oracle", "sample": sample_text(cpu)}
    elif cpu is not None:
        line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": cpu.get("why", "unavailable")}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample()))
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
