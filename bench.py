#!/usr/bin/env python
"""Benchmark: time to a 1e-6 relative residual (and Mdof/s) of the GMRES +
sweeping-preconditioner solve of the 2-D heterogeneous workload
(1000^2 interior cells + 20 PML cells per side = 1039^2 unknowns, seeded
random-field + layer medium, one point source, J = 16 slabs, X-sweep,
complex64 preconditioner, FP64 GMRES).

One step = hz_factor + hz_solve (factorise every slab, then solve to 1e-6).
Inputs are resident in HBM when the timed region starts; L2 is flushed
(256 MiB write) between timed steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank solves its own replica of the workload (the
path has no data-path exchange for one right-hand side): value = all ranks'
dof / max-over-ranks time.  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import resource
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-6 rel. residual (s) and Mdof/s; mixed+batched vs plain FP64 on GB300"
CONFIG_INDEX = 2


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 8-source batched leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-gradient leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the configuration 3 and 3-D legs of the default line")
    ap.add_argument("--n3d", type=int, default=64,
                    help="interior cells per axis of the reduced 3-D legs (configs 4 and 5)")
    ap.add_argument("--workload", type=int, default=CONFIG_INDEX, choices=[1, 2, 3, 4, 5],
                    help="benchmark configuration (default 2, the headline workload; 4 and 5 "
                         "run at --n3d interior cells unless --n is given)")
    ap.add_argument("--n", type=int, default=0,
                    help="profiling only: the workload's recipe at this interior size (not a bench line)")
    ap.add_argument("--J", type=int, default=0, help="profiling only: slab count with --n")
    ap.add_argument("--autotune", action="store_true",
                    help="time the autotuner's candidates first and run with its choice "
                         "(default: the automatic parameters, on which the committed ncu "
                         "figures were taken)")
    ap.add_argument("--write-traffic", nargs=3, metavar=("CSV", "COMMAND", "WORKLOAD"),
                    help="write profiles/traffic.json from an ncu DRAM-bytes capture of the "
                         "bench's mixed run on WORKLOAD (its config.workload string) and exit")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="print the per-kernel table of an ncu launch list and exit")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 GEMM peak (burst) times the
    nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x 1.1/2.25"
    return 1900.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


def _sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("sm_max_mhz", 2070.0))
    return 2070.0


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.idx = gpu_index
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.idx is not None:
                cmd += ["-i", str(self.idx)]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# kernels whose DRAM traffic profiles/traffic.json records: bench tag -> (kernel
# name patterns summed per launch, the sources that define them).  An entry is
# used only while the hash of those sources matches the one stored with it.
TRAFFIC_KERNELS = {
    "slab_factor": (["slab_factor_fused_kernel"],
                    ["slab.cuh", "slab_c64.cu", "slab_c128.cu", "ptx.cuh", "hz_internal.h"]),
    "stencil_c64": (["op_pair_kernel_c64"], ["stencil.cu", "hz_internal.h"]),
    "stencil_c128": (["op_kernel<double"], ["stencil.cu", "hz_internal.h"]),
    "slab_factor3d_update": (["tc_pack_kernel", "gj_update_tc_kernel"],
                             ["slab3d.cu", "tc.cuh", "ptx.cuh", "hz_internal.h"]),
    "slab3_gemv": (["tc_vpack_kernel", "slab3_gemm_tc_kernel", "slab3_gemm_reduce_kernel"],
                   ["slab3d.cu", "tc.cuh", "ptx.cuh", "hz_internal.h"]),
}


def _src_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1412_0464_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(tag, workload=None, precision=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    this workload and precision and its kernel's sources are unchanged since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or tag not in TRAFFIC_KERNELS:
        return None
    d = json.load(open(p))
    if workload is not None and d.get("bench_workload") != workload:
        return None
    if precision is not None and d.get("precision") != precision:
        return None
    e = d.get("kernels", {}).get(tag)
    if e is None or e.get("source_hash") != _src_hash(TRAFFIC_KERNELS[tag][1]):
        return None
    return e.get("dram_bytes_per_launch")


def _ncu_rows(path):
    """(kernel name, metric, value) rows of an `ncu --csv` log."""
    import csv
    rows = []
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    for r in csv.DictReader(lines):
        try:
            v = float(r["Metric Value"].replace(",", ""))
        except (KeyError, ValueError):
            continue
        rows.append((r["ID"], r["Kernel Name"], r["Metric Name"], v))
    return rows


def write_traffic(csv_path, command, workload):
    """profiles/traffic.json from an ncu capture of dram__bytes_read.sum and
    dram__bytes_write.sum (one pass, no replay)."""
    rows = _ncu_rows(csv_path)
    per = {}
    for lid, name, metric, v in rows:
        if metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per.setdefault((lid, name), 0.0)
            per[(lid, name)] += v
    out = {"command": command, "workload": workload, "bench_workload": workload, "precision": "mixed",
           "note": "DRAM bytes (read + write) per launch, mean over the captured launches; "
                   "a tag that sums two kernels (pack + update, GEMM + reduce) adds their means",
           "kernels": {}}
    for tag, (pats, files) in TRAFFIC_KERNELS.items():
        total, ok = 0.0, True
        counts = []
        for pat in pats:
            vals = [v for (lid, name), v in per.items() if pat in name.split("(")[0]]
            if not vals:
                ok = False
                break
            total += sum(vals) / len(vals)
            counts.append(len(vals))
        if ok:
            out["kernels"][tag] = {"dram_bytes_per_launch": total, "launches_captured": counts,
                                   "source_hash": _src_hash(files)}
    p = os.path.join(ROOT, "profiles", "traffic.json")
    old = json.load(open(p)).get("kernels", {}) if os.path.exists(p) else {}
    for tag, e in old.items():              # keep entries of kernels this capture did not see
        if tag not in out["kernels"] and tag in TRAFFIC_KERNELS:
            out["kernels"][tag] = e
    with open(p, "w") as f:
        json.dump(out, f, indent=1)
    return out


def _short_kernel_name(name):
    """Kernel name without the namespaces, the return type and the argument list."""
    for pre in ("(anonymous namespace)::", "<unnamed>::", "unnamed>::", "void ", "hz::"):
        name = name.replace(pre, "")
    return name.split("(")[0].strip()


def summarize_launches(csv_path):
    """Markdown table of an ncu launch list: launches, total time, share and mean
    time per launch per kernel, and, when the capture has them, the mean DRAM
    rate and the mean utilisations (DRAM, SM, FMA / FP64 / tensor pipes) over
    the kernel's launches."""
    rows = _ncu_rows(csv_path)
    per = {}
    for lid, name, metric, v in rows:
        k = _short_kernel_name(name)
        per.setdefault((lid, k), {})[metric] = v
    agg = {}
    for (lid, k), m in per.items():
        a = agg.setdefault(k, {"n": 0, "t": 0.0, "bytes": 0.0, "u": {}})
        a["n"] += 1
        a["t"] += m.get("gpu__time_duration.sum", 0.0)
        a["bytes"] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        for key, v in m.items():
            if key.endswith("pct_of_peak_sustained_elapsed") or key.endswith("pct_of_peak_sustained_active"):
                a["u"].setdefault(key, []).append(v)
    tot = sum(v["t"] for v in agg.values()) or 1.0
    short = [("gpu__dram_throughput", "DRAM %"), ("sm__throughput", "SM %"),
             ("sm__pipe_fma_cycles", "FMA pipe %"), ("sm__pipe_fp64_cycles", "FP64 pipe %"),
             ("sm__pipe_tensor_cycles", "tensor pipe %")]
    have = [(p, h) for p, h in short if any(any(k.startswith(p) for k in a["u"]) for a in agg.values())]
    hdr = "| kernel | launches | total (ms) | share | per launch (us) |"
    if any(a["bytes"] > 0 for a in agg.values()):
        hdr += " DRAM GB/s |"
    hdr += "".join(f" {h} |" for _, h in have)
    lines = [hdr, "|" + "---|" * (hdr.count("|") - 1)]
    for k, a in sorted(agg.items(), key=lambda kv: -kv[1]["t"]):
        row = f"| `{k}` | {a['n']} | {a['t'] / 1e6:.3f} | {a['t'] / tot:.3f} | {a['t'] / 1e3 / a['n']:.1f} |"
        if "DRAM GB/s" in hdr:
            row += f" {a['bytes'] / a['t'] if a['t'] else 0:.0f} |"
        for p, _ in have:
            vals = [x for key, v in a["u"].items() if key.startswith(p) for x in v]
            row += f" {sum(vals) / len(vals):.1f} |" if vals else " — |"
        lines.append(row)
    return "\n".join(lines)


def adjoint_leg(hz, synth, stream, flush, n=512, reps=3, cfg=None):
    """hz_grad on the 2-D adjoint workload (smooth random medium, blurred start
    model, 8 sources and 16 receivers, two-grid, J = 4, mixed), or on `cfg`:
    one gradient step = hz_factor at the start model + hz_grad (forward and
    adjoint solves of the sources, misfit, gradient).  The observed data are
    the receiver values of the true model's solution computed by the same
    solver."""
    import numpy as np
    import torch
    cfg = synth.adjoint_workload_2d(n) if cfg is None else cfg
    m_true, m0 = synth.medium(cfg, "true"), synth.medium(cfg, "start")
    c_pml = float(np.mean(1.0 / np.sqrt(m0)))
    src = np.array([np.ravel_multi_index(tuple(int(v) for v in idx), cfg.shape)
                    for idx in synth.source_nodes(cfg)])
    rec = synth.receivers(cfg)
    st = hz.Solver.from_workload(cfg, m=m_true, c_pml=c_pml)
    st.factor()
    u, _ = st.solve(torch.from_numpy(synth.sources(cfg)).cuda())
    d = u.reshape(cfg.n_src, -1)[:, torch.from_numpy(rec).cuda()].contiguous()
    st.close()
    s0 = hz.Solver.from_workload(cfg, m=m0, c_pml=c_pml)
    s0.factor()
    s0.grad(src, rec, d)
    ts, phi, info = [], 0.0, {}
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s0.factor()
        phi, g, info = s0.grad(src, rec, d)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    s0.close()
    t = statistics.mean(ts) / 1000.0
    return {"workload": f"{workload_string(cfg)}, mixed, {cfg.n_src} sources, {cfg.n_rec} receivers",
            "step": "hz_factor + hz_grad (forward + adjoint solves, misfit, gradient)",
            "time_s": t, "value": 2 * cfg.n_src * cfg.ndof / t / 1e6,
            "unit": "Mdof/s (dof x solves: forward and adjoint per source)",
            "misfit": phi, "iters_max": info.get("iters_max"), "relres_max": info.get("relres_max")}


def workload_leg(hz, synth, cfg, stream, flush, reps=3, note=None, precision=None):
    """hz_factor + hz_solve of every source of `cfg` in one multi-right-hand-side
    call: time to 1e-6 (CUDA events, L2 flushed between repetitions), Mdof/s
    counted as dof x right-hand sides, and the factorisation's share."""
    import torch
    m = synth.medium(cfg)
    b = torch.from_numpy(synth.sources(cfg)).cuda()
    kw = {} if precision is None else {"precision": precision}
    s = hz.Solver.from_workload(cfg, m=m, **kw)
    s.factor()
    s.solve(b)
    ts, tf, st = [], [], {}
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        s.factor()
        e1.record(stream)
        _, st = s.solve(b)
        e2.record(stream)
        e2.synchronize()
        ts.append(e0.elapsed_time(e2))
        tf.append(e0.elapsed_time(e1))
    s.close()
    t = statistics.mean(ts) / 1000.0
    out = {"workload": workload_string(cfg), "n_rhs": cfg.n_src,
           "precision": precision or cfg.precision, "step": "hz_factor + hz_solve",
           "time_to_solution_s": t, "factor_s": statistics.mean(tf) / 1000.0,
           "value": cfg.ndof * cfg.n_src / t / 1e6, "unit": "Mdof/s (dof x right-hand sides)",
           "iters_max": st.get("iters_max"), "relres_max": st.get("relres_max")}
    if note:
        out["note"] = note
    return out


def workload_string(cfg):
    """The workload name both arms report in config.workload."""
    dims = "x".join(str(s) for s in cfg.shape)
    return (f"{cfg.name}: {dims} dof, J={cfg.J}, {cfg.sweep}-sweep, w_dd={cfg.w_dd}"
            + (", two-grid" if cfg.two_grid else ""))


def oracle_solve(cfg):
    """One oracle time-to-solution sample: set-up (assembly and a sparse LU of
    every slab: the factorisation) and the GMRES solve of the first source to
    the workload's tolerance.  Returns (seconds, iterations, cpu seconds)."""
    import synth
    from oracle.problem import Problem
    b = synth.sources(cfg)[0]
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    p = Problem(cfg)
    _, info = p.solve(b)
    t = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return t, info["iters"], cpu


def cpu_baseline(cfg):
    """The FP64 oracle, as it stands, on the same workload: one full time to
    solution (set-up + GMRES to the tolerance), measured, not extrapolated."""
    t, iters, cpu = oracle_solve(cfg)
    return {"value": cfg.ndof / t / 1e6, "unit": "Mdof/s",
            "cores": max(1, round(cpu / t)), "kind": "oracle",
            "sample": (f"one full solve of the {workload_string(cfg)} workload: oracle set-up "
                       f"(assembly + SuperLU of every slab) and GMRES to {cfg.tol:g} "
                       f"({iters} iterations), {t:.2f} s measured"),
            "time_to_solution_s": t, "iters": iters, "host_cores_available": os.cpu_count()}


def replica_throughput(ms_step, dof_per_rank, ws, device):
    """Whole-job Mdof/s of ws independent replicas: every rank solved dof_per_rank
    unknowns; the job time is the slowest rank's (max over ranks)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms_step)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t)
    return ms_step, ws * dof_per_rank / (ms_step / 1000.0) / 1e6


def reference_arm(args):
    """The oracle as it stands, timed on the host cores: each step is one full
    time to solution of the same workload (set-up + GMRES to the tolerance)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import synth
    cfg = synth.workload(args.workload)
    for _ in range(args.warmup):
        oracle_solve(cfg)
    ts, cpus, iters = [], [], 0
    for _ in range(args.steps):
        t, iters, cpu = oracle_solve(cfg)
        ts.append(t)
        cpus.append(cpu)
    t_step = statistics.mean(ts)
    value = cfg.ndof / t_step / 1e6
    cores = max(1, round(sum(cpus) / sum(ts)))
    line = {"metric": METRIC, "value": value, "unit": "Mdof/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic (seeded random-field + layer medium, point source)",
            "impl": "reference",
            "config": {"workload": workload_string(cfg), "n_rhs": 1,
                       "step": "oracle set-up (assembly + SuperLU of every slab) + GMRES to 1e-6"},
            "cpu_baseline": {"value": value, "unit": "Mdof/s", "kind": "oracle", "cores": cores,
                             "sample": (f"each step one full oracle solve ({iters} GMRES "
                                        f"iterations), {t_step:.2f} s mean over {args.steps}")},
            "e2e": {"value": value, "unit": "Mdof/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "time_to_solution_s": t_step, "iters": iters}
    print(json.dumps(line))
    return 0


def main():
    args = _args()
    if args.write_traffic:
        out = write_traffic(*args.write_traffic)
        print(json.dumps({t: e["dram_bytes_per_launch"] for t, e in out["kernels"].items()}))
        return
    if args.summarize_launches:
        print(summarize_launches(args.summarize_launches))
        return
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1412_0464_gb300 as hz
    import synth
    if rank == 0:
        hz.build()
    if ws > 1:
        torch.distributed.barrier()
    cfg = synth.workload(args.workload)
    if args.n:
        cfg = synth.scaled_workload(args.workload, args.n, J=args.J or None)
    elif cfg.dim == 3:      # the full 3-D configurations do not fit (dense slab factors)
        cfg = synth.scaled_workload(args.workload, args.n3d, J=args.J or None)
    m = synth.medium(cfg)
    b = synth.sources(cfg)
    # run-time tuning parameters (segment count / 3-D outer block) from the
    # autotuner: timed once per device and workload shape, outside the timed steps
    tuned = {}
    if args.autotune:
        from paper_1412_0464_gb300 import autotune
        tuned_entry = autotune.tune(cfg, m=m)
        tuned = tuned_entry["params"]
    solver = hz.Solver.from_workload(cfg, m=m, **tuned)
    f_dev = torch.from_numpy(b).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        solver.factor()
        return solver.solve(f_dev)

    for _ in range(args.warmup):
        u, st = step()
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gidx = vis.split(",")[local] if vis and vis.split(",")[local].strip().isdigit() else (local if ws > 1 else None)
    clocks = ClockSampler(gidx)
    launches0 = solver.stats()["kernel_launches"]
    clocks.start()
    barrier()
    total_ms = 0.0
    iters, relres, solve_s = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, st = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters.append(st["iters_max"])
        relres.append(st["relres_max"])
        solve_s.append(st["t_solve_s"])
    barrier()
    gpu_launches = solver.stats()["kernel_launches"] - launches0
    # Per-kernel durations: the same K steps once more with a CUDA event pair
    # around every tagged launch on its own stream.  The events separate the
    # launches (no prologue overlap between consecutive kernels), so `value`
    # comes from the uninstrumented steps above and this pass only feeds the
    # roofline and the kernel breakdown.
    solver.enable_timing(True)
    inst_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        inst_ms += e0.elapsed_time(e1)
    barrier()
    clk = clocks.stop()
    tags = ["slab_rhs", "slab_fwd_pass1", "slab_carry", "slab_carry_bound", "slab_fwd_bwd1",
            "slab_bwd", "slab_solve", "slab_factor", "slab_middle", "segment_product",
            "segment_prefix", "stencil_c64", "stencil_c128",
            "slab_factor3d_schur", "slab_factor3d_panel", "slab_factor3d_rowmod",
            "slab_factor3d_update", "slab_factor3d_inner", "slab_factor3d_writeout", "slab3_gemv",
            "slab_solve3d"]
    kt = {t: solver.kernel_timing(t) for t in tags}
    solver.enable_timing(False)
    ms_step, value = replica_throughput(total_ms / args.steps, cfg.ndof * cfg.n_src, ws, "cuda")

    # end to end through the C ABI with host buffers (pinned), copies included
    f_host = torch.from_numpy(b).pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()          # the result lands in pinned memory
    e2e_ms = []
    for i in range(max(2, min(args.steps, 3)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.factor()
        solver.solve_host(f_host, out=u_host)
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_ms = statistics.mean(e2e_ms[1:])
    nbytes = cfg.ndof * cfg.n_src * 16

    # Roofline of the dominant kernel (largest summed device time over the
    # timed steps).  The factorisation is bounded by FP32 arithmetic (complex64
    # Gauss-Jordan, 8 W^3 flop per block row plus the 48 W^2 flop Schur update):
    # peak = SMs x 128 FP32 lanes x 2 flop x maximum SM clock.  The substitution
    # kernels are bounded by HBM: peak = the measured copy bandwidth.
    peak, peak_kind = _peaks()
    per_kernel = {t: {"ms": v[0], "launches": v[1], "bytes": v[2]} for t, v in kt.items() if v[1] > 0}
    widths = [solver.slab_info(j)["W"] for j in range(1, cfg.J + 1)]
    ny_sweep = (cfg.n // 2 + 2 * cfg.w_out - 1) if cfg.two_grid else cfg.N
    factor_flop = sum((ny_sweep - 1) * (8.0 * w ** 3 + 48.0 * w ** 2) for w in widths)
    props = torch.cuda.get_device_properties(local)
    sm_max = _sm_max_mhz()
    # the factorisation runs in the preconditioner precision: complex64 work is
    # bound by the FP32 FMA pipe, complex128 work by the (much narrower) FP64 one;
    # the peak is measured on this device by hz_alu_peak (FMA chains on all SMs)
    fprec = "mixed" if cfg.precision == "mixed" else "fp64"
    alu_peak = hz.alu_peak(fprec)
    alu_derived = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    indiv = {t: v for t, v in per_kernel.items() if t not in ("slab_solve", "slab_solve3d")}
    dom = max(indiv, key=lambda t: indiv[t]["ms"])
    # the kernels that stream the slab operators from HBM (the carries move a few products
    # each and are latency-bound; the stencils are reported separately below); in 3-D the
    # per-layer GEMV with the stored dense inverse
    hbm_tags = [t for t in indiv
                if t in ("slab_rhs", "slab_fwd_pass1", "slab_fwd_bwd1", "slab_bwd", "slab3_gemv")]
    dom_hbm = max(hbm_tags, key=lambda t: indiv[t]["ms"])

    def hbm_line(tag):
        d = indiv[tag]
        ach = d["bytes"] / (d["ms"] / 1000.0) / 1e9
        return {"bound": "hbm", "kernel": tag, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_kind, "traffic": _traffic(tag, workload_string(cfg), cfg.precision),
                "avg_launch_us": 1000 * d["ms"] / d["launches"],
                "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "share_of_device_time": d["ms"] / sum(v["ms"] for v in indiv.values())}

    if dom == "slab_factor":
        d = indiv[dom]
        ach = factor_flop / (d["ms"] / d["launches"] / 1000.0) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": ach / alu_peak,
                    "peak_source": (f"measured {'FP32' if fprec == 'mixed' else 'FP64'} FMA "
                                    "throughput (hz_alu_peak)"),
                    "peak_fp32_derived": alu_derived,
                    "traffic": _traffic(dom, workload_string(cfg), cfg.precision), "avg_launch_us": 1000 * d["ms"] / d["launches"],
                    "algorithmic_flop_per_launch": factor_flop,
                    "share_of_device_time": d["ms"] / sum(v["ms"] for v in indiv.values())}
        roofline["hbm_kernel"] = hbm_line(dom_hbm)
    elif dom == "slab_factor3d_update":
        # the rank-128 complex GEMM update (outer blocks) of the 3-D Gauss-Jordan
        # inverse; its tag carries the algorithmic flop, 8 B (B - 128) 128 per
        # chain and block.  complex64: tcgen05 kind::tf32 with three TF32 passes
        # per real product, so the tensor pipe executes 3x the algorithmic flop;
        # complex128: FP64 SIMT
        d = indiv[dom]
        ach = d["bytes"] / (d["ms"] / 1000.0) / 1e12
        common = {"kernel": dom, "achieved": ach, "unit": "TFLOP/s", "traffic": _traffic(dom, workload_string(cfg), cfg.precision),
                  "avg_launch_us": 1000 * d["ms"] / d["launches"],
                  "algorithmic_flop_per_launch": d["bytes"] / d["launches"],
                  "share_of_device_time": d["ms"] / sum(v["ms"] for v in indiv.values())}
        if fprec == "mixed":
            tpk, tsrc = _tf32_peak()
            roofline = {"bound": "tensor", "peak": tpk, "frac": ach / tpk, "peak_source": tsrc,
                        "tensor_pipe_frac": 3.0 * ach / tpk,
                        "note": "3xTF32 split: executed TF32 flop = 3 x algorithmic", **common}
        else:
            roofline = {"bound": "alu", "peak": alu_peak, "frac": ach / alu_peak,
                        "peak_source": "measured FP64 FMA throughput (hz_alu_peak)", **common}
        roofline["hbm_kernel"] = hbm_line(dom_hbm)
    else:
        roofline = hbm_line(dom)
    # the matrix-free stencil kernels (Eq. 40 apply / residual / Jacobi): complex64
    # in the two-grid smoother, complex128 for the GMRES operator (FP64 pipe)
    roofline["stencil"] = {t: hbm_line(t) for t in ("stencil_c64", "stencil_c128") if t in indiv}
    sol = per_kernel.get("slab_solve")
    if sol:
        roofline["slab_solve_sequence"] = {
            "achieved_gbs": sol["bytes"] / (sol["ms"] / 1000.0) / 1e9,
            "avg_us": 1000 * sol["ms"] / sol["launches"], "solves": sol["launches"],
            "note": "whole subdomain solve (all its kernels), method-minimal bytes (operators read twice)"}

    line = {"metric": METRIC, "value": value, "unit": "Mdof/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 preconditioner / c128 GMRES" if cfg.precision == "mixed" else "c128",
            "data": "synthetic (seeded random-field + layer medium, point source)",
            "config": {"workload": workload_string(cfg),
                       "n_rhs": cfg.n_src, "step": "hz_factor + hz_solve",
                       "autotune": ({"params": tuned, "candidates_ms": tuned_entry["ms"]}
                                    if args.autotune else "off (automatic parameters)"),
                       "l2": "flushed (256 MiB write) between timed steps",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "time_to_solution_s": ms_step / 1000.0, "solve_only_s": statistics.mean(solve_s),
            "iters": max(iters), "relres": max(relres),
            "e2e": {"value": cfg.ndof * cfg.n_src / (e2e_ms / 1000.0) / 1e6, "unit": "Mdof/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "roofline": roofline, "kernels": per_kernel,
            "kernel_timing": {"pass": "a second pass of the K timed steps with CUDA events around "
                                      "every tagged launch", "ms_per_step": inst_ms / args.steps},
            "clocks": clk, "gpu_launches": gpu_launches}
    solver.close()

    # (3-D: the complex128 dense-block inverses run on GB300's narrow FP64 pipe;
    # no FP64 arm there)
    if rank == 0 and ws == 1 and not args.no_fp64_arm and cfg.dim == 2:
        s64 = hz.Solver.from_workload(cfg, m=m, precision="fp64")
        s64.factor()
        s64.solve(f_dev)
        ts, it64 = [], 0
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s64.factor()
            _, st64 = s64.solve(f_dev)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            it64 = st64["iters_max"]
        t64 = statistics.mean(ts) / 1000.0
        line["fp64_arm"] = {"time_to_solution_s": t64, "value": cfg.ndof / t64 / 1e6,
                            "unit": "Mdof/s", "iters": it64,
                            "speedup_mixed_vs_fp64": t64 / (ms_step / 1000.0)}
        s64.close()
    if rank == 0 and ws == 1 and not args.no_batched and cfg.n_src == 1 and not args.n:
        # the same workload with 8 seeded sources solved together (multiple
        # right-hand sides through every kernel): one factorisation + one solve
        import dataclasses
        cfg8 = dataclasses.replace(cfg, n_src=8)
        b8 = torch.from_numpy(synth.sources(cfg8)).cuda()
        s8 = hz.Solver.from_workload(cfg8, m=m)
        s8.factor()
        s8.solve(b8)
        ts, it8, rr8 = [], 0, 0.0
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s8.factor()
            _, st8 = s8.solve(b8)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            it8, rr8 = st8["iters_max"], st8["relres_max"]
        t8 = statistics.mean(ts) / 1000.0
        line["batched"] = {"n_rhs": 8, "time_to_solution_s": t8,
                           "value": 8 * cfg.ndof / t8 / 1e6, "unit": "Mdof/s (dof x right-hand sides)",
                           "iters_max": it8, "relres_max": rr8,
                           "speedup_per_rhs_vs_single": 8 * (ms_step / 1000.0) / t8}
        s8.close()
    if rank == 0 and ws == 1 and not args.no_adjoint and not args.n and args.workload == 2:
        line["adjoint"] = adjoint_leg(hz, synth, stream, flush)
    if rank == 0 and ws == 1 and not args.no_extra and not args.n and args.workload == 2:
        # the other configurations, as side legs of the headline line: the large
        # 2-D two-grid workload at full size, and the 3-D workloads at n3d
        # interior cells per axis (their full sizes need more than the GPU's
        # memory for dense slab factors)
        line["config3"] = workload_leg(hz, synth, synth.workload(3), stream, flush, reps=2)
        c4 = synth.scaled_workload(4, args.n3d)
        line["config4_3d"] = workload_leg(
            hz, synth, c4, stream, flush, reps=2,
            note=f"configuration 4 recipe at {args.n3d}^3 interior cells (reduced), "
                 f"{c4.n_src} sources as right-hand sides of one solve")
        c5 = synth.scaled_workload(5, args.n3d)
        line["config5_3d_gradient"] = adjoint_leg(hz, synth, stream, flush, reps=2, cfg=c5)
        line["config5_3d_gradient"]["note"] = (
            f"configuration 5 recipe at {args.n3d}^3 interior cells (reduced), two-grid")
    if (rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload != 3
            and cfg.dim == 2):
        line["cpu_baseline"] = cpu_baseline(cfg)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
