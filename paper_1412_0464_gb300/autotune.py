"""Autotuner for the library's run-time tuning parameters.

The kernels' tile shapes follow from the slab width W at compile time.  Two
choices are left to run time, and this module picks them by timing:

* ``segments`` (2-D): the block-row segments of the parallel-in-y slab
  substitution.  The automatic value is about 2 N_y^(2/3), capped by the SM
  count; the candidates are that value and its neighbours.
* ``block_3d`` (3-D): the outer block width of the two-level Gauss-Jordan
  inverse, i.e. the depth of the delayed update that runs on the tensor
  cores: 64, 128 or 256.

A candidate is timed through the C ABI as one factorisation plus one
preconditioner application (the work of a solve step that depends on the
parameters), after a warm-up, with CUDA events on the current stream.  The
fastest candidate is stored in a JSON cache keyed by the workload's shape,
precision, sweep, two-grid flag and the device name, so that it is timed once
per machine.  Both parameters change only the order of floating-point
operations, not the method.
"""

from __future__ import annotations

import json
import os
import time

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1412_0464_gb300",
                             "autotune.json")


def cache_path() -> str:
    return os.environ.get("HZ_AUTOTUNE_CACHE", DEFAULT_CACHE)


def workload_key(cfg, device: str, over: dict | None = None) -> str:
    """Cache key: everything that changes the timed work, and the device."""
    over = dict(over or {})
    prec = over.get("precision", cfg.precision)
    sweep = over.get("sweep", cfg.sweep)
    two = over.get("two_grid", cfg.two_grid)
    nr = over.get("max_rhs", cfg.n_src)
    dims = "x".join(str(c) for c in cfg.cells)
    return (f"{device}|dim{cfg.dim}|{dims}|w{cfg.w_out}|J{over.get('J', cfg.J)}|"
            f"wdd{over.get('w_dd', cfg.w_dd)}|{prec}|{sweep}|tg{int(bool(two))}|rhs{nr}|"
            f"{getattr(cfg, 'boundary', 'pml')}")


def candidates(cfg, sms: int = 152) -> list[dict]:
    """Parameter sets to time for the workload."""
    if cfg.dim == 3:
        return [{"block_3d": b} for b in (64, 128, 256)]
    ny = cfg.cells[0] // 2 + 2 * cfg.w_out - 1 if cfg.two_grid else cfg.shape[0]
    auto = min(2 * round(ny ** (2.0 / 3.0)), 2 * sms)
    cands = {0}
    for f in (0.5, 0.75, 1.25):
        p = int(round(auto * f))
        if 2 <= p <= ny // 2:
            cands.add(p)
    return [{"segments": p} for p in sorted(cands)]


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(times: dict) -> str:
    """The fastest candidate; ties go to the first listed (the default)."""
    best = None
    for name, ms in times.items():
        if best is None or ms < times[best]:
            best = name
    return best


def _time_candidate(hz, cfg, m, f, params: dict, reps: int, over: dict) -> float:
    import torch
    s = hz.Solver.from_workload(cfg, m=m, **params, **over)
    try:
        s.factor()
        s.precond(f)                              # warm-up (allocations, first launches)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            t0.record()
            s.factor()
            s.precond(f)
            t1.record()
            t1.synchronize()
            best = min(best, t0.elapsed_time(t1))
        return best
    finally:
        s.close()


def tune(cfg, m=None, reps: int = 3, force: bool = False, path: str | None = None,
         **over) -> dict:
    """Time the candidates for ``cfg`` (a ``synth.Workload``; ``over`` as for
    ``Solver.from_workload``) and return ``{"params": best, "ms": {...}}``,
    from the cache unless ``force``."""
    import torch

    import paper_1412_0464_gb300 as hz
    import synth
    dev = torch.cuda.get_device_name()
    key = workload_key(cfg, dev, over)
    if not force:
        hit = load_cache(path).get(key)
        if hit is not None:
            return hit
    m = synth.medium(cfg) if m is None else m
    nr = over.get("max_rhs", cfg.n_src)
    b = synth.sources(cfg)[:nr]
    f = torch.from_numpy(b).cuda()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cands = candidates(cfg, sms)
    times = {}
    for c in cands:
        times[json.dumps(c, sort_keys=True)] = _time_candidate(hz, cfg, m, f, c, reps, over)
    best = choose(times)
    entry = {"params": json.loads(best), "ms": times, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    store(key, entry, path)
    return entry


def tuned_solver(cfg, m=None, path: str | None = None, **over):
    """``Solver.from_workload`` with the cached (or freshly timed) best parameters."""
    import paper_1412_0464_gb300 as hz
    entry = tune(cfg, m=m, path=path, **over)
    return hz.Solver.from_workload(cfg, m=m, **entry["params"], **over)
