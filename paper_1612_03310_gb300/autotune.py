"""Autotuner of the launch choices (see mithra_set_tuning in include/mithra.h).

It times candidate choices with the library's per-kernel CUDA events on a
scratch simulation built from the same grid and bunch (the caller's
simulation is never advanced), keeps the fastest potential-update choice and
the fastest particle-step choice independently (the two kernels do not share
knobs), and caches the result per (device, precision, grid, particle count)
in a JSON file so that later runs of the same shape skip the search.

The candidates: the direct stencil and the two marching stencils (TMA ring,
registers) with a range of plane runs per CTA; the per-particle push and the tiled push with 1 .. max
persistent CTAs per SM, then, for the tiled push with the best CTA count, a
range of sparse-tile thresholds (tiles below it skip the shared-memory
staging).  A threshold only acts from the next re-sort, so every push
candidate gets one untimed step before it is timed.
"""
from __future__ import annotations

import json
import os
import threading

from . import mithra

CACHE_DIR = os.environ.get("MITHRA_TUNING_CACHE",
                           os.path.join(os.path.expanduser("~"), ".cache", "mithra_gb300"))
_lock = threading.Lock()


def _cache_path() -> str:
    return os.path.join(CACHE_DIR, "tuning.json")


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    try:
        os.makedirs(CACHE_DIR, exist_ok=True)
        tmp = _cache_path() + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, _cache_path())
    except OSError:
        pass


def device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "cuda"


def key_of(grid: dict, n_particles: int, precision: int) -> str:
    # particle counts are bucketed by powers of two
    nb = max(int(n_particles), 1).bit_length()
    return (f"v2|{device_name()}|p{precision}|{grid['nx']}x{grid['ny']}x{grid['nz']}|"
            f"n2^{nb}|sub{grid.get('n_sub', 1)}")


def _kernel_ms(sim, steps: int) -> dict:
    sim.profile(True)
    sim.step(steps)
    kt = sim.kernel_times()
    sim.profile(False)
    return {k: (ms / n if n else 0.0) for k, (ms, n) in kt.items()}


def stencil_candidates(grid: dict) -> list[dict]:
    out = [dict(stencil_variant=0, lz=0)]
    for lz in (8, 16, 24, 32, 48, 64, 96, 128):
        if lz <= grid["nz"]:
            out.append(dict(stencil_variant=1, lz=lz))
    for lz in (4, 8, 16, 32, 64):
        if lz <= grid["nz"]:
            out.append(dict(stencil_variant=2, lz=lz))
    return out


def push_candidates(max_per_sm: int = 3) -> list[dict]:
    out = [dict(push_variant=0, push_ctas_per_sm=0, push_sparse_below=0)]
    for c in range(1, max_per_sm + 1):
        out.append(dict(push_variant=1, push_ctas_per_sm=c, push_sparse_below=0))
    return out


SPARSE_THRESHOLDS = (16, 32, 64, 128)


def sparse_candidates(best: dict) -> list[dict]:
    """Sparse-tile thresholds on top of the best tiled-push choice."""
    if best.get("push_variant") != 1:
        return []
    return [dict(best, push_sparse_below=s) for s in SPARSE_THRESHOLDS]


def tune(grid: dict, undulator: dict | None, bunch: dict | None, precision: int,
         steps: int = 4, warmup: int = 2, stream: int | None = None,
         use_cache: bool = True) -> dict:
    """Returns the best mithra_tuning fields for this shape, timing on a
    scratch simulation when the cache has no entry."""
    n = 0 if bunch is None else len(bunch["x"])
    key = key_of(grid, n, precision)
    with _lock:
        cache = _load() if use_cache else {}
        if key in cache:
            return dict(cache[key]["tuning"])
    sim = mithra.Simulation(grid, undulator, bunch, precision=precision, stream=stream)
    try:
        sim.step(warmup)
        trials = []
        best_st, best_st_ms = None, float("inf")
        for c in stencil_candidates(grid):
            try:
                sim.set_tuning(**c)
            except mithra.MithraError:
                continue
            ms = _kernel_ms(sim, steps)["potential_step"]
            trials.append(dict(c, ms=ms))
            if ms < best_st_ms:
                best_st, best_st_ms = c, ms
        best_pu = dict(push_variant=0, push_ctas_per_sm=0, push_sparse_below=0)
        best_pu_ms = float("inf")
        if n > 0:
            def trial(c):
                nonlocal best_pu, best_pu_ms
                try:
                    sim.set_tuning(**c)
                except mithra.MithraError:
                    return
                sim.step(1)  # the re-sort applies the candidate's tile lists
                ms = _kernel_ms(sim, steps)["push"]
                trials.append(dict(c, ms=ms))
                if ms < best_pu_ms:
                    best_pu, best_pu_ms = c, ms
            for c in push_candidates():
                trial(c)
            for c in sparse_candidates(best_pu):
                trial(c)
    finally:
        sim.close()
    best = dict(best_st or dict(stencil_variant=0, lz=0))
    best.update(best_pu)
    with _lock:
        cache = _load()
        cache[key] = dict(tuning=best, stencil_ms=best_st_ms, push_ms=best_pu_ms, trials=trials)
        _store(cache)
    return best


def record(grid: dict, n_particles: int, precision: int) -> dict | None:
    """The cached entry (choice, best times, all trials) of a shape."""
    return _load().get(key_of(grid, n_particles, precision))


def apply(sim, grid: dict, undulator: dict | None, bunch: dict | None, precision: int,
          **kw) -> dict:
    """Tunes (or looks up) this shape and applies the choice to sim."""
    best = tune(grid, undulator, bunch, precision, **kw)
    sim.set_tuning(**best)
    return best
