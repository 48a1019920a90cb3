"""A JSON cache of tuning choices, so that a later job on the same kind of GPU
reuses them instead of timing again.

Entries are keyed by (GPU name, process, precision, number of points k) for the
kernel variant of a single process (rex_autotune), and by (GPU name, precision,
batch composition, k) for the slot-group count and the per-process tile costs of a
persistent multi-process launch (rex_multi_autotune).  Each entry keeps the choice and the timings it was
made from.  The file is rewritten whole (through a temporary file and a rename),
so a crash cannot leave it half written; an unreadable file counts as empty.
"""
import json
import os
import tempfile
from typing import Callable, Sequence


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _write(path: str, d: dict) -> None:
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tune_cache.", dir=folder)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def variant_key(gpu: str, process: str, precision: int, k: int) -> str:
    return f"variant|{gpu}|{process}|{precision}|{k}"


def slot_groups_key(gpu: str, precision: int, batches: Sequence[tuple], k: int) -> str:
    """batches: (process name, events) per batch, in launch order."""
    comp = ",".join(f"{name}:{n}" for name, n in batches)
    return f"slot_groups|{gpu}|{precision}|{comp}|{k}"


def cached_choice(path: str, key: str, tune: Callable[[], tuple], apply: Callable[[int, dict], None]) -> dict:
    """The cached choice for key, applied; on a miss, tune() -> (choice, timings, extra)
    is run, its choice applied and stored.  extra is a dict of further tuned values that
    apply(choice, extra) restores.  Returns the entry and whether it came from the file."""
    d = _read(path)
    e = d.get(key)
    if isinstance(e, dict) and isinstance(e.get("choice"), int):
        extra = e.get("extra") if isinstance(e.get("extra"), dict) else {}
        apply(e["choice"], extra)
        return {"choice": e["choice"], "ms": e.get("ms"), "extra": extra, "cached": True}
    choice, ms, extra = tune()
    apply(int(choice), extra)
    d = _read(path)               # another job may have written meanwhile
    d[key] = {"choice": int(choice), "ms": [float(x) for x in ms], "extra": extra}
    _write(path, d)
    return {"choice": int(choice), "ms": list(ms), "extra": extra, "cached": False}


def autotune_process(proc, momenta, w_in, points, w_out, path: str, stream=None, gpu: str | None = None) -> dict:
    """rex_autotune through the cache: the variant for (GPU, process, precision, k)."""
    key = variant_key(gpu or gpu_name(), proc.name, proc.precision, len(points))

    def tune():
        ms = proc.autotune(momenta, w_in, points, w_out, stream=stream)
        return proc.variant, ms, {}   # rex_autotune keeps the fastest

    def apply(v, extra):
        proc.variant = v

    return cached_choice(path, key, tune, apply)


def autotune_multi(multi, batches, points, path: str, stream=None, gpu: str | None = None) -> dict:
    """rex_multi_autotune through the cache: slot groups and tile costs for the batch
    composition.  batches: [(Process, momenta, w_in, w_out)] as for Multi.reweight."""
    comp = [(b[0].name, int(b[1].shape[0])) for b in batches]
    key = slot_groups_key(gpu or gpu_name(), multi.precision, comp, len(points))

    def tune():
        ms = multi.autotune(batches, points, stream=stream)
        return multi.slot_groups, ms, {"tile_us": {b[0].name: multi.tile_cost(b[0]) for b in batches}}

    def apply(g, extra):
        multi.slot_groups = g
        costs = extra.get("tile_us", {})
        for b in batches:
            if isinstance(costs.get(b[0].name), (int, float)):
                multi.set_tile_cost(b[0], costs[b[0].name])

    return cached_choice(path, key, tune, apply)
