"""Choose the launch schedule of the FP32-mixed kernels by timing them.

Two knobs, set through the C ABI:
  * the thread-tile shape (sale_set_tiling / sale_batch_set_schedule): a
    block covers tx x ty cells (or nodes) of one k plane; four shapes from
    32x8 to 128x2 trade coalescing width against the rows of neighbours a
    block re-reads from L2;
  * for a batch, the order of the meshes' tiles in each launch (input order,
    or largest mesh first so that the long-running tiles start early).

No knob changes a result: every cell's arithmetic is the same whatever the
block it lands in, and the time-step minimum is exact.  So tuning may run on
the live state, as ordinary cycles (bench.py tunes during its warm-up).

Choices are cached in a JSON file keyed by device name, kind and sizes:
$SALE_TUNE_CACHE, else ~/.cache/sale_gb300/tune.json; pass cache=None to
neither read nor write it.
"""
from __future__ import annotations

import ctypes as C
import json
import statistics
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sale_gb300", "tune.json")


def cache_path():
    return os.environ.get("SALE_TUNE_CACHE", DEFAULT_CACHE)


def load_cache(path):
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path, key, value):
    """Merge one entry into the cache file (written atomically)."""
    data = load_cache(path)
    data[key] = value
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(candidates, time_fn, repeats=3):
    """The candidate with the smallest median time over `repeats` timings
    (statistics.median: the middle one for an odd count, the mean of the
    two middle ones for an even count), with every candidate's median.
    time_fn(candidate) returns milliseconds."""
    times = {}
    for c in candidates:
        times[c] = statistics.median(float(time_fn(c)) for _ in range(repeats))
    best = min(candidates, key=lambda c: (times[c], candidates.index(c)))
    return best, times


def tile_shapes():
    """[(shape id, tx, ty)] of the FP32-mixed kernels."""
    from . import sale

    out = []
    shape = 0
    while True:
        tx, ty = C.c_int(0), C.c_int(0)
        if sale.sale_tile_shape(shape, C.byref(tx), C.byref(ty)) != sale.SALE_OK:
            return out
        out.append((shape, tx.value, ty.value))
        shape += 1


def _device_name(stream):
    import torch

    return torch.cuda.get_device_name(stream.device)


def _timer(stream, run):
    """Milliseconds of run() on `stream`, by CUDA events recorded on it."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def tune_state(st, cycles=16, repeats=3, cache="default", remap_every=1):
    """Pick and set the fastest tile shape of an FP32-mixed State.  Advances
    the state by about (1 + repeats) * cycles cycles per shape.  Returns
    {"shape", "tile", "ms_per_cycle": {shape: ms}, "cached"}."""
    md = st.md
    path = cache_path() if cache == "default" else cache
    key = f"{_device_name(st.stream)}|state|{md.nx}x{md.ny}x{md.nz}|remap{remap_every}"
    shapes = tile_shapes()
    if path:
        hit = load_cache(path).get(key)
        if hit is not None and 0 <= int(hit.get("shape", -1)) < len(shapes):
            st.set_tiling(int(hit["shape"]))
            return {"shape": int(hit["shape"]), "tile": shapes[int(hit["shape"])][1:], "cached": True,
                    "ms_per_cycle": hit.get("ms_per_cycle", {})}

    def time_shape(shape):
        return _timer(st.stream, lambda: st.run_to_time(max_cycles=cycles, remap_every=remap_every)) / cycles

    ids = [s for s, _, _ in shapes]
    warmed = set()

    def timed(shape):
        st.set_tiling(shape)
        if shape not in warmed:  # first run captures the graph
            st.run_to_time(max_cycles=cycles, remap_every=remap_every)
            warmed.add(shape)
        return time_shape(shape)

    best, times = choose(ids, timed, repeats)
    st.set_tiling(best)
    res = {"shape": best, "tile": shapes[best][1:], "cached": False,
           "ms_per_cycle": {str(k): v for k, v in times.items()}}
    if path:
        store_cache(path, key, {"shape": best, "ms_per_cycle": res["ms_per_cycle"]})
    return res


def tune_batch(b, cycles=4, repeats=3, cache="default"):
    """Pick and set the fastest (tile shape, mesh order) of a Batch.  Advances
    every mesh by about (1 + repeats) * cycles cycles per candidate."""
    import hashlib

    path = cache_path() if cache == "default" else cache
    sizes = ",".join(f"{md.nx}x{md.ny}x{md.nz}" for md, _ in b.instances)
    key = f"{_device_name(b.stream)}|batch|{len(b.instances)}|{hashlib.sha1(sizes.encode()).hexdigest()[:16]}"
    shapes = tile_shapes()
    if path:
        hit = load_cache(path).get(key)
        if hit is not None and 0 <= int(hit.get("shape", -1)) < len(shapes) and hit.get("order") in (0, 1):
            b.set_schedule(int(hit["shape"]), int(hit["order"]))
            return {"shape": int(hit["shape"]), "order": int(hit["order"]), "tile": shapes[int(hit["shape"])][1:],
                    "cached": True, "ms_per_cycle": hit.get("ms_per_cycle", {})}

    cands = [(s, o) for s, _, _ in shapes for o in (0, 1)]
    warmed = set()

    def timed(c):
        b.set_schedule(*c)
        if c not in warmed:
            b.run(cycles)
            warmed.add(c)
        return _timer(b.stream, lambda: b.run(cycles)) / cycles

    best, times = choose(cands, timed, repeats)
    b.set_schedule(*best)
    res = {"shape": best[0], "order": best[1], "tile": shapes[best[0]][1:], "cached": False,
           "ms_per_cycle": {f"{s},{o}": v for (s, o), v in times.items()}}
    if path:
        store_cache(path, key, {"shape": best[0], "order": best[1], "ms_per_cycle": res["ms_per_cycle"]})
    return res
