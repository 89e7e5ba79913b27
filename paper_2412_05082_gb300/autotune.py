"""Autotuner for the batched form's tile shapes.

tiles_for: for every degree k (2D) it times the batched V-cycle graph of a
small batch of problems of that degree at a representative size for each
candidate tile shape (patches per thread block of the fused multiplicative-
smoother kernel) and keeps the fastest.

tune_batch: tiles for one given batch, timed on that batch's own V-cycle
graph: the per-degree tiles of tiles_for are the start, then one pass of
coordinate descent over the batch's degrees tries every candidate for one
degree with the others fixed.  The degrees' patch launches of one color run
concurrently and compete for the SMs, so the best tile of a degree can depend
on the mix.

Results are cached as JSON keyed by dimension, degree (or the batch's
problem list) and device architecture, in $BIHARM_TUNE_CACHE or
~/.cache/biharm_gb300/tiles.json.
"""

import json
import os

CANDIDATES = (1, 2, 3, 4, 6, 8, 12, 16, 24, 32)


def cache_path():
    p = os.environ.get("BIHARM_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "biharm_gb300", "tiles.json")


def _arch():
    import torch
    cap = torch.cuda.get_device_capability()
    return "sm_%d%d_%s" % (cap[0], cap[1], torch.cuda.get_device_name().replace(" ", "_"))


def load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(c):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def tune_degree(k, level=None, problems=4, reps=5, verbose=False, precision=0):
    """Best patches-per-block for degree k in the V-cycle precision `precision`
    (FP64 or the FP32 V-cycle with FP64 defects); returns (best, {pb: ms})."""
    import torch
    import paper_2412_05082_gb300 as bh
    if level is None:  # about 2e5 unknowns per problem
        level = max(2, min(9, int(round(__import__("math").log2(450.0 / k)))))
    params = [bh.default_params(2, k, level, precision=precision) for _ in range(problems)]
    times = {}
    with bh.Batch(params) as batch:
        for pb in CANDIDATES:
            try:
                batch.set_tile(k, pb)
            except bh.BiharmError:
                continue
            times[pb] = batch.vcycle_time(reps)
            if verbose:
                print("k=%d pb=%d: %.3f ms" % (k, pb, times[pb]))
    torch.cuda.synchronize()
    best = min(times, key=times.get)
    return best, times


def tiles_for(degrees, refresh=False, verbose=False, precision=0):
    """{k: patches per block} for the 2D degrees, tuned once per device and
    V-cycle precision."""
    cache = load_cache()
    arch = _arch()
    out, dirty = {}, False
    for k in sorted(set(degrees)):
        key = "d2_k%d_p%d_%s" % (k, precision, arch)
        if refresh or key not in cache:
            best, times = tune_degree(k, verbose=verbose, precision=precision)
            cache[key] = {"patches_per_block": best, "ms": times}
            dirty = True
        out[k] = int(cache[key]["patches_per_block"])
    if dirty:
        save_cache(cache)
    return out


def apply(batch, degrees, refresh=False):
    for k, pb in tiles_for(degrees, refresh).items():
        batch.set_tile(k, pb)


def tune_batch(batch, problems, refresh=False, reps=5, verbose=False):
    """{k: patches per block} for `batch`, built from `problems` (a list of
    (d, k, level)); applied to the batch before returning."""
    import paper_2412_05082_gb300 as bh
    degrees = sorted({k for _, k, _ in problems})
    precision = batch.params[0].precision
    cache = load_cache()
    key = "batch_p%d_%s_%s" % (precision, "-".join("%d.%d.%d" % p for p in sorted(problems)),
                               _arch())
    if not refresh and key in cache:
        tiles = {int(k): int(v) for k, v in cache[key]["tiles"].items()}
        for k, pb in tiles.items():
            batch.set_tile(k, pb)
        return tiles
    tiles = tiles_for(degrees, precision=precision)
    for k, pb in tiles.items():
        batch.set_tile(k, pb)
    best = batch.vcycle_time(reps)
    for k in degrees:
        for pb in CANDIDATES:
            if pb == tiles[k]:
                continue
            try:
                batch.set_tile(k, pb)
            except bh.BiharmError:
                continue
            t = batch.vcycle_time(reps)
            if verbose:
                print("k=%d pb=%d: %.3f ms (best %.3f)" % (k, pb, t, best))
            if t < best:
                best, tiles[k] = t, pb
        batch.set_tile(k, tiles[k])
    cache[key] = {"tiles": tiles, "vcycle_ms": best}
    save_cache(cache)
    return tiles
