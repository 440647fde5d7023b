"""Autotuner for the batched engine's configuration.

The batched launch's knobs (``swa_batch_config``) change speed, never
results:

- the height of a uint8 SAT tile (64 or 32 rows: shorter tiles mean more
  tiles and look-back records, taller ones more shared memory per warp);
- the image order (as given, or largest first, which lets small images fill
  the tail);
- the order of each image's tiles in the work queue (along anti-diagonals,
  or row by row);
- the look-back mode (edge records, or corner records from the tile above
  and to the left);
- the warps per build block (9, as many as shared memory holds, or 8);
- how many images of the same kind share the build's work queue at a time
  (8, their tickets merged by progress, or 1, image after image).

``tune`` times every combination (64 candidates) on a deterministic sample
of the batch's images with CUDA events and keeps the fastest.  Results are
cached in a JSON file keyed by the device and a coarse description of the
batch, so a later batch of the same kind skips the search.  The cache file
is ``$SWA_TUNE_CACHE`` if set, else
``~/.cache/paper_2410_16291_gb300/tune.json``.
"""
from __future__ import annotations

import itertools
import json
import math
import os

AXES = (("u8_tile_rows", (64, 32)), ("order", (0, 1)), ("ticket_order", (0, 1)),
        ("lookback", (0, 1)), ("warps", (9, 8)), ("interleave", (8, 1)))
# Every combination, the library's defaults first.
CANDIDATES = tuple(dict(zip([k for k, _ in AXES], v))
                   for v in itertools.product(*[vals for _, vals in AXES]))
KEY_VERSION = 3


def cache_path() -> str:
    p = os.environ.get("SWA_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2410_16291_gb300",
                        "tune.json")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def batch_key(device: str, shapes, dtypes) -> str:
    """Coarse class of a batch: device, image count (power-of-two bucket),
    mean image size (power-of-two bucket in pixels) and uint16 share
    (quarters)."""
    n = len(shapes)
    px = sum(r * c for r, c in shapes) / max(1, n)
    u16 = sum(1 for d in dtypes if d == "u16") / max(1, n)
    return "v%d|%s|n%d|px%d|u16q%d" % (KEY_VERSION, device,
                                       1 << max(0, int(math.log2(max(1, n)))),
                                       int(math.log2(max(1.0, px))), int(round(u16 * 4)))


def choose(times: dict) -> dict:
    """The candidate with the smallest time (first on ties)."""
    best = min(range(len(CANDIDATES)), key=lambda i: (times.get(i, float("inf")), i))
    return dict(CANDIDATES[best])


def sample_indices(n: int, k: int) -> list:
    """k indices spread evenly over range(n) (all of them if n <= k)."""
    if n <= k:
        return list(range(n))
    return sorted({int(i * n / k) for i in range(k)})


def tune(images, windows, dtypes=None, sample: int = 24, reps: int = 3, use_cache: bool = True,
         timer=None) -> dict:
    """Pick the batch configuration for these images (CUDA tensors) and
    windows.  ``timer(cfg, imgs, wins)`` may replace the GPU timing (tests)."""
    import paper_2410_16291_gb300 as swa
    shapes = [tuple(t.shape) for t in images]
    if dtypes is None:
        dtypes = ["u8" if str(t.dtype).endswith("uint8") else "u16" for t in images]
    device = "cpu"
    if timer is None:
        import torch
        device = torch.cuda.get_device_name()
    key = batch_key(device, shapes, dtypes)
    cache = load_cache() if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key]["config"])
    idx = sample_indices(len(images), sample)
    imgs = [images[i] for i in idx]
    wins = [windows[i] for i in idx]

    def gpu_time(cfg, imgs, wins):
        import torch
        b = swa.Batch(imgs, wins, **cfg)
        b.run()
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        for _ in range(reps):
            b.run()
        e1.record(s)
        b.sync()
        ms = e0.elapsed_time(e1) / reps
        b.free()
        return ms

    timer = timer or gpu_time
    times = {i: timer(dict(c), imgs, wins) for i, c in enumerate(CANDIDATES)}
    best = choose(times)
    if use_cache:
        cache[key] = {"config": best, "ms": {str(i): times[i] for i in times},
                      "sample": len(idx)}
        save_cache(cache)
    return best
