"""Tile-shape autotuner with an on-disk cache.

The timing itself is native (``lbd_autotune`` times every compiled tile shape on
the context's own state with CUDA events); this module only remembers the
winner per (device name, nx, ny, precision, walls) in a JSON file so that later
runs skip the search.
"""
import json
import os

CACHE = os.environ.get("LBD_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json"))


def kernels_tag():
    """Short hash of the CUDA sources the library is built from: a winner
    measured on other kernels is not reused."""
    import hashlib
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:12]


def _key(device, nx, ny, precision, flags=0):
    walls = "|walls" if flags & 16 else ""
    return "%s|%s|%dx%d|%s%s" % (kernels_tag(), device, nx, ny,
                                 "fp64" if precision == 0 else "fp32", walls)


def load_cache(path=CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key, tile, path=CACHE):
    cache = load_cache(path)
    cache[key] = list(tile)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(sim, device, reps=20, path=CACHE, refresh=False):
    """Set sim's tile from the cache, or search, store and set it.  Returns the tile."""
    key = _key(device, sim.nx, sim.ny, sim.params.precision, sim.params.flags)
    cache = load_cache(path)
    if key in cache and not refresh:
        tile = tuple(cache[key])
        try:
            sim.set_tile(*tile)
            return tile
        except RuntimeError:  # a shape the library no longer accepts here: search again
            pass
    tile = tuple(sim.autotune(reps))
    store(key, tile, path)
    return tile
