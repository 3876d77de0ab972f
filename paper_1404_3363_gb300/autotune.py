"""Cached launch shapes for batches (ivv_batch_autotune), one table per GPU.

The library times the candidate shapes itself; this module keeps the winners
in a JSON file keyed by the GPU (name, SM count, compute capability) and by
the batch's signature (volumes, image sizes, precision), so a batch of the
same shape on the same kind of GPU starts with its tuned shapes.
"""
from __future__ import annotations

import hashlib
import json
import os


def cache_path() -> str:
    return os.environ.get("IVV_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "ivv_gb300", "batch_tuning.json")


def gpu_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|sm%d%d|%dSM" % (p.name, p.major, p.minor, p.multi_processor_count)


def batch_signature(items, precision=0) -> str:
    """items: (volume, camera, width, height, tf) as passed to ivv.Batch."""
    h = hashlib.sha256()
    vols = {}
    for vol, _cam, w, hgt, _tf in items:
        vid = vols.setdefault(id(vol), len(vols))
        info = vol.info()
        h.update(("%d:%d:%d:%d:%d:%d;" % (vid, info["n_blocks"], info["n_faces"], info["degree"], w, hgt)).encode())
    h.update(("p%d" % precision).encode())
    return h.hexdigest()[:24]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned(batch, items, precision=0, reps=3, path=None):
    """Apply the cached shapes of this batch on this GPU, or autotune and
    cache them.  Returns (tuning dict, ms per frame or None, 'cache'|'tuned')."""
    path = path or cache_path()
    table = _load(path)
    key = gpu_key() + "|" + batch_signature(items, precision)
    if key in table:
        batch.tuning = table[key]["tuning"]
        return table[key]["tuning"], table[key].get("ms"), "cache"
    best, ms = batch.autotune(reps=reps)
    table[key] = {"tuning": best, "ms": ms}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return best, ms, "tuned"
