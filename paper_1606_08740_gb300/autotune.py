"""Tile autotuner for stencil systems.

Each system's sweep tiling (tile shape variant and z depth) is picked from its own grid shape,
radius, precision and history length only, never from the rest of a batch, so a system's
arithmetic and reduction order are the same alone and in any batch. Candidates are timed
natively by ``aar_tune_stencil`` (CUDA events around the Richardson sweep); results are cached
in a JSON file keyed by (nx, ny, nz, radius, precision, m).
"""
from __future__ import annotations

import json
import os
import threading

from . import aar

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("AAR_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "aar_gb300", "tiles.json"))


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path: str, table: dict) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home just means no cache


def key(desc: aar.StencilDesc, precision: int, m: int) -> str:
    return f"{desc.nx}x{desc.ny}x{desc.nz}/r{desc.radius}/p{precision}/m{m}"


def tune(descs, precision: int = aar.MIXED, m: int = 7, path: str | None = None, stream=None):
    """Set tile hints on every descriptor (in place) and return {shape key: (variant, zc, ms)}."""
    path = path or cache_path()
    with _lock:
        table = _load(path)
        chosen = {}
        dirty = False
        for d in descs:
            k = key(d, precision, m)
            if k not in table:
                probe = aar.StencilDesc.from_buffer_copy(d)
                probe.tile_variant = probe.tile_zc = 0
                v, z, ms = aar.tune_stencil(probe, precision, m, stream)
                table[k] = [v, z, ms]
                dirty = True
            v, z, ms = table[k]
            d.tile_variant, d.tile_zc = int(v), int(z)
            chosen[k] = (int(v), int(z), float(ms))
        if dirty:
            _save(path, table)
    return chosen
