"""The oracle's own functions on several host threads: the all-core CPU
baseline (test infrastructure only; the library never imports it).

Nothing of the oracle is rewritten here. Its C functions are called as they
are, through the same ctypes wrappers; ctypes releases the interpreter lock
for the length of each foreign call, so calls on disjoint inputs run on
separate cores. Work is split only where the oracle's result is a
concatenation or a set of independent results, so the threaded result is
identical to the single call's:
* capture: the oracle emits fragments in (triangle, row, column) order, so
  contiguous triangle ranges, captured separately (each a sub-scene with the
  whole scene's vertices and quantisation cube) and concatenated in order,
  give exactly one call's records once each range's triangle ids are
  shifted by the range's first triangle;
* novel views: each view is rendered by one call, one view per thread.
The POFA sort stays one call.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import fragments as _fragments
from . import render as _render


def default_threads() -> int:
    """Host threads to use: every core the process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # not on Linux
        return os.cpu_count() or 1


def _sub_scene(scene, t0: int, t1: int):
    """Triangles [t0, t1) of `scene` with its vertices, materials and cube (a shallow copy)."""
    sub = object.__new__(type(scene))
    sub.__dict__.update(scene.__dict__)
    sub.idx = np.ascontiguousarray(scene.idx[t0:t1])
    sub.tri_material = np.ascontiguousarray(scene.tri_material[t0:t1])
    return sub


def fragments(scene, mode: int, camera=None, pitch: float = 0.0, threads: int = None) -> np.ndarray:
    """The records of `oracle.fragments(scene, mode, camera, pitch)`, computed
    over contiguous triangle ranges on `threads` host threads."""
    threads = threads or default_threads()
    T = int(scene.idx.shape[0])
    cuts = np.linspace(0, T, max(1, min(threads * 4, T)) + 1).astype(np.int64)
    ranges = [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]

    def one(r):
        rec = _fragments(_sub_scene(scene, r[0], r[1]), mode, camera, pitch)[0]
        rec["tri"] += np.uint32(r[0])
        return rec

    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, ranges))
    return np.concatenate(parts) if parts else _fragments(scene, mode, camera, pitch)[0]


def render_views(records, scene, views, lights, k: int = 1, threads: int = None):
    """[(vis, rgba)] of `oracle.render` for every view, one view per thread."""
    threads = threads or default_threads()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda v: _render(records, scene, v, lights, k), views))
