"""One scene's FHV split over ranks: Morton-range ownership of the POFA with
one all-to-all of records, and rendering by a min-reduce of visibility words.

The method's data-parallel path shards by fragment (Sections 3.2 and 3.3):
capture is independent per triangle, the POFA is a sort by Morton key, and a
splat keeps, per pixel, the fragment with the smallest (depth, index) key.
Across ranks that becomes:

* capture: the triangles are cut into contiguous ranges of about equal
  estimated samples (`sample_weights`, `balanced_bounds`); every rank builds
  the POFA of its range straight from the triangles
  (`fhv_build_pofa_direct` on a slice of the scene, with the whole scene's
  triangle ids). Alternatively a rank passes records it captured otherwise,
  and compacts them (`fhv_compact_pofa`, sorted by key).
* build: from every rank's local sorted records and per-octant counts, the
  ranks all-reduce the record counts of the octants of a coarse level and
  cut the Morton order into contiguous ranges of about equal size, one per
  rank. Each rank's sorted records for a range form one contiguous slice
  (its bounds are the local offsets of the range's first octants), so one
  all-to-all sends every slice to the range's owner, which compacts what it
  receives. The owners' results, in rank order, are the POFA of all records
  byte for byte, and rank r's records start at the global index
  base_r = sum of the counts of ranks < r.
* render: every rank splats its records numbered from base_r
  (`fhv_splat_visibility`); the element-wise unsigned minimum over ranks is
  the visibility of the whole POFA. Every rank then shades the pixels whose
  winner it holds (`fhv_shade_owned`, zeros elsewhere) and the images are
  summed: each pixel comes from exactly one rank, so the sum is exact.

The local steps run in the library's kernels (`DeviceOps`); the collectives go
through torch.distributed (`Comm`: NCCL on device tensors, gloo through host
memory). Both are passed in, so the orchestration here is the same whatever
executes the local steps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist

from . import fhv

HIST_LEVEL = 6  # octree level whose octants the ownership ranges are cut at (capped at the depth)
_SIGN = -(1 << 63)  # int64 with only the top bit set


class Comm:
    """The collectives of the sharded path over a torch.distributed group."""

    def __init__(self, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.direct = dist.get_backend(group) == "nccl"  # NCCL takes device tensors; gloo host tensors

    def _io(self, t: torch.Tensor) -> torch.Tensor:
        return t if self.direct else t.cpu()

    def all_reduce_sum(self, t: torch.Tensor) -> torch.Tensor:
        """Element-wise sum over ranks."""
        x = self._io(t).clone()
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=self.group)
        return x.to(t.device)

    def all_reduce_min_u64(self, t: torch.Tensor) -> torch.Tensor:
        """Element-wise unsigned minimum of int64 tensors holding uint64 words
        (flipping the top bit maps unsigned order onto signed order)."""
        x = torch.bitwise_xor(self._io(t), _SIGN)
        dist.all_reduce(x, op=dist.ReduceOp.MIN, group=self.group)
        return torch.bitwise_xor(x, _SIGN).to(t.device)

    def all_gather_int(self, v: int) -> list:
        """One integer from every rank, in rank order."""
        x = torch.tensor([int(v)], dtype=torch.int64)
        x = x.cuda() if self.direct else x
        out = [torch.empty_like(x) for _ in range(self.world)]
        dist.all_gather(out, x, group=self.group)
        return [int(o.item()) for o in out]

    def all_to_all_rows(self, rows: torch.Tensor, counts: list) -> torch.Tensor:
        """rows [n, c]: the first counts[0] rows go to rank 0, the next
        counts[1] to rank 1, ...; returns the rows received, in rank order."""
        send = torch.tensor(counts, dtype=torch.int64)
        send = send.cuda() if self.direct else send
        recv = torch.empty_like(send)
        dist.all_to_all_single(recv, send, group=self.group)
        rc = [int(v) for v in recv.cpu().tolist()]
        c = rows.shape[1]
        x = self._io(rows).contiguous().view(-1)
        out = torch.empty(sum(rc) * c, dtype=rows.dtype, device=x.device)
        dist.all_to_all_single(out, x, [v * c for v in rc], [v * c for v in counts], group=self.group)
        return out.view(-1, c).to(rows.device)


def sample_weights(scene, mode: int, pitch: float, cam=None) -> np.ndarray:
    """Estimated capture work of every triangle, in samples: its area over
    the sample pitch squared as the capture sees it (in its own plane for
    FHV_CAPTURE_NORMAL, projected on the three axis planes for
    FHV_CAPTURE_AXIS3, on the view plane for FHV_CAPTURE_VIEW), plus one for
    its setup. Only the ratios matter: they cut the triangles into ranges of
    about equal work."""
    p = np.asarray(scene.pos, np.float64)[np.asarray(scene.idx, np.int64)]
    a = 0.5 * np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])  # area vectors
    if mode == fhv.FHV_CAPTURE_VIEW:
        h = float(cam.pitch)
        area = np.abs(a @ np.asarray(cam.fwd, np.float64))
    elif mode == fhv.FHV_CAPTURE_AXIS3:
        h = float(pitch)
        area = np.abs(a).sum(axis=1)
    else:
        h = float(pitch)
        area = np.linalg.norm(a, axis=1)
    return area / (h * h) + 1.0


def balanced_bounds(hist: np.ndarray, world: int) -> np.ndarray:
    """Cuts the octants of one level (their global record counts `hist`, in
    Morton order) into `world` contiguous ranges of about equal record count:
    returns bounds b_0 = 0 <= b_1 <= ... <= b_world = len(hist); rank r owns
    octants [b_r, b_{r+1}). Integer counts are cut exactly; fractional
    weights (the per-triangle sample estimates) keep their fractions."""
    hist = np.asarray(hist)
    exact = np.issubdtype(hist.dtype, np.integer) or hist.dtype == np.bool_
    hist = hist.astype(np.int64 if exact else np.float64)
    prefix = np.cumsum(hist)
    total = prefix[-1].item() if hist.size else 0
    b = np.zeros(world + 1, dtype=np.int64)
    b[world] = hist.size
    for r in range(1, world):
        # records before rank r's range: at least r / world of them
        target = (total * r + world - 1) // world if exact else total * r / world
        b[r] = min(max(int(np.searchsorted(prefix, target, side="left")) + 1, int(b[r - 1])), hist.size)
        if total == 0:
            b[r] = hist.size
    return b


@dataclass
class LocalPofa:
    """A compaction's result as the sharded path reads it."""
    rec: torch.Tensor  # [n, 2] int64: the sorted 16-byte records
    off: torch.Tensor  # per-octant offsets, all levels
    cnt: torch.Tensor  # per-octant counts, all levels
    level_base: object  # level -> index of the level's first octant in off / cnt


class DeviceOps:
    """The local steps on this rank's GPU, through the library's kernels."""

    def __init__(self, depth: int, device="cuda"):
        self.depth = depth
        self.device = device

    def compact(self, rec: torch.Tensor) -> LocalPofa:
        """rec [n, 2] int64 records in any order -> sorted records + offsets."""
        n = rec.shape[0]
        n_oct = fhv.fhv_level_offset(self.depth + 1)
        off = torch.empty(n_oct, dtype=torch.int32, device=self.device)
        cnt = torch.empty(n_oct, dtype=torch.int32, device=self.device)
        out = torch.empty((max(n, 1), 2), dtype=torch.int64, device=self.device)
        ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, self.depth, max(n, 1)).workspace_bytes,
                           self.device)
        src = rec.contiguous() if n else torch.zeros((1, 2), dtype=torch.int64, device=self.device)
        fhv.fhv_compact_pofa(src, n, None, self.depth, out, off, cnt, ws)
        return LocalPofa(out[:n], off, cnt, fhv.fhv_level_offset)

    def capture(self, scene, t0: int, t1: int, mode: int, cam, pitch: float) -> LocalPofa:
        """The POFA of triangles [t0, t1) of `scene` (a DeviceScene) built
        straight from them, with the whole scene's triangle ids: a first call
        without output learns the count, the second stores the records."""
        sl = scene.slice(t0, t1)
        m = fhv.fhv_level_offset(self.depth + 1)
        off = torch.empty(m, dtype=torch.int32, device=self.device)
        cnt = torch.empty(m, dtype=torch.int32, device=self.device)
        count = torch.zeros(2, dtype=torch.int64, device=self.device)

        def ws(cap):
            return fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_DIRECT, t1 - t0, 1, 1, self.depth,
                                                     cap).workspace_bytes, self.device)

        fhv.fhv_build_pofa_direct(sl, mode, cam, pitch, self.depth, None, 0, count, off, cnt, ws(0))
        n = int(count[0].item())
        out = torch.empty((max(n, 1), 2), dtype=torch.int64, device=self.device)
        fhv.fhv_build_pofa_direct(sl, mode, cam, pitch, self.depth, out, n, count, off, cnt, ws(n))
        return LocalPofa(out[:n], off, cnt, fhv.fhv_level_offset)

    def splat(self, rec: torch.Tensor, base: int, scene, cam, k: int) -> torch.Tensor:
        """Visibility keys of this rank's records, numbered from `base`."""
        vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device=self.device)
        ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES, self.device)
        fhv.fhv_splat_visibility(rec if rec.shape[0] else None, rec.shape[0], None, base, scene, cam, k, vis, ws)
        return vis

    def shade(self, rec: torch.Tensor, base: int, scene, albedo, lights, n_lights: int, cam,
              vis: torch.Tensor) -> torch.Tensor:
        """Colours of the pixels whose winner this rank holds; zero elsewhere."""
        rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device=self.device)
        ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES, self.device)
        fhv.fhv_shade_owned(rec if rec.shape[0] else None, rec.shape[0], None, base, scene, albedo, lights, n_lights,
                            cam, vis, rgba, ws)
        return rgba


@dataclass
class ShardedPofa:
    """This rank's contiguous slice of the POFA of all ranks' records."""
    rec: torch.Tensor  # [n_r, 2] int64: this rank's slice of the POFA
    base: int  # global index of its first record
    total: int  # records over all ranks
    bounds: np.ndarray  # ownership ranges (octants of level `level`)
    level: int


def build_pofa(local_rec: torch.Tensor, depth: int, comm: Comm, ops) -> ShardedPofa:
    """The POFA of all ranks' records (each rank passes the [n, 2] int64
    records it captured); returns this rank's contiguous slice of it."""
    return _exchange(ops.compact(local_rec), depth, comm, ops)


def capture_pofa(scene, src, mode: int, cam, pitch: float, depth: int, comm: Comm, ops) -> ShardedPofa:
    """The POFA of a whole scene captured by all ranks: `scene` (the host
    scene, the same on every rank) gives the triangle ranges, contiguous and
    of about equal estimated samples; rank r builds the POFA of its range
    from `src` (what `ops` captures from: a DeviceScene for DeviceOps) and
    the exchange follows. Returns this rank's contiguous slice."""
    b = balanced_bounds(sample_weights(scene, mode, pitch, cam), comm.world)
    mine = ops.capture(src, int(b[comm.rank]), int(b[comm.rank + 1]), mode, cam, pitch)
    return _exchange(mine, depth, comm, ops)


def _exchange(mine: LocalPofa, depth: int, comm: Comm, ops) -> ShardedPofa:
    """Morton-range ownership from the ranks' local POFAs: histogram,
    ranges, one all-to-all of records, compaction of what each owner
    receives."""
    level = min(HIST_LEVEL, depth)
    lb = mine.level_base(level)
    n_bins = 8 ** level
    hist = comm.all_reduce_sum(mine.cnt[lb: lb + n_bins].to(torch.int64))
    bounds = balanced_bounds(hist.cpu().numpy(), comm.world)
    # this rank's records of each owner's range: one contiguous slice each
    n_local = int(mine.rec.shape[0])
    inner = np.minimum(bounds[1:-1], n_bins - 1)  # a bound at the end of the level reads a valid entry, then n_local
    idx = torch.as_tensor(lb + inner, dtype=torch.int64).to(mine.off.device)
    cut = mine.off[idx].to(torch.int64).cpu().tolist() if inner.size else []
    cut = [0] + [n_local if b >= n_bins else c for b, c in zip(bounds[1:-1], cut)] + [n_local]
    counts = [cut[r + 1] - cut[r] for r in range(comm.world)]
    received = comm.all_to_all_rows(mine.rec, counts)
    del mine, idx  # the local index (dense octree arrays) is not needed past the exchange
    owned = ops.compact(received)
    sizes = comm.all_gather_int(owned.rec.shape[0])
    return ShardedPofa(owned.rec, sum(sizes[: comm.rank]), sum(sizes), bounds, level)


def render(sp: ShardedPofa, scene, albedo, lights, n_lights: int, cam, k: int, comm: Comm, ops):
    """Visibility and image of the whole POFA, identical on every rank."""
    vis = comm.all_reduce_min_u64(ops.splat(sp.rec, sp.base, scene, cam, k))
    rgba = comm.all_reduce_sum(ops.shade(sp.rec, sp.base, scene, albedo, lights, n_lights, cam, vis))
    return vis, rgba
