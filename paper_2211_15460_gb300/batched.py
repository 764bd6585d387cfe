"""Many novel views of many scenes in one call (fhv_render_views).

`build_sources` captures each scene (1-Pass/Normal POFL, then POFA) with the
regular calls and keeps only the POFA records and the material tables;
`BatchedViews` lays out the source and view descriptors on the device,
renders every view with one fhv_render_views call, can replay that call from
a CUDA graph, and `autotune` picks the work decomposition (views per item,
fragments per item, pixels per item, CTAs per SM, splat mode) by timing candidates,
caching the choice in a JSON file keyed by GPU and workload.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np

from . import fhv, scenes

DEFAULT_CONFIG = (8, 2048, 4096, 0, 0)


class BuiltSource:
    """The POFA records of one scene plus what shading needs."""

    def __init__(self, scene, records, n, device_scene):
        self.scene = scene
        self.records = records  # int64 [2 n]
        self.n = n
        self.ds = device_scene


def build_sources(workloads, device="cuda"):
    """Capture each workload's scene into a POFA (depth = workload.depth) and
    keep the records. Dense per-depth arrays are allocated once and reused."""
    import torch

    out = []
    dense = {}
    for w in workloads:
        d = w.depth
        if d not in dense:
            dense.clear()
            torch.cuda.empty_cache()
            m = fhv.fhv_level_offset(d + 1)
            dense[d] = (torch.empty(1 << (3 * d), dtype=torch.int32, device=device),
                        torch.empty(max(fhv.fhv_level_offset(d), 4), dtype=torch.int32, device=device),
                        torch.empty(m, dtype=torch.int32, device=device), torch.empty(m, dtype=torch.int32, device=device))
        leaf, levels, off, cnt = dense[d]
        ds = fhv.DeviceScene(w.scene, device)
        ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, w.scene.n_tri, 1, 1, d, 0).workspace_bytes, device)
        cap = max(1024, w.capture.width * w.capture.height * 2)
        while True:
            fb = fhv.FragBuf(cap, device)
            fhv.fhv_build_pofl(ds, fhv.FHV_CAPTURE_NORMAL, w.capture, w.normal_pitch, d, leaf, levels, fb, ws)
            st, n = fhv.fhv_get_count(fb)
            if st != fhv.FHV_ERR_OVERFLOW:
                break
            cap = n
        pofa = torch.empty(max(n, 1) * 2, dtype=torch.int64, device=device)
        wsc = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, d, n).workspace_bytes, device)
        fhv.fhv_compact_pofa(fb.rec, n, None, d, pofa, off, cnt, wsc)
        torch.cuda.synchronize()
        out.append(BuiltSource(w.scene, pofa, n, ds))
        del fb, ws, wsc
    dense.clear()
    torch.cuda.empty_cache()
    return out


class BatchedViews:
    """Views of several built sources, rendered by one fhv_render_views call."""

    def __init__(self, sources, views_per_source, lights, footprint_k=1, device="cuda"):
        import torch

        self.sources = sources
        self.k = int(footprint_k)
        self.lights = torch.from_numpy(np.ascontiguousarray(lights, np.float32).reshape(-1)).to(device)
        self.n_lights = int(np.asarray(lights).reshape(-1, 8).shape[0])
        src_structs = []
        for s in sources:
            x = fhv.fhv_splat_source()
            x.d_frag, x.n_max, x.d_n = s.records.data_ptr(), s.n, None
            x.tri_material, x.albedo = s.ds.tri_material.data_ptr(), s.ds.albedo.data_ptr()
            x.cube_min[:] = s.ds.cube_min
            x.cube_side = s.ds.cube_side
            src_structs.append(x)
        self.cams, self.view_src, self.vis, self.rgba = [], [], [], []
        view_structs = []
        for si, cams in enumerate(views_per_source):
            for cam in cams:
                v = fhv.fhv_view()
                v.cam = fhv.camera_struct(cam)
                v.source = si
                vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device=device)
                rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device=device)
                v.d_vis, v.d_rgba = vis.data_ptr(), rgba.data_ptr()
                self.cams.append(cam)
                self.view_src.append(si)
                self.vis.append(vis)
                self.rgba.append(rgba)
                view_structs.append(v)
        self.n_views = len(view_structs)
        self.d_sources = fhv.device_structs(src_structs, device)
        self.d_views = fhv.device_structs(view_structs, device)
        self.ws = fhv.workspace(fhv.fhv_batch_workspace_size(self.n_views), device)
        self.config = fhv.fhv_batch_config(*DEFAULT_CONFIG)
        self.config_tuple = tuple(DEFAULT_CONFIG)
        self.graph = None

    def set_config(self, cfg):
        """Use the work decomposition `cfg` (an fhv_batch_config tuple; a
        missing splat_mode field means 0) from now on."""
        cfg = tuple(cfg) + (0,) * (5 - len(cfg))
        self.config = fhv.fhv_batch_config(*cfg)
        self.config_tuple = cfg
        self.graph = None

    def render(self, stream=None):
        """Every view of every source in one fhv_render_views call."""
        fhv.fhv_render_views(self.d_sources, len(self.sources), self.d_views, self.n_views, self.lights, self.n_lights,
                             self.k, self.config, self.ws, stream)

    def capture_graph(self):
        """Record one render call into a CUDA graph (replayed by `replay`)."""
        import torch

        self.render()  # warm (first call sets kernel attributes outside capture)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.render(s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g

    def replay(self):
        """Replay the CUDA graph recorded by capture_graph."""
        self.graph.replay()

    def render_one_by_one(self, stream=None):
        """The same views through fhv_render_view, one call per view."""
        for i, cam in enumerate(self.cams):
            s = self.sources[self.view_src[i]]
            fhv.fhv_render_view(s.records, s.n, None, s.ds, s.ds.albedo, self.lights, self.n_lights, cam, self.k,
                                self.vis[i], self.rgba[i], self.ws_single, stream)

    @property
    def ws_single(self):
        """Workspace of the one-call-per-view comparison, allocated on first use."""
        if not hasattr(self, "_ws_single"):
            self._ws_single = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
        return self._ws_single


def _time(fn, reps):
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_cache_path():
    """JSON file of autotuned decompositions (FHV_TUNE_CACHE, else under ~/.cache)."""
    return os.environ.get("FHV_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fhv_gb300", "batch_tune.json"))


_DIGEST = None


def library_digest():
    """Short digest of the loaded libfhv.so: a rebuilt library is tuned anew."""
    global _DIGEST
    if _DIGEST is None:
        import hashlib

        with open(fhv.library_path(), "rb") as f:
            _DIGEST = hashlib.sha1(f.read()).hexdigest()[:12]
    return _DIGEST


def autotune(bv: BatchedViews, reps=3, candidates=None, signature=None):
    """Pick the fastest work decomposition for this batch; cached by GPU name
    and workload signature. Returns (config, ms, table)."""
    import torch

    sig = signature or f"views{bv.n_views}_src{len(bv.sources)}_frags{sum(s.n for s in bv.sources)}"
    key = f"{torch.cuda.get_device_name()}|{library_digest()}|{sig}"
    path = tune_cache_path()
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        cfg = tuple(cache[key]["config"])
        bv.set_config(cfg)
        return cfg, cache[key]["ms"], cache[key].get("table", [])
    if candidates is None:
        candidates = list(itertools.product((1, 4, 8, 16, 32), (512, 1024, 2048), (2048, 8192), (0,), (0, 4)))
    table = []
    for cfg in candidates:
        bv.set_config(cfg)
        table.append((cfg, _time(bv.render, reps)))
    best = min(table, key=lambda t: t[1])
    bv.set_config(best[0])
    cache[key] = {"config": list(best[0]), "ms": best[1], "table": [[list(c), m] for c, m in table]}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best[0], best[1], table


# --------------------------------------------------------------- workloads

def batched_workloads(n_scenes=16, width=1280, height=720, n_views=64, seed=300, lo=10_000, hi=2_000_000):
    """Seeded scenes of uneven size (geometric from `lo` to `hi` triangles),
    cycling spheres / heightfield with boxes / boxes only; depth 10 above
    500k triangles, else 9; `n_views` orbit views each (360 degrees). Sphere
    radii shrink as the cube root of 8 / count, boxes have sides
    U[0.005, 0.05]."""
    ws = []
    for s in range(n_scenes):
        target = lo * (hi / lo) ** (s / max(n_scenes - 1, 1))
        kind = s % 3
        if kind == 0:  # radii shrink with the count (constant total volume as for 8 spheres)
            ns = max(1, int(round(target / 960)))
            sc = scenes.spheres_scene(seed + s, n_spheres=ns, radius_scale=min(1.0, (8.0 / ns) ** (1.0 / 3.0)))
        elif kind == 1:
            grid = max(8, int(round((target / 2) ** 0.5)) + 1)
            sc = scenes.terrain_scene(seed + s, grid=grid, n_boxes=max(1, grid // 8))
        else:
            sc = scenes.boxes_scene(seed + s, n_boxes=max(1, int(round(target / 12))))
        cap = scenes.orbit_camera(sc, width, height)
        views = [scenes.orbit_camera(sc, width, height, orbit_deg=360.0 * v / n_views) for v in range(n_views)]
        depth = 10 if sc.n_tri > 500_000 else 9
        lights = np.stack([scenes.directional_light((1.0, 1.0, 1.0), (0.8, 0.8, 0.8)),
                           scenes.point_light(sc.center + np.array([0.0, 1.0, 0.0]), (0.3, 0.3, 0.3))])
        ws.append(scenes.Workload(f"batch{s}", sc, cap, depth, views, lights))
    return ws
