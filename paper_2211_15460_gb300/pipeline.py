"""The plain FHV path of one workload, end to end, on one GPU.

Allocates every device array with PyTorch and calls the C ABI in the
paper's order: PPFL capture (Section 3.2), POFL build, POFA compaction, then
one splat + shade per novel view (Section 3.3). Nothing synchronises the host
inside a step; the POFL counter feeds compaction and rendering on the device.
Independent calls run on their own streams, forked from and joined back into
the caller's stream: the PPFL capture (latency-bound raster kernels) beside
the POFL build and compaction (dense octree passes), and the novel views
beside each other. Each concurrent call has its own workspace. Fragment
buffers are sized by a first capture and re-allocated when it overflows, as
Section 3.1 prescribes for the next frame.
"""
from __future__ import annotations

import numpy as np

from . import fhv


class PlainFHV:
    """The plain path on one workload: device scene, buffers and workspaces allocated once, then steps of
    PPFL capture, POFL build, POFA compaction and every novel view (Sections 3.1-3.3)."""
    def __init__(self, workload, device="cuda", ppfl_capacity=None, pofl_capacity=None, pofl_mode=None):
        import torch

        self.w = workload
        self.device = device
        self.scene = fhv.DeviceScene(workload.scene, device)
        self.lights = torch.from_numpy(np.ascontiguousarray(workload.lights, np.float32).reshape(-1)).to(device)
        self.n_lights = int(workload.lights.shape[0])
        cap = workload.capture
        self.W, self.H = cap.width, cap.height
        self.depth = workload.depth
        self.mode = fhv.FHV_CAPTURE_NORMAL if pofl_mode is None else pofl_mode
        T = workload.scene.n_tri
        self.ws_capture = fhv.workspace(  # POFL build
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, T, self.W, self.H, self.depth, 0).workspace_bytes, device)
        self.ws_ppfl = fhv.workspace(  # PPFL capture (may run concurrently)
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_PPFL, T, self.W, self.H, 1, 0).workspace_bytes, device)
        self.head = torch.empty(self.W * self.H, dtype=torch.int32, device=device)
        nleaf = 1 << (3 * self.depth)
        self.leaf_head = torch.empty(nleaf, dtype=torch.int32, device=device)
        self.levels = torch.empty(max(fhv.fhv_level_offset(self.depth), 4), dtype=torch.int32, device=device)
        n_oct = fhv.fhv_level_offset(self.depth + 1)
        self.off = torch.empty(n_oct, dtype=torch.int32, device=device)
        self.cnt = torch.empty(n_oct, dtype=torch.int32, device=device)
        self.ws_views = [fhv.workspace(fhv.FHV_RENDER_WS_BYTES, device) for _ in workload.views]
        self.ws_render = self.ws_views[0]
        self.side = torch.cuda.Stream(device=device)
        self.view_streams = [torch.cuda.Stream(device=device) for _ in workload.views]
        self.vis = [torch.empty(v.width * v.height, dtype=torch.int64, device=device) for v in workload.views]
        self.rgba = [torch.empty(v.width * v.height * 4, dtype=torch.float32, device=device) for v in workload.views]
        self._alloc_ppfl(ppfl_capacity or self.W * self.H * 4)
        self._alloc_pofl(pofl_capacity or self.W * self.H * 4)
        self.size_buffers()

    # ---------------------------------------------------------------- memory
    def _alloc_ppfl(self, cap):
        self.ppfl = fhv.FragBuf(cap, self.device)

    def _alloc_pofl(self, cap):
        import torch

        self.pofl = fhv.FragBuf(cap, self.device)
        self._pofl_built = False  # a new fragment buffer: the next build resets every head
        self.pofa = torch.empty(max(cap, 1) * 2, dtype=torch.int64, device=self.device)
        self.ws_compact = fhv.workspace(
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, self.depth, cap).workspace_bytes, self.device)

    def size_buffers(self):
        """Capture once; re-allocate any list that overflowed (Section 3.1)."""
        self.capture_ppfl()
        st, n = fhv.fhv_get_count(self.ppfl)
        if st == fhv.FHV_ERR_OVERFLOW:
            self._alloc_ppfl(n)
            self.capture_ppfl()
        self.build_pofl()
        st, n = fhv.fhv_get_count(self.pofl)
        if st == fhv.FHV_ERR_OVERFLOW:
            self._alloc_pofl(n)
            self.build_pofl()
        self.n_ppfl = fhv.fhv_get_count(self.ppfl)[1]
        self.n_pofl = fhv.fhv_get_count(self.pofl)[1]

    # ----------------------------------------------------------------- stages
    def capture_ppfl(self, stream=None):
        """FHV_PPFL capture from the workload's capture camera."""
        fhv.fhv_capture_ppfl(self.scene, self.w.capture, self.head, self.ppfl, self.ws_ppfl, stream)

    def build_pofl(self, stream=None):
        """POFL build; after the first one, the lists are rebuilt in place
        (only the heads the previous build wrote are reset)."""
        cam = self.w.capture
        build = fhv.fhv_build_pofl_reuse if self._pofl_built else fhv.fhv_build_pofl
        build(self.scene, self.mode, cam, self.w.normal_pitch, self.depth, self.leaf_head, self.levels, self.pofl,
              self.ws_capture, stream)
        self._pofl_built = True

    def compact_pofa(self, stream=None):
        """FHV_POFA compaction of the POFL's records (count read on the device):
        the complete octree index, or after use_sparse_index() the sparse one."""
        if getattr(self, "index", None) is not None:
            fhv.fhv_compact_pofa_sparse(self.pofl.rec, self.pofl.capacity, self.pofl.count, self.depth, self.pofa,
                                        self.index, self.index_capacity, self.level_base, self.ws_sparse, stream)
            return
        fhv.fhv_compact_pofa(self.pofl.rec, self.pofl.capacity, self.pofl.count, self.depth, self.pofa, self.off,
                             self.cnt, self.ws_compact, stream)

    def use_sparse_index(self, on: bool = True):
        """Switch the compaction to the sparse octree index (only occupied
        octants of every level; the records are the same). The index is sized
        by a first call and re-allocated from the size it reports."""
        import torch

        if not on:
            self.index = None
            return
        d = self.depth
        s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, d, self.pofl.capacity)
        self.ws_sparse = fhv.workspace(s.workspace_bytes, self.device)
        self.level_base = torch.zeros(d + 4, dtype=torch.int64, device=self.device)
        self.index_capacity = 0
        self.index = torch.empty(2, dtype=torch.int64, device=self.device)
        self.compact_pofa()
        need = int(self.level_base[d + 1].item())
        self.index_capacity = need
        self.index = torch.empty(max(need, 1) * 2, dtype=torch.int64, device=self.device)
        self.compact_pofa()

    def render(self, v: int, stream=None):
        """Novel view `v` by splatting the POFA."""
        fhv.fhv_render_view(self.pofa, self.pofl.capacity, self.pofl.count, self.scene, self.scene.albedo, self.lights,
                            self.n_lights, self.w.views[v], self.w.footprint_k, self.vis[v], self.rgba[v],
                            self.ws_views[v], stream)

    def build(self, stream=None):
        """POFL build, then POFA compaction."""
        self.build_pofl(stream)
        self.compact_pofa(stream)

    def render_all(self, stream=None):
        """Every novel view of the workload, in order."""
        for v in range(len(self.w.views)):
            self.render(v, stream)

    def step(self, stream=None, concurrent=True):
        """One pass of the whole path: build the FHV, render every view.
        Enqueued on `stream` (default: the current stream), with the PPFL
        capture and the views on forked streams joined back into it
        (concurrent=False keeps every call on `stream`, in order)."""
        import torch

        if not concurrent:
            self.capture_ppfl(stream)
            self.build(stream)
            self.render_all(stream)
            return
        main = stream if stream is not None else torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(main)
        self.side.wait_event(fork)
        self.capture_ppfl(self.side)
        self.build_pofl(main)
        self.compact_pofa(main)
        built = torch.cuda.Event()
        built.record(main)
        for v, vs in enumerate(self.view_streams):
            vs.wait_event(built)
            self.render(v, vs)
        for s in [self.side] + self.view_streams:
            done = torch.cuda.Event()
            done.record(s)
            main.wait_event(done)



class StreamingSteps:
    """Repeated end-to-end steps of a PlainFHV: every step uploads the scene
    from pinned host memory, runs the path and reads the images and the
    POFL fragment count back to pinned host memory. Uploads and read-backs
    run on their own streams beside the computation of the neighbouring
    steps: the scene inputs and the images alternate between two device
    sets (a set is written again only after the step that read it, or the
    copy that read it, has finished), and the count is snapshotted on the
    device at the end of its step."""

    def __init__(self, p: PlainFHV):
        import torch

        self.p = p
        sc, w = p.w.scene, p.w
        self.host_in = [torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32 else
                                         np.ascontiguousarray(a)).pin_memory()
                        for a in (sc.idx, sc.pos, sc.nrm, sc.tri_material, sc.albedo, w.lights.reshape(-1))]
        second = fhv.DeviceScene(sc, p.device)
        self.scenes = [p.scene, second]
        self.lights = [p.lights, torch.empty_like(p.lights)]
        self.dev_in = [[d.idx, d.pos, d.nrm, d.tri_material, d.albedo, li] for d, li in zip(self.scenes, self.lights)]
        self.rgba_sets = [list(p.rgba), [torch.empty_like(t) for t in p.rgba]]
        self.host_out = [[torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in p.rgba] for _ in range(2)]
        self.count_dev = [torch.zeros(2, dtype=torch.int64, device=p.device) for _ in range(2)]
        self.count_host = [torch.zeros(2, dtype=torch.int64).pin_memory() for _ in range(2)]
        self.up = torch.cuda.Stream(device=p.device)
        self.copy = torch.cuda.Stream(device=p.device)
        self.used = [None, None]  # set s's inputs were last read by the step that recorded this
        self.copied = [None, None]  # set s's images were last read back by the copy that recorded this
        self.k = 0

    @property
    def h2d_bytes(self) -> int:
        """Bytes copied host to device per step (the scene's arrays)."""
        return sum(t.numel() * t.element_size() for t in self.host_in)

    @property
    def d2h_bytes(self) -> int:
        """Bytes copied device to host per step (every view's image and the fragment count)."""
        return sum(t.numel() * t.element_size() for t in self.host_out[0]) + self.count_host[0].numel() * 8

    def step(self):
        """Enqueue one step; returns the index of the host buffers its results land in."""
        import torch

        p, s = self.p, self.k % 2
        main = torch.cuda.current_stream()
        if self.used[s] is not None:
            self.up.wait_event(self.used[s])
        with torch.cuda.stream(self.up):
            for h, d in zip(self.host_in, self.dev_in[s]):
                d.view(-1).copy_(h.view(-1), non_blocking=True)
        uploaded = torch.cuda.Event()
        uploaded.record(self.up)
        main.wait_event(uploaded)
        if self.copied[s] is not None:
            main.wait_event(self.copied[s])  # this image set's previous read-back is done
        p.scene, p.lights, p.rgba = self.scenes[s], self.lights[s], self.rgba_sets[s]
        p.step(main)
        self.count_dev[s].copy_(p.pofl.count)
        done = torch.cuda.Event()
        done.record(main)
        self.used[s] = done
        self.copy.wait_event(done)
        with torch.cuda.stream(self.copy):
            for h, d in zip(self.host_out[s], self.rgba_sets[s]):
                h.copy_(d, non_blocking=True)
            self.count_host[s].copy_(self.count_dev[s], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(self.copy)
        self.copied[s] = ev
        self.k += 1
        return s

    def finish(self):
        """Waits for every copy enqueued so far; leaves set 0 bound to the PlainFHV."""
        import torch

        torch.cuda.current_stream().wait_stream(self.copy)
        self.copy.synchronize()
        self.p.scene, self.p.lights, self.p.rgba = self.scenes[0], self.lights[0], self.rgba_sets[0]


class PofaViews:
    """One scene built straight into an FHV_POFA and seen from every novel
    view of its workload in one batched call: fragment capture into the
    global fragment list (Section 3.1; three-axis capture for the stress
    workload, Section 3.2's 3-Pass/1-Way), POFA compaction with the complete
    octree index (Section 3.2, Table 4), and the views splatted and shaded
    by one fhv_render_views call (Section 3.3; Section 5 submits several
    viewpoints together). The fragment buffer is sized by a first capture."""

    def __init__(self, workload, mode=None, device="cuda"):
        import torch

        from . import batched

        self.w = workload
        self.device = device
        self.mode = fhv.FHV_CAPTURE_AXIS3 if mode is None else mode
        self.depth = workload.depth
        sc = workload.scene
        self.scene = fhv.DeviceScene(sc, device)
        self.ws_capture = fhv.workspace(
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, sc.n_tri, 1, 1, self.depth, 0).workspace_bytes, device)
        probe = fhv.FragBuf(0, device, links=False)
        self.capture(frags=probe)
        self.n = fhv.fhv_get_count(probe)[1]
        del probe
        self.frags = fhv.FragBuf(self.n, device, links=False)
        n_oct = fhv.fhv_level_offset(self.depth + 1)
        self.off = torch.empty(n_oct, dtype=torch.int32, device=device)
        self.cnt = torch.empty(n_oct, dtype=torch.int32, device=device)
        self.pofa = torch.empty(max(self.n, 1) * 2, dtype=torch.int64, device=device)
        self.ws_compact = fhv.workspace(
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, self.depth, self.n).workspace_bytes, device)
        self.views = batched.BatchedViews([batched.BuiltSource(sc, self.pofa, self.n, self.scene)], [workload.views],
                                          workload.lights, workload.footprint_k, device)

    def tune_views(self, reps=2):
        """Pick the batched renderer's decomposition for these views (views per
        chunk; one fragment per thread, with or without the pixel election and the per-chunk depth pre-test, or runs of
        four) by timing a few candidates on
        the built POFA; cached like every autotuned choice. Returns
        (config, ms, table)."""
        from . import batched

        cands = [(g, 2048, 8192, 0, m) for g in (8, 16) for m in (0, 4, 5, 2)]
        return batched.autotune(self.views, reps=reps, candidates=cands,
                                signature=f"{self.w.name}_views{len(self.w.views)}_frags{self.n}")

    def capture(self, stream=None, frags=None, scene=None):
        """Fragment capture of the scene into the global fragment list (no lists)."""
        fhv.fhv_capture_fragments(scene or self.scene, self.mode, None if self.mode != fhv.FHV_CAPTURE_VIEW
                                  else self.w.capture, self.w.normal_pitch, frags or self.frags, self.ws_capture,
                                  stream)

    def compact(self, stream=None):
        """FHV_POFA compaction of the captured records (count read on the device)."""
        fhv.fhv_compact_pofa(self.frags.rec, self.n, self.frags.count, self.depth, self.pofa, self.off, self.cnt,
                             self.ws_compact, stream)

    def alloc_sparse(self):
        """Buffers of the sparse-index compaction (records into their own
        array; index sized by a first call, re-allocated if it overflows)."""
        import torch

        d = self.depth
        s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, d, self.n)
        self.sparse_pofa = torch.empty(max(self.n, 1) * 2, dtype=torch.int64, device=self.device)
        self.level_base = torch.zeros(d + 2 + 2, dtype=torch.int64, device=self.device)
        self.ws_sparse = fhv.workspace(s.workspace_bytes, self.device)
        self.index_capacity = 0
        self.index = torch.empty(2, dtype=torch.int64, device=self.device)
        self.compact_sparse()
        need = int(self.level_base[d + 1].item())
        self.index_capacity = need
        self.index = torch.empty(max(need, 1) * 2, dtype=torch.int64, device=self.device)
        self.compact_sparse()

    def compact_sparse(self, stream=None):
        """FHV_POFA compaction with the sparse index (only occupied octants, every level)."""
        fhv.fhv_compact_pofa_sparse(self.frags.rec, self.n, self.frags.count, self.depth, self.sparse_pofa,
                                    self.index, self.index_capacity, self.level_base, self.ws_sparse, stream)

    def render(self, stream=None, views=None):
        """Every novel view, one batched call."""
        (views or self.views).render(stream)

    def step(self, stream=None):
        """One pass of the whole path: capture, compaction, every view."""
        self.capture(stream)
        self.compact(stream)
        self.render(stream)


class StreamingPofaSteps:
    """End-to-end steps of a PofaViews through the public API: every step
    uploads the scene's arrays from pinned host memory, builds the POFA,
    renders every view and reads every image and the fragment count back to
    pinned host memory. Uploads and read-backs run on their own streams
    beside the neighbouring steps' computation; the device scene and the
    views' images alternate between two sets (a set is written again only
    after the step and the copy that read it have finished)."""

    def __init__(self, p: PofaViews):
        import torch

        from . import batched

        self.p = p
        sc, w = p.w.scene, p.w
        self.host_in = [torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32 else
                                         np.ascontiguousarray(a)).pin_memory()
                        for a in (sc.idx, sc.pos, sc.nrm, sc.tri_material, sc.albedo)]
        second = fhv.DeviceScene(sc, p.device)
        self.scenes = [p.scene, second]
        self.views = [p.views, batched.BatchedViews([batched.BuiltSource(sc, p.pofa, p.n, second)], [w.views],
                                                     w.lights, w.footprint_k, p.device)]
        self.views[1].set_config(tuple(p.views.config_tuple))
        self.dev_in = [[d.idx, d.pos, d.nrm, d.tri_material, d.albedo] for d in self.scenes]
        self.host_out = [[torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in v.rgba] for v in self.views]
        self.count_dev = [torch.zeros(2, dtype=torch.int64, device=p.device) for _ in range(2)]
        self.count_host = [torch.zeros(2, dtype=torch.int64).pin_memory() for _ in range(2)]
        self.up = torch.cuda.Stream(device=p.device)
        self.copy = torch.cuda.Stream(device=p.device)
        self.used = [None, None]
        self.copied = [None, None]
        self.k = 0

    @property
    def h2d_bytes(self) -> int:
        """Bytes copied host to device per step (the scene's arrays)."""
        return sum(t.numel() * t.element_size() for t in self.host_in)

    @property
    def d2h_bytes(self) -> int:
        """Bytes copied device to host per step (every view's image and the fragment count)."""
        return sum(t.numel() * t.element_size() for t in self.host_out[0]) + self.count_host[0].numel() * 8

    def step(self):
        """Enqueue one step; returns the index of the host buffers its results land in."""
        import torch

        p, s = self.p, self.k % 2
        main = torch.cuda.current_stream()
        if self.used[s] is not None:
            self.up.wait_event(self.used[s])
        with torch.cuda.stream(self.up):
            for h, d in zip(self.host_in, self.dev_in[s]):
                d.view(-1).copy_(h.view(-1), non_blocking=True)
        uploaded = torch.cuda.Event()
        uploaded.record(self.up)
        main.wait_event(uploaded)
        if self.copied[s] is not None:
            main.wait_event(self.copied[s])
        p.capture(main, scene=self.scenes[s])
        p.compact(main)
        p.render(main, views=self.views[s])
        self.count_dev[s].copy_(p.frags.count)
        done = torch.cuda.Event()
        done.record(main)
        self.used[s] = done
        self.copy.wait_event(done)
        with torch.cuda.stream(self.copy):
            for h, d in zip(self.host_out[s], self.views[s].rgba):
                h.copy_(d, non_blocking=True)
            self.count_host[s].copy_(self.count_dev[s], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(self.copy)
        self.copied[s] = ev
        self.k += 1
        return s

    def finish(self):
        """Waits for every copy enqueued so far."""
        import torch

        torch.cuda.current_stream().wait_stream(self.copy)
        self.copy.synchronize()
