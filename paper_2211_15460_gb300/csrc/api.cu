// api.cu -- the C ABI of include/fhv.h: argument checks on the host, carving
// of the caller's workspace, and the launch sequence of each call. No entry
// point allocates memory.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.h"

using namespace fhv;

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

bool scene_ok(const fhv_scene* s) {
  if (!s) return false;
  if (!finite_pos(s->cube_side)) return false;
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(s->cube_min[c])) return false;
  if (s->n_tri > 0 && (!s->idx || !s->pos || !s->nrm || s->n_vtx == 0)) return false;
  if ((unsigned long long)s->tri_base + s->n_tri >= 0xffffffffull) return false;
  return true;
}

bool camera_ok(const fhv_ortho_camera* c) {
  if (!c) return false;
  if (!finite_pos(c->pitch) || c->width < 1 || c->height < 1) return false;
  if ((unsigned long long)c->width * (unsigned long long)c->height > (1ull << 31)) return false;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->origin[k]) || !std::isfinite(c->right[k]) || !std::isfinite(c->up[k]) ||
        !std::isfinite(c->fwd[k]))
      return false;
  return true;
}

bool frags_ok(const fhv_frag_buf* f, bool need_next = true) {
  if (!f || !f->d_count || !aligned16(f->d_count)) return false;
  if (f->capacity > 0x7fffffffull) return false;
  if (f->capacity > 0 && (!f->rec || !aligned16(f->rec))) return false;
  if (need_next && f->capacity > 0 && (!f->next || !aligned16(f->next))) return false;
  return true;
}

fhv_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FHV_OK : FHV_ERR_CUDA; }

void fill_scene(CaptureArgs& a, const fhv_scene* s) {
  a.idx = s->idx;
  a.pos = s->pos;
  a.nrm = s->nrm;
  a.n_tri = s->n_tri;
  a.n_vtx = s->n_vtx;
  a.tri_base = s->tri_base;
  for (int c = 0; c < 3; ++c) a.cube_min[c] = s->cube_min[c];
  a.cube_side = s->cube_side;
}

fhv_status capture_common(CaptureArgs& a, const fhv_scene* scene, const fhv_frag_buf* frags, void* d_ws,
                          size_t ws_bytes, unsigned long long n_slots, unsigned long long n_levels,
                          fhv_stream_t stream) {
  if (a.passes < 1) a.passes = 1;
  if ((unsigned long long)scene->n_tri * (unsigned long long)a.passes > 0xffffffffull) return FHV_ERR_UNSUPPORTED;
  a.n_setup = scene->n_tri * (uint32_t)a.passes;
  const CaptureWs w = capture_ws(a.n_setup);
  if (!d_ws || !aligned16(d_ws) || ws_bytes < w.total) return FHV_ERR_INVALID_ARG;
  char* ws = (char*)d_ws;
  fill_scene(a, scene);
  a.rec = reinterpret_cast<Rec*>(frags->rec);
  a.next = frags->next;
  a.capacity = frags->capacity;
  a.count = reinterpret_cast<unsigned long long*>(frags->d_count);
  a.hdr = reinterpret_cast<WsHeader*>(ws);
  a.big_setup = reinterpret_cast<TriSetup*>(ws + w.off_setup);
  a.big_meta = reinterpret_cast<unsigned long long*>(ws + w.off_meta);
  a.big_pref = reinterpret_cast<unsigned long long*>(ws + w.off_pref);
  a.big_chunk = reinterpret_cast<unsigned long long*>(ws + w.off_chunk);
  RangeFill f[4];
  int nf = 0;
  f[nf++] = RangeFill{ws, kHeaderBytes / 8ull, 0ull, 8};  // header
  if (!a.sparse_reset) f[nf++] = RangeFill{a.count, 1ull, 0ull, 8};
  const int n_first = nf;
  if (!a.sparse_reset && a.head && n_slots) f[nf++] = RangeFill{a.head, n_slots, 0xffffffffull, 4};
  if (a.levels && n_levels) f[nf++] = RangeFill{a.levels, n_levels, 0ull, 4};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  return cuda_status(launch_capture(a, f, n_first, nf, s));
}

// Projection of an octant-keyed capture: the camera (FHV_CAPTURE_VIEW) or
// the sample pitch (FHV_CAPTURE_NORMAL / FHV_CAPTURE_AXIS3).
bool set_capture_mode(CaptureArgs& a, fhv_capture_mode mode, const fhv_ortho_camera* cam, float pitch) {
  if (mode == FHV_CAPTURE_VIEW) {
    if (!camera_ok(cam)) return false;
    for (int c = 0; c < 3; ++c) {
      a.origin[c] = cam->origin[c];
      a.right[c] = cam->right[c];
      a.up[c] = cam->up[c];
    }
    a.pitch = cam->pitch;
    a.width = cam->width;
    a.height = cam->height;
    a.passes = 1;
  } else if (mode == FHV_CAPTURE_NORMAL || mode == FHV_CAPTURE_AXIS3) {
    if (!finite_pos(pitch)) return false;
    a.pitch = pitch;
    a.passes = mode == FHV_CAPTURE_AXIS3 ? 3 : 1;
  } else {
    return false;
  }
  a.mode = mode;
  return true;
}

// Workspace of the direct POFA build: the capture's (header first), then the
// compaction's (its own header slot unused: both stages share the first).
unsigned long long direct_ws_bytes(uint32_t n_setup, int depth, unsigned long long capacity) {
  return capture_ws(n_setup).total + compact_ws(depth, capacity).total;
}

}  // namespace

static fhv_status build_pofl(const fhv_scene* scene, fhv_capture_mode mode, const fhv_ortho_camera* cam, float pitch,
                             int depth, int32_t* d_leaf_head, uint32_t* d_levels, const fhv_frag_buf* frags,
                             void* d_ws, size_t ws_bytes, fhv_stream_t stream, int reuse) {
  if (!scene_ok(scene) || !frags_ok(frags) || depth < 1 || depth > 11) return FHV_ERR_INVALID_ARG;
  if (!d_leaf_head || !aligned16(d_leaf_head) || !d_levels || !aligned16(d_levels)) return FHV_ERR_INVALID_ARG;
  CaptureArgs a;
  memset(&a, 0, sizeof(a));
  if (!set_capture_mode(a, mode, cam, pitch)) return FHV_ERR_INVALID_ARG;
  a.sparse_reset = reuse;
  a.keymode = 1;
  a.depth = depth;
  a.head = d_leaf_head;
  a.levels = d_levels;
  return capture_common(a, scene, frags, d_ws, ws_bytes, 1ull << (3 * depth), level_offset(depth), stream);
}

extern "C" {

uint64_t fhv_level_offset(int level) {
  if (level < 0 || level > 12) return 0;
  return level_offset(level);
}

fhv_status fhv_memory_model(fhv_layout layout, uint64_t n_pixels, int depth, double avg_depth_complexity,
                            uint64_t n_fragments, uint32_t list_record_bytes, uint32_t array_record_bytes,
                            uint64_t* bytes) {
  if (!bytes) return FHV_ERR_INVALID_ARG;
  if ((layout == FHV_LAYOUT_POFL || layout == FHV_LAYOUT_POFA) && (depth < 0 || depth > 12))
    return FHV_ERR_INVALID_ARG;
  if (!(avg_depth_complexity >= 0.0)) return FHV_ERR_INVALID_ARG;
  const unsigned long long octants = ((1ull << (3 * (depth + 1))) - 1ull) / 7ull;
  const unsigned long long prealloc =
      (unsigned long long)std::ceil((double)n_pixels * avg_depth_complexity) * (unsigned long long)list_record_bytes;
  switch (layout) {
    case FHV_LAYOUT_PPFL:
      *bytes = n_pixels * 4ull + prealloc;
      return FHV_OK;
    case FHV_LAYOUT_POFL:
      *bytes = octants * 4ull + prealloc;
      return FHV_OK;
    case FHV_LAYOUT_POFA:
      *bytes = octants * 8ull + n_fragments * (unsigned long long)array_record_bytes;
      return FHV_OK;
  }
  return FHV_ERR_INVALID_ARG;
}

fhv_status fhv_query_sizes(fhv_layout layout, uint32_t n_tri, int32_t width, int32_t height, int depth,
                           uint64_t n_fragments, fhv_sizes* out) {
  if (!out) return FHV_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  switch (layout) {
    case FHV_LAYOUT_PPFL: {
      if (width < 1 || height < 1) return FHV_ERR_INVALID_ARG;
      out->workspace_bytes = capture_ws(n_tri).total;
      out->n_index_entries = (uint64_t)width * (uint64_t)height;
      out->index_bytes = out->n_index_entries * 4ull;
      out->fragment_bytes = n_fragments * (sizeof(fhv_record) + 4ull);
      return FHV_OK;
    }
    case FHV_LAYOUT_POFL: {
      if (depth < 1 || depth > 11) return FHV_ERR_INVALID_ARG;
      if ((unsigned long long)n_tri * 3ull > 0xffffffffull) return FHV_ERR_UNSUPPORTED;
      out->workspace_bytes = capture_ws(n_tri * 3u).total;  // covers FHV_CAPTURE_AXIS3
      out->n_index_entries = (1ull << (3 * depth)) + level_offset(depth);
      out->index_bytes = out->n_index_entries * 4ull;
      out->fragment_bytes = n_fragments * (sizeof(fhv_record) + 4ull);
      return FHV_OK;
    }
    case FHV_LAYOUT_POFA_DIRECT: {
      if (depth < 1 || depth > 11 || n_fragments >= 0xffffffffull) return FHV_ERR_INVALID_ARG;
      if ((unsigned long long)n_tri * 3ull > 0xffffffffull) return FHV_ERR_UNSUPPORTED;
      out->workspace_bytes = direct_ws_bytes(n_tri * 3u, depth, n_fragments);  // covers FHV_CAPTURE_AXIS3
      out->n_index_entries = level_offset(depth + 1);
      out->index_bytes = out->n_index_entries * 8ull;
      out->fragment_bytes = n_fragments * sizeof(fhv_record);
      return FHV_OK;
    }
    case FHV_LAYOUT_POFA_SPARSE: {
      if (depth < 1 || depth > 11 || n_fragments >= 0xffffffffull) return FHV_ERR_INVALID_ARG;
      out->workspace_bytes = sparse_ws(depth, n_fragments).total;
      // occupied octants of level l: at most min(8^l, n)
      unsigned long long e = 0;
      for (int l = 0; l <= depth; ++l) e += std::min(1ull << (3 * l), (unsigned long long)n_fragments);
      out->n_index_entries = e;
      out->index_bytes = e * sizeof(fhv_octant_entry);
      out->fragment_bytes = n_fragments * sizeof(fhv_record);
      return FHV_OK;
    }
    case FHV_LAYOUT_POFA: {
      if (depth < 1 || depth > 11) return FHV_ERR_INVALID_ARG;
      out->workspace_bytes = compact_ws(depth, n_fragments).total;
      out->n_index_entries = level_offset(depth + 1);
      out->index_bytes = out->n_index_entries * 8ull;
      out->fragment_bytes = n_fragments * sizeof(fhv_record);
      return FHV_OK;
    }
  }
  return FHV_ERR_INVALID_ARG;
}

fhv_status fhv_capture_ppfl(const fhv_scene* scene, const fhv_ortho_camera* cam, int32_t* d_head,
                            const fhv_frag_buf* frags, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_capture_ppfl");
  if (!scene_ok(scene) || !camera_ok(cam) || !d_head || !aligned16(d_head) || !frags_ok(frags))
    return FHV_ERR_INVALID_ARG;
  CaptureArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = FHV_CAPTURE_VIEW;
  for (int c = 0; c < 3; ++c) {
    a.origin[c] = cam->origin[c];
    a.right[c] = cam->right[c];
    a.up[c] = cam->up[c];
  }
  a.pitch = cam->pitch;
  a.width = cam->width;
  a.height = cam->height;
  a.keymode = 0;
  a.head = d_head;
  a.levels = nullptr;
  return capture_common(a, scene, frags, d_ws, ws_bytes, (unsigned long long)cam->width * cam->height, 0ull, stream);
}

fhv_status fhv_build_pofl(const fhv_scene* scene, fhv_capture_mode mode, const fhv_ortho_camera* cam, float pitch,
                          int depth, int32_t* d_leaf_head, uint32_t* d_levels, const fhv_frag_buf* frags, void* d_ws,
                          size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_build_pofl");
  return build_pofl(scene, mode, cam, pitch, depth, d_leaf_head, d_levels, frags, d_ws, ws_bytes, stream, 0);
}

fhv_status fhv_build_pofl_reuse(const fhv_scene* scene, fhv_capture_mode mode, const fhv_ortho_camera* cam,
                                float pitch, int depth, int32_t* d_leaf_head, uint32_t* d_levels,
                                const fhv_frag_buf* frags, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_build_pofl_reuse");
  return build_pofl(scene, mode, cam, pitch, depth, d_leaf_head, d_levels, frags, d_ws, ws_bytes, stream, 1);
}

fhv_status fhv_capture_fragments(const fhv_scene* scene, fhv_capture_mode mode, const fhv_ortho_camera* cam,
                                 float pitch, const fhv_frag_buf* frags, void* d_ws, size_t ws_bytes,
                                 fhv_stream_t stream) {
  ApiRange range_("fhv_capture_fragments");
  if (!scene_ok(scene) || !frags_ok(frags, false)) return FHV_ERR_INVALID_ARG;
  CaptureArgs a;
  memset(&a, 0, sizeof(a));
  if (!set_capture_mode(a, mode, cam, pitch)) return FHV_ERR_INVALID_ARG;
  a.keymode = 2;
  a.head = nullptr;
  a.levels = nullptr;
  fhv_frag_buf f = *frags;
  f.next = nullptr;
  return capture_common(a, scene, &f, d_ws, ws_bytes, 0ull, 0ull, stream);
}

fhv_status fhv_build_pofa_direct(const fhv_scene* scene, fhv_capture_mode mode, const fhv_ortho_camera* cam,
                                 float pitch, int depth, fhv_record* d_pofa, uint64_t capacity, uint64_t* d_count,
                                 uint32_t* d_off, uint32_t* d_cnt, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_build_pofa_direct");
  if (!scene_ok(scene) || depth < 1 || depth > 11 || capacity >= 0xffffffffull) return FHV_ERR_INVALID_ARG;
  if (!d_count || !aligned16(d_count) || !d_off || !d_cnt || !aligned16(d_off) || !aligned16(d_cnt))
    return FHV_ERR_INVALID_ARG;
  if (capacity > 0 && (!d_pofa || !aligned16(d_pofa))) return FHV_ERR_INVALID_ARG;
  CaptureArgs a;
  memset(&a, 0, sizeof(a));
  if (!set_capture_mode(a, mode, cam, pitch)) return FHV_ERR_INVALID_ARG;
  if ((unsigned long long)scene->n_tri * (unsigned long long)a.passes > 0xffffffffull) return FHV_ERR_UNSUPPORTED;
  a.n_setup = scene->n_tri * (uint32_t)a.passes;
  const CaptureWs w = capture_ws(a.n_setup);
  const CompactWs wc = compact_ws(depth, capacity);
  if (!d_ws || !aligned16(d_ws) || ws_bytes < direct_ws_bytes(a.n_setup, depth, capacity)) return FHV_ERR_INVALID_ARG;
  char* ws = (char*)d_ws;
  char* ws2 = ws + w.total;
  fill_scene(a, scene);
  a.keymode = 1;
  a.depth = depth;
  a.count = reinterpret_cast<unsigned long long*>(d_count);
  a.hdr = reinterpret_cast<WsHeader*>(ws);
  a.big_setup = reinterpret_cast<TriSetup*>(ws + w.off_setup);
  a.big_meta = reinterpret_cast<unsigned long long*>(ws + w.off_meta);
  a.big_pref = reinterpret_cast<unsigned long long*>(ws + w.off_pref);
  a.big_chunk = reinterpret_cast<unsigned long long*>(ws + w.off_chunk);
  CompactArgs c;
  memset(&c, 0, sizeof(c));
  c.n_max = capacity;
  c.d_n = &a.hdr->n_kept;
  c.depth = depth;
  c.out = reinterpret_cast<Rec*>(d_pofa);
  c.off = d_off;
  c.cnt = d_cnt;
  c.hdr = a.hdr;
  c.tile_state = reinterpret_cast<unsigned long long*>(ws2 + wc.off_state);
  c.huge_list = reinterpret_cast<unsigned long long*>(ws2 + wc.off_huge);
  c.huge_max = wc.huge_max;
  c.scratch = reinterpret_cast<Rec*>(ws2 + wc.off_scratch);
  RangeFill f[4];
  int nf = 0;
  f[nf++] = RangeFill{ws, kHeaderBytes / 8ull, 0ull, 8};  // shared header
  f[nf++] = RangeFill{d_count, 1ull, 0ull, 8};
  f[nf++] = RangeFill{c.tile_state, wc.tiles, 0ull, 8};
  const int T = depth > 4 ? depth - 4 : 0;
  if (T >= 1) f[nf++] = RangeFill{d_cnt + level_offset(T), 1ull << (3 * T), 0ull, 4};  // tile-parent counters
  return cuda_status(launch_pofa_direct(a, c, f, nf, nf, reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_compact_pofa(const fhv_record* d_in, uint64_t n_max, const uint64_t* d_n, int depth, fhv_record* d_pofa,
                            uint32_t* d_off, uint32_t* d_cnt, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_compact_pofa");
  if (depth < 1 || depth > 11 || n_max >= 0xffffffffull) return FHV_ERR_INVALID_ARG;
  if (!d_off || !d_cnt || !aligned16(d_off) || !aligned16(d_cnt)) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (!d_in || !d_pofa || !aligned16(d_in) || !aligned16(d_pofa))) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (const void*)d_in < (const void*)(d_pofa + n_max) && (const void*)d_pofa < (const void*)(d_in + n_max))
    return FHV_ERR_INVALID_ARG;
  if (d_n && !aligned16(d_n)) return FHV_ERR_INVALID_ARG;
  const CompactWs w = compact_ws(depth, n_max);
  if (!d_ws || !aligned16(d_ws) || ws_bytes < w.total) return FHV_ERR_INVALID_ARG;
  char* ws = (char*)d_ws;
  CompactArgs a;
  memset(&a, 0, sizeof(a));
  a.in = reinterpret_cast<const Rec*>(d_in);
  a.n_max = n_max;
  a.d_n = reinterpret_cast<const unsigned long long*>(d_n);
  a.depth = depth;
  a.out = reinterpret_cast<Rec*>(d_pofa);
  a.off = d_off;
  a.cnt = d_cnt;
  a.hdr = reinterpret_cast<WsHeader*>(ws);
  a.tile_state = reinterpret_cast<unsigned long long*>(ws + w.off_state);
  a.huge_list = reinterpret_cast<unsigned long long*>(ws + w.off_huge);
  a.huge_max = w.huge_max;
  a.scratch = reinterpret_cast<Rec*>(ws + w.off_scratch);
  RangeFill f[3];
  int nf = 0;
  f[nf++] = RangeFill{ws, (w.off_state + w.tiles * 8ull) / 8ull, 0ull, 8};  // header + tile states
  const int T = depth > 4 ? depth - 4 : 0;
  if (T >= 1) f[nf++] = RangeFill{d_cnt + level_offset(T), 1ull << (3 * T), 0ull, 4};  // tile-parent counters
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_fill(f, nf, s) != cudaSuccess) return FHV_ERR_CUDA;
  return cuda_status(launch_compact(a, s));
}

fhv_status fhv_compact_pofa_sparse(const fhv_record* d_in, uint64_t n_max, const uint64_t* d_n, int depth,
                                   fhv_record* d_pofa, fhv_octant_entry* d_index, uint64_t index_capacity,
                                   uint64_t* d_level_base, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_compact_pofa_sparse");
  if (depth < 1 || depth > 11 || n_max >= 0xffffffffull) return FHV_ERR_INVALID_ARG;
  if (!d_level_base || !aligned16(d_level_base)) return FHV_ERR_INVALID_ARG;
  if (index_capacity > 0 && (!d_index || !aligned16(d_index))) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (!d_in || !d_pofa || !aligned16(d_in) || !aligned16(d_pofa))) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (const void*)d_in < (const void*)(d_pofa + n_max) && (const void*)d_pofa < (const void*)(d_in + n_max))
    return FHV_ERR_INVALID_ARG;
  if (d_n && !aligned16(d_n)) return FHV_ERR_INVALID_ARG;
  const SparseWs w = sparse_ws(depth, n_max);
  if (!d_ws || !aligned16(d_ws) || ws_bytes < w.total) return FHV_ERR_INVALID_ARG;
  char* ws = (char*)d_ws;
  SparseArgs a;
  memset(&a, 0, sizeof(a));
  a.in = reinterpret_cast<const Rec*>(d_in);
  a.n_max = n_max;
  a.d_n = reinterpret_cast<const unsigned long long*>(d_n);
  a.depth = depth;
  a.B = w.B;
  a.leaf_bits = 3 * (depth - w.B);
  a.out = reinterpret_cast<Rec*>(d_pofa);
  a.scratch = reinterpret_cast<Rec*>(ws + w.off_scratch);
  a.n_buckets = w.n_buckets;
  a.bcnt = reinterpret_cast<uint32_t*>(ws + w.off_bcnt);
  a.boff = reinterpret_cast<uint32_t*>(ws + w.off_boff);
  a.bcur = reinterpret_cast<uint32_t*>(ws + w.off_bcur);
  a.blist = reinterpret_cast<uint32_t*>(ws + w.off_blist);
  a.chunk_sum = reinterpret_cast<uint32_t*>(ws + w.off_chunk);
  a.level_total = reinterpret_cast<unsigned long long*>(ws + w.off_chunk + round256(w.n_chunks * 4ull));
  a.n_tiles = w.n_tiles;
  a.tile_lvl = reinterpret_cast<uint32_t*>(ws + w.off_tiles);
  a.index = d_index;
  a.index_capacity = index_capacity;
  a.level_base = reinterpret_cast<unsigned long long*>(d_level_base);
  a.huge = reinterpret_cast<unsigned long long*>(ws + w.off_huge);
  a.huge_max = w.huge_max;
  a.hdr = reinterpret_cast<WsHeader*>(ws);
  RangeFill f[2];
  f[0] = RangeFill{ws, kHeaderBytes / 8ull, 0ull, 8};
  f[1] = RangeFill{a.bcnt, w.n_buckets, 0ull, 4};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_fill(f, 2, s) != cudaSuccess) return FHV_ERR_CUDA;
  return cuda_status(launch_compact_sparse(a, s));
}

fhv_status fhv_render_view(const fhv_record* d_frag, uint64_t n_max, const uint64_t* d_n, const fhv_scene* scene,
                           const float* d_albedo, const float* d_lights, int n_lights, const fhv_ortho_camera* cam,
                           int footprint_k, uint64_t* d_vis, float* d_rgba, void* d_ws, size_t ws_bytes,
                           fhv_stream_t stream) {
  ApiRange range_("fhv_render_view");
  if (!scene_ok(scene) || !camera_ok(cam) || footprint_k < 1 || footprint_k > 16) return FHV_ERR_INVALID_ARG;
  if (n_lights < 0 || n_lights > 64 || (n_lights > 0 && !d_lights)) return FHV_ERR_INVALID_ARG;
  if (!std::isfinite(cam->z0) || !std::isfinite(cam->z1) || !(cam->z1 > cam->z0)) return FHV_ERR_INVALID_ARG;
  if (n_max >= (1ull << kIdxBits)) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (!d_frag || !aligned16(d_frag) || !scene->tri_material || !d_albedo)) return FHV_ERR_INVALID_ARG;
  if (!d_vis || !d_rgba || !aligned16(d_vis) || !aligned16(d_rgba)) return FHV_ERR_INVALID_ARG;
  if (!d_ws || !aligned16(d_ws) || ws_bytes < FHV_RENDER_WS_BYTES) return FHV_ERR_INVALID_ARG;
  RenderArgs a;
  memset(&a, 0, sizeof(a));
  a.rec = reinterpret_cast<const Rec*>(d_frag);
  a.n_max = n_max;
  a.d_n = reinterpret_cast<const unsigned long long*>(d_n);
  a.tri_material = scene->tri_material;
  a.albedo = d_albedo;
  a.lights = d_lights;
  a.n_lights = n_lights;
  for (int c = 0; c < 3; ++c) {
    a.cube_min[c] = scene->cube_min[c];
    a.origin[c] = cam->origin[c];
    a.right[c] = cam->right[c];
    a.up[c] = cam->up[c];
    a.fwd[c] = cam->fwd[c];
  }
  a.cube_side = scene->cube_side;
  a.pitch = cam->pitch;
  a.width = cam->width;
  a.height = cam->height;
  a.z0 = cam->z0;
  a.z1 = cam->z1;
  a.k = footprint_k;
  a.vis = reinterpret_cast<unsigned long long*>(d_vis);
  a.rgba = d_rgba;
  a.hdr = reinterpret_cast<WsHeader*>(d_ws);
  RangeFill f[2];
  f[0] = RangeFill{d_ws, kHeaderBytes / 8ull, 0ull, 8};
  f[1] = RangeFill{d_vis, (unsigned long long)cam->width * cam->height, ~0ull, 8};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_fill(f, 2, s) != cudaSuccess) return FHV_ERR_CUDA;
  return cuda_status(launch_render(a, s));
}

fhv_status fhv_wait_probe(int kind, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  if (kind < 0 || kind > 2) return FHV_ERR_INVALID_ARG;
  if (!d_ws || !aligned16(d_ws) || ws_bytes < FHV_WAIT_PROBE_WS_BYTES) return FHV_ERR_INVALID_ARG;
  RangeFill f[1];
  f[0] = RangeFill{d_ws, FHV_WAIT_PROBE_WS_BYTES / 8ull, 0ull, 8};  // header and look-back states
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_fill(f, 1, s) != cudaSuccess) return FHV_ERR_CUDA;
  return cuda_status(launch_wait_probe(d_ws, kind, s));
}

fhv_status fhv_pofa_leaf_index(const fhv_record* d_pofa, uint64_t n_max, const uint64_t* d_n, int depth,
                               uint64_t* d_leaf, uint32_t* d_off, uint32_t* d_cnt, uint64_t* d_m, void* d_ws,
                               size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_pofa_leaf_index");
  if (depth < 1 || depth > 11 || n_max >= 0xffffffffull) return FHV_ERR_INVALID_ARG;
  if (!d_m || !aligned16(d_m) || (d_n && !aligned16(d_n))) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (!d_pofa || !aligned16(d_pofa) || !d_leaf || !d_off || !d_cnt)) return FHV_ERR_INVALID_ARG;
  const unsigned long long tiles = leaf_index_tiles(n_max);
  if (!d_ws || !aligned16(d_ws) || ws_bytes < FHV_LEAF_INDEX_WS_BYTES(n_max)) return FHV_ERR_INVALID_ARG;
  LeafIndexArgs a;
  memset(&a, 0, sizeof(a));
  a.pofa = reinterpret_cast<const Rec*>(d_pofa);
  a.n_max = n_max;
  a.d_n = reinterpret_cast<const unsigned long long*>(d_n);
  a.depth = depth;
  a.leaf = reinterpret_cast<unsigned long long*>(d_leaf);
  a.off = d_off;
  a.cnt = d_cnt;
  a.d_m = reinterpret_cast<unsigned long long*>(d_m);
  a.tile_off = reinterpret_cast<unsigned long long*>(d_ws);
  a.tile_sum = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(d_ws) + tiles * 8ull);
  return cuda_status(launch_leaf_index(a, reinterpret_cast<cudaStream_t>(stream)));
}

// Fills the fields of RenderArgs shared by the split render entry points.
static bool split_render_args(RenderArgs& a, const fhv_record* d_frag, uint64_t n_max, const uint64_t* d_n,
                              uint64_t index_base, const fhv_scene* scene, const fhv_ortho_camera* cam,
                              uint64_t* d_vis, void* d_ws, size_t ws_bytes) {
  if (!scene_ok(scene) || !camera_ok(cam)) return false;
  if (!std::isfinite(cam->z0) || !std::isfinite(cam->z1) || !(cam->z1 > cam->z0)) return false;
  if (n_max >= (1ull << kIdxBits) || index_base >= (1ull << kIdxBits) || n_max > (1ull << kIdxBits) - index_base)
    return false;
  if (n_max > 0 && (!d_frag || !aligned16(d_frag))) return false;
  if (!d_vis || !aligned16(d_vis) || !d_ws || !aligned16(d_ws) || ws_bytes < FHV_RENDER_WS_BYTES) return false;
  memset(&a, 0, sizeof(a));
  a.rec = reinterpret_cast<const Rec*>(d_frag);
  a.n_max = n_max;
  a.d_n = reinterpret_cast<const unsigned long long*>(d_n);
  a.tri_material = scene->tri_material;
  for (int c = 0; c < 3; ++c) {
    a.cube_min[c] = scene->cube_min[c];
    a.origin[c] = cam->origin[c];
    a.right[c] = cam->right[c];
    a.up[c] = cam->up[c];
    a.fwd[c] = cam->fwd[c];
  }
  a.cube_side = scene->cube_side;
  a.pitch = cam->pitch;
  a.width = cam->width;
  a.height = cam->height;
  a.z0 = cam->z0;
  a.z1 = cam->z1;
  a.vis = reinterpret_cast<unsigned long long*>(d_vis);
  a.hdr = reinterpret_cast<WsHeader*>(d_ws);
  a.index_base = index_base;
  return true;
}

fhv_status fhv_splat_visibility(const fhv_record* d_frag, uint64_t n_max, const uint64_t* d_n, uint64_t index_base,
                                const fhv_scene* scene, const fhv_ortho_camera* cam, int footprint_k,
                                uint64_t* d_vis, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_splat_visibility");
  RenderArgs a;
  if (footprint_k < 1 || footprint_k > 16) return FHV_ERR_INVALID_ARG;
  if (!split_render_args(a, d_frag, n_max, d_n, index_base, scene, cam, d_vis, d_ws, ws_bytes))
    return FHV_ERR_INVALID_ARG;
  a.k = footprint_k;
  RangeFill f[2];
  f[0] = RangeFill{d_ws, kHeaderBytes / 8ull, 0ull, 8};
  f[1] = RangeFill{d_vis, (unsigned long long)cam->width * cam->height, ~0ull, 8};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_fill(f, 2, s) != cudaSuccess) return FHV_ERR_CUDA;
  return cuda_status(launch_splat(a, s));
}

fhv_status fhv_shade_owned(const fhv_record* d_frag, uint64_t n_max, const uint64_t* d_n, uint64_t index_base,
                           const fhv_scene* scene, const float* d_albedo, const float* d_lights, int n_lights,
                           const fhv_ortho_camera* cam, const uint64_t* d_vis, float* d_rgba, void* d_ws,
                           size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_shade_owned");
  RenderArgs a;
  if (n_lights < 0 || n_lights > 64 || (n_lights > 0 && !d_lights)) return FHV_ERR_INVALID_ARG;
  if (!split_render_args(a, d_frag, n_max, d_n, index_base, scene, cam, const_cast<uint64_t*>(d_vis), d_ws,
                         ws_bytes))
    return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (!scene->tri_material || !d_albedo)) return FHV_ERR_INVALID_ARG;
  if (!d_rgba || !aligned16(d_rgba)) return FHV_ERR_INVALID_ARG;
  a.albedo = d_albedo;
  a.lights = d_lights;
  a.n_lights = n_lights;
  a.rgba = d_rgba;
  a.k = 1;
  return cuda_status(launch_shade_owned(a, reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_raycast_pofa(const fhv_record* d_pofa, uint64_t n_max, const uint32_t* d_off, const uint32_t* d_cnt,
                            int depth, const fhv_scene* scene, const float* d_albedo, const float* d_alpha,
                            float t_stop, const float* d_lights, int n_lights, const fhv_ortho_camera* cam,
                            uint64_t* d_vis, float* d_rgba, void* d_ws, size_t ws_bytes, fhv_stream_t stream) {
  ApiRange range_("fhv_raycast_pofa");
  if (!scene_ok(scene) || !camera_ok(cam) || depth < 1 || depth > kRayMaxDepth) return FHV_ERR_INVALID_ARG;
  if (n_lights < 0 || n_lights > 64 || (n_lights > 0 && !d_lights)) return FHV_ERR_INVALID_ARG;
  if (!std::isfinite(cam->z0) || !std::isfinite(cam->z1) || !(cam->z1 > cam->z0)) return FHV_ERR_INVALID_ARG;
  if (!(t_stop >= 0.0f && t_stop < 1.0f)) return FHV_ERR_INVALID_ARG;
  if (n_max >= (1ull << kIdxBits)) return FHV_ERR_INVALID_ARG;
  if (!d_off || !d_cnt || !aligned16(d_off) || !aligned16(d_cnt)) return FHV_ERR_INVALID_ARG;
  if (n_max > 0 && (!d_pofa || !aligned16(d_pofa) || !scene->tri_material || !d_albedo)) return FHV_ERR_INVALID_ARG;
  if (!d_vis || !d_rgba || !aligned16(d_vis) || !aligned16(d_rgba)) return FHV_ERR_INVALID_ARG;
  if (!d_ws || !aligned16(d_ws) || ws_bytes < FHV_RENDER_WS_BYTES) return FHV_ERR_INVALID_ARG;
  RayArgs a;
  memset(&a, 0, sizeof(a));
  a.pofa = reinterpret_cast<const Rec*>(d_pofa);
  a.n_max = n_max;
  a.off = d_off;
  a.cnt = d_cnt;
  a.depth = depth;
  a.tri_material = scene->tri_material;
  a.albedo = d_albedo;
  a.alpha = d_alpha;
  a.t_stop = t_stop;
  a.lights = d_lights;
  a.n_lights = n_lights;
  for (int c = 0; c < 3; ++c) {
    a.cube_min[c] = scene->cube_min[c];
    a.origin[c] = cam->origin[c];
    a.right[c] = cam->right[c];
    a.up[c] = cam->up[c];
    a.fwd[c] = cam->fwd[c];
  }
  a.cube_side = scene->cube_side;
  a.pitch = cam->pitch;
  a.width = cam->width;
  a.height = cam->height;
  a.z0 = cam->z0;
  a.z1 = cam->z1;
  // Octant bounds in (screen s, screen t, quantised depth q), in double.
  // Margins: the float32 projection of a fragment and the float32 sums of
  // the bounds each err by a few dozen units in the last place of the
  // largest intermediate magnitude (ms, mq below take 2^-16 of it, several
  // times that), plus a constant.
  const double side = scene->cube_side, ip = 1.0 / (double)cam->pitch;
  const double qs = 16777216.0 / ((double)cam->z1 - (double)cam->z0);
  double rc[3], l1r = 0, l1u = 0, l1f = 0, Ms = 0, Mq = 0;
  for (int c = 0; c < 3; ++c) {
    rc[c] = (double)scene->cube_min[c] + 0.5 * side - (double)cam->origin[c];
    l1r += std::fabs((double)cam->right[c]);
    l1u += std::fabs((double)cam->up[c]);
    l1f += std::fabs((double)cam->fwd[c]);
    const double mag = std::fabs((double)cam->origin[c]) + std::fabs((double)scene->cube_min[c]) + side;
    Ms += mag * (std::fabs((double)cam->right[c]) + std::fabs((double)cam->up[c]));
    Mq += mag * std::fabs((double)cam->fwd[c]);
  }
  Ms = Ms * ip + (double)cam->width + (double)cam->height;
  Mq = (Mq + std::fabs((double)cam->z0) + std::fabs((double)cam->z1)) * qs;
  const double ms = Ms * std::ldexp(1.0, -16) + std::ldexp(1.0, -10);
  const double mq = Mq * std::ldexp(1.0, -16) + 4.0;
  auto dot = [](const double* v, const float* w) { return v[0] * w[0] + v[1] * w[1] + v[2] * w[2]; };
  a.root[0] = (float)(dot(rc, cam->right) * ip + 0.5 * cam->width);
  a.root[1] = (float)(dot(rc, cam->up) * ip + 0.5 * cam->height);
  a.root[2] = (float)((dot(rc, cam->fwd) - (double)cam->z0) * qs);
  double cc[3];
  for (int c = 0; c < 3; ++c) cc[c] = (double)scene->cube_min[c] - (double)cam->origin[c];
  a.corner[0] = (float)(dot(cc, cam->right) * ip + 0.5 * cam->width);
  a.corner[1] = (float)(dot(cc, cam->up) * ip + 0.5 * cam->height);
  a.corner[2] = (float)((dot(cc, cam->fwd) - (double)cam->z0) * qs);
  for (int l = 0; l <= depth; ++l) {
    const double h = std::ldexp(side, -(l + 1));  // half side of a level-l octant
    a.ext[l][0] = (float)(h * l1r * ip + ms + 0.5);
    a.ext[l][1] = (float)(h * l1u * ip + ms + 0.5);
    a.ext[l][2] = (float)(h * l1f * qs + mq);
    const double side_l = 2.0 * h;  // side of a level-l octant
    for (int ax = 0; ax < 3; ++ax) {
      a.step[l][3 * ax + 0] = (float)(side_l * cam->right[ax] * ip);
      a.step[l][3 * ax + 1] = (float)(side_l * cam->up[ax] * ip);
      a.step[l][3 * ax + 2] = (float)(side_l * cam->fwd[ax] * qs);
    }
    if (l < depth) {
      const double hc = std::ldexp(side, -(l + 2));  // half side of its children
      for (int ax = 0; ax < 3; ++ax) {
        a.child[l][3 * ax + 0] = (float)(hc * cam->right[ax] * ip);
        a.child[l][3 * ax + 1] = (float)(hc * cam->up[ax] * ip);
        a.child[l][3 * ax + 2] = (float)(hc * cam->fwd[ax] * qs);
      }
    }
  }
  a.vis = reinterpret_cast<unsigned long long*>(d_vis);
  a.rgba = d_rgba;
  a.hdr = reinterpret_cast<WsHeader*>(d_ws);
  a.slabs = reinterpret_cast<unsigned char*>(d_ws) + kHeaderBytes;
  a.n_slabs = (uint32_t)std::min<unsigned long long>(256ull, (ws_bytes - kHeaderBytes) / kRaySlabBytes);
  RangeFill f[1];
  f[0] = RangeFill{d_ws, kHeaderBytes / 8ull, 0ull, 8};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_fill(f, 1, s) != cudaSuccess) return FHV_ERR_CUDA;
  return cuda_status(launch_raycast(a, s));
}

// ------------------------------------------------------- learned gap-filler

static bool conv_pair_ok(int cin, int cout) {
  return (cin == 8 || cin == 16 || cin == 32) && (cout == 16 || cout == 32);
}

fhv_status fhv_conv3x3_bf16(const void* d_x, int n, int h, int w, int cin, const void* d_weight, const float* d_bias,
                            int cout, int relu, const void* d_mask, void* d_y, void* d_ws, fhv_stream_t stream) {
  ApiRange range_("fhv_conv3x3_bf16");
  if (n < 1 || h < 1 || w < 1 || !conv_pair_ok(cin, cout)) return FHV_ERR_INVALID_ARG;
  if ((long long)n * h * w >= (1ll << 40)) return FHV_ERR_INVALID_ARG;
  if (!d_x || !d_weight || !d_y || !aligned16(d_x) || !aligned16(d_weight) || !aligned16(d_y)) return FHV_ERR_INVALID_ARG;
  if (d_mask && !aligned16(d_mask)) return FHV_ERR_INVALID_ARG;
  if (!d_ws || !aligned16(d_ws)) return FHV_ERR_INVALID_ARG;
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.x = reinterpret_cast<const __nv_bfloat16*>(d_x);
  a.weight = reinterpret_cast<const __nv_bfloat16*>(d_weight);
  a.bias = d_bias;
  a.mask = reinterpret_cast<const __nv_bfloat16*>(d_mask);
  a.y = reinterpret_cast<__nv_bfloat16*>(d_y);
  a.n = n;
  a.h = h;
  a.w = w;
  a.cin = cin;
  a.cout = cout;
  a.relu = relu ? 1 : 0;
  a.hdr = reinterpret_cast<WsHeader*>(d_ws);
  return cuda_status(launch_conv_fwd(a, reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_conv3x3_wgrad_bf16(const void* d_x, const void* d_dy, int n, int h, int w, int cin, int cout,
                                  float* d_dweight, float* d_dbias, void* d_ws, fhv_stream_t stream) {
  ApiRange range_("fhv_conv3x3_wgrad_bf16");
  if (n < 1 || h < 1 || w < 1 || !conv_pair_ok(cin, cout)) return FHV_ERR_INVALID_ARG;
  if ((long long)n * h * w >= (1ll << 40)) return FHV_ERR_INVALID_ARG;
  if (!d_x || !d_dy || !d_dweight || !aligned16(d_x) || !aligned16(d_dy) || !aligned16(d_dweight))
    return FHV_ERR_INVALID_ARG;
  if (!d_ws || !aligned16(d_ws)) return FHV_ERR_INVALID_ARG;
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.x = reinterpret_cast<const __nv_bfloat16*>(d_x);
  a.dy = reinterpret_cast<const __nv_bfloat16*>(d_dy);
  a.dweight = d_dweight;
  a.dbias = d_dbias;
  a.n = n;
  a.h = h;
  a.w = w;
  a.cin = cin;
  a.cout = cout;
  a.hdr = reinterpret_cast<WsHeader*>(d_ws);
  return cuda_status(launch_conv_wgrad(a, reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_conv3x3_flip_bf16(const void* d_weight, int cin, int cout, void* d_flipped, fhv_stream_t stream) {
  if (!d_weight || !d_flipped || cin < 1 || cout < 1 || cin > 1024 || cout > 1024) return FHV_ERR_INVALID_ARG;
  return cuda_status(launch_conv_flip(reinterpret_cast<const __nv_bfloat16*>(d_weight), cin, cout,
                                      reinterpret_cast<__nv_bfloat16*>(d_flipped),
                                      reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_splat_features(const uint64_t* d_vis, const float* d_rgba, const fhv_record* d_frag,
                              const fhv_ortho_camera* cam, void* d_feat, fhv_stream_t stream) {
  if (!camera_ok(cam) || !d_vis || !d_rgba || !d_feat || !aligned16(d_rgba) || !aligned16(d_feat))
    return FHV_ERR_INVALID_ARG;
  if (!d_frag || !aligned16(d_frag)) return FHV_ERR_INVALID_ARG;
  return cuda_status(launch_splat_features(reinterpret_cast<const unsigned long long*>(d_vis),
                                           reinterpret_cast<const float4*>(d_rgba),
                                           reinterpret_cast<const Rec*>(d_frag), cam->right, cam->up,
                                           (long long)cam->width * cam->height,
                                           reinterpret_cast<__nv_bfloat16*>(d_feat),
                                           reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_gapfill_loss(const void* d_out, const void* d_base, const float* d_target, uint64_t pixels,
                            float grad_scale, double* d_loss_sum, void* d_grad, fhv_stream_t stream) {
  if (!d_out || !d_target || !aligned16(d_out) || !aligned16(d_target)) return FHV_ERR_INVALID_ARG;
  if ((d_grad && !aligned16(d_grad)) || (d_base && !aligned16(d_base))) return FHV_ERR_INVALID_ARG;
  if (pixels >= (1ull << 40) || !std::isfinite(grad_scale)) return FHV_ERR_INVALID_ARG;
  return cuda_status(launch_gapfill_loss(reinterpret_cast<const __nv_bfloat16*>(d_out),
                                         reinterpret_cast<const __nv_bfloat16*>(d_base),
                                         reinterpret_cast<const float4*>(d_target), (long long)pixels, grad_scale,
                                         d_loss_sum, reinterpret_cast<__nv_bfloat16*>(d_grad),
                                         reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_gapfill_compose(const void* d_out, const void* d_base, uint64_t pixels, float* d_rgba,
                               fhv_stream_t stream) {
  if (!d_out || !d_rgba || !aligned16(d_out) || !aligned16(d_rgba)) return FHV_ERR_INVALID_ARG;
  if ((d_base && !aligned16(d_base)) || pixels >= (1ull << 40)) return FHV_ERR_INVALID_ARG;
  return cuda_status(launch_gapfill_compose(reinterpret_cast<const __nv_bfloat16*>(d_out),
                                            reinterpret_cast<const __nv_bfloat16*>(d_base), (long long)pixels,
                                            reinterpret_cast<float4*>(d_rgba),
                                            reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_adam_bf16(float* d_param, float* d_grad, float* d_m, float* d_v, uint64_t n, float lr, float beta1,
                         float beta2, float eps, int step, void* d_out_bf16, fhv_stream_t stream) {
  if (!d_param || !d_grad || !d_m || !d_v || step < 1 || n >= (1ull << 40)) return FHV_ERR_INVALID_ARG;
  if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return FHV_ERR_INVALID_ARG;
  return cuda_status(launch_adam(d_param, d_grad, d_m, d_v, (long long)n, lr, beta1, beta2, eps, step,
                                 reinterpret_cast<__nv_bfloat16*>(d_out_bf16),
                                 reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_atomic_probe(uint64_t* d_buf, uint64_t n_words, int ops_per_thread, int returning,
                            uint64_t* ops_total, fhv_stream_t stream) {
  if (!d_buf || n_words < 4 || !aligned16(d_buf) || ops_per_thread < 1 || ops_per_thread > (1 << 16) ||
      returning < 0 || returning > 2)
    return FHV_ERR_INVALID_ARG;
  if (ops_total) *ops_total = (uint64_t)sm_count() * 8ull * 256ull * (uint64_t)ops_per_thread;
  return cuda_status(launch_atomic_probe(reinterpret_cast<unsigned long long*>(d_buf), n_words, ops_per_thread,
                                         returning, reinterpret_cast<cudaStream_t>(stream)));
}

fhv_status fhv_get_count(const fhv_frag_buf* frags, uint64_t* host_count, fhv_stream_t stream) {
  if (!frags || !frags->d_count || !host_count) return FHV_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long v = 0;
  if (cudaMemcpyAsync(&v, frags->d_count, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FHV_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FHV_ERR_CUDA;
  *host_count = v;
  return v > frags->capacity ? FHV_ERR_OVERFLOW : FHV_OK;
}

fhv_status fhv_read_status(const void* d_ws, uint32_t* host_status, fhv_stream_t stream) {
  if (!d_ws || !host_status) return FHV_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  if (cudaMemcpyAsync(&v, d_ws, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FHV_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FHV_ERR_CUDA;
  *host_status = v;
  return (v & FHV_DEV_TIMEOUT) ? FHV_ERR_TIMEOUT : FHV_OK;
}

const char* fhv_status_str(fhv_status st) {
  switch (st) {
    case FHV_OK: return "ok";
    case FHV_ERR_INVALID_ARG: return "invalid argument";
    case FHV_ERR_OVERFLOW: return "fragment buffer overflow";
    case FHV_ERR_CUDA: return "CUDA error";
    case FHV_ERR_TIMEOUT: return "bounded device wait expired";
    case FHV_ERR_UNSUPPORTED: return "unsupported input";
  }
  return "unknown status";
}

}  // extern "C"
