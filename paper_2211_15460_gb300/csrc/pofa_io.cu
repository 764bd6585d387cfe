// pofa_io.cu -- a built FHV_POFA to and from a file (host buffers only).
// The paper keeps an FHV across frames and re-creates it only when the
// scene changes (Section 4); saving one lets a later run skip its creation.
// Plain C stdio, no device calls.
#include <cstdio>
#include <cstring>

#include "../../include/fhv.h"

namespace {

const char kMagic[8] = {'F', 'H', 'V', 'P', 'O', 'F', 'A', '1'};

bool write_all(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

unsigned long long dense_entries(int depth) { return fhv_level_offset(depth + 1); }

fhv_status read_header(FILE* f, fhv_pofa_header* h) {
  char magic[8];
  if (!read_all(f, magic, 8) || memcmp(magic, kMagic, 8) != 0) return FHV_ERR_INVALID_ARG;
  if (!read_all(f, h, sizeof(*h))) return FHV_ERR_INVALID_ARG;
  if (h->depth < 1 || h->depth > 11 || (h->index_kind != 0 && h->index_kind != 1) || h->n_records >= 0xffffffffull)
    return FHV_ERR_INVALID_ARG;
  if (h->index_kind == 0 && h->n_index_entries != dense_entries(h->depth)) return FHV_ERR_INVALID_ARG;
  return FHV_OK;
}

}  // namespace

extern "C" fhv_status fhv_pofa_save(const char* path, int depth, const fhv_record* h_pofa, uint64_t n,
                                    const uint32_t* h_off, const uint32_t* h_cnt, const fhv_octant_entry* h_index,
                                    const uint64_t* h_level_base) {
  if (!path || depth < 1 || depth > 11 || n >= 0xffffffffull || (n > 0 && !h_pofa)) return FHV_ERR_INVALID_ARG;
  const bool dense = h_off && h_cnt;
  const bool sparse = h_index && h_level_base;
  if (dense == sparse) return FHV_ERR_INVALID_ARG;  // exactly one index
  fhv_pofa_header h;
  memset(&h, 0, sizeof(h));
  h.depth = depth;
  h.index_kind = dense ? 0 : 1;
  h.n_records = n;
  h.n_index_entries = dense ? dense_entries(depth) : h_level_base[depth + 1];
  FILE* f = fopen(path, "wb");
  if (!f) return FHV_ERR_INVALID_ARG;
  bool ok = write_all(f, kMagic, 8) && write_all(f, &h, sizeof(h)) && write_all(f, h_pofa, n * sizeof(fhv_record));
  if (dense) {
    ok = ok && write_all(f, h_off, h.n_index_entries * 4) && write_all(f, h_cnt, h.n_index_entries * 4);
  } else {
    ok = ok && write_all(f, h_level_base, (size_t)(depth + 2) * 8) &&
         write_all(f, h_index, h.n_index_entries * sizeof(fhv_octant_entry));
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? FHV_OK : FHV_ERR_INVALID_ARG;
}

extern "C" fhv_status fhv_pofa_load_header(const char* path, fhv_pofa_header* out) {
  if (!path || !out) return FHV_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return FHV_ERR_INVALID_ARG;
  const fhv_status st = read_header(f, out);
  fclose(f);
  return st;
}

extern "C" fhv_status fhv_pofa_load(const char* path, fhv_record* h_pofa, uint64_t record_capacity, uint32_t* h_off,
                                    uint32_t* h_cnt, fhv_octant_entry* h_index, uint64_t index_capacity,
                                    uint64_t* h_level_base) {
  if (!path) return FHV_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return FHV_ERR_INVALID_ARG;
  fhv_pofa_header h;
  fhv_status st = read_header(f, &h);
  if (st == FHV_OK) {
    const bool dense = h.index_kind == 0;
    if (h.n_records > record_capacity || (h.n_records > 0 && !h_pofa)) st = FHV_ERR_OVERFLOW;
    else if (dense && (!h_off || !h_cnt)) st = FHV_ERR_INVALID_ARG;
    else if (!dense && (!h_level_base || (h.n_index_entries > 0 && !h_index))) st = FHV_ERR_INVALID_ARG;
    else if (!dense && h.n_index_entries > index_capacity) st = FHV_ERR_OVERFLOW;
  }
  if (st == FHV_OK) {
    bool ok = read_all(f, h_pofa, h.n_records * sizeof(fhv_record));
    if (h.index_kind == 0) {
      ok = ok && read_all(f, h_off, h.n_index_entries * 4) && read_all(f, h_cnt, h.n_index_entries * 4);
    } else {
      ok = ok && read_all(f, h_level_base, (size_t)(h.depth + 2) * 8) &&
           h_level_base[h.depth + 1] == h.n_index_entries &&
           read_all(f, h_index, h.n_index_entries * sizeof(fhv_octant_entry));
    }
    if (!ok) st = FHV_ERR_INVALID_ARG;  // truncated or inconsistent file
  }
  fclose(f);
  return st;
}
