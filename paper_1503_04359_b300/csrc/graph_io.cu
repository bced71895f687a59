// Graph files: a built graph written to disk and read back without a
// rebuild (no sort, no renumbering; the stored CSR is checked and adopted).
//
// Layout (little-endian): a 64-byte header, then the sections
//   row offsets  (n+1) x int32 or int64, in the internal vertex order
//   columns      n_entries x int32
//   new2orig     n x int32 (renumbered graphs only)
// each padded with zeros to a multiple of 8 bytes. The header carries a
// checksum of the payload: four interleaved FNV-1a streams over its 64-bit
// words (word i feeds stream i mod 4), combined by FNV-1a at the end.
//
// Sections move between the device and the file through two pinned staging
// buffers, so the copy of one chunk overlaps the disk transfer of the other
// and the host never holds more than 2 x kStageBytes of the graph.
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "graph.cuh"

namespace dobfs {
namespace {

constexpr char kMagic[8] = {'D', 'O', 'B', 'F', 'S', 'C', 'S', 'R'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kFileOff64 = 1u, kFileReindexed = 2u;
constexpr size_t kStageBytes = size_t(64) << 20;  // a multiple of 32 bytes
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull, kFnvPrime = 0x100000001b3ull;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t flags;         // kFileOff64 | kFileReindexed
  int64_t n_vertices;
  int64_t n_entries;
  uint64_t checksum;
  uint64_t reserved[3];
};
static_assert(sizeof(FileHeader) == 64, "graph file header is 64 bytes");

struct Checksum {
  uint64_t h[4] = {kFnvBasis, kFnvBasis, kFnvBasis, kFnvBasis};
  uint64_t words = 0;
  // bytes: a multiple of 8
  void add(const void* p, size_t bytes) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    const size_t nw = bytes / 8;
    size_t i = 0;
    // align the stream index to 0 so the unrolled loop feeds streams 0..3
    for (; i < nw && ((words + i) & 3u); ++i) mix(words + i, load(b + 8 * i));
    for (; i + 4 <= nw; i += 4) {
      h[0] = (h[0] ^ load(b + 8 * i)) * kFnvPrime;
      h[1] = (h[1] ^ load(b + 8 * i + 8)) * kFnvPrime;
      h[2] = (h[2] ^ load(b + 8 * i + 16)) * kFnvPrime;
      h[3] = (h[3] ^ load(b + 8 * i + 24)) * kFnvPrime;
    }
    for (; i < nw; ++i) mix(words + i, load(b + 8 * i));
    words += nw;
  }
  uint64_t value() const {
    uint64_t r = kFnvBasis;
    for (uint64_t x : h) r = (r ^ x) * kFnvPrime;
    return (r ^ words) * kFnvPrime;
  }

 private:
  static uint64_t load(const unsigned char* p) {
    uint64_t w;
    memcpy(&w, p, 8);
    return w;
  }
  void mix(uint64_t idx, uint64_t w) { h[idx & 3u] = (h[idx & 3u] ^ w) * kFnvPrime; }
};

size_t pad8(size_t bytes) { return (bytes + 7) & ~size_t(7); }

// Two pinned buffers and their copy events.
struct Staging {
  unsigned char* buf[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~Staging() {
    for (int i = 0; i < 2; ++i) {
      if (ev[i]) {
        cudaEventSynchronize(ev[i]);
        cudaEventDestroy(ev[i]);
      }
      if (buf[i]) cudaFreeHost(buf[i]);
    }
  }
  int init() {
    for (int i = 0; i < 2; ++i) {
      if (cudaMallocHost((void**)&buf[i], kStageBytes) != cudaSuccess) {
        cudaGetLastError();
        buf[i] = nullptr;
        return set_error(DOBFS_ERR_OOM, "pinned staging allocation of %zu bytes failed", kStageBytes);
      }
      DOBFS_CUDA_TRY(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    }
    return DOBFS_OK;
  }
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

// Device section -> file (padded to 8 bytes), chunk k+1's copy overlapping chunk k's write.
int write_section(Staging& st, FILE* f, const void* dev, size_t bytes, Checksum& ck, cudaStream_t s,
                  const char* path) {
  const size_t total = pad8(bytes);
  const size_t chunks = (total + kStageBytes - 1) / kStageBytes;
  auto issue = [&](size_t k) -> int {
    const size_t lo = k * kStageBytes, len = std::min(kStageBytes, total - lo);
    const size_t data = lo < bytes ? std::min(len, bytes - lo) : 0;
    unsigned char* b = st.buf[k & 1];
    if (data) DOBFS_CUDA_TRY(cudaMemcpyAsync(b, (const unsigned char*)dev + lo, data, cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaEventRecord(st.ev[k & 1], s));
    if (len > data) memset(b + data, 0, len - data);  // zero padding (host side, not touched by the copy)
    return DOBFS_OK;
  };
  if (chunks > 0) DOBFS_TRY(issue(0));
  for (size_t k = 0; k < chunks; ++k) {
    DOBFS_CUDA_TRY(cudaEventSynchronize(st.ev[k & 1]));
    if (k + 1 < chunks) DOBFS_TRY(issue(k + 1));
    const size_t len = std::min(kStageBytes, total - k * kStageBytes);
    ck.add(st.buf[k & 1], len);
    if (fwrite(st.buf[k & 1], 1, len, f) != len) return set_error(DOBFS_ERR_IO, "write to %s failed", path);
  }
  return DOBFS_OK;
}

// File -> device section (the file holds pad8(bytes)); chunk k's read overlaps chunk k-1's copy.
int read_section(Staging& st, FILE* f, void* dev, size_t bytes, Checksum& ck, cudaStream_t s, const char* path) {
  const size_t total = pad8(bytes);
  const size_t chunks = (total + kStageBytes - 1) / kStageBytes;
  for (size_t k = 0; k < chunks; ++k) {
    unsigned char* b = st.buf[k & 1];
    DOBFS_CUDA_TRY(cudaEventSynchronize(st.ev[k & 1]));  // chunk k-2's copy out of b is done
    const size_t lo = k * kStageBytes, len = std::min(kStageBytes, total - lo);
    if (fread(b, 1, len, f) != len) return set_error(DOBFS_ERR_IO, "%s: file is truncated", path);
    ck.add(b, len);
    const size_t data = lo < bytes ? std::min(len, bytes - lo) : 0;
    if (data) DOBFS_CUDA_TRY(cudaMemcpyAsync((unsigned char*)dev + lo, b, data, cudaMemcpyHostToDevice, s));
    DOBFS_CUDA_TRY(cudaEventRecord(st.ev[k & 1], s));
  }
  return DOBFS_OK;
}

int save_impl(dobfs_graph* g, const char* path, cudaStream_t s, bool* created) {
  Staging st;
  DOBFS_TRY(st.init());
  File out;
  out.f = fopen(path, "wb");
  if (!out.f) return set_error(DOBFS_ERR_IO, "cannot open %s for writing", path);
  *created = true;
  FileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.flags = (g->off64 ? kFileOff64 : 0u) | (g->reindexed ? kFileReindexed : 0u);
  h.n_vertices = g->n;
  h.n_entries = g->nnz;
  // header first with a zero checksum, rewritten once the payload is known
  if (fwrite(&h, sizeof(h), 1, out.f) != 1) return set_error(DOBFS_ERR_IO, "write to %s failed", path);
  Checksum ck;
  const size_t ob = (g->off64 ? 8 : 4) * (size_t)(g->n + 1);
  DOBFS_TRY(write_section(st, out.f, g->off.ptr, ob, ck, s, path));
  DOBFS_TRY(write_section(st, out.f, g->cols.ptr, sizeof(int32_t) * (size_t)g->nnz, ck, s, path));
  if (g->reindexed) DOBFS_TRY(write_section(st, out.f, g->new2orig.ptr, sizeof(int32_t) * (size_t)g->n, ck, s, path));
  h.checksum = ck.value();
  if (fseek(out.f, 0, SEEK_SET) != 0 || fwrite(&h, sizeof(h), 1, out.f) != 1)
    return set_error(DOBFS_ERR_IO, "write to %s failed", path);
  const int rc = fclose(out.f);
  out.f = nullptr;
  if (rc != 0) return set_error(DOBFS_ERR_IO, "closing %s failed", path);
  return DOBFS_OK;
}

int load_impl(dobfs_graph* g, FILE* f, const FileHeader& h, uint32_t flags, cudaStream_t s, const char* path) {
  g->nnz = h.n_entries;
  g->off64 = (h.flags & kFileOff64) != 0;
  g->reindexed = (h.flags & kFileReindexed) != 0;
  const size_t ob = (g->off64 ? 8 : 4) * (size_t)(g->n + 1);
  DOBFS_TRY(g->off.alloc(ob, s));
  DOBFS_TRY(g->cols.alloc(sizeof(int32_t) * (size_t)(g->nnz + 4), s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(g->cols.as<int32_t>() + g->nnz, 0, sizeof(int32_t) * 4, s));
  if (g->reindexed) {
    DOBFS_TRY(g->new2orig.alloc(sizeof(int32_t) * (size_t)g->n, s));
    DOBFS_TRY(g->orig2new.alloc(sizeof(int32_t) * (size_t)g->n, s));
  }
  {
    Staging st;
    DOBFS_TRY(st.init());
    Checksum ck;
    DOBFS_TRY(read_section(st, f, g->off.ptr, ob, ck, s, path));
    DOBFS_TRY(read_section(st, f, g->cols.ptr, sizeof(int32_t) * (size_t)g->nnz, ck, s, path));
    if (g->reindexed) DOBFS_TRY(read_section(st, f, g->new2orig.ptr, sizeof(int32_t) * (size_t)g->n, ck, s, path));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    unsigned char extra;
    if (fread(&extra, 1, 1, f) != 0) return set_error(DOBFS_ERR_IO, "%s: data after the last section", path);
    if (ck.value() != h.checksum) return set_error(DOBFS_ERR_IO, "%s: checksum mismatch (corrupt file)", path);
  }
  return adopt_csr(g, (flags & DOBFS_GRAPH_VALIDATE) != 0, s);
}

}  // namespace
}  // namespace dobfs

using namespace dobfs;

extern "C" {

int dobfs_graph_save(const dobfs_graph* gc, const char* path, void* stream) {
  clear_error();
  if (!gc || !path) return set_error(DOBFS_ERR_INVALID, "NULL argument");
  dobfs_graph* g = const_cast<dobfs_graph*>(gc);
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  if (g->last_stream) DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
  bool created = false;
  const int rc = save_impl(g, path, s, &created);
  if (rc != DOBFS_OK && created) remove(path);  // no partial file is left behind
  return rc;
}

int dobfs_graph_load(const char* path, uint32_t flags, void* stream, dobfs_graph** out) {
  clear_error();
  if (!out) return set_error(DOBFS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!path) return set_error(DOBFS_ERR_INVALID, "path is NULL");
  if (flags & ~(uint32_t)DOBFS_GRAPH_VALIDATE)
    return set_error(DOBFS_ERR_INVALID, "dobfs_graph_load takes no flag but DOBFS_GRAPH_VALIDATE");
  cudaStream_t s = (cudaStream_t)stream;
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return set_error(DOBFS_ERR_IO, "cannot open %s", path);
  FileHeader h;
  if (fread(&h, sizeof(h), 1, in.f) != 1) return set_error(DOBFS_ERR_IO, "%s: file is truncated", path);
  if (memcmp(h.magic, kMagic, 8) != 0) return set_error(DOBFS_ERR_IO, "%s is not a dobfs graph file", path);
  if (h.version != kVersion)
    return set_error(DOBFS_ERR_IO, "%s: graph file version %u, this library reads %u", path, h.version, kVersion);
  if ((h.flags & ~(kFileOff64 | kFileReindexed)) != 0 || h.n_entries < 0 ||
      (!(h.flags & kFileOff64) && h.n_entries > (int64_t)INT32_MAX))
    return set_error(DOBFS_ERR_IO, "%s: bad graph file header", path);
  dobfs_graph* g = nullptr;
  DOBFS_TRY(new_graph(h.n_vertices, s, &g));
  cudaEvent_t e0, e1;
  int rc = start_timer(s, &e0, &e1);
  if (rc == DOBFS_OK) rc = load_impl(g, in.f, h, flags, s, path);
  return finish_graph(g, rc, e0, e1, out);
}

}  // extern "C"
