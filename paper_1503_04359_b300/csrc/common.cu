// Error plumbing, allocator hook and device queries of libdobfs.
#include <mutex>

#include "common.cuh"

namespace dobfs {

namespace {
thread_local char t_last_error[1024] = "";

std::mutex g_alloc_mu;
dobfs_alloc_fn g_alloc = nullptr;
dobfs_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
}  // namespace

int set_error(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
  va_end(ap);
  return status;
}

void clear_error() { t_last_error[0] = '\0'; }

void* dev_alloc(size_t bytes, cudaStream_t stream) {
  if (bytes == 0) bytes = 16;
  if (kBoundsCheck) bytes += kBoundsSlackBytes;
  dobfs_alloc_fn fa;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    fa = g_alloc;
    ctx = g_alloc_ctx;
  }
  if (fa) return fa(bytes, (void*)stream, ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return nullptr;
  }
  return p;
}

void dev_free(void* p, cudaStream_t stream) {
  if (!p) return;
  dobfs_free_fn ff;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    ff = g_free;
    ctx = g_alloc_ctx;
  }
  if (ff) {
    ff(p, (void*)stream, ctx);
    return;
  }
  cudaFree(p);
}

int DevBuf::alloc(size_t n_bytes, cudaStream_t s) {
  reset();
  stream = s;
  ptr = dev_alloc(n_bytes, s);
  if (!ptr) return set_error(DOBFS_ERR_OOM, "device allocation of %zu bytes failed", n_bytes);
  bytes = n_bytes;
  return DOBFS_OK;
}

void DevBuf::reset() {
  if (ptr) dev_free(ptr, stream);
  ptr = nullptr;
  bytes = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    n = c > 0 ? c : 148;
  }
  return n;
}

const char* bounds_site_name(int site) {
  static const char* const names[kBcSiteCount] = {
      "none", "top-down frontier entry", "top-down row offsets", "top-down neighbour ID",
      "top-down next-queue position", "top-down chunk record", "queue/bitmap conversion",
      "bottom-up first neighbour", "bottom-up row offsets", "bottom-up neighbour ID", "bottom-up deferred row",
      "output parent or map entry", "batched row offsets", "batched neighbour ID", "batched chunk record"};
  return site > 0 && site < kBcSiteCount ? names[site] : "unknown site";
}

}  // namespace dobfs

extern "C" {

int dobfs_set_allocator(dobfs_alloc_fn alloc, dobfs_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return dobfs::set_error(DOBFS_ERR_INVALID, "dobfs_set_allocator: give both functions or neither");
  std::lock_guard<std::mutex> lk(dobfs::g_alloc_mu);
  dobfs::g_alloc = alloc;
  dobfs::g_free = free_fn;
  dobfs::g_alloc_ctx = ctx;
  return DOBFS_OK;
}

const char* dobfs_last_error(void) { return dobfs::t_last_error; }

}  // extern "C"
