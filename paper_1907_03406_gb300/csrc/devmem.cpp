// Device memory helpers and the dry-run validator (see devmem.h).
#include "devmem.h"

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>

#include "factor.h"

namespace sgf {

namespace {
struct Registry {
  std::mutex mu;
  std::map<uintptr_t, size_t> live;  // base -> bytes
  uintptr_t next = (uintptr_t)1 << 40;
  int64_t violations = 0;
  int64_t checks = 0;
  std::ostringstream log;
};
Registry& reg() {
  static Registry r;
  return r;
}
}  // namespace

static bool g_skip_checks = false;

bool dry_run() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("SGF_DRY_RUN");
    v = (e && (e[0] == '1' || e[0] == '2')) ? 1 : 0;
    // SGF_DRY_RUN=2: no range checks (times the host-side task building alone)
    g_skip_checks = e && e[0] == '2';
  }
  return v == 1;
}

static void* fake_alloc(size_t bytes) {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  uintptr_t p = r.next;
  r.live[p] = bytes;
  r.next += ((bytes + 255) & ~(size_t)255) + 4096;  // guard gap between ranges
  return (void*)p;
}

static void fake_free(void* p) {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  if (p) r.live.erase((uintptr_t)p);
}

static std::atomic<int64_t> g_alloc_events{0};
void note_alloc_event() { g_alloc_events.fetch_add(1, std::memory_order_relaxed); }
int64_t alloc_events() { return g_alloc_events.load(std::memory_order_relaxed); }

static void check_aligned(void* p) {
  if (reinterpret_cast<uintptr_t>(p) & 15) throw SgfError(SGF_ERR_CUDA, "device allocation not 16-byte aligned");
}

void* dev_malloc(size_t bytes) {
  if (dry_run()) return fake_alloc(bytes);
  void* p = nullptr;
  note_alloc_event();
  SGF_CK(cudaMalloc(&p, bytes + kAllocTail));
  check_aligned(p);
  return p;
}
void dev_free(void* p) {
  if (dry_run()) return fake_free(p);
  if (p) cudaFree(p);
}
void* dev_malloc_async(size_t bytes, cudaStream_t s) {
  if (dry_run()) return fake_alloc(bytes);
  {
    // keep freed stream-ordered memory cached in this process (the default
    // release threshold of 0 hands it back at every synchronisation, and each
    // factorization would reserve its work buffers again)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev >= 0 && dev < 64 && !done[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      done[dev] = true;
    }
  }
  void* p = nullptr;
  note_alloc_event();
  cudaError_t e = cudaMallocAsync(&p, bytes + kAllocTail, s);
  if (e == cudaErrorMemoryAllocation) {
    // the pool may be holding freed blocks of earlier factorizations: hand
    // them back to the device and try once more
    cudaGetLastError();
    cudaStreamSynchronize(s);
    dev_release_cached();
    e = cudaMallocAsync(&p, bytes + kAllocTail, s);
  }
  SGF_CK(e);
  check_aligned(p);
  return p;
}
void dev_release_cached() {
  if (dry_run()) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
}
void dev_free_async(void* p, cudaStream_t s) {
  if (dry_run()) return fake_free(p);
  if (p) cudaFreeAsync(p, s);
}
void dev_memset(void* p, int v, size_t bytes, cudaStream_t s) {
  if (dry_run()) return check_range(p, bytes, "memset");
  SGF_CK(cudaMemsetAsync(p, v, bytes, s));
}
void dev_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (dry_run()) return check_range(dst, bytes, "h2d");
  SGF_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
}
void dev_d2h(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (dry_run()) {
    check_range(src, bytes, "d2h");
    std::memset(dst, 0, bytes);
    return;
  }
  SGF_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
  SGF_CK(cudaStreamSynchronize(s));
}
void dev_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (dry_run()) {
    check_range(dst, bytes, "d2d dst");
    check_range(src, bytes, "d2d src");
    return;
  }
  SGF_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
}
void dev_sync(cudaStream_t s) {
  if (dry_run()) return;
  SGF_CK(cudaStreamSynchronize(s));
}

void check_range(const void* p, size_t bytes, const char* what) {
  if (!dry_run() || bytes == 0 || g_skip_checks) return;
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  r.checks++;
  const uintptr_t a = (uintptr_t)p;
  auto it = r.live.upper_bound(a);
  bool ok = false;
  if (it != r.live.begin()) {
    --it;
    ok = a >= it->first && a + bytes <= it->first + it->second;
  }
  if (!ok) {
    if (r.violations < 20) r.log << what << ": [" << std::hex << a << ", +" << std::dec << bytes << ") outside any allocation\n";
    r.violations++;
  }
}

void check_block_superset(const void* p, int64_t M, int64_t N, int64_t ld, size_t es, const char* what) {
  if (!dry_run() || M <= 0 || N <= 0 || g_skip_checks) return;
  const uintptr_t a = (uintptr_t)p;
  const uintptr_t a0 = a & ~uintptr_t(15);
  const uintptr_t e1 = (a + (size_t)((M - 1) + (N - 1) * ld + 1) * es + 15) & ~uintptr_t(15);
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  r.checks++;
  auto it = r.live.upper_bound(a0);
  bool ok = false;
  if (it != r.live.begin()) {
    --it;
    ok = a0 >= it->first && e1 <= it->first + it->second + kAllocTail;
  }
  if (!ok) {
    if (r.violations < 20)
      r.log << what << ": aligned superset [" << std::hex << a0 << ", " << e1 << std::dec << ") outside any allocation and its tail\n";
    r.violations++;
  }
}

void check_block(const void* p, int64_t M, int64_t N, int64_t ld, size_t es, const char* what) {
  if (!dry_run() || M <= 0 || N <= 0) return;
  if (M > ld) {
    Registry& r = reg();
    std::lock_guard<std::mutex> g(r.mu);
    if (r.violations < 20) r.log << what << ": rows " << M << " exceed leading dimension " << ld << "\n";
    r.violations++;
    return;
  }
  check_range(p, (size_t)((M - 1) + (N - 1) * ld + 1) * es, what);
}

Plan::~Plan() {
  if (cache.map) dev_free(cache.map);
  if (cache.perm) dev_free(cache.perm);
  if (cache.ld) dev_free(cache.ld);
  if (cache.kref) dev_free(cache.kref);
  for (int t = 0; t < 2; ++t) {
    if (cache.phi1[t]) dev_free(cache.phi1[t]);
    for (void* p : cache.reexp[t])
      if (p) dev_free(p);
  }
}

int64_t dry_run_violations() { return reg().violations; }
void dry_run_reset() {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  r.violations = 0;
  r.checks = 0;
  r.log.str("");
}
std::string dry_run_report() {
  return "checked " + std::to_string(reg().checks) + " ranges\n" + reg().log.str();
}

}  // namespace sgf
