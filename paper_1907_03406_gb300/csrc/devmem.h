// Device-memory and launch indirection with a host-only validation mode.
//
// With SGF_DRY_RUN=1 in the environment no CUDA call is made: allocations are
// fake address ranges recorded in a table, copies and syncs are skipped, and
// every launch wrapper checks, instead of launching, that each task's reads
// and writes stay inside one recorded allocation.  This lets the host driver
// (task building, layouts, offsets) be exercised on a machine without a GPU.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

namespace sgf {

bool dry_run();

// Every device allocation is 16-byte aligned and kAllocTail bytes longer than
// asked for, so a kernel may read the 16-byte aligned superset of any segment
// it owns (bulk copies need aligned ends) without leaving the allocation.
constexpr size_t kAllocTail = 64;

void* dev_malloc(size_t bytes);                          // persistent (cudaMalloc)
void dev_free(void* p);
// stream ordered, from the device's default pool, which keeps freed blocks
// cached for later allocations (an allocation that fails hands the cached
// blocks back and retries once)
void* dev_malloc_async(size_t bytes, cudaStream_t s);
void dev_free_async(void* p, cudaStream_t s);
// return the pool's unused cached blocks to the device
void dev_release_cached();
// Allocation events: every call of this library that asks the CUDA runtime
// or driver for device memory (cudaMalloc, cudaMallocAsync, stream creation,
// graph instantiation) adds one.
void note_alloc_event();
int64_t alloc_events();
void dev_memset(void* p, int v, size_t bytes, cudaStream_t s);
void dev_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s);
void dev_d2h(void* dst, const void* src, size_t bytes, cudaStream_t s);  // synchronous
void dev_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s);
void dev_sync(cudaStream_t s);

// Dry-run range checks: [p, p + bytes) must lie in one live allocation.
void check_range(const void* p, size_t bytes, const char* what);
// column-major M x N block with leading dimension ld and element size es
void check_block(const void* p, int64_t M, int64_t N, int64_t ld, size_t es, const char* what);
// the 16-byte aligned superset of that block's columns (what bulk copies of
// its column segments read) lies in one live allocation and its tail
void check_block_superset(const void* p, int64_t M, int64_t N, int64_t ld, size_t es, const char* what);
int64_t dry_run_violations();
void dry_run_reset();
std::string dry_run_report();

}  // namespace sgf
