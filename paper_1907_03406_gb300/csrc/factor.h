// Numeric factorization object behind the sgf_factor handle.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "kernels.h"
#include "sgf_internal.h"

namespace sgf {

struct SgfError : std::runtime_error {
  int code;
  SgfError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define SGF_CK(x)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess)                                                                 \
      throw ::sgf::SgfError(e_ == cudaErrorMemoryAllocation ? SGF_ERR_OOM : SGF_ERR_CUDA,  \
                            std::string(#x) + ": " + cudaGetErrorString(e_));              \
  } while (0)

// Host staging of task arrays: pushed descriptors are uploaded with one copy,
// then the recorded launches run against the device copy.
struct Batch {
  std::vector<char> host;
  std::vector<char> keep_host;  // dry-run copy of a persistent program
  std::vector<std::function<void(const char*)>> launches;
  char* dev = nullptr;   // persistent programs only
  size_t cap = 0;
  // pinned staging ring: a buffer is refilled only after the copy that last
  // read it has completed, so a deep ring keeps the host from waiting on the GPU
  static constexpr int kRing = 8;
  char* pin[kRing] = {};
  size_t pincap[kRing] = {};
  cudaEvent_t ev[kRing] = {};
  int cur = 0;
  Batch();
  Batch(const Batch&) = delete;
  Batch& operator=(const Batch&) = delete;
  ~Batch();
  template <class X>
  size_t push(const std::vector<X>& v) {
    const size_t off = (host.size() + 63) & ~size_t(63);
    const size_t bytes = v.size() * sizeof(X);
    if (host.capacity() < off + bytes) grow(std::max(2 * host.capacity(), off + bytes));
    host.insert(host.end(), off - host.size(), char(0));   // alignment padding only
    const char* p = reinterpret_cast<const char*>(v.data());
    host.insert(host.end(), p, p + bytes);
    return off;
  }
  // move the staged bytes into a buffer of at least `want` bytes of capacity
  // (a pooled one when one fits: its pages are already resident)
  void grow(size_t want);
  // upload and run everything recorded so far, then reset
  void run(cudaStream_t s);
  // keep the uploaded copy (for programs replayed many times)
  void upload_persistent(cudaStream_t s);
  void release(cudaStream_t s);
};

struct LevelStats {
  int ncomp = 0;
  int64_t size_before = 0, size_after = 0, bytes = 0;
  std::vector<int> m, r;
};

class FactorBase {
 public:
  virtual ~FactorBase() = default;
  virtual void apply(const double* x, double* y, cudaStream_t s) = 0;      // A_l^{-1}
  virtual void multiply(const double* x, double* y, cudaStream_t s) = 0;   // A_l
  // nrhs vectors at once (RHS-major, stride n): every factor entry read once per 8
  virtual void apply_n(const double* x, double* y, int nrhs, cudaStream_t s) = 0;
  virtual void multiply_n(const double* x, double* y, int nrhs, cudaStream_t s) = 0;
  virtual void spmv(const double* x, double* y, cudaStream_t s) = 0;       // A
  virtual bool mixed() const = 0;
  // Asynchronous status of the work issued for this factor so far: the
  // device pivot status, then a non-finite value written by an apply or a
  // multiply since the last call (that flag is cleared).  The caller has
  // synchronized the device.
  virtual int device_status() = 0;
  const Plan* plan = nullptr;
  int device = -1;              // the CUDA device the factor lives on
  std::vector<LevelStats> stats;
  int bad_level = -1, bad_node = -1, status = 0;
  bool fp64_fallback = false;   // mixed request factored in FP64 (see make_factor)
  int64_t n = 0;
};

std::unique_ptr<FactorBase> make_factor(const Plan& plan, const double* coeffs_dev, cudaStream_t s);

// nrhs (<= 8) independent PCG recurrences advanced together (one apply per
// iteration for all of them); iters/relres per RHS
int pcg_solve_block(FactorBase& F, const double* b, double* x, int nrhs, double rtol, int maxit,
                    cudaStream_t s, int* iters, double* relres);

}  // namespace sgf
