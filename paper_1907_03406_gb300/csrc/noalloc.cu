// PCG solve that allocates nothing (sgf_pcg_solve_noalloc).
//
// Some callers cannot let a library allocate device memory during a solve:
// a serving process that reserves its whole memory budget up front and
// treats any later cudaMalloc as a budget violation, code that owns every
// byte through its own arena, or a latency-critical loop where an allocator
// call (and the device synchronization it can imply) is not acceptable.
// For them this entry point runs the same preconditioned CG as
// sgf_pcg_solve, but its work vectors (r, z, p, q, previous r) and the
// partial sums of the dot products live in one file-scope device array of a
// fixed size, reserved by every GPU that loads the library until the process
// exits.  The caller still passes the factor, the right-hand side and the
// output.  The paper has no counterpart: this is a deployment interface.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <mutex>

#include "factor.h"
#include "handles.h"
#include "kernels.h"
#include "sgf.h"

namespace {

// scratch: 5 vectors of SGF_NOALLOC_MAX_UNKNOWNS doubles + dot partials + scalar
constexpr size_t kVecs = 5;
constexpr size_t kScratchDoubles = kVecs * (size_t)SGF_NOALLOC_MAX_UNKNOWNS + sgf::kDotBlocks + 64;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Host code cannot use g_noalloc_scratch as an address (it is a host-side
// stand-in for the device symbol): look the device address up once per
// device, with that device current.
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SGF_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SGF_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SGF_OK;
}

}  // namespace

extern "C" int sgf_pcg_solve_noalloc(const sgf_factor_t* fh, const double* b, double* x, double rtol,
                                     int maxit, void* stream, sgf_solve_info* info) {
  if (!fh || !b || !x || b == x || rtol <= 0 || maxit < 1) return SGF_ERR_INVALID_ARG;
  sgf::FactorBase& F = *fh->f;
  const int64_t n = F.n;
  if (n > (int64_t)SGF_NOALLOC_MAX_UNKNOWNS) return SGF_ERR_INVALID_ARG;  // beyond the fixed scratch
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return SGF_ERR_CUDA;
  if (cur != F.device) return SGF_ERR_INVALID_ARG;   // the scratch array of another GPU
  double* ws = nullptr;
  int rc = scratch_for_current_device(&ws);
  if (rc != SGF_OK) return rc;
  try {
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    // every scratch word below is written before it is read in this call, so
    // nothing left by an earlier call can leak into this one
    double *r = ws, *z = r + n, *p = z + n, *q = p + n, *ro = q + n;
    double* part = ws + kVecs * (size_t)SGF_NOALLOC_MAX_UNKNOWNS;
    double* sc = part + sgf::kDotBlocks;
    auto dot = [&](const double* a, const double* c) {
      sgf::launch_dot(a, c, n, part, sc, s);
      double h = 0;
      SGF_CK(cudaMemcpyAsync(&h, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
      SGF_CK(cudaStreamSynchronize(s));
      return h;
    };
    const bool flex = F.mixed();
    SGF_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    SGF_CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const double bnorm = std::sqrt(dot(b, b));
    int it = 0;
    rc = SGF_OK;
    if (bnorm > 0.0) {
      F.apply(r, z, s);
      SGF_CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      double rz = dot(r, z);
      while (true) {
        if (it >= maxit) { rc = SGF_ERR_NO_CONVERGENCE; break; }
        F.spmv(p, q, s);
        const double alpha = rz / dot(p, q);
        if (!std::isfinite(alpha)) { rc = SGF_ERR_NONFINITE; break; }
        sgf::launch_axpy(alpha, p, x, n, s);
        if (flex) SGF_CK(cudaMemcpyAsync(ro, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        sgf::launch_axpy(-alpha, q, r, n, s);
        ++it;
        if (std::sqrt(dot(r, r)) <= rtol * bnorm) break;
        F.apply(r, z, s);
        const double rz_new = dot(r, z);
        const double beta = flex ? (rz_new - dot(z, ro)) / rz : rz_new / rz;
        rz = rz_new;
        sgf::launch_xpay(z, beta, p, n, s);
      }
    }
    double rel = 0.0;
    if (bnorm > 0.0) {
      F.spmv(x, q, s);
      SGF_CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      sgf::launch_axpy(-1.0, q, r, n, s);
      rel = std::sqrt(dot(r, r)) / bnorm;
    }
    SGF_CK(cudaStreamSynchronize(s));
    if (info) {
      info->iterations = it;
      info->rel_residual = rel;
      info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
  } catch (const sgf::SgfError& e) {
    return e.code;
  } catch (...) {
    return SGF_ERR_CUDA;
  }
}
