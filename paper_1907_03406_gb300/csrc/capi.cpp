// C ABI of the SGF library (declared in include/sgf.h).  Every entry point
// converts internal exceptions into status codes; nothing throws across it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <string>

#include "devmem.h"
#include "factor.h"
#include "prof.h"
#include "sgf.h"
#include "sgf_internal.h"

#include "handles.h"

namespace {
thread_local std::string g_last_error;

template <class F>
int guarded(F&& fn) {
  try {
    return fn();
  } catch (const sgf::SgfError& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return SGF_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return SGF_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

const char* sgf_status_string(int s) {
  switch (s) {
    case SGF_OK: return "ok";
    case SGF_ERR_INVALID_ARG: return "invalid argument";
    case SGF_ERR_NOT_SPD: return "matrix not SPD (non-positive pivot)";
    case SGF_ERR_NONFINITE: return "non-finite value";
    case SGF_ERR_OOM: return "out of memory";
    case SGF_ERR_NO_CONVERGENCE: return "PCG did not converge";
    case SGF_ERR_TIMEOUT: return "device wait timed out";
    case SGF_ERR_CUDA: return "CUDA error";
    case SGF_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char* sgf_last_error(void) { return g_last_error.c_str(); }

int sgf_analyze(const sgf_grid* grid, int stencil, const sgf_opts* opts, sgf_plan** out) {
  if (!out) return SGF_ERR_INVALID_ARG;
  *out = nullptr;
  return guarded([&] {
    auto p = std::make_unique<sgf_plan>();
    std::string err;
    int rc = sgf::analyze(grid, stencil, opts, p->p, err);
    if (rc != SGF_OK) {
      g_last_error = err;
      return rc;
    }
    *out = p.release();
    return (int)SGF_OK;
  });
}

void sgf_plan_destroy(sgf_plan* plan) { delete plan; }

int sgf_plan_info(const sgf_plan* plan, int* nlevels, int64_t* n) {
  if (!plan) return SGF_ERR_INVALID_ARG;
  if (nlevels) *nlevels = (int)plan->p.lev.size();
  if (n) *n = plan->p.n;
  return SGF_OK;
}

int sgf_plan_export_level(const sgf_plan* plan, int level, int* nnodes, int* npairs, int* npost,
                          int* codes, int* flags, int* child_ptr, int* child_idx, int* pairs,
                          int* post) {
  if (!plan || level < 0 || level >= (int)plan->p.lev.size()) return SGF_ERR_INVALID_ARG;
  const sgf::LevelSym& L = plan->p.lev[level];
  if (nnodes) *nnodes = L.nnodes;
  if (npairs) *npairs = (int)L.pairs.size() / 2;
  if (npost) *npost = (int)L.post.size() / 2;
  if (codes) std::copy(L.code.begin(), L.code.end(), codes);
  if (flags)
    for (int i = 0; i < L.nnodes; ++i) flags[i] = (L.interior[i] ? 1 : 0) | (L.cell_dim[i] << 4) | (L.eligible[i] ? 2 : 0);
  if (child_ptr) {
    if (L.child_ptr.empty()) std::fill(child_ptr, child_ptr + L.nnodes + 1, 0);
    else std::copy(L.child_ptr.begin(), L.child_ptr.end(), child_ptr);
  }
  if (child_idx) std::copy(L.child_idx.begin(), L.child_idx.end(), child_idx);
  if (pairs) std::copy(L.pairs.begin(), L.pairs.end(), pairs);
  if (post) std::copy(L.post.begin(), L.post.end(), post);
  return SGF_OK;
}

int sgf_plan_footprint(const sgf_plan* plan, size_t* b64, size_t* bmx) {
  if (!plan) return SGF_ERR_INVALID_ARG;
  // structural bound: every node kept at its uncompressed size
  const sgf::Plan& P = plan->p;
  double words = 0;
  for (size_t li = 0; li < P.lev.size(); ++li) {
    sgf::LevelLayout lay;
    sgf::build_layout(P.lev[li], P.mcap[li], lay);
    // diagonal blocks (A, L, L^{-1}), panels (A, W, W^T), level vectors, Phi
    words += 3.0 * lay.dg_size + 3.0 * lay.up_size + 3.0 * lay.vec_size + P.pi * lay.vec_size;
  }
  const double extra = 64.0 * P.npts;  // stencil arrays, maps, vectors
  if (b64) *b64 = (size_t)(8.0 * words + extra);
  if (bmx) *bmx = (size_t)(4.0 * words + extra);
  return SGF_OK;
}

int sgf_plan_get_tuning(const sgf_plan* plan, sgf_tuning* out) {
  if (!plan || !out) return SGF_ERR_INVALID_ARG;
  *out = plan->p.tune;
  return SGF_OK;
}

int sgf_plan_set_tuning(sgf_plan* plan, const sgf_tuning* t) {
  if (!plan || !t || !sgf::tuning_valid(*t)) return SGF_ERR_INVALID_ARG;
  plan->p.tune = *t;
  return SGF_OK;
}

// Grid search over launch shapes.  The factor shapes (front_small x
// tensor_cores, single precision only) change only the factorization and the
// GEMV budgets only the apply programs, so they are searched one after the
// other: each factor shape by the faster of two timed factorizations, then,
// with the best one, each GEMV budget (x op T chunk width in single
// precision) by napply timed applications of A_l^{-1} (its factorization
// untimed).
int sgf_autotune(sgf_plan* plan, const double* coeffs_dev, void* stream, int napply, sgf_tuning* best,
                 double* best_ms) {
  if (!plan || !coeffs_dev || napply < 0) return SGF_ERR_INVALID_ARG;
  if (sgf::dry_run()) return SGF_ERR_UNSUPPORTED;
  const sgf_tuning saved = plan->p.tune;
  const int rc = guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    const bool mixed = plan->p.opts.precision == SGF_PREC_MIXED;
    const int64_t n = plan->p.n;
    double* x = (double*)sgf::dev_malloc(sizeof(double) * n);
    double* y = (double*)sgf::dev_malloc(sizeof(double) * n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SGF_CK(cudaEventCreate(&e0));
    SGF_CK(cudaEventCreate(&e1));
    struct Cleanup {
      double *x, *y;
      cudaEvent_t a, b;
      ~Cleanup() {
        sgf::dev_free(x);
        sgf::dev_free(y);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
      }
    } cleanup{x, y, e0, e1};
    sgf::dev_memset(x, 0, sizeof(double) * n, s);   // any fixed vector times the same
    auto elapsed = [&] {
      SGF_CK(cudaEventSynchronize(e1));
      float ms = 0;
      SGF_CK(cudaEventElapsedTime(&ms, e0, e1));
      return (double)ms;
    };
    {
      auto f = sgf::make_factor(plan->p, coeffs_dev, s);   // warm-up: caches, pools, module loading
      if (napply > 0) f->apply(x, y, s);
      sgf::dev_sync(s);
    }
    sgf_tuning cur = saved;
    double t_factor = 0;
    {
      struct Shape { int fs, tc, tcmin; };
      std::vector<Shape> shapes;
      if (mixed) {
        for (int fs : {512, 256})
          for (int tcmin : {32, 64, 128}) shapes.push_back({fs, saved.tensor_cores ? saved.tensor_cores : 1, tcmin});
      } else {
        shapes.push_back({saved.front_small, saved.tensor_cores, saved.tc_min_dim});
      }
      double bt = 1e300;
      for (const auto& sh : shapes) {
        plan->p.tune = saved;
        plan->p.tune.front_small = sh.fs;
        plan->p.tune.tensor_cores = sh.tc;
        plan->p.tune.tc_min_dim = sh.tcmin;
        double t = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
          SGF_CK(cudaEventRecord(e0, s));
          auto f = sgf::make_factor(plan->p, coeffs_dev, s);
          SGF_CK(cudaEventRecord(e1, s));
          t = std::min(t, elapsed());
        }
        if (t < bt) {
          bt = t;
          cur = plan->p.tune;
        }
      }
      t_factor = bt;
    }
    double t_apply = 0;
    if (napply > 0) {
      const int budgets[5][2] = {{4096, 32768}, {8192, 65536}, {16384, 131072}, {32768, 131072}, {32768, 262144}};
      std::vector<sgf_tuning> cand;
      for (int cols : mixed ? std::vector<int>{32, 64} : std::vector<int>{saved.gemv_cols})
        for (const auto& bgt : budgets) {
          sgf_tuning c = cur;
          c.gemv_min_elems = bgt[0];
          c.gemv_max_elems = bgt[1];
          c.gemv_cols = cols;
          cand.push_back(c);
        }
      double bt = 1e300;
      sgf_tuning bc = cur;
      for (const sgf_tuning& c : cand) {
        plan->p.tune = c;
        auto f = sgf::make_factor(plan->p, coeffs_dev, s);
        f->apply(x, y, s);   // first use: the program's graph is captured
        SGF_CK(cudaEventRecord(e0, s));
        for (int k = 0; k < napply; ++k) f->apply(x, y, s);
        SGF_CK(cudaEventRecord(e1, s));
        const double t = elapsed();
        if (t < bt) {
          bt = t;
          bc = plan->p.tune;
        }
      }
      cur = bc;
      t_apply = bt;
    }
    plan->p.tune = cur;
    if (best) *best = cur;
    if (best_ms) *best_ms = t_factor + t_apply;
    return (int)SGF_OK;
  });
  if (rc != SGF_OK) plan->p.tune = saved;
  return rc;
}

int sgf_factor(const sgf_plan* plan, const double* coeffs_dev, void* stream, sgf_factor_t** out) {
  if (!out) return SGF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!plan || !coeffs_dev) return SGF_ERR_INVALID_ARG;
  return guarded([&] {
    auto f = std::make_unique<sgf_factor_s>();
    f->plan = plan;
    f->f = sgf::make_factor(plan->p, coeffs_dev, (cudaStream_t)stream);
    *out = f.release();
    return (int)SGF_OK;
  });
}

void sgf_factor_destroy(sgf_factor_t* f) { delete f; }

int sgf_factor_level_stats(const sgf_factor_t* f, int level, int* ncomp, int64_t* before,
                           int64_t* after, int64_t* bytes) {
  if (!f || level < 0 || level >= (int)f->f->stats.size()) return SGF_ERR_INVALID_ARG;
  const auto& s = f->f->stats[level];
  if (ncomp) *ncomp = s.ncomp;
  if (before) *before = s.size_before;
  if (after) *after = s.size_after;
  if (bytes) *bytes = s.bytes;
  return SGF_OK;
}

int sgf_factor_ranks(const sgf_factor_t* f, int level, int* m, int* r) {
  if (!f || level < 0 || level >= (int)f->f->stats.size()) return SGF_ERR_INVALID_ARG;
  const auto& s = f->f->stats[level];
  if (m) std::copy(s.m.begin(), s.m.end(), m);
  if (r) std::copy(s.r.begin(), s.r.end(), r);
  return SGF_OK;
}

int sgf_factor_precision(const sgf_factor_t* f) {
  if (!f) return -1;
  return f->f->mixed() ? SGF_PREC_MIXED : SGF_PREC_FP64;
}

int sgf_factor_status(const sgf_factor_t* f, int* bl, int* bn) {
  if (!f) return SGF_ERR_INVALID_ARG;
  if (bl) *bl = f->f->bad_level;
  if (bn) *bn = f->f->bad_node;
  return f->f->status;
}

static int apply_common(const sgf_factor_t* f, const double* x, double* y, int nrhs, void* stream,
                        int which) {
  if (!f || !x || !y || nrhs < 1 || x == y) return SGF_ERR_INVALID_ARG;
  return guarded([&] {
    const int64_t n = f->f->n;
    if (which == 0) f->f->apply_n(x, y, nrhs, (cudaStream_t)stream);
    else if (which == 1) f->f->multiply_n(x, y, nrhs, (cudaStream_t)stream);
    else
      for (int j = 0; j < nrhs; ++j) f->f->spmv(x + j * n, y + j * n, (cudaStream_t)stream);
    if (!sgf::dry_run()) SGF_CK(cudaGetLastError());
    return (int)SGF_OK;
  });
}

int sgf_apply(const sgf_factor_t* f, const double* x, double* y, int nrhs, void* stream) {
  return apply_common(f, x, y, nrhs, stream, 0);
}
int sgf_apply_forward(const sgf_factor_t* f, const double* x, double* y, int nrhs, void* stream) {
  return apply_common(f, x, y, nrhs, stream, 1);
}
int sgf_spmv(const sgf_factor_t* f, const double* x, double* y, int nrhs, void* stream) {
  return apply_common(f, x, y, nrhs, stream, 2);
}

int sgf_pcg_solve(const sgf_factor_t* f, const double* b, double* x, int nrhs, double rtol, int maxit,
                  void* stream, sgf_solve_info* info) {
  if (!f || !b || !x || nrhs < 1 || rtol <= 0 || maxit < 1 || b == x) return SGF_ERR_INVALID_ARG;
  return guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SGF_CK(cudaEventCreate(&e0));
    SGF_CK(cudaEventCreate(&e1));
    SGF_CK(cudaEventRecord(e0, s));
    int worst = SGF_OK, itmax = 0;
    double resmax = 0;
    const int64_t n = f->f->n;
    for (int j = 0; j < nrhs; j += 8) {
      const int k = std::min(8, nrhs - j);
      int it[8];
      double rr[8];
      int rc = sgf::pcg_solve_block(*f->f, b + j * n, x + j * n, k, rtol, maxit, s, it, rr);
      if (rc != SGF_OK) worst = rc;
      for (int q = 0; q < k; ++q) {
        itmax = std::max(itmax, it[q]);
        resmax = std::max(resmax, rr[q]);
      }
    }
    SGF_CK(cudaEventRecord(e1, s));
    SGF_CK(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
      info->iterations = itmax;
      info->rel_residual = resmax;
      info->seconds = ms * 1e-3;
    }
    return worst;
  });
}

int sgf_solve_host(const sgf_plan* plan, const double* coeffs_host, const double* b_host,
                   double* x_host, int nrhs, double rtol, int maxit, void* stream,
                   sgf_solve_info* info) {
  if (!plan || !coeffs_host || !b_host || !x_host || nrhs < 1) return SGF_ERR_INVALID_ARG;
  return guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    const sgf::Plan& P = plan->p;
    const size_t nb = sizeof(double) * P.n * nrhs;
    double *dc = nullptr, *db = nullptr, *dx = nullptr;
    SGF_CK(cudaMallocAsync((void**)&dc, sizeof(double) * P.npts, s));
    SGF_CK(cudaMallocAsync((void**)&db, nb, s));
    SGF_CK(cudaMallocAsync((void**)&dx, nb, s));
    SGF_CK(cudaMemcpyAsync(dc, coeffs_host, sizeof(double) * P.npts, cudaMemcpyHostToDevice, s));
    SGF_CK(cudaMemcpyAsync(db, b_host, nb, cudaMemcpyHostToDevice, s));
    sgf_factor_t* f = nullptr;
    int rc = sgf_factor(plan, dc, stream, &f);
    if (rc == SGF_OK) {
      rc = sgf_pcg_solve(f, db, dx, nrhs, rtol, maxit, stream, info);
      SGF_CK(cudaMemcpyAsync(x_host, dx, nb, cudaMemcpyDeviceToHost, s));
      SGF_CK(cudaStreamSynchronize(s));
      sgf_factor_destroy(f);
    }
    cudaFreeAsync(dc, s);
    cudaFreeAsync(db, s);
    cudaFreeAsync(dx, s);
    SGF_CK(cudaStreamSynchronize(s));
    return rc;
  });
}

}  // extern "C"

extern "C" {
// Dry-run validation report (SGF_DRY_RUN=1): number of out-of-range task
// accesses seen since the last reset, and a text log of the first ones.
int64_t sgf_dry_run_violations(int reset) {
  int64_t v = sgf::dry_run_violations();
  if (reset) sgf::dry_run_reset();
  return v;
}
const char* sgf_dry_run_report(void) {
  thread_local std::string s;
  s = sgf::dry_run_report();
  return s.c_str();
}
}

extern "C" {
void sgf_profile_reset(int timing) { sgf::prof_reset(timing); }
int sgf_profile_read(int kind, int64_t* launches, double* ms, double* flops, double* bytes) {
  long long l = 0;
  int rc = sgf::prof_read(kind, &l, ms, flops, bytes);
  if (rc) return SGF_ERR_INVALID_ARG;
  if (launches) *launches = l;
  return SGF_OK;
}
const char* sgf_profile_kind_name(int kind) { return sgf::prof_name(kind); }

int sgf_sync(const sgf_factor_t* f) {
  if (!f) return SGF_ERR_INVALID_ARG;
  return guarded([&] {
    if (sgf::dry_run()) return (int)SGF_OK;
    int cur = -1;
    SGF_CK(cudaGetDevice(&cur));
    if (cur != f->f->device) throw sgf::SgfError(SGF_ERR_INVALID_ARG, "factor lives on another device");
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) throw sgf::SgfError(SGF_ERR_CUDA, std::string("device: ") + cudaGetErrorString(e));
    return f->f->device_status();
  });
}

int sgf_memory_stats(int64_t* alloc_events, int64_t* pool_used_bytes) {
  if (alloc_events) *alloc_events = sgf::alloc_events();
  if (pool_used_bytes) {
    *pool_used_bytes = 0;
    if (!sgf::dry_run()) {
      int dev = 0;
      cudaMemPool_t pool;
      uint64_t used = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
          cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
        return SGF_ERR_CUDA;
      *pool_used_bytes = (int64_t)used;
    }
  }
  return SGF_OK;
}

int sgf_release_cached_memory(void) {
  if (!sgf::dry_run() && cudaDeviceSynchronize() != cudaSuccess) return SGF_ERR_CUDA;
  sgf::dev_release_cached();
  return SGF_OK;
}
}
