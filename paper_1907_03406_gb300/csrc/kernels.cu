// Device kernels of the SGF hot path (sm_103a).
//
// Dense factor work is expressed as batched tile tasks built on the host:
//  * k_gemm  - one CTA per 64x64 output tile, C = beta C + alpha sum op(A) op(B)
//              over a list of contributions (owner-computes: a Schur target
//              tile sums its interiors in a fixed order, no atomics);
//  * k_diag  - in-shared-memory Cholesky of a <= 64x64 diagonal tile and the
//              inverse of its factor (the pivot step of the blocked
//              potrf/trsm/trtri sweep);
//  * k_copy  - tile copies / transposes / identity / zero fills;
//  * k_qrcp  - one CTA per node: Householder QR with column pivoting of the
//              filtered interaction matrix, numeric rank, explicit Q1
//              (Eq. (QR)).
// The apply of A_l^{-1} (Sec. 4.7) is batched matrix-vector work:
//  * k_gemv_n / k_gemv_t - y = beta y + sum alpha op(A) (x - x2), optionally
//              skipping the zero half of a lower-triangular A.
// Plus the stencil assembly, the FP64 SpMV and deterministic dot products of
// the PCG loop (Sec. 7).
#include <cuda_runtime.h>

#include <cstdint>

#include "devmem.h"
#include "kernels.h"
#include "prof.h"

namespace sgf {

namespace {

constexpr int kThreads = 256;
constexpr int kKC = 16;  // K chunk of the tile GEMM

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ void report(DevStatus* st, int code, int level, int node) {
  if (st && atomicCAS(&st->code, 0, code) == 0) {
    st->level = level;
    st->node = node;
  }
}

// ---------------------------------------------------------------------------
// tile GEMM
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gemm(const GemmTask<T>* __restrict__ tasks,
                                                   const GemmContrib<T>* __restrict__ cons) {
  const GemmTask<T> tk = tasks[blockIdx.x];
  __shared__ T As[kKC][kTile + 1];
  __shared__ T Bs[kKC][kTile + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[r][s] = T(0);
  for (int c = tk.c_begin; c < tk.c_begin + tk.c_count; ++c) {
    const GemmContrib<T> cb = cons[c];
    const bool ta = cb.flags & kTransA, tb = cb.flags & kTransB;
    for (int k0 = 0; k0 < cb.K; k0 += kKC) {
#pragma unroll
      for (int q = 0; q < (kKC * kTile) / kThreads; ++q) {
        const int e = threadIdx.x + kThreads * q;
        int i, kk;
        if (!ta) { i = e & 63; kk = e >> 6; } else { kk = e & 15; i = e >> 4; }
        T v = T(0);
        if (i < tk.M && k0 + kk < cb.K)
          v = ta ? cb.A[(size_t)(k0 + kk) + (size_t)i * cb.lda] : cb.A[(size_t)i + (size_t)(k0 + kk) * cb.lda];
        As[kk][i] = v;
        int j;
        if (!tb) { kk = e & 15; j = e >> 4; } else { j = e & 63; kk = e >> 6; }
        v = T(0);
        if (j < tk.N && k0 + kk < cb.K)
          v = tb ? cb.B[(size_t)j + (size_t)(k0 + kk) * cb.ldb] : cb.B[(size_t)(k0 + kk) + (size_t)j * cb.ldb];
        Bs[kk][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
        T a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          a[r] = As[kk][ty + 16 * r];
          b[r] = Bs[kk][tx + 16 * r];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = ty + 16 * r, j = tx + 16 * s;
      if (i < tk.M && j < tk.N) {
        T* p = tk.C + (size_t)i + (size_t)j * tk.ldc;
        T v = tk.alpha * acc[r][s];
        if (tk.beta) v += *p;
        *p = v;
      }
    }
}

// ---------------------------------------------------------------------------
// diagonal tile: Cholesky + inverse of the factor
// ---------------------------------------------------------------------------
constexpr int kPitch = kTile + 1;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_diag(const DiagTask<T>* __restrict__ tasks,
                                                   DevStatus* st, int level) {
  const DiagTask<T> tk = tasks[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  T* V = S + kTile * kPitch;
  __shared__ int bad;
  const int n = tk.n;
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int i = e % n, j = e / n;
    S[i * kPitch + j] = tk.A[(size_t)i + (size_t)j * tk.lda];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T d = S[j * kPitch + j];
      if (!(d > T(0)) || !isfinite(d)) {
        bad = isfinite(d) ? 1 : 2;
        d = T(1);
      }
      S[j * kPitch + j] = sqrt(d);
    }
    __syncthreads();
    const T dj = S[j * kPitch + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += kThreads) S[i * kPitch + j] /= dj;
    __syncthreads();
    const int w = n - j - 1;
    for (int p = threadIdx.x; p < w * w; p += kThreads) {
      const int i = j + 1 + p / w, k = j + 1 + p % w;
      if (k <= i) S[i * kPitch + k] -= S[i * kPitch + j] * S[k * kPitch + j];
    }
    __syncthreads();
  }
  // V = L^{-1}, row by row (row i needs rows < i)
  for (int i = 0; i < n; ++i) {
    for (int c = threadIdx.x; c <= i; c += kThreads) {
      T s = (c == i) ? T(1) : T(0);
      for (int k = c; k < i; ++k) s -= S[i * kPitch + k] * V[k * kPitch + c];
      V[i * kPitch + c] = s / S[i * kPitch + i];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int i = e % n, j = e / n;
    tk.A[(size_t)i + (size_t)j * tk.lda] = (i >= j) ? S[i * kPitch + j] : T(0);
    tk.Li[(size_t)i + (size_t)j * tk.ldli] = (i >= j) ? V[i * kPitch + j] : T(0);
  }
  if (threadIdx.x == 0 && bad) report(st, bad == 1 ? SGF_ERR_NOT_SPD : SGF_ERR_NONFINITE, level, tk.node);
}

// ---------------------------------------------------------------------------
// tile copies
// ---------------------------------------------------------------------------
template <typename S, typename D>
__global__ void __launch_bounds__(kThreads) k_copy(const CopyTask<S, D>* __restrict__ tasks) {
  const CopyTask<S, D> tk = tasks[blockIdx.x];
  const int n = tk.rows * tk.cols;
  for (int e = threadIdx.x; e < n; e += kThreads) {
    const int i = e % tk.rows, j = e / tk.rows;
    D v;
    switch (tk.mode) {
      case kCopy: v = (D)tk.src[(size_t)i + (size_t)j * tk.lds]; break;
      case kCopyT: v = (D)tk.src[(size_t)j + (size_t)i * tk.lds]; break;
      case kIdentity: v = (i == j) ? D(1) : D(0); break;
      case kCopyLower: v = (i >= j) ? (D)tk.src[(size_t)i + (size_t)j * tk.lds] : D(0); break;
      default: v = D(0); break;
    }
    tk.dst[(size_t)i + (size_t)j * tk.ldd] = v;
  }
}

// ---------------------------------------------------------------------------
// column-pivoted Householder QR, rank and Q1 (one CTA per node)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_qrcp(const QrTask<T>* __restrict__ tasks, int* ranks,
                                                   double tau, DevStatus* st, int level) {
  const QrTask<T> tk = tasks[blockIdx.x];
  const int m = tk.m, c = tk.c;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* norms = reinterpret_cast<double*>(smraw);   // c
  double* betas = norms + c;                          // min(m, c)
  T* v = reinterpret_cast<T*>(betas + (m < c ? m : c));  // m
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ double s_bcast;
  __shared__ int s_piv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
  T* A = tk.A;
  for (int j = warp; j < c; j += nw) {
    double s = 0;
    for (int i = lane; i < m; i += 32) {
      const double a = (double)A[(size_t)i + (size_t)j * m];
      s += a * a;
    }
    s = warp_sum(s);
    if (lane == 0) norms[j] = s;
  }
  __syncthreads();
  const int kmax = m < c ? m : c;
  int r = 0;
  double ref = 0;
  for (int k = 0; k < kmax; ++k) {
    // pivot: largest remaining column norm, lowest index on ties
    double best = -1.0;
    int bi = c;
    for (int j = k + threadIdx.x; j < c; j += kThreads) {
      const double x = norms[j];
      if (x > best || (x == best && j < bi)) { best = x; bi = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = rv[0];
      int p = ri[0];
      for (int w = 1; w < nw; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < p)) { b = rv[w]; p = ri[w]; }
      s_bcast = b;
      s_piv = p;
    }
    __syncthreads();
    const double nrm = sqrt(s_bcast > 0 ? s_bcast : 0.0);
    const int p = s_piv;
    if (k == 0) ref = nrm;
    if (!(nrm > tau * ref) || ref == 0.0) break;
    if (p != k) {
      for (int i = threadIdx.x; i < m; i += kThreads) {
        const T a = A[(size_t)i + (size_t)k * m];
        A[(size_t)i + (size_t)k * m] = A[(size_t)i + (size_t)p * m];
        A[(size_t)i + (size_t)p * m] = a;
      }
      if (threadIdx.x == 0) {
        const double t = norms[k];
        norms[k] = norms[p];
        norms[p] = t;
      }
    }
    __syncthreads();
    // Householder vector of A[k:m, k]
    double s = 0;
    for (int i = k + threadIdx.x; i < m; i += kThreads) {
      const T a = A[(size_t)i + (size_t)k * m];
      v[i] = a;
      s += (double)a * (double)a;
    }
    s = warp_sum(s);
    if (lane == 0) rv[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0;
      for (int w = 0; w < nw; ++w) tot += rv[w];
      const double normx = sqrt(tot);
      const double x0 = (double)v[k];
      const double alpha = x0 >= 0 ? -normx : normx;
      double beta = 0;
      if (normx > 0) {
        beta = 1.0 / (alpha * (alpha - x0));
        v[k] = (T)(x0 - alpha);
      }
      betas[k] = beta;
      A[(size_t)k + (size_t)k * m] = v[k];
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += kThreads) A[(size_t)i + (size_t)k * m] = v[i];
    const double beta = betas[k];
    // apply H = I - beta v v^T to the trailing columns and refresh their norms
    for (int j = k + 1 + warp; j < c; j += nw) {
      T* col = A + (size_t)j * m;
      double w = 0;
      for (int i = k + lane; i < m; i += 32) w += (double)v[i] * (double)col[i];
      w = warp_sum(w);
      const double f = beta * w;
      double s2 = 0;
      for (int i = k + lane; i < m; i += 32) {
        const T a = (T)((double)col[i] - f * (double)v[i]);
        col[i] = a;
        if (i > k) s2 += (double)a * (double)a;
      }
      s2 = warp_sum(s2);
      if (lane == 0) norms[j] = s2;
    }
    __syncthreads();
    r = k + 1;
  }
  if (threadIdx.x == 0) ranks[blockIdx.x] = r;
  // Q1 = H_0 ... H_{r-1} [I_r; 0]
  T* Q = tk.Q1;
  for (int e = threadIdx.x; e < m * r; e += kThreads) {
    const int i = e % m, j = e / m;
    Q[(size_t)i + (size_t)j * m] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    for (int i = k + threadIdx.x; i < m; i += kThreads) v[i] = A[(size_t)i + (size_t)k * m];
    __syncthreads();
    const double beta = betas[k];
    for (int j = k + warp; j < r; j += nw) {
      T* col = Q + (size_t)j * m;
      double w = 0;
      for (int i = k + lane; i < m; i += 32) w += (double)v[i] * (double)col[i];
      w = warp_sum(w);
      const double f = beta * w;
      for (int i = k + lane; i < m; i += 32) col[i] = (T)((double)col[i] - f * (double)v[i]);
    }
    __syncthreads();
  }
  (void)st;
  (void)level;
}

// ---------------------------------------------------------------------------
// batched GEMV
// ---------------------------------------------------------------------------
// op(A) = A: chunk of <= 64 output rows; 4 groups of 64 threads split the columns
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gemv_n(const GemvTask<T>* __restrict__ tasks,
                                                     const GemvContrib<T>* __restrict__ cons) {
  const GemvTask<T> tk = tasks[blockIdx.x];
  const int r = threadIdx.x & 63, g = threadIdx.x >> 6;
  T acc = T(0);
  if (r < tk.M) {
    for (int c = tk.c_begin; c < tk.c_begin + tk.c_count; ++c) {
      const GemvContrib<T> cb = cons[c];
      int kend = cb.K;
      if (cb.tri) kend = min(kend, cb.tri - 1 + r + 1);  // lower triangular: j <= row
      const T* a = cb.A + r;
      T part = T(0);
#pragma unroll 4
      for (int j = g; j < kend; j += 4) {
        T xv = cb.x[j];
        if (cb.x2) xv -= cb.x2[j];
        part = fma(a[(size_t)j * cb.lda], xv, part);
      }
      acc = fma(cb.alpha, part, acc);
    }
  }
  __shared__ T red[4][64];
  red[g][r] = acc;
  __syncthreads();
  if (g == 0 && r < tk.M) {
    const T s = (red[0][r] + red[1][r]) + (red[2][r] + red[3][r]);
    tk.y[r] = tk.beta ? tk.y[r] + s : s;
  }
}

// op(A) = A^T: chunk of <= 32 outputs (columns of A); one warp per output
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gemv_t(const GemvTask<T>* __restrict__ tasks,
                                                     const GemvContrib<T>* __restrict__ cons) {
  const GemvTask<T> tk = tasks[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = warp; o < tk.M; o += kThreads / 32) {
    T acc = T(0);
    for (int c = tk.c_begin; c < tk.c_begin + tk.c_count; ++c) {
      const GemvContrib<T> cb = cons[c];
      const int i0 = cb.tri ? (cb.tri - 1 + o) : 0;  // lower triangular: i >= column
      const T* a = cb.A + (size_t)o * cb.lda;
      T part = T(0);
#pragma unroll 4
      for (int i = i0 + lane; i < cb.K; i += 32) {
        T xv = cb.x[i];
        if (cb.x2) xv -= cb.x2[i];
        part = fma(a[i], xv, part);
      }
      part = warp_sum(part);
      acc = fma(cb.alpha, part, acc);
    }
    if (lane == 0) tk.y[o] = tk.beta ? tk.y[o] + acc : acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_veccopy(const VecCopyTask* __restrict__ tasks,
                                                      const T* __restrict__ src, T* __restrict__ dst) {
  const VecCopyTask tk = tasks[blockIdx.x];
  for (int i = threadIdx.x; i < tk.len; i += kThreads) dst[tk.dst + i] = src[tk.src + i];
}

// ---------------------------------------------------------------------------
// stencil assembly, SpMV, vector kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

template <typename T>
__global__ void k_assemble(const double* __restrict__ coef, int nx, int ny, int nz, unsigned dm,
                           double w, const int64_t* __restrict__ map, int64_t dgsz, T* dg, T* up,
                           double* sd, double* sx, double* sy, double* sz) {
  const int64_t npts = (int64_t)nx * ny * nz;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((int64_t)nx * ny));
  const double k = coef[p];
  double t[6];
  t[0] = x > 0 ? harmonic(coef[p - 1], k) : ((dm & 1u) ? w * k : 0.0);
  t[1] = x < nx - 1 ? harmonic(k, coef[p + 1]) : ((dm & 2u) ? w * k : 0.0);
  t[2] = y > 0 ? harmonic(coef[p - nx], k) : ((dm & 4u) ? w * k : 0.0);
  t[3] = y < ny - 1 ? harmonic(k, coef[p + nx]) : ((dm & 8u) ? w * k : 0.0);
  const int64_t pl = (int64_t)nx * ny;
  if (nz > 1) {
    t[4] = z > 0 ? harmonic(coef[p - pl], k) : ((dm & 16u) ? w * k : 0.0);
    t[5] = z < nz - 1 ? harmonic(k, coef[p + pl]) : ((dm & 32u) ? w * k : 0.0);
  } else {
    t[4] = t[5] = 0.0;
  }
  double d = 0.0;
  for (int q = 0; q < 6; ++q) d = d + t[q];
  sd[p] = d;
  sx[p] = x < nx - 1 ? t[1] : 0.0;
  sy[p] = y < ny - 1 ? t[3] : 0.0;
  sz[p] = z < nz - 1 ? t[5] : 0.0;
  if (map) {
    for (int q = 0; q < 7; ++q) {
      const int64_t o = map[p * 7 + q];
      if (o < 0) continue;
      const T v = (T)(q == 6 ? d : -t[q]);
      if (o < dgsz) dg[o] = v; else up[o - dgsz] = v;
    }
  }
}

__global__ void k_spmv(const double* __restrict__ sd, const double* __restrict__ sx,
                       const double* __restrict__ sy, const double* __restrict__ sz, int nx, int ny,
                       int nz, const double* __restrict__ x, double* __restrict__ yv) {
  const int64_t npts = (int64_t)nx * ny * nz;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const int xi = (int)(p % nx), yi = (int)((p / nx) % ny), zi = (int)(p / ((int64_t)nx * ny));
  const int64_t pl = (int64_t)nx * ny;
  double acc = sd[p] * x[p];
  if (xi > 0) acc -= sx[p - 1] * x[p - 1];
  if (xi < nx - 1) acc -= sx[p] * x[p + 1];
  if (yi > 0) acc -= sy[p - nx] * x[p - nx];
  if (yi < ny - 1) acc -= sy[p] * x[p + nx];
  if (zi > 0) acc -= sz[p - pl] * x[p - pl];
  if (zi < nz - 1) acc -= sz[p] * x[p + pl];
  yv[p] = acc;
}

__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              double* __restrict__ partials) {
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    s = fma(a[i], b[i], s);
  s = warp_sum(s);
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t += w[k];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_dot_final(const double* __restrict__ partials, int np, double* result) {
  double s = 0;
  for (int i = threadIdx.x; i < np; i += kThreads) s += partials[i];
  s = warp_sum(s);
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t += w[k];
    result[0] = t;
  }
}

template <typename T>
__global__ void k_gather(const double* __restrict__ src, const int64_t* __restrict__ perm,
                         T* __restrict__ dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)src[perm[i]];
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ src, const int64_t* __restrict__ perm,
                          double* __restrict__ dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[perm[i]] = (double)src[i];
}

__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}

__global__ void k_xpay(const double* __restrict__ z, double b, double* __restrict__ p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = fma(b, p[i], z[i]);
}

inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
template <typename T>
void launch_gemm(const GemmTask<T>* tasks, const GemmContrib<T>* cons, int n, cudaStream_t s) {
  if (dry_run()) {
    const size_t es = sizeof(T);
    for (int i = 0; i < n; ++i) {
      const GemmTask<T>& t = tasks[i];
      if (t.M > kTile || t.N > kTile || t.M < 1 || t.N < 1) check_range(nullptr, 1, "gemm tile shape");
      check_block(t.C, t.M, t.N, t.ldc, es, "gemm C");
      for (int c = t.c_begin; c < t.c_begin + t.c_count; ++c) {
        const GemmContrib<T>& q = cons[c];
        if (q.flags & kTransA) check_block(q.A, q.K, t.M, q.lda, es, "gemm A^T");
        else check_block(q.A, t.M, q.K, q.lda, es, "gemm A");
        if (q.flags & kTransB) check_block(q.B, t.N, q.K, q.ldb, es, "gemm B^T");
        else check_block(q.B, q.K, t.N, q.ldb, es, "gemm B");
      }
    }
    return;
  }
  if (n <= 0) return;
  ProfScope ps(P_GEMM, s);
  k_gemm<T><<<n, kThreads, 0, s>>>(tasks, cons);
}

template <typename T>
void launch_diag(const DiagTask<T>* tasks, int n, DevStatus* st, int level, cudaStream_t s) {
  if (dry_run()) {
    for (int i = 0; i < n; ++i) {
      if (tasks[i].n > kTile || tasks[i].n < 1) check_range(nullptr, 1, "diag tile shape");
      check_block(tasks[i].A, tasks[i].n, tasks[i].n, tasks[i].lda, sizeof(T), "diag A");
      check_block(tasks[i].Li, tasks[i].n, tasks[i].n, tasks[i].ldli, sizeof(T), "diag Li");
    }
    return;
  }
  if (n <= 0) return;
  const size_t sm = 2 * sizeof(T) * kTile * kPitch;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  ProfScope ps(P_DIAG, s);
  k_diag<T><<<n, kThreads, sm, s>>>(tasks, st, level);
}

template <typename S, typename D>
void launch_copy(const CopyTask<S, D>* tasks, int n, cudaStream_t s) {
  if (dry_run()) {
    for (int i = 0; i < n; ++i) {
      const CopyTask<S, D>& t = tasks[i];
      if (t.rows > kTile || t.cols > kTile) check_range(nullptr, 1, "copy tile shape");
      check_block(t.dst, t.rows, t.cols, t.ldd, sizeof(D), "copy dst");
      if (t.mode == kCopy || t.mode == kCopyLower) check_block(t.src, t.rows, t.cols, t.lds, sizeof(S), "copy src");
      if (t.mode == kCopyT) check_block(t.src, t.cols, t.rows, t.lds, sizeof(S), "copyT src");
    }
    return;
  }
  if (n <= 0) return;
  ProfScope ps(P_COPY, s);
  k_copy<S, D><<<n, kThreads, 0, s>>>(tasks);
}

template <typename T>
void launch_qrcp(const QrTask<T>* tasks, int n, int* ranks, double tau, int max_m, int max_c,
                 DevStatus* st, int level, cudaStream_t s) {
  if (dry_run()) {
    for (int i = 0; i < n; ++i) {
      const QrTask<T>& t = tasks[i];
      if (t.m > max_m || t.c > max_c) check_range(nullptr, 1, "qr size above launch bound");
      check_block(t.A, t.m, t.c, t.m, sizeof(T), "qr A");
      check_block(t.Q1, t.m, t.m < t.c ? t.m : t.c, t.m, sizeof(T), "qr Q1");
    }
    check_range(ranks, sizeof(int) * n, "qr ranks");
    return;
  }
  if (n <= 0) return;
  const int kmin = max_m < max_c ? max_m : max_c;
  const size_t sm = sizeof(double) * (size_t)(max_c + kmin) + sizeof(T) * (size_t)max_m + 16;
  cudaFuncSetAttribute(k_qrcp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ProfScope ps(P_QR, s);
  k_qrcp<T><<<n, kThreads, sm, s>>>(tasks, ranks, tau, st, level);
}

template <typename T>
static void check_gemv(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, bool trans) {
  for (int i = 0; i < n; ++i) {
    const GemvTask<T>& t = tasks[i];
    if (t.M > (trans ? 32 : 64) || t.M < 1) check_range(nullptr, 1, "gemv chunk shape");
    check_range(t.y, sizeof(T) * t.M, "gemv y");
    for (int c = t.c_begin; c < t.c_begin + t.c_count; ++c) {
      const GemvContrib<T>& q = cons[c];
      if (trans) check_block(q.A, q.K, t.M, q.lda, sizeof(T), "gemvT A");
      else check_block(q.A, t.M, q.K, q.lda, sizeof(T), "gemv A");
      check_range(q.x, sizeof(T) * q.K, "gemv x");
      if (q.x2) check_range(q.x2, sizeof(T) * q.K, "gemv x2");
    }
  }
}

template <typename T>
void launch_gemv_n(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, cudaStream_t s) {
  if (dry_run()) return check_gemv(tasks, cons, n, false);
  if (n <= 0) return;
  ProfScope ps(P_GEMV_N, s);
  k_gemv_n<T><<<n, kThreads, 0, s>>>(tasks, cons);
}

template <typename T>
void launch_gemv_t(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, cudaStream_t s) {
  if (dry_run()) return check_gemv(tasks, cons, n, true);
  if (n <= 0) return;
  ProfScope ps(P_GEMV_T, s);
  k_gemv_t<T><<<n, kThreads, 0, s>>>(tasks, cons);
}

template <typename T>
void launch_veccopy(const VecCopyTask* tasks, int n, const T* src, T* dst, cudaStream_t s) {
  if (dry_run()) {
    for (int i = 0; i < n; ++i) {
      check_range(src + tasks[i].src, sizeof(T) * tasks[i].len, "veccopy src");
      check_range(dst + tasks[i].dst, sizeof(T) * tasks[i].len, "veccopy dst");
    }
    return;
  }
  if (n <= 0) return;
  ProfScope ps(P_VECCOPY, s);
  k_veccopy<T><<<n, kThreads, 0, s>>>(tasks, src, dst);
}

template <typename T>
void launch_assemble_scalar(const double* coef, int nx, int ny, int nz, unsigned dm, double w,
                            const int64_t* map, int64_t dgsz, T* dg, T* up, double* sd, double* sx,
                            double* sy, double* sz, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz;
  if (dry_run()) {
    check_range(map, 8 * 7 * n, "assemble map");
    for (double* a : {sd, sx, sy, sz}) check_range(a, 8 * n, "assemble stencil arrays");
    return;
  }
  ProfScope ps(P_ASSEMBLE, s);
  k_assemble<T><<<blocks_for(n), kThreads, 0, s>>>(coef, nx, ny, nz, dm, w, map, dgsz, dg, up, sd, sx, sy, sz);
}

void launch_spmv_stencil(const double* sd, const double* sx, const double* sy, const double* sz,
                         int nx, int ny, int nz, const double* x, double* y, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz;
  if (dry_run()) return;
  prof_work(13.0 * n, 48.0 * n);
  ProfScope ps(P_SPMV, s);
  k_spmv<<<blocks_for(n), kThreads, 0, s>>>(sd, sx, sy, sz, nx, ny, nz, x, y);
}

void launch_dot(const double* a, const double* b, int64_t n, double* partials, double* result,
                cudaStream_t s) {
  if (dry_run()) return;
  prof_work(2.0 * n, 16.0 * n);
  ProfScope ps(P_DOT, s);
  k_dot_partial<<<kDotBlocks, kThreads, 0, s>>>(a, b, n, partials);
  k_dot_final<<<1, kThreads, 0, s>>>(partials, kDotBlocks, result);
}

template <typename T>
void launch_gather(const double* src, const int64_t* perm, T* dst, int64_t n, cudaStream_t s) {
  if (dry_run()) {
    check_range(perm, 8 * n, "gather perm");
    check_range(dst, sizeof(T) * n, "gather dst");
    return;
  }
  if (n <= 0) return;
  prof_work(0, (16.0 + sizeof(T)) * n);
  ProfScope ps(P_VEC, s);
  k_gather<T><<<blocks_for(n), kThreads, 0, s>>>(src, perm, dst, n);
}
template <typename T>
void launch_scatter(const T* src, const int64_t* perm, double* dst, int64_t n, cudaStream_t s) {
  if (dry_run()) {
    check_range(perm, 8 * n, "scatter perm");
    check_range(src, sizeof(T) * n, "scatter src");
    return;
  }
  if (n <= 0) return;
  prof_work(0, (16.0 + sizeof(T)) * n);
  ProfScope ps(P_VEC, s);
  k_scatter<T><<<blocks_for(n), kThreads, 0, s>>>(src, perm, dst, n);
}

void launch_axpy(double a, const double* x, double* y, int64_t n, cudaStream_t s) {
  if (dry_run()) return;
  if (n <= 0) return;
  prof_work(2.0 * n, 24.0 * n);
  ProfScope ps(P_VEC, s);
  k_axpy<<<blocks_for(n), kThreads, 0, s>>>(a, x, y, n);
}
void launch_xpay(const double* z, double b, double* p, int64_t n, cudaStream_t s) {
  if (dry_run()) return;
  if (n <= 0) return;
  prof_work(2.0 * n, 24.0 * n);
  ProfScope ps(P_VEC, s);
  k_xpay<<<blocks_for(n), kThreads, 0, s>>>(z, b, p, n);
}

#define SGF_INST(T)                                                                              \
  template void launch_gemm<T>(const GemmTask<T>*, const GemmContrib<T>*, int, cudaStream_t);   \
  template void launch_diag<T>(const DiagTask<T>*, int, DevStatus*, int, cudaStream_t);         \
  template void launch_copy<T, T>(const CopyTask<T, T>*, int, cudaStream_t);                    \
  template void launch_qrcp<T>(const QrTask<T>*, int, int*, double, int, int, DevStatus*, int,  \
                               cudaStream_t);                                                    \
  template void launch_gemv_n<T>(const GemvTask<T>*, const GemvContrib<T>*, int, cudaStream_t); \
  template void launch_gemv_t<T>(const GemvTask<T>*, const GemvContrib<T>*, int, cudaStream_t); \
  template void launch_veccopy<T>(const VecCopyTask*, int, const T*, T*, cudaStream_t);         \
  template void launch_assemble_scalar<T>(const double*, int, int, int, unsigned, double,       \
                                          const int64_t*, int64_t, T*, T*, double*, double*,    \
                                          double*, double*, cudaStream_t);                       \
  template void launch_gather<T>(const double*, const int64_t*, T*, int64_t, cudaStream_t);     \
  template void launch_scatter<T>(const T*, const int64_t*, double*, int64_t, cudaStream_t);

SGF_INST(double)
SGF_INST(float)
template void launch_copy<double, float>(const CopyTask<double, float>*, int, cudaStream_t);

}  // namespace sgf
