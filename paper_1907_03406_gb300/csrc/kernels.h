// Launch wrappers of the SGF device kernels (implemented in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "sgf_internal.h"

namespace sgf {

// First device-side failure (pivot <= 0 / non-finite / size limits).
struct DevStatus {
  int code;   // 0 or an SGF_ERR_* value
  int level;
  int node;
  int nonfinite;   // an apply or multiply wrote a NaN / infinity (sgf_sync reads and clears it)
};

template <typename T>
void launch_gemm(const GemmTask<T>* tasks, const GemmContrib<T>* contribs, int ntasks,
                 cudaStream_t s);
// FP32 GEMM tasks of up to kTileTC x kTileTC on the 5th-generation tensor
// cores, FP32 accumulators in tensor memory.  Every operand is split into
// nparts TF32 parts and the products p_i q_j with i + j < nparts are summed:
// nparts = 2 is the 3xTF32 scheme (products accurate to ~2^-21), nparts = 3
// carries them to FP32 accuracy with six products.
void launch_gemm_tc(const GemmTask<float>* tasks, const GemmContrib<float>* contribs, int ntasks, int nparts,
                    cudaStream_t s);
// tensor-core GEMMs for the FP32 factor unless SGF_TENSOR_CORES=0
bool gemm_tc_enabled();
// Programmatic dependent launch of the apply kernels (k_gemv_n, k_gemv_t,
// k_vgather, k_veccopy) on this thread, set while an apply program is
// captured into a graph: each such launch may start while the previous
// kernel drains; its blocks stage their task lists and prefetch their matrix
// columns into L2 (data no earlier kernel of the program writes), then wait
// for the previous grid's completion before reading vectors or writing
// results.  Off when SGF_DEPENDENT_LAUNCH=0.
void set_dependent_launch(bool on);
bool dependent_launch_enabled();
template <typename T>
void launch_diag(const DiagTask<T>* tasks, int ntasks, DevStatus* st, int level, cudaStream_t s);
// whole blocked Cholesky + inverse of small fronts, one CTA each
// (up to 512 rows in single precision; in double precision the tiled sweep
// over many CTAs is faster beyond one tile)
template <typename T>
constexpr int front_small() {
  return sizeof(T) == 8 ? 64 : 512;
}
// fronts up to kFrontTiny always take the one-CTA kernel (when front_small
// allows); larger ones only in batches of at least kFrontBatchMin (about one
// per SM)
constexpr int kFrontTiny = 128;
constexpr int kFrontBatchMin = 152;
template <typename T>
void launch_front(const FrontTask<T>* tasks, int ntasks, DevStatus* st, int level, cudaStream_t s);
template <typename S, typename D>
void launch_copy(const CopyTask<S, D>* tasks, int ntasks, cudaStream_t s);
// pivoted QR: tasks whose m * c_eff fits in cap_elems work in shared memory
template <typename T>
void launch_qrcp(const QrTask<T>* tasks, int ntasks, int* ranks, double tau, int max_m, int max_c,
                 long long cap_elems, cudaStream_t s);
size_t qr_smem_bytes(int m, int c, size_t elem_size, long long cap_elems);
// nr right-hand sides interleaved (nr in 1, 2, 4, 8)
// max_m: largest chunk of the launch's CTA tasks (op N bands up to 256 rows
// use a narrower kernel).  wtasks / nw: chunks too small to fill a CTA
// (unsplit, at most kGemvWarpElems elements; op N bands of at most
// kGemvWarpRowsMax rows), run in the same launch one per warp, eight to a
// block after the CTA tasks' blocks (best ordered largest first).
constexpr int kGemvWarpRowsMax = 128;
constexpr int kGemvWarpElems = 4 * 1024;
template <typename T>
void launch_gemv_n(const GemvTask<T>* tasks, const GemvContrib<T>* contribs, int ntasks, int nr, int max_m,
                   cudaStream_t s, const GemvTask<T>* wtasks = nullptr, int nw = 0);
// cols: the chunk width the tasks were built with (kGemvCols, or
// kGemvColsMax in single precision)
template <typename T>
void launch_gemv_t(const GemvTask<T>* tasks, const GemvContrib<T>* contribs, int ntasks, int nr, int cols,
                   cudaStream_t s, const GemvTask<T>* wtasks = nullptr, int nw = 0);
// dst[p * nr + q] = src[idx[p] * nr + q], p < n
template <typename T>
void launch_vgather(const T* src, const int* idx, T* dst, int n, int nr, cudaStream_t s);
template <typename T>
void launch_veccopy(const VecCopyTask* tasks, int ntasks, const T* src, T* dst, cudaStream_t s);

// Scalar stencil assembly (Sec. 7.1): FP64 SpMV diagonals and, through the
// element map (stride 7 per point: x-, x+, y-, y+, z-, z+, diag; offsets into
// the concatenation [Dg | Up], -1 = skip), the level-1 dense blocks.
template <typename T>
void launch_assemble_scalar(const double* coef, int nx, int ny, int nz, unsigned dirichlet,
                            double bweight, const int64_t* map, int64_t dg_size, T* dg, T* up,
                            double* sd, double* sx, double* sy, double* sz, cudaStream_t s);

// Q1 elasticity: level-1 3x3 blocks through the 27-per-point map (ld[p] =
// size of p's level-1 node) and the FP64 27-block BSR copy for the SpMV.
template <typename T>
void launch_assemble_q1(const double* E, const double* kref, int nx, int ny, int nz, const int64_t* map,
                        const int* ld, int64_t dg_size, T* dg, T* up, double* bsr, cudaStream_t s);
void launch_spmv_bsr27(const double* bsr, int nx, int ny, int nz, const double* x, double* y,
                       cudaStream_t s);

// y = A x for the assembled 5/7-point operator, FP64.
void launch_spmv_stencil(const double* sd, const double* sx, const double* sy, const double* sz,
                         int nx, int ny, int nz, const double* x, double* y, cudaStream_t s);

// Deterministic dot product: partials (>= kDotBlocks doubles) then result[0].
constexpr int kDotBlocks = 304;
void launch_dot(const double* a, const double* b, int64_t n, double* partials, double* result,
                cudaStream_t s);

// natural-order RHS-major (nrhs x n) <-> interleaved level-1 vectors (nr >= nrhs)
template <typename T>
void launch_gather(const double* src, const int64_t* perm, T* dst, int64_t n, int nrhs, int nr,
                   cudaStream_t s);
// nonfinite (may be null): raised to 1 when a value written is NaN or infinite
template <typename T>
void launch_scatter(const T* src, const int64_t* perm, double* dst, int64_t n, int nrhs, int nr,
                    cudaStream_t s, int* nonfinite = nullptr);

// block PCG helpers on RHS-major FP64 vectors (nrhs <= 8)
struct Coef8 {
  double v[8];
};
void launch_dot_n(const double* a, const double* b, int64_t n, int nrhs, double* partials,
                  double* result, cudaStream_t s);  // partials: nrhs * kDotBlocks
// mode 0: y_q += a_q x_q ; mode 1: y_q = x_q + a_q y_q
void launch_axpy_n(const Coef8& a, const double* x, double* y, int64_t n, int nrhs, int mode,
                   cudaStream_t s);

// PCG step length on the device (Sec. 7): alpha_q = rz_q / pq_q where
// act.v[q] != 0, else 0, written to coef[q] and -alpha_q to coef[8 + q];
// flag[q] = 1 (else 0) where alpha_q is not finite, its coefficients then 0
void launch_pcg_alpha(const double* pq, const double* rz, const Coef8& act, int nrhs, double* coef,
                      double* flag, cudaStream_t s);
// x_q += alpha_q p_q; ro_q = r_q (when ro is given); r_q -= alpha_q q_q, with
// alpha_q = coef[q] and -alpha_q = coef[8 + q] read on the device
void launch_pcg_xr(const double* coef, const double* p, const double* q, double* x, double* r, double* ro,
                   int64_t n, int nrhs, cudaStream_t s);

// y = a*x + y (FP64)
void launch_axpy(double a, const double* x, double* y, int64_t n, cudaStream_t s);
// p = z + b*p (FP64)
void launch_xpay(const double* z, double b, double* p, int64_t n, cudaStream_t s);

}  // namespace sgf
