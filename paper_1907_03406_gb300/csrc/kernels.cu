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

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <vector>

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


// FP32 variant: each thread owns a 4x4 block of consecutive rows / columns so
// every operand fetch from shared memory is one 16-byte load; the next K chunk
// is prefetched into registers while the current one is multiplied.
constexpr int kPitchF = kTile + 4;  // keeps 16-byte alignment, breaks bank aliasing

__device__ __forceinline__ void gemm_load_chunk(const GemmContrib<float>& cb, int M, int N, int k0,
                                                float ra[4], float rb[4]) {
  const bool ta = cb.flags & kTransA, tb = cb.flags & kTransB;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + kThreads * q;
    int i, kk;
    if (!ta) { i = e & 63; kk = e >> 6; } else { kk = e & 15; i = e >> 4; }
    float v = 0.f;
    if (i < M && k0 + kk < cb.K)
      v = ta ? cb.A[(size_t)(k0 + kk) + (size_t)i * cb.lda] : cb.A[(size_t)i + (size_t)(k0 + kk) * cb.lda];
    ra[q] = v;
    int j;
    if (!tb) { kk = e & 15; j = e >> 4; } else { j = e & 63; kk = e >> 6; }
    v = 0.f;
    if (j < N && k0 + kk < cb.K)
      v = tb ? cb.B[(size_t)j + (size_t)(k0 + kk) * cb.ldb] : cb.B[(size_t)(k0 + kk) + (size_t)j * cb.ldb];
    rb[q] = v;
  }
}

__device__ __forceinline__ void gemm_store_chunk(const GemmContrib<float>& cb, float (*As)[kPitchF],
                                                 float (*Bs)[kPitchF], const float ra[4], const float rb[4]) {
  const bool ta = cb.flags & kTransA, tb = cb.flags & kTransB;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + kThreads * q;
    int i, kk;
    if (!ta) { i = e & 63; kk = e >> 6; } else { kk = e & 15; i = e >> 4; }
    As[kk][i] = ra[q];
    int j;
    if (!tb) { kk = e & 15; j = e >> 4; } else { j = e & 63; kk = e >> 6; }
    Bs[kk][j] = rb[q];
  }
}

template <>
__global__ void __launch_bounds__(kThreads) k_gemm<float>(const GemmTask<float>* __restrict__ tasks,
                                                          const GemmContrib<float>* __restrict__ cons) {
  const GemmTask<float> tk = tasks[blockIdx.x];
  __shared__ __align__(16) float As[2][kKC][kPitchF];
  __shared__ __align__(16) float Bs[2][kKC][kPitchF];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
  for (int c = tk.c_begin; c < tk.c_begin + tk.c_count; ++c) {
    const GemmContrib<float> cb = cons[c];
    float ra[4], rb[4];
    gemm_load_chunk(cb, tk.M, tk.N, 0, ra, rb);
    __syncthreads();  // previous contribution done with the buffers
    gemm_store_chunk(cb, As[0], Bs[0], ra, rb);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < cb.K; k0 += kKC) {
      const bool more = k0 + kKC < cb.K;
      if (more) gemm_load_chunk(cb, tk.M, tk.N, k0 + kKC, ra, rb);
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
      }
      if (more) {
        gemm_store_chunk(cb, As[buf ^ 1], Bs[buf ^ 1], ra, rb);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ty * 4 + r;
    if (i >= tk.M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = tx * 4 + q;
      if (j < tk.N) {
        float* p = tk.C + (size_t)i + (size_t)j * tk.ldc;
        float v = tk.alpha * acc[r][q];
        if (tk.beta) v += *p;
        *p = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tensor-core tile GEMM (FP32 operands as split TF32 products, FP32 accumulation)
// ---------------------------------------------------------------------------
// One CTA per kTileTC x kTileTC output tile (M, N <= 128); the contributions'
// K ranges are walked in raw chunks of kRawK values and, within them, in
// chunks of kTcKC.  Seventeen warps, specialized, with no CTA barrier in the
// main loop:
//  * warps 0-7 (producers: warps 0-3 for op(A), 4-7 for op(B)^T, thread q of
//    a group owning row q of its operand) bring each raw chunk of both
//    operands one chunk ahead into one of two raw shared-memory stages with
//    cp.async.bulk (a copy per row of a K-contiguous operand, per k-row of a
//    row-contiguous one; the node blocks have odd leading dimensions, so each
//    copy takes the 16-byte aligned superset of its segment), then split
//    their row of each raw chunk
//    into NPART TF32 parts (each the remainder so far rounded to nearest
//    TF32, so v = p0 + p1 [+ p2] up to the last part's rounding), store them
//    K-major in the no-swizzle canonical layout (core matrices of 8 rows x 16
//    bytes, 128 bytes apart along K, kTcKC / 4 * 128 bytes apart along rows)
//    into operand stage c mod kStages and arrive on its "full" mbarrier; a
//    producer-only barrier after each raw chunk frees its raw stage;
//  * one thread of warp 8 waits for "full", issues per 8-wide K step the
//    split products (NPART = 2: p0q0 + p0q1 + p1q0, the 3xTF32 scheme;
//    NPART = 3: also p0q2 + p1q1 + p2q0) as tcgen05.mma kind::tf32 (M = N =
//    128) and commits to the stage's "empty" mbarrier so the producers refill
//    it.  The tensor cores accumulate with truncation, whose error grows
//    linearly with the number of additions, so a partial sum only covers
//    kTcFlush chunks: groups of chunks alternate between two 128-column
//    tensor-memory accumulators ("acc full" commits, "acc empty" arrivals);
//  * warps 9-16 (accumulators; warp w reads tensor-memory lanes 32 (w mod 4)
//    .. + 31, columns 64 ((w - 9) / 4) .. + 63) read every finished partial
//    with tcgen05.ld and add it to FP32 registers (round to nearest), then
//    write C = beta C + alpha sum.
// Rows of an operand beyond the task's M / N and K positions beyond a
// contribution's K are stored as zeros.  Every mbarrier wait is bounded; a
// wait that gives up stops the pipeline, waits (bounded) for the products in
// flight, poisons the tile with NaN (reported downstream as a non-finite
// factor) instead of hanging, and the tensor memory is released on every path.
constexpr int kTcKC = 16;
constexpr int kTcFlush = 2;                  // chunks per tensor-memory partial sum
constexpr int kTcProdWarps = 8;              // warps 0-7
constexpr int kTcProd = kTcProdWarps * 32;
constexpr int kTcMmaWarp = 8;
constexpr int kTcAccWarp0 = 9;               // warps 9-16
constexpr int kTcAccWarps = 8;
constexpr int kTcAccCols = kTileTC * 4 / kTcAccWarps;   // columns per accumulator warp
constexpr int kTcThreads = (kTcAccWarp0 + kTcAccWarps) * 32;
constexpr int kTcPartA = kTileTC * kTcKC;    // floats of one operand part per stage
constexpr int kTcPitchR = 136;               // raw k-row of a row-contiguous operand: 128 values + alignment slack
constexpr int kTcWaitIters = 1 << 22;

// Shared memory: kStages split-operand stages, then two raw stages (each
// op(A) then op(B)^T, kRawOp floats apiece) of kRawK values of K.  A raw
// row (K-contiguous operand, pitch kPitchK) holds the aligned superset of
// kRawK values; the pitch is 12 mod 32 words, so eight consecutive rows'
// 16-byte reads meet eight different bank groups.
template <int NPART>
struct TcCfg {
  static constexpr int kStages = 2;
  static constexpr int kStage = 2 * NPART * kTcPartA;   // A and B parts
  static constexpr int kRawK = NPART == 2 ? 64 : 32;
  static constexpr int kPitchK = NPART == 2 ? 76 : 44;
  static constexpr int kRawOp = kTileTC * kPitchK > kRawK * kTcPitchR ? kTileTC * kPitchK : kRawK * kTcPitchR;
  static constexpr size_t kSmem = sizeof(float) * ((size_t)kStages * kStage + 4 * (size_t)kRawOp);
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  constexpr uint32_t lbo = 128, sbo = (kTcKC / 4) * 128;
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(lbo >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version; base offset 0, no swizzle
  return d;
}
// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major, M = N = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTileTC >> 3) << 17) |
                              ((uint32_t)(kTileTC >> 4) << 24);

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < kTcWaitIters; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// v rounded to TF32 (nearest, ties away from zero); v - result is exact
__device__ __forceinline__ float tf32_hi(float v) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(v));
  return __uint_as_float(h);
}

// The producers' position in the task's chunk sequence: contribution c (its
// fields held in registers: every cp.async clobbers memory, so fields read
// through a pointer would be reloaded before each copy), K offset k0.
struct TcCursor {
  int c, k0;
  GemmContrib<float> cb;
};

__device__ __forceinline__ void tc_cursor_load(TcCursor& u, const GemmContrib<float>* __restrict__ cons, int cend) {
  while (u.c < cend && cons[u.c].K <= 0) ++u.c;
  if (u.c < cend) u.cb = cons[u.c];
}

__device__ __forceinline__ void tc_cursor_next(TcCursor& u, const GemmContrib<float>* __restrict__ cons, int cend,
                                               int step) {
  u.k0 += step;
  if (u.k0 >= u.cb.K) {
    u.k0 = 0;
    ++u.c;
    tc_cursor_load(u, cons, cend);
  }
}

// Producer thread q (0..127) of one operand issues its bulk copy of a raw
// chunk of that operand (R rows, element (r, k) at X[r + k ldx] when
// rows_contig, else at X[k + r ldx]; K offset k0, kc <= kRawK values) into
// the operand's half of a raw stage, and arrives on the stage's mbarrier
// with the bytes it expects (every producer thread arrives, with 0 bytes
// when it has nothing to copy).  K contiguous: thread q copies row q's kc
// values; rows contiguous: thread q (< kc) copies k-row q's R values and
// records where that k-row starts in its superset in the shift table.  A
// bulk copy needs 16-byte aligned ends, so each takes the aligned superset
// of its segment: at most 12 bytes either side, inside the allocation and
// its tail (every device allocation keeps one).
template <int NPART>
__device__ __forceinline__ void tc_issue(const float* X, int ldx, bool rows_contig, int k0, int kc, int R, int q,
                                         uint32_t sraw, uint32_t bar, unsigned char* shtab) {
  using Cfg = TcCfg<NPART>;
  uintptr_t a = 0;
  uint32_t dst = 0, nb = 0;
  if (rows_contig) {
    if (q < kc && R > 0) {
      a = reinterpret_cast<uintptr_t>(X + (size_t)(k0 + q) * ldx);
      nb = (uint32_t)(((a + sizeof(float) * R + 15) & ~uintptr_t(15)) - (a & ~uintptr_t(15)));
      dst = sraw + 4u * q * kTcPitchR;
      shtab[q] = (unsigned char)((a & 15) >> 2);   // published by the arrival below
    }
  } else {
    if (q < R && kc > 0) {
      a = reinterpret_cast<uintptr_t>(X + (size_t)q * ldx + k0);
      nb = (uint32_t)(((a + sizeof(float) * kc + 15) & ~uintptr_t(15)) - (a & ~uintptr_t(15)));
      dst = sraw + 4u * q * Cfg::kPitchK;
    }
  }
  if (nb) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(nb) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     dst),
                 "l"(a & ~uintptr_t(15)), "r"(nb), "r"(bar)
                 : "memory");
  } else {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
  }
}

// Producer thread q takes row q of its operand, values kk0 .. kk0 + 15 of
// the raw chunk (zero for rows >= R and k >= kc), splits them into NPART
// parts and stores them in the canonical K-major layout.  Where a segment
// starts in its superset: K contiguous, the row's own address (one shift
// for all its values, applied by branch-free selects on 16-byte reads);
// rows contiguous, the shift table the issuing threads wrote.
template <int NPART>
__device__ __forceinline__ void tc_split(const float* raw, const unsigned char* shtab, const float* X, int ldx,
                                         bool rows_contig, int k0, int kk0, int kc, int R, int q, float* dst) {
  using Cfg = TcCfg<NPART>;
  float v[16];
  if (rows_contig) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int kk = kk0 + j;
      v[j] = (q < R && kk < kc) ? raw[kk * kTcPitchR + shtab[kk] + q] : 0.f;
    }
  } else {
    const int sh = (int)((reinterpret_cast<uintptr_t>(X + (size_t)q * ldx + k0) & 15) >> 2);
    float a[20];
    const float* rp = raw + q * Cfg::kPitchK + kk0;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const float4 f = *reinterpret_cast<const float4*>(rp + 4 * m);
      a[4 * m] = f.x;
      a[4 * m + 1] = f.y;
      a[4 * m + 2] = f.z;
      a[4 * m + 3] = f.w;
    }
    const bool s1 = sh & 1, s2 = sh & 2, live = q < R;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float w0 = s1 ? a[j + 1] : a[j];
      const float w1 = s1 ? a[j + 3] : a[j + 2];
      const float w = s2 ? w1 : w0;
      v[j] = (live && kk0 + j < kc) ? w : 0.f;
    }
  }
#pragma unroll
  for (int kq = 0; kq < kTcKC / 4; ++kq) {
    const int off = (q >> 3) * (kTcKC / 4) * 32 + kq * 32 + (q & 7) * 4;   // floats
#pragma unroll
    for (int part = 0; part < NPART; ++part) {
      float4 o;
      float* po = reinterpret_cast<float*>(&o);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float h = tf32_hi(v[4 * kq + e]);
        po[e] = h;
        v[4 * kq + e] = __fsub_rn(v[4 * kq + e], h);
      }
      *reinterpret_cast<float4*>(dst + part * kTcPartA + off) = o;
    }
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

template <int NPART>
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_tc(const GemmTask<float>* __restrict__ tasks,
                                                           const GemmContrib<float>* __restrict__ cons) {
  using Cfg = TcCfg<NPART>;
  constexpr int kStages = Cfg::kStages;
  const GemmTask<float> tk = tasks[blockIdx.x];
  extern __shared__ __align__(1024) unsigned char tc_smraw[];
  float* stg = reinterpret_cast<float*>(tc_smraw);   // kStages x [A parts | B parts]
  float* raw = stg + kStages * Cfg::kStage;           // 2 x [A | B] raw chunks
  // full[s], empty[s], acc_full[2], acc_empty[2], done, raw_full[2]
  __shared__ __align__(8) uint64_t mbar[2 * kStages + 7];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_bad;
  __shared__ unsigned char shtab[2][2][64];   // [raw stage][operand][k-row]: start of a row-contiguous k-row
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
  auto full = [&](int st) { return mb + 8u * st; };
  auto empty = [&](int st) { return mb + 8u * (kStages + st); };
  auto acc_full = [&](int b) { return mb + 8u * (2 * kStages + b); };
  auto acc_empty = [&](int b) { return mb + 8u * (2 * kStages + 2 + b); };
  const uint32_t done = mb + 8u * (2 * kStages + 4);
  auto raw_full = [&](int rs) { return mb + 8u * (2 * kStages + 5 + rs); };
  if (warp == kTcMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                 "r"(2 * kTileTC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(full(st)), "r"(kTcProd) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty(st)) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(acc_full(b)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(acc_empty(b)), "r"(kTcAccWarps * 32) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(done) : "memory");
    for (int rs = 0; rs < 2; ++rs)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(raw_full(rs)), "r"(kTcProd) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_bad = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int M = tk.M, N = tk.N, cend = tk.c_begin + tk.c_count;
  int nch = 0;
  for (int c = tk.c_begin; c < cend; ++c) nch += (max(cons[c].K, 0) + kTcKC - 1) / kTcKC;
  const int ngrp = (nch + kTcFlush - 1) / kTcFlush;

  if (warp < kTcProdWarps) {
    // ---- producers: raw chunk rc (kRawK values of K of one contribution) is
    // bulk-copied into raw stage rc mod 2 one chunk ahead; once it has landed
    // (its mbarrier) each thread splits its row of it, 16 values at a time,
    // into the operand stages (c mod kStages for the task's c-th 16-value
    // chunk).  Warps 0-3 take op(A), 4-7 op(B)^T.  A producer-only barrier
    // after each raw chunk frees its stage for the copies two chunks on.  A
    // producer whose wait gives up keeps walking the loop (arriving and
    // meeting the barrier, so no other producer waits for it in vain)
    // without storing.
    const int mat = warp >> 2, q = tid & (kTileTC - 1);
    const int R = mat ? N : M;
    const uint32_t raw0 = (uint32_t)__cvta_generic_to_shared(raw);
    TcCursor is{tk.c_begin, 0, {}};   // next raw chunk to copy
    tc_cursor_load(is, cons, cend);
    TcCursor sp = is;                 // raw chunk being split
    auto issue = [&](int rc) {
      const int rs = rc & 1, kc = min(Cfg::kRawK, is.cb.K - is.k0);
      const uint32_t dst = raw0 + 4u * (uint32_t)((2 * rs + mat) * Cfg::kRawOp);
      if (mat == 0)
        tc_issue<NPART>(is.cb.A, is.cb.lda, !(is.cb.flags & kTransA), is.k0, kc, R, q, dst, raw_full(rs), shtab[rs][0]);
      else
        tc_issue<NPART>(is.cb.B, is.cb.ldb, (is.cb.flags & kTransB) != 0, is.k0, kc, R, q, dst, raw_full(rs), shtab[rs][1]);
      tc_cursor_next(is, cons, cend, Cfg::kRawK);
    };
    bool bad = false;
    int c = 0;
    if (is.c < cend) issue(0);
    for (int rc = 0; sp.c < cend; ++rc) {
      if (is.c < cend) issue(rc + 1);
      if (!bad && !tc_wait(raw_full(rc & 1), (uint32_t)((rc >> 1) & 1))) bad = true;
      const float* rawop = raw + (2 * (rc & 1) + mat) * Cfg::kRawOp;
      const unsigned char* sht = shtab[rc & 1][mat];
      const int kc = min(Cfg::kRawK, sp.cb.K - sp.k0);
      for (int kk0 = 0; kk0 < kc; kk0 += kTcKC, ++c) {
        const int st = c % kStages;
        if (!bad && c >= kStages && !tc_wait(empty(st), (uint32_t)(((c / kStages) + 1) & 1))) bad = true;
        if (!bad) {
          float* dst = stg + st * Cfg::kStage + mat * NPART * kTcPartA;
          if (mat == 0)
            tc_split<NPART>(rawop, sht, sp.cb.A, sp.cb.lda, !(sp.cb.flags & kTransA), sp.k0, kk0, kc, R, q, dst);
          else
            tc_split<NPART>(rawop, sht, sp.cb.B, sp.cb.ldb, (sp.cb.flags & kTransB) != 0, sp.k0, kk0, kc, R, q, dst);
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(full(st)) : "memory");
        }
      }
      tc_cursor_next(sp, cons, cend, Cfg::kRawK);
      asm volatile("bar.sync 1, %0;\n" ::"n"(kTcProd) : "memory");   // raw stage rc mod 2 read by every producer
    }
    if (bad) atomicExch(&s_bad, 1);
  } else if (warp == kTcMmaWarp) {
    // ---- MMA issue (one thread)
    if (lane == 0) {
      bool bad = false;
      for (int g = 0; g < ngrp && !bad; ++g) {
        const int b = g & 1;
        if (g >= 2 && !tc_wait(acc_empty(b), (uint32_t)(((g >> 1) + 1) & 1))) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(b * kTileTC);
        const int c1 = min(nch, (g + 1) * kTcFlush);
        for (int c = g * kTcFlush; c < c1; ++c) {
          const int st = c % kStages;
          if (!tc_wait(full(st), (uint32_t)((c / kStages) & 1))) {
            bad = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t sA = (uint32_t)__cvta_generic_to_shared(stg + st * Cfg::kStage);
          const uint32_t sB = sA + 4u * NPART * kTcPartA;
#pragma unroll
          for (int ks = 0; ks < kTcKC / 8; ++ks) {
            const uint32_t ko = ks * 2 * 128;   // two core matrices along K per step
            // products p_i q_j with i + j < NPART, the small ones first
#pragma unroll
            for (int deg = NPART - 1; deg >= 0; --deg)
#pragma unroll
              for (int i = 0; i <= deg; ++i) {
                const int j = deg - i;
                const uint64_t ad = tc_desc(sA + 4u * i * kTcPartA + ko);
                const uint64_t bd = tc_desc(sB + 4u * j * kTcPartA + ko);
                const uint32_t accum = (c > g * kTcFlush || ks > 0 || deg < NPART - 1 || i > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                    "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accum)
                    : "memory");
              }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           empty(st))
                       : "memory");
        }
        // the group's partial sum is complete once its products are
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         acc_full(b))
                     : "memory");
      }
      // tracks every product issued above, whether or not the loops finished
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                   : "memory");
      if (bad) atomicExch(&s_bad, 1);
    }
    __syncwarp();
  } else {
    // ---- accumulators: warp w reads tensor-memory lanes 32 (w mod 4) .. + 31
    // (the lane quadrant a warp may access), columns col0 .. col0 + 63
    const int qd = warp & 3;
    const int row = 32 * qd + lane;
    const int col0 = kTcAccCols * ((warp - kTcAccWarp0) >> 2);
    float acc[kTcAccCols];
#pragma unroll
    for (int j = 0; j < kTcAccCols; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int g = 0; g < ngrp; ++g) {
      const int b = g & 1;
      if (ok && !tc_wait(acc_full(b), (uint32_t)((g >> 1) & 1))) ok = false;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int h = 0; h < kTcAccCols / 16; ++h) {
        uint32_t r0[16];
        tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * kTileTC + col0 + 16 * h), r0);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[16 * h + t] += __uint_as_float(r0[t]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acc_empty(b)) : "memory");
    }
    if (!ok) atomicExch(&s_bad, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // (1) every role has finished its loop and recorded failures
    const bool poisoned = s_bad != 0;
    // the task is read again here rather than kept live through the loop
    const GemmTask<float> te = tasks[blockIdx.x];
    if (row < te.M) {
      float* pc = te.C + (size_t)row + (size_t)col0 * te.ldc;
#pragma unroll
      for (int jj = 0; jj < kTcAccCols; ++jj) {
        if (col0 + jj < te.N) {
          if (nch == 0) {
            if (!te.beta) *pc = 0.f;
          } else {
            float v = poisoned ? __int_as_float(0x7fc00000) : te.alpha * acc[jj];
            if (te.beta) v += *pc;
            *pc = v;
          }
        }
        pc += te.ldc;
      }
    }
    return;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();   // (1)
  if (warp == kTcMmaWarp) {
    // the tensor memory is released only once every product issued has
    // completed (the commit tracks them all), or the bounded wait gave up
    tc_wait(done, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * kTileTC)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// diagonal tile: Cholesky + inverse of the factor
// ---------------------------------------------------------------------------
constexpr int kPitch = kTile + 1;

// Cholesky of the n x n tile A (ld lda) in shared memory S, L^{-1} in V;
// writes L (strict upper part zeroed) back to A and L^{-1} to Li.  Returns
// 0, 1 (pivot <= 0) or 2 (non-finite pivot), the same in every thread.
//
// Right-looking with one barrier per column: every thread reads the pivot d_j
// itself, the trailing update uses the unscaled column (a_ik -= a_ij a_kj /
// d_j), and the columns are scaled by d_j^{-1/2} once at the end.  The inverse
// is a forward substitution per column of V, each owned by four lanes of one
// warp, so its row steps need only warp synchronisation.
template <typename T>
__device__ int diag_tile(T* A, int lda, T* Li, int ldli, int n, T* S, T* V) {
  __shared__ int bad;
  __shared__ T dinv[kTile];   // d_j^{-1/2}
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int i = e % n, j = e / n;
    S[i * kPitch + j] = A[(size_t)i + (size_t)j * lda];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int mybad = 0;
  for (int j = 0; j < n; ++j) {
    T d = S[j * kPitch + j];
    if (!(d > T(0)) || !isfinite(d)) {
      mybad = isfinite(d) ? 1 : 2;
      d = T(1);
    }
    const T rd = T(1) / d;
    // trailing lower triangle, 16 x 16 thread grid; column j itself is read only
    for (int i = j + 1 + ty; i < n; i += 16) {
      const T lij = S[i * kPitch + j] * rd;
      for (int k = j + 1 + tx; k <= i; k += 16) S[i * kPitch + k] -= lij * S[k * kPitch + j];
    }
    if (threadIdx.x == 0) {
      dinv[j] = T(1) / sqrt(d);
      if (mybad) S[j * kPitch + j] = d;   // failed pivot: continue with 1 (status reported)
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && mybad) bad = mybad;
  // scale: L_ij = a_ij d_j^{-1/2} (diagonal: sqrt(d_j))
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int i = e / n, j = e % n;
    if (j <= i) S[i * kPitch + j] *= dinv[j];
  }
  __syncthreads();
  {
    const int c = threadIdx.x >> 2, part = threadIdx.x & 3;
    for (int i = 0; i < n; ++i) {
      T sum = T(0);
      if (c < i)
        for (int k = c + part; k < i; k += 4) sum = fma(S[i * kPitch + k], V[k * kPitch + c], sum);
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      if (part == 0 && c <= i) V[i * kPitch + c] = ((c == i ? T(1) : T(0)) - sum) / S[i * kPitch + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int i = e % n, j = e / n;
    A[(size_t)i + (size_t)j * lda] = (i >= j) ? S[i * kPitch + j] : T(0);
    Li[(size_t)i + (size_t)j * ldli] = (i >= j) ? V[i * kPitch + j] : T(0);
  }
  __syncthreads();
  return bad;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_diag(const DiagTask<T>* __restrict__ tasks,
                                                   DevStatus* st, int level) {
  const DiagTask<T> tk = tasks[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  T* V = S + kTile * kPitch;
  const int bad = diag_tile<T>(tk.A, tk.lda, tk.Li, tk.ldli, tk.n, S, V);
  if (threadIdx.x == 0 && bad) report(st, bad == 1 ? SGF_ERR_NOT_SPD : SGF_ERR_NONFINITE, level, tk.node);
}

// C[M x N] = beta C + alpha op(A) op(B), M, N <= 64, by the whole CTA, with
// shared staging As/Bs (kKC x (kTile + 1) each).  The next K chunk is loaded
// into registers while the current one is multiplied, so the global load
// latency overlaps the arithmetic.  Ends with a barrier.
template <typename T>
__device__ void cta_gemm(T* C, int ldc, int M, int N, T alpha, int beta, const T* A, int lda, bool ta,
                         const T* B, int ldb, bool tb, int K, T (*As)[kTile + 1], T (*Bs)[kTile + 1]) {
  constexpr int NL = (kKC * kTile) / kThreads;   // elements of A (and of B) per thread per chunk
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = T(0);
  T ra[NL], rb[NL];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + kThreads * q;
      int i, kk;
      if (!ta) { i = e & 63; kk = e >> 6; } else { kk = e & 15; i = e >> 4; }
      ra[q] = (i < M && k0 + kk < K)
                  ? (ta ? A[(size_t)(k0 + kk) + (size_t)i * lda] : A[(size_t)i + (size_t)(k0 + kk) * lda])
                  : T(0);
      int j;
      if (!tb) { kk = e & 15; j = e >> 4; } else { j = e & 63; kk = e >> 6; }
      rb[q] = (j < N && k0 + kk < K)
                  ? (tb ? B[(size_t)j + (size_t)(k0 + kk) * ldb] : B[(size_t)(k0 + kk) + (size_t)j * ldb])
                  : T(0);
    }
  };
  if (K > 0) load(0);
  for (int k0 = 0; k0 < K; k0 += kKC) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + kThreads * q;
      if (!ta) As[e >> 6][e & 63] = ra[q]; else As[e & 15][e >> 4] = ra[q];
      if (!tb) Bs[e & 15][e >> 4] = rb[q]; else Bs[e >> 6][e & 63] = rb[q];
    }
    __syncthreads();
    if (k0 + kKC < K) load(k0 + kKC);
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
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = ty + 16 * r, j = tx + 16 * q;
      if (i < M && j < N) {
        T* p = C + (size_t)i + (size_t)j * ldc;
        T v = alpha * acc[r][q];
        if (beta) v += *p;
        *p = v;
      }
    }
  __syncthreads();
}

// FP32 CTA tile product with the k_gemm<float> scheme: 4x4 blocks of
// consecutive rows / columns per thread, 16-byte shared-memory operand reads,
// double-buffered chunks with the next chunk prefetched into registers.
__device__ void cta_gemm_f(float* C, int ldc, int M, int N, float alpha, int beta, const float* A, int lda,
                           bool ta, const float* B, int ldb, bool tb, int K, float (*As)[kKC][kPitchF],
                           float (*Bs)[kKC][kPitchF]) {
  GemmContrib<float> cb;
  cb.A = A;
  cb.B = B;
  cb.lda = lda;
  cb.ldb = ldb;
  cb.K = K;
  cb.flags = (ta ? kTransA : 0) | (tb ? kTransB : 0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
  if (K > 0) {
    float ra[4], rb[4];
    gemm_load_chunk(cb, M, N, 0, ra, rb);
    gemm_store_chunk(cb, As[0], Bs[0], ra, rb);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += kKC) {
      const bool more = k0 + kKC < K;
      if (more) gemm_load_chunk(cb, M, N, k0 + kKC, ra, rb);
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
      }
      if (more) {
        gemm_store_chunk(cb, As[buf ^ 1], Bs[buf ^ 1], ra, rb);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ty * 4 + r;
    if (i >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = tx * 4 + q;
      if (j < N) {
        float* p = C + (size_t)i + (size_t)j * ldc;
        float v = alpha * acc[r][q];
        if (beta) v += *p;
        *p = v;
      }
    }
  }
  __syncthreads();
}

// Shared staging of the front kernel's tile products after S and V: the FP32
// kernel uses the double-buffered 16-byte layout, FP64 the plain one.
template <typename T>
struct FrontStage {
  static size_t bytes() { return 2 * sizeof(T) * kKC * (kTile + 1); }
  static __device__ void gemm(T* C, int ldc, int M, int N, T alpha, int beta, const T* A, int lda, bool ta,
                              const T* B, int ldb, bool tb, int K, unsigned char* st) {
    T (*As)[kTile + 1] = reinterpret_cast<T (*)[kTile + 1]>(st);
    cta_gemm<T>(C, ldc, M, N, alpha, beta, A, lda, ta, B, ldb, tb, K, As, As + kKC);
  }
};
template <>
struct FrontStage<float> {
  static size_t bytes() { return 2 * 2 * sizeof(float) * kKC * kPitchF; }
  static __device__ void gemm(float* C, int ldc, int M, int N, float alpha, int beta, const float* A, int lda,
                              bool ta, const float* B, int ldb, bool tb, int K, unsigned char* st) {
    float (*As)[kKC][kPitchF] = reinterpret_cast<float (*)[kKC][kPitchF]>(st);
    cta_gemm_f(C, ldc, M, N, alpha, beta, A, lda, ta, B, ldb, tb, K, As, As + 2);
  }
};

// Whole blocked Cholesky of an m x m front D with L^{-1} in Li, one CTA per
// front (small fronts): the same diagonal-tile / panel / trailing-update
// sweep as the multi-launch path, without a launch per step.
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) k_front(const FrontTask<T>* __restrict__ tasks,
                                                    DevStatus* st, int level) {
  const FrontTask<T> tk = tasks[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  T* V = S + kTile * kPitch;
  unsigned char* stg = reinterpret_cast<unsigned char*>(V + kTile * kPitch);   // 16-byte aligned
  const int m = tk.m;
  T* D = tk.D;
  T* Li = tk.Li;
  const int nt = (m + kTile - 1) / kTile;
  int bad = 0;
  for (int k = 0; k < nt; ++k) {
    const int r0 = k * kTile, nk = min(kTile, m - r0), r1 = r0 + nk;
    T* Likk = Li + r0 + (size_t)r0 * m;
    const int b = diag_tile<T>(D + r0 + (size_t)r0 * m, m, Likk, m, nk, S, V);
    if (b && !bad) bad = b;
    for (int ri = r1; ri < m; ri += kTile) {
      T* C = D + ri + (size_t)r0 * m;
      FrontStage<T>::gemm(C, m, min(kTile, m - ri), nk, T(1), 0, C, m, false, Likk, m, true, nk, stg);
    }
    for (int j0 = 0; j0 < r0; j0 += kTile) {
      T* C = Li + r0 + (size_t)j0 * m;
      FrontStage<T>::gemm(C, m, nk, min(kTile, r0 - j0), T(1), 0, Likk, m, false, C, m, false, nk, stg);
    }
    for (int rj = r1; rj < m; rj += kTile) {
      const int nj = min(kTile, m - rj);
      for (int ri = rj; ri < m; ri += kTile)
        FrontStage<T>::gemm(D + ri + (size_t)rj * m, m, min(kTile, m - ri), nj, T(-1), 1, D + ri + (size_t)r0 * m, m,
                    false, D + rj + (size_t)r0 * m, m, true, nk, stg);
    }
    for (int ri = r1; ri < m; ri += kTile)
      for (int j0 = 0; j0 < r1; j0 += kTile)
        FrontStage<T>::gemm(Li + ri + (size_t)j0 * m, m, min(kTile, m - ri), min(kTile, r1 - j0), T(-1), 1,
                    D + ri + (size_t)r0 * m, m, false, Li + r0 + (size_t)j0 * m, m, false, nk, stg);
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
    if (tk.mode == kMirror) {   // upper entries of the tile from their transposes
      if (i < j) tk.dst[(size_t)i + (size_t)j * tk.ldd] = (D)tk.src[(size_t)j + (size_t)i * tk.lds];
      continue;
    }
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
// Columns that are exactly zero (monomials on the flat axes of a face or edge
// cell, Sec. 3.1) are dropped before the sweep; pivoting swaps entries of a
// column map instead of moving data; the pivot of step k is the largest of
// the per-warp maxima recorded while step k-1 refreshed the trailing column
// norms.  The matrix is copied to shared memory when m * c_eff fits in the
// launch's capacity, else the sweep runs on the global workspace.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_qrcp(const QrTask<T>* __restrict__ tasks, int* ranks,
                                                   double tau, long long cap_elems) {
  using Acc = T;  // column sweeps in the working precision (FP64 is ~1/64 rate here)
  const QrTask<T> tk = tasks[blockIdx.x];
  const int m = tk.m, c = tk.c;
  const int kmn = m < c ? m : c;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* norms = reinterpret_cast<double*>(smraw);   // c
  double* betas = norms + c;                          // kmn
  int* colmap = reinterpret_cast<int*>(betas + kmn);  // c
  uintptr_t vp = (reinterpret_cast<uintptr_t>(colmap + c) + 15) & ~uintptr_t(15);
  T* v = reinterpret_cast<T*>(vp);                    // m
  uintptr_t mp = (reinterpret_cast<uintptr_t>(v + m) + 15) & ~uintptr_t(15);
  T* Ms = reinterpret_cast<T*>(mp);                   // cap_elems
  __shared__ double pv[kThreads / 32];
  __shared__ int pj[kThreads / 32];
  __shared__ double s_x;
  __shared__ int s_i;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
  T* A = tk.A;
  for (int j = warp; j < c; j += nw) {
    Acc sq = 0;
    for (int i = lane; i < m; i += 32) {
      const Acc a = A[(size_t)i + (size_t)j * m];
      sq = fma(a, a, sq);
    }
    sq = warp_sum(sq);
    if (lane == 0) norms[j] = (double)sq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int j = 0; j < c; ++j)
      if (norms[j] > 0.0) {
        norms[cnt] = norms[j];
        colmap[cnt] = j;
        ++cnt;
      }
    s_i = cnt;
  }
  __syncthreads();
  const int ce = s_i;
  const bool in_smem = (long long)m * ce <= cap_elems;
  T* M = A;
  if (in_smem) {
    for (int q = warp; q < ce; q += nw) {
      const T* src = A + (size_t)colmap[q] * m;
      for (int i = lane; i < m; i += 32) Ms[(size_t)i + (size_t)q * m] = src[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ce; q += kThreads) colmap[q] = q;
    M = Ms;
  }
  // initial per-warp maxima over all columns
  {
    double best = -1.0;
    int bj = 1 << 30;
    for (int j = warp; j < ce; j += nw)
      if (norms[j] > best) { best = norms[j]; bj = j; }
    if (lane == 0) { pv[warp] = best; pj[warp] = bj; }
  }
  __syncthreads();
  const int kmax = m < ce ? m : ce;
  int r = 0;
  double ref = 0;
  for (int k = 0; k < kmax; ++k) {
    if (threadIdx.x == 0) {
      double b = pv[0];
      int p = pj[0];
      for (int w = 1; w < nw; ++w)
        if (pv[w] > b || (pv[w] == b && pj[w] < p)) { b = pv[w]; p = pj[w]; }
      s_x = b;
      s_i = p;
      if (p != k && p < ce) {
        const int t = colmap[k]; colmap[k] = colmap[p]; colmap[p] = t;
        const double u = norms[k]; norms[k] = norms[p]; norms[p] = u;
      }
    }
    __syncthreads();
    const double nrm = sqrt(s_x > 0 ? s_x : 0.0);
    if (k == 0) ref = nrm;
    if (!(nrm > tau * ref) || ref == 0.0) break;
    T* col = M + (size_t)colmap[k] * m;
    Acc sq = 0;
    for (int i = k + threadIdx.x; i < m; i += kThreads) {
      const T a = col[i];
      v[i] = a;
      sq = fma(a, a, sq);
    }
    sq = warp_sum(sq);
    if (lane == 0) pv[warp] = (double)sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0;
      for (int w = 0; w < nw; ++w) tot += pv[w];
      const double normx = sqrt(tot);
      const double x0 = (double)v[k];
      const double alpha = x0 >= 0 ? -normx : normx;
      double beta = 0;
      if (normx > 0) {
        beta = 1.0 / (alpha * (alpha - x0));
        v[k] = (T)(x0 - alpha);
      }
      betas[k] = beta;
      col[k] = v[k];
    }
    __syncthreads();
    const double beta = betas[k];
    double best = -1.0;
    int bj = 1 << 30;
    for (int j = k + 1 + warp; j < ce; j += nw) {
      T* cj = M + (size_t)colmap[j] * m;
      Acc w = 0;
      for (int i = k + lane; i < m; i += 32) w = fma(v[i], cj[i], w);
      w = warp_sum(w);
      const Acc f = (Acc)beta * w;
      Acc s2 = 0;
      for (int i = k + lane; i < m; i += 32) {
        const T a = fma(-f, v[i], cj[i]);
        cj[i] = a;
        if (i > k) s2 = fma(a, a, s2);
      }
      s2 = warp_sum(s2);
      if (lane == 0) norms[j] = (double)s2;
      if ((double)s2 > best) { best = (double)s2; bj = j; }
    }
    if (lane == 0) { pv[warp] = best; pj[warp] = bj; }
    __syncthreads();
    r = k + 1;
  }
  if (threadIdx.x == 0) ranks[tk.slot] = r;
  // Q1 = H_0 ... H_{r-1} [I_r; 0]
  T* Q = tk.Q1;
  for (int e = threadIdx.x; e < m * r; e += kThreads) {
    const int i = e % m, j = e / m;
    Q[(size_t)i + (size_t)j * m] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    const T* col = M + (size_t)colmap[k] * m;
    for (int i = k + threadIdx.x; i < m; i += kThreads) v[i] = col[i];
    __syncthreads();
    const double beta = betas[k];
    for (int j = k + warp; j < r; j += nw) {
      T* qc = Q + (size_t)j * m;
      Acc w = 0;
      for (int i = k + lane; i < m; i += 32) w = fma(v[i], qc[i], w);
      w = warp_sum(w);
      const Acc f = (Acc)beta * w;
      for (int i = k + lane; i < m; i += 32) qc[i] = fma(-f, v[i], qc[i]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// batched GEMV
// ---------------------------------------------------------------------------
// Contributions of a task staged in shared memory with the flat prefix of
// their useful lengths (pre[c] .. pre[c + 1] is contribution c).
template <typename T>
struct GemvStage {
  GemvContrib<T> c[kGemvMaxC];
  int kb[kGemvMaxC];
  int pre[kGemvMaxC + 1];
};

template <typename T>
__device__ __forceinline__ void gemv_stage(const GemvTask<T>& tk, const GemvContrib<T>* __restrict__ cons,
                                           bool trans, GemvStage<T>& S) {
  const int t = threadIdx.x;
  if (t < 32) {
    int len = 0;
    if (t < tk.c_count) {
      const GemvContrib<T> c = cons[tk.c_begin + t];
      int kb, ke;
      gemv_useful(trans, c.tri, c.upper, c.K, tk.M, &kb, &ke);
      S.c[t] = c;
      S.kb[t] = kb;
      len = ke - kb;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, len, o);
      if (t >= o) len += v;
    }
    S.pre[t + 1] = len;
    if (t == 0) S.pre[0] = 0;
  }
  __syncthreads();
}

// A task's result element e (= output * NR + rhs): written to y when the
// chunk is not split, else to the task's partial.
template <typename T>
__device__ __forceinline__ void gemv_put(const GemvTask<T>& tk, int e, T v, int ne) {
  if (tk.nsplit == 1) {
    T* y = tk.y + e;
    *y = tk.beta ? *y + v : v;
  } else {
    tk.part[(size_t)tk.split * ne + e] = v;
  }
}

// Split tasks: after every partial of this task is written, the last of the
// chunk's tasks to arrive adds the partials in split order, writes y and
// re-arms the counter for the next launch.  Nothing waits.
template <typename T>
__device__ __forceinline__ void gemv_finish(const GemvTask<T>& tk, int ne) {
  if (tk.nsplit == 1) return;
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(tk.cnt, 1) == tk.nsplit - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = threadIdx.x; e < ne; e += kThreads) {
    T v = T(0);
    for (int sp = 0; sp < tk.nsplit; ++sp) v += __ldcg(tk.part + (size_t)sp * ne + e);
    T* y = tk.y + e;
    *y = tk.beta ? *y + v : v;
  }
  if (threadIdx.x == 0) *tk.cnt = 0;
}

// Bulk prefetch of the 16-byte-aligned interior of [p, p + bytes) into L2
// (no registers held, nothing returned; the ragged ends are left to the loads).
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = (a + 15) & ~uintptr_t(15), hi = (a + bytes) & ~uintptr_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// Programmatic dependent launch: every block of an apply kernel lets the next
// kernel of the program launch as soon as it has started (once all blocks
// have, the next grid may fill the SMs this one frees), and waits for the
// previous grid's completion and memory flush before it touches a vector.
// Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Warp-granular GEMVs for chunks too small to fill a CTA (unsplit tasks of
// at most kGemvWarpElems elements, see GemvList::emit): they ride in the same
// launch as the CTA tasks, eight to a block, one per warp, with no shared
// staging and no barrier.  Each output's sum runs over its contributions in
// order, lane l taking the rows (op T) or columns (op N) l, l + 32, ... of
// each, then a butterfly (op T) - the same order for every NR.
//
// op(A) = A^T: the warp walks the chunk's outputs CW at a time (their loads
// interleaved); each column is read only over its useful rows (a triangular
// block's zero half is skipped per column).
template <typename T, int NR>
__device__ __forceinline__ void gemv_tw_one(const GemvTask<T>& tk, const GemvContrib<T>* __restrict__ cons, int lane) {
  constexpr int CW = NR <= 2 ? 4 : 2;
  constexpr int U = sizeof(T) == 4 ? 4 : 2;   // row steps in flight
  for (int o0 = 0; o0 < tk.M; o0 += CW) {
    T acc[CW][NR];
#pragma unroll
    for (int u = 0; u < CW; ++u)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[u][q] = T(0);
    for (int c = tk.c_begin; c < tk.c_begin + tk.c_count; ++c) {
      const GemvContrib<T> cb = cons[c];
      const T* col[CW];
      int lo[CW], hi[CW];
      int rlo = cb.K, rhi = 0;
#pragma unroll
      for (int u = 0; u < CW; ++u) {
        const int o = o0 + u;
        col[u] = cb.A + (size_t)o * cb.lda;
        lo[u] = 0;
        hi[u] = o < tk.M ? cb.K : 0;
        if (cb.tri && o < tk.M) {
          if (cb.upper) hi[u] = min(cb.K, cb.tri + o);   // rows <= absolute column tri - 1 + o
          else lo[u] = cb.tri - 1 + o;                    // rows >= it
        }
        if (hi[u] > lo[u]) {
          rlo = min(rlo, lo[u]);
          rhi = max(rhi, hi[u]);
        }
      }
#pragma unroll U
      for (int i = rlo + lane; i < rhi; i += 32) {
        T xv[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          T v = cb.x[(size_t)i * NR + q];
          if (cb.x2) v -= cb.x2[(size_t)i * NR + q];
          xv[q] = cb.alpha * v;
        }
        T av[CW];
#pragma unroll
        for (int u = 0; u < CW; ++u) av[u] = (i >= lo[u] && i < hi[u]) ? col[u][i] : T(0);
#pragma unroll
        for (int u = 0; u < CW; ++u)
#pragma unroll
          for (int q = 0; q < NR; ++q) acc[u][q] = fma(av[u], xv[q], acc[u][q]);
      }
    }
#pragma unroll
    for (int u = 0; u < CW; ++u) {
      const int o = o0 + u;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const T v = warp_sum(acc[u][q]);
        if (lane == 0 && o < tk.M) {
          T* y = tk.y + (size_t)o * NR + q;
          *y = tk.beta ? *y + v : v;
        }
      }
    }
  }
}

// op(A) = A, chunks of at most kGemvWarpRows rows: lane l owns rows l, l + 32,
// ... of the band (RP of them), so no reduction is needed; the warp walks
// the columns of every contribution in order, U at a time.
constexpr int kGemvWarpRows = kGemvWarpRowsMax;
template <typename T, int NR>
__device__ __forceinline__ void gemv_nw_one(const GemvTask<T>& tk, const GemvContrib<T>* __restrict__ cons, int lane) {
  constexpr int RP = kGemvWarpRows / 32;
  constexpr int U = 4;   // columns in flight
  T acc[RP][NR];
#pragma unroll
  for (int r = 0; r < RP; ++r)
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[r][q] = T(0);
  for (int c = tk.c_begin; c < tk.c_begin + tk.c_count; ++c) {
    const GemvContrib<T> cb = cons[c];
    int kb, ke;
    gemv_useful(false, cb.tri, cb.upper, cb.K, tk.M, &kb, &ke);
#pragma unroll U
    for (int j = kb; j < ke; ++j) {
      const T* colp = cb.A + (size_t)j * cb.lda;
      const int rmin = cb.tri ? j - (cb.tri - 1) : 0;   // a lower-triangular block's zero rows
      T xv[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        T v = cb.x[(size_t)j * NR + q];
        if (cb.x2) v -= cb.x2[(size_t)j * NR + q];
        xv[q] = cb.alpha * v;
      }
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        const int row = lane + 32 * r;
        const T a = (row < tk.M && row >= rmin) ? colp[row] : T(0);
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[r][q] = fma(a, xv[q], acc[r][q]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RP; ++r) {
    const int row = lane + 32 * r;
    if (row < tk.M) {
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        T* y = tk.y + (size_t)row * NR + q;
        *y = tk.beta ? *y + acc[r][q] : acc[r][q];
      }
    }
  }
}

// blocks beyond the CTA tasks carry the warp tasks, one per warp
template <typename T, int NR, bool TRANS>
__device__ __forceinline__ void gemv_warp_block(const GemvTask<T>* __restrict__ wtasks, int nw,
                                                const GemvContrib<T>* __restrict__ cons, int block) {
  pdl_trigger();
  pdl_wait();   // x and y are written by earlier kernels
  const int t = block * (kThreads / 32) + (threadIdx.x >> 5);
  if (t >= nw) return;
  const GemvTask<T> tk = wtasks[t];
  if (TRANS) gemv_tw_one<T, NR>(tk, cons, threadIdx.x & 31);
  else gemv_nw_one<T, NR>(tk, cons, threadIdx.x & 31);
}

// One column of an op N step: its x entries (scaled) and the band rows of the
// current pass (zero outside the band and, for a lower-triangular block,
// above the diagonal).
template <typename T, int NR, int MP>
__device__ __forceinline__ void gemv_n_col(const GemvStage<T>& S, int& c, int f, int r0, int lane, int M,
                                           T (&av)[MP], T (&xv)[NR]) {
  while (f >= S.pre[c + 1]) ++c;
  const GemvContrib<T>& cb = S.c[c];
  const int j = S.kb[c] + (f - S.pre[c]);
  const T* col = cb.A + (size_t)j * cb.lda;
  const int rmin = cb.tri ? j - (cb.tri - 1) : 0;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    T v = cb.x[(size_t)j * NR + q];
    if (cb.x2) v -= cb.x2[(size_t)j * NR + q];
    xv[q] = cb.alpha * v;
  }
#pragma unroll
  for (int t = 0; t < MP; ++t) {
    const int r = r0 + lane + 32 * t;
    av[t] = (r < M && r >= rmin) ? col[r] : T(0);
  }
}

// op(A) = A: a band of <= 32 * MT rows (MT = 8 or 16, chosen per launch from
// its largest band).  The task's column segments are first prefetched into L2
// (thread t takes flat columns t, t + 256, ...).  Warp w then takes the flat
// columns k_lo + w, k_lo + w + 8, ..., two per step so that two columns' loads
// are in flight; its lanes read the column's band rows (coalesced, 32
// consecutive rows per load) into per-row accumulators, and the eight warps'
// partial rows are added in warp order.  For NR > 1 the band is swept in
// passes of fewer rows so the registers stay bounded; each row's sum runs
// over the same columns in the same order for every NR.
template <typename T, int NR, int MT>
__global__ void __launch_bounds__(kThreads) k_gemv_n(const GemvTask<T>* __restrict__ tasks,
                                                     const GemvContrib<T>* __restrict__ cons, int ncta,
                                                     const GemvTask<T>* __restrict__ wtasks, int nw) {
  constexpr int kWarps = kThreads / 32;
  constexpr int MP = MT / NR > 0 ? MT / NR : 1;   // 32-row groups per pass
  // two columns per step unless that would cost too many registers (FP64, wide bands)
  constexpr bool kTwo = sizeof(T) == 4 || MP <= 8;
  if ((int)blockIdx.x >= ncta) return gemv_warp_block<T, NR, false>(wtasks, nw, cons, blockIdx.x - ncta);
  pdl_trigger();
  const GemvTask<T> tk = tasks[blockIdx.x];
  __shared__ GemvStage<T> S;
  __shared__ T red[kWarps][32 * MP * NR];
  gemv_stage(tk, cons, false, S);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    int c = 0;
    for (int f = tk.k_lo + threadIdx.x; f < tk.k_hi; f += kThreads) {
      while (f >= S.pre[c + 1]) ++c;
      const GemvContrib<T>& cb = S.c[c];
      const int j = S.kb[c] + (f - S.pre[c]);
      const int rs = cb.tri ? max(0, j - (cb.tri - 1)) : 0;
      l2_prefetch(cb.A + (size_t)j * cb.lda + rs, sizeof(T) * (size_t)(tk.M - rs));
    }
  }
  pdl_wait();   // x, y and the partials are written by earlier kernels
  for (int r0 = 0; r0 < tk.M; r0 += 32 * MP) {
    T acc[MP][NR];
#pragma unroll
    for (int t = 0; t < MP; ++t)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[t][q] = T(0);
    int c = 0;
    for (int f = tk.k_lo + w; f < tk.k_hi; f += (kTwo ? 2 : 1) * kWarps) {
      T av0[MP], xv0[NR], av1[MP], xv1[NR];
      gemv_n_col<T, NR, MP>(S, c, f, r0, lane, tk.M, av0, xv0);
      const bool two = kTwo && f + kWarps < tk.k_hi;
      int c1 = c;
      if (two) {
        gemv_n_col<T, NR, MP>(S, c1, f + kWarps, r0, lane, tk.M, av1, xv1);
      } else {
#pragma unroll
        for (int t = 0; t < MP; ++t) av1[t] = T(0);
#pragma unroll
        for (int q = 0; q < NR; ++q) xv1[q] = T(0);
      }
#pragma unroll
      for (int t = 0; t < MP; ++t)
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[t][q] = fma(av0[t], xv0[q], acc[t][q]);
      if (two) {
#pragma unroll
        for (int t = 0; t < MP; ++t)
#pragma unroll
          for (int q = 0; q < NR; ++q) acc[t][q] = fma(av1[t], xv1[q], acc[t][q]);
      }
      c = c1;
    }
#pragma unroll
    for (int t = 0; t < MP; ++t)
#pragma unroll
      for (int q = 0; q < NR; ++q) red[w][(lane + 32 * t) * NR + q] = acc[t][q];
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * MP * NR; e += kThreads) {
      const int r = r0 + e / NR;
      if (r < tk.M) {
        T v = T(0);
#pragma unroll
        for (int k = 0; k < kWarps; ++k) v += red[k][e];
        gemv_put(tk, r0 * NR + e, v, tk.M * NR);
      }
    }
    __syncthreads();
  }
  gemv_finish(tk, tk.M * NR);
}

// op(A) = A^T: <= 8 CW outputs, column o of A handled by warp o % 8 (CW
// columns per warp, their loads interleaved).  The task's column
// segments are prefetched into L2 first; lanes then stride over the flat rows
// of each contribution, and the lane sums are combined by a butterfly.
template <typename T, int NR, int CW>
__global__ void __launch_bounds__(kThreads, NR <= 2 ? 4 : 2)
    k_gemv_t(const GemvTask<T>* __restrict__ tasks, const GemvContrib<T>* __restrict__ cons, int ncta,
             const GemvTask<T>* __restrict__ wtasks, int nw) {
  constexpr int kWarps = kThreads / 32;
  if ((int)blockIdx.x >= ncta) return gemv_warp_block<T, NR, true>(wtasks, nw, cons, blockIdx.x - ncta);
  pdl_trigger();
  const GemvTask<T> tk = tasks[blockIdx.x];
  __shared__ GemvStage<T> S;
  gemv_stage(tk, cons, true, S);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // prefetch: one (contribution, column) segment per thread
  for (int sidx = threadIdx.x; sidx < tk.c_count * tk.M; sidx += kThreads) {
    const int c = sidx / tk.M, o = sidx - c * tk.M;
    const int f0 = max(S.pre[c], tk.k_lo), f1 = min(S.pre[c + 1], tk.k_hi);
    if (f0 >= f1) continue;
    const GemvContrib<T>& cb = S.c[c];
    int i0 = S.kb[c] + (f0 - S.pre[c]);
    int i1 = S.kb[c] + (f1 - S.pre[c]);
    if (cb.tri && !cb.upper) i0 = max(i0, cb.tri - 1 + o);
    if (cb.tri && cb.upper) i1 = min(i1, cb.tri + o);   // rows <= tri - 1 + o
    if (i1 > i0) l2_prefetch(cb.A + (size_t)o * cb.lda + i0, sizeof(T) * (size_t)(i1 - i0));
  }
  pdl_wait();   // x, y and the partials are written by earlier kernels
  T acc[CW][NR];
#pragma unroll
  for (int u = 0; u < CW; ++u)
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[u][q] = T(0);
  if (w < tk.M) {
    for (int c = 0; c < tk.c_count; ++c) {
      const int f0 = max(S.pre[c], tk.k_lo), f1 = min(S.pre[c + 1], tk.k_hi);
      if (f0 >= f1) continue;
      const GemvContrib<T>& cb = S.c[c];
      const int i0 = S.kb[c] + (f0 - S.pre[c]), i1 = S.kb[c] + (f1 - S.pre[c]);
      const T* a = cb.A + (size_t)w * cb.lda;
      const size_t cstep = (size_t)kWarps * cb.lda;
      const int cmin = cb.tri ? cb.tri - 1 + w : 0;   // absolute column of u = 0
      int is = i0;   // first row of the scalar loop below
      if constexpr (sizeof(T) == 4) {
        // a dense contribution whose columns start on 16 bytes (the apply's
        // blocks have padded leading dimensions) and whose rows start on a
        // multiple of 4: lane l reads rows i0 + 4 l .. + 3 of each column with
        // one 16-byte load, then 128 rows on; the rest (< 4 rows) is scalar.
        // The choice does not depend on NR, so every NR sums in one order.
        if (!cb.tri && (i0 & 3) == 0 && (cb.lda & 3) == 0 && (reinterpret_cast<uintptr_t>(cb.A) & 15) == 0) {
          const int iv1 = i0 + ((i1 - i0) & ~3);
          constexpr int kVecUnroll = CW * NR <= 4 ? 2 : 1;
#pragma unroll kVecUnroll
          for (int i = i0 + 4 * lane; i < iv1; i += 128) {
            float xv[4][NR];
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                float v = cb.x[(size_t)(i + e) * NR + q];
                if (cb.x2) v -= cb.x2[(size_t)(i + e) * NR + q];
                xv[e][q] = cb.alpha * v;
              }
            float4 av[CW];
#pragma unroll
            for (int u = 0; u < CW; ++u)
              av[u] = w + kWarps * u < tk.M ? *reinterpret_cast<const float4*>(a + u * cstep + i)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < CW; ++u)
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                acc[u][q] = fma(av[u].x, xv[0][q], acc[u][q]);
                acc[u][q] = fma(av[u].y, xv[1][q], acc[u][q]);
                acc[u][q] = fma(av[u].z, xv[2][q], acc[u][q]);
                acc[u][q] = fma(av[u].w, xv[3][q], acc[u][q]);
              }
          }
          is = iv1;
        }
      }
      constexpr int kUnroll = (sizeof(T) == 4 && NR <= 2 && CW <= 4) ? 4 : 2;   // row steps in flight
#pragma unroll kUnroll
      for (int i = is + lane; i < i1; i += 32) {
        T xv[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          T v = cb.x[(size_t)i * NR + q];
          if (cb.x2) v -= cb.x2[(size_t)i * NR + q];
          xv[q] = cb.alpha * v;
        }
        T av[CW];
#pragma unroll
        for (int u = 0; u < CW; ++u) {
          const int o = w + kWarps * u;
          // triangular: rows above (lower) or below (upper) the column's
          // absolute index are zero
          const bool in_tri = !cb.tri || (cb.upper ? i <= cmin + kWarps * u : i >= cmin + kWarps * u);
          av[u] = (o < tk.M && in_tri) ? a[u * cstep + i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < CW; ++u)
#pragma unroll
          for (int q = 0; q < NR; ++q) acc[u][q] = fma(av[u], xv[q], acc[u][q]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < CW; ++u) {
    const int o = w + kWarps * u;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const T v = warp_sum(acc[u][q]);
      if (lane == 0 && o < tk.M) gemv_put(tk, o * NR + q, v, tk.M * NR);
    }
  }
  gemv_finish(tk, tk.M * NR);
}



// dst[p * nr + q] = src[idx[p] * nr + q]: gathers scattered level-vector
// entries into one contiguous vector (nr interleaved right-hand sides)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_vgather(const T* __restrict__ src, const int* __restrict__ idx,
                                                      T* __restrict__ dst, int n, int nr) {
  pdl_trigger();
  pdl_wait();
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= (int64_t)n * nr) return;
  const int64_t p = e / nr, q = e - p * nr;
  dst[e] = src[(int64_t)idx[p] * nr + q];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_veccopy(const VecCopyTask* __restrict__ tasks, int n,
                                                      const T* __restrict__ src, T* __restrict__ dst) {
  // one task per warp (a node's kept values: tens to hundreds), eight to a block
  pdl_trigger();
  const int t = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  pdl_wait();
  if (t >= n) return;
  const VecCopyTask tk = tasks[t];
  for (int i = threadIdx.x & 31; i < tk.len; i += 32) dst[tk.dst + i] = src[tk.src + i];
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

// Q1 elasticity (Sec. 7.1.3 on hexahedra): the 3x3 block between point p and
// its neighbour at offset o sums E_e * Kref over the (up to 8) elements that
// contain both nodes, in (ez, ey, ex) order.  Point x index i is node x = i + 1
// (the clamped x = 0 nodes are removed); elements ex x ey x ez with
// ex = nx, ey = ny - 1, ez = nz - 1.
template <typename T>
__global__ void k_assemble_q1(const double* __restrict__ E, const double* __restrict__ kref, int nx,
                              int ny, int nz, const int64_t* __restrict__ map, const int* __restrict__ ld,
                              int64_t dgsz, T* dg, T* up, double* __restrict__ bsr) {
  const int64_t npts = (int64_t)nx * ny * nz;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts * 27) return;
  const int64_t p = id / 27;
  const int o = (int)(id % 27);
  const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((int64_t)nx * ny));
  const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
  double blk[9];
  for (int k = 0; k < 9; ++k) blk[k] = 0.0;
  const int qx = x + dx, qy = y + dy, qz = z + dz;
  const bool inside = qx >= 0 && qx < nx && qy >= 0 && qy < ny && qz >= 0 && qz < nz;
  if (inside) {
    const int EX = nx, EY = ny - 1, EZ = nz - 1;
    const int X = x + 1, QX = qx + 1;
    for (int ez = max(z, qz) - 1; ez <= min(z, qz); ++ez) {
      if (ez < 0 || ez >= EZ) continue;
      for (int ey = max(y, qy) - 1; ey <= min(y, qy); ++ey) {
        if (ey < 0 || ey >= EY) continue;
        for (int ex = max(X, QX) - 1; ex <= min(X, QX); ++ex) {
          if (ex < 0 || ex >= EX) continue;
          const double e = E[ex + (int64_t)EX * (ey + (int64_t)EY * ez)];
          const int ap = (X - ex) + 2 * (y - ey) + 4 * (z - ez);
          const int aq = (QX - ex) + 2 * (qy - ey) + 4 * (qz - ez);
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) blk[3 * i + j] += e * kref[(3 * ap + i) * 24 + 3 * aq + j];
        }
      }
    }
  }
  for (int k = 0; k < 9; ++k) bsr[id * 9 + k] = blk[k];
  const int64_t base = map[id];
  if (base >= 0) {
    const int m = ld[p];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int64_t off = base + i + (int64_t)j * m;
        const T v = (T)blk[3 * i + j];
        if (off < dgsz) dg[off] = v; else up[off - dgsz] = v;
      }
  }
}

__global__ void k_spmv_bsr27(const double* __restrict__ bsr, int nx, int ny, int nz,
                             const double* __restrict__ x, double* __restrict__ yv) {
  const int64_t npts = (int64_t)nx * ny * nz;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const int px = (int)(p % nx), py = (int)((p / nx) % ny), pz = (int)(p / ((int64_t)nx * ny));
  double acc[3] = {0.0, 0.0, 0.0};
  for (int o = 0; o < 27; ++o) {
    const int qx = px + o % 3 - 1, qy = py + (o / 3) % 3 - 1, qz = pz + o / 9 - 1;
    if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
    const int64_t q = qx + (int64_t)nx * (qy + (int64_t)ny * qz);
    const double* b = bsr + (p * 27 + o) * 9;
    const double x0 = x[3 * q], x1 = x[3 * q + 1], x2 = x[3 * q + 2];
    for (int i = 0; i < 3; ++i) acc[i] = fma(b[3 * i], x0, fma(b[3 * i + 1], x1, fma(b[3 * i + 2], x2, acc[i])));
  }
  for (int i = 0; i < 3; ++i) yv[3 * p + i] = acc[i];
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

// natural-order RHS-major vectors <-> interleaved level-1 vectors
// nrhs dot products a_q . b_q (RHS-major vectors of length n), the same
// fixed-order reduction per RHS as k_dot_partial / k_dot_final
__global__ void k_dot_partial_n(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                double* __restrict__ partials) {
  const int q = blockIdx.y;
  const double* aq = a + (int64_t)q * n;
  const double* bq = b + (int64_t)q * n;
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    s = fma(aq[i], bq[i], s);
  s = warp_sum(s);
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t += w[k];
    partials[(int64_t)q * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_dot_final_n(const double* __restrict__ partials, int np, double* result) {
  const int q = blockIdx.x;
  double s = 0;
  for (int i = threadIdx.x; i < np; i += kThreads) s += partials[(int64_t)q * np + i];
  s = warp_sum(s);
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t += w[k];
    result[q] = t;
  }
}

// y_q = a_q x_q + y_q for q < nrhs (mode 0); p_q = z_q + a_q p_q (mode 1)
__global__ void k_axpy_n(Coef8 a, const double* __restrict__ x, double* __restrict__ y, int64_t n, int nrhs,
                         int mode) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < nrhs; ++q) {
    const int64_t k = (int64_t)q * n + i;
    y[k] = mode == 0 ? fma(a.v[q], x[k], y[k]) : fma(a.v[q], y[k], x[k]);
  }
}

// PCG step length per right-hand side q (one thread each): rz_q / pq_q where
// active, 0 where not or where the quotient is not finite (flagged)
__global__ void k_pcg_alpha(const double* __restrict__ pq, const double* __restrict__ rz, Coef8 act, int nrhs,
                            double* __restrict__ coef, double* __restrict__ flag) {
  const int q = threadIdx.x;
  if (q >= nrhs) return;
  const double a = act.v[q] != 0.0 ? rz[q] / pq[q] : 0.0;
  const bool bad = !isfinite(a);
  coef[q] = bad ? 0.0 : a;
  coef[8 + q] = bad ? 0.0 : -a;
  flag[q] = bad ? 1.0 : 0.0;
}

// x_q += alpha_q p_q, ro_q = r_q (optional), r_q -= alpha_q q_q in one pass,
// alpha_q and -alpha_q read from device memory
__global__ void k_pcg_xr(const double* __restrict__ coef, const double* __restrict__ p,
                         const double* __restrict__ qv, double* __restrict__ x, double* __restrict__ r,
                         double* __restrict__ ro, int64_t n, int nrhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < nrhs; ++q) {
    const int64_t k = (int64_t)q * n + i;
    const double rk = r[k];
    x[k] = fma(coef[q], p[k], x[k]);
    if (ro) ro[k] = rk;
    r[k] = fma(coef[8 + q], qv[k], rk);
  }
}

template <typename T>
__global__ void k_gather(const double* __restrict__ src, const int64_t* __restrict__ perm,
                         T* __restrict__ dst, int64_t n, int nrhs, int nr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p = perm[i];
  for (int q = 0; q < nr; ++q) dst[i * nr + q] = q < nrhs ? (T)src[(int64_t)q * n + p] : T(0);
}

// also raises *nonfinite (when given) if a value written is NaN or infinite:
// the flag costs no traffic unless it fires
template <typename T>
__global__ void k_scatter(const T* __restrict__ src, const int64_t* __restrict__ perm,
                          double* __restrict__ dst, int64_t n, int nrhs, int nr, int* nonfinite) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p = perm[i];
  bool bad = false;
  for (int q = 0; q < nrhs; ++q) {
    const double v = (double)src[i * nr + q];
    bad |= !isfinite(v);
    dst[(int64_t)q * n + p] = v;
  }
  if (bad && nonfinite) atomicOr(nonfinite, 1);
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

bool gemm_tc_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("SGF_TENSOR_CORES");
    return !(e && e[0] == '0');
  }();
  return on;
}

void launch_gemm_tc(const GemmTask<float>* tasks, const GemmContrib<float>* cons, int n, int nparts, cudaStream_t s) {
  if (dry_run()) {
    if (nparts != 2 && nparts != 3) check_range(nullptr, 1, "tc gemm split parts");
    for (int i = 0; i < n; ++i) {
      const GemmTask<float>& t = tasks[i];
      if (t.M > kTileTC || t.N > kTileTC || t.M < 1 || t.N < 1) check_range(nullptr, 1, "tc gemm tile shape");
      check_block(t.C, t.M, t.N, t.ldc, sizeof(float), "tc gemm C");
      for (int c = t.c_begin; c < t.c_begin + t.c_count; ++c) {
        const GemmContrib<float>& q = cons[c];
        // (the bulk copies read the 16-byte aligned supersets of the segments)
        if (q.flags & kTransA) check_block_superset(q.A, q.K, t.M, q.lda, sizeof(float), "tc gemm A^T");
        else check_block_superset(q.A, t.M, q.K, q.lda, sizeof(float), "tc gemm A");
        if (q.flags & kTransB) check_block_superset(q.B, t.N, q.K, q.ldb, sizeof(float), "tc gemm B^T");
        else check_block_superset(q.B, q.K, t.N, q.ldb, sizeof(float), "tc gemm B");
      }
    }
    return;
  }
  if (n <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<2>::kSmem);
    cudaFuncSetAttribute(k_gemm_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<3>::kSmem);
    attr = true;
  }
  ProfScope ps(P_GEMM, s);
  if (nparts == 2) k_gemm_tc<2><<<n, kTcThreads, TcCfg<2>::kSmem, s>>>(tasks, cons);
  else k_gemm_tc<3><<<n, kTcThreads, TcCfg<3>::kSmem, s>>>(tasks, cons);
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

template <typename T>
void launch_front(const FrontTask<T>* tasks, int n, DevStatus* st, int level, cudaStream_t s) {
  if (dry_run()) {
    for (int i = 0; i < n; ++i) {
      check_block(tasks[i].D, tasks[i].m, tasks[i].m, tasks[i].m, sizeof(T), "front D");
      check_block(tasks[i].Li, tasks[i].m, tasks[i].m, tasks[i].m, sizeof(T), "front Li");
    }
    return;
  }
  if (n <= 0) return;
  const size_t sm = 2 * sizeof(T) * kTile * kPitch + FrontStage<T>::bytes();
  cudaFuncSetAttribute(k_front<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ProfScope ps(P_DIAG, s);
  k_front<T><<<n, kThreads, sm, s>>>(tasks, st, level);
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
      if (t.mode == kMirror) {
        if (t.rows != t.cols) check_range(nullptr, 1, "mirror tile shape");
        check_block(t.src, t.rows, t.cols, t.lds, sizeof(S), "mirror src");
      }
    }
    return;
  }
  if (n <= 0) return;
  ProfScope ps(P_COPY, s);
  k_copy<S, D><<<n, kThreads, 0, s>>>(tasks);
}

size_t qr_smem_bytes(int m, int c, size_t es, long long cap_elems) {
  const int kmn = m < c ? m : c;
  return 8 * (size_t)(c + kmn) + 4 * (size_t)c + 16 + es * (size_t)m + 16 + es * (size_t)cap_elems + 64;
}

template <typename T>
void launch_qrcp(const QrTask<T>* tasks, int n, int* ranks, double tau, int max_m, int max_c,
                 long long cap_elems, cudaStream_t s) {
  if (dry_run()) {
    for (int i = 0; i < n; ++i) {
      const QrTask<T>& t = tasks[i];
      if (t.m > max_m || t.c > max_c) check_range(nullptr, 1, "qr size above launch bound");
      check_block(t.A, t.m, t.c, t.m, sizeof(T), "qr A");
      check_block(t.Q1, t.m, t.m < t.c ? t.m : t.c, t.m, sizeof(T), "qr Q1");
      check_range(ranks + t.slot, sizeof(int), "qr rank slot");
    }
    return;
  }
  if (n <= 0) return;
  const size_t sm = qr_smem_bytes(max_m, max_c, sizeof(T), cap_elems);
  cudaFuncSetAttribute(k_qrcp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ProfScope ps(P_QR, s);
  k_qrcp<T><<<n, kThreads, sm, s>>>(tasks, ranks, tau, cap_elems);
}

template <typename T>
static void check_gemv(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, bool trans, int nr,
                       int max_m) {
  for (int i = 0; i < n; ++i) {
    const GemvTask<T>& t = tasks[i];
    if (t.M > (trans ? kGemvColsMax : kGemvBand) || t.M < 1 || t.M > max_m) check_range(nullptr, 1, "gemv chunk shape");
    if (t.c_count < 0 || t.c_count > kGemvMaxC) check_range(nullptr, 1, "gemv contribution count");
    check_range(t.y, sizeof(T) * t.M * nr, "gemv y");
    int total = 0;
    for (int c = t.c_begin; c < t.c_begin + t.c_count; ++c) {
      const GemvContrib<T>& q = cons[c];
      if (trans) check_block(q.A, q.K, t.M, q.lda, sizeof(T), "gemvT A");
      else check_block(q.A, t.M, q.K, q.lda, sizeof(T), "gemv A");
      check_range(q.x, sizeof(T) * q.K * nr, "gemv x");
      if (q.x2) check_range(q.x2, sizeof(T) * q.K * nr, "gemv x2");
      if (q.upper && (!trans || !q.tri)) check_range(nullptr, 1, "gemv upper triangle needs op T");
      int kb, ke;
      gemv_useful(trans, q.tri, q.upper, q.K, t.M, &kb, &ke);
      total += ke - kb;
    }
    if (t.k_lo < 0 || t.k_hi > total || (t.k_lo >= t.k_hi && total > 0))
      check_range(nullptr, 1, "gemv flat range");
    if (t.nsplit > 1) {
      if (t.split < 0 || t.split >= t.nsplit) check_range(nullptr, 1, "gemv split index");
      check_range(t.part, sizeof(T) * (size_t)t.nsplit * t.M * nr, "gemv partials");
      check_range(t.cnt, sizeof(int), "gemv counter");
    } else if (t.nsplit != 1) {
      check_range(nullptr, 1, "gemv split count");
    }
  }
}

template <typename T>
static void check_warp_tasks(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, bool trans, int nr) {
  if (n <= 0) return;
  for (int i = 0; i < n; ++i)
    if (tasks[i].nsplit != 1 || (!trans && tasks[i].M > kGemvWarpRowsMax)) check_range(nullptr, 1, "warp gemv task shape");
  check_gemv(tasks, cons, n, trans, nr, trans ? kGemvColsMax : kGemvWarpRowsMax);
}

namespace {
thread_local bool t_dependent = false;

// <<<grid, kThreads>>> launch, with the programmatic-serialization attribute
// while dependent launch is on for this thread
template <typename... KArgs, typename... Args>
void launch_apply_kernel_smem(void (*kern)(KArgs...), unsigned grid, size_t smem, cudaStream_t s, Args... args) {
  if (!t_dependent) {
    kern<<<grid, kThreads, smem, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // a failed launch is reported like a <<<>>> launch: by the caller's
  // cudaGetLastError, or by the end of the stream capture it belongs to
  (void)cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
template <typename... KArgs, typename... Args>
void launch_apply_kernel(void (*kern)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
  launch_apply_kernel_smem(kern, grid, 0, s, args...);
}
}  // namespace

bool dependent_launch_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("SGF_DEPENDENT_LAUNCH");
    return !(e && e[0] == '0');
  }();
  return on;
}

void set_dependent_launch(bool on) { t_dependent = on && dependent_launch_enabled(); }

// grid: the CTA tasks, then one block per eight warp tasks
inline unsigned gemv_grid(int n, int nw) { return (unsigned)(n + (nw + kThreads / 32 - 1) / (kThreads / 32)); }

template <typename T, int NR>
static void gemv_n_mt(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, int max_m,
                      const GemvTask<T>* wt, int nw, cudaStream_t s) {
  if (max_m <= 256) launch_apply_kernel(k_gemv_n<T, NR, 8>, gemv_grid(n, nw), s, tasks, cons, n, wt, nw);
  else launch_apply_kernel(k_gemv_n<T, NR, 16>, gemv_grid(n, nw), s, tasks, cons, n, wt, nw);
}

template <typename T>
void launch_gemv_n(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, int nr, int max_m,
                   cudaStream_t s, const GemvTask<T>* wtasks, int nw) {
  if (dry_run()) {
    check_warp_tasks(wtasks, cons, nw, false, nr);
    return check_gemv(tasks, cons, n, false, nr, max_m);
  }
  if (n + nw <= 0) return;
  ProfScope ps(P_GEMV_N, s);
  switch (nr) {
    case 1: gemv_n_mt<T, 1>(tasks, cons, n, max_m, wtasks, nw, s); break;
    case 2: gemv_n_mt<T, 2>(tasks, cons, n, max_m, wtasks, nw, s); break;
    case 4: gemv_n_mt<T, 4>(tasks, cons, n, max_m, wtasks, nw, s); break;
    default: gemv_n_mt<T, 8>(tasks, cons, n, max_m, wtasks, nw, s); break;
  }
}

// the 64-wide chunks exist in single precision only (double-precision
// accumulators of 8 columns x 8 right-hand sides would not fit the registers)
template <typename T, int NR>
static void gemv_t_cw(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, int cols,
                      const GemvTask<T>* wt, int nw, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (cols > kGemvCols) {
      launch_apply_kernel(k_gemv_t<T, NR, kGemvColsMax / (kThreads / 32)>, gemv_grid(n, nw), s, tasks, cons, n, wt, nw);
      return;
    }
  }
  launch_apply_kernel(k_gemv_t<T, NR, kGemvCols / (kThreads / 32)>, gemv_grid(n, nw), s, tasks, cons, n, wt, nw);
}

template <typename T>
void launch_gemv_t(const GemvTask<T>* tasks, const GemvContrib<T>* cons, int n, int nr, int cols, cudaStream_t s,
                   const GemvTask<T>* wtasks, int nw) {
  if (dry_run()) {
    check_warp_tasks(wtasks, cons, nw, true, nr);
    return check_gemv(tasks, cons, n, true, nr, cols);
  }
  if (n + nw <= 0) return;
  ProfScope ps(P_GEMV_T, s);
  switch (nr) {
    case 1: gemv_t_cw<T, 1>(tasks, cons, n, cols, wtasks, nw, s); break;
    case 2: gemv_t_cw<T, 2>(tasks, cons, n, cols, wtasks, nw, s); break;
    case 4: gemv_t_cw<T, 4>(tasks, cons, n, cols, wtasks, nw, s); break;
    default: gemv_t_cw<T, 8>(tasks, cons, n, cols, wtasks, nw, s); break;
  }
}

template <typename T>
void launch_vgather(const T* src, const int* idx, T* dst, int n, int nr, cudaStream_t s) {
  if (dry_run()) {
    // (idx is task data in the batch, read here on the host like task lists)
    check_range(dst, sizeof(T) * (size_t)n * nr, "vgather dst");
    for (int p = 0; p < n; ++p) check_range(src + (size_t)idx[p] * nr, sizeof(T) * nr, "vgather src");
    return;
  }
  if (n <= 0) return;
  ProfScope ps(P_VECCOPY, s);
  const int64_t tot = (int64_t)n * nr;
  launch_apply_kernel(k_vgather<T>, (unsigned)((tot + kThreads - 1) / kThreads), s, src, idx, dst, n, nr);
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
  launch_apply_kernel(k_veccopy<T>, (unsigned)((n + kThreads / 32 - 1) / (kThreads / 32)), s, tasks, n, src, dst);
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

template <typename T>
void launch_assemble_q1(const double* E, const double* kref, int nx, int ny, int nz, const int64_t* map,
                        const int* ld, int64_t dgsz, T* dg, T* up, double* bsr, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz * 27;
  if (dry_run()) {
    check_range(map, 8 * n, "assemble_q1 map");
    check_range(bsr, 8 * 9 * n, "assemble_q1 bsr");
    return;
  }
  ProfScope ps(P_ASSEMBLE, s);
  k_assemble_q1<T><<<blocks_for(n), kThreads, 0, s>>>(E, kref, nx, ny, nz, map, ld, dgsz, dg, up, bsr);
}

void launch_spmv_bsr27(const double* bsr, int nx, int ny, int nz, const double* x, double* y, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz;
  if (dry_run()) return;
  prof_work(2.0 * 243 * n, (243.0 * 8 + 48) * n);
  ProfScope ps(P_SPMV, s);
  k_spmv_bsr27<<<blocks_for(n), kThreads, 0, s>>>(bsr, nx, ny, nz, x, y);
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
void launch_gather(const double* src, const int64_t* perm, T* dst, int64_t n, int nrhs, int nr,
                   cudaStream_t s) {
  if (dry_run()) {
    check_range(perm, 8 * n, "gather perm");
    check_range(dst, sizeof(T) * n * nr, "gather dst");
    return;
  }
  if (n <= 0) return;
  prof_work(0, (8.0 + (8.0 + sizeof(T)) * nrhs) * n);
  ProfScope ps(P_VEC, s);
  k_gather<T><<<blocks_for(n), kThreads, 0, s>>>(src, perm, dst, n, nrhs, nr);
}
template <typename T>
void launch_scatter(const T* src, const int64_t* perm, double* dst, int64_t n, int nrhs, int nr,
                    cudaStream_t s, int* nonfinite) {
  if (dry_run()) {
    check_range(perm, 8 * n, "scatter perm");
    check_range(src, sizeof(T) * n * nr, "scatter src");
    return;
  }
  if (n <= 0) return;
  prof_work(0, (8.0 + (8.0 + sizeof(T)) * nrhs) * n);
  ProfScope ps(P_VEC, s);
  k_scatter<T><<<blocks_for(n), kThreads, 0, s>>>(src, perm, dst, n, nrhs, nr, nonfinite);
}

void launch_dot_n(const double* a, const double* b, int64_t n, int nrhs, double* partials, double* result,
                  cudaStream_t s) {
  if (dry_run() || nrhs <= 0) return;
  prof_work(2.0 * n * nrhs, 16.0 * n * nrhs);
  ProfScope ps(P_DOT, s);
  k_dot_partial_n<<<dim3(kDotBlocks, nrhs), kThreads, 0, s>>>(a, b, n, partials);
  k_dot_final_n<<<nrhs, kThreads, 0, s>>>(partials, kDotBlocks, result);
}

void launch_axpy_n(const Coef8& a, const double* x, double* y, int64_t n, int nrhs, int mode, cudaStream_t s) {
  if (dry_run() || n <= 0 || nrhs <= 0) return;
  prof_work(2.0 * n * nrhs, 24.0 * n * nrhs);
  ProfScope ps(P_VEC, s);
  k_axpy_n<<<blocks_for(n), kThreads, 0, s>>>(a, x, y, n, nrhs, mode);
}

void launch_pcg_alpha(const double* pq, const double* rz, const Coef8& act, int nrhs, double* coef, double* flag,
                      cudaStream_t s) {
  if (dry_run() || nrhs <= 0) return;
  ProfScope ps(P_VEC, s);
  k_pcg_alpha<<<1, 32, 0, s>>>(pq, rz, act, nrhs, coef, flag);
}

void launch_pcg_xr(const double* coef, const double* p, const double* q, double* x, double* r, double* ro,
                   int64_t n, int nrhs, cudaStream_t s) {
  if (dry_run() || n <= 0 || nrhs <= 0) return;
  prof_work(4.0 * n * nrhs, (ro ? 56.0 : 48.0) * n * nrhs);
  ProfScope ps(P_VEC, s);
  k_pcg_xr<<<blocks_for(n), kThreads, 0, s>>>(coef, p, q, x, r, ro, n, nrhs);
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
  template void launch_front<T>(const FrontTask<T>*, int, DevStatus*, int, cudaStream_t);       \
  template void launch_copy<T, T>(const CopyTask<T, T>*, int, cudaStream_t);                    \
  template void launch_qrcp<T>(const QrTask<T>*, int, int*, double, int, int, long long,        \
                               cudaStream_t);                                                    \
  template void launch_gemv_n<T>(const GemvTask<T>*, const GemvContrib<T>*, int, int, int,      \
                                 cudaStream_t, const GemvTask<T>*, int);                         \
  template void launch_gemv_t<T>(const GemvTask<T>*, const GemvContrib<T>*, int, int, int,      \
                                 cudaStream_t, const GemvTask<T>*, int);                         \
  template void launch_veccopy<T>(const VecCopyTask*, int, const T*, T*, cudaStream_t);         \
  template void launch_vgather<T>(const T*, const int*, T*, int, int, cudaStream_t);           \
  template void launch_assemble_scalar<T>(const double*, int, int, int, unsigned, double,       \
                                          const int64_t*, int64_t, T*, T*, double*, double*,    \
                                          double*, double*, cudaStream_t);                       \
  template void launch_assemble_q1<T>(const double*, const double*, int, int, int,              \
                                      const int64_t*, const int*, int64_t, T*, T*, double*,      \
                                      cudaStream_t);                                             \
  template void launch_gather<T>(const double*, const int64_t*, T*, int64_t, int, int,          \
                                 cudaStream_t);                                                  \
  template void launch_scatter<T>(const T*, const int64_t*, double*, int64_t, int, int,         \
                                  cudaStream_t, int*);

SGF_INST(double)
SGF_INST(float)
template void launch_copy<double, float>(const CopyTask<double, float>*, int, cudaStream_t);

}  // namespace sgf
