// Internal data structures of the SGF library: the symbolic plan built by
// sgf_analyze on the host, per-level block layouts, and the task descriptors
// the batched device kernels consume.
#pragma once

#include <cstddef>
#include <array>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sgf.h"

#if defined(__CUDACC__)
#define SGF_HD __host__ __device__
#else
#define SGF_HD
#endif

namespace sgf {

// ---------------------------------------------------------------------------
// Symbolic plan (host)
// ---------------------------------------------------------------------------

// One level of the nested-dissection hierarchy (Sec. 5.1, Defs. 2.1-2.4).
// Node order: interiors first, then separators, each sorted by the cell code
// tuple (z, y, x); per axis code 2k = interval k, 2k+1 = separator k.
struct LevelSym {
  int t = 0;          // 1-based level
  int d = 0;          // cut spacing b * 2^(t-1)
  bool top = false;   // the single-node top level
  int nnodes = 0;
  std::vector<int> code;       // 3 per node: z, y, x
  std::vector<char> interior;  // per node
  std::vector<int> cell_dim;   // per node
  std::vector<int> box;        // 6 per node: lo x,y,z then hi x,y,z
  std::vector<int> act;        // per node: basis columns not identically zero
                               // (monomials free of the cell's flat axes)
  std::vector<char> eligible;  // per node: selected for compression
  std::vector<int> child_ptr;  // nnodes + 1 (levels > 1)
  std::vector<int> child_idx;  // previous-level node ids, canonical order
  std::vector<int> pairs;      // pre-elimination block pairs (u < v), 2 ints each
  std::vector<int> post;       // separator pairs after elimination (u < v)
  std::vector<int> pt_ptr, pt_idx;  // level 1: natural point ids per node
  std::vector<double> reexp;   // levels > 1: pi x pi (col-major) per child,
                               // indexed like child_idx (Sec. 4.4 merge)
};

struct Plan {
  sgf_grid grid{};
  int stencil = 0;
  sgf_opts opts{};
  int nx = 1, ny = 1, nz = 1;
  int64_t npts = 0, n = 0;
  int dof = 1;
  int pi = 1;                      // basis columns
  double tau = 1e-12;
  double nu = 0.3;                 // Poisson ratio (Q1 elasticity)
  std::vector<double> kref;        // Q1 element stiffness for E = 1 (24 x 24, row-major)
  std::vector<LevelSym> lev;
  // level-1 basis rows Phi (m x pi, col-major) per node, concatenated
  std::vector<double> phi1;
  std::vector<int64_t> phi1_off;
  // structural upper bounds of node sizes per level (for the footprint)
  std::vector<std::vector<int>> mcap;
  // level-1 assembly: per point 7 destinations (x-, x+, y-, y+, z-, z+, diag)
  // in the concatenation [diagonal blocks | upper panels] of the level-1
  // layout (-1 = not stored) - for Q1 elasticity 27 per point, the (0, 0)
  // entry of each 3x3 neighbour block - and the natural DOF of each level-1
  // vector slot
  std::vector<int64_t> asm_map, perm1;
  std::vector<int> asm_ld;         // Q1: level-1 node size of every point
  // launch shapes (sgf_tuning; see sgf_plan_set_tuning)
  sgf_tuning tune{4096, 32768, 512, 1, 32, 64};

  // device copies of the plan's constant data, built on first use
  struct DevCache {
    int device = -1;
    int64_t* map = nullptr;
    int64_t* perm = nullptr;
    int* ld = nullptr;
    double* kref = nullptr;
    void* phi1[2] = {nullptr, nullptr};          // [double, float]
    std::vector<void*> reexp[2];                 // per level, [double, float]
  };
  mutable std::mutex cache_mu;
  mutable DevCache cache;
  ~Plan();
};

// Per-level dense block layout for given node sizes.  Every node owns a full
// m x m diagonal block and an "upper panel" holding its blocks with higher
// numbered neighbours, side by side (column-major, leading dimension m):
// interiors hold their separator blocks (pre-elimination pattern), separators
// hold their separator blocks of the post-elimination pattern (fill included).
struct LevelLayout {
  std::vector<int> m;
  std::vector<int64_t> dg_off;   // diagonal block offset (elements)
  int64_t dg_size = 0;
  std::vector<int> up_ptr;       // nnodes + 1 into up_nb / up_col
  std::vector<int> up_nb;        // neighbour node ids (> owner), ascending
  std::vector<int> up_col;       // column offset of each neighbour block
  std::vector<int64_t> up_off;   // panel start (elements)
  std::vector<int> up_w;         // panel width (columns)
  int64_t up_size = 0;
  std::vector<int64_t> vec_off;  // offset of each node in a level vector
  int64_t vec_size = 0;

  // column offset of block (u, v), u < v, inside u's panel; -1 if absent
  int col_of(int u, int v) const;
};

void build_layout(const LevelSym& L, const std::vector<int>& m, LevelLayout& out);

int analyze(const sgf_grid* g, int stencil, const sgf_opts* o, Plan& plan, std::string& err);

// ---------------------------------------------------------------------------
// Device task descriptors (one CTA per task unless stated)
// ---------------------------------------------------------------------------
constexpr int kTile = 64;
constexpr int kTileTC = 128;   // rows and columns of a tensor-core GEMM tile

template <typename T>
struct GemmTask {        // C[M x N] = beta*C + alpha * sum_c op(A_c) op(B_c)
  T* C;
  int ldc, M, N;         // M, N <= kTile (kTileTC on the tensor-core path)
  int c_begin, c_count;  // contribution range
  T alpha;
  int beta;              // 0 or 1
};

enum : int { kTransA = 1, kTransB = 2 };

template <typename T>
struct GemmContrib {
  const T* A;            // op(A) is M x K
  const T* B;            // op(B) is K x N
  int lda, ldb, K, flags;
};

// kMirror: in place on a square diagonal tile, upper part <- transpose of
// the lower part (src == dst)
enum : int { kCopy = 0, kCopyT = 1, kZero = 2, kIdentity = 3, kCopyLower = 4, kMirror = 5 };

template <typename S, typename D>
struct CopyTask {        // dst[rows x cols] <- mode(src), rows, cols <= kTile
  const S* src;
  D* dst;
  int lds, ldd, rows, cols, mode, pad;
};

template <typename T>
struct DiagTask {        // in-place Cholesky of an n x n tile (n <= kTile) and its inverse
  T* A;                  // tile, ld = lda; gets L (strict upper part zeroed)
  T* Li;                 // gets L^{-1}, ld = ldli
  int lda, ldli, n, node;
};

template <typename T>
struct FrontTask {       // blocked Cholesky of D (m x m, ld m) and L^{-1} into Li (zero on entry)
  T* D;
  T* Li;
  int m, node;
};

template <typename T>
struct QrTask {          // column-pivoted Householder QR of A (m x c, ld = m)
  T* A;                  // in/out workspace
  T* Q1;                 // out: m x r, ld = m (r = kept rank)
  int m, c, node, slot;  // slot: index of the rank output
};

// Batched GEMV.  A chunk is y[M] = beta*y + sum_c alpha_c op(A_c) (x_c - x2_c)
// over its contributions c; op N chunks are bands of <= kGemvBand rows, op T
// chunks hold 32 or 64 (kGemvColsMax, a tuning choice in single precision)
// columns of A; one CTA works on one task.  The
// contributions' useful indices (columns for op N, rows for op T; see
// gemv_useful) are concatenated into one flat range, and a chunk may be split
// into nsplit pieces of that range, each a task.  A split task writes its
// partial sums to part[split]; the last of the chunk's tasks to arrive (an
// atomic counter) adds the partials in split order and writes y, so the
// result does not depend on scheduling.
constexpr int kGemvBand = 512;
constexpr int kGemvCols = 32;      // op T chunk width in double precision and by default
constexpr int kGemvColsMax = 64;
constexpr int kGemvMaxC = 32;   // contributions per task

template <typename T>
struct GemvTask {
  T* y;
  T* part;               // nsplit > 1: [nsplit][M][nr] partial sums of the chunk
  int* cnt;              // nsplit > 1: arrival counter, zero between launches
  int M, c_begin, c_count, beta;
  int k_lo, k_hi;        // flat range of this task over contributions c_begin..
  int split, nsplit;
};

template <typename T>
struct GemvContrib {
  const T* A;            // column-major, ld = lda; op(A) is M x K
  const T* x;            // K
  const T* x2;           // K or nullptr (subtracted from x)
  int lda, K;
  int tri;               // 0: dense A; t > 0: A is (part of) a triangular matrix
                         // whose first row (op N) / column (op T) in this chunk
                         // has absolute index t - 1: the zero half is skipped
  int upper;             // tri, op T only: upper triangle (rows <= column) instead
                         // of lower (rows >= column)
  T alpha;
};

// Useful index range [kb, ke) of a contribution to a chunk of M outputs: all K
// for a dense block; for a lower-triangular one the columns j <= last row (op
// N) or the rows i >= first column (op T); for an upper-triangular one (op T)
// the rows i <= last column.
bool tuning_valid(const sgf_tuning& t);

SGF_HD inline void gemv_useful(bool trans, int tri, int upper, int K, int M, int* kb, int* ke) {
  if (!tri) {
    *kb = 0;
    *ke = K;
  } else if (trans && !upper) {
    *kb = tri - 1 < K ? tri - 1 : K;
    *ke = K;
  } else {
    *kb = 0;
    *ke = tri - 1 + M < K ? tri - 1 + M : K;
  }
}

struct VecCopyTask {     // dst[i] = src[i] for i < len (level-vector gathers)
  int64_t src, dst;
  int len, pad;
};

}  // namespace sgf
