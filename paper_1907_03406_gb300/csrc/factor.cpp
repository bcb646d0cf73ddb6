// Host driver of the SGF numeric factorization (Algorithm 4.1) and of the
// apply programs of Sec. 4.7.
//
// Per level, with the node sizes known (level 1 from the grid, higher levels
// from the ranks read back after the previous level):
//  1. elimination of the interiors (Sec. 4.1): a batched blocked sweep over
//     the fronts [A_II | A_IS | I] (diagonal tile Cholesky + inverse, panel,
//     trailing update) gives L_I, W_IS = L_I^{-1} A_IS and L_I^{-1}; then the
//     Schur products A_SS' -= W_IS^T W_IS' are accumulated owner-computes,
//     every target tile summing its interiors in index order;
//  2. compression of the selected separators (Sec. 3.2, Sec. 4.2), all from
//     the post-elimination matrix (compressions inside a level commute: the
//     filtered interaction matrix of a node only sees its neighbours through
//     M^_BN Phi_N, which earlier compressions leave unchanged because
//     L_N^T Phi_N lies in the range of Q1_N): the same blocked sweep on
//     [A_BB | A_B,nbrs | I] gives L_B, M^_BN, L_B^{-1}; the filtered
//     interaction matrix N = [L_B^T Phi_B | M^_BN Phi_N ...] (Eq.
//     (N-definition)) goes through column-pivoted QR (Eq. (QR)); rank
//     r = #{|R_kk| > tau |R_11|}; the node is compressed when r < m;
//  3. surviving blocks (Eq. (M')): Q1_B^T L_B^{-1} A_BN L_N^{-T} Q1_N when both
//     ends are compressed (one end: drop the other factor), identity on the
//     compressed diagonal, Phi_B <- Q1_B^T L_B^T Phi_B (Eq. (phi-update));
//  4. merge into the next level (Sec. 4.3-4.4): parents gather children's
//     kept variables, blocks and re-expanded Phi.
// The top node gets a dense Cholesky (Sec. 4.5).
//
// The steps of Sec. 4.7, written with the triangular factors,
//  forward:  y_I = L_I^{-1} b_I;  b_S -= W_IS^T y_I;  c_B = L_B^{-1} b_B;
//            kept_B = Q1_B^T c_B;  gather to the next level
//  top:      x = L^{-T} L^{-1} b
//  backward: x_B = L_B^{-T} (c_B + Q1_B (x_kept - kept_B));
//            x_I = L_I^{-T} (y_I - sum_S W_IS x_S)
// are applied through dense blocks formed at the end of each level, Z =
// L_I^{-T} W_IS = A_II^{-1} A_IS, A_II^{-1}, Qf = L_B^{-T} Q1_B, B^{-1} =
// L_B^{-T} L_B^{-1} and A_top^{-1}, each step one batched matrix-vector
// product of dense blocks (the same bytes, no triangular phases):
//  forward:  b_S -= Z^T b_I;  kept_B = Qf^T b_B;  gather to the next level
//  top:      x = A_top^{-1} b
//  backward: x_B = B^{-1} b_B + Qf (x_kept - kept_B);
//            x_I = A_II^{-1} b_I - sum_S Z x_S
// The Q2 part of a compressed node is its decoupled identity block (Eq. (M')):
// its forward value Q2^T c_B comes back unchanged, which is what
// c_B - Q1 Q1^T c_B restores.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <type_traits>

#include "devmem.h"
#include "factor.h"
#include "prof.h"

namespace sgf {

namespace {
// Host staging buffers and pinned upload buffers keep their capacity across
// factorizations on the same thread (page-locking megabytes per
// factorization costs milliseconds).  A pinned buffer is returned only after
// the last copy from it has completed.
std::vector<std::vector<char>>& host_pool() {
  thread_local std::vector<std::vector<char>> p;
  return p;
}
// keep at most 16 buffers, the largest ones
void host_pool_put(std::vector<char>&& v) {
  if (v.capacity() == 0) return;
  v.clear();
  auto& p = host_pool();
  if (p.size() < 16) {
    p.push_back(std::move(v));
    return;
  }
  size_t k = 0;
  for (size_t i = 1; i < p.size(); ++i)
    if (p[i].capacity() < p[k].capacity()) k = i;
  if (p[k].capacity() < v.capacity()) p[k] = std::move(v);
}
struct PinnedPool {
  std::vector<std::pair<char*, size_t>> bufs;
  ~PinnedPool() {
    for (auto& b : bufs) cudaFreeHost(b.first);
  }
};
PinnedPool& pinned_pool() {
  thread_local PinnedPool p;
  return p;
}
}  // namespace

void Batch::run(cudaStream_t s) {
  char* d = nullptr;
  if (!host.empty()) {
    if (dry_run()) {
      d = host.data();
    } else {
      // pinned staging ring: a buffer is refilled only after the copy that
      // last read it has completed
      const int i = cur;
      cur = (cur + 1) % kRing;
      if (ev[i]) SGF_CK(cudaEventSynchronize(ev[i]));
      else SGF_CK(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
      if (!pin[i] && !pinned_pool().bufs.empty()) {   // reuse a pooled buffer
        pin[i] = pinned_pool().bufs.back().first;
        pincap[i] = pinned_pool().bufs.back().second;
        pinned_pool().bufs.pop_back();
      }
      if (pincap[i] < host.size()) {
        if (pin[i]) cudaFreeHost(pin[i]);
        pincap[i] = std::max(host.size() + host.size() / 2, size_t(1) << 20);
        SGF_CK(cudaHostAlloc((void**)&pin[i], pincap[i], cudaHostAllocDefault));
      }
      std::memcpy(pin[i], host.data(), host.size());
      d = (char*)dev_malloc_async(host.size(), s);
      SGF_CK(cudaMemcpyAsync(d, pin[i], host.size(), cudaMemcpyHostToDevice, s));
      SGF_CK(cudaEventRecord(ev[i], s));
    }
  }
  for (auto& f : launches) f(d);
  if (!dry_run()) {
    SGF_CK(cudaGetLastError());
    if (d) dev_free_async(d, s);   // stream ordered, after the launches above
  }
  host.clear();
  launches.clear();
}


Batch::Batch() {}

void Batch::grow(size_t want) {
  auto& p = host_pool();
  int best = -1;   // the smallest pooled buffer that is large enough
  for (int i = 0; i < (int)p.size(); ++i)
    if (p[i].capacity() >= want && (best < 0 || p[i].capacity() < p[best].capacity())) best = i;
  std::vector<char> v;
  if (best >= 0) {
    v.swap(p[best]);
    p.erase(p.begin() + best);
  } else {
    v.reserve(want);
  }
  v.assign(host.begin(), host.end());
  host.swap(v);
  host_pool_put(std::move(v));
}

Batch::~Batch() {
  host_pool_put(std::move(host));
  for (int i = 0; i < kRing; ++i) {
    if (ev[i]) {
      cudaEventSynchronize(ev[i]);
      cudaEventDestroy(ev[i]);
    }
    if (pin[i]) {
      auto& q = pinned_pool().bufs;
      if (q.size() < 2 * kRing) q.push_back({pin[i], pincap[i]});
      else cudaFreeHost(pin[i]);
    }
  }
}

void Batch::upload_persistent(cudaStream_t s) {
  if (host.empty()) return;
  if (dry_run()) {
    keep_host.swap(host);
    dev = keep_host.data();
    return;
  }
  dev = (char*)dev_malloc_async(host.size(), s);
  cap = host.size();
  dev_h2d(dev, host.data(), host.size(), s);
  dev_sync(s);
  host.clear();
}

void Batch::release(cudaStream_t s) {
  if (dev && !dry_run()) dev_free_async(dev, s);
  dev = nullptr;
  cap = 0;
}

namespace {

// apply programs replayed as CUDA graphs unless SGF_APPLY_GRAPH=0
bool apply_graph() {
  static const bool on = [] {
    const char* e = std::getenv("SGF_APPLY_GRAPH");
    return !(e && e[0] == '0');
  }();
  return on;
}

// Launch shapes of the factorization or program build running on this thread
// (the plan's sgf_tuning), set for its duration by TuneScope.
thread_local const sgf_tuning* t_tune = nullptr;
struct TuneScope {
  const sgf_tuning* prev;
  explicit TuneScope(const sgf_tuning* t) : prev(t_tune) { t_tune = t; }
  ~TuneScope() { t_tune = prev; }
};
inline const sgf_tuning& active_tuning() {
  static const sgf_tuning def{4096, 32768, 512, 1, 32, 64};
  return t_tune ? *t_tune : def;
}

// Vectors handed out with the capacity they reached in earlier use on this
// thread (task lists are rebuilt for every factorization; growing them from
// empty each time costs reallocation copies).
template <class V>
struct VecPool {
  static std::vector<V>& pool() {
    thread_local std::vector<V> p;
    return p;
  }
  static V get() {
    auto& p = pool();
    if (p.empty()) return V();
    V v = std::move(p.back());
    p.pop_back();
    v.clear();
    return v;
  }
  static void put(V&& v) {
    auto& p = pool();
    if (p.size() < 16) p.push_back(std::move(v));
  }
};

template <class V>
struct Pooled {
  V v = VecPool<V>::get();
  Pooled() = default;
  Pooled(const Pooled&) = delete;
  Pooled& operator=(const Pooled&) = delete;
  ~Pooled() { VecPool<V>::put(std::move(v)); }
};

template <typename T>
struct Spec {
  const T* A;
  int lda;
  bool ta;
  const T* B;
  int ldb;
  bool tb;
  int K;
};

template <typename T>
struct GemmList {
  Pooled<std::vector<GemmTask<T>>> tp, sp;
  Pooled<std::vector<GemmContrib<T>>> cp;
  std::vector<GemmTask<T>>& t = tp.v;    // tensor-core tiles (kTileTC x kTileTC)
  std::vector<GemmTask<T>>& ts = sp.v;   // CUDA-core tiles (kTile x kTile)
  std::vector<GemmContrib<T>>& c = cp.v;
  // FP32 products of blocks with both dimensions >= tc_min_dim go to the
  // tensor cores as split TF32 products (tensor_cores: 2 = six products,
  // FP32-accurate; 1 = three, the 3xTF32 scheme); the rest, and all of FP64,
  // to the CUDA cores
  const int tcmode = std::is_same<T, float>::value && gemm_tc_enabled() ? active_tuning().tensor_cores : 0;
  const int tcmin = active_tuning().tc_min_dim;
  bool use_tc(int M, int N) const { return tcmode != 0 && M >= tcmin && N >= tcmin; }
  void add(T* C, int ldc, int M, int N, T alpha, int beta, std::initializer_list<Spec<T>> specs) {
    add_range(C, ldc, M, N, alpha, beta, specs.begin(), specs.end());
  }
  void add(T* C, int ldc, int M, int N, T alpha, int beta, const std::vector<Spec<T>>& specs) {
    add_range(C, ldc, M, N, alpha, beta, specs.data(), specs.data() + specs.size());
  }
  void add_range(T* C, int ldc, int M, int N, T alpha, int beta, const Spec<T>* sb, const Spec<T>* se) {
    if (M <= 0 || N <= 0) return;
    const bool tc = use_tc(M, N);
    const int tm = tc ? kTileTC : kTile, tn = tc ? kTileTC : kTile;
    std::vector<GemmTask<T>>& dst = tc ? t : ts;
    for (int j0 = 0; j0 < N; j0 += tn)
      for (int i0 = 0; i0 < M; i0 += tm) {
        GemmTask<T> g;
        g.C = C + i0 + (size_t)j0 * ldc;
        g.ldc = ldc;
        g.M = std::min(tm, M - i0);
        g.N = std::min(tn, N - j0);
        g.c_begin = (int)c.size();
        g.alpha = alpha;
        g.beta = beta;
        int cnt = 0;
        for (const Spec<T>* sp = sb; sp != se; ++sp) {
          const Spec<T>& s = *sp;
          if (s.K <= 0) continue;
          GemmContrib<T> q;
          q.A = s.ta ? s.A + (size_t)i0 * s.lda : s.A + i0;
          q.B = s.tb ? s.B + j0 : s.B + (size_t)j0 * s.ldb;
          q.lda = s.lda;
          q.ldb = s.ldb;
          q.K = s.K;
          q.flags = (s.ta ? kTransA : 0) | (s.tb ? kTransB : 0);
          c.push_back(q);
          ++cnt;
        }
        g.c_count = cnt;
        dst.push_back(g);
      }
  }
  // tasks of another list, after this list's (contribution indices shifted)
  void append(const GemmList& o) {
    const int base = (int)c.size();
    t.reserve(t.size() + o.t.size());
    for (GemmTask<T> g : o.t) {
      g.c_begin += base;
      t.push_back(g);
    }
    ts.reserve(ts.size() + o.ts.size());
    for (GemmTask<T> g : o.ts) {
      g.c_begin += base;
      ts.push_back(g);
    }
    c.insert(c.end(), o.c.begin(), o.c.end());
  }
  // C[M x N] = Li B with Li lower triangular (M x M): a row band starting at
  // i0 needs only the first min(M, i0 + band) rows of B
  void add_lowtri(T* C, int ldc, int M, int N, const T* Li, int ldli, const T* B, int ldb) {
    const int tm = use_tc(M, N) ? kTileTC : kTile;
    for (int i0 = 0; i0 < M; i0 += tm) {
      const int K = std::min(M, i0 + tm);
      add(C + i0, ldc, std::min(tm, M - i0), N, T(1), 0, {{Li + i0, ldli, false, B, ldb, false, K}});
    }
  }
  // C = Li^T Li (M x M, symmetric) with Li lower triangular: for each row
  // band only the column tiles up to and including the diagonal (its lower
  // part; the caller mirrors the upper triangle from it)
  void add_lowtri_tt_lower(T* C, int ldc, int M, const T* Li, int ldli) {
    const int tm = use_tc(M, M) ? kTileTC : kTile;
    for (int i0 = 0; i0 < M; i0 += tm)
      add(C + i0, ldc, std::min(tm, M - i0), std::min(M, i0 + tm), T(1), 0,
          {{Li + i0 + (size_t)i0 * ldli, ldli, true, Li + i0, ldli, false, M - i0}});
  }
  // C[M x N] = Li^T B with Li lower triangular (M x M): the row band starting
  // at i0 needs only rows i0.. of B (column i0 + r of Li is zero above row
  // i0 + r)
  void add_lowtri_t(T* C, int ldc, int M, int N, const T* Li, int ldli, const T* B, int ldb) {
    const int tm = use_tc(M, N) ? kTileTC : kTile;
    for (int i0 = 0; i0 < M; i0 += tm)
      add(C + i0, ldc, std::min(tm, M - i0), N, T(1), 0,
          {{Li + i0 + (size_t)i0 * ldli, ldli, true, B + i0, ldb, false, M - i0}});
  }
  static void work(const std::vector<GemmTask<T>>& v, const std::vector<GemmContrib<T>>& c, double& fl, double& by) {
    fl = by = 0;
    for (const auto& g : v) {
      for (int k = g.c_begin; k < g.c_begin + g.c_count; ++k) {
        fl += 2.0 * g.M * g.N * c[k].K;
        by += (double)sizeof(T) * ((double)g.M * c[k].K + (double)c[k].K * g.N);
      }
      by += (double)sizeof(T) * g.M * g.N * (g.beta ? 2 : 1);
    }
  }
  void emit(Batch& b, cudaStream_t s) {
    if (t.empty() && ts.empty()) return;
    const size_t oc = b.push(c);
    if (!t.empty()) {
      double fl, by;
      work(t, c, fl, by);
      const size_t ot = b.push(t);
      const int n = (int)t.size(), parts = tcmode == 1 ? 2 : 3;
      // launch-log description: tiles, full 128 x 128 tiles, the K sums
      std::shared_ptr<std::string> note;
      if (prof_logging()) {
        double ksum = 0, kmax = 0, full = 0, cmax = 0;
        for (const auto& g : t) {
          double k = 0;
          for (int q = g.c_begin; q < g.c_begin + g.c_count; ++q) k += c[q].K;
          ksum += k;
          kmax = std::max(kmax, k);
          cmax = std::max(cmax, (double)g.c_count);
          full += g.M == kTileTC && g.N == kTileTC;
        }
        char buf[192];
        std::snprintf(buf, sizeof buf, "tc tiles %d full %.0f kavg %.0f kmax %.0f cmax %.0f", n, full, ksum / n, kmax,
                      cmax);
        note = std::make_shared<std::string>(buf);
      }
      b.launches.push_back([=](const char* d) {
        if (note) prof_note(note->c_str());
        prof_work(fl, by);
        if constexpr (std::is_same<T, float>::value)
          launch_gemm_tc((const GemmTask<float>*)(d + ot), (const GemmContrib<float>*)(d + oc), n, parts, s);
      });
    }
    if (!ts.empty()) {
      double fl, by;
      work(ts, c, fl, by);
      const size_t ot = b.push(ts);
      const int n = (int)ts.size();
      // launch-log description: tiles, their mean output shape and K
      std::shared_ptr<std::string> note;
      if (prof_logging()) {
        double sm = 0, sn = 0, sk = 0;
        for (const auto& g : ts) {
          sm += g.M;
          sn += g.N;
          for (int q = g.c_begin; q < g.c_begin + g.c_count; ++q) sk += c[q].K;
        }
        char buf[160];
        std::snprintf(buf, sizeof buf, "simt tiles %d mavg %.1f navg %.1f kavg %.0f", n, sm / n, sn / n, sk / n);
        note = std::make_shared<std::string>(buf);
      }
      b.launches.push_back([=](const char* d) {
        if (note) prof_note(note->c_str());
        prof_work(fl, by);
        launch_gemm<T>((const GemmTask<T>*)(d + ot), (const GemmContrib<T>*)(d + oc), n, s);
      });
    }
    t.clear();
    ts.clear();
    c.clear();
  }
};

template <typename S, typename D>
struct CopyList {
  Pooled<std::vector<CopyTask<S, D>>> tp;
  std::vector<CopyTask<S, D>>& t = tp.v;
  // dst (rows x cols, ld ldd) <- mode(src); src is rows x cols (cols x rows for kCopyT)
  void add(const S* src, int lds, D* dst, int ldd, int rows, int cols, int mode) {
    for (int j0 = 0; j0 < cols; j0 += kTile)
      for (int i0 = 0; i0 < rows; i0 += kTile) {
        CopyTask<S, D> k;
        k.dst = dst + i0 + (size_t)j0 * ldd;
        k.ldd = ldd;
        k.rows = std::min(kTile, rows - i0);
        k.cols = std::min(kTile, cols - j0);
        k.lds = lds;
        int md = mode;
        if (mode == kIdentity) md = (i0 == j0) ? kIdentity : kZero;
        if (mode == kCopyLower) md = i0 > j0 ? kCopy : (i0 == j0 ? kCopyLower : kZero);
        k.mode = md;
        k.src = src ? (md == kCopyT ? src + j0 + (size_t)i0 * lds : src + i0 + (size_t)j0 * lds) : nullptr;
        k.pad = 0;
        t.push_back(k);
      }
  }
  void append(const CopyList& o) { t.insert(t.end(), o.t.begin(), o.t.end()); }
  void emit(Batch& b, cudaStream_t s) {
    if (t.empty()) return;
    const size_t ot = b.push(t);
    const int n = (int)t.size();
    b.launches.push_back([=](const char* d) { launch_copy<S, D>((const CopyTask<S, D>*)(d + ot), n, s); });
    t.clear();
  }
};

// Upper triangle of an m x m block (leading dimension ld, m by default) <-
// the transpose of its lower triangle: makes the symmetric inverses the
// apply reads exactly symmetric after only their lower part was formed.
template <typename T>
void add_mirror(CopyList<T, T>& cl, T* Li, int m, int ld = 0) {
  if (ld <= 0) ld = m;
  for (int j0 = 0; j0 < m; j0 += kTile)
    for (int i0 = 0; i0 <= j0; i0 += kTile) {
      const int ni = std::min(kTile, m - i0), nj = std::min(kTile, m - j0);
      if (i0 == j0) cl.add(Li + i0 + (size_t)i0 * ld, ld, Li + i0 + (size_t)i0 * ld, ld, ni, ni, kMirror);
      else cl.add(Li + j0 + (size_t)i0 * ld, ld, Li + i0 + (size_t)j0 * ld, ld, ni, nj, kCopyT);
    }
}

template <typename T>
struct Front {
  T* D;   // m x m, ld m (lower part used)
  int m;
  T* P;   // m x s panel, ld m
  int s;
  T* Li;  // m x m, ld m, zero on entry
  int node;
};

// Blocked right-looking Cholesky of D with the triangular solves of the panel
// and of the identity (giving L^{-1}), batched over all fronts.
template <typename T>
void run_fronts(const std::vector<Front<T>>& Fall, Batch& b, cudaStream_t s, DevStatus* st, int level) {
  // Small fronts without a panel: one CTA does the whole sweep.  Beyond
  // front_small the tile sweep spread over many CTAs wins (one CTA pays a
  // memory latency per tile product), and so it does for fronts above
  // kFrontTiny when the batch holds too few of them to occupy every SM.
  const int small_max = std::is_same<T, float>::value ? active_tuning().front_small : front_small<T>();
  int nfit = 0;
  for (const auto& f : Fall)
    if (f.s == 0 && f.m <= small_max) ++nfit;
  const int cut = nfit >= kFrontBatchMin ? small_max : std::min(kFrontTiny, small_max);
  std::vector<FrontTask<T>> small;
  std::vector<Front<T>> F;
  for (const auto& f : Fall) {
    if (f.s == 0 && f.m <= cut) small.push_back({f.D, f.Li, f.m, f.node});
    else F.push_back(f);
  }
  if (!small.empty()) {
    const size_t of = b.push(small);
    const int nf = (int)small.size();
    double fl = 0;
    for (const auto& f : small) fl += 2.0 * (2.0 / 3.0) * f.m * (double)f.m * f.m;
    b.launches.push_back([=](const char* d) {
      prof_work(fl, 0);
      launch_front<T>((const FrontTask<T>*)(d + of), nf, st, level, s);
    });
  }
  int kmax = 0;
  for (const auto& f : F) kmax = std::max(kmax, (f.m + kTile - 1) / kTile);
  for (int k = 0; k < kmax; ++k) {
    std::vector<DiagTask<T>> dt;
    GemmList<T> panel, update;
    for (const auto& f : F) {
      const int m = f.m, nt = (m + kTile - 1) / kTile;
      if (k >= nt) continue;
      const int r0 = k * kTile, nk = std::min(kTile, m - r0), r1 = r0 + nk;
      T* Dkk = f.D + r0 + (size_t)r0 * m;
      T* Likk = f.Li + r0 + (size_t)r0 * m;
      dt.push_back({Dkk, Likk, m, m, nk, f.node});
      // panel: L_ik = A_ik L_kk^{-T} (i > k); X_k = L_kk^{-1} B_k for the RHS
      for (int ri = r1; ri < m; ri += kTile) {
        const int ni = std::min(kTile, m - ri);
        T* C = f.D + ri + (size_t)r0 * m;
        panel.add(C, m, ni, nk, T(1), 0, {{C, m, false, Likk, m, true, nk}});
      }
      if (f.s > 0) panel.add(f.P + r0, m, nk, f.s, T(1), 0, {{Likk, m, false, f.P + r0, m, false, nk}});
      if (r0 > 0) panel.add(f.Li + r0, m, nk, r0, T(1), 0, {{Likk, m, false, f.Li + r0, m, false, nk}});
      // trailing update
      if (r1 < m) {
        const T* Lcol = f.D + r1 + (size_t)r0 * m;  // rows r1.., the k-th tile column
        for (int rj = r1; rj < m; rj += kTile) {
          const int nj = std::min(kTile, m - rj);
          update.add(f.D + rj + (size_t)rj * m, m, m - rj, nj, T(-1), 1,
                     {{f.D + rj + (size_t)r0 * m, m, false, f.D + rj + (size_t)r0 * m, m, true, nk}});
        }
        if (f.s > 0) update.add(f.P + r1, m, m - r1, f.s, T(-1), 1, {{Lcol, m, false, f.P + r0, m, false, nk}});
        update.add(f.Li + r1, m, m - r1, r1, T(-1), 1, {{Lcol, m, false, f.Li + r0, m, false, nk}});
      }
    }
    if (!dt.empty()) {
      const size_t od = b.push(dt);
      const int nd = (int)dt.size();
      b.launches.push_back([=](const char* d) { launch_diag<T>((const DiagTask<T>*)(d + od), nd, st, level, s); });
    }
    panel.emit(b, s);
    update.emit(b, s);
  }
}

template <typename T>
T* dalloc(std::vector<void*>& keep, size_t count, cudaStream_t s, bool zero = true) {
  if (count == 0) count = 1;
  T* p = (T*)dev_malloc_async(count * sizeof(T), s);
  keep.push_back(p);
  if (zero) dev_memset(p, 0, count * sizeof(T), s);
  return p;
}

template <typename T>
T* walloc(std::vector<void*>& work, size_t count, cudaStream_t s, bool zero = true) {
  if (count == 0) count = 1;
  T* p = (T*)dev_malloc_async(count * sizeof(T), s);
  work.push_back(p);
  if (zero) dev_memset(p, 0, count * sizeof(T), s);
  return p;
}

template <typename T>
struct InteriorRec {
  int node, m, s;
  T *L, *Li, *W;   // Li: only while the level is factored
  // for the apply: Z = L^{-T} W = A_II^{-1} A_IS (m x s) and its transpose
  // Zt (s x m), and Ai = L^{-T} L^{-1} = A_II^{-1} (m x m), all column-major
  // with leading dimensions ldm = pad(m), lds = pad(s) (columns start on a
  // 32-byte sector)
  T *Z, *Zt, *Ai;
  int ldm, lds;
  std::vector<std::pair<int, int>> nb;  // (separator, column offset in W)
};

template <typename T>
struct SepRec {
  int node, m, k;   // k = kept size
  bool comp;
  int64_t dst;      // offset of the kept part in the next level vector
  T *L, *Li, *Q1;   // compressed only
  // for the apply (compressed only): Qf = L_B^{-T} Q1 (m x k), its transpose
  // Qft (k x m) and Ab = L_B^{-T} L_B^{-1} = B^{-1} (m x m), column-major
  // with leading dimensions ldm = pad(m), ldk = pad(k)
  T *Qf, *Qft, *Ab;
  int ldm, ldk;
};

template <typename T>
struct LevelRec {
  LevelLayout lay;
  std::vector<InteriorRec<T>> in;
  std::vector<SepRec<T>> sep;
};

// a fixed sequence of batched launches (replayed as one CUDA graph)
template <typename T>
struct Program {
  using Op = std::function<void(const char*, cudaStream_t)>;
  struct Acct { int kind; double flops, bytes; };
  Batch b;
  std::vector<Op> ops;
  std::vector<Acct> acct;      // launch accounting added per replay
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<void*> mem;      // split-GEMV partial sums and counters
  // launches of one part of the program, recorded before the parts are put
  // in apply order (they share the program's staging batch and memory)
  struct Piece {
    std::vector<Op> ops;
    std::vector<Acct> acct;
  };
  std::vector<Piece> down, up;   // per level: the part before / after the top
  int levels_built = 0;
};

// where GemvList::emit and friends record: a program's batch and memory with
// the launch list of one of its pieces
template <typename T>
struct ProgramSink {
  Batch& b;
  std::vector<void*>& mem;
  std::vector<typename Program<T>::Op>& ops;
  std::vector<typename Program<T>::Acct>& acct;
};

// Element budget of one GEMV task (one CTA): the launch's elements spread
// over about eight CTAs per SM, kept within the tuning's range (by default 4K
// to 32K elements: small launches get more, shorter tasks; large ones long
// enough to hide the start-up latency).
constexpr double kGemvCtas = 152.0 * 8.0;

template <typename T>
struct GemvList {
  std::vector<GemvTask<T>> t;
  std::vector<GemvContrib<T>> c;
  bool trans = false;
  int nr = 1;  // interleaved right-hand sides
  std::string tag;   // phase and level, for the launch log
  // op T chunk width: the tuning's in single precision, kGemvCols in double
  const int cols = std::is_same<T, float>::value ? active_tuning().gemv_cols : kGemvCols;
  explicit GemvList(int nr_ = 1) : nr(nr_) {}
  struct In {
    const T* A;
    int lda;
    const T* x;
    const T* x2;
    int K;
    bool tri;
    T alpha;
    bool upper = false;   // tri: the upper triangle (op T: rows <= column)
  };
  // y[M] = beta y + sum alpha op(A)(x - x2); op N chunks of kGemvBand rows,
  // op T chunks of `cols` columns (one unsplit task each until emit)
  void add(T* y, int M, int beta, const std::vector<In>& ins) {
    if (M <= 0) return;
    const int chunk = trans ? cols : kGemvBand;
    for (int i0 = 0; i0 < M; i0 += chunk) {
      GemvTask<T> g{};
      g.y = y + (size_t)i0 * nr;
      g.M = std::min(chunk, M - i0);
      g.c_begin = (int)c.size();
      g.beta = beta;
      g.nsplit = 1;
      int cnt = 0, total = 0;
      for (const auto& in : ins) {
        if (in.K <= 0) continue;
        GemvContrib<T> q;
        q.A = trans ? in.A + (size_t)i0 * in.lda : in.A + i0;
        q.x = in.x;
        q.x2 = in.x2;
        q.lda = in.lda;
        q.K = in.K;
        q.tri = in.tri ? i0 + 1 : 0;
        q.upper = in.upper ? 1 : 0;
        q.alpha = in.alpha;
        int kb, ke;
        gemv_useful(trans, q.tri, q.upper, q.K, g.M, &kb, &ke);
        total += ke - kb;
        c.push_back(q);
        ++cnt;
      }
      g.c_count = cnt;
      g.k_hi = total;
      t.push_back(g);
    }
  }

  void append(const GemvList& o) {
    const int base = (int)c.size();
    for (GemvTask<T> g : o.t) {
      g.c_begin += base;
      t.push_back(g);
    }
    c.insert(c.end(), o.c.begin(), o.c.end());
  }
  // Split chunks into tasks of about `budget` elements (and at most kGemvMaxC
  // contributions each); returns the number of partial elements and counters
  // the split chunks need.  Depends on the shapes only, not on nr.
  void split(double budget, std::vector<GemvTask<T>>& out, size_t& npart, int& ncnt) const {
    npart = 0;
    ncnt = 0;
    std::vector<int> pre;
    std::vector<GemvTask<T>> pcs;
    for (size_t gi = 0; gi < t.size(); ++gi) {
      const GemvTask<T>& g = t[gi];
      pre.assign(1, 0);
      for (int k = 0; k < g.c_count; ++k) {
        const GemvContrib<T>& q = c[g.c_begin + k];
        int kb, ke;
        gemv_useful(trans, q.tri, q.upper, q.K, g.M, &kb, &ke);
        pre.push_back(pre.back() + ke - kb);
      }
      const int total = pre.back();
      if (total == 0) {          // nothing to add: y = beta y
        GemvTask<T> h = g;
        h.c_count = 0;
        h.k_lo = h.k_hi = 0;
        out.push_back(h);
        continue;
      }
      const int span = std::max(1, (int)(budget / g.M));
      const int npieces = std::max(1, (total + span - 1) / span);
      if (npieces == 1 && g.c_count <= kGemvMaxC) {   // unsplit
        out.push_back(g);
        continue;
      }
      pcs.clear();
      const int len = (total + npieces - 1) / npieces;
      int cf = 0;
      for (int a = 0; a < total;) {
        while (pre[cf + 1] <= a) ++cf;
        const int b = std::min({total, a + len, pre[std::min(cf + kGemvMaxC, g.c_count)]});
        int cl = cf;
        while (pre[cl + 1] < b) ++cl;
        GemvTask<T> h = g;
        h.c_begin = g.c_begin + cf;
        h.c_count = cl - cf + 1;
        h.k_lo = a - pre[cf];
        h.k_hi = b - pre[cf];
        pcs.push_back(h);
        a = b;
      }
      const int ns = (int)pcs.size();
      for (int k = 0; k < ns; ++k) {
        GemvTask<T> h = pcs[k];
        h.split = k;
        h.nsplit = ns;
        // offsets for now; made pointers once the buffers exist
        h.part = (T*)(uintptr_t)(npart * sizeof(T));
        h.cnt = (int*)(uintptr_t)((size_t)ncnt * sizeof(int));
        out.push_back(h);
      }
      if (ns > 1) {
        npart += (size_t)ns * g.M * nr;
        ++ncnt;
      }
    }
  }

  template <class Prog>
  void emit(Prog& P, cudaStream_t s) {
    if (t.empty()) return;
    double fl = 0, by = 0, el_all = 0;
    for (const auto& g : t) {
      by += (double)sizeof(T) * g.M * nr * (g.beta ? 2 : 1);
      for (int k = g.c_begin; k < g.c_begin + g.c_count; ++k) {
        // elements of A read: the lower-triangular ones only when tri is set
        double el = (double)g.M * c[k].K;
        if (c[k].tri) {
          const double lo = c[k].tri - 1, hi = lo + g.M;  // absolute rows / columns of the chunk
          el = (trans && !c[k].upper) ? (double)g.M * c[k].K - 0.5 * (hi * (hi - 1) - lo * (lo - 1))
                                      : 0.5 * ((hi) * (hi + 1) - lo * (lo + 1));
        }
        fl += 2.0 * el;
        el_all += el;
        by += (double)sizeof(T) * (el + (double)c[k].K * nr * (c[k].x2 ? 2.0 : 1.0));
      }
    }
    const sgf_tuning& tu = active_tuning();
    const double budget = std::min((double)tu.gemv_max_elems, std::max((double)tu.gemv_min_elems, el_all / kGemvCtas));
    std::vector<GemvTask<T>> tasks;
    size_t npart = 0;
    int ncnt = 0;
    split(budget, tasks, npart, ncnt);
    T* part = nullptr;
    int* cnt = nullptr;
    if (ncnt > 0) {
      part = (T*)dev_malloc_async(npart * sizeof(T), s);
      cnt = (int*)dev_malloc_async((size_t)ncnt * sizeof(int), s);
      dev_memset(cnt, 0, (size_t)ncnt * sizeof(int), s);
      P.mem.push_back(part);
      P.mem.push_back(cnt);
    }
    for (auto& h : tasks) {
      if (h.nsplit > 1) {
        h.part = part + (uintptr_t)h.part / sizeof(T);
        h.cnt = cnt + (uintptr_t)h.cnt / sizeof(int);
      } else {
        h.part = nullptr;
        h.cnt = nullptr;
      }
    }
    // chunks too small to fill a CTA are run one per warp (eight to a block,
    // largest first) in the same launch; split and large chunks keep a CTA each
    std::vector<GemvTask<T>> wt, ct;
    for (const GemvTask<T>& h : tasks) {
      const double el = (double)h.M * (h.k_hi - h.k_lo);
      if (h.nsplit == 1 && el <= kGemvWarpElems && (trans || h.M <= kGemvWarpRowsMax)) wt.push_back(h);
      else ct.push_back(h);
    }
    std::stable_sort(wt.begin(), wt.end(), [](const GemvTask<T>& a, const GemvTask<T>& b) {
      return (double)a.M * (a.k_hi - a.k_lo) > (double)b.M * (b.k_hi - b.k_lo);
    });
    const size_t oc = P.b.push(c);
    const size_t ot = ct.empty() ? 0 : P.b.push(ct), ow = wt.empty() ? 0 : P.b.push(wt);
    const int n = (int)ct.size(), nw = (int)wt.size();
    const bool tr = trans;
    const int r = nr, cw = cols;
    int max_m = 1;
    for (const auto& h : ct) max_m = std::max(max_m, h.M);
    P.acct.push_back({tr ? P_GEMV_T : P_GEMV_N, fl * r, by});
    // launch-log description: phase, CTA / warp tasks, the largest task's
    // elements and contributions, the split budget
    std::shared_ptr<std::string> note;
    if (prof_logging()) {
      double emax = 0;
      int cmax = 0, mmax = 0, nsp = 0;
      for (const auto& h : tasks) {
        emax = std::max(emax, (double)h.M * (h.k_hi - h.k_lo));
        cmax = std::max(cmax, h.c_count);
        mmax = std::max(mmax, h.M);
        nsp += h.nsplit > 1;
      }
      char buf[256];
      std::snprintf(buf, sizeof buf, "%s cta %d warp %d split %d el %.3g emax %.0f cmax %d mmax %d budget %.0f",
                    tag.c_str(), n, nw, nsp, el_all, emax, cmax, mmax, budget);
      note = std::make_shared<std::string>(buf);
    }
    P.ops.push_back([=](const char* d, cudaStream_t st) {
      if (note) prof_note(note->c_str());
      prof_work(fl * r, by);
      const GemvTask<T>* cta = (const GemvTask<T>*)(d + ot);
      const GemvTask<T>* wtk = nw > 0 ? (const GemvTask<T>*)(d + ow) : nullptr;
      if (tr) launch_gemv_t<T>(cta, (const GemvContrib<T>*)(d + oc), n, r, cw, st, wtk, nw);
      else launch_gemv_n<T>(cta, (const GemvContrib<T>*)(d + oc), n, r, max_m, st, wtk, nw);
    });
    t.clear();
    c.clear();
  }
};

void emit_veccopy_impl(std::vector<VecCopyTask>& v, Batch& b,
                       std::vector<std::function<void(const char*, cudaStream_t)>>& ops,
                       std::function<void(const VecCopyTask*, int, cudaStream_t)> fn) {
  if (v.empty()) return;
  const size_t ov = b.push(v);
  const int n = (int)v.size();
  ops.push_back([=](const char* d, cudaStream_t s) { fn((const VecCopyTask*)(d + ov), n, s); });
  v.clear();
}

template <typename T>
class FactorImpl final : public FactorBase {
 public:
  FactorImpl(const Plan& P, const double* coeffs, cudaStream_t s) {
    plan = &P;
    n = P.n;
    tune_ = P.tune;   // a factor keeps the launch shapes it was made with
    if (!dry_run()) SGF_CK(cudaGetDevice(&device));
    st_ = (DevStatus*)dev_malloc_async(sizeof(DevStatus), s);
    dev_memset(st_, 0, sizeof(DevStatus), s);
    try {
      build(coeffs, s);
      trace(s, 0, "apply programs + top");
    } catch (...) {
      release();
      throw;
    }
  }
  ~FactorImpl() override { release(); }
  bool mixed() const override { return sizeof(T) == 4; }

  int device_status() override {
    if (dry_run()) return SGF_OK;
    DevStatus h;
    SGF_CK(cudaMemcpy(&h, st_, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.code) return h.code;
    if (h.nonfinite) {
      SGF_CK(cudaMemset(&st_->nonfinite, 0, sizeof(int)));
      return SGF_ERR_NONFINITE;
    }
    return SGF_OK;
  }

  void apply(const double* x, double* y, cudaStream_t s) override { apply_n(x, y, 1, s); }
  void multiply(const double* x, double* y, cudaStream_t s) override { multiply_n(x, y, 1, s); }
  void apply_n(const double* x, double* y, int nrhs, cudaStream_t s) override { run_n(true, x, y, nrhs, s); }
  void multiply_n(const double* x, double* y, int nrhs, cudaStream_t s) override { run_n(false, x, y, nrhs, s); }

  // up to kMaxNr right-hand sides per program run (RHS-major, stride n)
  void run_n(bool inverse, const double* x, double* y, int nrhs, cudaStream_t s) {
    std::lock_guard<std::mutex> g(prog_mu_);   // one program run at a time per factor
    for (int j = 0; j < nrhs; j += kMaxNr) {
      const int k = std::min(kMaxNr, nrhs - j);
      const int nr = k == 1 ? 1 : k == 2 ? 2 : k <= 4 ? 4 : 8;
      run_program(program(inverse, nr, s), nr, x + (int64_t)j * n, y + (int64_t)j * n, k, s);
    }
  }
  void spmv(const double* x, double* y, cudaStream_t s) override {
    if (bsr_) launch_spmv_bsr27(bsr_, plan->nx, plan->ny, plan->nz, x, y, s);
    else launch_spmv_stencil(sd_, sx_, sy_, sz_, plan->nx, plan->ny, plan->nz, x, y, s);
  }

 private:
  std::vector<void*> keep_;
  DevStatus* st_ = nullptr;
  double *sd_ = nullptr, *sx_ = nullptr, *sy_ = nullptr, *sz_ = nullptr;
  double* bsr_ = nullptr;   // Q1 elasticity: 27 FP64 3x3 blocks per point
  const int64_t* perm1_ = nullptr;
  std::vector<LevelRec<T>> lev_;
  int mtop_ = 0;
  T *Ltop_ = nullptr, *Litop_ = nullptr;
  T* Atop_ = nullptr;   // the top block's inverse L^{-T} L^{-1}, which the apply reads
  std::vector<T*> vb_;  // per non-top level: [v | w | kept], 3 * vec_size
  T* vtop_ = nullptr;   // [v | w], 2 * mtop
  Program<T> inv_[4], fwd_[4];   // nr = 1, 2, 4, 8 right-hand sides, built on first use
  sgf_tuning tune_{};
  std::mutex prog_mu_;

  // Everything the factor holds came from the stream-ordered pool; after the
  // device is idle it goes back to the pool (no unmapping, so the next
  // factorization of a plan of this size allocates without driver calls).
  void release() {
    if (!dry_run()) cudaDeviceSynchronize();
    cudaStream_t s0 = nullptr;
    for (void* p : keep_) dev_free_async(p, s0);
    keep_.clear();
    if (st_) dev_free_async(st_, s0);
    st_ = nullptr;
    for (int k = 0; k < 4; ++k)
      for (Program<T>* P : {&inv_[k], &fwd_[k]}) {
        if (!dry_run()) {
          if (P->b.dev) dev_free_async(P->b.dev, s0);
          if (P->exec) cudaGraphExecDestroy(P->exec);
          if (P->graph) cudaGraphDestroy(P->graph);
        }
        for (void* m : P->mem) dev_free_async(m, s0);
        P->mem.clear();
        P->b.dev = nullptr;
        P->exec = nullptr;
        P->graph = nullptr;
      }
  }

  void check_status(cudaStream_t s) {
    dev_sync(s);
    DevStatus h;
    dev_d2h(&h, st_, sizeof(h), s);
    if (h.code) {
      bad_level = h.level;
      bad_node = h.node;
      status = h.code;
      throw SgfError(h.code, "non-positive or non-finite pivot at level " + std::to_string(h.level) +
                                 ", node " + std::to_string(h.node));
    }
  }

  void run_program(Program<T>& P, int nr, const double* x, double* y, int nrhs, cudaStream_t s) {
    T* v1 = lev_.empty() ? vtop_ : vb_[0];
    launch_gather<T>(x, perm1_, v1, n, nrhs, nr, s);
    if (dry_run() || !apply_graph()) {
      // SGF_APPLY_GRAPH=0: the program's launches issued one by one (each
      // counted and, with profiling, timed on its own)
      for (auto& op : P.ops) op(P.b.dev, s);
    } else {
      if (!P.exec) capture(P);
      {
        double fl = 0, by = 0;
        for (const auto& a : P.acct) {
          prof_count(a.kind, a.flops, a.bytes);
          fl += a.flops;
          by += a.bytes;
        }
        prof_work(fl, by);
        ProfScope ps(P_APPLY, s);
        SGF_CK(cudaGraphLaunch(P.exec, s));
      }
    }
    launch_scatter<T>(v1, perm1_, y, n, nrhs, nr, s, &st_->nonfinite);
  }

  // record the program's launches once on a private stream
  void capture(Program<T>& P) {
    cudaStream_t cs;
    note_alloc_event();
    SGF_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    prof_capture(true);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      // every kernel after the first may launch programmatically (its
      // prologue overlaps the previous kernel's tail)
      for (size_t i = 0; i < P.ops.size(); ++i) {
        set_dependent_launch(i > 0);
        P.ops[i](P.b.dev, cs);
      }
      set_dependent_launch(false);
      e = cudaStreamEndCapture(cs, &P.graph);
    }
    prof_capture(false);
    cudaStreamDestroy(cs);
    SGF_CK(e);
    note_alloc_event();
    SGF_CK(cudaGraphInstantiate(&P.exec, P.graph, 0));
  }

  // device copies of the plan's constant data (assembly map, DOF order,
  // level-1 bases, re-expansion matrices), uploaded once per plan and device
  struct PlanData {
    const int64_t* map;
    const int64_t* perm;
    const int* ld;
    const double* kref;
    const T* phi1;
    std::vector<const T*> reexp;
  };
  static PlanData plan_data(const Plan& P, cudaStream_t s) {
    std::lock_guard<std::mutex> g(P.cache_mu);
    Plan::DevCache& C = P.cache;
    int dev = 0;
    if (!dry_run()) SGF_CK(cudaGetDevice(&dev));
    if (C.device >= 0 && C.device != dev)
      throw SgfError(SGF_ERR_INVALID_ARG, "plan data cached on another device");
    const int ti = sizeof(T) == 8 ? 0 : 1;
    if (!C.map) {
      C.device = dev;
      C.map = (int64_t*)dev_malloc(std::max<size_t>(P.asm_map.size(), 1) * 8);
      dev_h2d(C.map, P.asm_map.data(), P.asm_map.size() * 8, s);
      C.perm = (int64_t*)dev_malloc(std::max<size_t>(P.perm1.size(), 1) * 8);
      dev_h2d(C.perm, P.perm1.data(), P.perm1.size() * 8, s);
      if (!P.kref.empty()) {
        C.ld = (int*)dev_malloc(std::max<size_t>(P.asm_ld.size(), 1) * 4);
        dev_h2d(C.ld, P.asm_ld.data(), P.asm_ld.size() * 4, s);
        C.kref = (double*)dev_malloc(P.kref.size() * 8);
        dev_h2d(C.kref, P.kref.data(), P.kref.size() * 8, s);
      }
      dev_sync(s);
    }
    if (!C.phi1[ti]) {
      std::vector<T> h(P.phi1.size());
      for (size_t i = 0; i < h.size(); ++i) h[i] = (T)P.phi1[i];
      C.phi1[ti] = dev_malloc(std::max<size_t>(h.size(), 1) * sizeof(T));
      dev_h2d(C.phi1[ti], h.data(), h.size() * sizeof(T), s);
      C.reexp[ti].assign(P.lev.size(), nullptr);
      for (size_t li = 1; li < P.lev.size(); ++li) {
        const auto& r = P.lev[li].reexp;
        std::vector<T> hr(r.size());
        for (size_t i = 0; i < hr.size(); ++i) hr[i] = (T)r[i];
        C.reexp[ti][li] = dev_malloc(std::max<size_t>(hr.size(), 1) * sizeof(T));
        dev_h2d(C.reexp[ti][li], hr.data(), hr.size() * sizeof(T), s);
      }
      dev_sync(s);
    }
    PlanData d;
    d.map = C.map;
    d.perm = C.perm;
    d.ld = C.ld;
    d.kref = C.kref;
    d.phi1 = (const T*)C.phi1[ti];
    for (void* p : C.reexp[ti]) d.reexp.push_back((const T*)p);
    return d;
  }

  // SGF_TRACE=1: synchronize and print the wall time of each factor phase
  bool trace_on_ = std::getenv("SGF_TRACE") != nullptr;
  std::chrono::steady_clock::time_point trace_t0_ = std::chrono::steady_clock::now();
  // (wall time since the previous mark, and the host time spent before this
  // mark's synchronisation, i.e. building and issuing the phase)
  void trace(cudaStream_t s, int level, const char* what) {
    if (!trace_on_) return;
    const auto issued = std::chrono::steady_clock::now();
    if (!dry_run()) cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[sgf trace] level %d %-22s %8.3f ms  (host %7.3f ms)\n", level, what,
                 std::chrono::duration<double, std::milli>(now - trace_t0_).count(),
                 std::chrono::duration<double, std::milli>(issued - trace_t0_).count());
    trace_t0_ = now;
  }

  void build(const double* coeffs, cudaStream_t s) {
    const Plan& P = *plan;
    TuneScope tscope(&tune_);
    trace(s, 0, "start");
    const int pi = P.pi;
    Batch b;
    // ---- level 1 sizes, layout, assembly --------------------------------
    const LevelSym& L1 = P.lev[0];
    std::vector<int> m(L1.nnodes);
    for (int i = 0; i < L1.nnodes; ++i) m[i] = (L1.pt_ptr[i + 1] - L1.pt_ptr[i]) * P.dof;
    LevelLayout lay;
    build_layout(L1, m, lay);
    T* Dg = dalloc<T>(keep_, lay.dg_size, s);
    T* Up = dalloc<T>(keep_, lay.up_size, s);
    const PlanData pd = plan_data(P, s);
    perm1_ = pd.perm;
    if (P.stencil == SGF_STENCIL_Q1_ELASTIC_3D) {
      bsr_ = dalloc<double>(keep_, (size_t)P.npts * 27 * 9, s, false);
      launch_assemble_q1<T>(coeffs, pd.kref, P.nx, P.ny, P.nz, pd.map, pd.ld, lay.dg_size, Dg, Up, bsr_, s);
    } else {
      sd_ = dalloc<double>(keep_, P.npts, s);
      sx_ = dalloc<double>(keep_, P.npts, s);
      sy_ = dalloc<double>(keep_, P.npts, s);
      sz_ = dalloc<double>(keep_, P.npts, s);
      const double w = P.stencil == SGF_STENCIL_7PT_FV_3D ? 2.0 : 1.0;
      launch_assemble_scalar<T>(coeffs, P.nx, P.ny, P.nz, P.grid.dirichlet, w, pd.map, lay.dg_size, Dg, Up,
                                sd_, sx_, sy_, sz_, s);
    }
    if (!dry_run()) SGF_CK(cudaGetLastError());
    trace(s, 1, "assembly");
    // level-1 Phi: a working copy (merges write the next level's)
    T* Phi = nullptr;
    std::vector<void*> phiw;
    Phi = walloc<T>(phiw, std::max<size_t>(P.phi1.size(), 1), s, false);
    dev_d2d(Phi, pd.phi1, P.phi1.size() * sizeof(T), s);

    for (size_t li = 0; li < P.lev.size(); ++li) {
      const LevelSym& L = P.lev[li];
      const int lvl = (int)li + 1;
      LevelStats ls;
      ls.m = m;
      ls.r = m;
      if (L.top) {
        mtop_ = m[0];
        Ltop_ = Dg;
        Litop_ = dalloc<T>(keep_, (size_t)mtop_ * mtop_, s);
        std::vector<Front<T>> F = {{Dg, mtop_, nullptr, 0, Litop_, 0}};
        if (mtop_ > 0) run_fronts<T>(F, b, s, st_, lvl);
        b.run(s);
        if (mtop_ > 0) {   // stream ordered after the top factor
          Atop_ = dalloc<T>(keep_, (size_t)mtop_ * mtop_, s, false);
          GemmList<T> ga;
          ga.add_lowtri_tt_lower(Atop_, mtop_, mtop_, Litop_, mtop_);
          ga.emit(b, s);
          b.run(s);
          CopyList<T, T> cm;
          add_mirror(cm, Atop_, mtop_);
          cm.emit(b, s);
          b.run(s);
        }
        trace(s, lvl, "top factor issued");
        // the apply program is built on the host while the GPU finishes the
        // top factor; a failed pivot below discards it with the factor
        build_programs(s);
        check_status(s);
        ls.size_before = ls.size_after = mtop_;
        ls.bytes = (int64_t)2 * mtop_ * mtop_ * sizeof(T);
        stats.push_back(ls);
        for (void* p : phiw) dev_free_async(p, s);
        free_work(s);
        break;
      }
      LevelRec<T> rec;
      rec.lay = lay;
      const int nn = L.nnodes;
      // ---------------- 1. eliminate interiors --------------------------
      std::vector<int64_t> li_off(nn, -1);
      int64_t li_tot = 0;
      for (int i = 0; i < nn; ++i)
        if (L.interior[i] && m[i] > 0) { li_off[i] = li_tot; li_tot += (int64_t)m[i] * m[i]; }
      T* LiI = dalloc<T>(keep_, li_tot, s);
      int64_t w_tot = 0;
      std::vector<int64_t> w_off(nn, -1);
      for (int i = 0; i < nn; ++i)
        if (L.interior[i] && m[i] > 0) { w_off[i] = w_tot; w_tot += (int64_t)m[i] * lay.up_w[i]; }
      T* Wb = dalloc<T>(keep_, w_tot, s, false);
      std::vector<Front<T>> F;
      for (int i = 0; i < nn; ++i) {
        if (!L.interior[i] || m[i] == 0) continue;
        F.push_back({Dg + lay.dg_off[i], m[i], nullptr, 0, LiI + li_off[i], i});
        InteriorRec<T> r;
        r.node = i;
        r.m = m[i];
        r.s = lay.up_w[i];
        r.L = Dg + lay.dg_off[i];
        r.Li = LiI + li_off[i];
        r.W = Wb + w_off[i];
        r.Z = r.Zt = r.Ai = nullptr;
        r.ldm = r.lds = 0;
        for (int k = lay.up_ptr[i]; k < lay.up_ptr[i + 1]; ++k) r.nb.push_back({lay.up_nb[k], lay.up_col[k]});
        rec.in.push_back(r);
      }
      run_fronts<T>(F, b, s, st_, lvl);
      b.run(s);
      trace(s, lvl, "interior fronts");
      {
        // W_I = L_I^{-1} A_I,S (Sec. 4.1), one launch over all interiors
        GemmList<T> gw;
        for (const auto& r : rec.in)
          if (r.s > 0) gw.add_lowtri(r.W, r.m, r.m, r.s, r.Li, r.m, Up + lay.up_off[r.node], r.m);
        gw.emit(b, s);
      }
      {
        // Schur complement, owner-computes per target block.  Targets are
        // numbered (diagonal block of S: S; block (Sa, Sb), Sa < Sb: nn + its
        // index in Sa's neighbour list); the (target, contribution) pairs are
        // bucketed by target with a stable counting sort, so each target sums
        // its contributions in interior order.
        struct Pair { int id; Spec<T> sp; };
        const int nin = (int)rec.in.size();
        const int ntg = nn + (int)lay.up_nb.size();
        auto tid = [&](int Sa, int Sb) {
          if (Sa == Sb) return Sa;
          auto bgn = lay.up_nb.begin() + lay.up_ptr[Sa], end = lay.up_nb.begin() + lay.up_ptr[Sa + 1];
          auto it = std::lower_bound(bgn, end, Sb);
          if (it == end || *it != Sb) throw SgfError(SGF_ERR_CUDA, "internal: missing fill block");
          return nn + (int)(it - lay.up_nb.begin());
        };
        Pooled<std::vector<Pair>> pp;
        std::vector<Pair>& pairs = pp.v;
        for (int k = 0; k < nin; ++k) {
          const auto& r = rec.in[k];
          for (size_t a = 0; a < r.nb.size(); ++a)
            for (size_t c = a; c < r.nb.size(); ++c)
              pairs.push_back({tid(r.nb[a].first, r.nb[c].first),
                               {r.W + (size_t)r.nb[a].second * r.m, r.m, true,
                                r.W + (size_t)r.nb[c].second * r.m, r.m, false, r.m}});
        }
        std::vector<int> start(ntg + 1, 0);
        for (const Pair& q : pairs) ++start[q.id + 1];
        for (int k = 0; k < ntg; ++k) start[k + 1] += start[k];
        Pooled<std::vector<Spec<T>>> sp;
        std::vector<Spec<T>>& sorted = sp.v;
        sorted.resize(start[ntg]);
        {
          std::vector<int> fill(start.begin(), start.end() - 1);
          for (const Pair& q : pairs) sorted[fill[q.id]++] = q.sp;
        }
        GemmList<T> gl;
        {
          GemmList<T>& G = gl;
          for (int k = 0; k < ntg; ++k) {
            if (start[k] == start[k + 1]) continue;
            int Sa, Sb;
            T* C;
            if (k < nn) {
              Sa = Sb = k;
              C = Dg + lay.dg_off[Sa];
            } else {
              const int u = k - nn;
              Sa = (int)(std::upper_bound(lay.up_ptr.begin(), lay.up_ptr.end(), u) - lay.up_ptr.begin()) - 1;
              Sb = lay.up_nb[u];
              C = Up + lay.up_off[Sa] + (size_t)lay.up_col[u] * m[Sa];
            }
            G.add_range(C, m[Sa], m[Sa], m[Sb], T(-1), 1, sorted.data() + start[k], sorted.data() + start[k + 1]);
          }
        }
        gl.emit(b, s);
        b.run(s);
      }
      trace(s, lvl, "W + Schur");
      // ---------------- 2. compression, phase 1 --------------------------
      std::vector<std::vector<int>> nball(nn);
      for (size_t p = 0; p < L.post.size(); p += 2) {
        nball[L.post[p]].push_back(L.post[p + 1]);
        nball[L.post[p + 1]].push_back(L.post[p]);
      }
      for (auto& v : nball) std::sort(v.begin(), v.end());
      std::vector<int> E;
      for (int i = 0; i < nn; ++i)
        if (!L.interior[i] && L.eligible[i] && m[i] > 0) E.push_back(i);
      const int ne = (int)E.size();
      std::vector<int64_t> o_mm(ne), o_ms(ne), o_mc(ne), o_mp(ne);
      std::vector<int> sw(ne), cw(ne);
      int64_t t_mm = 0, t_ms = 0, t_mc = 0, t_mp = 0;
      int max_m = 1, max_c = 1;
      // gofs[B][k]: column offset of neighbour nball[B][k] in B's gathered block
      std::vector<std::vector<int>> gofs(nn);
      std::vector<int> eidx(nn, -1);
      // Nest-2-2: per compressed node, the neighbours (indices into nball) that
      // are lower-dimensional separators on its rim - boxes at most one grid
      // step apart on every axis; their whole blocks M^_BE join N
      const bool rim = P.opts.scheme == SGF_SCHEME_NEST_2_2;
      std::vector<std::vector<int>> adj(ne);
      auto touching = [&](int B, int X) {
        if (L.interior[X] || L.cell_dim[X] >= P.grid.dim - 1) return false;
        for (int a = 0; a < 3; ++a) {
          const int gap = std::max({0, L.box[6 * X + a] - L.box[6 * B + 3 + a], L.box[6 * B + a] - L.box[6 * X + 3 + a]});
          if (gap > 1) return false;
        }
        return true;
      };
      auto gcol = [&](int B, int N) {
        const auto& v = nball[B];
        const auto it = std::lower_bound(v.begin(), v.end(), N);
        return gofs[B][it - v.begin()];
      };
      for (int e = 0; e < ne; ++e) {
        const int B = E[e];
        eidx[B] = e;
        int sB = 0;
        gofs[B].reserve(nball[B].size());
        for (int N : nball[B]) { gofs[B].push_back(sB); sB += m[N]; }
        sw[e] = sB;
        cw[e] = pi * (1 + (int)nball[B].size());
        if (rim)
          for (size_t k = 0; k < nball[B].size(); ++k)
            if (m[nball[B][k]] > 0 && touching(B, nball[B][k])) {
              adj[e].push_back((int)k);
              cw[e] += m[nball[B][k]];
            }
        o_mm[e] = t_mm; t_mm += (int64_t)m[B] * m[B];
        o_ms[e] = t_ms; t_ms += (int64_t)m[B] * sB;
        o_mc[e] = t_mc; t_mc += (int64_t)m[B] * cw[e];
        o_mp[e] = t_mp; t_mp += (int64_t)m[B] * pi;
        max_m = std::max(max_m, m[B]);
        max_c = std::max(max_c, cw[e]);
      }
      if (qr_smem_bytes(max_m, max_c, sizeof(T), 0) > 220 * 1024)
        throw SgfError(SGF_ERR_UNSUPPORTED, "node too large for the QR kernel");
      T* Dw = dalloc<T>(keep_, t_mm, s, false);
      T* LiB = dalloc<T>(keep_, t_mm, s);
      T* Q1 = dalloc<T>(keep_, t_mm, s, false);
      T* G = walloc<T>(work_, t_ms, s, false);
      T* Mh = walloc<T>(work_, t_ms, s, false);
      T* Nm = walloc<T>(work_, t_mc, s, false);
      T* LtP = walloc<T>(work_, t_mp, s, false);
      int* dranks = walloc<int>(work_, ne, s);
      {
        CopyList<T, T> cl;
        for (int e = 0; e < ne; ++e) {
          const int B = E[e];
          cl.add(Dg + lay.dg_off[B], m[B], Dw + o_mm[e], m[B], m[B], m[B], kCopyLower);
          for (size_t k = 0; k < nball[B].size(); ++k) {
            const int N = nball[B][k];
            T* dst = G + o_ms[e] + (size_t)gofs[B][k] * m[B];
            if (N > B) {
              const int col = lay.col_of(B, N);
              cl.add(Up + lay.up_off[B] + (size_t)col * m[B], m[B], dst, m[B], m[B], m[N], kCopy);
            } else {
              const int col = lay.col_of(N, B);
              cl.add(Up + lay.up_off[N] + (size_t)col * m[N], m[N], dst, m[B], m[B], m[N], kCopyT);
            }
          }
        }
        cl.emit(b, s);
        b.run(s);
      }
      {
        std::vector<Front<T>> FB;
        for (int e = 0; e < ne; ++e) FB.push_back({Dw + o_mm[e], m[E[e]], nullptr, 0, LiB + o_mm[e], E[e]});
        run_fronts<T>(FB, b, s, st_, lvl);
        {
          // M^_B,nbrs = L_B^{-1} A_B,nbrs (Eq. (compr-scale))
          GemmList<T> gm;
          for (int e = 0; e < ne; ++e)
            if (sw[e] > 0) gm.add_lowtri(Mh + o_ms[e], m[E[e]], m[E[e]], sw[e], LiB + o_mm[e], m[E[e]], G + o_ms[e], m[E[e]]);
          gm.emit(b, s);
        }
        CopyList<T, T> cz;
        for (int e = 0; e < ne; ++e) {
          const int mb = m[E[e]];
          for (int j0 = kTile; j0 < mb; j0 += kTile)
            cz.add(nullptr, 0, Dw + o_mm[e] + (size_t)j0 * mb, mb, std::min(j0, mb), std::min(kTile, mb - j0), kZero);
        }
        cz.emit(b, s);
        GemmList<T> gl;
        for (int e = 0; e < ne; ++e) {
          const int B = E[e], mb = m[B];
          T* Nb = Nm + o_mc[e];
          gl.add(Nb, mb, mb, pi, T(1), 0, {{Dw + o_mm[e], mb, true, Phi + lay.vec_off[B] * pi, mb, false, mb}});
          for (size_t k = 0; k < nball[B].size(); ++k) {
            const int N = nball[B][k];
            gl.add(Nb + (size_t)(k + 1) * pi * mb, mb, mb, pi, T(1), 0,
                   {{Mh + o_ms[e] + (size_t)gofs[B][k] * mb, mb, false, Phi + lay.vec_off[N] * pi, m[N], false, m[N]}});
          }
        }
        gl.emit(b, s);
        if (rim) {   // the rim blocks, whole, after the polynomial columns
          CopyList<T, T> ca;
          for (int e = 0; e < ne; ++e) {
            const int B = E[e], mb = m[B];
            size_t col = (size_t)pi * (1 + nball[B].size());
            for (int k : adj[e]) {
              const int X = nball[B][k];
              ca.add(Mh + o_ms[e] + (size_t)gofs[B][k] * mb, mb, Nm + o_mc[e] + col * mb, mb, mb, m[X], kCopy);
              col += m[X];
            }
          }
          ca.emit(b, s);
        }
        b.run(s);
        CopyList<T, T> cp;
        for (int e = 0; e < ne; ++e) cp.add(Nm + o_mc[e], m[E[e]], LtP + o_mp[e], m[E[e]], m[E[e]], pi, kCopy);
        cp.emit(b, s);
        // shared-memory sweep when m x (columns not identically zero) fits
        std::vector<QrTask<T>> qs, qg;
        int sm_m = 1, sm_c = 1, g_m = 1, g_c = 1;
        long long cap = 0;
        const size_t budget = 200 * 1024;
        for (int e = 0; e < ne; ++e) {
          const int B = E[e];
          int ce = L.act[B];
          for (int N : nball[B]) ce += L.act[N];
          for (int k : adj[e]) ce += m[nball[B][k]];
          ce = std::min(ce, cw[e]);
          QrTask<T> q{Nm + o_mc[e], Q1 + o_mm[e], m[B], cw[e], B, e};
          const long long need = (long long)m[B] * ce;
          if (qr_smem_bytes(std::max(sm_m, m[B]), std::max(sm_c, cw[e]), sizeof(T), std::max(cap, need)) <= budget) {
            qs.push_back(q);
            sm_m = std::max(sm_m, m[B]);
            sm_c = std::max(sm_c, cw[e]);
            cap = std::max(cap, need);
          } else {
            qg.push_back(q);
            g_m = std::max(g_m, m[B]);
            g_c = std::max(g_c, cw[e]);
          }
        }
        const double tau = P.tau;
        for (int pass = 0; pass < 2; ++pass) {
          auto& q = pass == 0 ? qs : qg;
          if (q.empty()) continue;
          double fl = 0;
          for (const auto& t : q) fl += 4.0 * t.m * t.c * std::min(t.m, t.c);
          const size_t oq = b.push(q);
          const int nq = (int)q.size();
          const int mm = pass == 0 ? sm_m : g_m, mc = pass == 0 ? sm_c : g_c;
          const long long cp = pass == 0 ? cap : 0;
          b.launches.push_back([=](const char* d) {
            prof_work(fl, 0);
            launch_qrcp<T>((const QrTask<T>*)(d + oq), nq, dranks, tau, mm, mc, cp, s);
          });
        }
        b.run(s);
      }
      trace(s, lvl, "compression issued");
      // the level below is complete: record its parts of the apply program
      // while the GPU works through this level (the host waits next)
      if (li >= 1) {
        prebuild_level((int)li - 1, lay.vec_size, s);
        trace(s, lvl, "apply parts, level below");
      }
      check_status(s);
      trace(s, lvl, "compression to QR");
      std::vector<int> rk(ne, 0);
      if (ne) dev_d2h(rk.data(), dranks, ne * sizeof(int), s);
      if (dry_run())  // a deterministic stand-in that exercises both outcomes
        for (int e = 0; e < ne; ++e) rk[e] = std::max(1, std::min({m[E[e]] - (E[e] % 2), cw[e], (2 * m[E[e]] + 2) / 3 + (E[e] % 2) * m[E[e]]}));
      // ---------------- 3. surviving blocks ------------------------------
      std::vector<char> comp(nn, 0);
      std::vector<int> kk(nn, 0), rr(nn, 0);
      for (int i = 0; i < nn; ++i) kk[i] = L.interior[i] ? 0 : m[i];
      for (int i = 0; i < nn; ++i) rr[i] = m[i];
      for (int e = 0; e < ne; ++e) {
        const int B = E[e];
        rr[B] = rk[e];
        if (rk[e] < m[B]) { comp[B] = 1; kk[B] = rk[e]; ls.ncomp++; }
      }
      ls.r = rr;
      for (int i = 0; i < nn; ++i) if (!L.interior[i]) { ls.size_before += m[i]; ls.size_after += kk[i]; }
      // next level sizes and layout
      const LevelSym& Ln = P.lev[li + 1];
      std::vector<int> parent(nn, -1), oc(nn, 0), slot(nn, -1);
      std::vector<int> mn(Ln.nnodes, 0);
      for (int D = 0; D < Ln.nnodes; ++D)
        for (int k = Ln.child_ptr[D]; k < Ln.child_ptr[D + 1]; ++k) {
          const int C = Ln.child_idx[k];
          parent[C] = D;
          slot[C] = k;
          oc[C] = mn[D];
          mn[D] += kk[C];
        }
      LevelLayout layn;
      build_layout(Ln, mn, layn);
      T* Dgn = dalloc<T>(keep_, layn.dg_size, s);
      T* Upn = Ln.top ? nullptr : dalloc<T>(keep_, layn.up_size, s);
      std::vector<void*> phin;
      T* Phin = walloc<T>(phin, (size_t)layn.vec_size * pi, s);
      // Phi update and L^{-T} Q1
      std::vector<int64_t> o_rp(ne, 0), o_mr(ne, 0);
      int64_t t_rp = 0, t_mr = 0;
      for (int e = 0; e < ne; ++e)
        if (comp[E[e]]) {
          o_rp[e] = t_rp; t_rp += (int64_t)rk[e] * pi;
          o_mr[e] = t_mr; t_mr += (int64_t)m[E[e]] * rk[e];
        }
      T* PhiC = walloc<T>(work_, t_rp, s, false);
      T* Yh = walloc<T>(work_, t_mr, s, false);
      {
        GemmList<T> gl;
        for (int e = 0; e < ne; ++e) {
          const int B = E[e], mb = m[B], r = rk[e];
          if (!comp[B]) continue;
          gl.add(PhiC + o_rp[e], r, r, pi, T(1), 0, {{Q1 + o_mm[e], mb, true, LtP + o_mp[e], mb, false, mb}});
          gl.add(Yh + o_mr[e], mb, mb, r, T(1), 0, {{LiB + o_mm[e], mb, true, Q1 + o_mm[e], mb, false, mb}});
        }
        gl.emit(b, s);
        b.run(s);
      }
      // two-sided transforms of the separator blocks
      struct Src { const T* p; int ld; };
      std::vector<Src> src(L.post.size() / 2);
      {
        std::vector<int64_t> ko(src.size(), -1), to(src.size(), -1);
        int64_t kt = 0, tt = 0;
        for (size_t q = 0; q < src.size(); ++q) {
          const int C = L.post[2 * q], Cp = L.post[2 * q + 1];
          if (comp[C] || comp[Cp]) { ko[q] = kt; kt += (int64_t)kk[C] * kk[Cp]; }
          if (comp[C] && comp[Cp]) { to[q] = tt; tt += (int64_t)m[C] * kk[Cp]; }
        }
        T* Kb = walloc<T>(work_, kt, s, false);
        T* T1 = walloc<T>(work_, tt, s, false);
        GemmList<T> g1, g2;
        for (size_t q = 0; q < src.size(); ++q) {
          const int C = L.post[2 * q], Cp = L.post[2 * q + 1];
          const T* X = Up + lay.up_off[C] + (size_t)lay.col_of(C, Cp) * m[C];
          if (!comp[C] && !comp[Cp]) { src[q] = {X, m[C]}; continue; }
          const int e = eidx[C], ep = eidx[Cp];
          T* K = Kb + ko[q];
          if (comp[C] && !comp[Cp]) {
            g1.add(K, kk[C], kk[C], m[Cp], T(1), 0,
                   {{Q1 + o_mm[e], m[C], true, Mh + o_ms[e] + (size_t)gcol(C, Cp) * m[C], m[C], false, m[C]}});
          } else if (!comp[C] && comp[Cp]) {
            g1.add(K, m[C], m[C], kk[Cp], T(1), 0, {{X, m[C], false, Yh + o_mr[ep], m[Cp], false, m[Cp]}});
          } else {
            T* T1q = T1 + to[q];
            g1.add(T1q, m[C], m[C], kk[Cp], T(1), 0,
                   {{Mh + o_ms[e] + (size_t)gcol(C, Cp) * m[C], m[C], false, Yh + o_mr[ep], m[Cp], false, m[Cp]}});
            g2.add(K, kk[C], kk[C], kk[Cp], T(1), 0, {{Q1 + o_mm[e], m[C], true, T1q, m[C], false, m[C]}});
          }
          src[q] = {K, kk[C]};
        }
        g1.emit(b, s);
        g2.emit(b, s);
        b.run(s);
      }
      // ---------------- 4. merge into the next level --------------------
      {
        const T* R = pd.reexp[li + 1];
        CopyList<T, T> cl;
        GemmList<T> gl;
        for (int C = 0; C < nn; ++C) {
          if (L.interior[C] || kk[C] == 0) continue;
          const int D = parent[C];
          const int mD = mn[D];
          T* dd = Dgn + layn.dg_off[D] + oc[C] + (size_t)oc[C] * mD;
          if (comp[C]) cl.add(nullptr, 0, dd, mD, kk[C], kk[C], kIdentity);
          else cl.add(Dg + lay.dg_off[C], m[C], dd, mD, m[C], m[C], kCopy);
          const T* phiC = comp[C] ? PhiC + o_rp[eidx[C]] : Phi + lay.vec_off[C] * pi;
          gl.add(Phin + layn.vec_off[D] * pi + oc[C], mD, kk[C], pi, T(1), 0,
                 {{phiC, kk[C], false, R + (size_t)slot[C] * pi * pi, pi, false, pi}});
        }
        for (size_t q = 0; q < src.size(); ++q) {
          const int C = L.post[2 * q], Cp = L.post[2 * q + 1];
          const int D = parent[C], Ep = parent[Cp];
          const int rC = kk[C], rCp = kk[Cp];
          if (D == Ep) {
            const int mD = mn[D];
            cl.add(src[q].p, src[q].ld, Dgn + layn.dg_off[D] + oc[C] + (size_t)oc[Cp] * mD, mD, rC, rCp, kCopy);
            cl.add(src[q].p, src[q].ld, Dgn + layn.dg_off[D] + oc[Cp] + (size_t)oc[C] * mD, mD, rCp, rC, kCopyT);
          } else if (D < Ep) {
            const int col = layn.col_of(D, Ep);
            if (col < 0) throw SgfError(SGF_ERR_CUDA, "internal: missing merged block");
            cl.add(src[q].p, src[q].ld, Upn + layn.up_off[D] + (size_t)(col + oc[Cp]) * mn[D] + oc[C], mn[D], rC, rCp, kCopy);
          } else {
            const int col = layn.col_of(Ep, D);
            if (col < 0) throw SgfError(SGF_ERR_CUDA, "internal: missing merged block");
            cl.add(src[q].p, src[q].ld, Upn + layn.up_off[Ep] + (size_t)(col + oc[C]) * mn[Ep] + oc[Cp], mn[Ep], rCp, rC, kCopyT);
          }
        }
        cl.emit(b, s);
        gl.emit(b, s);
        b.run(s);
      }
      trace(s, lvl, "two-sided + merge");
      // ---------------- records for the apply ----------------------------
      for (int C = 0; C < nn; ++C) {
        if (L.interior[C]) continue;
        SepRec<T> sr;
        sr.node = C;
        sr.m = m[C];
        sr.k = kk[C];
        sr.comp = comp[C];
        sr.dst = layn.vec_off[parent[C]] + oc[C];
        sr.L = sr.Li = sr.Q1 = nullptr;
        sr.Qf = sr.Qft = sr.Ab = nullptr;
        sr.ldm = sr.ldk = 0;
        if (comp[C]) {
          const int e = eidx[C];
          sr.L = Dw + o_mm[e];
          sr.Li = LiB + o_mm[e];
          sr.Q1 = Q1 + o_mm[e];
        }
        rec.sep.push_back(sr);
      }
      // apply layout (the factor is done with the zero upper triangles of the
      // L^{-1} blocks at this point).  Interiors: the apply uses, instead of
      // L^{-1} and W, Z = L^{-T} W = A_II^{-1} A_IS, its transpose and
      // A_II^{-1} = L^{-T} L^{-1} (the same bytes in all, but only dense
      // blocks); their L^{-1} is freed.  Compressed separators likewise:
      // Qf = L_B^{-T} Q1, its transpose and B^{-1} = L_B^{-T} L_B^{-1}.
      {
        // leading dimensions rounded up to a 32-byte sector, so that every
        // column the apply reads starts on one
        constexpr int kApplyPad = 32 / (int)sizeof(T);   // elements per 32-byte sector
        auto pad = [](int x) { return (x + kApplyPad - 1) / kApplyPad * kApplyPad; };
        int64_t zs = 0, zts = 0, as = 0;
        for (auto& r : rec.in) {
          r.ldm = pad(r.m);
          r.lds = pad(r.s);
          zs += (int64_t)r.ldm * r.s;
          zts += (int64_t)r.lds * r.m;
          as += (int64_t)r.ldm * r.m;
        }
        for (auto& sr : rec.sep)
          if (sr.comp) {
            sr.ldm = pad(sr.m);
            sr.ldk = pad(sr.k);
            zs += (int64_t)sr.ldm * sr.k;
            zts += (int64_t)sr.ldk * sr.m;
            as += (int64_t)sr.ldm * sr.m;
          }
        T* Zb = dalloc<T>(keep_, zs, s, false);
        T* Ztb = dalloc<T>(keep_, zts, s, false);
        T* Ab = dalloc<T>(keep_, as, s, false);
        GemmList<T> gz;
        int64_t oz = 0, ozt = 0, oa = 0;
        for (auto& r : rec.in) {
          r.Z = Zb + oz;
          r.Zt = Ztb + ozt;
          r.Ai = Ab + oa;
          oz += (int64_t)r.ldm * r.s;
          ozt += (int64_t)r.lds * r.m;
          oa += (int64_t)r.ldm * r.m;
          if (r.s > 0) gz.add_lowtri_t(r.Z, r.ldm, r.m, r.s, r.Li, r.m, r.W, r.m);
          gz.add_lowtri_tt_lower(r.Ai, r.ldm, r.m, r.Li, r.m);
        }
        for (auto& sr : rec.sep) {
          if (!sr.comp) continue;
          sr.Qf = Zb + oz;
          sr.Qft = Ztb + ozt;
          sr.Ab = Ab + oa;
          oz += (int64_t)sr.ldm * sr.k;
          ozt += (int64_t)sr.ldk * sr.m;
          oa += (int64_t)sr.ldm * sr.m;
          if (sr.k > 0) gz.add_lowtri_t(sr.Qf, sr.ldm, sr.m, sr.k, sr.Li, sr.m, sr.Q1, sr.m);
          gz.add_lowtri_tt_lower(sr.Ab, sr.ldm, sr.m, sr.Li, sr.m);
        }
        gz.emit(b, s);
        b.run(s);
        CopyList<T, T> cm;
        for (auto& r : rec.in) {
          if (r.s > 0) cm.add(r.Z, r.ldm, r.Zt, r.lds, r.s, r.m, kCopyT);
          add_mirror(cm, r.Ai, r.m, r.ldm);   // the inverses exactly symmetric
        }
        for (const auto& sr : rec.sep)
          if (sr.comp) {
            if (sr.k > 0) cm.add(sr.Qf, sr.ldm, sr.Qft, sr.ldk, sr.k, sr.m, kCopyT);
            add_mirror(cm, sr.Ab, sr.m, sr.ldm);
          }
        cm.emit(b, s);
        b.run(s);
        // the L^{-1} blocks of interiors and compressed separators are not
        // read again
        for (T* li : {LiI, LiB}) {
          auto it = std::find(keep_.begin(), keep_.end(), (void*)li);
          if (it != keep_.end()) {
            keep_.erase(it);
            dev_free_async(li, s);
          }
        }
        for (auto& r : rec.in) r.Li = nullptr;
        for (auto& sr : rec.sep) sr.Li = nullptr;
      }
      int64_t bytes = 0;
      for (const auto& r : rec.in) bytes += ((int64_t)2 * r.m * r.m + (int64_t)3 * r.m * r.s) * sizeof(T);
      for (const auto& r : rec.sep)
        if (r.comp) bytes += ((int64_t)2 * r.m * r.m + (int64_t)3 * r.m * r.k) * sizeof(T);
      ls.bytes = bytes;
      stats.push_back(ls);
      lev_.push_back(std::move(rec));
      free_work(s);   // stream ordered: the host goes on building level t+1
      for (void* p : phiw) dev_free_async(p, s);
      phiw = phin;
      Phi = Phin;
      Dg = Dgn;
      Up = Upn;
      lay = layn;
      m = mn;
    }
    b.release(s);
    dev_sync(s);
  }

  std::vector<void*> work_;
  void free_work(cudaStream_t s) {
    for (void* p : work_) dev_free_async(p, s);
    work_.clear();
  }

  // ----------------------------------------------------------------------
  // apply programs
  // ----------------------------------------------------------------------
  static constexpr int kMaxNr = 8;
  // level-vector buffers [v | w | kept] of non-top level t
  void ensure_vb(int t, int64_t vec_size, cudaStream_t s) {
    if ((int)vb_.size() <= t) vb_.resize(t + 1, nullptr);
    if (!vb_[t]) vb_[t] = dalloc<T>(keep_, 3 * (size_t)kMaxNr * std::max<int64_t>(vec_size, 1), s);
  }
  // While the GPU factors level t + 1 (vec_size: its vector length), the host
  // records the single-RHS inverse program's parts for the finished level t.
  void prebuild_level(int t, int64_t next_vec_size, cudaStream_t s) {
    ensure_vb(t, lev_[t].lay.vec_size, s);
    ensure_vb(t + 1, next_vec_size, s);
    TuneScope tscope(&tune_);
    inverse_level(inv_[0], t, 1, s);
  }
  void build_programs(cudaStream_t s) {
    const int nl = (int)lev_.size();
    for (int t = 0; t < nl; ++t) ensure_vb(t, lev_[t].lay.vec_size, s);
    vtop_ = dalloc<T>(keep_, 2 * (size_t)kMaxNr * std::max(mtop_, 1), s);
    // the single-RHS inverse program is built and instantiated as a graph
    // here, so that applying the factor later allocates nothing (the other
    // programs are built on first use)
    Program<T>& P = program(true, 1, s);
    if (!dry_run() && apply_graph() && !P.exec) capture(P);
  }

  Program<T>& program(bool inverse, int nr, cudaStream_t s) {
    const int k = nr == 1 ? 0 : nr == 2 ? 1 : nr == 4 ? 2 : 3;
    Program<T>& P = inverse ? inv_[k] : fwd_[k];
    if (P.ops.empty()) {
      TuneScope tscope(&tune_);
      if (inverse) build_inverse(P, nr, s);
      else build_forward(P, nr, s);
      P.b.upload_persistent(s);
    }
    return P;
  }

  T* base(int t) { return t < (int)vb_.size() ? vb_[t] : vtop_; }

  // interior neighbours of each separator (owner-computes lists)
  std::vector<std::vector<std::pair<int, int>>> sep_interiors(const LevelRec<T>& R, int nnodes) {
    std::vector<std::vector<std::pair<int, int>>> out(nnodes);
    for (int a = 0; a < (int)R.in.size(); ++a)
      for (const auto& nb : R.in[a].nb) out[nb.first].push_back({a, nb.second});
    return out;
  }

  template <class Sink>
  void veccopy(Sink& P, std::vector<VecCopyTask>& v, const T* src, T* dst) {
    if (!v.empty()) {
      double by = 0;
      for (const auto& t : v) by += 2.0 * sizeof(T) * t.len;
      P.acct.push_back({P_VECCOPY, 0.0, by});
    }
    emit_veccopy_impl(v, P.b, P.ops, [src, dst](const VecCopyTask* t, int n, cudaStream_t s) {
      launch_veccopy<T>(t, n, src, dst, s);
    });
  }

  // A_l^{-1} x in apply order: for each level upward the interior solve and
  // separator update (down part), the top solve, then for each level
  // downward the back substitution (up part).  The parts of a level are
  // recorded as soon as the level is factored; the program is put together
  // once all are.
  void inverse_level(Program<T>& P, int t, int nr, cudaStream_t s) {
    if (t < P.levels_built) return;
    P.down.resize(t + 1);
    P.up.resize(t + 1);
    ProgramSink<T> d{P.b, P.mem, P.down[t].ops, P.down[t].acct};
    inverse_down(d, t, nr, s);
    ProgramSink<T> u{P.b, P.mem, P.up[t].ops, P.up[t].acct};
    inverse_up(u, t, nr, s);
    P.levels_built = t + 1;
  }

  void build_inverse(Program<T>& P, int nr, cudaStream_t s) {
    const int nl = (int)lev_.size();
    for (int t = P.levels_built; t < nl; ++t) inverse_level(P, t, nr, s);
    auto take = [&P](typename Program<T>::Piece& q) {
      for (auto& o : q.ops) P.ops.push_back(std::move(o));
      P.acct.insert(P.acct.end(), q.acct.begin(), q.acct.end());
      q = {};
    };
    for (int t = 0; t < nl; ++t) take(P.down[t]);
    ProgramSink<T> top{P.b, P.mem, P.ops, P.acct};
    inverse_top(top, nr, s);
    for (int t = nl - 1; t >= 0; --t) take(P.up[t]);
    P.down.clear();
    P.up.clear();
  }

  template <class Sink>
  void inverse_down(Sink& P, int t, int nr, cudaStream_t s) {
    const LevelRec<T>& R = lev_[t];
    const auto& lay = R.lay;
    const int64_t vs = lay.vec_size;
    T* v = base(t);
    T* w = v + vs * nr;
    T* kp = v + 2 * vs * nr;
    // every product is a column dot product: Z^T x through the columns of
    // Z (v_S -= A_SI A_II^{-1} v_I = W^T L^{-1} v_I), then for the
    // compressed separators Qf^T x (= Q1^T L_B^{-1} v_B)
    GemvList<T> f2(nr), f4(nr);
    f2.trans = f4.trans = true;
    f2.tag = "L" + std::to_string(t) + ".f2";
    f4.tag = "L" + std::to_string(t) + ".f4";
    auto si = sep_interiors(R, (int)lay.m.size());
    for (int S = 0; S < (int)si.size(); ++S) {
      if (si[S].empty()) continue;
      std::vector<typename GemvList<T>::In> ins;
      for (auto [a, col] : si[S]) {
        const auto& r = R.in[a];
        ins.push_back({r.Z + (size_t)col * r.ldm, r.ldm, v + nr * lay.vec_off[r.node], nullptr, r.m, false, T(-1)});
      }
      f2.add(v + nr * lay.vec_off[S], lay.m[S], 1, ins);
    }
    for (const auto& c : R.sep) {
      if (!c.comp) continue;
      f4.add(kp + nr * lay.vec_off[c.node], c.k, 0, {{c.Qf, c.ldm, v + nr * lay.vec_off[c.node], nullptr, c.m, false, T(1)}});
    }
    f2.emit(P, s);
    f4.emit(P, s);
    std::vector<VecCopyTask> vc;
    for (const auto& c : R.sep)
      if (c.k > 0) vc.push_back({nr * ((c.comp ? 2 * vs : 0) + lay.vec_off[c.node]), nr * c.dst, nr * c.k, 0});
    veccopy(P, vc, v, base(t + 1));
  }

  template <class Sink>
  void inverse_top(Sink& P, int nr, cudaStream_t s) {
    T* v = vtop_;
    T* w = vtop_ + (size_t)mtop_ * nr;
    GemvList<T> a(nr);
    a.trans = true;
    a.tag = "top";
    // x = A_top^{-1} v (A_top^{-1} = L^{-T} L^{-1} is symmetric: its columns
    // are its rows), into w, then copied back to v
    a.add(w, mtop_, 0, {{Atop_, mtop_, v, nullptr, mtop_, false, T(1)}});
    a.emit(P, s);
    std::vector<VecCopyTask> c;
    if (mtop_ > 0) c.push_back({(int64_t)mtop_ * nr, 0, mtop_ * nr, 0});
    veccopy(P, c, vtop_, vtop_);
  }

  template <class Sink>
  void inverse_up(Sink& P, int t, int nr, cudaStream_t s) {
    const LevelRec<T>& R = lev_[t];
    const auto& lay = R.lay;
    const int64_t vs = lay.vec_size;
    T* v = base(t);
    T* w = v + vs * nr;
    T* kp = v + 2 * vs * nr;
    T* vn = base(t + 1);
    std::vector<VecCopyTask> vc;
    for (const auto& c : R.sep)
      if (!c.comp && c.k > 0) vc.push_back({nr * c.dst, nr * lay.vec_off[c.node], nr * c.k, 0});
    veccopy(P, vc, vn, v);
    // compressed separators: x_B = B^{-1} v_B + Qf (vn - kp) (= L_B^{-T}
    // (L_B^{-1} v_B + Q1 (vn - kp))), one dense phase of column dot products
    // (B^{-1} is symmetric; the rows of Qf are the columns of Qf^T), into w_B
    GemvList<T> b2(nr), b3(nr);
    b2.trans = b3.trans = true;
    b2.tag = "L" + std::to_string(t) + ".b2";
    b3.tag = "L" + std::to_string(t) + ".b3";
    std::vector<char> in_w(lay.m.size(), 0);   // nodes whose result sits in w until the final copy
    std::vector<VecCopyTask> ic;
    for (const auto& c : R.sep) {
      if (!c.comp) continue;
      std::vector<typename GemvList<T>::In> ins = {{c.Ab, c.ldm, v + nr * lay.vec_off[c.node], nullptr, c.m, false, T(1)}};
      if (c.k > 0) ins.push_back({c.Qft, c.ldk, vn + nr * c.dst, kp + nr * lay.vec_off[c.node], c.k, false, T(1)});
      b2.add(w + nr * lay.vec_off[c.node], c.m, 0, ins);
      in_w[c.node] = 1;
      if (c.m > 0) ic.push_back({nr * (vs + lay.vec_off[c.node]), nr * lay.vec_off[c.node], nr * c.m, 0});
    }
    // x_I = A_II^{-1} v_I - Z x_S (= L^{-T} (L^{-1} v_I - W x_S)), into w_I
    // and then copied to v_I: the separator values of every interior are
    // gathered into one contiguous vector in Z's column order, so each row of
    // Z (a column of Z^T) is a single dense dot product, as is each row of
    // the symmetric A_II^{-1}
    std::vector<int> gidx;
    std::vector<int64_t> goff(R.in.size());
    for (size_t a = 0; a < R.in.size(); ++a) {
      const auto& r = R.in[a];
      goff[a] = (int64_t)gidx.size();
      gidx.resize(gidx.size() + r.s);
      for (auto [S, col] : r.nb)
        for (int j = 0; j < lay.m[S]; ++j) gidx[goff[a] + col + j] = (int)((in_w[S] ? vs : 0) + lay.vec_off[S] + j);
    }
    T* xs = nullptr;
    if (!gidx.empty()) {
      xs = (T*)dev_malloc_async(sizeof(T) * gidx.size() * nr, s);
      P.mem.push_back(xs);
    }
    for (size_t a = 0; a < R.in.size(); ++a) {
      const auto& r = R.in[a];
      std::vector<typename GemvList<T>::In> ins = {{r.Ai, r.ldm, v + nr * lay.vec_off[r.node], nullptr, r.m, false, T(1)}};
      if (r.s > 0) ins.push_back({r.Zt, r.lds, xs + nr * goff[a], nullptr, r.s, false, T(-1)});
      b3.add(w + nr * lay.vec_off[r.node], r.m, 0, ins);
      if (r.m > 0) ic.push_back({nr * (vs + lay.vec_off[r.node]), nr * lay.vec_off[r.node], nr * r.m, 0});
    }
    b2.emit(P, s);
    if (!gidx.empty()) {
      const size_t oi = P.b.push(gidx);
      const int ng = (int)gidx.size(), r = nr;
      const T* src = v;
      P.acct.push_back({P_VECCOPY, 0.0, 2.0 * sizeof(T) * ng * r + 4.0 * ng});
      P.ops.push_back([=](const char* d, cudaStream_t st) {
        launch_vgather<T>(src, (const int*)(d + oi), xs, ng, r, st);
      });
    }
    b3.emit(P, s);
    veccopy(P, ic, v, v);
  }

  // y = A_l x: the factors applied in the opposite order (G^T, B^T up, top
  // L L^T, then B, G down)
  void build_forward(Program<T>& P, int nr, cudaStream_t s) {
    const int nl = (int)lev_.size();
    for (int t = 0; t < nl; ++t) {
      const LevelRec<T>& R = lev_[t];
      const auto& lay = R.lay;
      const int64_t vs = lay.vec_size;
      T* v = base(t);
      T* w = v + vs * nr;
      T* kp = v + 2 * vs * nr;
      GemvList<T> a1(nr), a2(nr), c1(nr), c2(nr);
      a1.trans = c1.trans = c2.trans = true;
      for (const auto& r : R.in) {
        a1.add(w + nr * lay.vec_off[r.node], r.m, 0, {{r.L, r.m, v + nr * lay.vec_off[r.node], nullptr, r.m, true, T(1)}});
        std::vector<typename GemvList<T>::In> ins;
        for (auto [S, col] : r.nb)
          ins.push_back({r.W + (size_t)col * r.m, r.m, v + nr * lay.vec_off[S], nullptr, lay.m[S], false, T(1)});
        a2.add(w + nr * lay.vec_off[r.node], r.m, 1, ins);
      }
      for (const auto& c : R.sep) {
        if (!c.comp) continue;
        c1.add(w + nr * lay.vec_off[c.node], c.m, 0, {{c.L, c.m, v + nr * lay.vec_off[c.node], nullptr, c.m, true, T(1)}});
        c2.add(kp + nr * lay.vec_off[c.node], c.k, 0, {{c.Q1, c.m, w + nr * lay.vec_off[c.node], nullptr, c.m, false, T(1)}});
      }
      a1.emit(P, s);
      a2.emit(P, s);
      c1.emit(P, s);
      c2.emit(P, s);
      std::vector<VecCopyTask> vc;
      for (const auto& c : R.sep)
        if (c.k > 0) vc.push_back({nr * ((c.comp ? 2 * vs : 0) + lay.vec_off[c.node]), nr * c.dst, nr * c.k, 0});
      veccopy(P, vc, v, base(t + 1));
    }
    {
      T* v = vtop_;
      T* w = vtop_ + (size_t)mtop_ * nr;
      GemvList<T> a(nr), bn(nr);
      a.trans = true;
      a.add(w, mtop_, 0, {{Ltop_, mtop_, v, nullptr, mtop_, true, T(1)}});
      bn.add(v, mtop_, 0, {{Ltop_, mtop_, w, nullptr, mtop_, true, T(1)}});
      a.emit(P, s);
      bn.emit(P, s);
    }
    for (int t = nl - 1; t >= 0; --t) {
      const LevelRec<T>& R = lev_[t];
      const auto& lay = R.lay;
      const int64_t vs = lay.vec_size;
      T* v = base(t);
      T* w = v + vs * nr;
      T* kp = v + 2 * vs * nr;
      T* vn = base(t + 1);
      std::vector<VecCopyTask> vc;
      for (const auto& c : R.sep)
        if (!c.comp && c.k > 0) vc.push_back({nr * c.dst, nr * lay.vec_off[c.node], nr * c.k, 0});
      veccopy(P, vc, vn, v);
      GemvList<T> b1(nr), b2(nr), b3(nr), b4(nr);
      b3.trans = true;
      for (const auto& c : R.sep) {
        if (!c.comp) continue;
        b1.add(w + nr * lay.vec_off[c.node], c.m, 1, {{c.Q1, c.m, vn + nr * c.dst, kp + nr * lay.vec_off[c.node], c.k, false, T(1)}});
        b2.add(v + nr * lay.vec_off[c.node], c.m, 0, {{c.L, c.m, w + nr * lay.vec_off[c.node], nullptr, c.m, true, T(1)}});
      }
      // separators receive W^T x_I from their interiors, then x_I <- L_I x_I
      auto si = sep_interiors(R, (int)lay.m.size());
      for (int S = 0; S < (int)si.size(); ++S) {
        if (si[S].empty()) continue;
        std::vector<typename GemvList<T>::In> ins;
        for (auto [a, col] : si[S]) {
          const auto& r = R.in[a];
          ins.push_back({r.W + (size_t)col * r.m, r.m, w + nr * lay.vec_off[r.node], nullptr, r.m, false, T(1)});
        }
        b3.add(v + nr * lay.vec_off[S], lay.m[S], 1, ins);
      }
      for (const auto& r : R.in)
        b4.add(v + nr * lay.vec_off[r.node], r.m, 0, {{r.L, r.m, w + nr * lay.vec_off[r.node], nullptr, r.m, true, T(1)}});
      b1.emit(P, s);
      b2.emit(P, s);
      b3.emit(P, s);
      b4.emit(P, s);
    }
  }
};

}  // namespace

// Precision policy: the mixed path factors in FP32; if an FP32 pivot is not
// positive (or not finite) the whole problem is factored again in FP64, so a
// matrix that is SPD but too ill-conditioned for single precision still gets
// a factor; a genuinely non-SPD matrix fails in FP64 as well.
std::unique_ptr<FactorBase> make_factor(const Plan& plan, const double* coeffs, cudaStream_t s) {
  if (plan.opts.precision == SGF_PREC_MIXED) {
    try {
      return std::make_unique<FactorImpl<float>>(plan, coeffs, s);
    } catch (const SgfError& e) {
      if (e.code != SGF_ERR_NOT_SPD && e.code != SGF_ERR_NONFINITE) throw;
    }
    auto f = std::make_unique<FactorImpl<double>>(plan, coeffs, s);
    f->fp64_fallback = true;
    return f;
  }
  return std::make_unique<FactorImpl<double>>(plan, coeffs, s);
}

// ---------------------------------------------------------------------------
// PCG (Sec. 7), FP64 vectors; flexible beta with a single-precision factor;
// up to 8 independent recurrences advanced together (one apply per iteration)
// ---------------------------------------------------------------------------
int pcg_solve_block(FactorBase& F, const double* b, double* x, int nrhs, double rtol, int maxit,
                    cudaStream_t s, int* iters, double* relres) {
  const int64_t n = F.n;
  const int k = nrhs;
  if (k < 1 || k > 8) throw SgfError(SGF_ERR_INVALID_ARG, "block PCG takes 1..8 right-hand sides");
  const size_t kn = (size_t)k * n;
  double* buf = (double*)dev_malloc_async(sizeof(double) * (5 * kn + 8 * kDotBlocks + 64), s);
  double *r = buf, *z = r + kn, *p = z + kn, *q = p + kn, *ro = q + kn;
  double* part = ro + kn;
  // device scalars, 8 per slot: 0 r.r | 1 r.z | 2 z.ro | 3 p.q | 4-5 alpha,
  // -alpha | 6 non-finite alpha flags
  double* sc = part + 8 * kDotBlocks;
  double* coef = sc + 32;
  double* flag = sc + 48;
  double h[56];
  auto dot = [&](const double* a, const double* bb, int slot) { launch_dot_n(a, bb, n, k, part, sc + 8 * slot, s); };
  auto read = [&](int nslots) { dev_d2h(h, sc, sizeof(double) * 8 * nslots, s); };   // synchronizes
  const bool flex = F.mixed();
  // SGF_PCG_LOG=1: the recursive relative residual of the first right-hand
  // side after every iteration, to stderr
  static const bool plog = std::getenv("SGF_PCG_LOG") != nullptr;
  std::vector<double> bnorm(k), rz(k);
  std::vector<char> active(k);
  dev_memset(x, 0, kn * sizeof(double), s);
  dev_d2d(r, b, kn * sizeof(double), s);
  dot(b, b, 0);
  read(1);
  for (int j = 0; j < k; ++j) {
    bnorm[j] = std::sqrt(h[j]);
    active[j] = bnorm[j] > 0.0;
    iters[j] = 0;
  }
  int rc = SGF_OK;
  F.apply_n(r, z, k, s);
  dev_d2d(p, z, kn * sizeof(double), s);
  dot(r, z, 1);
  read(2);
  for (int j = 0; j < k; ++j) rz[j] = h[8 + j];
  int it = 0;
  auto any = [&] {
    for (int j = 0; j < k; ++j)
      if (active[j]) return true;
    return false;
  };
  // one host synchronisation per iteration: the step length is formed on the
  // device from the r.z and p.q in device memory; the host reads the
  // residual norms, the new r.z and the flags once the preconditioner ran
  while (any()) {
    if (it >= maxit) { rc = SGF_ERR_NO_CONVERGENCE; break; }
    for (int j = 0; j < k; ++j) F.spmv(p + (size_t)j * n, q + (size_t)j * n, s);
    dot(p, q, 3);
    Coef8 act{};
    for (int j = 0; j < k; ++j) act.v[j] = active[j] ? 1.0 : 0.0;
    launch_pcg_alpha(sc + 24, sc + 8, act, k, coef, flag, s);
    launch_pcg_xr(coef, p, q, x, r, flex ? ro : nullptr, n, k, s);
    ++it;
    for (int j = 0; j < k; ++j)
      if (active[j]) iters[j] = it;
    F.apply_n(r, z, k, s);
    dot(r, r, 0);
    dot(r, z, 1);
    if (flex) dot(z, ro, 2);
    read(7);
    if (plog && bnorm[0] > 0) std::fprintf(stderr, "[sgf pcg] %d %.6e\n", it, std::sqrt(h[0]) / bnorm[0]);
    Coef8 be{};
    for (int j = 0; j < k; ++j) {
      if (!active[j]) continue;
      if (h[48 + j] != 0.0) {   // this iteration's step length was not finite: x_j, r_j unchanged
        rc = SGF_ERR_NONFINITE;
        active[j] = 0;
        iters[j] = it - 1;
        continue;
      }
      if (std::sqrt(h[j]) <= rtol * bnorm[j]) { active[j] = 0; continue; }
      const double rzn = h[8 + j];
      be.v[j] = flex ? (rzn - h[16 + j]) / rz[j] : rzn / rz[j];
      rz[j] = rzn;
    }
    launch_axpy_n(be, z, p, n, k, 1, s);
  }
  // true residuals
  for (int j = 0; j < k; ++j) F.spmv(x + (size_t)j * n, q + (size_t)j * n, s);
  dev_d2d(r, b, kn * sizeof(double), s);
  Coef8 m1{};
  for (int j = 0; j < k; ++j) m1.v[j] = -1.0;
  launch_axpy_n(m1, q, r, n, k, 0, s);
  dot(r, r, 0);
  read(1);
  for (int j = 0; j < k; ++j) relres[j] = bnorm[j] > 0 ? std::sqrt(h[j]) / bnorm[j] : 0.0;
  dev_free_async(buf, s);
  return rc;
}

}  // namespace sgf
