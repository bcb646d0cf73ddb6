// Symbolic analysis for the SGF factorization (host C++).
//
// Partitions (Sec. 5.1): at level t the cut spacing is d = b * 2^(t-1); along
// an axis with N unknowns the separator layers sit at the coordinates i with
// (i+1) % d == 0 and i <= N-2, dropping the last one when fewer than d/2
// unknowns follow it.  A node is the set of unknowns sharing, on every axis,
// the same separator coordinate or the same interval between separators
// (Defs. 2.1-2.4).  Cells spanning intervals on every axis are the interiors
// eliminated by block Cholesky (Sec. 4.1); the others are separators, which
// Nest-All-All compresses when their cell dimension is >= 1 and Nest-2-All
// when it is dim-1 (Sec. 5.1).  The top level is the first without any
// separator.
//
// Block sparsity: level-1 blocks follow the stencil couplings; eliminating an
// interior couples all its separator neighbours pairwise (fill); compression
// keeps the block pattern; a level-(t+1) pair exists when two of its nodes'
// children were coupled after elimination at level t (Sec. 4.3).
//
// Node bases (Sec. 3.1): monomials of degree <= j of the local coordinates
// u = (x - c) / h of each node's cell box (u = 0 on flat axes), and the exact
// affine re-expansion matrices that express a parent's local monomials in a
// child's (Sec. 4.4 merge).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <numeric>
#include <unordered_set>
#include <vector>

#include "sgf_internal.h"

namespace sgf {

namespace {

std::vector<int> axis_separators(int N, int d) {
  std::vector<int> s;
  for (int i = 0; i <= N - 2; ++i)
    if ((i + 1) % d == 0) s.push_back(i);
  if (!s.empty() && (double)(N - 1 - s.back()) < d / 2.0) s.pop_back();
  return s;
}

// code of every coordinate: 2k inside interval k, 2k+1 on separator k
std::vector<int> axis_codes(int N, const std::vector<int>& seps) {
  std::vector<int> c(N);
  size_t k = 0;
  for (int i = 0; i < N; ++i) {
    if (k < seps.size() && seps[k] == i) {
      c[i] = 2 * (int)k + 1;
      ++k;
    } else {
      c[i] = 2 * (int)k;
    }
  }
  return c;
}

void code_extent(int N, const std::vector<int>& seps, int code, int& lo, int& hi) {
  int k = code / 2;
  if (code & 1) {
    lo = hi = seps[k];
    return;
  }
  lo = k > 0 ? seps[k - 1] + 1 : 0;
  hi = k < (int)seps.size() ? seps[k] - 1 : N - 1;
}

struct Offset { int dx, dy, dz; };

std::vector<Offset> positive_offsets(int stencil) {
  // one direction of every symmetric coupling
  if (stencil == SGF_STENCIL_5PT_2D) return {{1, 0, 0}, {0, 1, 0}};
  if (stencil == SGF_STENCIL_7PT_3D || stencil == SGF_STENCIL_7PT_FV_3D)
    return {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  std::vector<Offset> o;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int key = dx + 3 * dy + 9 * dz;
        if (key > 0) o.push_back({dx, dy, dz});
      }
  return o;
}

// monomial exponents of Pi^j in the column order of Sec. 3.1
std::vector<std::array<int, 3>> exponents(int dim, int degree) {
  std::vector<std::array<int, 3>> e = {{0, 0, 0}};
  if (dim == 3) {
    if (degree >= 1) { e.push_back({1, 0, 0}); e.push_back({0, 1, 0}); e.push_back({0, 0, 1}); }
    if (degree >= 2) {
      e.push_back({2, 0, 0}); e.push_back({0, 2, 0}); e.push_back({0, 0, 2});
      e.push_back({1, 1, 0}); e.push_back({0, 1, 1}); e.push_back({1, 0, 1});
    }
  } else {
    if (degree >= 1) { e.push_back({1, 0, 0}); e.push_back({0, 1, 0}); }
    if (degree >= 2) { e.push_back({2, 0, 0}); e.push_back({0, 2, 0}); e.push_back({1, 1, 0}); }
  }
  return e;
}

void frame_of(const int* box, double c[3], double h[3]) {
  for (int a = 0; a < 3; ++a) {
    c[a] = 0.5 * ((double)box[a] + (double)box[3 + a]);
    h[a] = 0.5 * ((double)box[3 + a] - (double)box[a]);
  }
}

double ipow(double x, int e) { return e == 0 ? 1.0 : (e == 1 ? x : x * x); }

// R (pi x pi, col-major) with Pi_parent(p) = Pi_child(p) R on the child's points
void reexpansion(const int* cbox, const int* pbox, const std::vector<std::array<int, 3>>& ex,
                 double* R) {
  double cc[3], hc[3], cp[3], hp[3], a[3], b[3];
  frame_of(cbox, cc, hc);
  frame_of(pbox, cp, hp);
  for (int ax = 0; ax < 3; ++ax) {
    a[ax] = hp[ax] > 0 ? hc[ax] / hp[ax] : 0.0;
    b[ax] = hp[ax] > 0 ? (cc[ax] - cp[ax]) / hp[ax] : 0.0;
  }
  const int pi = (int)ex.size();
  std::fill(R, R + pi * pi, 0.0);
  std::map<std::array<int, 3>, int> col;
  for (int i = 0; i < pi; ++i) col[ex[i]] = i;
  static const double binom[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
  for (int j = 0; j < pi; ++j) {
    const auto& e = ex[j];
    // (a_x u + b_x)^ex (a_y v + b_y)^ey (a_z w + b_z)^ez, expanded
    for (int kx = 0; kx <= e[0]; ++kx)
      for (int ky = 0; ky <= e[1]; ++ky)
        for (int kz = 0; kz <= e[2]; ++kz) {
          double v = binom[e[0]][kx] * ipow(a[0], kx) * ipow(b[0], e[0] - kx) *
                     binom[e[1]][ky] * ipow(a[1], ky) * ipow(b[1], e[1] - ky) *
                     binom[e[2]][kz] * ipow(a[2], kz) * ipow(b[2], e[2] - kz);
          R[col[{kx, ky, kz}] + (size_t)pi * j] += v;
        }
  }
}

// one isotropic scale per node keeps rotations rigid (1 for a single point)
void frame_rbm(const int* box, double c[3], double& s) {
  double h[3];
  frame_of(box, c, h);
  s = std::max(h[0], std::max(h[1], h[2]));
  if (!(s > 0)) s = 1.0;
}

// R (6 x 6, col-major): parent modes in the child's; u_parent = a u_child + b
void reexpansion_rbm(const int* cbox, const int* pbox, double* R) {
  double cc[3], cp[3], sc, sp;
  frame_rbm(cbox, cc, sc);
  frame_rbm(pbox, cp, sp);
  const double a = sc / sp;
  double b[3];
  for (int k = 0; k < 3; ++k) b[k] = (cc[k] - cp[k]) / sp;
  std::fill(R, R + 36, 0.0);
  for (int k = 0; k < 3; ++k) R[k + 6 * k] = 1.0;
  for (int k = 0; k < 3; ++k) {
    R[(3 + k) + 6 * (3 + k)] = a;
    // e_k x b in the translation rows of column 3 + k
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    R[i + 6 * (3 + k)] = -b[j];
    R[j + 6 * (3 + k)] = b[i];
  }
}

// 24 x 24 stiffness (row-major) of a unit-cube trilinear hexahedron with
// E = 1: B^T D B integrated by the 2 x 2 x 2 Gauss rule; node a at corner
// (a & 1, (a >> 1) & 1, (a >> 2) & 1), DOF 3 a + component.
void q1_element_stiffness(double nu, std::vector<double>& K) {
  const double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 1.0 / (2 * (1 + nu));
  double D[6][6] = {};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = lam + (i == j ? 2 * mu : 0.0);
  D[3][3] = D[4][4] = D[5][5] = mu;
  const double g[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  K.assign(24 * 24, 0.0);
  for (int gi = 0; gi < 8; ++gi) {
    const double pt[3] = {g[gi & 1], g[(gi >> 1) & 1], g[(gi >> 2) & 1]};
    double Bm[6][24] = {};
    for (int a = 0; a < 8; ++a) {
      double f[3], sg[3];
      for (int d = 0; d < 3; ++d) {
        const int cor = (a >> d) & 1;
        f[d] = cor ? pt[d] : 1.0 - pt[d];
        sg[d] = cor ? 1.0 : -1.0;
      }
      const double dx = sg[0] * f[1] * f[2], dy = f[0] * sg[1] * f[2], dz = f[0] * f[1] * sg[2];
      const int c = 3 * a;
      Bm[0][c] = dx; Bm[1][c + 1] = dy; Bm[2][c + 2] = dz;
      Bm[3][c] = dy; Bm[3][c + 1] = dx;
      Bm[4][c + 1] = dz; Bm[4][c + 2] = dy;
      Bm[5][c] = dz; Bm[5][c + 2] = dx;
    }
    double DB[6][24];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 24; ++j) {
        double acc = 0;
        for (int k = 0; k < 6; ++k) acc += D[i][k] * Bm[k][j];
        DB[i][j] = acc;
      }
    for (int i = 0; i < 24; ++i)
      for (int j = 0; j < 24; ++j) {
        double acc = 0;
        for (int k = 0; k < 6; ++k) acc += Bm[k][i] * DB[k][j];
        K[i * 24 + j] += 0.125 * acc;   // Gauss weight (1/2)^3
      }
  }
}

}  // namespace

bool tuning_valid(const sgf_tuning& t) {
  // front_small: at most the one-CTA front kernel's limit (512 rows)
  return t.gemv_min_elems >= 256 && t.gemv_min_elems <= t.gemv_max_elems && t.gemv_max_elems <= (1 << 20) &&
         t.front_small >= 64 && t.front_small <= 512 && t.tensor_cores >= 0 && t.tensor_cores <= 2 &&
         (t.gemv_cols == 32 || t.gemv_cols == 64) && t.tc_min_dim >= 1 && t.tc_min_dim <= 4096;
}

int LevelLayout::col_of(int u, int v) const {
  auto b = up_nb.begin() + up_ptr[u], e = up_nb.begin() + up_ptr[u + 1];
  auto it = std::lower_bound(b, e, v);
  if (it == e || *it != v) return -1;
  return up_col[it - up_nb.begin()];
}

void build_layout(const LevelSym& L, const std::vector<int>& m, LevelLayout& o) {
  const int nn = L.nnodes;
  o.m = m;
  o.dg_off.assign(nn, 0);
  o.vec_off.assign(nn, 0);
  int64_t off = 0, voff = 0;
  for (int i = 0; i < nn; ++i) {
    o.dg_off[i] = off;
    off += (int64_t)m[i] * m[i];
    o.vec_off[i] = voff;
    voff += m[i];
  }
  o.dg_size = off;
  o.vec_size = voff;
  // upper neighbours: interiors from the pre-elimination pattern, separators
  // from the post-elimination pattern
  std::vector<std::vector<int>> up(nn);
  for (size_t p = 0; p < L.pairs.size(); p += 2) {
    int u = L.pairs[p], v = L.pairs[p + 1];
    if (L.interior[u]) up[u].push_back(v);
  }
  for (size_t p = 0; p < L.post.size(); p += 2) up[L.post[p]].push_back(L.post[p + 1]);
  o.up_ptr.assign(nn + 1, 0);
  o.up_nb.clear();
  o.up_col.clear();
  o.up_off.assign(nn, 0);
  o.up_w.assign(nn, 0);
  off = 0;
  for (int u = 0; u < nn; ++u) {
    auto& v = up[u];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    o.up_off[u] = off;
    int col = 0;
    for (int w : v) {
      o.up_nb.push_back(w);
      o.up_col.push_back(col);
      col += m[w];
    }
    o.up_w[u] = col;
    o.up_ptr[u + 1] = (int)o.up_nb.size();
    off += (int64_t)m[u] * col;
  }
  o.up_size = off;
}

int analyze(const sgf_grid* g, int stencil, const sgf_opts* op, Plan& P, std::string& err) {
  if (!g || !op) { err = "null argument"; return SGF_ERR_INVALID_ARG; }
  if (stencil < 0 || stencil > SGF_STENCIL_Q1_ELASTIC_3D) { err = "bad stencil"; return SGF_ERR_INVALID_ARG; }
  const int dim = g->dim;
  if (dim != 2 && dim != 3) { err = "dim must be 2 or 3"; return SGF_ERR_INVALID_ARG; }
  if ((stencil == SGF_STENCIL_5PT_2D) != (dim == 2)) { err = "stencil/dim mismatch"; return SGF_ERR_INVALID_ARG; }
  const bool elastic = stencil == SGF_STENCIL_Q1_ELASTIC_3D;
  if (elastic) {
    if (g->dof != 3) { err = "Q1 elasticity has 3 DOFs per point"; return SGF_ERR_INVALID_ARG; }
    if (op->basis != SGF_BASIS_RBM) { err = "Q1 elasticity uses the rigid-body-mode basis"; return SGF_ERR_UNSUPPORTED; }
    if (g->dirichlet != SGF_FACE_XM) { err = "Q1 elasticity: only the clamped x- face"; return SGF_ERR_UNSUPPORTED; }
    if (g->n[1] < 2 || g->n[2] < 2) { err = "Q1 elasticity needs >= 2 nodes in y and z"; return SGF_ERR_INVALID_ARG; }
  } else if (g->dof != 1) {
    err = "scalar stencils have 1 DOF per point";
    return SGF_ERR_INVALID_ARG;
  }
  for (int a = 0; a < dim; ++a)
    if (g->n[a] < 1 || g->n[a] > (1 << 14)) { err = "grid size out of range"; return SGF_ERR_INVALID_ARG; }
  if (op->leaf < 2) { err = "leaf must be >= 2"; return SGF_ERR_INVALID_ARG; }
  if (op->degree < 0 || op->degree > 2) { err = "degree must be 0, 1 or 2"; return SGF_ERR_INVALID_ARG; }
  if (!elastic && op->basis != SGF_BASIS_POLY) { err = "scalar problems use the polynomial basis"; return SGF_ERR_UNSUPPORTED; }
  if (op->scheme < 0 || op->scheme > 4) { err = "bad scheme"; return SGF_ERR_INVALID_ARG; }
  const bool general = op->scheme == SGF_SCHEME_GEN_ALL_ALL;
  if (op->precision != SGF_PREC_FP64 && op->precision != SGF_PREC_MIXED) { err = "bad precision"; return SGF_ERR_INVALID_ARG; }

  P.grid = *g;
  P.stencil = stencil;
  P.opts = *op;
  P.nx = g->n[0];
  P.ny = g->n[1];
  P.nz = dim == 3 ? g->n[2] : 1;
  P.npts = (int64_t)P.nx * P.ny * P.nz;
  if (P.npts > (int64_t)1 << 30) { err = "grid too large"; return SGF_ERR_INVALID_ARG; }
  P.dof = g->dof;
  P.n = P.npts * P.dof;
  const auto ex = exponents(dim, op->degree);
  P.pi = elastic ? 6 : (int)ex.size();
  P.nu = op->nu > 0 ? op->nu : 0.3;
  if (elastic && !(P.nu < 0.5)) { err = "Poisson ratio must be < 0.5"; return SGF_ERR_INVALID_ARG; }
  P.tau = op->tau > 0 ? op->tau : (op->precision == SGF_PREC_MIXED ? 1e-6 : 1e-12);
  const int N[3] = {P.nx, P.ny, P.nz};

  std::vector<int> prev_node_of_point;  // level-t node of every point
  int t = 1;
  while (true) {
    LevelSym L;
    L.t = t;
    const int64_t dd = (int64_t)op->leaf << (t - 1);
    L.d = dd > (1 << 30) ? (1 << 30) : (int)dd;
    std::vector<int> seps[3];
    bool any = false;
    int KG[3] = {1, 1, 1};   // general partitions: cells per axis
    for (int a = 0; a < 3; ++a) {
      if (general) {
        if (N[a] > 1) KG[a] = (N[a] + L.d - 1) / L.d;
        any = any || KG[a] > 1;
      } else {
        if (N[a] > 1) seps[a] = axis_separators(N[a], L.d);
        any = any || !seps[a].empty();
      }
    }
    if (!any) {
      L.top = true;
      L.nnodes = 1;
      L.code = {0, 0, 0};
      L.interior = {0};
      L.cell_dim = {dim};
      L.box = {0, 0, 0, P.nx - 1, P.ny - 1, P.nz - 1};
      L.eligible = {0};
      if (P.lev.empty()) {
        L.pt_ptr = {0, (int)P.npts};
        L.pt_idx.resize(P.npts);
        std::iota(L.pt_idx.begin(), L.pt_idx.end(), 0);
      } else {
        const LevelSym& pv = P.lev.back();
        L.child_ptr = {0};
        for (int c = 0; c < pv.nnodes; ++c)
          if (!pv.interior[c]) L.child_idx.push_back(c);
        L.child_ptr.push_back((int)L.child_idx.size());
      }
      P.lev.push_back(std::move(L));
      break;
    }
    std::vector<int> cx, cy, cz;
    int KX, KY, KZ;
    if (general) {   // code 2k for the k-th run of d vertices (no separator codes)
      auto gcodes = [&](int n) {
        std::vector<int> c(n);
        for (int i = 0; i < n; ++i) c[i] = 2 * (i / L.d);
        return c;
      };
      cx = gcodes(P.nx);
      cy = gcodes(P.ny);
      cz = gcodes(P.nz);
      KX = 2 * KG[0] - 1;
      KY = 2 * KG[1] - 1;
      KZ = 2 * KG[2] - 1;
    } else {
      cx = axis_codes(P.nx, seps[0]);
      cy = axis_codes(P.ny, seps[1]);
      cz = axis_codes(P.nz, seps[2]);
      KX = 2 * (int)seps[0].size() + 1;
      KY = 2 * (int)seps[1].size() + 1;
      KZ = 2 * (int)seps[2].size() + 1;
    }
    // enumerate cells, sort interiors first then by (z, y, x) code
    struct Cell { int z, y, x; bool in; };
    std::vector<Cell> cells;
    cells.reserve((size_t)KX * KY * KZ);
    for (int z = 0; z < KZ; ++z)
      for (int y = 0; y < KY; ++y)
        for (int x = 0; x < KX; ++x) {
          if (general && (x % 2 || y % 2 || z % 2)) continue;   // no separator cells
          cells.push_back({z, y, x, !general && (x % 2 == 0) && (y % 2 == 0) && (z % 2 == 0)});
        }
    std::stable_sort(cells.begin(), cells.end(), [](const Cell& a, const Cell& b) {
      if (a.in != b.in) return a.in;
      if (a.z != b.z) return a.z < b.z;
      if (a.y != b.y) return a.y < b.y;
      return a.x < b.x;
    });
    L.nnodes = (int)cells.size();
    std::vector<int> table((size_t)KX * KY * KZ);
    L.code.resize(3 * L.nnodes);
    L.interior.resize(L.nnodes);
    L.cell_dim.resize(L.nnodes);
    L.box.resize(6 * L.nnodes);
    L.eligible.resize(L.nnodes);
    for (int i = 0; i < L.nnodes; ++i) {
      const Cell& c = cells[i];
      table[((size_t)c.z * KY + c.y) * KX + c.x] = i;
      L.code[3 * i] = c.z;
      L.code[3 * i + 1] = c.y;
      L.code[3 * i + 2] = c.x;
      L.interior[i] = c.in;
      int cd = (c.x % 2 == 0) + (c.y % 2 == 0) + (dim == 3 ? (c.z % 2 == 0) : 0);
      L.cell_dim[i] = cd;
      const int cc[3] = {c.x, c.y, c.z};
      for (int a = 0; a < 3; ++a) {
        if (general) {
          L.box[6 * i + a] = (cc[a] / 2) * L.d;
          L.box[6 * i + 3 + a] = std::min((cc[a] / 2 + 1) * L.d, N[a]) - 1;
        } else {
          code_extent(N[a], seps[a], cc[a], L.box[6 * i + a], L.box[6 * i + 3 + a]);
        }
      }
      bool el = false;
      if (!c.in && t >= std::max(1, op->compress_from_level)) {
        if (op->scheme == SGF_SCHEME_NEST_ALL_ALL) el = cd >= 1;
        else if (op->scheme == SGF_SCHEME_NEST_2_ALL || op->scheme == SGF_SCHEME_NEST_2_2) el = cd == dim - 1;
        else if (op->scheme == SGF_SCHEME_GEN_ALL_ALL) el = true;
      }
      L.eligible[i] = el;
    }
    std::vector<int> node_of_point(P.npts);
    for (int64_t p = 0; p < P.npts; ++p) {
      int x = (int)(p % P.nx), y = (int)((p / P.nx) % P.ny), z = (int)(p / ((int64_t)P.nx * P.ny));
      node_of_point[p] = table[((size_t)cz[z] * KY + cy[y]) * KX + cx[x]];
    }
    if (P.lev.empty()) {
      L.pt_ptr.assign(L.nnodes + 1, 0);
      for (int64_t p = 0; p < P.npts; ++p) L.pt_ptr[node_of_point[p] + 1]++;
      for (int i = 0; i < L.nnodes; ++i) L.pt_ptr[i + 1] += L.pt_ptr[i];
      L.pt_idx.resize(P.npts);
      std::vector<int> fill(L.pt_ptr.begin(), L.pt_ptr.end() - 1);
      for (int64_t p = 0; p < P.npts; ++p) L.pt_idx[fill[node_of_point[p]]++] = (int)p;
    } else {
      const LevelSym& pv = P.lev.back();
      std::vector<std::vector<int>> kids(L.nnodes);
      for (int c = 0; c < pv.nnodes; ++c) {
        if (pv.interior[c]) continue;
        const int* b = &pv.box[6 * c];
        int64_t p = b[0] + (int64_t)P.nx * (b[1] + (int64_t)P.ny * b[2]);
        kids[node_of_point[p]].push_back(c);
      }
      L.child_ptr.assign(1, 0);
      for (int i = 0; i < L.nnodes; ++i) {
        for (int c : kids[i]) L.child_idx.push_back(c);
        L.child_ptr.push_back((int)L.child_idx.size());
      }
    }
    prev_node_of_point.swap(node_of_point);
    P.lev.push_back(std::move(L));
    ++t;
    if (t > 40) { err = "too many levels"; return SGF_ERR_INVALID_ARG; }
  }
  // children of the top level need the same treatment (handled above)

  // ---- block patterns -------------------------------------------------
  auto finish_post = [&](LevelSym& L) {
    std::vector<std::vector<int>> nb(L.nnodes);
    for (size_t p = 0; p < L.pairs.size(); p += 2) {
      nb[L.pairs[p]].push_back(L.pairs[p + 1]);
      nb[L.pairs[p + 1]].push_back(L.pairs[p]);
    }
    std::vector<int64_t> keys;
    for (size_t p = 0; p < L.pairs.size(); p += 2) {
      int u = L.pairs[p], v = L.pairs[p + 1];
      if (!L.interior[u] && !L.interior[v]) keys.push_back((int64_t)u * L.nnodes + v);
    }
    for (int I = 0; I < L.nnodes; ++I) {
      if (!L.interior[I]) continue;
      auto& s = nb[I];
      std::sort(s.begin(), s.end());
      for (size_t a = 0; a < s.size(); ++a)
        for (size_t b = a + 1; b < s.size(); ++b) keys.push_back((int64_t)s[a] * L.nnodes + s[b]);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    L.post.clear();
    for (int64_t k : keys) {
      L.post.push_back((int)(k / L.nnodes));
      L.post.push_back((int)(k % L.nnodes));
    }
  };
  if (!P.lev[0].top) {
    LevelSym& L1 = P.lev[0];
    std::vector<int> node_of(P.npts);
    for (int i = 0; i < L1.nnodes; ++i)
      for (int k = L1.pt_ptr[i]; k < L1.pt_ptr[i + 1]; ++k) node_of[L1.pt_idx[k]] = i;
    std::vector<int64_t> keys;
    for (auto o : positive_offsets(stencil)) {
      for (int64_t p = 0; p < P.npts; ++p) {
        int x = (int)(p % P.nx), y = (int)((p / P.nx) % P.ny), z = (int)(p / ((int64_t)P.nx * P.ny));
        int qx = x + o.dx, qy = y + o.dy, qz = z + o.dz;
        if (qx < 0 || qx >= P.nx || qy < 0 || qy >= P.ny || qz < 0 || qz >= P.nz) continue;
        int u = node_of[p], v = node_of[qx + (int64_t)P.nx * (qy + (int64_t)P.ny * qz)];
        if (u == v) continue;
        keys.push_back((int64_t)std::min(u, v) * L1.nnodes + std::max(u, v));
      }
      std::sort(keys.begin(), keys.end());
      keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    }
    for (int64_t k : keys) {
      L1.pairs.push_back((int)(k / L1.nnodes));
      L1.pairs.push_back((int)(k % L1.nnodes));
    }
    finish_post(L1);
    for (size_t li = 1; li < P.lev.size(); ++li) {
      LevelSym& L = P.lev[li];
      const LevelSym& pv = P.lev[li - 1];
      if (L.top) break;
      std::vector<int> parent(pv.nnodes, -1);
      for (int D = 0; D < L.nnodes; ++D)
        for (int k = L.child_ptr[D]; k < L.child_ptr[D + 1]; ++k) parent[L.child_idx[k]] = D;
      std::vector<int64_t> pk;
      for (size_t p = 0; p < pv.post.size(); p += 2) {
        int a = parent[pv.post[p]], b = parent[pv.post[p + 1]];
        if (a != b) pk.push_back((int64_t)std::min(a, b) * L.nnodes + std::max(a, b));
      }
      std::sort(pk.begin(), pk.end());
      pk.erase(std::unique(pk.begin(), pk.end()), pk.end());
      for (int64_t k : pk) {
        L.pairs.push_back((int)(k / L.nnodes));
        L.pairs.push_back((int)(k % L.nnodes));
      }
      finish_post(L);
    }
  }

  // ---- bases and re-expansion (Sec. 3.1, Sec. 4.4) ---------------------
  {
    const LevelSym& L1 = P.lev[0];
    P.phi1_off.assign(L1.nnodes + 1, 0);
    for (int i = 0; i < L1.nnodes; ++i)
      P.phi1_off[i + 1] = P.phi1_off[i] + (int64_t)(L1.pt_ptr[i + 1] - L1.pt_ptr[i]) * P.dof * P.pi;
    P.phi1.assign(P.phi1_off.back(), 0.0);
    for (int i = 0; elastic && i < L1.nnodes; ++i) {
      // rigid-body modes (Sec. 7.2): translations, rotations about x, y, z in
      // local coordinates (x - c) / s with one scale per node
      double c[3], s;
      frame_rbm(&L1.box[6 * i], c, s);
      const int np = L1.pt_ptr[i + 1] - L1.pt_ptr[i], m = 3 * np;
      double* F = &P.phi1[P.phi1_off[i]];
      for (int r = 0; r < np; ++r) {
        const int64_t p = L1.pt_idx[L1.pt_ptr[i] + r];
        const double u = ((double)(p % P.nx) - c[0]) / s, v = ((double)((p / P.nx) % P.ny) - c[1]) / s,
                     w = ((double)(p / ((int64_t)P.nx * P.ny)) - c[2]) / s;
        for (int k = 0; k < 3; ++k) F[3 * r + k + (size_t)m * k] = 1.0;
        F[3 * r + 1 + (size_t)m * 3] = -w; F[3 * r + 2 + (size_t)m * 3] = v;
        F[3 * r + 0 + (size_t)m * 4] = w;  F[3 * r + 2 + (size_t)m * 4] = -u;
        F[3 * r + 0 + (size_t)m * 5] = -v; F[3 * r + 1 + (size_t)m * 5] = u;
      }
    }
    for (int i = 0; !elastic && i < L1.nnodes; ++i) {
      double c[3], h[3];
      frame_of(&L1.box[6 * i], c, h);
      const int m = L1.pt_ptr[i + 1] - L1.pt_ptr[i];
      double* F = &P.phi1[P.phi1_off[i]];
      for (int r = 0; r < m; ++r) {
        int64_t p = L1.pt_idx[L1.pt_ptr[i] + r];
        double xyz[3] = {(double)(p % P.nx), (double)((p / P.nx) % P.ny), (double)(p / ((int64_t)P.nx * P.ny))};
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = h[a] > 0 ? (xyz[a] - c[a]) / h[a] : 0.0;
        for (int j = 0; j < P.pi; ++j)
          F[r + (size_t)m * j] = ipow(u[0], ex[j][0]) * ipow(u[1], ex[j][1]) * ipow(u[2], ex[j][2]);
      }
    }
    for (size_t li = 1; li < P.lev.size(); ++li) {
      LevelSym& L = P.lev[li];
      const LevelSym& pv = P.lev[li - 1];
      L.reexp.assign(L.child_idx.size() * (size_t)P.pi * P.pi, 0.0);
      for (int D = 0; D < L.nnodes; ++D)
        for (int k = L.child_ptr[D]; k < L.child_ptr[D + 1]; ++k) {
          double* R = &L.reexp[(size_t)k * P.pi * P.pi];
          if (elastic) reexpansion_rbm(&pv.box[6 * L.child_idx[k]], &L.box[6 * D], R);
          else reexpansion(&pv.box[6 * L.child_idx[k]], &L.box[6 * D], ex, R);
        }
    }
  }

  // ---- basis columns that can be nonzero on each node -------------------
  for (auto& L : P.lev) {
    L.act.assign(L.nnodes, 0);
    for (int i = 0; i < L.nnodes; ++i) {
      if (elastic) {
        // translations, plus a rotation about axis k when another axis varies
        bool var[3];
        for (int a = 0; a < 3; ++a) var[a] = L.box[6 * i + a] != L.box[6 * i + 3 + a];
        int cnt = 3;
        for (int k = 0; k < 3; ++k) cnt += var[(k + 1) % 3] || var[(k + 2) % 3];
        L.act[i] = cnt;
        continue;
      }
      int cnt = 0;
      for (const auto& e : ex) {
        bool ok = true;
        for (int a = 0; a < 3; ++a)
          if (e[a] > 0 && L.box[6 * i + a] == L.box[6 * i + 3 + a]) ok = false;
        cnt += ok;
      }
      L.act[i] = cnt;
    }
  }

  // ---- level-1 assembly destinations -----------------------------------
  if (elastic) {
    const LevelSym& L1 = P.lev[0];
    std::vector<int> m1(L1.nnodes);
    for (int i = 0; i < L1.nnodes; ++i) m1[i] = (L1.pt_ptr[i + 1] - L1.pt_ptr[i]) * 3;
    LevelLayout lay;
    build_layout(L1, m1, lay);
    std::vector<int> node_of(P.npts), lpos(P.npts);
    P.perm1.assign(P.n, 0);
    for (int u = 0; u < L1.nnodes; ++u)
      for (int k = L1.pt_ptr[u]; k < L1.pt_ptr[u + 1]; ++k) {
        const int p = L1.pt_idx[k];
        node_of[p] = u;
        lpos[p] = k - L1.pt_ptr[u];
        for (int c = 0; c < 3; ++c) P.perm1[lay.vec_off[u] + 3 * lpos[p] + c] = 3 * (int64_t)p + c;
      }
    // per point and neighbour offset (dx + 3 dy + 9 dz over {-1,0,1}^3): the
    // offset of the 3x3 block's (0, 0) entry in [diagonal blocks | panels]
    P.asm_map.assign(P.npts * 27, -1);
    for (int64_t p = 0; p < P.npts; ++p) {
      const int x = (int)(p % P.nx), y = (int)((p / P.nx) % P.ny), z = (int)(p / ((int64_t)P.nx * P.ny));
      const int u = node_of[p], lp = lpos[p];
      for (int o = 0; o < 27; ++o) {
        const int qx = x + o % 3 - 1, qy = y + (o / 3) % 3 - 1, qz = z + o / 9 - 1;
        if (qx < 0 || qx >= P.nx || qy < 0 || qy >= P.ny || qz < 0 || qz >= P.nz) continue;
        const int64_t q = qx + (int64_t)P.nx * (qy + (int64_t)P.ny * qz);
        const int v = node_of[q], lq = lpos[q];
        if (u == v) {
          P.asm_map[p * 27 + o] = lay.dg_off[u] + 3 * lp + (int64_t)3 * lq * m1[u];
        } else if (u < v) {
          const int col = lay.col_of(u, v);
          if (col < 0) { err = "internal: missing level-1 block"; return SGF_ERR_INVALID_ARG; }
          P.asm_map[p * 27 + o] = lay.dg_size + lay.up_off[u] + (int64_t)(col + 3 * lq) * m1[u] + 3 * lp;
        }
      }
    }
    P.asm_ld.assign(P.npts, 0);
    for (int64_t p = 0; p < P.npts; ++p) P.asm_ld[p] = m1[node_of[p]];
    q1_element_stiffness(P.nu, P.kref);
  } else {
    const LevelSym& L1 = P.lev[0];
    std::vector<int> m1(L1.nnodes);
    for (int i = 0; i < L1.nnodes; ++i) m1[i] = (L1.pt_ptr[i + 1] - L1.pt_ptr[i]) * P.dof;
    LevelLayout lay;
    build_layout(L1, m1, lay);
    std::vector<int> node_of(P.npts), lpos(P.npts);
    P.perm1.assign(P.npts, 0);
    for (int u = 0; u < L1.nnodes; ++u)
      for (int k = L1.pt_ptr[u]; k < L1.pt_ptr[u + 1]; ++k) {
        const int p = L1.pt_idx[k];
        node_of[p] = u;
        lpos[p] = k - L1.pt_ptr[u];
        P.perm1[lay.vec_off[u] + lpos[p]] = p;
      }
    P.asm_map.assign(P.npts * 7, -1);
    const int64_t nxy = (int64_t)P.nx * P.ny;
    for (int64_t p = 0; p < P.npts; ++p) {
      const int x = (int)(p % P.nx), y = (int)((p / P.nx) % P.ny), z = (int)(p / nxy);
      const int u = node_of[p], lp = lpos[p];
      const int64_t nbq[6] = {x > 0 ? p - 1 : -1, x < P.nx - 1 ? p + 1 : -1,
                              y > 0 ? p - P.nx : -1, y < P.ny - 1 ? p + P.nx : -1,
                              z > 0 ? p - nxy : -1, z < P.nz - 1 ? p + nxy : -1};
      for (int q = 0; q < 6; ++q) {
        if (nbq[q] < 0) continue;
        const int v = node_of[nbq[q]], lq = lpos[nbq[q]];
        if (u == v) {
          P.asm_map[p * 7 + q] = lay.dg_off[u] + lp + (int64_t)lq * m1[u];
        } else if (u < v) {
          const int col = lay.col_of(u, v);
          if (col < 0) { err = "internal: missing level-1 block"; return SGF_ERR_INVALID_ARG; }
          P.asm_map[p * 7 + q] = lay.dg_size + lay.up_off[u] + (int64_t)(col + lq) * m1[u] + lp;
        }
      }
      P.asm_map[p * 7 + 6] = lay.dg_off[u] + lp + (int64_t)lp * m1[u];
    }
  }

  // ---- structural size bounds (no compression) -------------------------
  P.mcap.resize(P.lev.size());
  for (size_t li = 0; li < P.lev.size(); ++li) {
    const LevelSym& L = P.lev[li];
    P.mcap[li].assign(L.nnodes, 0);
    for (int i = 0; i < L.nnodes; ++i) {
      if (li == 0) {
        P.mcap[li][i] = (L.pt_ptr[i + 1] - L.pt_ptr[i]) * P.dof;
      } else {
        int s = 0;
        for (int k = L.child_ptr[i]; k < L.child_ptr[i + 1]; ++k) s += P.mcap[li - 1][L.child_idx[k]];
        P.mcap[li][i] = s;
      }
    }
  }
  return SGF_OK;
}

}  // namespace sgf
