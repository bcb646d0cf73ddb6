"""Sparse Geometric Factorization, Algorithm 4.1, restated step by step in FP64.

The current matrix is kept as a dictionary of dense blocks between the nodes
of the current level (key (u, v) with u <= v; the (v, u) block is the
transpose).  Each level does, in the paper's order:

1. Elimination of every interior I (Sec. 4.1, Eq. (elimination)):
   L = chol(A_II), W_S = L^{-1} A_IS for each neighbour S, and
   A_SS' <- A_SS' - W_S^T W_S' for every pair of neighbours (fill included).
2. Compression of every selected separator B, one after the other on the
   current matrix (Sec. 3.2 and Sec. 4.2):
   scale with M_BB = L L^T (Eq. (compr-scale)), M^_BN = L^{-1} M_BN;
   filtered interaction matrix N = [L^T Phi_B, M^_BN1 Phi_N1, ...]
   (Eq. (N-definition)); column-pivoted QR  N P = Q R  (Eq. (QR), LAPACK
   geqp3 as in Sec. 7); rank r = #{k : |R_kk| > tau |R_11|}; Q1 = Q[:, :r].
   The node is compressed when r < m: its block row becomes
   [I_r | Q1^T M^_BN ...], the Q2 variables decouple with identity diagonal
   (Eq. (M')), and Phi_B <- Q1^T L^T Phi_B (Eq. (phi-update)).  When r = m the
   node is left as it is: with Q square the step is only a change of basis.
3. Coarsening (Sec. 4.3) and Phi merge (Sec. 4.4): every parent node gathers
   its children's surviving variables, the blocks between them, and the
   stacked children's Phi (re-expressed in the parent's local monomials).
4. At the top level (one node) an exact Cholesky factorization (Sec. 4.5).

The apply of A_l^{-1} (Sec. 4.7) runs the recorded factors forward
(G^{-1}, B^{-1} per level, merge), solves with the top factor, and runs them
backward (B^{-T}, G^{-T}).  `multiply` applies A_l itself (the factors in the
opposite order), which is what the preservation checks of Prop. 6.1 need.

Readings (the paper leaves these open):
* tau = 1e-12 relative to |R_11| (the paper only says "e.g. pivoted QR");
* 0-cells are never compressed (Sec. 5.1 notes it makes no difference);
* Nest-2-All compresses only separators of codimension 1;
* Nest-2-2 (Sec. 5.1) compresses the same nodes, with the scaled blocks
  M^_BE = L^{-1} A_BE to every lower-dimensional separator E whose box
  touches B's (at most one grid step apart on every axis) appended to N as
  whole columns, so span(Q1) holds them and those interactions are kept
  exactly; one pivoted QR with the usual rank rule gives Q1;
* scheme "none" disables compression, which gives exact block Cholesky;
* Gen-All-All (Sec. 5.2) runs on general partitions
  (build_hierarchy(general=True)): no interiors, every node is compressed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from .basis import Basis
from .partition import Hierarchy


@dataclass
class Options:
    scheme: str = "nest_all_all"     # "nest_all_all" | "nest_2_all" | "nest_2_2" | "gen_all_all" | "none"
    tau: float = 1e-12
    compress_from_level: int = 1
    basis: str = "poly"              # "poly" | "rbm"
    degree: int = 2
    order: str = "sequential"        # "sequential" (Sec. 3.2 recursion) | "level"
    # sensitivity probe for tests: perturb every entry of N by a relative
    # rounding-level amount (seeded) before the pivoted QR
    qr_noise: float = 0.0
    qr_noise_seed: int = 0


def _eligible(lev, i, dim, opts: Options) -> bool:
    if opts.scheme == "none" or lev.t < opts.compress_from_level or lev.interior[i]:
        return False
    cd = int(lev.cell_dim[i])
    if opts.scheme == "nest_all_all":
        return cd >= 1
    if opts.scheme in ("nest_2_all", "nest_2_2"):
        return cd == dim - 1
    if opts.scheme == "gen_all_all":   # Sec. 5.2: every node of a general partition
        return True
    raise ValueError(opts.scheme)


def adjacent_low(lev, B, X, dim) -> bool:
    """Nest-2-2: X is a separator of lower dimension than the compressed
    cells (cell_dim < dim - 1) whose box touches B's box."""
    if lev.interior[X] or int(lev.cell_dim[X]) >= dim - 1:
        return False
    lo_b, hi_b = lev.box[B]
    lo_x, hi_x = lev.box[X]
    gap = np.maximum(0, np.maximum(lo_x - hi_b, lo_b - hi_x))
    return bool(np.all(gap <= 1))


def _get(blk, u, v):
    return blk[(u, v)] if u <= v else blk[(v, u)].T


def _set(blk, u, v, X):
    if u <= v:
        blk[(u, v)] = X
    else:
        blk[(v, u)] = X.T


def point_coords(H: Hierarchy) -> np.ndarray:
    nx, ny, nz = H.n
    p = np.arange(nx * ny * nz)
    return np.stack([p % nx, (p // nx) % ny, p // (nx * ny)], axis=1).astype(np.float64)


def dof_list(points, dof):
    if dof == 1:
        return np.asarray(points, dtype=np.int64)
    return (dof * np.asarray(points, dtype=np.int64)[:, None] + np.arange(dof)[None, :]).ravel()


class SGFFactor:
    """The factors of A_l for one matrix A on one hierarchy."""

    def __init__(self, A, H: Hierarchy, opts: Options = Options(), order_seed=None):
        self.A = A.tocsr()
        self.H = H
        self.opts = opts
        self.basis = Basis(H.dim, opts.degree, opts.basis, H.dof)
        self.order_seed = order_seed
        self.ops = []
        self.comp_info = {}     # (t, node) -> dict(m, r, ncols, q2n, nnorm)
        self.pivots_min = np.inf
        self._factorize()

    # ------------------------------------------------------------------ factor
    def _chol(self, X):
        L = sla.cholesky(X, lower=True)
        self.pivots_min = min(self.pivots_min, float(np.min(np.diag(L))))
        return L

    def _factorize(self):
        H, A, dof, opts = self.H, self.A, self.H.dof, self.opts
        xyz = point_coords(H)
        lev1 = H.levels[0]
        self.vars1 = [dof_list(p, dof) for p in lev1.points]
        sizes = {i: len(v) for i, v in enumerate(self.vars1)}
        blk = {}
        for i, v in enumerate(self.vars1):
            blk[(i, i)] = A[v][:, v].toarray()
        nbr = {i: set() for i in range(lev1.nnodes)}
        for (u, v) in lev1.pattern:
            blk[(u, v)] = A[self.vars1[u]][:, self.vars1[v]].toarray()
            nbr[u].add(v)
            nbr[v].add(u)
        phi = {i: self.basis.evaluate(xyz[lev1.points[i]], lev1.box[i]) for i in range(lev1.nnodes)}
        rng = np.random.default_rng(self.order_seed) if self.order_seed is not None else None
        noise_rng = np.random.default_rng(opts.qr_noise_seed)

        for li, lev in enumerate(H.levels):
            t = lev.t
            if lev.top:
                L = self._chol(blk[(0, 0)])
                self.ops.append(("top", L))
                break
            # 1. eliminate interiors
            for I in lev.interiors():
                S_list = sorted(nbr[I])
                if sizes[I] == 0:
                    # an interior whose region holds no surviving variable
                    for S in S_list:
                        nbr[S].discard(I)
                        del blk[(min(I, S), max(I, S))]
                    del blk[(I, I)]
                    del nbr[I]
                    continue
                L = self._chol(blk[(I, I)])
                W = [sla.solve_triangular(L, _get(blk, I, S), lower=True) for S in S_list]
                for a, S in enumerate(S_list):
                    for b in range(a, len(S_list)):
                        S2 = S_list[b]
                        upd = W[a].T @ W[b]
                        key = (min(S, S2), max(S, S2))
                        if key in blk:
                            _set(blk, S, S2, _get(blk, S, S2) - upd)
                        else:
                            _set(blk, S, S2, -upd)
                            nbr[S].add(S2)
                            nbr[S2].add(S)
                for S in S_list:
                    nbr[S].discard(I)
                    del blk[(min(I, S), max(I, S))]
                del blk[(I, I)]
                del nbr[I]
                self.ops.append(("elim", t, I, L, S_list, W))
            # 2. compress selected separators, sequentially on the current matrix
            order = [B for B in lev.separators() if _eligible(lev, B, H.dim, opts)]
            if rng is not None:
                order = [order[k] for k in rng.permutation(len(order))]
            # "level": every node sees the post-elimination matrix (see below)
            src_blk, src_phi = (dict(blk), dict(phi)) if opts.order == "level" else (blk, phi)
            level_q = {}
            for B in order:
                m = sizes[B]
                N_list = sorted(nbr[B])
                L = self._chol(_get(src_blk, B, B))
                Mh = [sla.solve_triangular(L, _get(src_blk, B, N), lower=True) for N in N_list]
                cols = [L.T @ src_phi[B]] + [Mh[k] @ src_phi[N] for k, N in enumerate(N_list)]
                adj = [Mh[k] for k, N in enumerate(N_list)
                       if opts.scheme == "nest_2_2" and adjacent_low(lev, B, N, H.dim)]
                Nmat = np.hstack(cols + adj)
                if opts.qr_noise > 0:
                    Nmat = Nmat * (1.0 + opts.qr_noise * noise_rng.standard_normal(Nmat.shape))
                Q, R, _ = sla.qr(Nmat, pivoting=True)
                d = np.abs(np.diag(R))
                r = int(np.sum(d > opts.tau * d[0])) if d.size and d[0] > 0 else 0
                A_adj = np.hstack(adj) if adj else np.zeros((m, 0))
                info = dict(m=m, r=r, ncols=Nmat.shape[1], nnorm=float(np.linalg.norm(Nmat)),
                            adj_cols=A_adj.shape[1], adj_norm=float(np.linalg.norm(A_adj)),
                            adj_q2=float(np.linalg.norm(Q[:, r:].T @ A_adj)) if r < m else 0.0,
                            rdiag=d / d[0] if d.size and d[0] > 0 else d,
                            q2n=float(np.linalg.norm(Q[:, r:].T @ Nmat)) if r < m else 0.0,
                            compressed=r < m)
                self.comp_info[(t, B)] = info
                if r < m:
                    Q1 = Q[:, :r]
                    if opts.order == "level":
                        level_q[B] = (L, Q1)
                    else:
                        blk[(B, B)] = np.eye(r)
                        for k, N in enumerate(N_list):
                            _set(blk, B, N, Q1.T @ Mh[k])
                    phi[B] = Q1.T @ (L.T @ src_phi[B])
                    sizes[B] = r
                    self.ops.append(("comp", t, B, L, Q, r))
            if opts.order == "level":
                # all compressions of the level from the post-elimination matrix:
                # block (B, N) <- [Q1_B^T L_B^{-1}] A_BN [L_N^{-T} Q1_N], a factor
                # for each compressed end (equal to the sequential recursion when
                # the truncated part Q2^T N vanishes, Sec. 3.2)
                for (u, v), X in list(src_blk.items()):
                    if u == v:
                        if u in level_q:
                            blk[(u, u)] = np.eye(level_q[u][1].shape[1])
                        continue
                    Y = X
                    if u in level_q:
                        Lu, Qu = level_q[u]
                        Y = Qu.T @ sla.solve_triangular(Lu, Y, lower=True)
                    if v in level_q:
                        Lv, Qv = level_q[v]
                        Y = sla.solve_triangular(Lv, Y.T, lower=True).T @ Qv
                    blk[(u, v)] = Y
            # 3. coarsen and merge
            nxt = H.levels[li + 1]
            parent, offset = {}, {}
            new_sizes = {}
            for D, kids in enumerate(nxt.children):
                o = 0
                for C in kids:
                    parent[C] = D
                    offset[C] = o
                    o += sizes[C]
                new_sizes[D] = o
            new_blk = {}
            new_nbr = {D: set() for D in range(nxt.nnodes)}
            for D in range(nxt.nnodes):
                new_blk[(D, D)] = np.zeros((new_sizes[D], new_sizes[D]))
            for (u, v), X in blk.items():
                D, E = parent[u], parent[v]
                key = (min(D, E), max(D, E))
                if key not in new_blk:
                    new_blk[key] = np.zeros((new_sizes[key[0]], new_sizes[key[1]]))
                    new_nbr[D].add(E)
                    new_nbr[E].add(D)
                ou, ov = offset[u], offset[v]
                if D <= E:
                    new_blk[key][ou:ou + X.shape[0], ov:ov + X.shape[1]] = X
                else:
                    new_blk[key][ov:ov + X.shape[1], ou:ou + X.shape[0]] = X.T
                if D == E and u != v:
                    new_blk[key][ov:ov + X.shape[1], ou:ou + X.shape[0]] = X.T
            new_phi = {}
            for D, kids in enumerate(nxt.children):
                parts = [phi[C] @ self.basis.reexpansion(lev.box[C], nxt.box[D]) for C in kids]
                new_phi[D] = np.vstack(parts) if parts else np.zeros((0, self.basis.pi))
            self.ops.append(("merge", t, [(D, list(kids), [sizes[C] for C in kids])
                                          for D, kids in enumerate(nxt.children)]))
            blk, nbr, sizes, phi = new_blk, new_nbr, new_sizes, new_phi
            if nxt.top:
                pass

    # ------------------------------------------------------------------- apply
    def _scatter_in(self, b):
        return {i: b[v].copy() for i, v in enumerate(self.vars1)}

    def _gather_out(self, vec, n):
        x = np.zeros(n)
        for i, v in enumerate(self.vars1):
            x[v] = vec[i]
        return x

    def solve(self, b):
        """x = A_l^{-1} b (Sec. 4.7)."""
        b = np.asarray(b, dtype=np.float64)
        vec = self._scatter_in(b)
        saved = []
        for op in self.ops:
            kind = op[0]
            if kind == "elim":
                _, t, I, L, S_list, W = op
                y = sla.solve_triangular(L, vec[I], lower=True)
                for S, Ws in zip(S_list, W):
                    vec[S] = vec[S] - Ws.T @ y
                saved.append(y)
            elif kind == "comp":
                _, t, B, L, Q, r = op
                z = Q.T @ sla.solve_triangular(L, vec[B], lower=True)
                saved.append(z[r:])
                vec[B] = z[:r]
            elif kind == "merge":
                new = {}
                for D, kids, szs in op[2]:
                    new[D] = np.concatenate([vec[C] for C in kids]) if kids else np.zeros(0)
                saved.append(vec)
                vec = new
            elif kind == "top":
                L = op[1]
                vec[0] = sla.cho_solve((L, True), vec[0])
        for op in reversed(self.ops):
            kind = op[0]
            if kind == "top":
                continue
            s = saved.pop()
            if kind == "merge":
                old = s
                for D, kids, szs in op[2]:
                    o = 0
                    for C, sz in zip(kids, szs):
                        old[C] = vec[D][o:o + sz]
                        o += sz
                vec = old
            elif kind == "comp":
                _, t, B, L, Q, r = op
                vec[B] = sla.solve_triangular(L.T, Q @ np.concatenate([vec[B], s]), lower=False)
            elif kind == "elim":
                _, t, I, L, S_list, W = op
                rhs = s.copy()
                for S, Ws in zip(S_list, W):
                    rhs -= Ws @ vec[S]
                vec[I] = sla.solve_triangular(L.T, rhs, lower=False)
        return self._gather_out(vec, b.size)

    def multiply(self, x):
        """y = A_l x with A_l = G1 B1 G2 ... Gl Gl^T ... B1^T G1^T (Sec. 2.1)."""
        x = np.asarray(x, dtype=np.float64)
        vec = self._scatter_in(x)
        saved = []
        for op in self.ops:
            kind = op[0]
            if kind == "elim":               # G^T = [[L^T, W], [0, I]]
                _, t, I, L, S_list, W = op
                acc = L.T @ vec[I]
                for S, Ws in zip(S_list, W):
                    acc = acc + Ws @ vec[S]
                vec[I] = acc
                saved.append(None)
            elif kind == "comp":             # B^T = diag(Q^T L^T, I)
                _, t, B, L, Q, r = op
                z = Q.T @ (L.T @ vec[B])
                saved.append(z[r:])
                vec[B] = z[:r]
            elif kind == "merge":
                new = {}
                for D, kids, szs in op[2]:
                    new[D] = np.concatenate([vec[C] for C in kids]) if kids else np.zeros(0)
                saved.append(vec)
                vec = new
            elif kind == "top":
                L = op[1]
                vec[0] = L @ (L.T @ vec[0])
        for op in reversed(self.ops):
            kind = op[0]
            if kind == "top":
                continue
            s = saved.pop()
            if kind == "merge":
                old = s
                for D, kids, szs in op[2]:
                    o = 0
                    for C, sz in zip(kids, szs):
                        old[C] = vec[D][o:o + sz]
                        o += sz
                vec = old
            elif kind == "comp":             # B = diag(L Q, I)
                _, t, B, L, Q, r = op
                vec[B] = L @ (Q @ np.concatenate([vec[B], s]))
            elif kind == "elim":             # G = [[L, 0], [W^T, I]]
                _, t, I, L, S_list, W = op
                xi = vec[I]
                for S, Ws in zip(S_list, W):
                    vec[S] = vec[S] + Ws.T @ xi
                vec[I] = L @ xi
        return self._gather_out(vec, x.size)

    # --------------------------------------------------------------- summaries
    def ranks(self):
        """{(level, node): (m, r, compressed)} for every compression attempt."""
        return {k: (v["m"], v["r"], v["compressed"]) for k, v in self.comp_info.items()}

    def dense_operator(self):
        n = self.A.shape[0]
        return np.stack([self.multiply(e) for e in np.eye(n)], axis=1)

    def dense_inverse(self):
        n = self.A.shape[0]
        return np.stack([self.solve(e) for e in np.eye(n)], axis=1)


def factorize(A, H, opts: Options = Options(), order_seed=None) -> SGFFactor:
    return SGFFactor(A, H, opts, order_seed)
