// Batched HODLR (weak-admissibility H-matrix) arithmetic on GPU panels.
//
// The H-operations cyclic reduction needs (Section 2.2.2, Eq. elim: "+_H,
// -_H, ._H, ^{-H}") are written in a level-flat form, so that every step is
// one batched GEMM over all planes of a CR level and all clusters of a HODLR
// level:
//
//  * matvec  Y = M^_{>=l} W : leaf products + per level  c = V|c^T W|c,
//    Y|c^1 += U|c^1 c  (M^_{>=l} keeps the leaves and the levels >= l).
//  * inverse (recursive Woodbury): with X^_{>=l+1} the inverse of the
//    level-(l+1) diagonal blocks, every node t of level l gives
//        X_t = diag(X1, X2) - P_t Kt^{-1} Q_t^T ,
//        P = X^ U_l,  Q = X^T V_l,  Kt = I + [[0, V12^T P2],[V21^T P1, 0]],
//    so  X = blkdiag(leaf^{-1}) - sum over all nodes of rank-2K terms; this
//    sum is exact and is converted to standard HODLR form level by level.
//  * product C = A B: the block of C at level l0 cluster c is
//        A^|c B|c,c^1 + A|c,c^1 B^|c^1 + sum_{l<l0} U^A_l|c T_l V^B_l|c^1^T,
//    T_l(c') = V^A_l|c'^1^T U^B_l|c'^1, i.e. low-rank factors built from
//    matvecs; leaves collect A_leaf B_leaf + sum_l (U^A_l T_l)|leaf V^B_l|leaf^T.
//  * sums: terms are concatenated per level and recompressed once.
#pragma once

#include <algorithm>
#include <vector>

#include "acr_internal.h"

namespace acr {

template <class T>
Op<T> opm(T* p, long rs, long cs, long ps, long c1, int sib = 0, int sh = 0, long c2 = 0) {
  Op<T> o;
  o.p = p; o.rs = rs; o.cs = cs; o.ps = ps; o.c1 = c1; o.c2 = c2; o.sh = sh; o.sib = sib;
  return o;
}

template <class T>
void axpy2d(Ctx& c, int P, long rows, int cols, T alpha, const T* src, long sld, long sps, T* dst, long dld,
            long dps);

// Y = alpha * (leaf part + sum_l [level l of M restricted to the first ncol[l]
// columns of W]) + beta * Y   (trans: M^T).  W, Y: m x w per plane.
// Coefficients c_l = V_l|c^T W|c[:, :ncol[l]] per level (batched reductions),
// then one fused expansion of the leaf product and all levels.  A level with
// ncol[l] = 0 is skipped; the plain product is ncol[l] = w for every level.
template <class T>
void hmatvec_cols(Ctx& c, const HMat<T>& A, bool trans, Pan<T> W, Pan<T> Y, int w, const int* ncol, T alpha,
                  T beta) {
  const int P = A.P, m = A.m, b = A.b, nleaf = m / b;
  if (P <= 0 || w <= 0) return;
  DBuf<T> cbs[MAXL];
  for (int l = 0; l < A.L; ++l) {
    const int K = A.K[l], nc = ncol[l];
    if (K == 0 || nc == 0) continue;
    const int s = m >> (l + 1), nclus = 1 << (l + 1);
    T* Cf = trans ? A.U[l] : A.V[l];
    cbs[l] = DBuf<T>(c, (size_t)P * nclus * K * nc);
    c.tag = "mv_coef";
    gemm<T>(c, K, nc, s, P, nclus, T(1), opm<T>(Cf, 1, K, A.pps[l], (long)s * K),
            opm<T>(W.p, W.ld, 1, W.ps, (long)s * W.ld), T(0), opm<T>(cbs[l].p, nc, 1, (long)nclus * K * nc, (long)K * nc));
  }
  if (b > 64) {
    c.tag = "mv_leaf";
    gemm<T>(c, b, w, b, P, nleaf, alpha, opm<T>(A.leaf, trans ? 1 : b, trans ? b : 1, A.lps, (long)b * b),
            opm<T>(W.p, W.ld, 1, W.ps, (long)b * W.ld), beta, opm<T>(Y.p, Y.ld, 1, Y.ps, (long)b * Y.ld));
    for (int l = 0; l < A.L; ++l) {
      const int K = A.K[l], nc = ncol[l];
      if (K == 0 || nc == 0) continue;
      const int s = m >> (l + 1), nclus = 1 << (l + 1);
      T* Ex = trans ? A.V[l] : A.U[l];
      c.tag = "mv_expand";
      gemm<T>(c, s, nc, K, P, nclus, alpha, opm<T>(Ex, K, 1, A.pps[l], (long)s * K),
              opm<T>(cbs[l].p, nc, 1, (long)nclus * K * nc, (long)K * nc, 1), T(1),
              opm<T>(Y.p, Y.ld, 1, Y.ps, (long)s * Y.ld));
    }
    return;
  }
  HexpArgs<T> ha;
  ha.m = m; ha.b = b; ha.w = w; ha.leaf_trans = trans ? 1 : 0;
  ha.leaf = A.leaf; ha.lps = A.lps;
  ha.W = W.p; ha.wld = W.ld; ha.wps = W.ps;
  ha.Y = Y.p; ha.yld = Y.ld; ha.yps = Y.ps;
  ha.alpha = alpha; ha.beta = beta;
  for (int l = 0; l < A.L; ++l) {
    const int K = A.K[l], nc = ncol[l];
    if (K == 0 || nc == 0) continue;
    const int i = ha.nl++;
    ha.U[i] = trans ? A.V[l] : A.U[l];
    ha.ups[i] = A.pps[l]; ha.C[i] = cbs[l].p; ha.K[i] = K; ha.s[i] = m >> (l + 1); ha.nclus[i] = 1 << (l + 1);
    ha.ncol[i] = nc;
  }
  c.tag = "mv_expand";
  hexpand<T>(c, ha, P);
}

// Y = alpha * M^_{>=lmin} W + beta * Y  (trans: M^T): the leaf part and levels lmin.. of M.
template <class T>
void hmatvec(Ctx& c, const HMat<T>& A, int lmin, bool trans, Pan<T> W, Pan<T> Y, int w, T alpha, T beta) {
  int ncol[MAXL] = {};
  for (int l = std::max(lmin, 0); l < A.L; ++l) ncol[l] = w;
  hmatvec_cols<T>(c, A, trans, W, Y, w, ncol, alpha, beta);
}

// Sum (Woodbury) form of the inverse of P HODLR matrices.
template <class T>
struct WSum {
  int P = 0, m = 0, L = 0, b = 0;
  DBuf<T> leafinv;            // [P][m*b]
  DBuf<T> Pc[MAXL], Qc[MAXL];  // [P][m][K]
  DBuf<T> Kp[MAXL];           // [P][2^l][2K][2K], row-block-swapped coupling inverse
  int K[MAXL] = {};
  bool have[MAXL] = {};
};

// Y = X^_{>=lmin} W (overwrite); trans applies X^T.
template <class T>
void wsum_apply(Ctx& c, const WSum<T>& X, int lmin, bool trans, Pan<T> W, Pan<T> Y, int w) {
  const int P = X.P, m = X.m, b = X.b, nleaf = m / b;
  c.tag = "ws_leaf";
  gemm<T>(c, b, w, b, P, nleaf, T(1), opm<T>(X.leafinv.p, trans ? 1 : b, trans ? b : 1, (long)m * b, (long)b * b),
          opm<T>(W.p, W.ld, 1, W.ps, (long)b * W.ld), T(0), opm<T>(Y.p, Y.ld, 1, Y.ps, (long)b * Y.ld));
  for (int l = lmin; l < X.L; ++l) {
    if (!X.have[l]) continue;
    const int K = X.K[l], s = m >> (l + 1), nclus = 1 << (l + 1), nodes = nclus / 2;
    T* first = trans ? X.Pc[l].p : X.Qc[l].p;
    T* second = trans ? X.Qc[l].p : X.Pc[l].p;
    DBuf<T> cb(c, (size_t)P * nclus * K * w), db(c, (size_t)P * nclus * K * w);
    c.tag = "ws_coef";
    gemm<T>(c, K, w, s, P, nclus, T(1), opm<T>(first, 1, K, (long)m * K, (long)s * K),
            opm<T>(W.p, W.ld, 1, W.ps, (long)s * W.ld), T(0), opm<T>(cb.p, w, 1, (long)nclus * K * w, (long)K * w));
    const long K2 = 2L * K;
    c.tag = "ws_kmix";
    gemm<T>(c, (int)K2, w, (int)K2, P, nodes, T(1),
            opm<T>(X.Kp[l].p, trans ? 1 : K2, trans ? K2 : 1, (long)nodes * K2 * K2, K2 * K2),
            opm<T>(cb.p, w, 1, (long)nclus * K * w, K2 * w), T(0), opm<T>(db.p, w, 1, (long)nclus * K * w, K2 * w));
    c.tag = "ws_expand";
    gemm<T>(c, s, w, K, P, nclus, T(-1), opm<T>(second, K, 1, (long)m * K, (long)s * K),
            opm<T>(db.p, w, 1, (long)nclus * K * w, (long)K * w), T(1), opm<T>(Y.p, Y.ld, 1, Y.ps, (long)s * Y.ld));
  }
}

// Recursive-Woodbury inverse of the P HODLR matrices D (any plane stride).
// Inverses of all Woodbury couplings of one level, stored row-block-swapped
// (the operator applied to the stacked child coefficients):
//   M'_t = [[g1, I], [I, g2]],  g1 = g(2t), g2 = g(2t+1)  (K x K each).
// Block elimination: M'^{-1} = [[-g2 S, T], [S, -g1 T]] with S = (I - g1 g2)^{-1}
// and T = (I - g2 g1)^{-1} = I + g2 S g1 (push-through identity), so one
// pivoted inverse of order K and four batched products replace the inverse
// of order 2K (8x fewer pivoting flops; the products run on the GEMM path).
template <class T>
void coupling_inverse(Ctx& c, int P, int nodes, int K, T* g, T* Kp) {
  const long KK = (long)K * K, K2 = 2L * K, blk = 4L * KK;
  const long gps = 2L * nodes * KK;  // g: [P][2 nodes][K][K]
  const long bps = (long)nodes * blk;
  DBuf<T> S(c, (size_t)P * nodes * KK);
  set_identity_clusters<T>(c, P * nodes, K, K, S.p, K, KK);
  c.tag = "inv_schur";
  gemm<T>(c, K, K, K, P, nodes, T(-1), opm<T>(g, K, 1, gps, 2 * KK), opm<T>(g + KK, K, 1, gps, 2 * KK), T(1),
          opm<T>(S.p, K, 1, (long)nodes * KK, KK));
  batched_inverse<T>(c, P * nodes, K, S.p, KK);
  gemm<T>(c, K, K, K, P, nodes, T(-1), opm<T>(g + KK, K, 1, gps, 2 * KK), opm<T>(S.p, K, 1, (long)nodes * KK, KK),
          T(0), opm<T>(Kp, K2, 1, bps, blk));
  copy2d<T>(c, P * nodes, K, K, T(1), S.p, K, KK, Kp + K2 * K, K2, blk);
  set_identity_clusters<T>(c, P * nodes, K, K, Kp + K, K2, blk);
  gemm<T>(c, K, K, K, P, nodes, T(-1), opm<T>(Kp, K2, 1, bps, blk), opm<T>(g, K, 1, gps, 2 * KK), T(1),
          opm<T>(Kp + K, K2, 1, bps, blk));
  gemm<T>(c, K, K, K, P, nodes, T(-1), opm<T>(g, K, 1, gps, 2 * KK), opm<T>(Kp + K, K2, 1, bps, blk), T(0),
          opm<T>(Kp + K2 * K + K, K2, 1, bps, blk));
}

template <class T>
WSum<T> winverse(Ctx& c, const HMat<T>& D) {
  WSum<T> X;
  X.P = D.P; X.m = D.m; X.L = D.L; X.b = D.b;
  const int P = D.P, m = D.m, b = D.b, nleaf = m / b;
  X.leafinv = DBuf<T>(c, (size_t)P * m * b);
  copy2d<T>(c, P, m, b, T(1), D.leaf, b, D.lps, X.leafinv.p, b, (long)m * b);
  batched_inverse<T>(c, P * nleaf, b, X.leafinv.p, (long)b * b);
  for (int l = D.L - 1; l >= 0; --l) {
    const int K = D.K[l];
    X.K[l] = K;
    if (K == 0) continue;
    const int s = m >> (l + 1), nclus = 1 << (l + 1), nodes = nclus / 2;
    X.Pc[l] = DBuf<T>(c, (size_t)P * m * K);
    X.Qc[l] = DBuf<T>(c, (size_t)P * m * K);
    wsum_apply<T>(c, X, l + 1, false, Pan<T>{D.U[l], K, D.pps[l]}, Pan<T>{X.Pc[l].p, K, (long)m * K}, K);
    wsum_apply<T>(c, X, l + 1, true, Pan<T>{D.V[l], K, D.pps[l]}, Pan<T>{X.Qc[l].p, K, (long)m * K}, K);
    DBuf<T> g(c, (size_t)P * nclus * K * K);
    c.tag = "inv_g";
    gemm<T>(c, K, K, s, P, nclus, T(1), opm<T>(D.V[l], 1, K, D.pps[l], (long)s * K),
            opm<T>(X.Pc[l].p, K, 1, (long)m * K, (long)s * K), T(0),
            opm<T>(g.p, K, 1, (long)nclus * K * K, (long)K * K));
    X.Kp[l] = DBuf<T>(c, (size_t)P * nodes * 4 * K * K);
    coupling_inverse<T>(c, P, nodes, K, g.p, X.Kp[l].p);
    X.have[l] = true;
  }
  return X;
}

template <class T>
void hstore_finish(HStore<T>& H, int P, int m, int L, int b) {
  H.h.P = P; H.h.m = m; H.h.L = L; H.h.b = b;
  H.h.leaf = H.leaf.p;
  H.h.lps = (long)m * b;
  for (int l = 0; l < L; ++l) {
    H.h.U[l] = H.U[l].p;
    H.h.V[l] = H.V[l].p;
    H.h.pps[l] = (long)m * H.h.K[l];
  }
}

// Standard HODLR form of a Woodbury sum, recompressed level by level.
template <class T>
HStore<T> wsum_to_hodlr(Ctx& c, WSum<T>& X, double tol, bool exact, int* ranks_out) {
  const int P = X.P, m = X.m, b = X.b, L = X.L, nleaf = m / b;
  HStore<T> out;
  out.leaf = std::move(X.leafinv);
  DBuf<T> Z[MAXL];
  for (int l = 0; l < L; ++l) {
    if (!X.have[l]) continue;
    const int K = X.K[l], s = m >> (l + 1), nclus = 1 << (l + 1), nodes = nclus / 2;
    const long K2 = 2L * K;
    Z[l] = DBuf<T>(c, (size_t)P * m * K);
    // Z = P ~ Kinv[a][a] of the row's level-(l+1) child a (diagonal block of the swapped inverse)
    c.tag = "conv_z";
    gemm<T>(c, s, K, K, P, nclus, T(1), opm<T>(X.Pc[l].p, K, 1, (long)m * K, (long)s * K),
            opm<T>(X.Kp[l].p, K2, 1, (long)nodes * K2 * K2, K2 * K2, 0, 1, K2 * K + K), T(0),
            opm<T>(Z[l].p, K, 1, (long)m * K, (long)s * K));
    c.tag = "conv_leaf";
    gemm<T>(c, b, b, K, P, nleaf, T(-1), opm<T>(Z[l].p, K, 1, (long)m * K, (long)b * K),
            opm<T>(X.Qc[l].p, 1, K, (long)m * K, (long)b * K), T(1), opm<T>(out.leaf.p, b, 1, (long)m * b, (long)b * b));
  }
  for (int l0 = 0; l0 < L; ++l0) {
    int r = 0;
    for (int l = 0; l <= l0; ++l)
      if (X.have[l]) r += X.K[l];
    DBuf<T> Lf, Rf;
    if (r > 0) {
      Lf = DBuf<T>(c, (size_t)P * m * r);
      Rf = DBuf<T>(c, (size_t)P * m * r);
      int o = 0;
      if (X.have[l0]) {
        const int K = X.K[l0], s = m >> (l0 + 1), nclus = 1 << (l0 + 1), nodes = nclus / 2;
        const long K2 = 2L * K;
        c.tag = "conv_own";
        gemm<T>(c, s, K, K, P, nclus, T(-1), opm<T>(X.Pc[l0].p, K, 1, (long)m * K, (long)s * K),
                opm<T>(X.Kp[l0].p + K, K2, 1, (long)nodes * K2 * K2, K2 * K2, 0, 1, K2 * K - K), T(0),
                opm<T>(Lf.p, r, 1, (long)m * r, (long)s * r));
        copy2d<T>(c, P, m, K, T(1), X.Qc[l0].p, K, (long)m * K, Rf.p, r, (long)m * r);
        o += K;
      }
      for (int l = 0; l < l0; ++l) {
        if (!X.have[l]) continue;
        const int K = X.K[l];
        copy2d<T>(c, P, m, K, T(-1), Z[l].p, K, (long)m * K, Lf.p + o, r, (long)m * r);
        copy2d<T>(c, P, m, K, T(1), X.Qc[l].p, K, (long)m * K, Rf.p + o, r, (long)m * r);
        o += K;
      }
    }
    int Kout = 0;
    recompress_level<T>(c, P, m, l0, std::move(Lf), std::move(Rf), r, tol, exact, out.U[l0], out.V[l0], Kout);
    out.h.K[l0] = Kout;
    if (ranks_out) ranks_out[l0] = Kout;
  }
  hstore_finish(out, P, m, L, b);
  return out;
}

// A pending sum of HODLR terms before recompression.
template <class T>
struct FlatBlk {
  T* Lp; long ldL, psL;
  T* Rp; long ldR, psR;
  int w;
  T coef;
  int Pb;
};

template <class T>
struct Flat {
  int P = 0, m = 0, L = 0, b = 0;
  DBuf<T> leaf;
  std::vector<FlatBlk<T>> lv[MAXL];
  std::vector<DBuf<T>> owned;
  bool padded = false;
};

template <class T>
void flat_init(Ctx& c, Flat<T>& F, int P, int m, int L, int b) {
  F.P = P; F.m = m; F.L = L; F.b = b;
  F.leaf = DBuf<T>(c, (size_t)P * m * b, true);
}

template <class T>
void flat_add_hodlr(Ctx& c, Flat<T>& F, const HMat<T>& A, T coef) {
  axpy2d<T>(c, A.P, F.m, F.b, coef, A.leaf, F.b, A.lps, F.leaf.p, F.b, (long)F.m * F.b);
  if (A.P < F.P) F.padded = true;
  for (int l = 0; l < F.L; ++l)
    if (A.K[l] > 0) F.lv[l].push_back({A.U[l], A.K[l], A.pps[l], A.V[l], A.K[l], A.pps[l], A.K[l], coef, A.P});
}

// F += coef * A B  (A.P == B.P planes, <= F.P).
template <class T>
void flat_add_product(Ctx& c, Flat<T>& F, const HMat<T>& A, const HMat<T>& B, T coef) {
  const int Pb = A.P, m = F.m, b = F.b, L = F.L, nleaf = m / b;
  if (Pb <= 0) return;
  if (Pb < F.P) F.padded = true;
  T* Y1[MAXL] = {};
  T* Y2[MAXL] = {};
  T* Wl[MAXL] = {};
  long ld1 = 0, ld2 = 0;
  // Y1[l] = A^{(>l)} U^B_l and Y2[l] = (B^{(>l)})^T V^A_l for every level at
  // once: the panels of all levels side by side form one wide W, and level l'
  // of the other factor touches only the columns of levels l < l' (a prefix).
  for (int side = 0; side < 2; ++side) {
    const HMat<T>& M = side ? B : A;     // the HODLR factor applied
    const HMat<T>& Q = side ? A : B;     // whose panels are stacked
    int off[MAXL + 1] = {};
    for (int l = 0; l < L; ++l) off[l + 1] = off[l] + Q.K[l];
    const int wt = off[L];
    if (wt == 0) continue;
    DBuf<T> Wc(c, (size_t)Pb * m * wt);
    for (int l = 0; l < L; ++l)
      if (Q.K[l] > 0)
        copy2d<T>(c, Pb, m, Q.K[l], T(1), side ? Q.V[l] : Q.U[l], Q.K[l], Q.pps[l], Wc.p + off[l], wt, (long)m * wt);
    F.owned.emplace_back(c, (size_t)Pb * m * wt);
    T* Yall = F.owned.back().p;
    hmatvec_cols<T>(c, M, side == 1, Pan<T>{Wc.p, wt, (long)m * wt}, Pan<T>{Yall, wt, (long)m * wt}, wt, off, T(1),
                    T(0));
    for (int l = 0; l < L; ++l)
      if (Q.K[l] > 0) (side ? Y2 : Y1)[l] = Yall + off[l];
    (side ? ld2 : ld1) = wt;
  }
  for (int l = 0; l < L; ++l) {
    const int KA = A.K[l], KB = B.K[l], s = m >> (l + 1), nclus = 1 << (l + 1);
    if (KA > 0 && KB > 0) {
      DBuf<T> Tb(c, (size_t)Pb * nclus * KA * KB);
      c.tag = "prod_T";
      gemm<T>(c, KA, KB, s, Pb, nclus, T(1), opm<T>(A.V[l], 1, KA, A.pps[l], (long)s * KA, 1),
              opm<T>(B.U[l], KB, 1, B.pps[l], (long)s * KB, 1), T(0),
              opm<T>(Tb.p, KB, 1, (long)nclus * KA * KB, (long)KA * KB));
      F.owned.emplace_back(c, (size_t)Pb * m * KB);
      Wl[l] = F.owned.back().p;
      c.tag = "prod_W";
      gemm<T>(c, s, KB, KA, Pb, nclus, T(1), opm<T>(A.U[l], KA, 1, A.pps[l], (long)s * KA),
              opm<T>(Tb.p, KB, 1, (long)nclus * KA * KB, (long)KA * KB), T(0),
              opm<T>(Wl[l], KB, 1, (long)m * KB, (long)s * KB));
    }
  }
  c.tag = "prod_leaf";
  gemm<T>(c, b, b, b, Pb, nleaf, coef, opm<T>(A.leaf, b, 1, A.lps, (long)b * b),
          opm<T>(B.leaf, b, 1, B.lps, (long)b * b), T(1), opm<T>(F.leaf.p, b, 1, (long)m * b, (long)b * b));
  for (int l = 0; l < L; ++l) {
    if (!Wl[l]) continue;
    const int KB = B.K[l];
    c.tag = "prod_leafW";
    gemm<T>(c, b, b, KB, Pb, nleaf, coef, opm<T>(Wl[l], KB, 1, (long)m * KB, (long)b * KB),
            opm<T>(B.V[l], 1, KB, B.pps[l], (long)b * KB), T(1), opm<T>(F.leaf.p, b, 1, (long)m * b, (long)b * b));
  }
  for (int l0 = 0; l0 < L; ++l0) {
    const int KA = A.K[l0], KB = B.K[l0];
    if (KB > 0) F.lv[l0].push_back({Y1[l0], ld1, (long)m * ld1, B.V[l0], KB, B.pps[l0], KB, coef, Pb});
    if (KA > 0) F.lv[l0].push_back({A.U[l0], KA, A.pps[l0], Y2[l0], ld2, (long)m * ld2, KA, coef, Pb});
    for (int l = 0; l < l0; ++l)
      if (Wl[l]) F.lv[l0].push_back({Wl[l], B.K[l], (long)m * B.K[l], B.V[l], B.K[l], B.pps[l], B.K[l], coef, Pb});
  }
}

template <class T>
HStore<T> flat_finalize(Ctx& c, Flat<T>& F, double tol, bool exact, int* ranks_out) {
  const int P = F.P, m = F.m, L = F.L;
  HStore<T> out;
  out.leaf = std::move(F.leaf);
  for (int l0 = 0; l0 < L; ++l0) {
    int r = 0;
    for (auto& bk : F.lv[l0]) r += bk.w;
    DBuf<T> Lf, Rf;
    if (r > 0) {
      Lf = DBuf<T>(c, (size_t)P * m * r, F.padded);
      Rf = DBuf<T>(c, (size_t)P * m * r, F.padded);
      int o = 0;
      for (auto& bk : F.lv[l0]) {
        copy2d<T>(c, bk.Pb, m, bk.w, bk.coef, bk.Lp, bk.ldL, bk.psL, Lf.p + o, r, (long)m * r);
        copy2d<T>(c, bk.Pb, m, bk.w, T(1), bk.Rp, bk.ldR, bk.psR, Rf.p + o, r, (long)m * r);
        o += bk.w;
      }
    }
    int Kout = 0;
    recompress_level<T>(c, P, m, l0, std::move(Lf), std::move(Rf), r, tol, exact, out.U[l0], out.V[l0], Kout);
    out.h.K[l0] = Kout;
    if (ranks_out) ranks_out[l0] = Kout;
  }
  F.owned.clear();
  for (int l = 0; l < L; ++l) F.lv[l].clear();
  hstore_finish(out, P, m, L, F.b);
  return out;
}

}  // namespace acr
