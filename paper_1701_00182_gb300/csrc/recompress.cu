// Batched QR + SVD recompression of low-rank blocks (Section 2.1: every
// low-rank block is an outer product A B^T kept to a relative accuracy by SVD
// truncation; Section 3.1: the tolerance is enforced in every H-operation).
//
// For a block  M = L R^T  (L: s x r rows of cluster c, R: s x r rows of c^1):
//   1. orthogonalise both factors, L = Q_L R_L, R = Q_R R_R:
//        s <= 128  Householder QR of the whole factor in shared memory;
//        s >  128  Gram matrix (batched GEMM) + pivoted Cholesky, so that
//                  Q = L[:, piv] R11^{-1} is never formed;
//   2. core C = R_L R_R^T (r x r), one-sided (Hestenes) Jacobi SVD C = X S Y^T;
//   3. keep the k singular values > tol * sigma_1;
//   4. U = Q_L X_k S_k^{1/2},  V = Q_R Y_k S_k^{1/2}  (one GEMM each).
// When r exceeds the block size s the block is first made explicit (U = I,
// V = R L^T), which is exact.
#include <algorithm>
#include <cmath>

#include "../../include/acr.h"
#include "acr_internal.h"

namespace acr {

namespace {
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class T>
__device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : T(0);
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}
}  // namespace

// ---- Householder QR of an s x r factor (r <= s <= 128) ----------------------
// Segment j of 2*NB: side = j / NB (0: rows c of L, 1: rows c^1 of R) of block
// bi = j % NB.  Q (s x r) overwrites the factor, R (r x r) goes to Rout.
template <class T>
__global__ void __launch_bounds__(256) k_qr_small(int s, int r, int nclus, long NB, long mr, T* Lp, T* Rp,
                                                  T* Rout, int* piv, int* kk) {
  extern __shared__ unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);  // column major s x r
  T* tau = A + (long)s * r;
  __shared__ T red[32];
  const long j = blockIdx.x;
  const int side = (int)(j / NB);
  const long bi = j % NB;
  const long plane = bi / nclus;
  const int c = (int)(bi % nclus);
  const int cl = side ? (c ^ 1) : c;
  T* src = (side ? Rp : Lp) + plane * mr + (long)cl * s * r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (long e = tid; e < (long)s * r; e += blockDim.x) {
    int row = (int)(e / r), col = (int)(e % r);
    A[(long)col * s + row] = src[e];
  }
  __syncthreads();
  for (int q = 0; q < r; ++q) {
    T part = T(0);
    for (int i = q + 1 + tid; i < s; i += blockDim.x) part += A[(long)q * s + i] * A[(long)q * s + i];
    T xn2 = block_sum(part, red);
    T x0 = A[(long)q * s + q];
    T t = T(0), beta = x0, scal = T(0);
    if (xn2 > T(0)) {
      beta = -copysign(sqrt(x0 * x0 + xn2), x0);
      t = (beta - x0) / beta;
      scal = T(1) / (x0 - beta);
    }
    __syncthreads();
    for (int i = q + 1 + tid; i < s; i += blockDim.x) A[(long)q * s + i] *= scal;
    if (tid == 0) { tau[q] = t; A[(long)q * s + q] = beta; }
    __syncthreads();
    if (t != T(0)) {
      for (int k = q + 1 + warp; k < r; k += nw) {
        T w = (lane == 0) ? A[(long)k * s + q] : T(0);
        for (int i = q + 1 + lane; i < s; i += 32) w += A[(long)q * s + i] * A[(long)k * s + i];
        w = warp_sum(w) * t;
        if (lane == 0) A[(long)k * s + q] -= w;
        for (int i = q + 1 + lane; i < s; i += 32) A[(long)k * s + i] -= w * A[(long)q * s + i];
      }
    }
    __syncthreads();
  }
  T* R = Rout + j * (long)r * r;
  for (long e = tid; e < (long)r * r; e += blockDim.x) {
    int row = (int)(e / r), col = (int)(e % r);
    R[e] = (row <= col) ? A[(long)col * s + row] : T(0);
  }
  for (int i = tid; i < r; i += blockDim.x) piv[j * r + i] = i;
  if (tid == 0) kk[j] = r;
  __syncthreads();
  // Form Q = H_0 ... H_{r-1} [I; 0] in place (backward accumulation).
  for (int q = r - 1; q >= 0; --q) {
    const T t = tau[q];
    if (q < r - 1) {
      if (tid == 0) A[(long)q * s + q] = T(1);
      __syncthreads();
      for (int k = q + 1 + warp; k < r; k += nw) {
        T w = T(0);
        for (int i = q + lane; i < s; i += 32) w += A[(long)q * s + i] * A[(long)k * s + i];
        w = warp_sum(w) * t;
        for (int i = q + lane; i < s; i += 32) A[(long)k * s + i] -= w * A[(long)q * s + i];
      }
      __syncthreads();
    }
    for (int i = tid; i < s; i += blockDim.x) {
      if (i > q) A[(long)q * s + i] *= -t;
      else if (i < q) A[(long)q * s + i] = T(0);
    }
    if (tid == 0) A[(long)q * s + q] = T(1) - t;
    __syncthreads();
  }
  for (long e = tid; e < (long)s * r; e += blockDim.x) {
    int row = (int)(e / r), col = (int)(e % r);
    src[e] = A[(long)col * s + row];
  }
}

// ---- column balancing of the two Gram matrices of a block -------------------
// M = L R^T is unchanged by L_j *= a_j, R_j /= a_j.  With a_j = sqrt(|R_j|/|L_j|)
// both factors' columns carry the norm sqrt(|L_j| |R_j|) of their rank-one
// term, so the pivoted Cholesky thresholds below compare terms by their
// contribution to M.  Columns with a zero partner are dropped (a = 0).
template <class T>
__global__ void k_balance_scales(int r, long NB, const T* G, T* aL, T* aR) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NB * r; e += (long)gridDim.x * blockDim.x) {
    const long bi = e / r;
    const int j = (int)(e - bi * r);
    const T gl = G[(bi * r + j) * (long)r + j], gr = G[((NB + bi) * r + j) * (long)r + j];
    const T nl = sqrt(fmax(gl, T(0))), nr = sqrt(fmax(gr, T(0)));
    T a = T(0), b = T(0);
    if (nl > T(0) && nr > T(0)) {
      a = sqrt(nr / nl);
      b = T(1) / a;
    }
    aL[e] = a;
    aR[e] = b;
  }
}

// The Gram GEMM fills only the upper triangle (i <= j).  One CTA per pair of
// 32 x 32 tiles (ti <= tj) of one matrix reads the upper tile once and writes
// it and its mirror image, both scaled by a_i a_j, so every element of the
// full symmetric result is written exactly once from unscaled data.
template <class T>
__global__ void __launch_bounds__(256) k_mirror_scale(int r, long NB, T* G, const T* aL, const T* aR) {
  __shared__ T t[32][33];
  const long z = blockIdx.x;  // matrix: side = z / NB, block z % NB
  const int nt = (r + 31) / 32;
  T* M = G + z * (long)r * r;
  const T* a = aL ? ((z < NB) ? aL + z * r : aR + (z - NB) * r) : nullptr;  // null: mirror only
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int pr = blockIdx.y; pr < nt * nt; pr += gridDim.y) {
    const int ti = pr / nt, tj = pr % nt;
    if (ti > tj) continue;  // uniform over the CTA
    const int i0 = ti * 32, j0 = tj * 32;
    for (int ii = ty; ii < 32; ii += 8) {
      const int i = i0 + ii, j = j0 + tx;
      t[ii][tx] = (i < r && j < r && (ti < tj || ii <= tx)) ? M[(long)i * r + j] : T(0);
    }
    __syncthreads();
    for (int ii = ty; ii < 32; ii += 8) {
      const int i = i0 + ii, j = j0 + tx;
      if (i < r && j < r) {
        const T v = (ti < tj || ii <= tx) ? t[ii][tx] : t[tx][ii];
        M[(long)i * r + j] = a ? v * a[i] * a[j] : v;
      }
      if (ti < tj) {  // mirror tile (tj, ti): row j0 + ii, column i0 + tx
        const int mi = j0 + ii, mj = i0 + tx;
        if (mi < r && mj < r) M[(long)mi * r + mj] = a ? t[tx][ii] * a[mi] * a[mj] : t[tx][ii];
      }
    }
    __syncthreads();
  }
}

// ---- pivoted Cholesky of a Gram matrix --------------------------------------
// G (r x r, symmetric PSD) ~ P R^T R P^T.  Rows t of R are written at row
// off + t (off = kkall[j] on entry when `resume`, else 0; original column
// order, zero in already chosen columns), pivots at piv[off + t], and kkall[j]
// becomes off + (pivots found).  Stops when the largest remaining diagonal is
// <= max(eps * (largest initial diagonal of this G), eps_abs * dref[j])
// (dref: the first pass's largest initial diagonal; null = no absolute floor).
// dmax_out[j] (if given) receives this G's largest initial diagonal.
//
// A resumed pass factors the Gram matrix of the explicitly formed residual
// F1 = F - Q1 R1 of the first pass: its Schur complement is recomputed from
// data instead of by subtraction in Gram space, which is what limits a single
// FP32 pass (the FP32 Gram holds entries to ~1e-7 of the largest, so a
// column whose residual is below ~3e-3 of the largest cannot be resolved).
// Columns chosen by the first pass have exact zero residual and are never
// chosen again, so the rows of both passes form one upper-triangular factor
// in pivot order.
constexpr int kCholThreads = 1024;
template <class T>
__global__ void __launch_bounds__(kCholThreads) k_pchol(int r, const T* Gall, T eps, T eps_abs, const T* dref,
                                                        int resume, T* Rall, int* pivall, int* kkall, T* dmax_out) {
  extern __shared__ unsigned char smraw[];
  T* d = reinterpret_cast<T*>(smraw);
  T* colp = d + r;  // R[0..t)[p] of the current pivot column
  __shared__ T wv[32];
  __shared__ int wi[32];
  __shared__ T s_dp, s_dmax0;
  __shared__ int s_p;
  const long j = blockIdx.x;
  const T* G = Gall + j * (long)r * r;
  const int off = resume ? kkall[j] : 0;
  T* R = Rall + j * (long)r * r + (long)off * r;
  int* piv = pivall + j * r + off;
  const T floor_abs = dref ? eps_abs * dref[j] : T(0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < r; i += blockDim.x) d[i] = fmax(G[(long)i * r + i], T(0));
  __syncthreads();
  // columns chosen by earlier passes stay out (their rows here are exact zeros)
  for (int u = tid; u < off; u += blockDim.x) d[piv[u - off]] = T(-1);
  __syncthreads();
  int t = 0;
  const int tmax = r - off;
  for (; t < tmax; ++t) {
    T best = T(-1);
    int bi = 0x7fffffff;
    for (int i = tid; i < r; i += blockDim.x)
      if (d[i] > best) { best = d[i]; bi = i; }
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nw ? wv[lane] : T(-1);
      bi = lane < nw ? wi[lane] : 0x7fffffff;
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        s_dp = best;
        s_p = bi;
        if (t == 0) s_dmax0 = best;
      }
    }
    __syncthreads();
    const T dp = s_dp;
    const int p = s_p;
    if (!(dp > eps * s_dmax0) || !(dp > floor_abs) || !(dp > T(0))) break;
    for (int u = tid; u < t; u += blockDim.x) colp[u] = R[(long)u * r + p];
    __syncthreads();
    const T sq = sqrt(dp), isq = T(1) / sq;
    for (int i = tid; i < r; i += blockDim.x) {
      T v;
      if (d[i] < T(0)) {
        v = T(0);  // already chosen column
      } else if (i == p) {
        v = sq;
      } else {
        T v0 = G[(long)p * r + i], v1 = T(0), v2 = T(0), v3 = T(0);
        int u = 0;
        for (; u + 3 < t; u += 4) {  // four independent chains keep loads in flight
          v0 -= colp[u] * R[(long)u * r + i];
          v1 -= colp[u + 1] * R[(long)(u + 1) * r + i];
          v2 -= colp[u + 2] * R[(long)(u + 2) * r + i];
          v3 -= colp[u + 3] * R[(long)(u + 3) * r + i];
        }
        for (; u < t; ++u) v0 -= colp[u] * R[(long)u * r + i];
        v = ((v0 + v1) + (v2 + v3)) * isq;
      }
      R[(long)t * r + i] = v;
      if (i == p) d[i] = T(-1);
      else if (d[i] >= T(0)) d[i] = fmax(d[i] - v * v, T(0));
    }
    if (tid == 0) piv[t] = p;
    __syncthreads();
  }
  for (long e = (long)t * r + tid; e < (long)(r - off) * r; e += blockDim.x) R[e] = T(0);
  if (tid == 0) {
    kkall[j] = off + t;
    if (dmax_out) dmax_out[j] = s_dmax0;
  }
}

// ---- residual of the first pass ------------------------------------------------
// W = R11^{-1} R1 per block (k1 x r, row major, ld r) with R11[u][v] =
// R[u][piv[v]], so that F1 = F - F[:, piv] W is the part of F outside the
// span of its pivot columns.  One CTA per (block, chunk of C right-hand-side
// columns), right-looking back substitution as in the rebuild coefficients.
template <class T>
__global__ void __launch_bounds__(256) k_resid_coef(int r, const T* __restrict__ Rall, const int* __restrict__ pivall,
                                                    const int* __restrict__ kkall, T* __restrict__ Wall, int C) {
  extern __shared__ unsigned char smraw[];
  T* B = reinterpret_cast<T*>(smraw);  // k x C
  const long j = blockIdx.x;
  const int i0 = blockIdx.y * C;
  const int tc = threadIdx.x % C, g = threadIdx.x / C, G = blockDim.x / C;
  const int i = i0 + tc;
  const int k = kkall[j];
  const T* R = Rall + j * (long)r * r;
  const int* piv = pivall + j * r;
  T* W = Wall + j * (long)r * r;
  const bool act = i < r;
  for (int u = g; u < k; u += G) B[u * C + tc] = act ? R[(long)u * r + i] : T(0);
  __syncthreads();
  for (int u = k - 1; u >= 0; --u) {
    const int pu = piv[u];
    const T zu = B[u * C + tc] / R[(long)u * r + pu];
    const T* Rc = R + pu;
#pragma unroll 4
    for (int w = g; w < u; w += G) B[w * C + tc] -= Rc[(long)w * r] * zu;
    if (g == 0 && act) W[(long)u * r + i] = zu;
    __syncthreads();
  }
}

// F1 = F diag(a): the balanced copy of one side's factor; row i of cluster c
// of a plane belongs to block (plane, c ^ side) and uses that block's scales.
template <class T>
__global__ void k_scale_cols(int P, int m, int s, int nclus, int r, long NB, int side, const T* F, const T* a,
                             T* out) {
  const long nrow = (long)P * m;
  const int lane = threadIdx.x & 31;
  for (long rw = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; rw < nrow;
       rw += ((long)gridDim.x * blockDim.x) >> 5) {
    const long plane = rw / m;
    const int i = (int)(rw - plane * m);
    const T* sc = a + (plane * nclus + ((i / s) ^ side)) * (long)r;
    for (int u = lane; u < r; u += 32) out[rw * r + u] = F[rw * r + u] * sc[u];
  }
}

// ---- one-sided Jacobi SVD of the core ----------------------------------------
// C (row major, valid kL x kR) = X diag(sig) Y^T, sig sorted descending.
// X[i][t] (i < kL) and Y[i][t] (i < kR) row major with leading dimension r;
// rank = #{sig > tol sig_1}.  The wider side is orthogonalised column by
// column (Hestenes), with a round-robin tournament so the ncol/2 disjoint
// pairs of a step run on separate warps.  The working matrix lives in shared
// memory when it fits (ldw = nrow), otherwise in the global work buffer.
// One Hestenes rotation of columns (i, j) by one warp, the column segments
// held in registers (lane owns rows lane + 32 q).  Returns true if rotated.
template <class T, int RPT>
__device__ __forceinline__ bool jacobi_pair(T* wi, T* wj, int nrow, T* vi, T* vj, int ncol, T eps, T floor2,
                                            int lane) {
  T x[RPT], y[RPT];
  T a = 0, b = 0, g = 0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int idx = lane + 32 * q;
    x[q] = idx < nrow ? wi[idx] : T(0);
    y[q] = idx < nrow ? wj[idx] : T(0);
    a += x[q] * x[q];
    b += y[q] * y[q];
    g += x[q] * y[q];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  g = warp_sum(g);
  if (fmin(a, b) <= floor2) return false;  // a negligible column: its rotation cannot matter
  if (!(g != T(0) && fabs(g) > eps * sqrt(a * b))) return false;
  T zeta = (b - a) / (T(2) * g);
  T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
  T cs = T(1) / sqrt(T(1) + t * t), sn = cs * t;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int idx = lane + 32 * q;
    if (idx < nrow) {
      wi[idx] = cs * x[q] - sn * y[q];
      wj[idx] = sn * x[q] + cs * y[q];
    }
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int idx = lane + 32 * q;
    x[q] = idx < ncol ? vi[idx] : T(0);
    y[q] = idx < ncol ? vj[idx] : T(0);
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int idx = lane + 32 * q;
    if (idx < ncol) {
      vi[idx] = cs * x[q] - sn * y[q];
      vj[idx] = sn * x[q] + cs * y[q];
    }
  }
  return true;
}

constexpr int kJacThreads = 1024;
template <class T>
__global__ void __launch_bounds__(kJacThreads) k_jacobi(int r, const T* Call, const int* kk, long NB, T* Wall, T* Vall,
                                                        T* Xall, T* Yall, T* sigall, int* rankall, T tol,
                                                        int maxsweeps, int smem_elems, int* sweeps_out,
                                                        double* flops_out) {
  extern __shared__ unsigned char smraw[];
  T* sig = reinterpret_cast<T*>(smraw);
  int* ord = reinterpret_cast<int*>(sig + r);
  T* Ws = reinterpret_cast<T*>(ord + r + (r & 1));
  __shared__ int s_rot;
  const long bi = blockIdx.x;
  const T* C = Call + bi * (long)r * r;
  const int kL = kk[bi], kR = kk[NB + bi];
  // Orthogonalise the columns of the wider orientation (never more columns
  // than rows).  On a tie take the rows of C: they are graded (row t carries
  // the t-th pivoted-Cholesky row of the left factor, norms decreasing).
  const int trans = kL <= kR;
  const int nrow = trans ? kR : kL, ncol = trans ? kL : kR;
  const bool insm = (long)nrow * ncol <= smem_elems;
  const long ldw = insm ? nrow : r;
  T* W = insm ? Ws : Wall + bi * (long)r * r;  // column major
  T* V = Vall + bi * (long)r * r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // Rotate while the pair's cosine exceeds eps: 16 u (what the precision can
  // resolve) or a hundredth of the truncation tolerance, whichever is larger.
  // The cosine of two columns is only known to about u sqrt(nrow), so the
  // threshold never goes below 4 u sqrt(nrow).
  const T unit = sizeof(T) == 8 ? T(1.1e-16) : T(6e-8);
  const T eps = fmax(T(4) * unit * sqrt(T(nrow > 16 ? nrow : 16)), T(0.01) * tol);
  if (ncol == 0) {
    if (tid == 0) rankall[bi] = 0;
    for (int i = tid; i < r; i += blockDim.x) sigall[bi * r + i] = T(0);
    return;
  }
  for (long e = tid; e < (long)nrow * ncol; e += blockDim.x) {
    int row = (int)(e % nrow), col = (int)(e / nrow);
    W[(long)col * ldw + row] = trans ? C[(long)col * r + row] : C[(long)row * r + col];
  }
  for (long e = tid; e < (long)ncol * ncol; e += blockDim.x) {
    int row = (int)(e % ncol), col = (int)(e / ncol);
    V[(long)col * r + row] = (row == col) ? T(1) : T(0);
  }
  __shared__ T s_fro[32];
  {
    T part = T(0);
    for (long e = tid; e < (long)nrow * ncol; e += blockDim.x) {
      int row = (int)(e % nrow), col = (int)(e / nrow);
      T v = W[(long)col * ldw + row];
      part += v * v;
    }
    part = warp_sum(part);
    if (lane == 0) s_fro[warp] = part;
  }
  __syncthreads();
  T fro2 = T(0);
  for (int w = 0; w < nw; ++w) fro2 += s_fro[w];
  // Columns whose squared norm is below tau ||C||_F^2 lie far below the
  // truncation threshold; Jacobi leaves them alone (their pairwise cosines
  // are rounding noise and would never settle).
  // Columns at the rounding-noise level (norm ~ u ||C||) have random
  // directions and are left alone too (32 u ||C||_F); the truncation below
  // drops everything under this floor, so no unrotated column is kept.
  const T tau = fmax(T(1e-4) * tol * tol, T(1024) * unit * unit);
  const T floor2 = tau * fro2;
  const int ne = ncol + (ncol & 1);
  long long nevals = 0, nrots = 0;  // per warp (identical on its lanes)
  for (int sw = 0; sw < maxsweeps && ne > 1; ++sw) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step < ne - 1; ++step) {
      for (int k = warp; k < ne / 2; k += nw) {
        // Round-robin tournament: position 0 fixed, positions 1..ne-1 rotate.
        int i, jx;
        if (k == 0) {
          i = 0;
          jx = 1 + step;
        } else {
          int a = step + k;
          if (a >= ne - 1) a -= ne - 1;
          int b = step - k;
          if (b < 0) b += ne - 1;
          i = 1 + a;
          jx = 1 + b;
        }
        if (i >= ncol || jx >= ncol) continue;
        ++nevals;
        T* wi = W + (long)i * ldw;
        T* wj = W + (long)jx * ldw;
        T* vi = V + (long)i * r;
        T* vj = V + (long)jx * r;
        bool rotd;
        if (nrow <= 256) rotd = jacobi_pair<T, 8>(wi, wj, nrow, vi, vj, ncol, eps, floor2, lane);
        else if (sizeof(T) == 4 && nrow <= 512)
          rotd = jacobi_pair<T, (sizeof(T) == 4 ? 16 : 8)>(wi, wj, nrow, vi, vj, ncol, eps, floor2, lane);
        else {
          rotd = false;
          T a = 0, b = 0, g = 0;
          for (int q = lane; q < nrow; q += 32) {
            T x = wi[q], y = wj[q];
            a += x * x;
            b += y * y;
            g += x * y;
          }
          a = warp_sum(a);
          b = warp_sum(b);
          g = warp_sum(g);
          if (fmin(a, b) > floor2 && g != T(0) && fabs(g) > eps * sqrt(a * b)) {
            T zeta = (b - a) / (T(2) * g);
            T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
            T cs = T(1) / sqrt(T(1) + t * t), sn = cs * t;
            for (int q = lane; q < nrow; q += 32) {
              T x = wi[q], y = wj[q];
              wi[q] = cs * x - sn * y;
              wj[q] = sn * x + cs * y;
            }
            for (int q = lane; q < ncol; q += 32) {
              T x = vi[q], y = vj[q];
              vi[q] = cs * x - sn * y;
              vj[q] = sn * x + cs * y;
            }
            rotd = true;
          }
        }
        if (rotd) {
          ++nrots;
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (tid == 0 && sweeps_out) atomicMax(sweeps_out, sw + 1);
    if (!rot) break;
  }
  if (lane == 0 && flops_out && (nevals | nrots))
    atomicAdd(flops_out, 6.0 * (double)nevals * nrow + 6.0 * (double)nrots * (nrow + ncol));
  for (int col = warp; col < ncol; col += nw) {
    T a = 0;
    for (int q = lane; q < nrow; q += 32) a += W[(long)col * ldw + q] * W[(long)col * ldw + q];
    a = warp_sum(a);
    if (lane == 0) sig[col] = sqrt(a);
  }
  __syncthreads();
  for (int col = tid; col < ncol; col += blockDim.x) {
    int pos = 0;
    T v = sig[col];
    for (int o = 0; o < ncol; ++o) pos += (sig[o] > v) || (sig[o] == v && o < col);
    ord[pos] = col;
  }
  __syncthreads();
  T smax = sig[ord[0]];
  int rank = 0;
  if (smax > T(0)) {
    T thr = fmax(fmax(tol * smax, smax * unit * T(4)), sqrt(floor2));
    for (int t = 0; t < ncol; ++t) rank += sig[ord[t]] > thr;
  }
  T* X = Xall + bi * (long)r * r;
  T* Y = Yall + bi * (long)r * r;
  for (long e = tid; e < (long)rank * r; e += blockDim.x) {
    int t = (int)(e / r), i = (int)(e % r);
    int col = ord[t];
    T sc = sig[col];
    T wv = (i < nrow) ? W[(long)col * ldw + i] / sc : T(0);
    T vv = (i < ncol) ? V[(long)col * r + i] : T(0);
    // !trans: X = W/s (kL = nrow rows), Y = V (kR = ncol rows); trans: swapped.
    X[(long)i * r + t] = trans ? vv : wv;
    Y[(long)i * r + t] = trans ? wv : vv;
  }
  for (int i = tid; i < r; i += blockDim.x) sigall[bi * r + i] = (i < ncol) ? sig[ord[i]] : T(0);
  if (tid == 0) rankall[bi] = rank;
}

// ---- rank-revealing QR (column pivoting) of the core ---------------------------
// C Pi = Q R (Householder, columns chosen by largest remaining norm), stopped
// when the largest remaining column norm is <= tol * (largest initial column
// norm).  Output in the same form as the Jacobi SVD: C ~ X diag(sig) Y^T with
// X = Q_k (kL x k, orthonormal), sig_t = |R_tt|, Y[Pi(j)][t] = R[t][j] / sig_t.
constexpr int kQrcpThreads = 1024;
// frob = 1: stop instead when the remaining columns' squared norms sum to
// <= tol^2 * (largest initial), which bounds the truncation error of the whole
// block by tol * sigma_1 however many columns remain (explicit blocks).
// floor2 (per block, or null): squared column norm below which a column is
// rounding noise of the block's formation and is never chosen.
template <class T>
__global__ void __launch_bounds__(kQrcpThreads) k_qrcp(int r, const T* Call, const int* kk, long NB, T* Wall,
                                                       T* Xall, T* Yall, T* sigall, int* rankall, T tol,
                                                       int smem_elems, double* flops_out, int frob,
                                                       const T* floor2) {
  extern __shared__ unsigned char smraw[];
  T* nrm = reinterpret_cast<T*>(smraw);
  T* nrm0 = nrm + r;
  T* tau = nrm0 + r;
  int* perm = reinterpret_cast<int*>(tau + r);
  T* Ws = reinterpret_cast<T*>(perm + r + (r & 1));
  __shared__ T wv[32], ws[32];
  __shared__ int wi[32];
  __shared__ T s_thr2;
  __shared__ int s_p, s_stop;
  const long bi = blockIdx.x;
  const T* C = Call + bi * (long)r * r;
  const int kL = kk[bi], kR = kk[NB + bi];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const bool insm = (long)kL * kR <= smem_elems;
  const long ldw = insm ? kL : r;
  T* W = insm ? Ws : Wall + bi * (long)r * r;  // column major kL x kR
  T* X = Xall + bi * (long)r * r;
  T* Y = Yall + bi * (long)r * r;
  const int kmax = min(kL, kR);
  if (kmax == 0) {
    if (tid == 0) rankall[bi] = 0;
    for (int i = tid; i < r; i += blockDim.x) sigall[bi * r + i] = T(0);
    return;
  }
  for (long e = tid; e < (long)kL * kR; e += blockDim.x) {
    int row = (int)(e % kL), col = (int)(e / kL);
    W[(long)col * ldw + row] = C[(long)row * r + col];
  }
  __syncthreads();
  for (int col = warp; col < kR; col += nw) {
    T a = 0;
    for (int q = lane; q < kL; q += 32) a += W[(long)col * ldw + q] * W[(long)col * ldw + q];
    a = warp_sum(a);
    if (lane == 0) { nrm[col] = a; nrm0[col] = a; perm[col] = col; }
  }
  __syncthreads();
  int rank = 0;
  for (int st = 0; st < kmax; ++st) {
    // pivot: largest remaining column norm
    T best = T(-1), sum = T(0);
    int bi2 = 0x7fffffff;
    for (int j = st + tid; j < kR; j += blockDim.x) {
      sum += fmax(nrm[j], T(0));
      if (nrm[j] > best) { best = nrm[j]; bi2 = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi2, o);
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (ov > best || (ov == best && oi < bi2)) { best = ov; bi2 = oi; }
    }
    if (lane == 0) { wv[warp] = best; wi[warp] = bi2; ws[warp] = sum; }
    __syncthreads();
    if (tid == 0) {
      T b = T(-1), sm = T(0);
      int bb = st;
      for (int w = 0; w < nw; ++w) {
        sm += ws[w];
        if (wv[w] > b || (wv[w] == b && wi[w] < bb)) { b = wv[w]; bb = wi[w]; }
      }
      if (st == 0) s_thr2 = tol * tol * b;
      s_p = bb;
      s_stop = !((frob ? sm : b) > s_thr2) || !(b > (floor2 ? floor2[bi] : T(0)));
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != st) {
      for (int q = tid; q < kL; q += blockDim.x) {
        T t = W[(long)st * ldw + q];
        W[(long)st * ldw + q] = W[(long)p * ldw + q];
        W[(long)p * ldw + q] = t;
      }
      if (tid == 0) {
        T t = nrm[st]; nrm[st] = nrm[p]; nrm[p] = t;
        t = nrm0[st]; nrm0[st] = nrm0[p]; nrm0[p] = t;
        int ti = perm[st]; perm[st] = perm[p]; perm[p] = ti;
      }
    }
    __syncthreads();
    // Householder reflector of column st, rows st..kL-1
    T part = T(0);
    for (int q = st + 1 + tid; q < kL; q += blockDim.x) part += W[(long)st * ldw + q] * W[(long)st * ldw + q];
    T xn2 = block_sum(part, wv);
    T x0 = W[(long)st * ldw + st];
    T t = T(0), beta = x0, scal = T(0);
    if (xn2 > T(0)) {
      beta = -copysign(sqrt(x0 * x0 + xn2), x0);
      t = (beta - x0) / beta;
      scal = T(1) / (x0 - beta);
    }
    __syncthreads();
    for (int q = st + 1 + tid; q < kL; q += blockDim.x) W[(long)st * ldw + q] *= scal;
    if (tid == 0) { tau[st] = t; W[(long)st * ldw + st] = beta; }
    __syncthreads();
    for (int j = st + 1 + warp; j < kR; j += nw) {
      T w = T(0);
      if (t != T(0)) {
        w = (lane == 0) ? W[(long)j * ldw + st] : T(0);
        for (int q = st + 1 + lane; q < kL; q += 32) w += W[(long)st * ldw + q] * W[(long)j * ldw + q];
        w = warp_sum(w) * t;
        for (int q = st + 1 + lane; q < kL; q += 32) W[(long)j * ldw + q] -= w * W[(long)st * ldw + q];
      }
      if (lane == 0) {
        T rsj = W[(long)j * ldw + st] - w;
        W[(long)j * ldw + st] = rsj;
        T nn = nrm[j] - rsj * rsj;
        nrm[j] = nn;
      }
      __syncwarp();
      // norm downdate lost its digits: recompute from the remaining rows
      if (nrm[j] < T(0.05) * nrm0[j]) {
        T a = 0;
        for (int q = st + 1 + lane; q < kL; q += 32) a += W[(long)j * ldw + q] * W[(long)j * ldw + q];
        a = warp_sum(a);
        if (lane == 0) { nrm[j] = a; nrm0[j] = a; }
      }
    }
    __syncthreads();
    rank = st + 1;
  }
  // Y and sig from R (rows < rank), before Q overwrites the reflectors.
  for (long e = tid; e < (long)rank * kR; e += blockDim.x) {
    int tt = (int)(e / kR), j = (int)(e % kR);
    T d = fabs(W[(long)tt * ldw + tt]);
    T v = (j >= tt) ? W[(long)j * ldw + tt] : T(0);
    Y[(long)perm[j] * r + tt] = d > T(0) ? v / d : T(0);
  }
  for (int i = tid; i < r; i += blockDim.x) sigall[bi * r + i] = (i < rank) ? fabs(W[(long)i * ldw + i]) : T(0);
  __syncthreads();
  // Q_k = H_0 ... H_{k-1} [I; 0] in place (backward accumulation).
  for (int q = rank - 1; q >= 0; --q) {
    const T tq = tau[q];
    if (q < rank - 1) {
      if (tid == 0) W[(long)q * ldw + q] = T(1);
      __syncthreads();
      for (int j = q + 1 + warp; j < rank; j += nw) {
        T w = T(0);
        for (int i = q + lane; i < kL; i += 32) w += W[(long)q * ldw + i] * W[(long)j * ldw + i];
        w = warp_sum(w) * tq;
        for (int i = q + lane; i < kL; i += 32) W[(long)j * ldw + i] -= w * W[(long)q * ldw + i];
      }
      __syncthreads();
    }
    for (int i = tid; i < kL; i += blockDim.x) {
      if (i > q) W[(long)q * ldw + i] *= -tq;
      else if (i < q) W[(long)q * ldw + i] = T(0);
    }
    if (tid == 0) W[(long)q * ldw + q] = T(1) - tq;
    __syncthreads();
  }
  for (long e = tid; e < (long)rank * r; e += blockDim.x) {
    int tt = (int)(e / r), i = (int)(e % r);
    X[(long)i * r + tt] = (i < kL) ? W[(long)tt * ldw + i] : T(0);
  }
  if (tid == 0) {
    rankall[bi] = rank;
    if (flops_out) {  // reflector applications of the factorisation and of forming Q_k
      double f = 0;
      for (int q = 0; q < rank; ++q) f += 4.0 * (kL - q) * ((kR - q - 1) + (rank - q - 1));
      atomicAdd(flops_out, f);
    }
  }
}

// ---- coefficients of the rebuild ---------------------------------------------
// Z (zrows x Kout used of r x Kout, row major) per side of block bi such that
// the new factor is (factor columns) * Z:  QR path  Z[0:k, t] = X[:, t] sqrt(s_t)
// (rows of Q);  Gram path  Z[u, t] = z[u] a_{piv[u]},  R11 z = X[:, t] sqrt(s_t)
// with R11[u][v] = R[u][piv[v]] (upper triangular) and a the balancing scale;
// there the factor columns are the gathered pivots piv[0..k), so Z is compact.
// Rows k .. zrows-1 are zero.
//
// One CTA per (side, block, chunk of C columns); its 256 threads are C columns
// x G = 256 / C row groups.  The right-hand sides of the chunk sit in B (shared
// memory when k x C fits, else a global scratch slice with row stride ldb).
// Right-looking back substitution: at step u every thread forms
// z_u = b_u / R11[u][u] for its column and removes z_u R11[w][u] from the rows
// w < u of its group, so a step is one barrier and a k / G long update.
template <class T>
__global__ void __launch_bounds__(256) k_coef(int r, int Kout, long NB, int qr, const T* __restrict__ Rall,
                                              const int* __restrict__ pivall, const int* __restrict__ kkall,
                                              const T* __restrict__ Xall, const T* __restrict__ Yall,
                                              const T* __restrict__ sigall, const int* __restrict__ rankall,
                                              const T* __restrict__ scall, T* __restrict__ Zall, int C,
                                              T* __restrict__ gscratch, int zrows) {
  extern __shared__ unsigned char smraw[];
  const long j = blockIdx.x;
  const int side = (int)(j / NB);
  const long bi = j % NB;
  const int t0 = blockIdx.y * C;
  const int tc = threadIdx.x % C, g = threadIdx.x / C, G = blockDim.x / C;
  const int t = t0 + tc;
  const int rank = rankall[bi];
  const int k = kkall[j];
  T* Z = Zall + j * (long)r * Kout;
  if (t < Kout)
    for (int row = g; row < zrows; row += G) Z[(long)row * Kout + t] = T(0);
  if (t0 >= rank) return;  // uniform over the CTA
  const bool act = t < rank;
  const T* R = Rall + j * (long)r * r;
  const int* piv = pivall + j * r;
  const T* XY = (side ? Yall : Xall) + bi * (long)r * r;
  const T* sc = scall ? scall + j * (long)r : nullptr;
  const T sq = act ? sqrt(sigall[bi * r + t]) : T(0);
  if (qr) {
    __syncthreads();
    if (act)
      for (int u = g; u < k; u += G) Z[(long)u * Kout + t] = XY[(long)u * r + t] * sq * (sc ? sc[u] : T(1));
    return;
  }
  T* B;
  long ldb;
  if (gscratch) {
    ldb = (long)gridDim.y * C;  // padded so every thread of the grid owns its own column
    B = gscratch + j * (long)r * ldb + t0;
  } else {
    B = reinterpret_cast<T*>(smraw);
    ldb = C;
  }
  for (int u = g; u < k; u += G) B[(long)u * ldb + tc] = act ? XY[(long)u * r + t] * sq : T(0);
  __syncthreads();  // also orders the zero fill of Z before the writes below
  for (int u = k - 1; u >= 0; --u) {
    const int pu = piv[u];
    const T zu = B[(long)u * ldb + tc] / R[(long)u * r + pu];
    const T* Rc = R + pu;
#pragma unroll 4
    for (int w = g; w < u; w += G) B[(long)w * ldb + tc] -= Rc[(long)w * r] * zu;
    if (g == 0 && act) Z[(long)u * Kout + t] = zu * (sc ? sc[pu] : T(1));
    __syncthreads();
  }
}

// Columns piv[0..k) of each block's factor, side by side (zero up to kmax):
// out[plane][row][u] = F[plane][row][piv[u]] for the rows of cluster c, with the
// pivots of block c ^ side (the R factor of block b lives in cluster b ^ 1).
template <class T>
__global__ void k_gather_piv(int P, int m, int s, int nclus, int r, int kmax, long NB, int side, const T* F,
                             const int* pivall, const int* kkall, T* out) {
  const long nrow = (long)P * m;
  const int lane = threadIdx.x & 31;
  for (long rw = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; rw < nrow;
       rw += ((long)gridDim.x * blockDim.x) >> 5) {
    const long plane = rw / m;
    const int i = (int)(rw - plane * m);
    const long j = side * NB + plane * nclus + ((i / s) ^ side);
    const int* piv = pivall + j * r;
    const int k = kkall[j];
    const T* src = F + rw * r;
    T* dst = out + rw * kmax;
    for (int u = lane; u < kmax; u += 32) dst[u] = (u < k) ? src[piv[u]] : T(0);
  }
}

// Squared column norms of a factor over each cluster: out[(plane nclus + c)
// r + k] = sum over the rows i of cluster c of F[plane][i][k]^2.  CTA: 32
// columns x 8 row groups (rows coalesced 128 bytes at a time).
template <class T>
__global__ void __launch_bounds__(256) k_cluster_colnorm2(int m, int s, int nclus, int r, const T* F, float* out) {
  __shared__ float part[8][33];
  const long bc = blockIdx.x;  // plane * nclus + cluster
  const long plane = bc / nclus;
  const int c = (int)(bc % nclus);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int k = blockIdx.y * 32 + tx;
  const T* Fc = F + (plane * m + (long)c * s) * r;
  float a = 0.f;
  if (k < r)
    for (int i = ty; i < s; i += 8) {
      const float v = (float)Fc[(long)i * r + k];
      a += v * v;
    }
  part[ty][tx] = a;
  __syncthreads();
  if (ty == 0 && k < r) {
    float t = 0.f;
    for (int g = 0; g < 8; ++g) t += part[g][tx];
    out[bc * r + k] = t;
  }
}

// Rounding-noise floor of an explicit block M_c = L|c R|c^1^T formed by one
// GEMM: its error is ~ u sqrt(r) (sum_k |L_k|^2 |R_k|^2)^(1/2) in Frobenius
// norm, spread over s columns; floor2 = (4 x that / sqrt(s))^2 keeps every
// noise column below the stop of the pivoted QR.  One warp per block.
template <class T>
__global__ void k_explicit_floor(long NB, int s, int r, const float* nL, const float* nR, double u, T* floor2) {
  const long bi = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (bi >= NB) return;
  double acc = 0;
  for (int k = lane; k < r; k += 32) acc += (double)nL[bi * r + k] * nR[(bi ^ 1) * r + k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) floor2[bi] = T(16.0 * u * u * r * acc / s);
}

// Factors of blocks truncated in explicit form: block bi = (plane, cluster c)
// was given as C_bi = M_c^T ~ X diag(sig) Y^T, so M_c ~ (Y S^1/2)(X S^1/2)^T:
// U|c = Y sqrt(sig), V|c^1 = X sqrt(sig) (columns beyond the block's rank zero).
// One warp per output row of both panels.
template <class T>
__global__ void k_dense_uv(int P, int m, int s, int nclus, int r, int Kout, const T* __restrict__ Xall,
                           const T* __restrict__ Yall, const T* __restrict__ sigall, const int* __restrict__ rankall,
                           T* __restrict__ U, T* __restrict__ V) {
  const long nrow = (long)P * m;
  const int lane = threadIdx.x & 31;
  for (long rw = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; rw < nrow;
       rw += ((long)gridDim.x * blockDim.x) >> 5) {
    const long plane = rw / m;
    const int i = (int)(rw - plane * m);
    const int cl = i / s, ii = i - cl * s;
    const long bu = plane * nclus + cl, bv = plane * nclus + (cl ^ 1);
    const int ku = rankall[bu], kv = rankall[bv];
    for (int t = lane; t < Kout; t += 32) {
      U[rw * Kout + t] = t < ku ? Yall[(bu * r + ii) * (long)r + t] * sqrt(sigall[bu * r + t]) : T(0);
      V[rw * Kout + t] = t < kv ? Xall[(bv * r + ii) * (long)r + t] * sqrt(sigall[bv * r + t]) : T(0);
    }
  }
}

// Truncation of NB cores C_bi (valid kk[bi] x kk[NB + bi], row major, ld r):
// C ~ X diag(sig) Y^T with the ranks in `rank` (pivoted QR by default, or the
// one-sided Jacobi SVD).
template <class T>
static void truncate_cores(Ctx& c, int r, const T* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol,
                           DBuf<T>& Xo, DBuf<T>& Yo, DBuf<T>& sig, DBuf<int>& rank, const char* site, int frob,
                           const T* floor2 = nullptr, bool prefer_cluster = false) {
  DBuf<T> W(c, NB * (size_t)r * r);
  Xo = DBuf<T>(c, NB * (size_t)r * r);
  Yo = DBuf<T>(c, NB * (size_t)r * r);
  sig = DBuf<T>(c, NB * (size_t)r);
  rank = DBuf<int>(c, NB);
  const size_t cap = 200 * 1024;
  if (c.core_svd != 1) {
    size_t base2 = (size_t)r * (3 * sizeof(T) + sizeof(int)) + ((r & 1) ? sizeof(int) : 0);
    base2 = (base2 + 15) / 16 * 16;
    int se2 = (int)std::min<size_t>((size_t)r * r, cap > base2 ? (cap - base2) / sizeof(T) : 0);
    size_t sm2 = base2 + (size_t)se2 * sizeof(T);
    // Matrices beyond one CTA's shared memory: the cluster kernel keeps them on chip.  In FP32
    // the register-resident cluster kernel also takes the blocks the caller prefers there
    // (explicit blocks of 128+ rows; large cores in batches too small to fill the GPU with
    // one CTA each), where it measured faster than the one-CTA kernel.
    const bool reg = sizeof(T) == 4 && c.qrcp_reg && (prefer_cluster || c.qrcp_reg_all);
    if (((long)kmaxL * kmaxR > se2 || reg) && c.qrcp_cluster &&
        qrcp_cluster<T>(c, r, C, kk, NB, kmaxL, kmaxR, tol, frob, floor2, Xo.p, Yo.p, sig.p, rank.p, site))
      return;
    ACR_CUDA(cudaFuncSetAttribute(k_qrcp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    c.kbegin();
    const int thr = std::min(kQrcpThreads, std::max(64, (8 * std::max(kmaxL, kmaxR) + 31) / 32 * 32));
    k_qrcp<T><<<(unsigned)NB, thr, sm2, c.st>>>(r, C, kk, NB, W.p, Xo.p, Yo.p, sig.p, rank.p, T(tol), se2,
                                                c.d_jflops, frob, floor2);
    c.kend(KC_JACOBI, 0, (double)NB * sizeof(T) * 3.0 * r * r, site);
  } else {
    DBuf<T> Vw(c, NB * (size_t)r * r);
    size_t base = (size_t)r * (sizeof(T) + sizeof(int)) + ((r & 1) ? sizeof(int) : 0);
    base = (base + 15) / 16 * 16;
    int smem_elems = (int)std::min<size_t>((size_t)r * r, cap > base ? (cap - base) / sizeof(T) : 0);
    size_t sm = base + (size_t)smem_elems * sizeof(T);
    ACR_CUDA(cudaFuncSetAttribute(k_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    c.kbegin();
    k_jacobi<T><<<(unsigned)NB, kJacThreads, sm, c.st>>>(r, C, kk, NB, W.p, Vw.p, Xo.p, Yo.p, sig.p, rank.p, T(tol),
                                                         24, smem_elems, c.d_flag + 1, c.d_jflops);
    c.kend(KC_JACOBI, 0, (double)NB * sizeof(T) * 3.0 * r * r, site);
  }
}

// A block is truncated in explicit form (one GEMM forms it, one pivoted QR
// truncates it) when its concatenated width reaches its size and it is at
// most 512 rows (its pivoted QR then runs out of a cluster's shared memory);
// it is then also more accurate than the Gram route in FP32 (Householder
// instead of a squared condition number).
static bool explicit_block(int s, int r) { return s <= 512 && r >= s; }

// Per-site profile label of a recompression launch: kernel, block size s and
// whether the block was made explicit first.
static const char* site_name(Ctx& c, const char* kern, int s, bool dens) {
  if (!c.site_detail) return kern;
  char buf[96];
  std::snprintf(buf, sizeof(buf), "%s s=%d%s", kern, s, dens ? " dense" : "");
  return c.tagstore.insert(buf).first->c_str();
}

template <class T>
void recompress_level(Ctx& c, int P, int m, int lvl, DBuf<T>&& Left, DBuf<T>&& Right, int r, double tol, bool exact,
                      DBuf<T>& Uout, DBuf<T>& Vout, int& Kout) {
  const int s = m >> (lvl + 1);
  bool dens = false;
  const int nclus = 1 << (lvl + 1);
  const long NB = (long)P * nclus;
  DBuf<T> Lb = std::move(Left), Rb = std::move(Right);
  if (r <= 0) {
    Kout = 0;
    Uout.release();
    Vout.release();
    return;
  }
  if (!exact && explicit_block(s, r)) {
    // Explicit form: M_c^T = R|c^1 (L|c)^T (s x s) for every block (plane, c),
    // stored at cluster c; its pivoted QR truncated at tol gives the factors.
    DBuf<T> Mt(c, (size_t)P * m * s);
    {
      Op<T> A{Rb.p, r, 1, (long)m * r, (long)s * r, 0, 0, 1};
      Op<T> B{Lb.p, 1, r, (long)m * r, (long)s * r, 0, 0, 0};
      Op<T> C{Mt.p, s, 1, (long)m * s, (long)s * s, 0, 0, 0};
      c.tag = "explicit";
      gemm<T>(c, s, s, r, P, nclus, T(1), A, B, T(0), C);
    }
    DBuf<T> fl2(c, NB);
    {
      // 3xTF32 tensor-core products carry ~2^-22 relative error per product
      const double u = sizeof(T) == 8 ? 1.1e-16 : (c.tensor ? 2.4e-7 : 6e-8);
      DBuf<float> nrm(c, 2 * NB * (size_t)r);
      c.kbegin();
      const dim3 g((unsigned)NB, (unsigned)((r + 31) / 32));
      k_cluster_colnorm2<T><<<g, 256, 0, c.st>>>(m, s, nclus, r, Lb.p, nrm.p);
      k_cluster_colnorm2<T><<<g, 256, 0, c.st>>>(m, s, nclus, r, Rb.p, nrm.p + NB * r);
      k_explicit_floor<T><<<(unsigned)((NB * 32 + 255) / 256), 256, 0, c.st>>>(NB, s, r, nrm.p, nrm.p + NB * r, u,
                                                                            fl2.p);
      c.kend(KC_COPY, 0, (double)sizeof(T) * 2.0 * P * m * r, site_name(c, "copy:explicit_floor", s, true));
      c.launches += 2;
    }
    Lb.release();
    Rb.release();
    DBuf<int> kk(c, 2 * NB);
    fill<int>(c, kk.p, 2 * NB, s);
    DBuf<T> Xo, Yo, sig;
    DBuf<int> rank;
    // FP64: stop on the remaining columns' Frobenius norm (block error <= tol
    // sigma_1).  FP32: on the largest remaining column -- the Frobenius sum of
    // s rounding-level columns (~u sqrt(s) each) exceeds tol^2 at tol ~1e-6.
    truncate_cores<T>(c, s, Mt.p, kk.p, NB, s, s, tol, Xo, Yo, sig, rank, site_name(c, "qrcp", s, true),
                      sizeof(T) == 8 ? 1 : 0, fl2.p, s >= 128);
    std::vector<int> hr(NB);
    ACR_CUDA(cudaMemcpyAsync(hr.data(), rank.p, NB * sizeof(int), cudaMemcpyDeviceToHost, c.st));
    ACR_CUDA(cudaStreamSynchronize(c.st));
    Kout = 0;
    for (int v : hr) Kout = std::max(Kout, v);
    if (Kout == 0) {
      Uout.release();
      Vout.release();
      return;
    }
    Uout = DBuf<T>(c, (size_t)P * m * Kout);
    Vout = DBuf<T>(c, (size_t)P * m * Kout);
    c.kbegin();
    k_dense_uv<T><<<(unsigned)std::min<long>(((long)P * m * 32 + 255) / 256, 152L * 32), 256, 0, c.st>>>(
        P, m, s, nclus, s, Kout, Xo.p, Yo.p, sig.p, rank.p, Uout.p, Vout.p);
    c.kend(KC_COPY, 0, (double)sizeof(T) * 2.0 * P * m * (s + Kout), site_name(c, "copy:dense_uv", s, true));
    return;
  }
  if (r > s) {
    // Explicit block kept exact: U|c = I_s, V|c^1 = R|c^1 (L|c)^T.
    DBuf<T> U2(c, (size_t)P * m * s), V2(c, (size_t)P * m * s);
    set_identity_clusters<T>(c, P, m, s, U2.p, s, (long)m * s);
    Op<T> A{Rb.p, r, 1, (long)m * r, (long)s * r, 0, 0, 1};
    Op<T> B{Lb.p, 1, r, (long)m * r, (long)s * r, 0, 0, 0};
    Op<T> C{V2.p, s, 1, (long)m * s, (long)s * s, 0, 0, 1};
    c.tag = "densify";
    gemm<T>(c, s, s, r, P, nclus, T(1), A, B, T(0), C);
    Lb = std::move(U2);
    Rb = std::move(V2);
    r = s;
    dens = true;
  }
  if (exact) {
    Uout = std::move(Lb);
    Vout = std::move(Rb);
    Kout = r;
    return;
  }
  const bool qr = (s <= 128);
  DBuf<T> scale;
  DBuf<T> R(c, 2 * NB * r * (size_t)r);
  DBuf<int> piv(c, 2 * NB * (size_t)r), kk(c, 2 * NB);
  if (qr) {
    size_t sm = ((size_t)s * r + r) * sizeof(T);
    ACR_CUDA(cudaFuncSetAttribute(k_qr_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    c.kbegin();
    k_qr_small<T><<<(unsigned)(2 * NB), 256, sm, c.st>>>(s, r, nclus, NB, (long)m * r, Lb.p, Rb.p, R.p, piv.p,
                                                         kk.p);
    c.kend(KC_QR, 2.0 * NB * 4.0 * s * (double)r * r, 2.0 * NB * sizeof(T) * (2.0 * s * r + (double)r * r),
           site_name(c, "qr_small", s, dens));
  } else {
    DBuf<T> G(c, 2 * NB * r * (size_t)r);
    for (int side = 0; side < 2; ++side) {
      T* F = side ? Rb.p : Lb.p;
      Op<T> A{F, 1, r, (long)m * r, (long)s * r, 0, 0, side};
      Op<T> B{F, r, 1, (long)m * r, (long)s * r, 0, 0, side};
      Op<T> C{G.p + side * NB * r * (long)r, r, 1, (long)nclus * r * r, (long)r * r, 0, 0, 0};
      c.tag = "gram";
      gemm_sym<T>(c, r, s, P, nclus, T(1), A, B, T(0), C, false);
    }
    scale = DBuf<T>(c, 2 * NB * (size_t)r);
    c.kbegin();
    k_balance_scales<T><<<(unsigned)std::min<long>((NB * r + 255) / 256, 152L * 16), 256, 0, c.st>>>(
        r, NB, G.p, scale.p, scale.p + NB * r);
    const int nt = (r + 31) / 32;
    k_mirror_scale<T><<<dim3((unsigned)(2 * NB), (unsigned)std::min(nt * nt, 65535)), 256, 0, c.st>>>(
        r, NB, G.p, scale.p, scale.p + NB * r);
    c.kend(KC_COPY, 0, 2.0 * NB * sizeof(T) * 1.5 * r * r, site_name(c, "copy:balance", s, dens));
    c.launches += 1;
    // FP32: the Gram matrix resolves a column's residual down to ~3e-3 of the
    // largest (1e-5 on the squared diagonal); FP64 to ~3e-8.
    const double floor_rel = sizeof(T) == 8 ? 1e-15 : 1e-5;
    const double tau = 0.01 * tol * tol;  // squared column residual the tolerance asks for
    const double epsd = std::max(tau, floor_rel);
    size_t sm = 2 * (size_t)r * sizeof(T);
    if (sm > 48 * 1024) ACR_CUDA(cudaFuncSetAttribute(k_pchol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // one thread per Gram column (64 .. 1024): small blocks at deep levels do
    // not pay for idle warps in every per-pivot barrier
    const int thr = std::min(kCholThreads, std::max(64, (r + 31) / 32 * 32));
    DBuf<T> dmax(c, 2 * NB);
    c.kbegin();
    k_pchol<T><<<(unsigned)(2 * NB), thr, sm, c.st>>>(r, G.p, T(epsd), T(0), nullptr, 0, R.p, piv.p, kk.p, dmax.p);
    c.kend(KC_PCHOL, 0, 2.0 * NB * sizeof(T) * 2.0 * r * r, site_name(c, "pchol", s, dens));
    // Further passes while the floor stopped above the tolerance: each factors
    // the Gram matrix of the explicit residual F1 = F~ - F~[:, piv] R11^{-1} R1
    // (F~ = F diag(a), the balanced factor) and appends its rows to R.
    const int passes = tau < epsd ? c.chol_passes : 1;
    for (int pass = 1; pass < passes; ++pass) {
      std::vector<int> hk1(2 * NB);
      ACR_CUDA(cudaMemcpyAsync(hk1.data(), kk.p, 2 * NB * sizeof(int), cudaMemcpyDeviceToHost, c.st));
      ACR_CUDA(cudaStreamSynchronize(c.st));
      int k1 = 0;
      for (int v : hk1) k1 = std::max(k1, v);
      if (k1 == 0 || k1 >= r) break;
      DBuf<T> W(c, 2 * NB * (size_t)r * r, true);
      {
        int Cw = 32;
        while (Cw > 8 && (size_t)k1 * Cw * sizeof(T) > 100 * 1024) Cw /= 2;
        const size_t smw = (size_t)k1 * Cw * sizeof(T);
        if (smw > 200 * 1024) throw AcrError(ACR_ERR_RANK_CAP, "recompression rank too large for the residual pass");
        if (smw > 48 * 1024)
          ACR_CUDA(cudaFuncSetAttribute(k_resid_coef<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
        c.kbegin();
        k_resid_coef<T><<<dim3((unsigned)(2 * NB), (unsigned)((r + Cw - 1) / Cw)), 256, smw, c.st>>>(
            r, R.p, piv.p, kk.p, W.p, Cw);
        double f = 0;
        for (int v : hk1) f += (double)v * v * r;
        c.kend(KC_COEF, f, 2.0 * NB * sizeof(T) * 2.0 * r * r, "resid_coef");
      }
      DBuf<T> F1(c, (size_t)P * m * r), Gc1(c, (size_t)P * m * k1);
      for (int side = 0; side < 2; ++side) {
        const unsigned gblk = (unsigned)std::min<long>(((long)P * m * 32 + 255) / 256, 152L * 32);
        c.kbegin();
        k_scale_cols<T><<<gblk, 256, 0, c.st>>>(P, m, s, nclus, r, NB, side, side ? Rb.p : Lb.p,
                                                scale.p + side * NB * r, F1.p);
        c.kend(KC_COPY, 0, (double)sizeof(T) * 2.0 * P * m * r, "copy:scale_cols");
        c.kbegin();
        k_gather_piv<T><<<gblk, 256, 0, c.st>>>(P, m, s, nclus, r, k1, NB, side, F1.p, piv.p, kk.p, Gc1.p);
        c.kend(KC_COPY, 0, (double)sizeof(T) * 2.0 * P * m * k1, "copy:gather_piv");
        // F1 -= F1[:, piv] W  (the block of a row of cluster c is c ^ side)
        Op<T> A{Gc1.p, k1, 1, (long)m * k1, (long)s * k1, 0, 0, 0};
        Op<T> B{W.p + side * NB * (long)r * r, r, 1, (long)nclus * r * r, (long)r * r, 0, 0, side};
        Op<T> Cm{F1.p, r, 1, (long)m * r, (long)s * r, 0, 0, 0};
        c.tag = "resid";
        gemm<T>(c, s, r, k1, P, nclus, T(-1), A, B, T(1), Cm);
        Op<T> GA{F1.p, 1, r, (long)m * r, (long)s * r, 0, 0, side};
        Op<T> GB{F1.p, r, 1, (long)m * r, (long)s * r, 0, 0, side};
        Op<T> GC{G.p + side * NB * r * (long)r, r, 1, (long)nclus * r * r, (long)r * r, 0, 0, 0};
        c.tag = "gram2";
        gemm_sym<T>(c, r, s, P, nclus, T(1), GA, GB, T(0), GC, false);
      }
      c.kbegin();
      k_mirror_scale<T><<<dim3((unsigned)(2 * NB), (unsigned)std::min(nt * nt, 65535)), 256, 0, c.st>>>(
          r, NB, G.p, nullptr, nullptr);
      c.kend(KC_COPY, 0, 2.0 * NB * sizeof(T) * 1.5 * r * r, "copy:mirror");
      c.kbegin();
      k_pchol<T><<<(unsigned)(2 * NB), thr, sm, c.st>>>(r, G.p, T(floor_rel), T(tau), dmax.p, 1, R.p, piv.p,
                                                        kk.p, nullptr);
      c.kend(KC_PCHOL, 0, 2.0 * NB * sizeof(T) * 2.0 * r * r, site_name(c, "pchol2", s, dens));
    }
  }
  // Ranks of the two factorisations: the core only needs its leading
  // kL x kR block (the truncation kernels read nothing else).
  std::vector<int> hk(2 * NB);
  ACR_CUDA(cudaMemcpyAsync(hk.data(), kk.p, 2 * NB * sizeof(int), cudaMemcpyDeviceToHost, c.st));
  ACR_CUDA(cudaStreamSynchronize(c.st));
  int kmaxL = 0, kmaxR = 0;
  for (long i = 0; i < NB; ++i) {
    kmaxL = std::max(kmaxL, hk[i]);
    kmaxR = std::max(kmaxR, hk[NB + i]);
  }
  if (!qr) {  // pivoted Cholesky: step t updates r entries with t products each
    double f = 0;
    for (long i = 0; i < 2 * NB; ++i) f += (double)r * hk[i] * hk[i];
    c.kc_flops[KC_PCHOL] += f;
  }
  DBuf<T> Cc(c, NB * (size_t)r * r);
  {
    Op<T> A{R.p, r, 1, 0, (long)r * r, 0, 0, 0};
    Op<T> B{R.p + NB * r * (long)r, 1, r, 0, (long)r * r, 0, 0, 0};
    Op<T> C{Cc.p, r, 1, 0, (long)r * r, 0, 0, 0};
    c.tag = "core";
    gemm<T>(c, kmaxL, kmaxR, r, 1, (int)NB, T(1), A, B, T(0), C);
  }
  DBuf<T> Xo, Yo, sig;
  DBuf<int> rank;
  truncate_cores<T>(c, r, Cc.p, kk.p, NB, kmaxL, kmaxR, tol, Xo, Yo, sig, rank, site_name(c, "qrcp", s, dens), 0,
                    nullptr, (long)kmaxL * kmaxR >= 128 * 128 && NB <= 512);
  std::vector<int> hr(NB);
  ACR_CUDA(cudaMemcpyAsync(hr.data(), rank.p, NB * sizeof(int), cudaMemcpyDeviceToHost, c.st));
  ACR_CUDA(cudaStreamSynchronize(c.st));
  Kout = 0;
  for (int v : hr) Kout = std::max(Kout, v);
  if (Kout == 0) {
    Uout.release();
    Vout.release();
    return;
  }
  // Z and the rebuild use the leading kmax rows / factor columns: the
  // pivoted columns (Gram path, gathered below) or Q's first columns (QR path).
  const int kmax = std::max(kmaxL, kmaxR);
  DBuf<T> Z(c, 2 * NB * (size_t)r * Kout);
  DBuf<T> Bscr;
  c.kbegin();
  {
    // column chunk: the widest of 32 / 16 / 8 whose k x C right-hand sides fit
    // in 100 KB of shared memory (two CTAs per SM); else a global scratch.
    const size_t cap = 100 * 1024;
    int Cw = 32;
    while (Cw > 8 && (size_t)kmax * Cw * sizeof(T) > cap) Cw /= 2;
    size_t sm = 0;
    T* gs = nullptr;
    if (!qr) {
      if ((size_t)kmax * Cw * sizeof(T) > cap) {
        Bscr = DBuf<T>(c, 2 * NB * (size_t)r * (size_t)((Kout + Cw - 1) / Cw * Cw));
        gs = Bscr.p;
      } else {
        sm = (size_t)kmax * Cw * sizeof(T);
        if (sm > 48 * 1024)
          ACR_CUDA(cudaFuncSetAttribute(k_coef<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      }
    }
    dim3 grid((unsigned)(2 * NB), (unsigned)((Kout + Cw - 1) / Cw));
    k_coef<T><<<grid, 256, sm, c.st>>>(r, Kout, NB, qr ? 1 : 0, R.p, piv.p, kk.p, Xo.p, Yo.p, sig.p, rank.p,
                                       scale.p, Z.p, Cw, gs, kmax);
  }
  {  // back substitution: k^2 products per coefficient column, both sides
    double f = 0;
    if (!qr)
      for (long i = 0; i < 2 * NB; ++i) f += (double)hk[i] * hk[i] * hr[i % NB];
    c.kend(KC_COEF, f, 2.0 * NB * sizeof(T) * ((double)r * r + (double)r * Kout), site_name(c, "coef", s, dens));
  }
  Uout = DBuf<T>(c, (size_t)P * m * Kout);
  Vout = DBuf<T>(c, (size_t)P * m * Kout);
  for (int side = 0; side < 2; ++side) {
    T* F = side ? Rb.p : Lb.p;
    DBuf<T> Gc;
    Op<T> A{F, r, 1, (long)m * r, (long)s * r, 0, 0, 0};
    if (!qr) {
      Gc = DBuf<T>(c, (size_t)P * m * kmax);
      c.kbegin();
      k_gather_piv<T><<<(unsigned)std::min<long>(((long)P * m * 32 + 255) / 256, 152L * 32), 256, 0, c.st>>>(
          P, m, s, nclus, r, kmax, NB, side, F, piv.p, kk.p, Gc.p);
      c.kend(KC_COPY, 0, (double)sizeof(T) * 2.0 * P * m * kmax, site_name(c, "copy:gather_piv", s, dens));
      A = Op<T>{Gc.p, kmax, 1, (long)m * kmax, (long)s * kmax, 0, 0, 0};
    }
    Op<T> B{Z.p + side * NB * r * (long)Kout, Kout, 1, (long)nclus * r * Kout, (long)r * Kout, 0, 0, side};
    Op<T> C{(side ? Vout.p : Uout.p), Kout, 1, (long)m * Kout, (long)s * Kout, 0, 0, 0};
    c.tag = "rebuild";
    gemm<T>(c, s, Kout, kmax, P, nclus, T(1), A, B, T(0), C);
  }
}

template void recompress_level<float>(Ctx&, int, int, int, DBuf<float>&&, DBuf<float>&&, int, double, bool,
                                      DBuf<float>&, DBuf<float>&, int&);
template void recompress_level<double>(Ctx&, int, int, int, DBuf<double>&&, DBuf<double>&&, int, double, bool,
                                       DBuf<double>&, DBuf<double>&, int&);

}  // namespace acr
