// Dense FP64 factorisation of the coarsest plane (Eq. first_backSubs): the
// single block D^{(q)} left after the last reduction step is small enough to
// be factorised directly.  Blocked right-looking LU with partial pivoting
// (panels of 64 columns: each panel column is a pivot search + swap by one
// CTA and a row-parallel update of the panel, the panel's row swaps are then
// applied to the other columns, U12 comes from a unit-lower triangular solve,
// and the trailing block is updated by one FP64 GEMM), then the explicit
// inverse from A X = P by blocked forward and backward substitution (a
// triangular solve per diagonal block, a GEMM per off-diagonal update), so
// that the solve phase applies it as one FP64 product.
#include <algorithm>
#include <cmath>

#include "acr_internal.h"
#include "hodlr.cuh"

namespace acr {

namespace {
inline int nblk(long tot, int bs = 256, int cap = 152 * 32) {
  long b = (tot + bs - 1) / bs;
  return (int)std::max(1L, std::min<long>(b, cap));
}
constexpr int kNB = 64;  // panel width
}  // namespace

// Column col of the panel (columns k0..k0+jb-1): piv[col] = argmax over rows
// r >= col of |A[r][col]| (lowest index on ties), and rows col and piv[col]
// swapped across the panel.  One CTA.
__global__ void __launch_bounds__(1024) k_panel_pivot(int m, int col, int k0, int jb, double* A, int* piv) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double best = -1.0;
  int idx = 0x7fffffff;
  for (int r = col + tid; r < m; r += blockDim.x) {
    const double v = fabs(A[(long)r * m + col]);
    if (v > best) { best = v; idx = r; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > best || (ov == best && oi < idx)) { best = ov; idx = oi; }
  }
  if (lane == 0) { bv[warp] = best; bi[warp] = idx; }
  __syncthreads();
  if (tid == 0) {
    double b = -1.0;
    int bb = col;
    for (int w = 0; w < nw; ++w)
      if (bv[w] > b || (bv[w] == b && bi[w] < bb)) { b = bv[w]; bb = bi[w]; }
    s_p = bb;
    piv[col] = bb;
  }
  __syncthreads();
  const int p = s_p;
  if (p != col && tid < jb) {
    const double t = A[(long)col * m + k0 + tid];
    A[(long)col * m + k0 + tid] = A[(long)p * m + k0 + tid];
    A[(long)p * m + k0 + tid] = t;
  }
}

// Rows below col: multiplier l = A[r][col] / A[col][col] stored in place and
// the panel's remaining columns updated, one warp per row (lanes along the
// row).  A zero pivot sets flag and is replaced by a tiny one.
__global__ void k_panel_update(int m, int col, int k0, int jb, double* A, int* flag) {
  const int lane = threadIdx.x & 31;
  const double d0 = A[(long)col * m + col];
  const double d = (d0 != 0.0) ? d0 : 1e-300;
  if (d0 == 0.0 && blockIdx.x == 0 && threadIdx.x == 0 && flag) atomicExch(flag, 1);
  const double* prow = A + (long)col * m;
  const int c1 = k0 + jb;
  for (long r = col + 1 + ((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5); r < m;
       r += ((long)gridDim.x * blockDim.x) >> 5) {
    double* ar = A + r * m;
    const double l = ar[col] / d;  // every lane reads it before lane 0 overwrites it
    __syncwarp();
    for (int c2 = col + 1 + lane; c2 < c1; c2 += 32) ar[c2] -= l * prow[c2];
    if (lane == 0) ar[col] = l;
  }
}

// Row swaps k0..k0+jb-1 (in order) applied to the columns outside the panel.
__global__ void k_swap_rows(int m, int k0, int jb, double* A, const int* piv) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    if (j >= k0 && j < k0 + jb) continue;
    for (int i = k0; i < k0 + jb; ++i) {
      const int p = piv[i];
      if (p != i) {
        const double t = A[(long)i * m + j];
        A[(long)i * m + j] = A[(long)p * m + j];
        A[(long)p * m + j] = t;
      }
    }
  }
}

// B rows k0..k0+jb-1, columns c0.. (one thread per column) <- L11^{-1} B with
// L11 the unit lower block of T at (k0, k0) (upper = false), or U11^{-1} B
// with U11 its upper block, diagonal included (upper = true).
__global__ void __launch_bounds__(256) k_trsm_block(int m, int k0, int jb, const double* T, double* B, int c0,
                                                    int ncols, int upper) {
  __shared__ double t11[kNB][kNB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) t11[e / jb][e % jb] = T[(long)(k0 + e / jb) * m + k0 + e % jb];
  __syncthreads();
  for (int j = c0 + blockIdx.x * blockDim.x + threadIdx.x; j < c0 + ncols; j += gridDim.x * blockDim.x) {
    double* bj = B + (long)k0 * m + j;
    if (!upper) {
      for (int i = 1; i < jb; ++i) {
        double v = bj[(long)i * m];
        for (int t = 0; t < i; ++t) v -= t11[i][t] * bj[(long)t * m];
        bj[(long)i * m] = v;
      }
    } else {
      for (int i = jb - 1; i >= 0; --i) {
        double v = bj[(long)i * m];
        for (int t = i + 1; t < jb; ++t) v -= t11[i][t] * bj[(long)t * m];
        bj[(long)i * m] = v / t11[i][i];
      }
    }
  }
}

// X = P (the row interchanges applied to the identity): row i of X is e_{perm[i]}.
__global__ void k_perm_identity(int m, const int* piv, int* perm, double* X) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int k = 0; k < m; ++k) {
      const int p = piv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
}
__global__ void k_perm_fill(int m, const int* perm, double* X) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)m * m; e += (long)gridDim.x * blockDim.x) {
    const long i = e / m, j = e % m;
    X[e] = (perm[i] == j) ? 1.0 : 0.0;
  }
}

// Dense inverse of the m x m FP64 matrix A (overwritten by its LU factors).
void dense_inverse_fp64(Ctx& c, int m, double* A, double* Xinv) {
  DBuf<int> piv(c, m), perm(c, m);
  const int cgrid = std::min(152 * 4, (m + 255) / 256);
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int jb = std::min(kNB, m - k0), rest = m - k0 - jb;
    c.kbegin();
    for (int j = 0; j < jb; ++j) {
      const int col = k0 + j, rows = m - col - 1;
      k_panel_pivot<<<1, 1024, 0, c.st>>>(m, col, k0, jb, A, piv.p);
      if (rows > 0) k_panel_update<<<std::max(1, std::min((rows + 7) / 8, 152 * 8)), 256, 0, c.st>>>(m, col, k0, jb, A, c.d_flag);
    }
    c.launches += 2 * jb;
    k_swap_rows<<<cgrid, 256, 0, c.st>>>(m, k0, jb, A, piv.p);
    if (rest > 0) k_trsm_block<<<(rest + 255) / 256, 256, 0, c.st>>>(m, k0, jb, A, A, k0 + jb, rest, 0);
    c.kend(KC_GJ, (double)(m - k0) * jb * jb + (double)rest * jb * jb, 16.0 * (double)(m - k0) * jb);
    c.launches += 2;
    if (rest > 0) {
      c.tag = "coarse_lu";
      gemm<double>(c, rest, rest, jb, 1, 1, -1.0, opm<double>(A + (long)(k0 + jb) * m + k0, m, 1, 0, 0),
                   opm<double>(A + (long)k0 * m + k0 + jb, m, 1, 0, 0), 1.0,
                   opm<double>(A + (long)(k0 + jb) * m + k0 + jb, m, 1, 0, 0));
    }
  }
  // Xinv = U^{-1} L^{-1} P: A X = P by blocked forward then backward substitution.
  c.kbegin();
  k_perm_identity<<<1, 32, 0, c.st>>>(m, piv.p, perm.p, Xinv);
  k_perm_fill<<<nblk((long)m * m), 256, 0, c.st>>>(m, perm.p, Xinv);
  c.kend(KC_GJ, 0, 8.0 * (double)m * m);
  c.launches += 1;
  const int tgrid = (m + 255) / 256;
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int jb = std::min(kNB, m - k0), rest = m - k0 - jb;
    c.kbegin();
    k_trsm_block<<<tgrid, 256, 0, c.st>>>(m, k0, jb, A, Xinv, 0, m, 0);
    c.kend(KC_GJ, (double)m * jb * jb, 16.0 * (double)m * jb);
    if (rest > 0) {
      c.tag = "coarse_inv";
      gemm<double>(c, rest, m, jb, 1, 1, -1.0, opm<double>(A + (long)(k0 + jb) * m + k0, m, 1, 0, 0),
                   opm<double>(Xinv + (long)k0 * m, m, 1, 0, 0), 1.0, opm<double>(Xinv + (long)(k0 + jb) * m, m, 1, 0, 0));
    }
  }
  for (int k0 = (m - 1) / kNB * kNB; k0 >= 0; k0 -= kNB) {
    const int jb = std::min(kNB, m - k0);
    c.kbegin();
    k_trsm_block<<<tgrid, 256, 0, c.st>>>(m, k0, jb, A, Xinv, 0, m, 1);
    c.kend(KC_GJ, (double)m * jb * jb, 16.0 * (double)m * jb);
    if (k0 > 0) {
      c.tag = "coarse_inv";
      gemm<double>(c, k0, m, jb, 1, 1, -1.0, opm<double>(A + k0, m, 1, 0, 0), opm<double>(Xinv + (long)k0 * m, m, 1, 0, 0),
                   1.0, opm<double>(Xinv, m, 1, 0, 0));
    }
  }
}

template <class S, class D>
__global__ void k_cvt(long n, const S* a, D* b) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) b[i] = D(a[i]);
}

template <class S, class D>
void convert(Ctx& c, long n, const S* a, D* b) {
  if (n <= 0) return;
  c.kbegin();
  k_cvt<S, D><<<nblk(n), 256, 0, c.st>>>(n, a, b);
  c.kend(KC_COPY, 0, (double)(sizeof(S) + sizeof(D)) * n, "copy:convert");
}

template void convert<float, double>(Ctx&, long, const float*, double*);
template void convert<double, float>(Ctx&, long, const double*, float*);
template void convert<double, double>(Ctx&, long, const double*, double*);

}  // namespace acr
