// Dense FP64 factorisation of the coarsest plane (Eq. first_backSubs): the
// single block D^{(q)} left after the last reduction step is small enough to
// be factorised directly.  LU with partial pivoting, one pivot column at a
// time (pivot search, row swap + column scaling, rank-one trailing update,
// each a multi-CTA kernel whose traffic is the trailing matrix), then the
// explicit inverse from two triangular solves with the identity, so that the
// solve phase applies it as one FP64 product.
#include <algorithm>
#include <cmath>

#include "acr_internal.h"

namespace acr {

namespace {
inline int nblk(long tot, int bs = 256, int cap = 152 * 32) {
  long b = (tot + bs - 1) / bs;
  return (int)std::max(1L, std::min<long>(b, cap));
}
}  // namespace

// piv[k] = argmax_{r >= k} |A[r][k]| (one CTA).
__global__ void k_lu_pivot(int m, int k, const double* A, int* piv) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int idx = k;
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
    double v = fabs(A[(long)r * m + k]);
    if (v > best) { best = v; idx = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = idx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s && (bv[threadIdx.x + s] > bv[threadIdx.x] ||
                            (bv[threadIdx.x + s] == bv[threadIdx.x] && bi[threadIdx.x + s] < bi[threadIdx.x]))) {
      bv[threadIdx.x] = bv[threadIdx.x + s];
      bi[threadIdx.x] = bi[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) piv[k] = bi[0];
}

// Swap rows k and piv[k] (all m columns).
__global__ void k_lu_swap(int m, int k, double* A, const int* piv) {
  const int p = piv[k];
  if (p == k) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double t = A[(long)k * m + j];
    A[(long)k * m + j] = A[(long)p * m + j];
    A[(long)p * m + j] = t;
  }
}

// L multipliers of column k and the rank-one update of the trailing block.
// The multipliers are formed from the unscaled column inside the update, so
// one launch suffices; a zero pivot sets flag and is replaced by a tiny one.
__global__ void k_lu_update(int m, int k, double* A, int* flag) {
  const double d0 = A[(long)k * m + k];
  const double d = (d0 != 0.0) ? d0 : 1e-300;
  if (d0 == 0.0 && blockIdx.x == 0 && threadIdx.x == 0 && flag) atomicExch(flag, 1);
  const long rows = m - k - 1, cols = m - k - 1;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rows * (cols + 1); e += (long)gridDim.x * blockDim.x) {
    const long r = k + 1 + e / (cols + 1);
    const long cj = e % (cols + 1);  // 0: the multiplier itself, else trailing column k + cj
    const double l = A[r * m + k] / d;
    if (cj == 0) continue;
    A[r * m + k + cj] -= l * A[(long)k * m + k + cj];
  }
}

__global__ void k_lu_scale(int m, int k, double* A) {
  const double d = A[(long)k * m + k];
  for (int r = k + 1 + blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
    A[(long)r * m + k] = (d != 0.0) ? A[(long)r * m + k] / d : 0.0;
}

// X <- P X (apply the recorded row interchanges, in order, to an m x m matrix).
__global__ void k_lu_apply_piv(int m, double* X, const int* piv) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    for (int k = 0; k < m; ++k) {
      int p = piv[k];
      if (p != k) {
        double t = X[(long)k * m + j];
        X[(long)k * m + j] = X[(long)p * m + j];
        X[(long)p * m + j] = t;
      }
    }
}

// Forward step k of L Y = X (unit lower): rows below k lose L[r][k] * Y[k][:].
__global__ void k_lu_fwd(int m, int k, const double* LU, double* X) {
  const long rows = m - k - 1;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rows * m; e += (long)gridDim.x * blockDim.x) {
    const long r = k + 1 + e / m, j = e % m;
    X[r * m + j] -= LU[r * m + k] * X[(long)k * m + j];
  }
}

// Backward step k of U Z = Y: row k is divided by U[k][k], rows above lose U[r][k] * Z[k][:].
__global__ void k_lu_bwd_scale(int m, int k, const double* LU, double* X) {
  const double d = LU[(long)k * m + k];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) X[(long)k * m + j] /= d;
}
__global__ void k_lu_bwd(int m, int k, const double* LU, double* X) {
  const long rows = k;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rows * m; e += (long)gridDim.x * blockDim.x) {
    const long r = e / m, j = e % m;
    X[r * m + j] -= LU[r * m + k] * X[(long)k * m + j];
  }
}

// Dense inverse of the m x m FP64 matrix A (overwritten by its LU factors).
void dense_inverse_fp64(Ctx& c, int m, double* A, double* Xinv) {
  DBuf<int> piv(c, m);
  const int grid = 152 * 4;
  for (int k = 0; k < m; ++k) {
    c.kbegin();
    k_lu_pivot<<<1, 1024, 0, c.st>>>(m, k, A, piv.p);
    k_lu_swap<<<nblk(m), 256, 0, c.st>>>(m, k, A, piv.p);
    k_lu_update<<<grid, 256, 0, c.st>>>(m, k, A, c.d_flag);
    k_lu_scale<<<nblk(m), 256, 0, c.st>>>(m, k, A);
    c.kend(KC_GJ, 2.0 * (double)(m - k - 1) * (m - k - 1), 16.0 * (double)(m - k) * (m - k));
    c.launches += 3;
  }
  // Xinv = U^{-1} L^{-1} P  by solving A X = I column-block-wise.
  fill<double>(c, Xinv, (long)m * m, 0.0);
  set_identity_clusters<double>(c, 1, m, m, Xinv, m, (long)m * m);
  c.kbegin();
  k_lu_apply_piv<<<nblk(m), 256, 0, c.st>>>(m, Xinv, piv.p);
  c.kend(KC_GJ, 0, 16.0 * (double)m * m);
  for (int k = 0; k < m - 1; ++k) {
    c.kbegin();
    k_lu_fwd<<<grid, 256, 0, c.st>>>(m, k, A, Xinv);
    c.kend(KC_GJ, 2.0 * (double)(m - k - 1) * m, 24.0 * (double)(m - k - 1) * m);
  }
  for (int k = m - 1; k >= 0; --k) {
    c.kbegin();
    k_lu_bwd_scale<<<nblk(m), 256, 0, c.st>>>(m, k, A, Xinv);
    if (k > 0) k_lu_bwd<<<grid, 256, 0, c.st>>>(m, k, A, Xinv);
    c.kend(KC_GJ, 2.0 * (double)k * m, 24.0 * (double)k * m);
    c.launches += 1;
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
