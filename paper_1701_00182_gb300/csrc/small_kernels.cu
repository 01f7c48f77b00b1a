// Element-wise and per-block kernels of the ACR path: fills and panel copies,
// batched Gauss-Jordan inversion (leaves and Woodbury couplings), level-0
// HODLR assembly of the 7-point planes, RHS permutations, and the FP64
// 7-point stencil with its column reductions (residual, refinement, GMRES).
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

template <class T>
__global__ void k_fill(T* p, long n, T v) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] = v;
}
template <class T>
void fill(Ctx& c, T* p, long n, T v) {
  if (n <= 0) return;
  c.kbegin();
  k_fill<T><<<nblk(n), 256, 0, c.st>>>(p, n, v);
  c.kend(KC_COPY, 0, (double)sizeof(T) * n, "copy:fill");
}

// dst[p][row][j] = alpha * src[p][row][j], j < cols.  One warp per row (lanes
// along the row), so the index division happens once per row.
template <class T>
__global__ void k_copy2d(int P, long rows, int cols, T alpha, const T* src, long sld, long sps, T* dst,
                         long dld, long dps) {
  const long nrow = (long)P * rows;
  const int lane = threadIdx.x & 31;
  for (long rw = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; rw < nrow;
       rw += ((long)gridDim.x * blockDim.x) >> 5) {
    const long p = rw / rows, i = rw - p * rows;
    const T* sr = src + p * sps + i * sld;
    T* dr = dst + p * dps + i * dld;
    int j = lane;
    for (; j + 96 < cols; j += 128) {  // four loads in flight per lane
      const T a0 = sr[j], a1 = sr[j + 32], a2 = sr[j + 64], a3 = sr[j + 96];
      dr[j] = alpha * a0;
      dr[j + 32] = alpha * a1;
      dr[j + 64] = alpha * a2;
      dr[j + 96] = alpha * a3;
    }
    for (; j < cols; j += 32) dr[j] = alpha * sr[j];
  }
}
// Narrow rows (cols < 32): one thread per element, 32-bit index arithmetic
// (the caller checks the element count fits), so a warp covers several rows.
template <class T>
__global__ void k_copy2d_narrow(int P, int rows, int cols, T alpha, const T* __restrict__ src, long sld, long sps,
                                T* __restrict__ dst, long dld, long dps) {
  const unsigned tot = (unsigned)P * (unsigned)rows * (unsigned)cols;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const unsigned rw = e / (unsigned)cols, j = e - rw * (unsigned)cols;
    const unsigned p = rw / (unsigned)rows, i = rw - p * (unsigned)rows;
    dst[p * dps + i * dld + j] = alpha * src[p * sps + i * sld + j];
  }
}

template <class T>
void copy2d(Ctx& c, int P, long rows, int cols, T alpha, const T* src, long sld, long sps, T* dst, long dld,
            long dps) {
  long tot = (long)P * rows * cols;
  if (tot <= 0) return;
  if (c.check_bounds) {
    c.check_range(src, 0, (long)(P - 1) * sps + (rows - 1) * sld + cols - 1, sizeof(T), "copy2d src");
    c.check_range(dst, 0, (long)(P - 1) * dps + (rows - 1) * dld + cols - 1, sizeof(T), "copy2d dst");
  }
  c.kbegin();
  if (cols < 32 && tot < (1L << 31) && rows < (1L << 31))
    k_copy2d_narrow<T><<<nblk(tot), 256, 0, c.st>>>(P, (int)rows, cols, alpha, src, sld, sps, dst, dld, dps);
  else
    k_copy2d<T><<<nblk((long)P * rows * 32), 256, 0, c.st>>>(P, rows, cols, alpha, src, sld, sps, dst, dld, dps);
  c.kend(KC_COPY, 0, 2.0 * sizeof(T) * tot, c.site_detail ? (cols < 32 ? "copy:copy2d narrow" : "copy:copy2d") : "copy:copy2d");
}

// Every cluster (size s) of every plane: U|c = I_s  (panel of width s).
template <class T>
__global__ void k_identity(int P, int m, int s, T* U, long ld, long ps) {
  long tot = (long)P * m * s;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    long p = e / ((long)m * s);
    long r = e - p * (long)m * s;
    long i = r / s;
    int j = (int)(r - i * s);
    U[p * ps + i * ld + j] = ((int)(i % s) == j) ? T(1) : T(0);
  }
}
template <class T>
void set_identity_clusters(Ctx& c, int P, int m, int s, T* U, long ld, long ps) {
  long tot = (long)P * m * s;
  if (tot <= 0) return;
  c.kbegin();
  k_identity<T><<<nblk(tot), 256, 0, c.st>>>(P, m, s, U, ld, ps);
  c.kend(KC_COPY, 0, (double)sizeof(T) * tot, "copy:identity");
}

// In-place Gauss-Jordan inversion with partial (row) pivoting, one CTA per
// matrix of order n (row major, matrices `stride` elements apart).  A pivot
// below 64 u max|A| sets flag[0] = 1 and is replaced by that threshold so the
// kernel always finishes.
constexpr int kGJThreads = 1024;
template <class T>
__device__ __forceinline__ void argmax_shfl(T& v, int& i) {
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}
template <class T>
__global__ void __launch_bounds__(kGJThreads) k_gj_inverse(int n, T* A, long stride, int* flag) {
  extern __shared__ unsigned char smraw[];
  T* rowk = reinterpret_cast<T*>(smraw);
  T* fcol = rowk + n;
  int* piv = reinterpret_cast<int*>(fcol + n);
  __shared__ T wv[32];
  __shared__ int wi[32];
  __shared__ T s_thr;
  __shared__ int s_p;
  T* a = A + (long)blockIdx.x * stride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  T mx = T(0);
  for (long e = tid; e < (long)n * n; e += blockDim.x) mx = fmax(mx, fabs(a[e]));
  int dummy = 0;
  argmax_shfl(mx, dummy);
  if (lane == 0) wv[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    T m2 = T(0);
    for (int w = 0; w < nw; ++w) m2 = fmax(m2, wv[w]);
    const T eps = sizeof(T) == 8 ? T(1.1e-16) : T(6e-8);
    s_thr = m2 > T(0) ? T(64) * eps * m2 : T(1e-30);
  }
  __syncthreads();
  const T thr = s_thr;
  for (int k = 0; k < n; ++k) {
    T best = T(-1);
    int bi = 0x7fffffff;
    for (int i = k + tid; i < n; i += blockDim.x) {
      T v = fabs(a[(long)i * n + k]);
      if (v > best) { best = v; bi = i; }
    }
    argmax_shfl(best, bi);
    if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nw ? wv[lane] : T(-1);
      bi = lane < nw ? wi[lane] : 0x7fffffff;
      argmax_shfl(best, bi);
      if (lane == 0) s_p = (bi < n) ? bi : k;
    }
    __syncthreads();
    const int p = s_p;
    if (tid == 0) piv[k] = p;
    if (p != k) {
      for (int j = tid; j < n; j += blockDim.x) {
        T t = a[(long)k * n + j];
        a[(long)k * n + j] = a[(long)p * n + j];
        a[(long)p * n + j] = t;
      }
    }
    __syncthreads();
    T d = a[(long)k * n + k];
    if (!(fabs(d) > thr)) {
      if (tid == 0 && flag) atomicExch(flag, 1);
      d = (d < T(0)) ? -thr : thr;
    }
    const T inv = T(1) / d;
    for (int j = tid; j < n; j += blockDim.x) rowk[j] = (j == k) ? inv : a[(long)k * n + j] * inv;
    for (int i = tid; i < n; i += blockDim.x) fcol[i] = (i == k) ? T(0) : a[(long)i * n + k];
    __syncthreads();
    for (long e = tid; e < (long)n * n; e += blockDim.x) {
      int i = (int)(e / n), j = (int)(e - (long)i * n);
      if (i == k) {
        a[e] = rowk[j];
      } else {
        T f = fcol[i];
        if (f != T(0)) a[e] = ((j == k) ? T(0) : a[e]) - f * rowk[j];
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k) {
      for (int i = tid; i < n; i += blockDim.x) {
        T t = a[(long)i * n + k];
        a[(long)i * n + k] = a[(long)i * n + p];
        a[(long)i * n + p] = t;
      }
    }
    __syncthreads();
  }
}

template <class S, class D>
__global__ void k_convert(long n, const S* a, D* b) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) b[i] = D(a[i]);
}

template <class T>
int batched_inverse(Ctx& c, int nb, int n, T* A, long stride) {
  if (nb <= 0 || n <= 0) return 0;
  if (sizeof(T) == 4 && c.inverse_fp64 && stride == (long)n * n) {
    // Small inverses of the FP32 factorisation carried out in FP64.
    long tot = (long)nb * n * n;
    double* Ad = c.alloc<double>(tot);
    c.kbegin();
    k_convert<T, double><<<nblk(tot), 256, 0, c.st>>>(tot, A, Ad);
    c.kend(KC_COPY, 0, 12.0 * tot, "copy:inv_fp64");
    batched_inverse<double>(c, nb, n, Ad, stride);
    c.kbegin();
    k_convert<double, T><<<nblk(tot), 256, 0, c.st>>>(tot, Ad, A);
    c.kend(KC_COPY, 0, 12.0 * tot, "copy:inv_fp64");
    c.free(Ad, tot);
    return 0;
  }
  size_t sm = 2 * (size_t)n * sizeof(T) + (size_t)n * sizeof(int);
  if (sm > 48 * 1024) ACR_CUDA(cudaFuncSetAttribute(k_gj_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  if (sm > 200 * 1024) throw AcrError(4, "coupling matrix too large");
  c.kbegin();
  const int thr = n <= 64 ? 256 : kGJThreads;
  k_gj_inverse<T><<<nb, thr, sm, c.st>>>(n, A, stride, c.d_flag);
  c.kend(KC_GJ, 2.0 * nb * (double)n * n * n, 2.0 * nb * sizeof(T) * (double)n * n);
  return 0;
}

// ---- level-0 assembly --------------------------------------------------------

__device__ __forceinline__ double harm(double a, double b, double ih2) { return 2.0 * a * b / (a + b) * ih2; }

// Upwind weight of the first-order convection term toward the neighbour in
// direction +e_d (plus = true) or -e_d of a node with velocity component beta:
// beta du/dx_d is differenced against the upstream neighbour, so only that
// neighbour gets -|beta|/h and the diagonal gets +|beta|/h.
__device__ __forceinline__ double upw(double beta, bool plus, double ih) {
  return plus ? fmax(-beta, 0.0) * ih : fmax(beta, 0.0) * ih;
}

// One thread per row of a leaf block of plane k: the 5-point in-plane part
// restricted to the leaf, the full diagonal (6 faces + shift + convection),
// and the diagonal E (to plane k-1) and F (to plane k+1) entries.  vel: the
// convection velocity (3 planar components of n^3 values) or null.
template <class T>
__global__ void k_assemble_leaves(int n, int b, const double* kap, const double* vel, double shift, const int* perm,
                                  const int* iperm, T* DL, T* EL, T* FL) {
  const int m = n * n;
  const long N = (long)m * n;
  const int nleaf = m / b;
  const int k = blockIdx.x / nleaf, lf = blockIdx.x % nleaf;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h), ih = 1.0 / h;
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
    const int pos = lf * b + i;
    const int g = perm[pos];
    const int x = g % n, y = g / n;
    const long node = (long)k * m + g;
    const double kp = kap[node];
    const double bx = vel ? vel[node] : 0.0, by = vel ? vel[N + node] : 0.0, bz = vel ? vel[2 * N + node] : 0.0;
    T* drow = DL + ((long)k * nleaf + lf) * b * b + (long)i * b;
    T* erow = EL + ((long)k * nleaf + lf) * b * b + (long)i * b;
    T* frow = FL + ((long)k * nleaf + lf) * b * b + (long)i * b;
    for (int j = 0; j < b; ++j) { drow[j] = T(0); erow[j] = T(0); frow[j] = T(0); }
    double diag = shift + (fabs(bx) + fabs(by) + fabs(bz)) * ih;
    const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
    for (int d = 0; d < 4; ++d) {
      int xx = x + dx[d], yy = y + dy[d];
      if (xx < 0 || xx >= n || yy < 0 || yy >= n) { diag += kp * ih2; continue; }
      double cpq = harm(kp, kap[(long)k * m + xx + n * yy], ih2);
      diag += cpq;
      const double w = cpq + (d < 2 ? upw(bx, dx[d] > 0, ih) : upw(by, dy[d] > 0, ih));
      int q = iperm[xx + n * yy];
      if (q >= lf * b && q < lf * b + b) drow[q - lf * b] = T(-w);
    }
    if (k > 0) { double cz = harm(kp, kap[node - m], ih2); diag += cz; erow[i] = T(-(cz + upw(bz, false, ih))); }
    else diag += kp * ih2;
    if (k < n - 1) { double cz = harm(kp, kap[node + m], ih2); diag += cz; frow[i] = T(-(cz + upw(bz, true, ih))); }
    else diag += kp * ih2;
    drow[i] = T(diag);
  }
}

// One thread per (plane, cut edge) of a level: the exact low-rank factors of
// the off-diagonal blocks, one column per cut edge (p in the first child,
// q in the second):  U[p,e] = A[p][q],  U[q,e] = A[q][p],  V[p,e] = V[q,e] = 1,
// with A[p][q] = -(c_pq + upwind weight of row p toward q).
template <class T>
__global__ void k_assemble_cuts(int n, int nodes, int ncut, const double* kap, const double* vel, const int* perm,
                                const int* cp, const int* cq, T* U, T* V, long ld, long ps) {
  const int m = n * n;
  const long N = (long)m * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h), ih = 1.0 / h;
  long tot = (long)n * nodes * ncut;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    int k = (int)(e / ((long)nodes * ncut));
    int r = (int)(e - (long)k * nodes * ncut);
    int col = r % ncut;
    int p = cp[r], q = cq[r];
    const int gp = perm[p], gq = perm[q];
    double c = harm(kap[(long)k * m + gp], kap[(long)k * m + gq], ih2);
    double wp = c, wq = c;
    if (vel) {
      // neighbours differ in x (same row of the plane) or in y
      const bool xdir = (gp / n) == (gq / n);
      const bool qplus = xdir ? (gq % n) > (gp % n) : (gq / n) > (gp / n);
      const long off = xdir ? 0 : N;
      wp += upw(vel[off + (long)k * m + gp], qplus, ih);
      wq += upw(vel[off + (long)k * m + gq], !qplus, ih);
    }
    U[k * ps + (long)p * ld + col] = T(-wp);
    U[k * ps + (long)q * ld + col] = T(-wq);
    V[k * ps + (long)p * ld + col] = T(1);
    V[k * ps + (long)q * ld + col] = T(1);
  }
}

template <class T>
void assemble_level0(Ctx& c, const Geometry& geo, const double* kappa, const double* vel, double shift,
                     const int* d_perm, const int* d_iperm, const std::vector<const int*>& d_cutp,
                     const std::vector<const int*>& d_cutq, HMat<T> D, HMat<T> E, HMat<T> F) {
  const int n = geo.n, b = geo.leaf;
  const int nleaf = geo.m / b;
  c.kbegin();
  k_assemble_leaves<T><<<n * nleaf, std::min(b, 128), 0, c.st>>>(n, b, kappa, vel, shift, d_perm, d_iperm,
                                                                 D.leaf, E.leaf, F.leaf);
  c.kend(KC_ASSEMBLE, 0, 3.0 * sizeof(T) * (double)geo.m * b * n);
  for (int l = 0; l < geo.L; ++l) {
    int K = geo.ncut[l];
    fill<T>(c, D.U[l], (long)n * D.pps[l], T(0));
    fill<T>(c, D.V[l], (long)n * D.pps[l], T(0));
    long tot = (long)n * (1L << l) * K;
    c.kbegin();
    k_assemble_cuts<T><<<nblk(tot), 256, 0, c.st>>>(n, 1 << l, K, kappa, vel, d_perm, d_cutp[l], d_cutq[l],
                                                   D.U[l], D.V[l], K, D.pps[l]);
    c.kend(KC_ASSEMBLE, 0, 4.0 * sizeof(T) * (double)tot);
  }
}

// ---- RHS permutations --------------------------------------------------------
// F[k][pos][c] (row major per plane, nrhs contiguous) <-> x[perm[pos] + m k + c ld].

template <class T>
__global__ void k_permute_in(int n, int nrhs, const double* b, long ld, const int* perm, T* F) {
  __shared__ double tile[32][33];
  const int m = n * n;
  const long rowblk = blockIdx.x;  // over (k, pos/32)
  const int k = (int)(rowblk / ((m + 31) / 32));
  const int p0 = (int)(rowblk % ((m + 31) / 32)) * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    int c = c0 + yy, pos = p0 + tx;
    tile[yy][tx] = (c < nrhs && pos < m) ? b[(long)perm[pos] + (long)m * k + (long)c * ld] : 0.0;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    int pos = p0 + yy, c = c0 + tx;
    if (pos < m && c < nrhs) F[((long)k * m + pos) * nrhs + c] = T(tile[tx][yy]);
  }
}
template <class T>
void permute_in(Ctx& c, int n, int nrhs, const double* b, long ld, const int* d_perm, T* F) {
  int m = n * n;
  dim3 grid((unsigned)((long)n * ((m + 31) / 32)), (nrhs + 31) / 32);
  c.kbegin();
  k_permute_in<T><<<grid, dim3(32, 8), 0, c.st>>>(n, nrhs, b, ld, d_perm, F);
  c.kend(KC_PERMUTE, 0, (8.0 + sizeof(T)) * (double)n * m * nrhs);
}

template <class T>
__global__ void k_permute_out(int n, int nrhs, const T* F, const int* perm, double* x, long ld, int acc) {
  __shared__ double tile[32][33];
  const int m = n * n;
  const long rowblk = blockIdx.x;
  const int k = (int)(rowblk / ((m + 31) / 32));
  const int p0 = (int)(rowblk % ((m + 31) / 32)) * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    int pos = p0 + yy, c = c0 + tx;
    tile[yy][tx] = (pos < m && c < nrhs) ? (double)F[((long)k * m + pos) * nrhs + c] : 0.0;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    int c = c0 + yy, pos = p0 + tx;
    if (c < nrhs && pos < m) {
      double* dst = x + (long)perm[pos] + (long)m * k + (long)c * ld;
      *dst = acc ? *dst + tile[tx][yy] : tile[tx][yy];
    }
  }
}
template <class T>
void permute_out(Ctx& c, int n, int nrhs, const T* F, const int* d_perm, double* x, long ld, int accumulate) {
  int m = n * n;
  dim3 grid((unsigned)((long)n * ((m + 31) / 32)), (nrhs + 31) / 32);
  c.kbegin();
  k_permute_out<T><<<grid, dim3(32, 8), 0, c.st>>>(n, nrhs, F, d_perm, x, ld, accumulate);
  c.kend(KC_PERMUTE, 0, (8.0 * (1 + accumulate) + sizeof(T)) * (double)n * m * nrhs);
}

// ---- FP64 7-point stencil ------------------------------------------------------
// coef layout: [4][N] = diagonal (6 faces + shift), coupling to +x, +y, +z.

// Row coefficients of the FP64 operator, 7 planar arrays of n^3: [0] diagonal,
// [1 + 2d] weight of the neighbour at -e_d, [2 + 2d] at +e_d (d = x, y, z), so
// (A u)_p = coef0_p u_p - sum of weight x neighbour (zero where the neighbour
// lies on the boundary).  Diffusion: harmonic-mean face coefficients, boundary
// faces kappa_p / h^2; convection (vel, or null): first-order upwind.
__global__ void k_face_coef(int n, const double* kap, const double* vel, double shift, double* coef) {
  const long N = (long)n * n * n;
  const int m = n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h), ih = 1.0 / h;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
    const int ci[3] = {(int)(p % n), (int)((p / n) % n), (int)(p / m)};
    const long st[3] = {1, n, m};
    const double kp = kap[p];
    double d = shift;
    for (int ax = 0; ax < 3; ++ax) {
      const double be = vel ? vel[ax * N + p] : 0.0;
      d += fabs(be) * ih;
      for (int sg = 0; sg < 2; ++sg) {
        const bool plus = sg == 1;
        const bool in = plus ? ci[ax] < n - 1 : ci[ax] > 0;
        double w = 0.0;
        if (in) {
          const double c = harm(kp, kap[plus ? p + st[ax] : p - st[ax]], ih2);
          d += c;
          w = c + upw(be, plus, ih);
        } else {
          d += kp * ih2;
        }
        coef[(1 + 2 * ax + sg) * N + p] = w;
      }
    }
    coef[p] = d;
  }
}
void face_coefficients(Ctx& c, int n, const double* kappa, const double* vel, double shift, double* coef) {
  long N = (long)n * n * n;
  c.kbegin();
  k_face_coef<<<nblk(N), 256, 0, c.st>>>(n, kappa, vel, shift, coef);
  c.kend(KC_STENCIL, 0, (vel ? 11.0 : 8.0) * 8.0 * N);
}

// out = alpha * A x + beta * y (trans: A^T x); optional per-column partial
// sums of out^2 and y^2.  Row p of A^T takes, from the neighbour q = p + e,
// the weight of row q toward p (direction -e).
__global__ void k_stencil(int n, int nrhs, const double* __restrict__ coef, const double* __restrict__ x, long ld,
                          const double* y, double* out, double alpha, double beta, double* part, int trans) {
  const long N = (long)n * n * n;
  const int m = n * n;
  const int col = blockIdx.y;
  __shared__ double s1[256], s2[256];
  double a1 = 0, a2 = 0;
  const double* xc = x + (long)col * ld;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
    const int ci[3] = {(int)(p % n), (int)((p / n) % n), (int)(p / m)};
    const long st[3] = {1, n, m};
    double v = coef[p] * xc[p];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (ci[ax] > 0) {
        const long q = p - st[ax];
        v -= (trans ? coef[(2 + 2 * ax) * N + q] : coef[(1 + 2 * ax) * N + p]) * xc[q];
      }
      if (ci[ax] < n - 1) {
        const long q = p + st[ax];
        v -= (trans ? coef[(1 + 2 * ax) * N + q] : coef[(2 + 2 * ax) * N + p]) * xc[q];
      }
    }
    double yv = (beta != 0.0) ? y[(long)col * ld + p] : 0.0;
    double o = alpha * v + beta * yv;
    out[(long)col * ld + p] = o;
    a1 += o * o;
    a2 += yv * yv;
  }
  if (!part) return;
  s1[threadIdx.x] = a1;
  s2[threadIdx.x] = a2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { s1[threadIdx.x] += s1[threadIdx.x + s]; s2[threadIdx.x] += s2[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((long)col * gridDim.x + blockIdx.x) * 2] = s1[0];
    part[((long)col * gridDim.x + blockIdx.x) * 2 + 1] = s2[0];
  }
}

__global__ void k_reduce_pairs(int nrhs, int nparts, const double* part, double* out) {
  int col = blockIdx.x;
  __shared__ double s1[256], s2[256];
  double a1 = 0, a2 = 0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    a1 += part[((long)col * nparts + i) * 2];
    a2 += part[((long)col * nparts + i) * 2 + 1];
  }
  s1[threadIdx.x] = a1;
  s2[threadIdx.x] = a2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { s1[threadIdx.x] += s1[threadIdx.x + s]; s2[threadIdx.x] += s2[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[2 * col] = s1[0]; out[2 * col + 1] = s2[0]; }
}

void stencil_apply(Ctx& c, int n, int nrhs, const double* coef, const double* x, long ld, const double* y,
                   double* out, double alpha, double beta, double* norms_out, bool trans) {
  long N = (long)n * n * n;
  int nb = (int)std::min<long>((N + 255) / 256, 1024);
  double* part = nullptr;
  if (norms_out) part = c.alloc<double>((size_t)nb * nrhs * 2);
  c.kbegin();
  k_stencil<<<dim3(nb, nrhs), 256, 0, c.st>>>(n, nrhs, coef, x, ld, y, out, alpha, beta, part, trans ? 1 : 0);
  c.kend(KC_STENCIL, 15.0 * N * nrhs, 8.0 * (7.0 * N + N * nrhs * (2.0 + (beta != 0.0))));
  if (norms_out) {
    c.kbegin();
    k_reduce_pairs<<<nrhs, 256, 0, c.st>>>(nrhs, nb, part, norms_out);
    c.kend(KC_STENCIL, 0, 16.0 * nb * nrhs);
    c.free(part, (size_t)nb * nrhs * 2);
  }
}

// Same kernels as stencil_apply with norms, but the per-block partial sums and
// the per-column pairs live in caller-provided device scratch: part holds
// nb_max * nrhs * 2 doubles, pairs 2 * nrhs.  Every entry read is written
// earlier in the same call, so the scratch needs no clearing.  Allocates nothing.
void stencil_norms_scratch(cudaStream_t st, int n, int nrhs, const double* coef, const double* x, long ld,
                           const double* y, double* out, double* part, int nb_max, double* pairs) {
  long N = (long)n * n * n;
  int nb = (int)std::min<long>((N + 255) / 256, nb_max);
  k_stencil<<<dim3(nb, nrhs), 256, 0, st>>>(n, nrhs, coef, x, ld, y, out, -1.0, 1.0, part, 0);
  k_reduce_pairs<<<nrhs, 256, 0, st>>>(nrhs, nb, part, pairs);
}

// dL/dg_p = -kappa_p * sum over columns of lambda^T (dA/dkappa_p) u, with
// dc_pq/dkappa_p = 2 kappa_q^2 / ((kappa_p + kappa_q)^2 h^2) on interior faces
// and 1/h^2 on boundary faces (u = 0 outside).  One thread per node.
__global__ void k_grad_logkappa(int n, int nrhs, const double* __restrict__ kap, const double* __restrict__ u,
                                const double* __restrict__ lam, long ld, double* grad, int accumulate) {
  const long N = (long)n * n * n;
  const int m = n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
    const int xi = (int)(p % n), yi = (int)((p / n) % n), zi = (int)(p / m);
    const double kp = kap[p];
    const long nb[6] = {xi > 0 ? p - 1 : -1, xi < n - 1 ? p + 1 : -1, yi > 0 ? p - n : -1,
                        yi < n - 1 ? p + n : -1, zi > 0 ? p - m : -1, zi < n - 1 ? p + m : -1};
    double acc = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      const double up = u[(long)c * ld + p], lp = lam[(long)c * ld + p];
      for (int d = 0; d < 6; ++d) {
        const long q = nb[d];
        if (q < 0) {
          acc += lp * up * ih2;
        } else {
          const double kq = kap[q];
          const double dc = 2.0 * kq * kq / ((kp + kq) * (kp + kq)) * ih2;
          acc += dc * (lp - lam[(long)c * ld + q]) * (up - u[(long)c * ld + q]);
        }
      }
    }
    const double v = -kp * acc;
    grad[p] = accumulate ? grad[p] + v : v;
  }
}
void grad_logkappa(Ctx& c, int n, int nrhs, const double* kap, const double* u, const double* lam, long ld,
                   double* grad, int accumulate) {
  long N = (long)n * n * n;
  c.kbegin();
  k_grad_logkappa<<<nblk(N), 256, 0, c.st>>>(n, nrhs, kap, u, lam, ld, grad, accumulate);
  c.kend(KC_STENCIL, 40.0 * N * nrhs, 8.0 * (N + 2.0 * N * nrhs + N));
}

__global__ void k_col_dots(long N, const double* x, long ldx, const double* y, long ldy, double* part) {
  int col = blockIdx.y;
  __shared__ double s1[256];
  double a = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    a += x[(long)col * ldx + i] * y[(long)col * ldy + i];
  s1[threadIdx.x] = a;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) s1[threadIdx.x] += s1[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((long)col * gridDim.x + blockIdx.x) * 2] = s1[0];
    part[((long)col * gridDim.x + blockIdx.x) * 2 + 1] = 0.0;
  }
}
void col_dots(Ctx& c, long N, int nrhs, const double* x, long ldx, const double* y, long ldy, double* out) {
  int nb = (int)std::min<long>((N + 255) / 256, 512);
  double* part = c.alloc<double>((size_t)nb * nrhs * 2);
  double* pairs = c.alloc<double>((size_t)nrhs * 2);
  c.kbegin();
  k_col_dots<<<dim3(nb, nrhs), 256, 0, c.st>>>(N, x, ldx, y, ldy, part);
  c.kend(KC_STENCIL, 2.0 * N * nrhs, 16.0 * N * nrhs);
  c.kbegin();
  k_reduce_pairs<<<nrhs, 256, 0, c.st>>>(nrhs, nb, part, pairs);
  c.kend(KC_STENCIL, 0, 16.0 * nb * nrhs);
  c.kbegin();
  k_copy2d<double><<<1, 64, 0, c.st>>>(1, nrhs, 1, 1.0, pairs, 2, 0, out, 1, 0);
  c.kend(KC_COPY, 0, 16.0 * nrhs, "copy:norms");
  c.free(part, (size_t)nb * nrhs * 2);
  c.free(pairs, (size_t)nrhs * 2);
}

__global__ void k_col_axpy(long N, int nrhs, const double* a, const double* x, long ldx, double* y, long ldy,
                           int overwrite) {
  long tot = N * nrhs;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    int col = (int)(e / N);
    long i = e - (long)col * N;
    double v = a[col] * x[(long)col * ldx + i];
    if (overwrite) y[(long)col * ldy + i] = v;
    else y[(long)col * ldy + i] += v;
  }
}
void col_axpy(Ctx& c, long N, int nrhs, const double* a, const double* x, long ldx, double* y, long ldy) {
  c.kbegin();
  k_col_axpy<<<nblk(N * nrhs), 256, 0, c.st>>>(N, nrhs, a, x, ldx, y, ldy, 0);
  c.kend(KC_STENCIL, 2.0 * N * nrhs, 24.0 * N * nrhs);
}
void col_scale_copy(Ctx& c, long N, int nrhs, const double* a, const double* x, long ldx, double* y, long ldy) {
  c.kbegin();
  k_col_axpy<<<nblk(N * nrhs), 256, 0, c.st>>>(N, nrhs, a, x, ldx, y, ldy, 1);
  c.kend(KC_STENCIL, 2.0 * N * nrhs, 24.0 * N * nrhs);
}


// dst[p][row][j] += alpha * src[p][row][j], j < cols (one warp per row).
template <class T>
__global__ void k_axpy2d(int P, long rows, int cols, T alpha, const T* src, long sld, long sps, T* dst, long dld,
                         long dps) {
  const long nrow = (long)P * rows;
  const int lane = threadIdx.x & 31;
  for (long rw = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; rw < nrow;
       rw += ((long)gridDim.x * blockDim.x) >> 5) {
    const long p = rw / rows, i = rw - p * rows;
    const T* sr = src + p * sps + i * sld;
    T* dr = dst + p * dps + i * dld;
    for (int j = lane; j < cols; j += 32) dr[j] += alpha * sr[j];
  }
}
template <class T>
void axpy2d(Ctx& c, int P, long rows, int cols, T alpha, const T* src, long sld, long sps, T* dst, long dld,
            long dps) {
  long tot = (long)P * rows * cols;
  if (tot <= 0) return;
  if (c.check_bounds) {
    c.check_range(src, 0, (long)(P - 1) * sps + (rows - 1) * sld + cols - 1, sizeof(T), "axpy2d src");
    c.check_range(dst, 0, (long)(P - 1) * dps + (rows - 1) * dld + cols - 1, sizeof(T), "axpy2d dst");
  }
  c.kbegin();
  k_axpy2d<T><<<nblk((long)P * rows * 32), 256, 0, c.st>>>(P, rows, cols, alpha, src, sld, sps, dst, dld, dps);
  c.kend(KC_COPY, 0, 3.0 * sizeof(T) * tot, "copy:axpy2d");
}

// Dense m x m image of the leaf blocks of one HODLR matrix (off-diagonal zero).
template <class T>
__global__ void k_expand_leaves(int m, int b, const T* leaf, T* dense) {
  long tot = (long)m * b;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    long row = e / b;
    int j = (int)(e % b);
    long lf = row / b;
    dense[row * m + lf * b + j] = leaf[e];
  }
}
template <class T>
void expand_leaves(Ctx& c, int m, int b, const T* leaf, T* dense) {
  c.kbegin();
  k_expand_leaves<T><<<nblk((long)m * b), 256, 0, c.st>>>(m, b, leaf, dense);
  c.kend(KC_COPY, 0, 2.0 * sizeof(T) * (double)m * b, "copy:expand_leaves");
}

__global__ void k_exp_inplace(double* p, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] = exp(p[i]);
}
// flag = 1 if any entry is NaN or infinite (or, with positive, not > 0).
__global__ void k_flag_invalid(const double* p, long n, int positive, int* flag) {
  bool bad = false;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = p[i];
    bad |= !isfinite(v) || (positive && !(v > 0.0));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

void flag_invalid(Ctx& c, const double* p, long n, bool positive, int* flag) {
  c.kbegin();
  k_flag_invalid<<<nblk(n), 256, 0, c.st>>>(p, n, positive ? 1 : 0, flag);
  c.kend(KC_ASSEMBLE, 0, 8.0 * n);
}

void exp_inplace(Ctx& c, double* p, long n) {
  c.kbegin();
  k_exp_inplace<<<nblk(n), 256, 0, c.st>>>(p, n);
  c.kend(KC_ASSEMBLE, 0, 16.0 * n);
}

#define INST(T)                                                                                          \
  template void fill<T>(Ctx&, T*, long, T);                                                              \
  template void copy2d<T>(Ctx&, int, long, int, T, const T*, long, long, T*, long, long);                \
  template void set_identity_clusters<T>(Ctx&, int, int, int, T*, long, long);                           \
  template int batched_inverse<T>(Ctx&, int, int, T*, long);                                             \
  template void assemble_level0<T>(Ctx&, const Geometry&, const double*, const double*, double, const int*, \
                                   const int*,                                                           \
                                   const std::vector<const int*>&, const std::vector<const int*>&,       \
                                   HMat<T>, HMat<T>, HMat<T>);                                           \
  template void permute_in<T>(Ctx&, int, int, const double*, long, const int*, T*);                      \
  template void permute_out<T>(Ctx&, int, int, const T*, const int*, double*, long, int);                \
  template void axpy2d<T>(Ctx&, int, long, int, T, const T*, long, long, T*, long, long);                \
  template void expand_leaves<T>(Ctx&, int, int, const T*, T*);
INST(float)
INST(double)
template void fill<int>(Ctx&, int*, long, int);
#undef INST

}  // namespace acr
