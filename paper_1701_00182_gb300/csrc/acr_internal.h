// Internal declarations of the GB300 ACR library: device buffers, batched
// HODLR matrix views, the batched GEMM operand descriptor and the launchers.
//
// Layout conventions (all per plane, planes of one batch at a fixed stride):
//   * a plane's n^2 unknowns are permuted so every cluster of the 2D bisection
//     tree (Section 3.1) is a contiguous index range; the level-l clusters
//     (l = 1..L) have size m >> l, the leaves have size b = m >> L;
//   * HODLR leaves: 2^L dense b x b blocks, row major, leaf-major;
//   * HODLR level l (l = 0..L-1): two row-major m x K_l panels U_l, V_l.
//     For the level-(l+1) cluster c and its sibling c^1 the off-diagonal block
//     M[c, c^1] = U_l|c * (V_l|c^1)^T  (rows of c in U, rows of c^1 in V);
//     columns beyond a block's rank are zero.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <array>
#include <map>
#include <set>
#include <string>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

namespace acr {

constexpr int MAXL = 16;

struct AcrError : std::runtime_error {
  int code;
  AcrError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define ACR_CUDA(x)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess) {                                                             \
      if (e_ == cudaErrorMemoryAllocation) throw ::acr::AcrError(2, cudaGetErrorString(e_)); \
      throw ::acr::AcrError(5, std::string(#x) + ": " + cudaGetErrorString(e_));         \
    }                                                                                    \
  } while (0)

// Kernel classes for the per-class profile (CUDA events on the launch stream).
enum KClass { KC_GEMM, KC_SPLITK, KC_QR, KC_PCHOL, KC_JACOBI, KC_COEF, KC_GJ, KC_COPY, KC_ASSEMBLE, KC_PERMUTE,
              KC_STENCIL, KC_GEMM_TC, KC_HEXPAND, KC_TF32SPLIT, KC_N };

// Execution context of one handle: stream, scratch, counters, autotune cache.
struct Ctx {
  cudaStream_t st = nullptr;
  int* d_flag = nullptr;            // device status flags (breakdown ...)
  double* d_jflops = nullptr;       // device count of Jacobi SVD flops (pair evaluations + rotations)
  long long launches = 0;
  long long gemm_flops = 0;
  size_t live_bytes = 0, peak_bytes = 0, budget = 0;
  bool autotune = false;
  std::map<uintptr_t, size_t> live;  // allocation start -> bytes (for the operand extent check)
  bool check_bounds = false;  // ACR_CHECK_BOUNDS=1: verify every GEMM operand range on the host
  bool verify_gemm = false;   // ACR_GEMM_VERIFY=1: recompute every GEMM with the reference FMA tiling and report differences
  bool inverse_fp64 = false;  // FP32 factorisation: leaf and coupling inverses in FP64
  bool tensor = false;        // FP32 GEMMs of large tiles on the tensor cores (3xTF32)
  int force_cfg = -1;         // ACR_GEMM_CFG=<i>: every GEMM uses tiling i where it is valid (debugging)
  int chol_passes = 1;         // pivoted-Cholesky passes of the FP32 recompression (1 = Gram floor only)
  bool qrcp_cluster = true;    // pivoted QR of large cores / explicit blocks on a thread-block cluster
  bool qrcp_reg = true;        // FP32 blocks up to 512 x 512: the register-resident cluster variant (ACR_QRCP_REG=0: off)
  bool qrcp_reg_all = false;   // ACR_QRCP_REG=2: also the blocks that fit one CTA's shared memory
  bool qrcp_blocked = false;   // ACR_QRCP_BLOCKED=1: several pivots per cluster barrier (not yet run on a GPU)
  int core_svd = 0;           // core truncation: 0 / 2 pivoted QR (default), 1 Jacobi SVD
  void check_range(const void* base, long lo, long hi, size_t es, const char* what) const;
  bool profile = false;  // record CUDA events around every launch, accumulated per kernel class
  double kc_ms[16] = {}, kc_flops[16] = {}, kc_bytes[16] = {};
  long long kc_launch[16] = {};
  struct PendingEv { cudaEvent_t a, b; int cls; const char* tag; };
  const char* tag = "other";  // call site of the next GEMM (profile breakdown)
  bool site_detail = false;   // ACR_PROFILE_SITES=2: split each site by GEMM shape and tiling
  std::set<std::string> tagstore;
  std::map<std::string, std::pair<double, double>> site;  // tag -> (ms, flops)
  std::map<std::string, double> gap;  // tag (or class) of a launch -> device idle time before it (ms)
  std::vector<cudaEvent_t> evfree;
  std::vector<PendingEv> pend;
  cudaEvent_t evcur = nullptr;
  void kbegin();
  // name: label of a non-GEMM launch in the per-site profile (ACR_PROFILE_SITES=2; its bytes are recorded)
  void kend(int cls, double flops, double bytes, const char* name = nullptr);
  void kflush();
  void* dalloc_bytes(size_t bytes);
  void dfree(void* p, size_t bytes);
  template <class T> T* alloc(size_t n) { return static_cast<T*>(dalloc_bytes(n * sizeof(T))); }
  template <class T> void free(T* p, size_t n) { dfree(p, n * sizeof(T)); }
};

// Owned device buffer with size bookkeeping.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  Ctx* c = nullptr;
  DBuf() = default;
  DBuf(Ctx& ctx, size_t cnt, bool zero = false);
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; c = o.c; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release();
};

// Batched GEMM operand: element (i, j) of batch entry (plane, cluster c) is
//   p[plane*ps + (cc >> sh)*c1 + (cc & 1)*c2 + i*rs + j*cs],  cc = sib ? c^1 : c.
template <class T>
struct Op {
  T* p = nullptr;
  long rs = 0, cs = 0, ps = 0, c1 = 0, c2 = 0;
  int sh = 0, sib = 0;
};

// C = alpha * A(MxK) * B(KxN) + beta * C over nplanes x nclus batch entries.
template <class T>
void gemm(Ctx& c, int M, int N, int K, int nplanes, int nclus, T alpha, Op<T> A, Op<T> B, T beta,
          Op<T> C);

// C = alpha * A B + beta * C for symmetric C (M x M, A = B^T): the upper triangle is computed, then
// mirrored; with mirror = false the entries below the diagonal are left unspecified.
template <class T>
void gemm_sym(Ctx& c, int M, int K, int nplanes, int nclus, T alpha, Op<T> A, Op<T> B, T beta, Op<T> C,
              bool mirror = true);

// Fused HODLR x panel expansion (leaf product + every level's expansion).
template <class T>
struct HexpArgs {
  int m = 0, b = 0, w = 0, nl = 0, leaf_trans = 0;
  const T* leaf = nullptr;
  long lps = 0;
  const T* W = nullptr;
  long wld = 0, wps = 0;
  T* Y = nullptr;
  long yld = 0, yps = 0;
  T alpha = T(1), beta = T(0);
  const T* U[MAXL] = {};
  long ups[MAXL] = {};
  const T* C[MAXL] = {};
  int K[MAXL] = {}, s[MAXL] = {}, nclus[MAXL] = {};
  int ncol[MAXL] = {};  // level applies to the first ncol columns; its coefficient rows have stride ncol
};
template <class T>
void hexpand(Ctx& c, const HexpArgs<T>& a, int P);

// Panel view: rows m per plane, element (row, col) at p[plane*ps + row*ld + col].
template <class T>
struct Pan {
  T* p = nullptr;
  long ld = 0, ps = 0;
};

// View of P HODLR matrices (planes at stride lps / pps[l]).
template <class T>
struct HMat {
  int P = 0, m = 0, L = 0, b = 0;
  T* leaf = nullptr;
  long lps = 0;
  T* U[MAXL] = {};
  T* V[MAXL] = {};
  int K[MAXL] = {};
  long pps[MAXL] = {};
  HMat sub(int p0, int step, int count) const {
    HMat r = *this;
    r.P = count;
    r.leaf = leaf + (long)p0 * lps;
    r.lps = lps * step;
    for (int l = 0; l < L; ++l) {
      if (U[l]) { r.U[l] = U[l] + (long)p0 * pps[l]; r.V[l] = V[l] + (long)p0 * pps[l]; }
      r.pps[l] = pps[l] * step;
    }
    return r;
  }
  long bytes() const {
    long s = (long)P * m * b;
    for (int l = 0; l < L; ++l) s += 2L * P * m * K[l];
    return s * (long)sizeof(T);
  }
};

// Owner of a contiguous batch of HODLR matrices.
template <class T>
struct HStore {
  DBuf<T> leaf;
  DBuf<T> U[MAXL], V[MAXL];
  HMat<T> h;
  HStore() = default;
  HStore(HStore&&) = default;
  HStore& operator=(HStore&&) = default;
};

// Planner output (host): cluster tree of one n x n plane.
struct Geometry {
  int n = 0, m = 0, leaf = 0, L = 0;
  std::vector<int> perm;              // permuted position -> lexicographic in-plane index
  std::vector<int> ncut;              // per level: cut edges per node
  std::vector<std::vector<int>> cutp, cutq;  // per level: [node*ncut + e] positions
};
int plan_geometry(int n, int leaf, Geometry& g);  // 0 or ACR_ERR_ARG
// Leaves of the block cluster tree of one plane: (level, t, s, low rank); eta < 0 = weak.
int plan_blocks(int n, int leaf, double eta, std::vector<std::array<int, 4>>& out);  // 0 or 1 (bad argument)

// ---- small kernels (small_kernels.cu) -------------------------------------
template <class T> void fill(Ctx& c, T* p, long n, T v);
template <class T> void copy2d(Ctx& c, int P, long rows, int cols, T alpha, const T* src, long sld,
                               long sps, T* dst, long dld, long dps);
template <class T> void set_identity_clusters(Ctx& c, int P, int m, int s, T* U, long ld, long ps);
template <class T> int batched_inverse(Ctx& c, int nb, int n, T* A, long stride);  // in place GJ, returns 0
template <class T> void assemble_level0(Ctx& c, const Geometry& geo, const double* kappa, const double* vel,
                                        double shift, const int* d_perm, const int* d_iperm,
                                        const std::vector<const int*>& d_cutp,
                                        const std::vector<const int*>& d_cutq, HMat<T> D, HMat<T> E,
                                        HMat<T> F);
template <class T> void permute_in(Ctx& c, int n, int nrhs, const double* b, long ld, const int* d_perm,
                                   T* F);
template <class T> void permute_out(Ctx& c, int n, int nrhs, const T* F, const int* d_perm, double* x,
                                    long ld, int accumulate);
void stencil_apply(Ctx& c, int n, int nrhs, const double* coef, const double* x, long ld, const double* y,
                   double* out, double alpha, double beta, double* norms_out /*2*nrhs or null*/, bool trans = false);
template <class T> void expand_leaves(Ctx& c, int m, int b, const T* leaf, T* dense);
void exp_inplace(Ctx& c, double* p, long n);
// Sets *flag (device int) if an entry of p is NaN / infinite (or, with positive, not > 0).
void flag_invalid(Ctx& c, const double* p, long n, bool positive, int* flag);
void stencil_norms_scratch(cudaStream_t st, int n, int nrhs, const double* coef, const double* x, long ld,
                           const double* y, double* out, double* part, int nb_max, double* pairs);
void grad_logkappa(Ctx& c, int n, int nrhs, const double* kap, const double* u, const double* lam, long ld,
                   double* grad, int accumulate);
void face_coefficients(Ctx& c, int n, const double* kappa, const double* vel, double shift, double* coef);
void col_dots(Ctx& c, long N, int nrhs, const double* x, long ldx, const double* y, long ldy, double* out);
void col_axpy(Ctx& c, long N, int nrhs, const double* a /*device nrhs*/, const double* x, long ldx,
              double* y, long ldy);
void col_scale_copy(Ctx& c, long N, int nrhs, const double* a, const double* x, long ldx, double* y,
                    long ldy);

// ---- dense coarsest plane (coarse.cu) ---------------------------------------
void dense_inverse_fp64(Ctx& c, int m, double* A, double* Xinv);
template <class S, class D> void convert(Ctx& c, long n, const S* a, D* b);

// ---- cluster pivoted QR (qrcp_cluster.cu) -----------------------------------
// Truncation of NB matrices C_bi (valid kk[bi] x kk[NB + bi], row major, ld r)
// by a column-pivoted QR held in the distributed shared memory of a cluster
// of up to 8 CTAs: C ~ X diag(sig) Y^T, ranks in rank (the form of the one-CTA
// kernel).  frob: stop criterion on the remaining columns' Frobenius norm;
// floor2 (per block, or null): squared column norm that is never chosen.
// Returns false (nothing launched) when the matrices do not fit.
template <class T>
bool qrcp_cluster(Ctx& c, int r, const T* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol, int frob,
                  const T* floor2, T* X, T* Y, T* sig, int* rank, const char* site);

// The same truncation (FP32, blocks up to 512 x 512, column stop criterion)
// with up to 16 pivots chosen per round of cluster barriers from a sketch of
// the trailing matrix (qrcp_blocked.cu).  Returns false when it does not apply.
bool qrcp_blocked(Ctx& c, int r, const float* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol,
                  const float* floor2, float* X, float* Y, float* sig, int* rank, const char* site);

// ---- recompression (recompress.cu) ----------------------------------------
// Level-l recompression of the off-diagonal blocks  Left|c * Right|c^1 ^T  for
// every level-(l+1) cluster c of P planes.  Left/Right are [P][m][r] row
// major (ld r) and are consumed (freed or adopted).  Output panels have
// capacity *Kout.  tol < 0 (or exact) keeps blocks exact.
template <class T>
void recompress_level(Ctx& c, int P, int m, int lvl, DBuf<T>&& Left, DBuf<T>&& Right, int r, double tol,
                      bool exact, DBuf<T>& Uout, DBuf<T>& Vout, int& Kout);

}  // namespace acr
