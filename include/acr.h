/*
 * acr.h -- C ABI of the GB300 accelerated-cyclic-reduction (ACR) solver.
 *
 * Problem (Section 2.2.1, Eq. probSta, Eq. originalMatrix): the 7-point
 * finite-difference discretisation of  -div(kappa grad u) + shift*u = f  on
 * the unit cube with homogeneous Dirichlet conditions, n interior nodes per
 * axis (h = 1/(n+1)), N = n^3 unknowns.  Unknown (i,j,k), i,j,k in [0,n), is
 * stored at lexicographic index i + n*j + n*n*k; k is the plane axis along
 * which cyclic reduction runs, so A = tridiag(E_k, D_k, F_k) with n x n
 * blocks of size n^2.  kappa = exp(log_kappa) is attached to the nodes;
 * interior faces use the harmonic mean 2 k_p k_q / (k_p + k_q) / h^2 and a
 * boundary face of node p uses k_p / h^2.
 *
 * Method (Section 3, Algorithms 1-2, Eq. elim, Eq. all_backSubs): every plane
 * block is held as a hierarchical matrix with weak admissibility (HODLR) over
 * a 2D bisection cluster tree of the plane, with dense leaf blocks and
 * tolerance-truncated low-rank off-diagonal blocks.  Cyclic reduction
 * eliminates the even planes of each level with H-arithmetic (inverse,
 * products, sums, QR+SVD recompression), the last plane is inverted, and the
 * solve runs the forward reduction and the back-substitution sweeps.
 *
 * Memory and ownership.  Right-hand sides and solutions are FP64, column
 * major N x nrhs with leading dimension ld >= N, in caller-owned DEVICE
 * memory.  The handle owns every factor it allocates until acr_destroy.  All
 * work is enqueued on opts->cuda_stream (the legacy default stream if NULL);
 * calls return after the stream has finished the work unless stated
 * otherwise.  A handle is not thread safe.
 *
 * Errors.  Every int-returning call returns ACR_OK (0) or one of the
 * ACR_ERR_* codes below; acr_error_string gives a message.  No call traps the
 * GPU; a numerical breakdown inside a kernel (a zero leaf pivot) is recorded
 * in a device flag and reported as ACR_ERR_BREAKDOWN.  Every wait inside a
 * kernel (tensor-core MMA completion) is bounded in time; one that expires is
 * recorded in a device flag and reported by acr_factor as ACR_ERR_CUDA.
 */
#ifndef ACR_H_
#define ACR_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ACR_OK = 0,
  ACR_ERR_ARG = 1,           /* invalid argument (sizes, NULL, unsupported n/leaf) */
  ACR_ERR_OOM = 2,           /* a device allocation failed */
  ACR_ERR_BREAKDOWN = 3,     /* a leaf or coupling pivot was (numerically) zero */
  ACR_ERR_RANK_CAP = 4,      /* a block rank exceeded opts->max_rank */
  ACR_ERR_CUDA = 5,          /* a CUDA runtime call failed (no device, launch failure) */
  ACR_ERR_NOT_CONVERGED = 6  /* refinement / GMRES hit the iteration limit */
};

/* Working precision of the factorisation and of the inner solve sweeps. */
enum { ACR_FP64 = 0, ACR_FP32 = 1 };

typedef struct acr_handle_s* acr_handle;

typedef struct {
  int precision;          /* ACR_FP64 (default) or ACR_FP32 */
  double shift;           /* diagonal term: -omega^2 for Helmholtz, 0 otherwise */
  int max_rank;           /* 0 = unlimited; else a block rank above it fails with ACR_ERR_RANK_CAP */
  size_t mem_budget;      /* 0 = unlimited; else bytes the stored factors may hold: the CR levels are kept
                             while they fit; from the first level that does not, only a checkpoint of that
                             level's inputs is kept (nothing when it is level 0, which re-assembles from
                             kappa), and every solve call recomputes those levels and the coarsest plane,
                             uses them and frees them (see levels_stored, tail_recomputes) */
  int autotune;           /* 1 = time candidate GEMM tilings per shape class and keep the fastest */
  int nrhs_max;           /* solve workspace is sized for this many right-hand sides (default 64) */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = legacy default stream */
  int profile;            /* 1 = time every kernel launch with CUDA events (per-class totals in acr_stats) */
  int inverse_fp64;       /* ACR_FP32 only: 1 = leaf and Woodbury-coupling inverses computed in FP64 */
  int tensor_cores;       /* ACR_FP32 only: 1 = GEMM tiles and the fused HODLR expansion on the tcgen05
                             tensor cores with a 3xTF32 split (FP32-level accuracy; large products
                             through TMA-fed pre-split tiles) instead of FP32 FMA tiles */
  int core_svd;           /* truncation of the recompression core: 0 = default (rank-revealing QR with
                             column pivoting, both precisions), 1 = one-sided Jacobi SVD, 2 = pivoted QR */
  int coarse_dense_max;   /* coarsest plane factorised densely in FP64 when n^2 <= this (0 = default 4096,
                             negative = never; otherwise it is inverted as a HODLR matrix) */
  int graphs;             /* 1 = capture the solve sweeps once per (nrhs, transpose) as a CUDA graph and replay
                             it; with cuda_stream NULL the handle then runs on its own blocking stream */
  const double* velocity; /* NULL, or a convection velocity beta (3 planar arrays of n^3 doubles: beta_x, beta_y,
                             beta_z per node, host or device, copied at factor) adding beta . grad u by
                             first-order upwind differences (Section 5, Eq. codi: beta = alpha b(x)); the
                             operator is then non-symmetric and acr_solve_ir_transpose refines with A^T */
  int chol_passes;        /* ACR_FP32 recompression of blocks wider than 128 rows: passes of the pivoted
                             Cholesky (0 = default 1, at most 4).  One pass stops where the FP32 Gram matrix
                             stops resolving (column residuals ~3e-3 of the largest), so tol below that is
                             met only approximately; each further pass factors the Gram matrix of the
                             explicitly formed residual (2 passes reach the FP64 factorisation's ranks at
                             tol 1e-6).  FP32 rounding, not truncation, then bounds the preconditioner */
} acr_opts;

typedef struct {
  int n, leaf, levels_cr, levels_h;       /* grid size, leaf size, CR levels q, HODLR depth */
  int precision;
  double tol;
  int max_rank[16][16];                   /* [CR level r][HODLR level l], largest block rank of X_r; r = levels_cr-1... coarsest row q */
  int max_rank_d[16][16];                 /* same for the reduced diagonal blocks D^{(r)} */
  size_t factor_bytes;                    /* device bytes held by the stored factors */
  size_t peak_bytes;                      /* device high-water mark of the factorisation */
  double t_factor_ms;                     /* device time of the last acr_factor */
  double t_level_ms[16];                  /* per CR level */
  long long gemm_flops;                   /* algorithmic GEMM flops issued by the factorisation */
  long long kernel_launches;              /* kernels launched by the last call */
  /* Per kernel class, accumulated over the handle's life (times only with opts.profile = 1):
   * 0 batched GEMM (CUDA-core and mma.sync tilings), 1 split-K reduction, 2 Householder QR, 3 pivoted Cholesky, 4 core truncation (Jacobi SVD or pivoted QR),
   * 5 rebuild coefficients, 6 Gauss-Jordan inverse, 7 copies/fills, 8 assembly, 9 RHS permutation,
   * 10 FP64 stencil and column reductions, 11 FP32 GEMM tiles on the tcgen05 tensor cores (3xTF32),
   * 12 fused HODLR x panel expansion, 13 TF32 high/remainder split of GEMM operands into TMA tiles.
   * flops/bytes are algorithmic counts (each operand once). */
  double kc_ms[16];
  double kc_flops[16];
  double kc_bytes[16];
  long long kc_launches[16];
  int jacobi_sweeps_max;                  /* most Jacobi sweeps any core SVD of the factorisation needed */
  int graphs_captured;                    /* solve graphs captured so far */
  int coarse_dense;                       /* 1 if the coarsest plane has a dense FP64 inverse */
  int levels_stored;                      /* CR levels whose factors are kept (levels_cr without a memory budget) */
  long long tail_recomputes;              /* solve calls that recomputed the levels not kept */
} acr_stats;

/* Default options (FP64, shift 0, unlimited ranks and memory, autotune off, nrhs_max 64). */
void acr_default_opts(acr_opts* opts);

/*
 * acr_factor -- ACR elimination (Algorithm 1 with Eq. elim), Section 3.2.
 *   n          grid points per axis; a power of two, 2 <= n <= 1024.
 *   log_kappa  N = n^3 values g, kappa = exp(g), host or device memory (the
 *              pointer kind is detected), read during the call; NULL means
 *              kappa = 1 (constant-coefficient operator).
 *   tol        relative truncation tolerance of every low-rank block
 *              (Section 3.1): singular values <= tol * sigma_1 of the block
 *              are dropped.  tol = 0 keeps every block exact (no truncation).
 *   leaf       leaf size of the HODLR cluster tree; must divide n^2 into a
 *              power-of-two number of leaves, 4 <= leaf <= 128.
 *   opts       NULL for defaults.
 *   out        receives the handle (NULL on failure).
 */
int acr_factor(int n, const double* log_kappa, double tol, int leaf, const acr_opts* opts,
               acr_handle* out);

/*
 * acr_solve -- forward reduction, coarsest solve and back-substitution
 * (Algorithm 2, Eq. all_backSubs) with the stored factors: x = M^{-1} rhs,
 * M the ACR approximation of A.  rhs, x: device FP64, N x nrhs column major,
 * leading dimension ld >= N; x may alias rhs.  nrhs >= 1.
 */
int acr_solve(acr_handle h, const double* rhs, double* x, int nrhs, long ld);

/*
 * acr_solve_transpose -- x = M^{-T} rhs with the same factors, transposed
 * (derived from the block LDU form of Eq. schur_complement; the paper gives
 * no transpose solve).  Arguments as acr_solve.
 */
int acr_solve_transpose(acr_handle h, const double* rhs, double* x, int nrhs, long ld);

/*
 * acr_residual -- FP64 7-point residual r = b - A x (the relative residual
 * of Section 5).  b, x, r: device FP64, N x nrhs, leading dimension ld; r may
 * alias b.  rel_norms: host array of nrhs doubles receiving ||r||_2/||b||_2,
 * or NULL.
 */
int acr_residual(acr_handle h, const double* b, const double* x, double* r, int nrhs, long ld,
                 double* rel_norms);

/*
 * acr_residual_noalloc -- the same FP64 residual and relative norms as
 * acr_residual, for callers that may not allocate device memory while they
 * run (a memory budget reserved up front, or a loop that cannot absorb an
 * allocation's implicit synchronisation).  The paper has no counterpart; this
 * is a property of the library, not of the method.
 *   Arguments as acr_residual; rel_norms is a host array of nrhs doubles or NULL.
 *   nrhs must be 1..64: larger requests return ACR_ERR_ARG.
 * The call allocates nothing: its reduction scratch is a fixed ~1 MiB array
 * in device memory that every GPU using the library holds until the process
 * exits.  The first call on each device looks up that array's device address
 * (with that device current).  The call waits for the handle's stream (it
 * reads the norms back), so it must not be made while that stream is being
 * captured into a CUDA graph.  All calls share the array: calls that overlap
 * on the GPU (other streams, other threads) race and must be serialised by
 * the caller.  A failed launch returns ACR_ERR_CUDA.
 */
int acr_residual_noalloc(acr_handle h, const double* b, const double* x, double* r, int nrhs, long ld,
                         double* rel_norms);

/*
 * acr_solve_ir -- ACR as preconditioner inside FP64 iterative refinement
 * (Section 5: low-accuracy factorisation plus an iterative procedure):
 * x_0 = 0; repeat d = M^{-1}(b - A x); x += d until every column has
 * ||b - A x||/||b|| <= rtol or maxit corrections were applied.
 *   b, x     device FP64, N x nrhs, leading dimension ld (must not alias).
 *   iters    host int, receives the number of corrections (may be NULL).
 *   rel_res  host array of nrhs doubles, final relative residuals (may be NULL).
 * Returns ACR_ERR_NOT_CONVERGED if the tolerance was not met.
 */
int acr_solve_ir(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol, int maxit,
                 int* iters, double* rel_res);

/*
 * acr_solve_ir_transpose -- refinement with the transpose solve:
 * x_0 = 0; repeat x += M^{-T}(b - A^T x).  The FP64 residual applies the
 * transposed 7-point stencil: for the diffusion operator A^T = A, and with
 * opts.velocity set (non-symmetric upwind operator) it applies A^T, whose
 * row p holds the couplings of column p of A.  Arguments as acr_solve_ir.
 */
int acr_solve_ir_transpose(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol, int maxit,
                           int* iters, double* rel_res);

/*
 * acr_grad_logkappa -- adjoint coefficient gradient (the paper has no
 * adjoint; derived from the operator of Section 2.2.1):
 *   grad_p = - kappa_p sum_columns lambda^T (dA/dkappa_p) u
 * for the handle's kappa, i.e. dL/dlog(kappa_p) when lambda = A^{-T} dL/du.
 * u, lam: device FP64, N x nrhs, leading dimension ld; grad: device FP64,
 * N entries (overwritten; contributions of all columns are summed).
 */
int acr_grad_logkappa(acr_handle h, const double* u, const double* lam, double* grad, int nrhs, long ld);

/*
 * acr_solve_fgmres -- right-preconditioned flexible GMRES(restart) in FP64
 * with the ACR solve as preconditioner and modified Gram-Schmidt, run for
 * every column independently (all columns advance together).  For the
 * indefinite Helmholtz operator, where refinement alone need not converge.
 * Arguments as acr_solve_ir; maxit counts preconditioner applications.
 */
int acr_solve_fgmres(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol,
                     int restart, int maxit, int* iters, double* rel_res);

/*
 * acr_get_factor_block -- expand one stored factor block to a dense
 * n^2 x n^2 matrix in lexicographic in-plane order (i + n j), row major,
 * into HOST memory `dense` (n^4 doubles).  which: 0 = X (inverse of an
 * eliminated D), 1 = E, 2 = F (of that eliminated plane), 3 = G = E_j X_{j-1},
 * 4 = H = F_j X_{j+1} (of a kept plane), 5 = inverse of the coarsest block.
 * level: CR level r; index: position among the eliminated (0..n_r/2-1) or
 * kept (0..n_r/2-1) planes of that level.  For inspection and tests.
 */
int acr_get_factor_block(acr_handle h, int which, int level, int index, double* dense);

/* Statistics of the last factorisation / solve. */
int acr_get_stats(acr_handle h, acr_stats* s);

/* Release the handle and all device memory it owns.  NULL is ignored. */
void acr_destroy(acr_handle h);

/* Static message for a status code. */
const char* acr_error_string(int status);

/*
 * acr_plane_ordering -- host-only query of the 2D bisection cluster tree of
 * one plane (Section 3.1): perm (host, n^2 ints) receives the lexicographic
 * in-plane index of each permuted position; ncut (host, up to 32 ints)
 * receives, per HODLR level, the number of grid edges each bisection cuts
 * (the exact rank of the level's off-diagonal blocks of D).  Returns the
 * number of HODLR levels, or a negative status on bad arguments.  Needs no GPU.
 */
int acr_plane_ordering(int n, int leaf, int* perm, int* ncut);

/*
 * acr_plan_blocks -- host-only query of the block cluster tree of one plane
 * (Section 2.1: index set, cluster tree, block cluster tree, admissibility
 * condition).  Clusters are those of acr_plane_ordering; a cluster holds a
 * rectangle of grid nodes and its geometric region is their convex hull.
 * Standard admissibility (eta >= 0): a pair of clusters (t, s) of one level
 * is admissible -- one low-rank block -- when
 *     min(diam(t), diam(s)) <= eta * dist(t, s),
 * decided exactly in squared grid steps; otherwise it is split into the four
 * pairs of children, and pairs of leaves stay dense blocks.  eta < 0 selects
 * weak admissibility (the HODLR structure acr_factor uses: the two sibling
 * off-diagonal blocks of every node low rank, the diagonal leaves dense).
 *   blocks  (host) NULL, or room for `cap` blocks of four ints: level l, row
 *           cluster t, column cluster s (level-l clusters cover the permuted
 *           range [t m / 2^l, (t + 1) m / 2^l), m = n^2), and 1 = low rank,
 *           0 = dense; in depth-first order, row child before column child.
 *   nblocks (host) receives the number of blocks.
 * Returns ACR_OK; ACR_ERR_ARG for n or leaf invalid (as acr_plane_ordering),
 * eta not finite, nblocks NULL, or blocks non-NULL with cap below the count
 * (*nblocks is still set, nothing is written).  Needs no GPU.
 */
int acr_plan_blocks(int n, int leaf, double eta, int* blocks, long cap, long* nblocks);

#ifdef __cplusplus
}
#endif

#endif /* ACR_H_ */
