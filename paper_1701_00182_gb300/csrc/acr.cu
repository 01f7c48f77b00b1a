// Accelerated cyclic reduction on one GPU: factorisation (Algorithm 1 with the
// block updates of Eq. elim), solve (Algorithm 2, Eq. all_backSubs), the
// transpose solve, FP64 residual / refinement / FGMRES, and the C ABI.
//
// Plane bookkeeping.  At CR level r the planes present are the original
// planes 2^r (t+1) - 1, t = 0..n_r-1 ("positions"); even positions are
// eliminated, odd positions are kept (Eq. permuted_system, Eq. next_step).
// E of position 0 and F of the last position are zero matrices, so every
// product is uniform over the batch; the only ragged case, the kept plane
// without a right neighbour, is a batch one plane shorter whose missing
// plane contributes zeros.
//
// Stored per level r: X_e = D_e^{-1} (eliminated), E^{(r)}, F^{(r)} (all
// positions; the eliminated ones are used), G_j = E_j X_{j-1} and
// H_j = F_j X_{j+1} (kept).  Forward:  f_j -= G_j f_{j-1} + H_j f_{j+1};
// back:  u_e = X_e (f_e - E_e u_{e-1} - F_e u_{e+1}).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>

#include "../../include/acr.h"
#include "acr_internal.h"
#include "hodlr.cuh"

namespace acr {

void* Ctx::dalloc_bytes(size_t bytes) {
  if (bytes == 0) return nullptr;
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw AcrError(ACR_ERR_OOM, "device allocation failed");
  }
  live_bytes += bytes;
  peak_bytes = std::max(peak_bytes, live_bytes);
  live[(uintptr_t)p] = bytes;
  return p;
}

void Ctx::kbegin() {
  if (!profile) return;
  if (evfree.empty()) {
    cudaEvent_t e;
    ACR_CUDA(cudaEventCreate(&e));
    evfree.push_back(e);
  }
  evcur = evfree.back();
  evfree.pop_back();
  ACR_CUDA(cudaEventRecord(evcur, st));
}

void Ctx::kend(int cls, double flops, double bytes, const char* name) {
  ++launches;
  kc_launch[cls] += 1;
  kc_flops[cls] += flops;
  kc_bytes[cls] += bytes;
  if (!profile || !evcur) return;
  if (evfree.empty()) {
    cudaEvent_t e;
    ACR_CUDA(cudaEventCreate(&e));
    evfree.push_back(e);
  }
  cudaEvent_t b = evfree.back();
  evfree.pop_back();
  ACR_CUDA(cudaEventRecord(b, st));
  const bool g = cls == KC_GEMM || cls == KC_GEMM_TC || cls == KC_HEXPAND;
  const char* key = g ? tag : (site_detail ? name : nullptr);
  pend.push_back({evcur, b, cls, key});
  if (key) site[key].second += g ? flops : bytes;
  evcur = nullptr;
  if (pend.size() >= 8192) kflush();
}

void Ctx::kflush() {
  if (pend.empty()) return;
  ACR_CUDA(cudaStreamSynchronize(st));
  for (size_t i = 0; i < pend.size(); ++i) {
    auto& p = pend[i];
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      kc_ms[p.cls] += ms;
      if (p.tag) site[p.tag].first += ms;
    }
    // idle time of the stream between the previous launch and this one (host work, syncs)
    if (site_detail && i > 0 && cudaEventElapsedTime(&ms, pend[i - 1].b, p.a) == cudaSuccess)
      gap[p.tag ? std::string(p.tag) : "class " + std::to_string(p.cls)] += ms;
    evfree.push_back(p.a);
    evfree.push_back(p.b);
  }
  pend.clear();
}

void Ctx::check_range(const void* base, long lo, long hi, size_t es, const char* what) const {
  uintptr_t a = (uintptr_t)base + (intptr_t)lo * (intptr_t)es;
  uintptr_t b = (uintptr_t)base + (intptr_t)(hi + 1) * (intptr_t)es;
  auto it = live.upper_bound(a);
  if (it == live.begin()) throw AcrError(ACR_ERR_ARG, std::string("operand outside any allocation: ") + what);
  --it;
  if (a < it->first || b > it->first + it->second)
    throw AcrError(ACR_ERR_ARG, std::string("operand range exceeds its allocation: ") + what);
}

void Ctx::dfree(void* p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, st);
  live_bytes -= bytes;
  live.erase((uintptr_t)p);
}

template <class T>
DBuf<T>::DBuf(Ctx& ctx, size_t cnt, bool zero) : n(cnt), c(&ctx) {
  p = ctx.alloc<T>(cnt);
  if (zero && cnt) ACR_CUDA(cudaMemsetAsync(p, 0, cnt * sizeof(T), ctx.st));
}
template <class T>
void DBuf<T>::release() {
  if (p && c) c->free(p, n);
  p = nullptr;
  n = 0;
}
template struct DBuf<float>;
template struct DBuf<double>;
template struct DBuf<int>;

template <class T>
struct LevelF {
  HStore<T> X, E, F, G, H;
  int nr = 0, ne = 0;
};

template <class T>
struct FactorT {
  int q = 0;
  // Levels r0..q-1 and the coarsest plane are not kept (memory budget): they
  // are recomputed from the checkpoint of level r0's inputs (re-assembled from
  // kappa when r0 = 0) for every solve call, and freed after it.  -1: all kept.
  int r0 = -1;
  int tail_pins = 0;  // > 0 while a call holds the recomputed levels
  std::vector<LevelF<T>> lv;
  HStore<T> Xc;
  DBuf<double> Xdense;  // FP64 dense inverse of the coarsest plane (m <= coarse_dense_max)
  HStore<T> ckD, ckE, ckF;
  DBuf<T> Fint, tmp;
  int cap = 0;
  std::vector<std::pair<long, cudaGraphExec_t>> graphs;  // key nrhs*2 + transpose
  ~FactorT() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
  }
};

}  // namespace acr

using namespace acr;

struct acr_handle_s {
  Ctx ctx;
  int n = 0, leaf = 0, precision = ACR_FP64, nrhs_max = 64, max_rank = 0, coarse_dense_max = 4096;
  bool graphs = false;
  cudaStream_t own_stream = nullptr;
  double tol = 0, shift = 0;
  Geometry geo;
  DBuf<int> perm, iperm;
  std::vector<DBuf<int>> cutp, cutq;
  DBuf<double> kappa, coef, vel;
  long long tail_recomputes = 0;
  std::unique_ptr<FactorT<float>> f32;
  std::unique_ptr<FactorT<double>> f64;
  acr_stats stats{};
  ~acr_handle_s() {
    f32.reset();
    f64.reset();
    perm.release();
    iperm.release();
    cutp.clear();
    cutq.clear();
    kappa.release();
    coef.release();
    vel.release();
    if (ctx.st) cudaStreamSynchronize(ctx.st);
    const char* ps = std::getenv("ACR_PROFILE_SITES");
    if (ps && (ps[0] == '1' || ps[0] == '2') && !ctx.site.empty()) {
      ctx.kflush();
      for (auto& kv : ctx.site)
        std::fprintf(stderr, "acr gemm site %-14s %10.1f ms %10.3f TFLOP\n", kv.first.c_str(), kv.second.first,
                     kv.second.second / 1e12);
      for (auto& kv : ctx.gap)
        if (kv.second >= 1.0) std::fprintf(stderr, "acr idle before %-24s %10.1f ms\n", kv.first.c_str(), kv.second);
    }
    for (auto& p : ctx.pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    ctx.pend.clear();
    for (auto e : ctx.evfree) cudaEventDestroy(e);
    ctx.evfree.clear();
    if (ctx.d_flag) cudaFree(ctx.d_flag);
    ctx.d_flag = nullptr;
    if (ctx.d_jflops) cudaFree(ctx.d_jflops);
    ctx.d_jflops = nullptr;
    // The private stream goes last, and no call may name it afterwards.
    if (own_stream) {
      cudaStreamDestroy(own_stream);
      own_stream = nullptr;
      ctx.st = nullptr;
    }
  }
};

namespace {

thread_local std::string g_last_error;

template <class Fn>
int guard(Fn&& fn) {
  try {
    fn();
    return ACR_OK;
  } catch (const AcrError& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    return ACR_ERR_OOM;
  } catch (...) {
    return ACR_ERR_CUDA;
  }
}

void check_flag(acr_handle_s* h) {
  int fl[4] = {0, 0, 0, 0};
  ACR_CUDA(cudaMemcpyAsync(fl, h->ctx.d_flag, sizeof(fl), cudaMemcpyDeviceToHost, h->ctx.st));
  ACR_CUDA(cudaStreamSynchronize(h->ctx.st));
  h->stats.jacobi_sweeps_max = fl[1];
  if (fl[2]) {
    ACR_CUDA(cudaMemsetAsync(h->ctx.d_flag + 2, 0, sizeof(int), h->ctx.st));
    throw AcrError(ACR_ERR_CUDA, "a tensor-core GEMM gave up waiting for its MMAs (time limit)");
  }
  const int f = fl[0];
  if (f) {
    ACR_CUDA(cudaMemsetAsync(h->ctx.d_flag, 0, sizeof(int), h->ctx.st));
    throw AcrError(ACR_ERR_BREAKDOWN, "zero pivot in a leaf or coupling inverse");
  }
}

void max_into(int* dst, const int* src, int L) {
  for (int l = 0; l < L; ++l) dst[l] = std::max(dst[l], src[l]);
}

// Dense m x m image (row major, permuted order) of one HODLR matrix.
template <class T>
void expand_dense_device(Ctx& c, const HMat<T>& A1, T* d) {
  const int m = A1.m, b = A1.b, L = A1.L;
  ACR_CUDA(cudaMemsetAsync(d, 0, sizeof(T) * (size_t)m * m, c.st));
  expand_leaves<T>(c, m, b, A1.leaf, d);
  for (int l = 0; l < L; ++l) {
    const int K = A1.K[l];
    if (!K) continue;
    const int s = m >> (l + 1), nclus = 1 << (l + 1);
    c.tag = "expand";
    gemm<T>(c, s, s, K, 1, nclus, T(1), opm<T>(A1.U[l], K, 1, 0, (long)s * K),
            opm<T>(A1.V[l], 1, K, 0, (long)s * K, 1), T(0), opm<T>(d + s, m, 1, 0, (long)s * m + s, 0, 0, -2L * s));
  }
}

// Level-0 blocks of the operator (Eq. originalMatrix) in HODLR form.
template <class T>
void assemble_inputs(acr_handle_s* h, HStore<T>& D, HStore<T>& E, HStore<T>& F) {
  Ctx& c = h->ctx;
  const Geometry& g = h->geo;
  const int n = g.n, m = g.m, L = g.L, b = g.leaf;
  D = HStore<T>();
  E = HStore<T>();
  F = HStore<T>();
  D.leaf = DBuf<T>(c, (size_t)n * m * b);
  E.leaf = DBuf<T>(c, (size_t)n * m * b);
  F.leaf = DBuf<T>(c, (size_t)n * m * b);
  for (int l = 0; l < L; ++l) {
    D.U[l] = DBuf<T>(c, (size_t)n * m * g.ncut[l]);
    D.V[l] = DBuf<T>(c, (size_t)n * m * g.ncut[l]);
    D.h.K[l] = g.ncut[l];
  }
  hstore_finish(D, n, m, L, b);
  hstore_finish(E, n, m, L, b);
  hstore_finish(F, n, m, L, b);
  std::vector<const int*> cp, cq;
  for (int l = 0; l < L; ++l) {
    cp.push_back(h->cutp[l].p);
    cq.push_back(h->cutq[l].p);
  }
  assemble_level0<T>(c, g, h->kappa.p, h->vel.p, h->shift, h->perm.p, h->iperm.p, cp, cq, D.h, E.h, F.h);
}

// Device copy of a batch of HODLR matrices (the checkpoint of a level's inputs).
template <class T>
HStore<T> hstore_clone(Ctx& c, const HStore<T>& A) {
  HStore<T> B;
  B.h = A.h;
  const HMat<T>& a = A.h;
  if (a.P <= 0) return B;
  B.leaf = DBuf<T>(c, (size_t)a.P * a.m * a.b);
  copy2d<T>(c, 1, (long)a.P * a.m, a.b, T(1), a.leaf, a.b, 0, B.leaf.p, a.b, 0);
  for (int l = 0; l < a.L; ++l) {
    const int K = a.K[l];
    if (!K) continue;
    B.U[l] = DBuf<T>(c, (size_t)a.P * a.m * K);
    B.V[l] = DBuf<T>(c, (size_t)a.P * a.m * K);
    copy2d<T>(c, 1, (long)a.P * a.m, K, T(1), a.U[l], K, 0, B.U[l].p, K, 0);
    copy2d<T>(c, 1, (long)a.P * a.m, K, T(1), a.V[l], K, 0, B.V[l].p, K, 0);
  }
  hstore_finish(B, a.P, a.m, a.L, a.b);
  return B;
}

// One CR level (Eq. elim): the inverses of the eliminated planes, G and H of
// the kept planes, and the next level's D, E, F.  The level's E and F move
// into the stored factors.
template <class T>
void eliminate_level(acr_handle_s* h, int r, HStore<T>& D, HStore<T>& E, HStore<T>& F, LevelF<T>& lvf) {
  Ctx& c = h->ctx;
  const Geometry& g = h->geo;
  const int m = g.m, L = g.L, b = g.leaf;
  const double tol = h->tol;
  const bool exact = !(tol > 0);
  const int nr = D.h.P, ne = nr / 2;
  lvf.nr = nr;
  lvf.ne = ne;
  int rk[MAXL] = {};
  {
    WSum<T> ws = winverse<T>(c, D.h.sub(0, 2, ne));
    lvf.X = wsum_to_hodlr<T>(c, ws, tol, exact, rk);
    max_into(h->stats.max_rank[r], rk, L);
  }
  {
    Flat<T> fg;
    flat_init<T>(c, fg, ne, m, L, b);
    flat_add_product<T>(c, fg, E.h.sub(1, 2, ne), lvf.X.h, T(1));
    lvf.G = flat_finalize<T>(c, fg, tol, exact, nullptr);
  }
  if (ne > 1) {
    Flat<T> fh;
    flat_init<T>(c, fh, ne - 1, m, L, b);
    flat_add_product<T>(c, fh, F.h.sub(1, 2, ne - 1), lvf.X.h.sub(1, 1, ne - 1), T(1));
    lvf.H = flat_finalize<T>(c, fh, tol, exact, nullptr);
  }
  HStore<T> Dn, En, Fn;
  {
    Flat<T> fd;
    flat_init<T>(c, fd, ne, m, L, b);
    flat_add_hodlr<T>(c, fd, D.h.sub(1, 2, ne), T(1));
    flat_add_product<T>(c, fd, lvf.G.h, F.h.sub(0, 2, ne), T(-1));
    if (ne > 1) flat_add_product<T>(c, fd, lvf.H.h, E.h.sub(2, 2, ne - 1), T(-1));
    Dn = flat_finalize<T>(c, fd, tol, exact, rk);
    max_into(h->stats.max_rank_d[r + 1], rk, L);
  }
  {
    Flat<T> fe;
    flat_init<T>(c, fe, ne, m, L, b);
    flat_add_product<T>(c, fe, lvf.G.h, E.h.sub(0, 2, ne), T(-1));
    En = flat_finalize<T>(c, fe, tol, exact, nullptr);
  }
  {
    Flat<T> ff;
    flat_init<T>(c, ff, ne, m, L, b);
    if (ne > 1) flat_add_product<T>(c, ff, lvf.H.h, F.h.sub(2, 2, ne - 1), T(-1));
    Fn = flat_finalize<T>(c, ff, tol, exact, nullptr);
  }
  D = HStore<T>();
  lvf.E = std::move(E);
  lvf.F = std::move(F);
  D = std::move(Dn);
  E = std::move(En);
  F = std::move(Fn);
}

// Inverse of the coarsest plane (Eq. first_backSubs): dense FP64 when small
// enough, else the HODLR inverse in the working precision.
template <class T>
void coarsest(acr_handle_s* h, FactorT<T>& fac, HStore<T>& D, int r) {
  Ctx& c = h->ctx;
  const int m = h->geo.m, L = h->geo.L;
  const double tol = h->tol;
  const bool exact = !(tol > 0);
  if (m <= h->coarse_dense_max) {
    DBuf<T> dT(c, (size_t)m * m);
    expand_dense_device<T>(c, D.h, dT.p);
    DBuf<double> dD(c, (size_t)m * m);
    convert<T, double>(c, (long)m * m, dT.p, dD.p);
    dT.release();
    fac.Xdense = DBuf<double>(c, (size_t)m * m);
    dense_inverse_fp64(c, m, dD.p, fac.Xdense.p);
    h->stats.coarse_dense = 1;
  } else {
    int rk[MAXL] = {};
    WSum<T> ws = winverse<T>(c, D.h);
    fac.Xc = wsum_to_hodlr<T>(c, ws, tol, exact, rk);
    max_into(h->stats.max_rank[r], rk, L);
  }
}

template <class T>
long level_bytes(const LevelF<T>& l) {
  return l.X.h.bytes() + l.E.h.bytes() + l.F.h.bytes() + l.G.h.bytes() + l.H.h.bytes();
}

template <class T>
void factor_impl(acr_handle_s* h, FactorT<T>& fac) {
  Ctx& c = h->ctx;
  const Geometry& g = h->geo;
  const int n = g.n, m = g.m, L = g.L;
  HStore<T> D, E, F;
  assemble_inputs<T>(h, D, E, F);
  for (int l = 0; l < L; ++l) h->stats.max_rank_d[0][l] = g.ncut[l];
  cudaEvent_t e0, e1;
  ACR_CUDA(cudaEventCreate(&e0));
  ACR_CUDA(cudaEventCreate(&e1));
  // Memory budget: level r is kept when the store, its estimate (twice the
  // level's inputs) and a checkpoint of the next level's inputs (estimated as
  // the level's own inputs) fit.  From the first level that does not, only the
  // checkpoint of its inputs is kept, or nothing (the tail then starts at level
  // 0, re-assembled from kappa) when even that would not fit; those levels are
  // still computed here (ranks, breakdown checks) but not kept.  The store
  // never exceeds the budget.
  const long budget = (long)c.budget;
  long stored = 0;
  auto drop_from = [&](int r, HStore<T>& D, HStore<T>& E, HStore<T>& F) {
    const long inputs = D.h.bytes() + E.h.bytes() + F.h.bytes();
    if (r > 0 && stored + inputs <= budget) {
      fac.r0 = r;
      fac.ckD = hstore_clone<T>(c, D);
      fac.ckE = hstore_clone<T>(c, E);
      fac.ckF = hstore_clone<T>(c, F);
    } else {
      fac.r0 = 0;
      fac.lv.clear();
      stored = 0;
    }
  };
  int r = 0;
  while (D.h.P > 1) {
    if (budget && fac.r0 < 0 && stored + 3 * (D.h.bytes() + E.h.bytes() + F.h.bytes()) > budget)
      drop_from(r, D, E, F);
    ACR_CUDA(cudaEventRecord(e0, c.st));
    LevelF<T> lvf;
    eliminate_level<T>(h, r, D, E, F, lvf);
    if (fac.r0 < 0) {
      stored += level_bytes(lvf);
      fac.lv.push_back(std::move(lvf));
      if (budget && stored > budget) {  // the estimate was short: keep nothing
        fac.r0 = 0;
        fac.lv.clear();
        stored = 0;
      }
    }
    ACR_CUDA(cudaEventRecord(e1, c.st));
    ACR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    ACR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (r < 16) h->stats.t_level_ms[r] = ms;
    ++r;
  }
  fac.q = r;
  if (fac.r0 < 0 && budget) {
    const long m2 = (long)m * m;
    const long est = m <= h->coarse_dense_max ? 8 * m2 : 2 * D.h.bytes();
    if (stored + est > budget) drop_from(r, D, E, F);  // r0 = q: only the coarsest plane is recomputed
  }
  if (fac.r0 < 0) coarsest<T>(h, fac, D, r);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_flag(h);
  h->stats.levels_stored = fac.r0 < 0 ? fac.q : fac.r0;
  fac.cap = h->nrhs_max;
  fac.Fint = DBuf<T>(c, (size_t)n * m * fac.cap);
  fac.tmp = DBuf<T>(c, (size_t)std::max(1, n / 2) * m * fac.cap);
}

// Recompute the levels r0..q-1 and the coarsest plane from the checkpoint
// (held until tail_release).
template <class T>
void tail_acquire(acr_handle_s* h, FactorT<T>& fac) {
  if (fac.r0 < 0 || fac.tail_pins++ > 0) return;
  Ctx& c = h->ctx;
  try {
    HStore<T> D, E, F;
    if (fac.r0 == 0) {
      assemble_inputs<T>(h, D, E, F);
    } else {
      D = hstore_clone<T>(c, fac.ckD);
      E = hstore_clone<T>(c, fac.ckE);
      F = hstore_clone<T>(c, fac.ckF);
    }
    int r = fac.r0;
    while (D.h.P > 1) {
      LevelF<T> lvf;
      eliminate_level<T>(h, r, D, E, F, lvf);
      fac.lv.push_back(std::move(lvf));
      ++r;
    }
    coarsest<T>(h, fac, D, r);
    check_flag(h);
  } catch (...) {
    fac.lv.resize(fac.r0);
    fac.Xc = HStore<T>();
    fac.Xdense.release();
    fac.tail_pins = 0;
    throw;
  }
  h->tail_recomputes++;
}

template <class T>
void tail_release(FactorT<T>& fac) {
  if (fac.r0 < 0 || --fac.tail_pins > 0) return;
  fac.lv.resize(fac.r0);
  fac.Xc = HStore<T>();
  fac.Xdense.release();
}

template <class T>
long factor_bytes(const FactorT<T>& f) {
  long s = f.Xc.h.bytes() + (long)f.Xdense.n * 8 + f.ckD.h.bytes() + f.ckE.h.bytes() + f.ckF.h.bytes();
  for (auto& l : f.lv) s += l.X.h.bytes() + l.E.h.bytes() + l.F.h.bytes() + l.G.h.bytes() + l.H.h.bytes();
  return s;
}

// Coarsest plane: last <- X_c last (or X_c^T), through the HODLR inverse or
// the dense FP64 inverse.
template <class T>
void coarse_apply(Ctx& c, FactorT<T>& fac, Pan<T> last, Pan<T> tp, int m, int nrhs, bool trans) {
  if (fac.Xdense.p) {
    DBuf<double> f64(c, (size_t)m * nrhs), y64(c, (size_t)m * nrhs);
    convert<T, double>(c, (long)m * nrhs, last.p, f64.p);
    c.tag = "coarse";
    gemm<double>(c, m, nrhs, m, 1, 1, 1.0, opm<double>(fac.Xdense.p, trans ? 1 : m, trans ? m : 1, 0, 0),
                 opm<double>(f64.p, nrhs, 1, 0, 0), 0.0, opm<double>(y64.p, nrhs, 1, 0, 0));
    convert<double, T>(c, (long)m * nrhs, y64.p, last.p);
  } else {
    hmatvec<T>(c, fac.Xc.h, 0, trans, last, tp, nrhs, T(1), T(0));
    copy2d<T>(c, 1, m, nrhs, T(1), tp.p, nrhs, 0, last.p, nrhs, 0);
  }
}

// The forward-reduction / coarsest / back-substitution sweeps on the
// internal RHS buffer F (n planes of m x nrhs), M^{-1} or M^{-T}.
template <class T>
void sweeps(acr_handle_s* h, FactorT<T>& fac, T* Fint, T* tmp, int nrhs, bool trans) {
  Ctx& c = h->ctx;
  const int n = h->geo.n, m = h->geo.m, q = fac.q;
  const long pst = (long)m * nrhs;
  auto view = [&](int r, int pos0) {
    long step = 1L << r;
    return Pan<T>{Fint + (step * (pos0 + 1) - 1) * pst, nrhs, 2 * step * pst};
  };
  Pan<T> tp{tmp, nrhs, pst};
  Pan<T> last{Fint + (long)(n - 1) * pst, nrhs, 0};
  if (!trans) {
    for (int r = 0; r < q; ++r) {
      LevelF<T>& lv = fac.lv[r];
      hmatvec<T>(c, lv.G.h, 0, false, view(r, 0), view(r, 1), nrhs, T(-1), T(1));
      if (lv.ne > 1) hmatvec<T>(c, lv.H.h, 0, false, view(r, 2), view(r, 1), nrhs, T(-1), T(1));
    }
    coarse_apply<T>(c, fac, last, tp, m, nrhs, false);
    for (int r = q - 1; r >= 0; --r) {
      LevelF<T>& lv = fac.lv[r];
      const int ne = lv.ne;
      if (ne > 1) hmatvec<T>(c, lv.E.h.sub(2, 2, ne - 1), 0, false, view(r, 1), view(r, 2), nrhs, T(-1), T(1));
      hmatvec<T>(c, lv.F.h.sub(0, 2, ne), 0, false, view(r, 1), view(r, 0), nrhs, T(-1), T(1));
      hmatvec<T>(c, lv.X.h, 0, false, view(r, 0), tp, nrhs, T(1), T(0));
      Pan<T> v0 = view(r, 0);
      copy2d<T>(c, ne, m, nrhs, T(1), tmp, nrhs, pst, v0.p, nrhs, v0.ps);
    }
  } else {
    for (int r = 0; r < q; ++r) {
      LevelF<T>& lv = fac.lv[r];
      const int ne = lv.ne;
      hmatvec<T>(c, lv.X.h, 0, true, view(r, 0), tp, nrhs, T(1), T(0));
      Pan<T> v0 = view(r, 0);
      copy2d<T>(c, ne, m, nrhs, T(1), tmp, nrhs, pst, v0.p, nrhs, v0.ps);
      if (ne > 1) hmatvec<T>(c, lv.E.h.sub(2, 2, ne - 1), 0, true, view(r, 2), view(r, 1), nrhs, T(-1), T(1));
      hmatvec<T>(c, lv.F.h.sub(0, 2, ne), 0, true, view(r, 0), view(r, 1), nrhs, T(-1), T(1));
    }
    coarse_apply<T>(c, fac, last, tp, m, nrhs, true);
    for (int r = q - 1; r >= 0; --r) {
      LevelF<T>& lv = fac.lv[r];
      const int ne = lv.ne;
      hmatvec<T>(c, lv.G.h, 0, true, view(r, 1), view(r, 0), nrhs, T(-1), T(1));
      if (ne > 1) hmatvec<T>(c, lv.H.h, 0, true, view(r, 1), view(r, 2), nrhs, T(-1), T(1));
    }
  }
}

// x = M^{-1} rhs (or M^{-T}); accumulate adds into x.  With graphs enabled the
// sweeps for a given (nrhs, transpose) are captured once and replayed.
template <class T>
void solve_impl(acr_handle_s* h, FactorT<T>& fac, const double* rhs, double* x, int nrhs, long ld, bool trans,
                bool accumulate) {
  Ctx& c = h->ctx;
  const int n = h->geo.n, m = h->geo.m;
  DBuf<T> Fown, Town;
  T* Fint = fac.Fint.p;
  T* tmp = fac.tmp.p;
  const bool own = nrhs > fac.cap;
  if (own) {
    Fown = DBuf<T>(c, (size_t)n * m * nrhs);
    Town = DBuf<T>(c, (size_t)std::max(1, n / 2) * m * nrhs);
    Fint = Fown.p;
    tmp = Town.p;
  }
  permute_in<T>(c, n, nrhs, rhs, ld, h->perm.p, Fint);
  struct Pin {
    acr_handle_s* h;
    FactorT<T>& f;
    Pin(acr_handle_s* hh, FactorT<T>& ff) : h(hh), f(ff) { tail_acquire<T>(h, f); }
    ~Pin() { tail_release<T>(f); }
  } pin(h, fac);
  if (h->graphs && !own && c.st && fac.r0 < 0) {
    const long key = 2L * nrhs + (trans ? 1 : 0);
    cudaGraphExec_t ex = nullptr;
    for (auto& g : fac.graphs)
      if (g.first == key) ex = g.second;
    if (!ex) {
      const bool prof = c.profile, tune = c.autotune, chk = c.check_bounds, ver = c.verify_gemm;
      c.verify_gemm = false;  // no host synchronisation inside a capture
      c.profile = false;  // no event timing or host synchronisation inside a capture
      c.autotune = false;
      cudaGraph_t graph = nullptr;
      ACR_CUDA(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
      try {
        sweeps<T>(h, fac, Fint, tmp, nrhs, trans);
      } catch (...) {
        cudaStreamEndCapture(c.st, &graph);
        if (graph) cudaGraphDestroy(graph);
        c.profile = prof;
        c.autotune = tune;
        c.verify_gemm = ver;
        throw;
      }
      ACR_CUDA(cudaStreamEndCapture(c.st, &graph));
      c.profile = prof;
      c.autotune = tune;
      c.check_bounds = chk;
      c.verify_gemm = ver;
      cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
      cudaGraphDestroy(graph);
      ACR_CUDA(e);
      fac.graphs.push_back({key, ex});
      h->stats.graphs_captured++;
    }
    ACR_CUDA(cudaGraphLaunch(ex, c.st));
    c.launches += 1;
  } else {
    sweeps<T>(h, fac, Fint, tmp, nrhs, trans);
  }
  permute_out<T>(c, n, nrhs, Fint, h->perm.p, x, ld, accumulate ? 1 : 0);
}

void publish_profile(acr_handle_s* h) {
  h->ctx.kflush();
  if (h->ctx.d_jflops) {
    double jf = 0;
    if (cudaMemcpy(&jf, h->ctx.d_jflops, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess)
      h->ctx.kc_flops[KC_JACOBI] = jf;
  }
  for (int k = 0; k < KC_N; ++k) {
    h->stats.kc_ms[k] = h->ctx.kc_ms[k];
    h->stats.kc_flops[k] = h->ctx.kc_flops[k];
    h->stats.kc_bytes[k] = h->ctx.kc_bytes[k];
    h->stats.kc_launches[k] = h->ctx.kc_launch[k];
  }
}

// Holds the recomputed levels of a budgeted factorisation for one call.
struct TailPin {
  acr_handle_s* h;
  explicit TailPin(acr_handle_s* hh) : h(hh) {
    if (h->f64) tail_acquire<double>(h, *h->f64);
    else tail_acquire<float>(h, *h->f32);
  }
  ~TailPin() {
    if (h->f64) tail_release<double>(*h->f64);
    else tail_release<float>(*h->f32);
  }
};

void solve_any(acr_handle_s* h, const double* rhs, double* x, int nrhs, long ld, bool trans, bool acc) {
  if (h->f64) solve_impl<double>(h, *h->f64, rhs, x, nrhs, ld, trans, acc);
  else solve_impl<float>(h, *h->f32, rhs, x, nrhs, ld, trans, acc);
}

template <class T>
void expand_block(acr_handle_s* h, const HMat<T>& A1, double* dense_host) {
  Ctx& c = h->ctx;
  const int m = A1.m, b = A1.b, L = A1.L;
  DBuf<T> d(c, (size_t)m * m, true);
  expand_leaves<T>(c, m, b, A1.leaf, d.p);
  for (int l = 0; l < L; ++l) {
    const int K = A1.K[l];
    if (!K) continue;
    const int s = m >> (l + 1), nclus = 1 << (l + 1);
    gemm<T>(c, s, s, K, 1, nclus, T(1), opm<T>(A1.U[l], K, 1, 0, (long)s * K),
            opm<T>(A1.V[l], 1, K, 0, (long)s * K, 1), T(0), opm<T>(d.p + s, m, 1, 0, (long)s * m + s, 0, 0, -2L * s));
  }
  std::vector<T> hb((size_t)m * m);
  ACR_CUDA(cudaMemcpyAsync(hb.data(), d.p, hb.size() * sizeof(T), cudaMemcpyDeviceToHost, c.st));
  ACR_CUDA(cudaStreamSynchronize(c.st));
  const std::vector<int>& pm = h->geo.perm;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) dense_host[(size_t)pm[i] * m + pm[j]] = (double)hb[(size_t)i * m + j];
}

template <class T>
void get_block_impl(acr_handle_s* h, FactorT<T>& f, int which, int level, int index, double* dense) {
  if (which == 5) {
    if (f.Xdense.p) {
      const int m = h->geo.m;
      std::vector<double> hb((size_t)m * m);
      ACR_CUDA(cudaMemcpyAsync(hb.data(), f.Xdense.p, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, h->ctx.st));
      ACR_CUDA(cudaStreamSynchronize(h->ctx.st));
      const std::vector<int>& pm = h->geo.perm;
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) dense[(size_t)pm[i] * m + pm[j]] = hb[(size_t)i * m + j];
    } else {
      expand_block<T>(h, f.Xc.h.sub(0, 1, 1), dense);
    }
    return;
  }
  if (level < 0 || level >= (int)f.lv.size()) throw AcrError(ACR_ERR_ARG, "level out of range");
  LevelF<T>& lv = f.lv[level];
  const HMat<T>* A = nullptr;
  int pos = index;
  switch (which) {
    case 0: A = &lv.X.h; break;
    case 1: A = &lv.E.h; pos = 2 * index; break;
    case 2: A = &lv.F.h; pos = 2 * index; break;
    case 3: A = &lv.G.h; break;
    case 4: A = &lv.H.h; break;
    default: throw AcrError(ACR_ERR_ARG, "bad factor kind");
  }
  if (pos < 0 || pos >= A->P) throw AcrError(ACR_ERR_ARG, "index out of range");
  expand_block<T>(h, A->sub(pos, 1, 1), dense);
}

}  // namespace

int solve_ir_impl(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol, int maxit,
                         int* iters, double* rel_res, bool trans) {
  if (!h || !b || !x || nrhs < 1 || maxit < 1 || ld < (long)h->n * h->n * h->n || b == x) return ACR_ERR_ARG;
  bool conv = false;
  int it = 0;
  int st = guard([&] {
    Ctx& c = h->ctx;
    h->ctx.launches = 0;
    const long N = (long)h->n * h->n * h->n;
    DBuf<double> r(c, (size_t)ld * nrhs), nrm(c, 2 * (size_t)nrhs);
    TailPin pin(h);
    ACR_CUDA(cudaMemset2DAsync(x, ld * sizeof(double), 0, N * sizeof(double), nrhs, c.st));
    ACR_CUDA(cudaMemcpy2DAsync(r.p, ld * sizeof(double), b, ld * sizeof(double), N * sizeof(double), nrhs,
                               cudaMemcpyDeviceToDevice, c.st));
    std::vector<double> hn(2 * nrhs), rel(nrhs, 1.0);
    for (it = 1; it <= maxit; ++it) {
      solve_any(h, r.p, x, nrhs, ld, trans, true);
      stencil_apply(c, h->n, nrhs, h->coef.p, x, ld, b, r.p, -1.0, 1.0, nrm.p, trans);
      ACR_CUDA(cudaMemcpyAsync(hn.data(), nrm.p, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
      ACR_CUDA(cudaStreamSynchronize(c.st));
      bool all_ok = true, finite = true;
      for (int k = 0; k < nrhs; ++k) {
        rel[k] = hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : std::sqrt(hn[2 * k]);
        if (!(rel[k] <= rtol)) all_ok = false;  // NaN counts as not converged
        if (!std::isfinite(rel[k])) finite = false;
      }
      if (all_ok) { conv = true; break; }
      if (!finite) break;
    }
    if (it > maxit) it = maxit;
    if (rel_res) std::memcpy(rel_res, rel.data(), nrhs * sizeof(double));
    h->stats.kernel_launches = h->ctx.launches;
    publish_profile(h);
  });
  if (iters) *iters = it;
  if (st != ACR_OK) return st;
  return conv ? ACR_OK : ACR_ERR_NOT_CONVERGED;
}


namespace acr {
int handle_residual_view(acr_handle h, cudaStream_t* st, int* n, const double** coef) {
  if (!h || !h->coef.p) return ACR_ERR_ARG;
  *st = h->ctx.st;
  *n = h->n;
  *coef = h->coef.p;
  return ACR_OK;
}
}  // namespace acr

extern "C" {

void acr_default_opts(acr_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = ACR_FP64;
  o->nrhs_max = 64;
}

const char* acr_error_string(int s) {
  switch (s) {
    case ACR_OK: return "ok";
    case ACR_ERR_ARG: return "invalid argument";
    case ACR_ERR_OOM: return "out of device memory";
    case ACR_ERR_BREAKDOWN: return "numerical breakdown (zero pivot)";
    case ACR_ERR_RANK_CAP: return "block rank above the cap";
    case ACR_ERR_CUDA: return "CUDA runtime error";
    case ACR_ERR_NOT_CONVERGED: return "iteration limit reached before the tolerance";
    default: return "unknown status";
  }
}

int acr_plane_ordering(int n, int leaf, int* perm, int* ncut) {
  Geometry g;
  if (plan_geometry(n, leaf, g)) return -ACR_ERR_ARG;
  if (perm) std::memcpy(perm, g.perm.data(), g.perm.size() * sizeof(int));
  if (ncut)
    for (int l = 0; l < g.L && l < 32; ++l) ncut[l] = g.ncut[l];
  return g.L;
}

int acr_plan_blocks(int n, int leaf, double eta, int* blocks, long cap, long* nblocks) {
  if (!nblocks) return ACR_ERR_ARG;
  *nblocks = 0;
  std::vector<std::array<int, 4>> b;
  try {
    if (plan_blocks(n, leaf, eta, b)) return ACR_ERR_ARG;
  } catch (const std::bad_alloc&) {
    return ACR_ERR_OOM;
  }
  *nblocks = (long)b.size();
  if (blocks) {
    if (cap < (long)b.size()) return ACR_ERR_ARG;
    for (size_t i = 0; i < b.size(); ++i)
      for (int k = 0; k < 4; ++k) blocks[4 * i + k] = b[i][k];
  }
  return ACR_OK;
}

int acr_factor(int n, const double* log_kappa, double tol, int leaf, const acr_opts* opts, acr_handle* out) {
  if (!out) return ACR_ERR_ARG;
  *out = nullptr;
  acr_opts o;
  acr_default_opts(&o);
  if (opts) o = *opts;
  if (!(tol >= 0) || (o.precision != ACR_FP64 && o.precision != ACR_FP32)) return ACR_ERR_ARG;
  if (o.nrhs_max <= 0) o.nrhs_max = 64;
  auto h = std::make_unique<acr_handle_s>();
  if (plan_geometry(n, leaf, h->geo)) return ACR_ERR_ARG;
  int st = guard([&] {
    int dev = 0;
    ACR_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    Ctx& c = h->ctx;
    c.st = (cudaStream_t)o.cuda_stream;
    h->graphs = o.graphs != 0;
    if (h->graphs && !c.st) {
      // The legacy default stream cannot be captured: run on a private blocking
      // stream (it still orders with the legacy default stream).
      ACR_CUDA(cudaStreamCreate(&h->own_stream));
      c.st = h->own_stream;
    }
    c.budget = o.mem_budget;
    const char* cb = std::getenv("ACR_CHECK_BOUNDS");
    c.check_bounds = cb && cb[0] == '1';
    const char* qr = std::getenv("ACR_QRCP_REG");
    c.qrcp_reg = !(qr && qr[0] == '0');
    c.qrcp_reg_all = qr && qr[0] == '2';
    const char* qb = std::getenv("ACR_QRCP_BLOCKED");
    c.qrcp_blocked = qb && qb[0] == '1';
    const char* gv = std::getenv("ACR_GEMM_VERIFY");
    c.verify_gemm = gv && gv[0] == '1';
    const char* sd = std::getenv("ACR_PROFILE_SITES");
    c.site_detail = sd && sd[0] == '2';
    const char* fc = std::getenv("ACR_GEMM_CFG");
    c.force_cfg = fc ? std::atoi(fc) : -1;
    c.autotune = o.autotune != 0;
    c.profile = o.profile != 0;
    c.inverse_fp64 = o.inverse_fp64 != 0;
    c.tensor = o.tensor_cores != 0;
    c.core_svd = o.core_svd;
    c.chol_passes = o.chol_passes > 0 ? std::min(o.chol_passes, 4) : 1;
    ACR_CUDA(cudaMalloc(&c.d_flag, 4 * sizeof(int)));
    ACR_CUDA(cudaMemsetAsync(c.d_flag, 0, 4 * sizeof(int), c.st));
    ACR_CUDA(cudaMalloc(&c.d_jflops, sizeof(double)));
    ACR_CUDA(cudaMemsetAsync(c.d_jflops, 0, sizeof(double), c.st));
    h->n = n;
    h->leaf = leaf;
    h->tol = tol;
    h->shift = o.shift;
    h->precision = o.precision;
    h->nrhs_max = o.nrhs_max;
    h->max_rank = o.max_rank;
    h->coarse_dense_max = o.coarse_dense_max > 0 ? o.coarse_dense_max : (o.coarse_dense_max < 0 ? 0 : 4096);
    const Geometry& g = h->geo;
    const long N = (long)n * n * n;
    h->perm = DBuf<int>(c, g.m);
    h->iperm = DBuf<int>(c, g.m);
    std::vector<int> ip(g.m);
    for (int p = 0; p < g.m; ++p) ip[g.perm[p]] = p;
    ACR_CUDA(cudaMemcpyAsync(h->perm.p, g.perm.data(), g.m * sizeof(int), cudaMemcpyHostToDevice, c.st));
    ACR_CUDA(cudaMemcpyAsync(h->iperm.p, ip.data(), g.m * sizeof(int), cudaMemcpyHostToDevice, c.st));
    for (int l = 0; l < g.L; ++l) {
      h->cutp.emplace_back(c, g.cutp[l].size());
      h->cutq.emplace_back(c, g.cutq[l].size());
      ACR_CUDA(cudaMemcpyAsync(h->cutp[l].p, g.cutp[l].data(), g.cutp[l].size() * sizeof(int),
                               cudaMemcpyHostToDevice, c.st));
      ACR_CUDA(cudaMemcpyAsync(h->cutq[l].p, g.cutq[l].data(), g.cutq[l].size() * sizeof(int),
                               cudaMemcpyHostToDevice, c.st));
    }
    h->kappa = DBuf<double>(c, N);
    if (log_kappa) {
      cudaPointerAttributes at;
      cudaMemcpyKind kind = cudaMemcpyHostToDevice;
      if (cudaPointerGetAttributes(&at, log_kappa) == cudaSuccess && at.type == cudaMemoryTypeDevice)
        kind = cudaMemcpyDeviceToDevice;
      cudaGetLastError();
      ACR_CUDA(cudaMemcpyAsync(h->kappa.p, log_kappa, N * sizeof(double), kind, c.st));
      exp_inplace(c, h->kappa.p, N);
    } else {
      fill<double>(c, h->kappa.p, N, 1.0);
    }
    if (o.velocity) {
      h->vel = DBuf<double>(c, 3 * N);
      ACR_CUDA(cudaMemcpyAsync(h->vel.p, o.velocity, 3 * N * sizeof(double), cudaMemcpyDefault, c.st));
    }
    // Inputs the operator cannot be built from (kappa = exp(log_kappa) not a
    // positive finite number, a non-finite velocity or shift) are argument errors.
    if (!std::isfinite(o.shift)) throw AcrError(ACR_ERR_ARG, "shift is not finite");
    flag_invalid(c, h->kappa.p, N, true, c.d_flag + 3);
    if (h->vel.p) flag_invalid(c, h->vel.p, 3 * N, false, c.d_flag + 3);
    {
      int bad = 0;
      ACR_CUDA(cudaMemcpyAsync(&bad, c.d_flag + 3, sizeof(int), cudaMemcpyDeviceToHost, c.st));
      ACR_CUDA(cudaStreamSynchronize(c.st));
      if (bad) throw AcrError(ACR_ERR_ARG, "log_kappa or velocity holds NaN / infinite values");
    }
    h->coef = DBuf<double>(c, 7 * N);
    face_coefficients(c, n, h->kappa.p, h->vel.p, o.shift, h->coef.p);
    std::memset(&h->stats, 0, sizeof(h->stats));
    h->stats.n = n;
    h->stats.leaf = leaf;
    h->stats.levels_h = g.L;
    h->stats.precision = o.precision;
    h->stats.tol = tol;
    c.launches = 0;
    c.gemm_flops = 0;
    cudaEvent_t e0, e1;
    ACR_CUDA(cudaEventCreate(&e0));
    ACR_CUDA(cudaEventCreate(&e1));
    ACR_CUDA(cudaEventRecord(e0, c.st));
    if (o.precision == ACR_FP64) {
      h->f64 = std::make_unique<FactorT<double>>();
      factor_impl<double>(h.get(), *h->f64);
    } else {
      h->f32 = std::make_unique<FactorT<float>>();
      factor_impl<float>(h.get(), *h->f32);
    }
    ACR_CUDA(cudaEventRecord(e1, c.st));
    ACR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    ACR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->stats.t_factor_ms = ms;
    h->stats.levels_cr = h->f64 ? h->f64->q : h->f32->q;
    h->stats.factor_bytes = h->f64 ? factor_bytes(*h->f64) : factor_bytes(*h->f32);
    h->stats.peak_bytes = c.peak_bytes;
    h->stats.gemm_flops = c.gemm_flops;
    h->stats.kernel_launches = c.launches;
    publish_profile(h.get());
    if (h->max_rank > 0)
      for (int r = 0; r < 16; ++r)
        for (int l = 0; l < 16; ++l)
          if (h->stats.max_rank[r][l] > h->max_rank || h->stats.max_rank_d[r][l] > h->max_rank)
            throw AcrError(ACR_ERR_RANK_CAP, "rank cap exceeded");
  });
  if (st != ACR_OK) return st;
  *out = h.release();
  return ACR_OK;
}

int acr_solve(acr_handle h, const double* rhs, double* x, int nrhs, long ld) {
  if (!h || !rhs || !x || nrhs < 1 || ld < (long)h->n * h->n * h->n) return ACR_ERR_ARG;
  return guard([&] {
    h->ctx.launches = 0;
    solve_any(h, rhs, x, nrhs, ld, false, false);
    h->stats.kernel_launches = h->ctx.launches;
    ACR_CUDA(cudaStreamSynchronize(h->ctx.st));
    publish_profile(h);
  });
}

int acr_solve_transpose(acr_handle h, const double* rhs, double* x, int nrhs, long ld) {
  if (!h || !rhs || !x || nrhs < 1 || ld < (long)h->n * h->n * h->n) return ACR_ERR_ARG;
  return guard([&] {
    h->ctx.launches = 0;
    solve_any(h, rhs, x, nrhs, ld, true, false);
    h->stats.kernel_launches = h->ctx.launches;
    ACR_CUDA(cudaStreamSynchronize(h->ctx.st));
    publish_profile(h);
  });
}

int acr_residual(acr_handle h, const double* b, const double* x, double* r, int nrhs, long ld, double* rel) {
  if (!h || !b || !x || !r || nrhs < 1 || ld < (long)h->n * h->n * h->n) return ACR_ERR_ARG;
  return guard([&] {
    Ctx& c = h->ctx;
    DBuf<double> nrm(c, 2 * (size_t)nrhs);
    stencil_apply(c, h->n, nrhs, h->coef.p, x, ld, b, r, -1.0, 1.0, nrm.p);
    std::vector<double> hn(2 * nrhs);
    ACR_CUDA(cudaMemcpyAsync(hn.data(), nrm.p, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    ACR_CUDA(cudaStreamSynchronize(c.st));
    if (rel)
      for (int k = 0; k < nrhs; ++k) rel[k] = hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : std::sqrt(hn[2 * k]);
  });
}

int acr_solve_ir(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol, int maxit, int* iters,
                 double* rel_res) {
  return solve_ir_impl(h, b, x, nrhs, ld, rtol, maxit, iters, rel_res, false);
}

int acr_solve_ir_transpose(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol, int maxit,
                           int* iters, double* rel_res) {
  return solve_ir_impl(h, b, x, nrhs, ld, rtol, maxit, iters, rel_res, true);
}

int acr_grad_logkappa(acr_handle h, const double* u, const double* lam, double* grad, int nrhs, long ld) {
  if (!h || !u || !lam || !grad || nrhs < 1 || ld < (long)h->n * h->n * h->n) return ACR_ERR_ARG;
  return guard([&] {
    grad_logkappa(h->ctx, h->n, nrhs, h->kappa.p, u, lam, ld, grad, 0);
    ACR_CUDA(cudaStreamSynchronize(h->ctx.st));
  });
}

int acr_solve_fgmres(acr_handle h, const double* b, double* x, int nrhs, long ld, double rtol, int restart, int maxit,
                     int* iters, double* rel_res) {
  if (!h || !b || !x || nrhs < 1 || maxit < 1 || restart < 1 || restart > 200 || b == x ||
      ld < (long)h->n * h->n * h->n)
    return ACR_ERR_ARG;
  bool conv = false;
  int total = 0;
  int st = guard([&] {
    Ctx& c = h->ctx;
    h->ctx.launches = 0;
    const long N = (long)h->n * h->n * h->n;
    const int mrs = restart;
    // Krylov basis V_0..V_m and preconditioned directions Z_0..Z_{m-1}, each N x nrhs (ld N).
    DBuf<double> Vb(c, (size_t)(mrs + 1) * N * nrhs), Zb(c, (size_t)mrs * N * nrhs), w(c, (size_t)N * nrhs);
    DBuf<double> nrm(c, 2 * (size_t)nrhs), dv(c, (size_t)nrhs), coefd(c, (size_t)nrhs);
    TailPin pin(h);
    auto Vk = [&](int k) { return Vb.p + (size_t)k * N * nrhs; };
    auto Zk = [&](int k) { return Zb.p + (size_t)k * N * nrhs; };
    ACR_CUDA(cudaMemset2DAsync(x, ld * sizeof(double), 0, N * sizeof(double), nrhs, c.st));
    std::vector<double> bn(nrhs, 0), hn(2 * nrhs), rel(nrhs, 1.0), tmpv(nrhs);
    while (total < maxit && !conv) {
      // r = b - A x into V0 (column stride N)
      DBuf<double> rl(c, (size_t)ld * nrhs);
      stencil_apply(c, h->n, nrhs, h->coef.p, x, ld, b, rl.p, -1.0, 1.0, nrm.p);
      ACR_CUDA(cudaMemcpy2DAsync(Vk(0), N * sizeof(double), rl.p, ld * sizeof(double), N * sizeof(double), nrhs,
                                 cudaMemcpyDeviceToDevice, c.st));
      ACR_CUDA(cudaMemcpyAsync(hn.data(), nrm.p, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
      ACR_CUDA(cudaStreamSynchronize(c.st));
      std::vector<double> beta(nrhs);
      double worst = 0;
      for (int k = 0; k < nrhs; ++k) {
        bn[k] = std::sqrt(hn[2 * k + 1]);
        beta[k] = std::sqrt(hn[2 * k]);
        rel[k] = bn[k] > 0 ? beta[k] / bn[k] : 0;
        worst = (rel[k] <= worst) ? worst : rel[k];  // NaN propagates
      }
      if (worst <= rtol) { conv = true; break; }
      if (!std::isfinite(worst)) break;
      for (int k = 0; k < nrhs; ++k) tmpv[k] = beta[k] > 0 ? 1.0 / beta[k] : 0.0;
      ACR_CUDA(cudaMemcpyAsync(dv.p, tmpv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c.st));
      col_scale_copy(c, N, nrhs, dv.p, Vk(0), N, Vk(0), N);
      // Hessenberg per column, Givens rotations
      std::vector<double> H((size_t)nrhs * (mrs + 1) * mrs, 0.0), cs((size_t)nrhs * mrs), sn((size_t)nrhs * mrs),
          gv((size_t)nrhs * (mrs + 1), 0.0);
      for (int k = 0; k < nrhs; ++k) gv[(size_t)k * (mrs + 1)] = beta[k];
      auto Hat = [&](int k, int i, int j) -> double& { return H[((size_t)k * (mrs + 1) + i) * mrs + j]; };
      int jdone = 0;
      for (int j = 0; j < mrs && total < maxit; ++j) {
        solve_any(h, Vk(j), Zk(j), nrhs, N, false, false);
        ++total;
        stencil_apply(c, h->n, nrhs, h->coef.p, Zk(j), N, nullptr, w.p, 1.0, 0.0, nullptr);
        for (int i = 0; i <= j; ++i) {
          col_dots(c, N, nrhs, w.p, N, Vk(i), N, dv.p);
          ACR_CUDA(cudaMemcpyAsync(tmpv.data(), dv.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, c.st));
          ACR_CUDA(cudaStreamSynchronize(c.st));
          for (int k = 0; k < nrhs; ++k) {
            Hat(k, i, j) = tmpv[k];
            tmpv[k] = -tmpv[k];
          }
          ACR_CUDA(cudaMemcpyAsync(coefd.p, tmpv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c.st));
          col_axpy(c, N, nrhs, coefd.p, Vk(i), N, w.p, N);
        }
        col_dots(c, N, nrhs, w.p, N, w.p, N, dv.p);
        ACR_CUDA(cudaMemcpyAsync(tmpv.data(), dv.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, c.st));
        ACR_CUDA(cudaStreamSynchronize(c.st));
        std::vector<double> inv(nrhs);
        worst = 0;
        for (int k = 0; k < nrhs; ++k) {
          double hn1 = std::sqrt(std::max(tmpv[k], 0.0));
          Hat(k, j + 1, j) = hn1;
          inv[k] = hn1 > 0 ? 1.0 / hn1 : 0.0;
          for (int i = 0; i < j; ++i) {
            double a = Hat(k, i, j), bb = Hat(k, i + 1, j);
            double cc = cs[(size_t)k * mrs + i], ss = sn[(size_t)k * mrs + i];
            Hat(k, i, j) = cc * a + ss * bb;
            Hat(k, i + 1, j) = -ss * a + cc * bb;
          }
          double a = Hat(k, j, j), bb = Hat(k, j + 1, j);
          double den = std::hypot(a, bb);
          double cc = den > 0 ? a / den : 1.0, ss = den > 0 ? bb / den : 0.0;
          cs[(size_t)k * mrs + j] = cc;
          sn[(size_t)k * mrs + j] = ss;
          Hat(k, j, j) = den;
          Hat(k, j + 1, j) = 0;
          double g0 = gv[(size_t)k * (mrs + 1) + j];
          gv[(size_t)k * (mrs + 1) + j] = cc * g0;
          gv[(size_t)k * (mrs + 1) + j + 1] = -ss * g0;
          rel[k] = bn[k] > 0 ? std::fabs(gv[(size_t)k * (mrs + 1) + j + 1]) / bn[k] : 0;
          worst = (rel[k] <= worst) ? worst : rel[k];
        }
        ACR_CUDA(cudaMemcpyAsync(dv.p, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c.st));
        col_scale_copy(c, N, nrhs, dv.p, w.p, N, Vk(j + 1), N);
        jdone = j + 1;
        if (worst <= rtol * 0.5) break;
      }
      // y = R^{-1} g per column, x += Z y
      std::vector<double> y((size_t)nrhs * mrs, 0.0);
      for (int k = 0; k < nrhs; ++k)
        for (int i = jdone - 1; i >= 0; --i) {
          double v = gv[(size_t)k * (mrs + 1) + i];
          for (int q = i + 1; q < jdone; ++q) v -= Hat(k, i, q) * y[(size_t)k * mrs + q];
          double d = Hat(k, i, i);
          y[(size_t)k * mrs + i] = d != 0 ? v / d : 0.0;
        }
      for (int i = 0; i < jdone; ++i) {
        for (int k = 0; k < nrhs; ++k) tmpv[k] = y[(size_t)k * mrs + i];
        ACR_CUDA(cudaMemcpyAsync(coefd.p, tmpv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c.st));
        col_axpy(c, N, nrhs, coefd.p, Zk(i), N, x, ld);
      }
    }
    if (!conv) {
      DBuf<double> rl(c, (size_t)ld * nrhs);
      stencil_apply(c, h->n, nrhs, h->coef.p, x, ld, b, rl.p, -1.0, 1.0, nrm.p);
      ACR_CUDA(cudaMemcpyAsync(hn.data(), nrm.p, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
      ACR_CUDA(cudaStreamSynchronize(c.st));
      double worst = 0;
      for (int k = 0; k < nrhs; ++k) {
        rel[k] = hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : 0.0;
        worst = (rel[k] <= worst) ? worst : rel[k];
      }
      conv = worst <= rtol;
    }
    if (rel_res) std::memcpy(rel_res, rel.data(), nrhs * sizeof(double));
    h->stats.kernel_launches = h->ctx.launches;
    publish_profile(h);
  });
  if (iters) *iters = total;
  if (st != ACR_OK) return st;
  return conv ? ACR_OK : ACR_ERR_NOT_CONVERGED;
}

int acr_get_factor_block(acr_handle h, int which, int level, int index, double* dense) {
  if (!h || !dense) return ACR_ERR_ARG;
  return guard([&] {
    TailPin pin(h);
    if (h->f64) get_block_impl<double>(h, *h->f64, which, level, index, dense);
    else get_block_impl<float>(h, *h->f32, which, level, index, dense);
  });
}

int acr_get_stats(acr_handle h, acr_stats* s) {
  if (!h || !s) return ACR_ERR_ARG;
  h->stats.tail_recomputes = h->tail_recomputes;
  *s = h->stats;
  return ACR_OK;
}

void acr_destroy(acr_handle h) { delete h; }

}  // extern "C"
