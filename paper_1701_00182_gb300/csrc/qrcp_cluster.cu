// Rank-revealing QR with column pivoting (Householder, columns chosen by the
// largest remaining norm) of matrices too large for one CTA's shared memory,
// on a thread-block cluster.  This is the truncation of the recompression
// (Section 2.1: every low-rank block kept to a relative accuracy) for the
// large cores of the top HODLR levels and for the 256/512-row blocks that are
// truncated in explicit form.
//
// The kL x kR matrix is split by columns over the NC CTAs of a cluster (NC <=
// 8), each holding its columns in shared memory, so the whole factorisation
// runs out of on-chip memory.  Step st: warp 0 of every CTA publishes its best
// remaining column (largest norm), the sum of its remaining squared norms and
// that column's Householder vector; after one cluster barrier every CTA
// reduces the NC publications in the same order, so all take the same pivot p
// and the same stop decision, and copies p's vector over distributed shared
// memory; the owner of p keeps R's column in place; every CTA applies the
// reflector to its own remaining columns and downdates their norms.
// Columns are never moved: R stays in original column order.  The output has
// the form of the one-CTA kernel: C ~ X diag(sig) Y^T, X = Q_k (kL x k),
// sig_t = |R_tt|, Y[j][t] = R[t][j] / sig_t.  Q_k is formed afterwards from
// the reflectors (kept in global memory), its columns split over the CTAs.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "acr_internal.h"

namespace cg = cooperative_groups;

namespace acr {

namespace {

constexpr int kQT = 512;  // threads per CTA

template <class T>
__device__ __forceinline__ T wred_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
struct Pub {
  T best, sum, tau, beta;
  int idx;
};

}  // namespace

// Shared memory per CTA: W (ldw x cw, column major: the local columns, later
// Q's local columns), vloc (r), vpub (2 r), taus (r), nrm and nrm0 (cw),
// chosen step tj (cw ints).
//
// One cluster barrier per step: before it, warp 0 of every CTA picks its best
// remaining local column and publishes, besides its norm, that column's
// Householder vector (computed speculatively, W untouched); after it every
// CTA takes the same winner and copies the winner's vector.  The publications
// alternate between two buffers, so a CTA writing step st + 1's can never
// overwrite what another CTA still reads for step st (it would first have to
// pass step st + 1's barrier, which needs every CTA).
template <class T>
__global__ void __launch_bounds__(kQT)
    k_qrcp_cl(int r, const T* __restrict__ Call, const int* __restrict__ kk, long NB, int cw, int ldw,
              T* __restrict__ Vref, T* __restrict__ Xall, T* __restrict__ Yall, T* __restrict__ sigall,
              int* __restrict__ rankall, T tol, int frob, const T* __restrict__ floor2) {
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  extern __shared__ unsigned char smraw[];
  T* W = reinterpret_cast<T*>(smraw);
  T* vloc = W + (long)ldw * cw;
  T* vpub = vloc + r;
  T* taus = vpub + 2L * r;
  T* nrm = taus + r;
  T* nrm0 = nrm + cw;
  int* tj = reinterpret_cast<int*>(nrm0 + cw);
  __shared__ Pub<T> pub[2];
  __shared__ T s_thr2, s_tau, s_beta;
  __shared__ int s_p, s_stop;
  const long bi = blockIdx.x / NC;
  const T* C = Call + bi * (long)r * r;
  T* Vb = Vref + bi * (long)r * r;
  const int kL = kk[bi], kR = kk[NB + bi];
  const int kmax = min(kL, kR);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int c0 = q * cw;
  const int ncl = max(0, min(kR, c0 + cw) - c0);
  T* sig = sigall + bi * r;
  if (kmax == 0) {  // uniform over the cluster
    if (q == 0) {
      if (tid == 0) rankall[bi] = 0;
      for (int i = tid; i < r; i += blockDim.x) sig[i] = T(0);
    }
    return;
  }
  for (long e = tid; e < (long)ncl * kL; e += blockDim.x) {
    const int jl = (int)(e % ncl), i = (int)(e / ncl);
    W[(long)jl * ldw + i] = C[(long)i * r + c0 + jl];
  }
  __syncthreads();
  for (int jl = warp; jl < ncl; jl += nw) {
    T a = 0;
    for (int i = lane; i < kL; i += 32) a += W[(long)jl * ldw + i] * W[(long)jl * ldw + i];
    a = wred_sum(a);
    if (lane == 0) { nrm[jl] = a; nrm0[jl] = a; tj[jl] = -1; }
  }
  __syncthreads();
  int rank = 0;
  for (int st = 0; st < kmax; ++st) {
    const int buf = st & 1;
    if (warp == 0) {
      // best remaining local column, remaining squared norms
      T best = T(-1), sum = T(0);
      int bidx = 0x7fffffff;
      for (int jl = lane; jl < ncl; jl += 32) {
        if (tj[jl] >= 0) continue;
        const T nv = nrm[jl];
        sum += fmax(nv, T(0));
        if (nv > best) { best = nv; bidx = c0 + jl; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
      }
      // its Householder vector, rows st..kL-1 (speculative: W is not changed)
      T tau = T(0), beta = T(0);
      if (bidx != 0x7fffffff) {
        const T* col = W + (long)(bidx - c0) * ldw;
        T xn2 = T(0);
        for (int i = st + 1 + lane; i < kL; i += 32) xn2 += col[i] * col[i];
        xn2 = wred_sum(xn2);
        const T x0 = col[st];
        beta = x0;
        T scal = T(0);
        if (xn2 > T(0)) {
          beta = -copysign(sqrt(x0 * x0 + xn2), x0);
          tau = (beta - x0) / beta;
          scal = T(1) / (x0 - beta);
        }
        T* vp = vpub + (long)buf * r;
        for (int i = st + 1 + lane; i < kL; i += 32) vp[i] = col[i] * scal;
        if (lane == 0) vp[st] = T(1);
      }
      if (lane == 0) {
        pub[buf].best = best;
        pub[buf].idx = bidx;
        pub[buf].sum = sum;
        pub[buf].tau = tau;
        pub[buf].beta = beta;
      }
    }
    cluster.sync();
    if (warp == 0) {
      // the same reduction over the NC publications in every CTA
      T b = T(-1), sm = T(0), tw = T(0), bw = T(0);
      int bb = 0x7fffffff;
      if (lane < NC) {
        const Pub<T>* o = cluster.map_shared_rank(&pub[buf], lane);
        b = o->best;
        bb = o->idx;
        sm = o->sum;
        tw = o->tau;
        bw = o->beta;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, b, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bb, o);
        const T ot = __shfl_xor_sync(0xffffffffu, tw, o);
        const T obw = __shfl_xor_sync(0xffffffffu, bw, o);
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
        if (ov > b || (ov == b && oi < bb)) { b = ov; bb = oi; tw = ot; bw = obw; }
      }
      if (lane == 0) {
        if (st == 0) s_thr2 = tol * tol * b;
        s_p = bb;
        s_tau = tw;
        s_beta = bw;
        s_stop = !((frob ? sm : b) > s_thr2) || !(b > (floor2 ? floor2[bi] : T(0)));
      }
    }
    __syncthreads();
    if (s_stop) break;  // identical in every CTA of the cluster
    const int p = s_p;
    const int owner = p / cw, pl = p - owner * cw;
    const T tau = s_tau;
    {
      const T* vsrc = (q == owner) ? vpub + (long)buf * r : cluster.map_shared_rank(vpub + (long)buf * r, owner);
      for (int i = st + tid; i < kL; i += blockDim.x) vloc[i] = vsrc[i];
    }
    if (tid == 0) taus[st] = tau;
    if (q == owner) {
      // R's column p keeps rows 0..st; the reflector is kept for forming Q
      T* col = W + (long)pl * ldw;
      for (int i = st + 1 + tid; i < kL; i += blockDim.x) {
        Vb[(long)st * r + i] = vpub[(long)buf * r + i];
        col[i] = T(0);
      }
      if (tid == 0) {
        Vb[(long)st * r + st] = T(1);
        col[st] = s_beta;
        sig[st] = fabs(s_beta);
        tj[pl] = st;
      }
    }
    __syncthreads();
    // apply H = I - tau v v^T to the remaining local columns; row st becomes
    // R's row st.  A warp's columns go in groups of four so that their dot
    // products, reductions and updates overlap; the same warp then downdates
    // their norms.
    for (int jb = warp * 4; jb < ncl; jb += nw * 4) {
      T w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) w[u] = T(0);
      if (tau != T(0)) {
        for (int i = st + lane; i < kL; i += 32) {
          const T vi = vloc[i];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (jb + u < ncl) w[u] += vi * W[(long)(jb + u) * ldw + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = (jb + u < ncl && tj[jb + u] < 0) ? w[u] * tau : T(0);
        for (int i = st + lane; i < kL; i += 32) {
          const T vi = vloc[i];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (w[u] != T(0)) W[(long)(jb + u) * ldw + i] -= w[u] * vi;
        }
        __syncwarp();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jl = jb + u;
        if (jl >= ncl || tj[jl] >= 0) continue;  // uniform over the warp
        const T* cj = W + (long)jl * ldw;
        T nn = nrm[jl] - cj[st] * cj[st];
        if (nn < T(0.05) * nrm0[jl]) {  // the downdate lost its digits: recompute
          T a = 0;
          for (int i = st + 1 + lane; i < kL; i += 32) a += cj[i] * cj[i];
          a = wred_sum(a);
          if (lane == 0) nrm0[jl] = a;
          nn = a;
        }
        if (lane == 0) nrm[jl] = nn;
      }
    }
    __syncthreads();
    rank = st + 1;
  }
  cluster.sync();  // reflectors and sig of every step visible to the whole cluster
  // Y[j][t] = R[t][j] / sig_t for the local columns (R upper triangular in pivot order)
  T* Y = Yall + bi * (long)r * r;
  for (long e = tid; e < (long)ncl * rank; e += blockDim.x) {
    const int jl = (int)(e / rank), t = (int)(e % rank);
    const T d = sig[t];
    const T val = (tj[jl] < 0 || t <= tj[jl]) ? W[(long)jl * ldw + t] : T(0);
    Y[(long)(c0 + jl) * r + t] = d > T(0) ? val / d : T(0);
  }
  __syncthreads();
  // Q_k = H_0 ... H_{k-1} [I; 0]: this CTA's columns, in the space W held
  const int ck = (rank + NC - 1) / NC;
  const int t0 = q * ck, nloc = max(0, min(rank, t0 + ck) - t0);
  T* Q = W;
  for (long e = tid; e < (long)nloc * kL; e += blockDim.x) {
    const int tl = (int)(e / kL), i = (int)(e % kL);
    Q[(long)tl * ldw + i] = (i == t0 + tl) ? T(1) : T(0);
  }
  __syncthreads();
  for (int tp = min(rank, t0 + nloc) - 1; tp >= 0; --tp) {
    for (int i = tp + tid; i < kL; i += blockDim.x) vloc[i] = Vb[(long)tp * r + i];
    __syncthreads();
    const T tau = taus[tp];
    for (int tl = warp; tl < nloc; tl += nw) {
      if (t0 + tl < tp || tau == T(0)) continue;
      T* cq = Q + (long)tl * ldw;
      T w = T(0);
      for (int i = tp + lane; i < kL; i += 32) w += vloc[i] * cq[i];
      w = wred_sum(w) * tau;
      for (int i = tp + lane; i < kL; i += 32) cq[i] -= w * vloc[i];
    }
    __syncthreads();
  }
  T* X = Xall + bi * (long)r * r;
  for (long e = tid; e < (long)r * nloc; e += blockDim.x) {
    const int i = (int)(e / nloc), tl = (int)(e % nloc);
    X[(long)i * r + t0 + tl] = i < kL ? Q[(long)tl * ldw + i] : T(0);
  }
  if (q == 0) {
    for (int i = rank + tid; i < r; i += blockDim.x) sig[i] = T(0);
    if (tid == 0) rankall[bi] = rank;
  }
}

// Register-resident variant (FP32, blocks of at most 512 x 512).  The
// factorisation is bound by the reflector application, a rank-1 update of
// every remaining column per pivot step: with the columns in shared memory it
// streams the whole local matrix through the shared-memory pipe twice per
// step.  Here warp w of CTA q holds CPW columns (q * 16 * CPW + w * CPW + u)
// in registers, lane l rows l + 32 t (t < RPL), so the dot products and the
// update are register FMAs plus one shuffle reduction, and only the
// reflector (RPL values per lane) is read from shared memory.  Every warp
// computes, from its registers, the Householder vector of its own best
// remaining column (speculatively); one cluster barrier publishes the
// 16 x NC candidates, warp 0 of every CTA reduces them in the same order (same
// pivot, same stop decision everywhere) and every CTA copies the winner's
// vector over distributed shared memory.  Candidates and entries alternate
// between two buffers by step parity, so a CTA writing step st + 1's can never
// overwrite what another CTA still reads for step st.  Q_k is then formed
// from the reflectors in the same register layout, the next reflector
// prefetched into the other half of a double buffer while one is applied.
template <int RPL, int CPW>
__global__ void __launch_bounds__(kQT, 1)
    k_qrcp_reg(int r, int ldv, const float* __restrict__ Call, const int* __restrict__ kk, long NB,
               float* __restrict__ Vref, float* __restrict__ Xall, float* __restrict__ Yall,
               float* __restrict__ sigall, int* __restrict__ rankall, float tol, int frob,
               const float* __restrict__ floor2) {
  constexpr int NW = kQT / 32;
  constexpr int CW = NW * CPW;
  constexpr unsigned FULL = 0xffffffffu;
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  extern __shared__ float4 smraw4[];
  float* cand = reinterpret_cast<float*>(smraw4);  // [2][NW][ldv] candidate reflectors
  float* vloc = cand + 2L * NW * ldv;               // [2][ldv] the chosen reflector
  float* taus = vloc + 2L * ldv;                    // [ldv]
  float* sigs = taus + ldv;                         // [ldv]
  __shared__ float e_best[2][NW], e_sum[2][NW], e_tau[2][NW], e_beta[2][NW];
  __shared__ int e_idx[2][NW];
  __shared__ float s_thr2, s_tau, s_beta;
  __shared__ int s_p, s_src, s_stop;
  const long bi = blockIdx.x / NC;
  const float* C = Call + bi * (long)r * r;
  float* Vb = Vref + bi * (long)r * r;
  const int kL = kk[bi], kR = kk[NB + bi];
  const int kmax = min(kL, kR);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = q * CW + warp * CPW;  // this warp's first column
  float* sig = sigall + bi * r;
  if (kmax == 0) {  // uniform over the cluster
    if (q == 0) {
      if (tid == 0) rankall[bi] = 0;
      for (int i = tid; i < r; i += blockDim.x) sig[i] = 0.f;
    }
    return;
  }
  float W[RPL][CPW];
#pragma unroll
  for (int t = 0; t < RPL; ++t)
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      const int row = lane + 32 * t, col = c0 + u;
      W[t][u] = (row < kL && col < kR) ? C[(long)row * r + col] : 0.f;
    }
  // per column (replicated over the lanes): squared remaining norm, its last
  // exact value, and the step it was chosen at (-1 remaining, -2 absent)
  float nrm[CPW], nrm0[CPW];
  int tj[CPW];
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    float a = 0.f;
#pragma unroll
    for (int t = 0; t < RPL; ++t) a += W[t][u] * W[t][u];
    a = wred_sum(a);
    nrm[u] = a;
    nrm0[u] = a;
    tj[u] = (c0 + u < kR) ? -1 : -2;
  }
  for (int i = tid; i < 2 * ldv; i += blockDim.x) vloc[i] = 0.f;
  const float fl2 = floor2 ? floor2[bi] : 0.f;
  __syncthreads();
  int rank = 0;
  for (int st = 0; st < kmax; ++st) {
    const int buf = st & 1;
    const int ts = st >> 5, ls = st & 31;
    {
      // the warp's best remaining column and its Householder vector (rows st..kL-1)
      float best = -1.f, sum = 0.f, tau = 0.f, beta = 0.f;
      int ub = -1;
#pragma unroll
      for (int u = 0; u < CPW; ++u)
        if (tj[u] == -1) {
          sum += fmaxf(nrm[u], 0.f);
          if (nrm[u] > best) { best = nrm[u]; ub = u; }
        }
      if (ub >= 0) {
        float col[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          float v = 0.f;
#pragma unroll
          for (int u = 0; u < CPW; ++u)
            if (u == ub) v = W[t][u];
          col[t] = v;
        }
        float x0l = 0.f, xn2 = 0.f;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int row = lane + 32 * t;
          if (t == ts) x0l = col[t];
          if (row > st) xn2 += col[t] * col[t];
        }
        const float x0 = __shfl_sync(FULL, x0l, ls);
        xn2 = wred_sum(xn2);
        beta = x0;
        float scal = 0.f;
        if (xn2 > 0.f) {
          beta = -copysignf(sqrtf(x0 * x0 + xn2), x0);
          tau = (beta - x0) / beta;
          scal = 1.f / (x0 - beta);
        }
        float* cv = cand + ((long)buf * NW + warp) * ldv;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int row = lane + 32 * t;
          if (row > st && row < kL) cv[row] = col[t] * scal;
        }
        if (lane == 0) cv[st] = 1.f;
      }
      if (lane == 0) {
        e_best[buf][warp] = best;
        e_sum[buf][warp] = sum;
        e_tau[buf][warp] = tau;
        e_beta[buf][warp] = beta;
        e_idx[buf][warp] = ub >= 0 ? c0 + ub : 0x7fffffff;
      }
    }
    cluster.sync();
    if (warp == 0) {
      // the same reduction over the NC x NW candidates in every CTA
      // all loads of a lane's (at most four) entries are issued before any is used
      float ob[4], os[4], ot[4], obt[4];
      int oi[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = lane + 32 * e;
        ob[e] = -1.f; os[e] = 0.f; ot[e] = 0.f; obt[e] = 0.f; oi[e] = 0x7fffffff;
        if (m < NC * NW) {
          const int cta = m / NW, wq = m - cta * NW;
          ob[e] = *cluster.map_shared_rank(&e_best[buf][wq], cta);
          oi[e] = *cluster.map_shared_rank(&e_idx[buf][wq], cta);
          os[e] = *cluster.map_shared_rank(&e_sum[buf][wq], cta);
          ot[e] = *cluster.map_shared_rank(&e_tau[buf][wq], cta);
          obt[e] = *cluster.map_shared_rank(&e_beta[buf][wq], cta);
        }
      }
      float b = -1.f, sm = 0.f, tw = 0.f, bw = 0.f;
      int bb = 0x7fffffff, src = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sm += os[e];
        if (ob[e] > b || (ob[e] == b && oi[e] < bb)) { b = ob[e]; bb = oi[e]; tw = ot[e]; bw = obt[e]; src = lane + 32 * e; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(FULL, b, o);
        const int oi = __shfl_xor_sync(FULL, bb, o);
        const float ot = __shfl_xor_sync(FULL, tw, o);
        const float obw = __shfl_xor_sync(FULL, bw, o);
        const int os = __shfl_xor_sync(FULL, src, o);
        sm += __shfl_xor_sync(FULL, sm, o);
        if (ov > b || (ov == b && oi < bb)) { b = ov; bb = oi; tw = ot; bw = obw; src = os; }
      }
      if (lane == 0) {
        if (st == 0) s_thr2 = tol * tol * b;
        s_p = bb;
        s_tau = tw;
        s_beta = bw;
        s_src = src;
        s_stop = !((frob ? sm : b) > s_thr2) || !(b > fl2);
      }
    }
    __syncthreads();
    if (s_stop) break;  // identical in every CTA of the cluster
    const int p = s_p;
    const float tau = s_tau;
    {
      const int scta = s_src / NW, swarp = s_src - scta * NW;
      const float* vs = cand + ((long)buf * NW + swarp) * ldv;
      const float* vsrc = (scta == q) ? vs : cluster.map_shared_rank(vs, scta);
      for (int i = st + tid; i < kL; i += blockDim.x) vloc[i] = vsrc[i];
    }
    if (tid == 0) {
      taus[st] = tau;
      sigs[st] = fabsf(s_beta);
    }
    if (p >= c0 && p < c0 + CPW) {
      // this warp owns p: its column becomes R's column (rows 0..st), its reflector is kept for Q
      const int up = p - c0;
#pragma unroll
      for (int u = 0; u < CPW; ++u)
        if (u == up) {
          tj[u] = st;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int row = lane + 32 * t;
            if (row == st) W[t][u] = s_beta;
            else if (row > st) W[t][u] = 0.f;
          }
        }
      const float* vs = cand + ((long)buf * NW + warp) * ldv;
      for (int i = st + lane; i < kL; i += 32) Vb[(long)st * r + i] = vs[i];
    }
    __syncthreads();
    // apply H = I - tau v v^T to the remaining columns; row st becomes R's row st
    if (tau != 0.f) {
      float vr[RPL];
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        vr[t] = (row >= st && row < kL) ? vloc[row] : 0.f;
      }
      float w[CPW];
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < RPL; ++t) a += vr[t] * W[t][u];
        w[u] = a;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < CPW; ++u) w[u] += __shfl_xor_sync(FULL, w[u], o);
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
        if (tj[u] != -1) continue;  // uniform over the warp
        const float f = w[u] * tau;
#pragma unroll
        for (int t = 0; t < RPL; ++t) W[t][u] -= f * vr[t];
      }
    }
    // downdate the remaining norms by R's row st; recompute one that lost its digits
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      if (tj[u] != -1) continue;
      float xl = 0.f;
#pragma unroll
      for (int t = 0; t < RPL; ++t)
        if (t == ts) xl = W[t][u];
      const float x = __shfl_sync(FULL, xl, ls);
      float nn = nrm[u] - x * x;
      if (nn < 0.05f * nrm0[u]) {
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < RPL; ++t)
          if (lane + 32 * t > st) a += W[t][u] * W[t][u];
        a = wred_sum(a);
        nrm0[u] = a;
        nn = a;
      }
      nrm[u] = nn;
    }
    rank = st + 1;
  }
  cluster.sync();  // every step's reflector rows are in Vb and visible cluster-wide
  // Y[j][t] = R[t][j] / sig_t for this warp's columns
  float* Y = Yall + bi * (long)r * r;
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    if (tj[u] == -2) continue;
    const int j = c0 + u;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      if (row >= rank) continue;
      const float d = sigs[row];
      const float val = (tj[u] < 0 || row <= tj[u]) ? W[t][u] : 0.f;
      Y[(long)j * r + row] = d > 0.f ? val / d : 0.f;
    }
  }
  // Q_k = H_0 ... H_{k-1} [I; 0]: CTA q forms columns t0 .. t0 + nloc - 1, local column
  // tl in warp tl % NW, slot tl / NW (nloc <= CW since rank <= NC * CW)
  const int ck = (rank + NC - 1) / NC;
  const int t0 = q * ck, nloc = max(0, min(rank, t0 + ck) - t0);
#pragma unroll
  for (int t = 0; t < RPL; ++t)
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      const int tl = warp + NW * u;
      W[t][u] = (tl < nloc && lane + 32 * t == t0 + tl) ? 1.f : 0.f;
    }
  int vb = 0;
  if (rank > 0)
    for (int i = tid; i < kL; i += blockDim.x) vloc[i] = i >= rank - 1 ? Vb[(long)(rank - 1) * r + i] : 0.f;
  __syncthreads();
  for (int tp = rank - 1; tp >= 0; --tp) {
    if (tp > 0) {
      float* nx = vloc + (long)(vb ^ 1) * ldv;
      for (int i = tid; i < kL; i += blockDim.x) nx[i] = i >= tp - 1 ? Vb[(long)(tp - 1) * r + i] : 0.f;
    }
    const float tau = taus[tp];
    if (tau != 0.f && tp < t0 + nloc) {
      const float* cv = vloc + (long)vb * ldv;
      float vr[RPL];
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        vr[t] = row < kL ? cv[row] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
        const int tl = warp + NW * u;
        if (tl >= nloc || t0 + tl < tp) continue;  // uniform over the warp
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < RPL; ++t) a += vr[t] * W[t][u];
        a = wred_sum(a) * tau;
#pragma unroll
        for (int t = 0; t < RPL; ++t) W[t][u] -= a * vr[t];
      }
    }
    __syncthreads();
    vb ^= 1;
  }
  float* X = Xall + bi * (long)r * r;
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int tl = warp + NW * u;
    if (tl >= nloc) continue;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      if (row < r) X[(long)row * r + t0 + tl] = row < kL ? W[t][u] : 0.f;
    }
    for (int row = 32 * RPL + lane; row < r; row += 32) X[(long)row * r + t0 + tl] = 0.f;
  }
  if (q == 0) {
    for (int i = tid; i < r; i += blockDim.x) sig[i] = i < rank ? sigs[i] : 0.f;
    if (tid == 0) rankall[bi] = rank;
  }
}

template <int RPL, int CPW>
static bool launch_qrcp_reg(Ctx& c, int r, const float* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol,
                            int frob, const float* floor2, float* X, float* Y, float* sig, int* rank,
                            const char* site) {
  constexpr int CW = (kQT / 32) * CPW;
  const int NC = (kmaxR + CW - 1) / CW;
  const int ldv = (kmaxL + 3) / 4 * 4;
  const size_t sm = (2 * (size_t)(kQT / 32) + 4) * ldv * sizeof(float);
  if (NC > 8 || kmaxL > 32 * RPL) return false;
  ACR_CUDA(cudaFuncSetAttribute(k_qrcp_reg<RPL, CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(NB * NC));
  cfg.blockDim = dim3(kQT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = c.st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_qrcp_reg<RPL, CPW>, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  DBuf<float> Vref(c, NB * (size_t)r * r);
  c.kbegin();
  ACR_CUDA(cudaLaunchKernelEx(&cfg, k_qrcp_reg<RPL, CPW>, r, ldv, C, kk, NB, Vref.p, X, Y, sig, rank, (float)tol,
                              frob, floor2));
  c.kend(KC_JACOBI, 0, (double)NB * sizeof(float) * 3.0 * kmaxL * kmaxR, site);
  return true;
}

template <class T>
bool qrcp_cluster(Ctx& c, int r, const T* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol, int frob,
                  const T* floor2, T* X, T* Y, T* sig, int* rank, const char* site) {
  if constexpr (sizeof(T) == 4) {
    if (c.qrcp_blocked && !frob && qrcp_blocked(c, r, C, kk, NB, kmaxL, kmaxR, tol, floor2, X, Y, sig, rank, site))
      return true;
    if (c.qrcp_reg && kmaxL <= 512 && kmaxR <= 512) {
      const bool ok = kmaxL <= 128   ? launch_qrcp_reg<4, 8>(c, r, C, kk, NB, kmaxL, kmaxR, tol, frob, floor2, X, Y, sig,
                                                             rank, site)
                      : kmaxL <= 256 ? launch_qrcp_reg<8, 8>(c, r, C, kk, NB, kmaxL, kmaxR, tol, frob, floor2, X, Y,
                                                             sig, rank, site)
                                     : launch_qrcp_reg<16, 4>(c, r, C, kk, NB, kmaxL, kmaxR, tol, frob, floor2, X, Y,
                                                              sig, rank, site);
      if (ok) return true;
    }
  }
  const size_t cap = 220 * 1024;
  const int ldw = kmaxL | 1;  // odd: the column-major stores of a row run over distinct banks
  // The smallest cluster (<= 8 CTAs) whose CTAs fit several to an SM (each
  // step is a chain of short dependent phases: resident clusters hide each
  // other's latency), else the smallest that fits at all.  (16-CTA clusters
  // measured slower: their barrier dominates.)
  int NC = 0, cw = 0;
  size_t sm = 0;
  auto bytes = [&](int w) {
    return ((size_t)ldw * w + 4 * (size_t)r + 2 * (size_t)w) * sizeof(T) + (size_t)w * sizeof(int);
  };
  for (size_t lim : {(size_t)75 * 1024, cap})
    for (int nc : {1, 2, 4, 8}) {
      const int w = (kmaxR + nc - 1) / nc;
      if (!NC && bytes(w) <= lim) { NC = nc; cw = w; sm = bytes(w); }
    }
  if (NC == 0) return false;
  ACR_CUDA(cudaFuncSetAttribute(k_qrcp_cl<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(NB * NC));
  cfg.blockDim = dim3(kQT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = c.st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_qrcp_cl<T>, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  DBuf<T> Vref(c, NB * (size_t)r * r);
  c.kbegin();
  ACR_CUDA(cudaLaunchKernelEx(&cfg, k_qrcp_cl<T>, r, C, kk, NB, cw, ldw, Vref.p, X, Y, sig, rank, T(tol), frob,
                              floor2));
  c.kend(KC_JACOBI, 0, (double)NB * sizeof(T) * 3.0 * kmaxL * kmaxR, site);
  return true;
}

template bool qrcp_cluster<float>(Ctx&, int, const float*, const int*, long, int, int, double, int, const float*,
                                  float*, float*, float*, int*, const char*);
template bool qrcp_cluster<double>(Ctx&, int, const double*, const int*, long, int, int, double, int, const double*,
                                   double*, double*, double*, int*, const char*);

}  // namespace acr
