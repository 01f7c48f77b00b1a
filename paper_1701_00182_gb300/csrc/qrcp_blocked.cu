// Blocked-pivot variant of the register-resident cluster pivoted QR (FP32,
// blocks up to 512 x 512, column stop criterion): the truncation of the
// recompression (Section 2.1) with kBP pivots chosen per round of cluster
// barriers instead of one.
//
// Written from the sketch-pivoting scheme the pivot-selection study measured
// (b pivots from a pivoted QR of a random-sign sketch of the trailing matrix
// reach the one-pivot ranks within two on decaying and Schur-complement
// blocks).  Per block of at most kBP pivots:
//   1. every warp sketches its remaining columns, S = Omega A(st:, cols),
//      Omega kBL x (kL - st) with signs from a hash of (row, block, matrix);
//      cluster barrier; every CTA gathers the whole sketch;
//   2. every CTA runs the same pivoted Householder QR on the sketch: the same
//      npiv pivots everywhere;
//   3. the owners publish the pivot columns; cluster barrier; every CTA
//      gathers them and runs the same Householder QR of that panel (R11 and
//      the reflectors);
//   4. every warp applies the npiv reflectors to its other remaining columns
//      in registers, and, from the exact norm of their rows below the block
//      and their new rows inside it, the largest remaining norm after t
//      pivots for every t; cluster barrier; the first t at which it is at
//      most tol^2 x the largest initial norm (or the noise floor) ends the
//      factorisation at rank st + t, else all npiv pivots are kept.
// Pivots dropped at a stop stay ordinary columns: their rows of the kept
// reflectors come from R11.  Outputs as the other cluster kernels:
// C ~ X diag(sig) Y^T, X = Q_k, sig_t = |R_tt|, Y[j][t] = R[t][j] / sig_t.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "acr_internal.h"

namespace cg = cooperative_groups;

namespace acr {

namespace {

constexpr int kBT = 512;  // threads per CTA
constexpr int kBW = kBT / 32;
constexpr int kBP = 16;   // pivots per block
constexpr int kBL = 24;   // sketch rows (kBP + 8 of oversampling)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float bsum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// MurmurHash3's 32-bit finaliser (a bijective integer mixer): its low kBL bits
// give the sketch signs of one matrix row.
__device__ __forceinline__ unsigned fmix32(unsigned x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// Block-wide arg-max of (v, idx) with ties to the lower index; every thread
// gets the result.  rf / ri: kBW-entry scratch.
__device__ __forceinline__ void block_argmax(float& v, int& idx, float* rf, int* ri) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(kFull, v, o);
    const int oi = __shfl_xor_sync(kFull, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  __syncthreads();  // the scratch may still be read from a previous call
  if (lane == 0) { rf[warp] = v; ri[warp] = idx; }
  __syncthreads();
  v = lane < kBW ? rf[lane] : -1.f;
  idx = lane < kBW ? ri[lane] : 0x7fffffff;
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(kFull, v, o);
    const int oi = __shfl_xor_sync(kFull, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
}

__device__ __forceinline__ float block_sum(float v, float* rf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = bsum(v);
  __syncthreads();
  if (lane == 0) rf[warp] = v;
  __syncthreads();
  v = lane < kBW ? rf[lane] : 0.f;
  return bsum(v);
}

}  // namespace

template <int RPL, int CPW>
__global__ void __launch_bounds__(kBT, 1)
    k_qrcp_blk(int r, int ldv, const float* __restrict__ Call, const int* __restrict__ kk, long NB,
               float* __restrict__ Vref, float* __restrict__ Xall, float* __restrict__ Yall,
               float* __restrict__ sigall, int* __restrict__ rankall, float tol, const float* __restrict__ floor2) {
  constexpr int CW = kBW * CPW;  // columns per CTA
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int ncols = NC * CW;  // <= kBT (checked by the launcher)
  extern __shared__ float4 smraw4[];
  float* skl = reinterpret_cast<float*>(smraw4);  // [2][kBL][CW] this CTA's sketch columns
  float* ska = skl + 2 * kBL * CW;                 // [kBL][ncols] the gathered sketch
  float* pcl = ska + (long)kBL * ncols;            // [2][kBP][ldv] this CTA's pivot columns
  float* pan = pcl + 2L * kBP * ldv;               // [kBP][ldv] the gathered panel, then its reflectors
  float* taus = pan + (long)kBP * ldv;             // [ldv]
  float* sigs = taus + ldv;                        // [ldv]
  __shared__ float rf[kBW];
  __shared__ int ri[kBW];
  __shared__ float wmx[kBW][kBP + 1];
  __shared__ float stl[2][kBP + 1];  // this CTA's largest remaining norm after t pivots (published)
  __shared__ float R11[kBP][kBP];
  __shared__ float ptau[kBP], pbeta[kBP], svs[kBL];
  __shared__ int spiv[kBP];
  __shared__ float s_stau, s_scal, s_beta;
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
  int tj[CPW];  // step a column was chosen at; -1 remaining, -2 absent
  float wm = 0.f;
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int col = c0 + u;
    float a = 0.f;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      W[t][u] = (row < kL && col < kR) ? C[(long)row * r + col] : 0.f;
      a += W[t][u] * W[t][u];
    }
    a = bsum(a);
    tj[u] = col < kR ? -1 : -2;
    if (col < kR) wm = fmaxf(wm, a);
  }
  // the largest initial column norm over the cluster fixes the stop threshold
  if (lane == 0) rf[warp] = wm;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int w = 0; w < kBW; ++w) m = fmaxf(m, rf[w]);
    stl[1][0] = m;
  }
  cluster.sync();
  float gmax = 0.f;
  {
    float m = lane < NC ? *cluster.map_shared_rank(&stl[1][0], lane) : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    gmax = m;
  }
  const float thr = tol * tol * gmax;
  const float fl2 = floor2 ? floor2[bi] : 0.f;
  int st = 0;
  if ((gmax > thr) && (gmax > fl2)) {
    const unsigned seed = (unsigned)bi * 0x27d4eb2fu + 0x165667b1u;
    for (int blk = 0;; ++blk) {
      const int buf = blk & 1;
      // 1. sketch of this warp's remaining columns, rows st..kL-1
      {
        unsigned hs[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) hs[t] = fmix32((unsigned)(lane + 32 * t) * 0x9e3779b9u + (unsigned)blk * 0x85ebca77u + seed);
        for (int i = 0; i < kBL; ++i) {
          float s[CPW];
#pragma unroll
          for (int u = 0; u < CPW; ++u) s[u] = 0.f;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int row = lane + 32 * t;
            const bool in = row >= st && row < kL;
            const float sg = ((hs[t] >> i) & 1u) ? -1.f : 1.f;
#pragma unroll
            for (int u = 0; u < CPW; ++u) s[u] += in ? sg * W[t][u] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < CPW; ++u) {
            const float v = bsum(s[u]);
            if (lane == 0) skl[(buf * kBL + i) * CW + warp * CPW + u] = tj[u] == -1 ? v : 0.f;
          }
        }
      }
      cluster.sync();
      for (int e = tid; e < kBL * ncols; e += blockDim.x) {
        const int i = e / ncols, col = e - i * ncols, cta = col / CW, j = col - cta * CW;
        const float* src = skl + (buf * kBL + i) * CW + j;
        ska[e] = cta == q ? *src : *cluster.map_shared_rank(src, cta);
      }
      __syncthreads();
      // 2. the same pivoted Householder QR of the sketch in every CTA
      const int pmax = min(kBP, kL - st);
      int npiv = 0;
      for (int p = 0; p < pmax; ++p) {
        float cn = -1.f;
        int cidx = 0x7fffffff;
        if (tid < ncols) {
          cn = 0.f;
          for (int i = p; i < kBL; ++i) cn += ska[i * ncols + tid] * ska[i * ncols + tid];
          cidx = tid;
        }
        block_argmax(cn, cidx, rf, ri);
        if (!(cn > 0.f)) break;  // uniform: every thread holds the block's result
        if (warp == 0) {
          const float x = lane >= p && lane < kBL ? ska[lane * ncols + cidx] : 0.f;
          const float x0 = __shfl_sync(kFull, x, p);
          const float xn2 = bsum(lane > p ? x * x : 0.f);
          float beta = x0, tau = 0.f, scal = 0.f;
          if (xn2 > 0.f) {
            beta = -copysignf(sqrtf(x0 * x0 + xn2), x0);
            tau = (beta - x0) / beta;
            scal = 1.f / (x0 - beta);
          }
          if (lane < kBL) svs[lane] = lane < p ? 0.f : (lane == p ? 1.f : x * scal);
          if (lane == 0) {
            s_stau = tau;
            spiv[p] = cidx;
          }
        }
        __syncthreads();
        if (tid < ncols) {
          float w = 0.f;
          for (int i = p; i < kBL; ++i) w += svs[i] * ska[i * ncols + tid];
          w *= s_stau;
          for (int i = p; i < kBL; ++i) ska[i * ncols + tid] -= w * svs[i];
        }
        __syncthreads();
        npiv = p + 1;
      }
      if (npiv == 0) break;  // uniform over the cluster
      // 3. the owners publish the pivot columns (rows st..kL-1); every CTA gathers them
      for (int p = 0; p < npiv; ++p) {
        const int col = spiv[p];
        if (col >= c0 && col < c0 + CPW) {
#pragma unroll
          for (int u = 0; u < CPW; ++u)
            if (c0 + u == col) {
#pragma unroll
              for (int t = 0; t < RPL; ++t) {
                const int row = lane + 32 * t;
                if (row >= st && row < kL) pcl[((long)buf * kBP + p) * ldv + row] = W[t][u];
              }
            }
        }
      }
      cluster.sync();
      const int nr = kL - st;
      for (int e = tid; e < npiv * nr; e += blockDim.x) {
        const int p = e / nr, row = st + (e - p * nr), cta = spiv[p] / CW;
        const float* src = pcl + ((long)buf * kBP + p) * ldv + row;
        pan[(long)p * ldv + row] = cta == q ? *src : *cluster.map_shared_rank(src, cta);
      }
      __syncthreads();
      // the same Householder QR of the panel in every CTA: R11 and the reflectors (in pan)
      for (int p = 0; p < npiv; ++p) {
        const int row0 = st + p;
        float* cp = pan + (long)p * ldv;
        const int rr = row0 + 1 + tid;
        const float xv = rr < kL ? cp[rr] : 0.f;
        const float xn2 = block_sum(xv * xv, rf);
        if (tid == 0) {
          const float x0 = cp[row0];
          float beta = x0, tau = 0.f, scal = 0.f;
          if (xn2 > 0.f) {
            beta = -copysignf(sqrtf(x0 * x0 + xn2), x0);
            tau = (beta - x0) / beta;
            scal = 1.f / (x0 - beta);
          }
          s_beta = beta;
          s_stau = tau;
          s_scal = scal;
          R11[p][p] = beta;
          ptau[p] = tau;
          pbeta[p] = beta;
        }
        __syncthreads();
        if (rr < kL) cp[rr] = xv * s_scal;
        if (tid == 0) cp[row0] = 1.f;
        __syncthreads();
        const float tau = s_stau;
        const int j = p + 1 + warp;
        if (j < npiv) {
          float* cj = pan + (long)j * ldv;
          float w = 0.f;
          for (int row = row0 + lane; row < kL; row += 32) w += cp[row] * cj[row];
          w = bsum(w) * tau;
          for (int row = row0 + lane; row < kL; row += 32) cj[row] -= w * cp[row];
          __syncwarp();
          if (lane == 0) R11[p][j] = cj[row0];
        }
        __syncthreads();
      }
      // 4. apply the reflectors to this warp's other remaining columns
      bool isp[CPW];
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
        isp[u] = false;
        for (int p = 0; p < npiv; ++p) isp[u] |= spiv[p] == c0 + u;
      }
      for (int p = 0; p < npiv; ++p) {
        const float tau = ptau[p];
        if (tau == 0.f) continue;
        const float* cp = pan + (long)p * ldv;
        float vr[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int row = lane + 32 * t;
          vr[t] = (row >= st + p && row < kL) ? cp[row] : 0.f;
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
          for (int u = 0; u < CPW; ++u) w[u] += __shfl_xor_sync(kFull, w[u], o);
#pragma unroll
        for (int u = 0; u < CPW; ++u) {
          if (tj[u] != -1 || isp[u]) continue;  // uniform over the warp
          const float f = w[u] * tau;
#pragma unroll
          for (int t = 0; t < RPL; ++t) W[t][u] -= f * vr[t];
        }
      }
      // the largest remaining norm after t pivots, t = 1..npiv: exact norm below the block
      // plus the column's rows st + t .. st + npiv - 1
      {
        float mx[kBP + 1];
#pragma unroll
        for (int t = 0; t <= kBP; ++t) mx[t] = 0.f;
#pragma unroll
        for (int u = 0; u < CPW; ++u) {
          if (tj[u] != -1 || isp[u]) continue;
          float e = 0.f;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int row = lane + 32 * t;
            if (row >= st + npiv && row < kL) e += W[t][u] * W[t][u];
          }
          float rem = bsum(e);
          mx[kBP] = fmaxf(mx[kBP], rem);  // after all npiv pivots: the rows below the block
#pragma unroll
          for (int i = kBP - 1; i >= 0; --i) {
            if (i >= npiv) continue;
            const int row = st + i;
            float xl = 0.f;
#pragma unroll
            for (int t = 0; t < RPL; ++t)
              if (t == (row >> 5)) xl = W[t][u];
            const float x = __shfl_sync(kFull, xl, row & 31);
            rem += x * x;
            mx[i] = fmaxf(mx[i], rem);  // before pivot st + i: rows st + i .. below
          }
        }
        if (lane == 0)
#pragma unroll
          for (int t = 0; t <= kBP; ++t) wmx[warp][t] = mx[t];
      }
      __syncthreads();
      if (tid >= 1 && tid <= npiv) {
        const int t = tid;  // after t pivots: rows st + t .. remain
        float m = 0.f;
        for (int w = 0; w < kBW; ++w) m = fmaxf(m, t < npiv ? wmx[w][t] : 0.f);
        if (t == npiv) {  // nothing of the block's rows remains: the exact norms below it
          for (int w = 0; w < kBW; ++w) m = fmaxf(m, wmx[w][kBP]);
        }
        for (int tp = t; tp < npiv; ++tp) {  // pivot tp, not yet chosen: its R11 rows t..tp
          float a = 0.f;
          for (int i = t; i <= tp; ++i) a += R11[i][tp] * R11[i][tp];
          m = fmaxf(m, a);
        }
        stl[buf][t] = m;
      }
      cluster.sync();
      // every warp: the first t whose cluster-wide largest remaining norm is below the threshold
      int tstop = 0;
      for (int t = 1; t <= npiv; ++t) {
        float m = lane < NC ? *cluster.map_shared_rank(&stl[buf][t], lane) : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
        if (!(m > thr) || !(m > fl2)) { tstop = t; break; }
      }
      const int cnt = tstop ? tstop : npiv;
      for (int p = tid; p < cnt; p += blockDim.x) {
        taus[st + p] = ptau[p];
        sigs[st + p] = fabsf(pbeta[p]);
      }
      if (q == 0)
        for (int p = 0; p < cnt; ++p)
          for (int row = st + p + tid; row < kL; row += blockDim.x) Vb[(long)(st + p) * r + row] = pan[(long)p * ldv + row];
      // the pivot columns' R values (rows < st keep theirs); dropped pivots stay ordinary columns
      for (int p = 0; p < npiv; ++p) {
        const int col = spiv[p];
        if (col < c0 || col >= c0 + CPW) continue;
#pragma unroll
        for (int u = 0; u < CPW; ++u) {
          if (c0 + u != col) continue;
          if (p < cnt) tj[u] = st + p;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int row = lane + 32 * t;
            if (row < st) continue;
            const int i = row - st;
            if (p < cnt) W[t][u] = i <= p ? R11[min(i, kBP - 1)][p] : 0.f;
            else if (i < cnt) W[t][u] = R11[min(i, kBP - 1)][p];
          }
        }
      }
      st += cnt;
      __syncthreads();  // pan, spiv and R11 are rewritten by the next block
      if (tstop || st >= kmax) break;
    }
  }
  const int rank = st;
  cluster.sync();  // every block's reflector rows are in Vb and visible cluster-wide
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
  // Q_k = H_0 ... H_{k-1} [I; 0]: CTA q forms columns t0 .. t0 + nloc - 1 (local column tl in
  // warp tl % kBW, slot tl / kBW), the next reflector prefetched into the other half of vloc
  float* vloc = pan;  // [2][ldv]
  const int ck = (rank + NC - 1) / NC;
  const int t0 = q * ck, nloc = max(0, min(rank, t0 + ck) - t0);
#pragma unroll
  for (int t = 0; t < RPL; ++t)
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      const int tl = warp + kBW * u;
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
        const int tl = warp + kBW * u;
        if (tl >= nloc || t0 + tl < tp) continue;  // uniform over the warp
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < RPL; ++t) a += vr[t] * W[t][u];
        a = bsum(a) * tau;
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
    const int tl = warp + kBW * u;
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
static bool launch_blk(Ctx& c, int r, const float* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol,
                       const float* floor2, float* X, float* Y, float* sig, int* rank, const char* site) {
  constexpr int CW = kBW * CPW;
  const int NC = (kmaxR + CW - 1) / CW;
  const int ldv = (kmaxL + 3) / 4 * 4;
  if (NC > 8 || NC * CW > kBT || kmaxL > 32 * RPL) return false;
  const size_t sm = ((size_t)2 * kBL * CW + (size_t)kBL * NC * CW + (size_t)3 * kBP * ldv + 2 * (size_t)ldv) *
                    sizeof(float);
  if (sm > 200 * 1024) return false;
  ACR_CUDA(cudaFuncSetAttribute(k_qrcp_blk<RPL, CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(NB * NC));
  cfg.blockDim = dim3(kBT);
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
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_qrcp_blk<RPL, CPW>, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  DBuf<float> Vref(c, NB * (size_t)r * r);
  c.kbegin();
  ACR_CUDA(cudaLaunchKernelEx(&cfg, k_qrcp_blk<RPL, CPW>, r, ldv, C, kk, NB, Vref.p, X, Y, sig, rank, (float)tol,
                              floor2));
  c.kend(KC_JACOBI, 0, (double)NB * sizeof(float) * 3.0 * kmaxL * kmaxR, site);
  return true;
}

bool qrcp_blocked(Ctx& c, int r, const float* C, const int* kk, long NB, int kmaxL, int kmaxR, double tol,
                  const float* floor2, float* X, float* Y, float* sig, int* rank, const char* site) {
  if (kmaxL > 512 || kmaxR > 512) return false;
  if (kmaxL <= 128) return launch_blk<4, 8>(c, r, C, kk, NB, kmaxL, kmaxR, tol, floor2, X, Y, sig, rank, site);
  if (kmaxL <= 256) return launch_blk<8, 8>(c, r, C, kk, NB, kmaxL, kmaxR, tol, floor2, X, Y, sig, rank, site);
  return launch_blk<16, 4>(c, r, C, kk, NB, kmaxL, kmaxR, tol, floor2, X, Y, sig, rank, site);
}

}  // namespace acr
