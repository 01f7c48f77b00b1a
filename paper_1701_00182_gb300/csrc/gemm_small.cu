// CUDA-core tilings for the small, heavily batched products of the HODLR
// arithmetic, where a 128 x 128 tensor-core tile is mostly padding:
//
//  * k_gemm_skinny: C (M x N, M <= 32) = A B with B and C row-major -- the
//    coefficient reductions c = V|c^T W|c of the level-flat matvec and of the
//    Woodbury apply (M is a HODLR rank, N a panel width, K a cluster size).
//    One warp owns 32 * CPL columns (CPL = 1 or 2) of one batch entry and the
//    whole K range; lane l holds columns l, l + 32, so every B load and C store is one
//    coalesced 128-byte row segment.  A's columns are staged per warp in
//    shared memory and read as broadcasts.  These products read each B element
//    once and are bound by HBM bandwidth.
//  * k_gemm_v: 64 x 64, 64 x 128 and 128 x 64 tiles with 4 x 4 register
//    quadrants read from shared memory as 16-byte vectors, the next K tile
//    fetched into registers while the current one is consumed -- leaf-block
//    products, expansions with a small inner dimension and other tiles of a
//    few thousand outputs.
//
// Both follow the batched operand addressing of the other tilings (Op<T>,
// split-K partials in GArgs::partial) and serve FP32 and FP64.
#include "../../include/acr.h"
#include "acr_internal.h"
#include "tc_common.cuh"

namespace acr {

namespace {

template <class T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p);
  const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

template <class T>
constexpr int kSkKC = sizeof(T) == 8 ? 16 : 32;  // K rows of A staged per warp and chunk (static shared memory < 48 KB)
template <class T>
constexpr int kVBK = sizeof(T) == 8 ? 8 : 16;  // K depth of a vector-read tile (static shared memory < 48 KB)
constexpr int kSkKU = 8;   // B rows loaded ahead of their use

}  // namespace

template <class T, int MT, int CPL>
__global__ void __launch_bounds__(256) k_gemm_skinny(GArgs<T> g, int spe) {
  __shared__ __align__(16) T As[8][kSkKC<T>][MT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long slab = (long)blockIdx.x * 8 + warp;
  if (slab >= (long)g.batch * spe) return;  // warp-uniform; the kernel has no block barrier
  const int bi = (int)(slab / spe), sj = (int)(slab - (long)bi * spe);
  const int plane = bi / g.nclus, c = bi - plane * g.nclus;
  const int j0 = sj * 32 * CPL + lane;
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const T* __restrict__ A = opaddr(g.A, plane, c);
  const T* __restrict__ B = opaddr(g.B, plane, c);
  const long ars = g.A.rs, acs = g.A.cs, brs = g.B.rs;
  bool ok[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) ok[q] = j0 + 32 * q < g.N;
  T acc[MT][CPL];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int q = 0; q < CPL; ++q) acc[i][q] = T(0);
  T (*as)[MT] = As[warp];
  for (int k0 = kbeg; k0 < kend; k0 += kSkKC<T>) {
    const int kn = min(kSkKC<T>, kend - k0);
    __syncwarp();
    if (ars == 1) {
      for (int e = lane; e < kSkKC<T> * MT; e += 32) {
        const int i = e % MT, kk = e / MT;
        as[kk][i] = (i < g.M && kk < kn) ? A[i + (long)(k0 + kk) * acs] : T(0);
      }
    } else {
      for (int e = lane; e < kSkKC<T> * MT; e += 32) {
        const int kk = e % kSkKC<T>, i = e / kSkKC<T>;
        as[kk][i] = (i < g.M && kk < kn) ? A[(long)i * ars + (long)(k0 + kk) * acs] : T(0);
      }
    }
    __syncwarp();
    for (int kb = 0; kb < kn; kb += kSkKU) {
      T b[kSkKU][CPL];
#pragma unroll
      for (int u = 0; u < kSkKU; ++u) {
        const T* br = B + (long)(k0 + kb + u) * brs + j0;
#pragma unroll
        for (int q = 0; q < CPL; ++q) b[u][q] = (kb + u < kn && ok[q]) ? br[32 * q] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kSkKU; ++u) {
#pragma unroll
        for (int i = 0; i < MT; i += 4) {
          T a[4];
          ld4<T>(&as[kb + u][i], a);
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int q = 0; q < CPL; ++q) acc[i + v][q] = fma(a[v], b[u][q], acc[i + v][q]);
        }
      }
    }
  }
  if (g.partial) {
    T* P = g.partial + ((long)blockIdx.z * g.batch + bi) * (long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      if (i >= g.M) break;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (ok[q]) P[(long)i * g.N + j0 + 32 * q] = acc[i][q];
    }
    return;
  }
  T* C = opaddr(g.C, plane, c);
  const long crs = g.C.rs;
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    if (i >= g.M) break;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      if (!ok[q]) continue;
      T* cp = C + (long)i * crs + j0 + 32 * q;
      T v = g.alpha * acc[i][q];
      if (g.beta != T(0)) v += g.beta * *cp;
      *cp = v;
    }
  }
}

// Thread (tx, ty) owns rows ty*4 + {0..3} + 4*NTY*{0..TM/4-1} and columns
// tx*4 + {0..3} + 4*NTX*{0..TN/4-1} of the BM x BN tile.
template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256) k_gemm_v(GArgs<T> g) {
  constexpr int NTX = BN / TN, NTY = BM / TM;
  static_assert(NTX * NTY == 256 && TM % 4 == 0 && TN % 4 == 0, "tile shape");
  constexpr int PAD = 16 / sizeof(T);
  constexpr int LA = BM * BK / 256, LB = BK * BN / 256;
  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BN + PAD];
  const int bi = blockIdx.x;
  const int plane = bi / g.nclus, c = bi - plane * g.nclus;
  const int tilesN = (g.N + BN - 1) / BN;
  const int m0 = (blockIdx.y / tilesN) * BM, n0 = (blockIdx.y % tilesN) * BN;
  if (g.sym && m0 >= n0 + BN) return;  // tile strictly below the diagonal (uniform)
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const T* __restrict__ A = opaddr(g.A, plane, c);
  const T* __restrict__ B = opaddr(g.B, plane, c);
  const long ars = g.A.rs, acs = g.A.cs, brs = g.B.rs, bcs = g.B.cs;
  const bool a_kfast = (acs == 1), b_nfast = (bcs == 1);
  const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;
  T ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = tid + 256 * u;
      const int ii = a_kfast ? e / BK : e % BM, kk = a_kfast ? e % BK : e / BM;
      const int gi = m0 + ii, gk = k0 + kk;
      ra[u] = (gi < g.M && gk < kend) ? A[(long)gi * ars + (long)gk * acs] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = tid + 256 * u;
      const int jj = b_nfast ? e % BN : e / BK, kk = b_nfast ? e / BN : e % BK;
      const int gj = n0 + jj, gk = k0 + kk;
      rb[u] = (gk < kend && gj < g.N) ? B[(long)gk * brs + (long)gj * bcs] : T(0);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = tid + 256 * u;
      const int ii = a_kfast ? e / BK : e % BM, kk = a_kfast ? e % BK : e / BM;
      As[buf][kk][ii] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = tid + 256 * u;
      const int jj = b_nfast ? e % BN : e / BK, kk = b_nfast ? e / BN : e % BK;
      Bs[buf][kk][jj] = rb[u];
    }
  };
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  int buf = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int qa = 0; qa < TM / 4; ++qa) {
        T t[4];
        ld4<T>(&As[buf][kk][ty * 4 + qa * 4 * NTY], t);
#pragma unroll
        for (int v = 0; v < 4; ++v) av[qa * 4 + v] = t[v];
      }
#pragma unroll
      for (int qb = 0; qb < TN / 4; ++qb) {
        T t[4];
        ld4<T>(&Bs[buf][kk][tx * 4 + qb * 4 * NTX], t);
#pragma unroll
        for (int v = 0; v < 4; ++v) bv[qb * 4 + v] = t[v];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  auto row_of = [&](int i) { return m0 + ty * 4 + (i & 3) + (i >> 2) * 4 * NTY; };
  auto col_of = [&](int j) { return n0 + tx * 4 + (j & 3) + (j >> 2) * 4 * NTX; };
  if (g.partial) {
    T* P = g.partial + ((long)blockIdx.z * g.batch + bi) * (long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gi = row_of(i);
      if (gi >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gj = col_of(j);
        if (gj < g.N) P[(long)gi * g.N + gj] = acc[i][j];
      }
    }
    return;
  }
  T* C = opaddr(g.C, plane, c);
  const long crs = g.C.rs, ccs = g.C.cs;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = row_of(i);
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = col_of(j);
      if (gj >= g.N) continue;
      T* cp = C + (long)gi * crs + (long)gj * ccs;
      T v = g.alpha * acc[i][j];
      if (g.beta != T(0)) v += g.beta * *cp;
      *cp = v;
    }
  }
}

template <class T, int MT, int CPL>
static void launch_skinny_t(const GArgs<T>& g, long batch, int split, cudaStream_t st) {
  const int spe = (g.N + 32 * CPL - 1) / (32 * CPL);
  const long ctas = (batch * spe + 7) / 8;
  k_gemm_skinny<T, MT, CPL><<<dim3((unsigned)ctas, 1, (unsigned)split), 256, 0, st>>>(g, spe);
}

template <class T>
void launch_gemm_small(int kind, const GArgs<T>& g, dim3 grid, long batch, int split, cudaStream_t st) {
  switch (kind) {
    case 0: {  // skinny: M <= 32, B and C row-major; two columns per lane unless N <= 32
      if (g.M > 32 || g.B.cs != 1 || (!g.partial && g.C.cs != 1))
        throw AcrError(ACR_ERR_ARG, "one-warp-per-slab GEMM tiling needs M <= 32 and row-major B and C");
      const int mt = g.M <= 8 ? 8 : g.M <= 16 ? 16 : 32;
      const bool one = g.N <= 32;
      if (mt == 8) {
        if (one) launch_skinny_t<T, 8, 1>(g, batch, split, st);
        else launch_skinny_t<T, 8, 2>(g, batch, split, st);
      } else if (mt == 16) {
        if (one) launch_skinny_t<T, 16, 1>(g, batch, split, st);
        else launch_skinny_t<T, 16, 2>(g, batch, split, st);
      } else if constexpr (sizeof(T) == 8) {
        launch_skinny_t<T, 32, 1>(g, batch, split, st);  // two FP64 columns per lane would spill
      } else {
        if (one) launch_skinny_t<T, 32, 1>(g, batch, split, st);
        else launch_skinny_t<T, 32, 2>(g, batch, split, st);
      }
      break;
    }
    case 1: k_gemm_v<T, 64, 64, kVBK<T>, 4, 4><<<grid, 256, 0, st>>>(g); break;
    case 2: k_gemm_v<T, 64, 128, kVBK<T>, 4, 8><<<grid, 256, 0, st>>>(g); break;
    default: k_gemm_v<T, 128, 64, kVBK<T>, 8, 4><<<grid, 256, 0, st>>>(g); break;
  }
}

template void launch_gemm_small<float>(int, const GArgs<float>&, dim3, long, int, cudaStream_t);
template void launch_gemm_small<double>(int, const GArgs<double>&, dim3, long, int, cudaStream_t);

}  // namespace acr
