// Batched strided GEMM for the HODLR arithmetic: C = alpha A B + beta C over
// (plane, cluster) batch entries whose operands are located by Op<T>.
//
// Every product the H-arithmetic needs (leaf products, V^T W coefficient
// reductions over a cluster, U T expansions, Gram matrices, rebuilds) is one
// call.  Tall reductions with few batch entries are split along K into a
// scratch buffer and reduced by a second kernel.  Four register tilings exist;
// with autotuning enabled the fastest one per (precision, shape class) is
// measured once with CUDA events and cached for the process.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "acr_internal.h"
#include "tc_common.cuh"

namespace acr {

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm(GArgs<T> g) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int bi = blockIdx.x;
  const int plane = bi / g.nclus, c = bi - plane * g.nclus;
  const int tilesN = (g.N + BN - 1) / BN;
  const int m0 = (blockIdx.y / tilesN) * BM, n0 = (blockIdx.y % tilesN) * BN;
  if (g.sym && m0 >= n0 + BN) return;  // tile strictly below the diagonal
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const T* __restrict__ A = opaddr(g.A, plane, c);
  const T* __restrict__ B = opaddr(g.B, plane, c);
  const long ars = g.A.rs, acs = g.A.cs, brs = g.B.rs, bcs = g.B.cs;
  const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  const bool a_kfast = (acs == 1), b_nfast = (bcs == 1);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    if (a_kfast) {
      for (int e = tid; e < BM * BK; e += NT) {
        int ii = e / BK, kk = e % BK;
        int gi = m0 + ii, gk = k0 + kk;
        As[kk][ii] = (gi < g.M && gk < kend) ? A[(long)gi * ars + gk] : T(0);
      }
    } else {
      for (int e = tid; e < BM * BK; e += NT) {
        int ii = e % BM, kk = e / BM;
        int gi = m0 + ii, gk = k0 + kk;
        As[kk][ii] = (gi < g.M && gk < kend) ? A[(long)gi * ars + (long)gk * acs] : T(0);
      }
    }
    if (b_nfast) {
      for (int e = tid; e < BK * BN; e += NT) {
        int kk = e / BN, jj = e % BN;
        int gk = k0 + kk, gj = n0 + jj;
        Bs[kk][jj] = (gk < kend && gj < g.N) ? B[(long)gk * brs + gj] : T(0);
      }
    } else {
      for (int e = tid; e < BK * BN; e += NT) {
        int kk = e % BK, jj = e / BK;
        int gk = k0 + kk, gj = n0 + jj;
        Bs[kk][jj] = (gk < kend && gj < g.N) ? B[(long)gk * brs + (long)gj * bcs] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (g.partial) {
    T* P = g.partial + ((long)blockIdx.z * g.batch + bi) * (long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int gi = m0 + ty * TM + i;
      if (gi >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int gj = n0 + tx * TN + j;
        if (gj < g.N) P[(long)gi * g.N + gj] = acc[i][j];
      }
    }
    return;
  }
  T* C = opaddr(g.C, plane, c);
  const long crs = g.C.rs, ccs = g.C.cs;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int gi = m0 + ty * TM + i;
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gj = n0 + tx * TN + j;
      if (gj >= g.N) continue;
      T* cp = C + (long)gi * crs + (long)gj * ccs;
      T v = g.alpha * acc[i][j];
      if (g.beta != T(0)) v += g.beta * *cp;
      *cp = v;
    }
  }
}

// FP32 128 x 128 tile, BK = 8, 256 threads, 8 x 8 outputs per thread arranged
// as four 4 x 4 quadrants (rows ty*4 + {0, 64}, columns tx*4 + {0, 64}) so the
// shared-memory reads are float4 and bank-conflict free.  The next K tile is
// fetched into registers while the current one is consumed (double buffer).
__global__ void __launch_bounds__(256) k_gemm_f32_big(GArgs<float> g) {
  constexpr int BM = 128, BN = 128, BK = 8;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int bi = blockIdx.x;
  const int plane = bi / g.nclus, c = bi - plane * g.nclus;
  const int tilesN = (g.N + BN - 1) / BN;
  const int m0 = (blockIdx.y / tilesN) * BM, n0 = (blockIdx.y % tilesN) * BN;
  if (g.sym && m0 >= n0 + BN) return;
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const float* __restrict__ A = opaddr(g.A, plane, c);
  const float* __restrict__ B = opaddr(g.B, plane, c);
  const long ars = g.A.rs, acs = g.A.cs, brs = g.B.rs, bcs = g.B.cs;
  const bool a_kfast = (acs == 1), b_nfast = (bcs == 1);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // Each thread stages 4 elements of the A tile and 4 of the B tile.
  float ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int e = tid + 256 * u;
      int ii, kk;
      if (a_kfast) { ii = e >> 3; kk = e & 7; } else { ii = e & 127; kk = e >> 7; }
      int gi = m0 + ii, gk = k0 + kk;
      ra[u] = (gi < g.M && gk < kend) ? A[(long)gi * ars + (long)gk * acs] : 0.f;
      int jj, kb;
      if (b_nfast) { jj = e & 127; kb = e >> 7; } else { jj = e >> 3; kb = e & 7; }
      int gj = n0 + jj, gk2 = k0 + kb;
      rb[u] = (gk2 < kend && gj < g.N) ? B[(long)gk2 * brs + (long)gj * bcs] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int e = tid + 256 * u;
      int ii, kk;
      if (a_kfast) { ii = e >> 3; kk = e & 7; } else { ii = e & 127; kk = e >> 7; }
      As[buf][kk][ii] = ra[u];
      int jj, kb;
      if (b_nfast) { jj = e & 127; kb = e >> 7; } else { jj = e >> 3; kb = e & 7; }
      Bs[buf][kb][jj] = rb[u];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
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
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4 + 64]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4 + 64]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  auto row_of = [&](int i) { return m0 + ty * 4 + (i & 3) + ((i >> 2) << 6); };
  auto col_of = [&](int j) { return n0 + tx * 4 + (j & 3) + ((j >> 2) << 6); };
  if (g.partial) {
    float* P = g.partial + ((long)blockIdx.z * g.batch + bi) * (long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int gi = row_of(i);
      if (gi >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int gj = col_of(j);
        if (gj < g.N) P[(long)gi * g.N + gj] = acc[i][j];
      }
    }
    return;
  }
  float* C = opaddr(g.C, plane, c);
  const long crs = g.C.rs, ccs = g.C.cs;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int gi = row_of(i);
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int gj = col_of(j);
      if (gj >= g.N) continue;
      float* cp = C + (long)gi * crs + (long)gj * ccs;
      float v = g.alpha * acc[i][j];
      if (g.beta != 0.f) v += g.beta * *cp;
      *cp = v;
    }
  }
}

// ---- 3xTF32 tensor-core tile --------------------------------------------------
// FP32 GEMM on the tensor pipe: every operand x is split into a TF32 head
// h = tf32(x) and tail l = tf32(x - h), and a*b is accumulated in FP32 as
// a_l b_h + a_h b_l + a_h b_h (the a_l b_l term is below FP32 rounding), which
// keeps FP32-level accuracy.  mma.sync m16n8k8 (row.col), 128 x 128 x 16 tile,
// 8 warps of 64 x 32, double-buffered shared memory.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) k_gemm_tf32x3(GArgs<float> g) {
  constexpr int BM = 128, BN = 128, BK = 16, PAD = 8;
  __shared__ __align__(16) float As[2][BK][BM + PAD];
  __shared__ __align__(16) float Bs[2][BK][BN + PAD];
  const int bi = blockIdx.x;
  const int plane = bi / g.nclus, c = bi - plane * g.nclus;
  const int tilesN = (g.N + BN - 1) / BN;
  const int m0 = (blockIdx.y / tilesN) * BM, n0 = (blockIdx.y % tilesN) * BN;
  if (g.sym && m0 >= n0 + BN) return;
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const float* __restrict__ A = opaddr(g.A, plane, c);
  const float* __restrict__ B = opaddr(g.B, plane, c);
  const long ars = g.A.rs, acs = g.A.cs, brs = g.B.rs, bcs = g.B.cs;
  const bool a_kfast = (acs == 1), b_nfast = (bcs == 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;  // warp tile origin
  const int gq = lane >> 2, tq = lane & 3;                  // groupID, thread in group
  float ra[8], rb[8];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int e = tid + 256 * u;
      int ii, kk;
      if (a_kfast) { ii = e >> 4; kk = e & 15; } else { ii = e & 127; kk = e >> 7; }
      int gi = m0 + ii, gk = k0 + kk;
      ra[u] = (gi < g.M && gk < kend) ? A[(long)gi * ars + (long)gk * acs] : 0.f;
      int jj, kb;
      if (b_nfast) { jj = e & 127; kb = e >> 7; } else { jj = e >> 4; kb = e & 15; }
      int gj = n0 + jj, gk2 = k0 + kb;
      rb[u] = (gk2 < kend && gj < g.N) ? B[(long)gk2 * brs + (long)gj * bcs] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int e = tid + 256 * u;
      int ii, kk;
      if (a_kfast) { ii = e >> 4; kk = e & 15; } else { ii = e & 127; kk = e >> 7; }
      As[buf][kk][ii] = ra[u];
      int jj, kb;
      if (b_nfast) { jj = e & 127; kb = e >> 7; } else { jj = e >> 4; kb = e & 15; }
      Bs[buf][kb][jj] = rb[u];
    }
  };
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
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
    for (int ks = 0; ks < BK; ks += 8) {
      uint32_t ah[4][4], al[4][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int mr = wm + 16 * i + gq;
        split_tf32(As[buf][ks + tq][mr], ah[i][0], al[i][0]);
        split_tf32(As[buf][ks + tq][mr + 8], ah[i][1], al[i][1]);
        split_tf32(As[buf][ks + tq + 4][mr], ah[i][2], al[i][2]);
        split_tf32(As[buf][ks + tq + 4][mr + 8], ah[i][3], al[i][3]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nc = wn + 8 * j + gq;
        split_tf32(Bs[buf][ks + tq][nc], bh[j][0], bl[j][0]);
        split_tf32(Bs[buf][ks + tq + 4][nc], bh[j][1], bl[j][1]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          mma_tf32(acc[i][j], al[i], bh[j]);
          mma_tf32(acc[i][j], ah[i], bl[j]);
          mma_tf32(acc[i][j], ah[i], bh[j]);
        }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* P = g.partial ? g.partial + ((long)blockIdx.z * g.batch + bi) * (long)g.M * g.N : nullptr;
  float* C = g.partial ? nullptr : opaddr(g.C, plane, c);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gi = m0 + wm + 16 * i + gq + ((q & 2) ? 8 : 0);
        const int gj = n0 + wn + 8 * j + 2 * tq + (q & 1);
        if (gi >= g.M || gj >= g.N) continue;
        if (P) {
          P[(long)gi * g.N + gj] = acc[i][j][q];
        } else {
          float* cp = C + (long)gi * g.C.rs + (long)gj * g.C.cs;
          float v = g.alpha * acc[i][j][q];
          if (g.beta != 0.f) v += g.beta * *cp;
          *cp = v;
        }
      }
}

template <class T>
__global__ void k_splitk_reduce(GArgs<T> g, int nsplit) {
  long tot = (long)g.batch * g.M * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    long bi = e / ((long)g.M * g.N);
    long r = e - bi * (long)g.M * g.N;
    int i = (int)(r / g.N), j = (int)(r % g.N);
    if (g.sym && i > j) continue;
    T s = T(0);
    for (int q = 0; q < nsplit; ++q) s += g.partial[((long)q * g.batch + bi) * (long)g.M * g.N + r];
    int plane = (int)(bi / g.nclus), c = (int)(bi - (long)plane * g.nclus);
    T* cp = opaddr(g.C, plane, c) + (long)i * g.C.rs + (long)j * g.C.cs;
    T v = g.alpha * s;
    if (g.beta != T(0)) v += g.beta * *cp;
    *cp = v;
  }
}

template <class T>
__global__ void k_mirror(GArgs<T> g) {
  long tot = (long)g.batch * g.M * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    long bi = e / ((long)g.M * g.N);
    long r = e - bi * (long)g.M * g.N;
    int i = (int)(r / g.N), j = (int)(r % g.N);
    if (i <= j) continue;
    int plane = (int)(bi / g.nclus), c = (int)(bi - (long)plane * g.nclus);
    T* C = opaddr(g.C, plane, c);
    C[(long)i * g.C.rs + (long)j * g.C.cs] = C[(long)j * g.C.rs + (long)i * g.C.cs];
  }
}

template <class T>
__global__ void k_scale_c(GArgs<T> g) {
  long tot = (long)g.batch * g.M * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    long bi = e / ((long)g.M * g.N);
    long r = e - bi * (long)g.M * g.N;
    int i = (int)(r / g.N), j = (int)(r % g.N);
    int plane = (int)(bi / g.nclus), c = (int)(bi - (long)plane * g.nclus);
    T* cp = opaddr(g.C, plane, c) + (long)i * g.C.rs + (long)j * g.C.cs;
    *cp = (g.beta == T(0)) ? T(0) : g.beta * *cp;
  }
}

// ---- FP32 GEMM on the 5th-generation tensor cores (3xTF32) ---------------------
// 128 x 128 output tile per CTA, accumulated in tensor memory (128 lanes x 128
// FP32 columns).  Each 32-deep K slice of A and B is loaded by the CTA's 512
// threads (any strides, zero fill outside the operand), split into a TF32 high
// part and the rounded remainder, and stored K-major in the 128-byte-swizzled
// layout the tensor core reads (row r, 16-byte chunk q at r*128 + (q^(r%8))*16,
// 8-row atoms 1 KB apart).  One thread then issues A_hi B_hi + A_hi B_lo +
// A_lo B_hi as 3 x 4 MMAs of 128 x 128 x 8 and commits them to the slice's
// mbarrier.  Three shared-memory stages and two register sets keep the global
// loads of slices k+1 and k+2 in flight while the MMAs of slice k run.  The
// epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32 (w mod 4)
// .. +31, a quarter of the columns per w / 4).  Every mbarrier wait is bounded
// in time; on expiry the kernel sets an error flag, skips its epilogue and
// still frees its tensor memory.
namespace tc {
constexpr int BM = 128, BN = 128, BK = 32;
constexpr int NT = 512;                      // 16 warps
constexpr int TILE_BYTES = BM * BK * 4;      // 128 rows x 128 B
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A_hi, A_lo, B_hi, B_lo
constexpr int NSTAGE = 3;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;  // + slack for the 1 KB alignment
constexpr uint32_t TMEM_COLS = 128;
// instruction descriptor: D F32, A and B TF32, both K-major, N >> 3, M >> 4
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}  // namespace tc

// AK: A(i, k) is contiguous along k (A.cs == 1); BKC: B(k, j) is contiguous
// along k (B.rs == 1).  Lanes run along each operand's contiguous direction.
template <bool AK, bool BKC>
__global__ void __launch_bounds__(tc::NT, 1) k_gemm_tc05(GArgs<float> g, int* err) {
  constexpr int QT = (tc::BM * tc::BK / 4) / tc::NT;  // quads of A (and of B) per thread per slice
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t bars[tc::NSTAGE];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bi = blockIdx.x;
  const int plane = bi / g.nclus, c = bi - plane * g.nclus;
  const int tilesN = (g.N + tc::BN - 1) / tc::BN;
  const int m0 = (blockIdx.y / tilesN) * tc::BM, n0 = (blockIdx.y % tilesN) * tc::BN;
  if (g.sym && m0 >= n0 + tc::BN) return;  // tile strictly below the diagonal (uniform)
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + tc::BK - 1) / tc::BK : 0;
  const uint32_t raw_s = smem_u32(tc_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;
  unsigned char* base = tc_raw + (base_s - raw_s);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tc::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < tc::NSTAGE; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  const float* A = opaddr(g.A, plane, c);
  const float* B = opaddr(g.B, plane, c);
  const long ars = g.A.rs, acs = AK ? 1 : g.A.cs, brs = BKC ? 1 : g.B.rs, bcs = g.B.cs;
  // Fixed per thread for the whole K loop: the rows it loads, their first
  // element, whether they exist, and where their quads go in a stage.
  float ra0[QT][4], rb0[QT][4], ra1[QT][4], rb1[QT][4];
  const float* pa[QT];
  const float* pb[QT];
  bool va[QT], vb[QT];
  int qa[QT], qb[QT];
  uint32_t oa[QT], ob[QT];
#pragma unroll
  for (int it = 0; it < QT; ++it) {
    const int e = tid + tc::NT * it;
    int row = AK ? (e >> 3) : (e & 127), q = AK ? (e & 7) : (e >> 7);
    va[it] = m0 + row < g.M;
    qa[it] = 4 * q;
    pa[it] = A + (long)(va[it] ? m0 + row : 0) * ars + (long)(kbeg + 4 * q) * acs;
    oa[it] = row * 128 + ((q ^ (row & 7)) << 4);
    row = BKC ? (e >> 3) : (e & 127);
    q = BKC ? (e & 7) : (e >> 7);
    vb[it] = n0 + row < g.N;
    qb[it] = 4 * q;
    pb[it] = B + (long)(vb[it] ? n0 + row : 0) * bcs + (long)(kbeg + 4 * q) * brs;
    ob[it] = row * 128 + ((q ^ (row & 7)) << 4);
  }
  auto load = [&](int kc, float (&ra)[QT][4], float (&rb)[QT][4]) {
    const int kr = kend - kbeg - kc * tc::BK;  // k rows left in this slice (relative)
    const long ka = (long)kc * tc::BK * acs, kb = (long)kc * tc::BK * brs;
    if (kr >= tc::BK) {
#pragma unroll
      for (int it = 0; it < QT; ++it)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ra[it][j] = va[it] ? pa[it][ka + j * acs] : 0.f;
          rb[it][j] = vb[it] ? pb[it][kb + j * brs] : 0.f;
        }
    } else {
#pragma unroll
      for (int it = 0; it < QT; ++it)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ra[it][j] = (va[it] && qa[it] + j < kr) ? pa[it][ka + j * acs] : 0.f;
          rb[it][j] = (vb[it] && qb[it] + j < kr) ? pb[it][kb + j * brs] : 0.f;
        }
    }
  };
  // TF32 high part rounded to nearest (ties away from zero: add half an ulp of
  // bit 13 to the magnitude, clear the low 13 bits), and the rounded remainder.
  auto split4 = [](const float (&x)[4], float4& h, float4& l) {
    auto hi = [](float v) { return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u); };
    h.x = hi(x[0]); l.x = hi(x[0] - h.x);
    h.y = hi(x[1]); l.y = hi(x[1] - h.y);
    h.z = hi(x[2]); l.z = hi(x[2] - h.z);
    h.w = hi(x[3]); l.w = hi(x[3] - h.w);
  };
  auto store = [&](int s, const float (&ra)[QT][4], const float (&rb)[QT][4]) {
    unsigned char* st = base + s * tc::STAGE_BYTES;
#pragma unroll
    for (int it = 0; it < QT; ++it) {
      float4 h, l;
      split4(ra[it], h, l);
      *reinterpret_cast<float4*>(st + oa[it]) = h;
      *reinterpret_cast<float4*>(st + tc::TILE_BYTES + oa[it]) = l;
      split4(rb[it], h, l);
      *reinterpret_cast<float4*>(st + 2 * tc::TILE_BYTES + ob[it]) = h;
      *reinterpret_cast<float4*>(st + 3 * tc::TILE_BYTES + ob[it]) = l;
    }
  };
  auto issue = [&](int kc, int s) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t sa = base_s + s * tc::STAGE_BYTES;
#pragma unroll
    for (int kk = 0; kk < tc::BK / 8; ++kk) {
      const uint64_t ah = umma_desc_sw128(sa + kk * 32), al = umma_desc_sw128(sa + tc::TILE_BYTES + kk * 32);
      const uint64_t bh = umma_desc_sw128(sa + 2 * tc::TILE_BYTES + kk * 32),
                     bl = umma_desc_sw128(sa + 3 * tc::TILE_BYTES + kk * 32);
      umma_tf32(tmem, ah, bh, tc::IDESC, (kc > 0 || kk > 0) ? 1u : 0u);
      umma_tf32(tmem, ah, bl, tc::IDESC, 1u);
      umma_tf32(tmem, al, bh, tc::IDESC, 1u);
    }
    umma_commit(smem_u32(&bars[s]));
  };
  // One step: wait until the MMAs that last read stage kc % NSTAGE are done,
  // store slice kc there, one barrier (which also votes on the waits), start
  // the loads of slice kc + 2 into the freed registers, issue the MMAs.
  auto step = [&](int kc, float (&ra)[QT][4], float (&rb)[QT][4]) -> bool {
    const int s = kc % tc::NSTAGE;
    bool ok = true;
    if (kc >= tc::NSTAGE) ok = mbar_wait_bounded(smem_u32(&bars[s]), ((kc - tc::NSTAGE) / tc::NSTAGE) & 1);
    if (ok) store(s, ra, rb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) return false;
    if (kc + 2 < nk) load(kc + 2, ra, rb);
    if (tid == 0) issue(kc, s);
    return true;
  };

  bool ok = true;
  if (nk > 0) load(0, ra0, rb0);
  if (nk > 1) load(1, ra1, rb1);
  for (int kc = 0; kc < nk && ok; kc += 2) {
    ok = step(kc, ra0, rb0);
    if (ok && kc + 1 < nk) ok = step(kc + 1, ra1, rb1);
  }
  if (ok && nk > 0) ok = mbar_wait_bounded(smem_u32(&bars[(nk - 1) % tc::NSTAGE]), ((nk - 1) / tc::NSTAGE) & 1);
  if (!__syncthreads_and(ok)) s_ok = 0;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_ok) {
    // warp w reads TMEM lanes 32 (w mod 4) .. +31 and columns CW (w / 4) .. +CW-1
    constexpr int CW = tc::BN / (tc::NT / 128);
    const int lb = (warp & 3) * 32, cb = (warp >> 2) * CW;
    float* stg = reinterpret_cast<float*>(base) + warp * 32 * 17;  // stages are free now
#pragma unroll 1
    for (int ch = 0; ch < CW / 16; ++ch) {
      uint32_t r[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)(cb + ch * 16), r);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      }
      store_chunk(g, stg, r, lane, m0 + lb, n0 + cb + ch * 16, plane, c, bi);
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::TMEM_COLS));
}

template <bool AK, bool BKC>
void launch_tc05(dim3 grid, const GArgs<float>& g, cudaStream_t st, int* err) {
  ACR_CUDA(cudaFuncSetAttribute(k_gemm_tc05<AK, BKC>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
  k_gemm_tc05<AK, BKC><<<grid, tc::NT, tc::SMEM_BYTES, st>>>(g, err);
}

void launch_tc05_any(dim3 grid, const GArgs<float>& g, cudaStream_t st, int* err) {
  const bool ak = g.A.cs == 1, bk = g.B.rs == 1;
  if (ak && bk) launch_tc05<true, true>(grid, g, st, err);
  else if (ak) launch_tc05<true, false>(grid, g, st, err);
  else if (bk) launch_tc05<false, true>(grid, g, st, err);
  else launch_tc05<false, false>(grid, g, st, err);
}

namespace {

struct Cfg {
  int bm, bn, bk;
};
constexpr int kNCfg = 12;
constexpr Cfg kCfg[kNCfg] = {{64, 64, 16},   {128, 64, 8},   {32, 32, 32},   {128, 128, 8},
                             {128, 128, 8},  {128, 128, 16}, {128, 128, 32}, {128, 128, 32},
                             {32, 1024, 32}, {64, 64, 16},   {64, 128, 16},  {128, 64, 16}};

// Configurations 5 (mma.sync 3xTF32), 6 (tcgen05 3xTF32, in-kernel split) and
// 7 (tcgen05 3xTF32, pre-split tiles fed by TMA) exist for FP32 only; 8 (one
// warp per 32-128 columns, gemm_small.cu) needs M <= 32 and row-major B and C
// (skinny = true); 9-11 are the vector-read CUDA-core tiles of gemm_small.cu.
bool cfg_valid(int cfg, int es, bool tensor, bool skinny) {
  if (cfg == 8) return skinny;
  return cfg < 5 || cfg > 8 || (tensor && es == 4);
}

// The tile index of the grid's y dimension stays below its 65535 limit (the
// one-warp-per-slab tiling puts its slabs on x).
bool grid_ok(int cfg, int M, int N) {
  if (cfg == 8) return true;
  return (long)((M + kCfg[cfg].bm - 1) / kCfg[cfg].bm) * ((N + kCfg[cfg].bn - 1) / kCfg[cfg].bn) <= 65535;
}

template <class T>
void launch_cfg(int cfg, dim3 grid, const GArgs<T>& g, cudaStream_t st, int* err) {
  switch (cfg) {
    case 0: k_gemm<T, 64, 64, 16, 4, 4><<<grid, 256, 0, st>>>(g); break;
    case 1: k_gemm<T, 128, 64, 8, 8, 4><<<grid, 256, 0, st>>>(g); break;
    case 2: k_gemm<T, 32, 32, 32, 2, 2><<<grid, 256, 0, st>>>(g); break;
    case 3: k_gemm<T, 128, 128, 8, 8, 8><<<grid, 256, 0, st>>>(g); break;
    case 4:
      if constexpr (sizeof(T) == 4) k_gemm_f32_big<<<grid, 256, 0, st>>>(g);
      else k_gemm<T, 128, 128, 8, 8, 8><<<grid, 256, 0, st>>>(g);
      break;
    case 5:
      if constexpr (sizeof(T) == 4) k_gemm_tf32x3<<<grid, 256, 0, st>>>(g);
      else k_gemm<T, 128, 128, 8, 8, 8><<<grid, 256, 0, st>>>(g);
      break;
    case 8:
    case 9:
    case 10:
    case 11: launch_gemm_small<T>(cfg - 8, g, grid, g.batch, (int)grid.z, st); break;
    default:
      if constexpr (sizeof(T) == 4) {
        launch_tc05_any(grid, g, st, err);
      } else {
        k_gemm<T, 128, 128, 8, 8, 8><<<grid, 256, 0, st>>>(g);
      }
      break;
  }
}

int heuristic_cfg(int M, int N, int K, long batch, int es, bool tensor, bool skinny) {
  if (es == 4 && tensor && skinny) return 8;
  if (es == 4 && tensor && M >= 64 && N >= 32) return (M >= 768 && N >= 768 && K >= 2048) ? 7 : 6;
  if (M <= 32 && N <= 32) return 2;
  if (M >= 96 && N >= 96) return es == 4 ? (tensor ? 6 : 4) : 3;
  if (M >= 128 && N <= 64) return 1;
  return 0;
}

int split_for(int cfg, int M, int N, int K, long batch) {
  long tiles = batch * ((M + kCfg[cfg].bm - 1) / kCfg[cfg].bm) * ((N + kCfg[cfg].bn - 1) / kCfg[cfg].bn);
  if (tiles >= 2 * 152 || K < 512) return 1;
  long want = (4 * 152 + tiles - 1) / tiles;
  long maxs = K / 256;
  return (int)std::max(1L, std::min({want, maxs, 64L}));
}

std::mutex g_tune_mu;
std::vector<std::pair<unsigned long long, int>> g_tuned;
bool g_tune_loaded = false;

// ACR_TUNE_CACHE=<file>: the choices are read from the file at the first
// tuned product and every new choice is appended to it (one "key choice" line
// each), so a later process -- a profiler run of the same command, say --
// skips the timing.  Called with g_tune_mu held.
void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("ACR_TUNE_CACHE");
  if (!path || !path[0]) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  unsigned long long key;
  int choice;
  while (std::fscanf(f, "%llx %d", &key, &choice) == 2)
    if (choice >= 0 && choice < 2 * kNCfg) g_tuned.push_back({key, choice});
  std::fclose(f);
}

void tune_cache_append(unsigned long long key, int choice) {
  const char* path = std::getenv("ACR_TUNE_CACHE");
  if (!path || !path[0]) return;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "%llx %d\n", key, choice);
    std::fclose(f);
  }
}

// Tuning cache key: element size, tensor-core permission and the log2 classes
// of the shape (a handle that forbids the tensor cores never reuses a choice
// made by one that allows them).
// M, N and K fall in half-octave classes (v in [2^b, 1.5 * 2^b) or [1.5 * 2^b, 2^(b+1))), the batch
// in octaves; the operand layouts (which stride is 1) and whether the one-warp-per-slab tiling
// applies (M <= 32, which a class can straddle) are part of the key.
unsigned long long shape_key(int es, bool tensor, int M, int N, int K, long batch, int layout) {
  auto lg = [](long v) { int b = 0; while (v > 1) { v >>= 1; ++b; } return (unsigned long long)b; };
  auto lh = [&](long v) {
    const unsigned long long b = lg(v);
    return 2 * b + ((b >= 1 && v >= (3L << (b - 1))) ? 1 : 0);
  };
  return (unsigned long long)es | (lh(M) << 8) | (lh(N) << 16) | (lh(K) << 24) | (lg(batch) << 32) |
         ((unsigned long long)(tensor ? 1 : 0) << 48) | ((unsigned long long)layout << 49);
}

}  // namespace

template <class T>
static void run_gemm(Ctx& c, int cfg, int split, int M, int N, int K, long batch, GArgs<T> g) {
  const Cfg& f = kCfg[cfg];
  const KClass cls = (cfg == 6 && sizeof(T) == 4) ? KC_GEMM_TC : KC_GEMM;
  int tiles = ((M + f.bm - 1) / f.bm) * ((N + f.bn - 1) / f.bn);
  if (split > 1) {
    int kchunk = (K + split - 1) / split;
    kchunk = (kchunk + f.bk - 1) / f.bk * f.bk;
    split = (K + kchunk - 1) / kchunk;
    size_t pn = (size_t)split * batch * M * N;
    T* part = c.alloc<T>(pn);
    g.kchunk = kchunk;
    g.partial = part;
    const double es = sizeof(T);
    if (cfg == 7) {
      if constexpr (sizeof(T) == 4) gemm_tma(c, g, batch, split, c.d_flag + 2);
    } else {
      c.kbegin();
      launch_cfg<T>(cfg, dim3((unsigned)batch, tiles, split), g, c.st, c.d_flag + 2);
      c.kend(cls, (g.sym ? 1.0 * M * (N + 1) : 2.0 * M * N) * K * batch, es * batch * ((double)M * K + (double)K * N + (double)M * N * split));
    }
    long tot = batch * (long)M * N;
    int nb = (int)std::min<long>((tot + 255) / 256, 152L * 16);
    c.kbegin();
    k_splitk_reduce<T><<<nb, 256, 0, c.st>>>(g, split);
    c.kend(KC_SPLITK, (double)tot * split, es * tot * (split + 1 + (g.beta != T(0))));
    c.free(part, pn);
  } else {
    g.kchunk = K;
    g.partial = nullptr;
    if (cfg == 7) {
      if constexpr (sizeof(T) == 4) gemm_tma(c, g, batch, 1, c.d_flag + 2);
    } else {
      c.kbegin();
      launch_cfg<T>(cfg, dim3((unsigned)batch, tiles, 1), g, c.st, c.d_flag + 2);
      c.kend(cls, (g.sym ? 1.0 * M * (N + 1) : 2.0 * M * N) * K * batch,
             (double)sizeof(T) * batch * ((double)M * K + (double)K * N + (double)M * N * (1 + (g.beta != T(0)))));
    }
  }
}

// Debug check (ACR_GEMM_VERIFY=1): the chosen tiling and the reference FMA
// tiling (0) both compute alpha A B into scratch; the largest difference (upper
// triangle only for symmetric products) is compared with the reference's
// magnitude, and non-finite values the reference does not have are reported.
template <class T>
__global__ void k_cmp_max(const T* __restrict__ x, const T* __restrict__ y, long tot, int M, int N, int sym,
                          unsigned* out) {
  float md = 0.f, mr = 0.f;
  int bad = 0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const long r = e % ((long)M * N);
    if (sym && r / N > r % N) continue;
    const T a = x[e], b = y[e];
    if (!isfinite((double)a) && isfinite((double)b)) bad = 1;
    md = fmaxf(md, (float)fabs((double)a - (double)b));
    mr = fmaxf(mr, (float)fabs((double)b));
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(md));
    atomicMax(out + 1, __float_as_uint(mr));
    if (bad) atomicOr(out + 2, 1u);
  }
}

template <class T>
static void verify_choice(Ctx& c, int cfg, int split, int M, int N, int K, long batch, const GArgs<T>& g) {
  static std::atomic<int> reported{0};
  const size_t cn = (size_t)batch * M * N;
  T* s1 = c.alloc<T>(cn);
  T* s2 = c.alloc<T>(cn);
  unsigned* d = c.alloc<unsigned>(4);
  GArgs<T> gt = g;
  gt.beta = T(0);
  gt.C.rs = N; gt.C.cs = 1; gt.C.ps = (long)g.nclus * M * N; gt.C.c1 = (long)M * N;
  gt.C.c2 = 0; gt.C.sh = 0; gt.C.sib = 0;
  gt.C.p = s1;
  run_gemm<T>(c, cfg, split, M, N, K, batch, gt);
  gt.C.p = s2;
  run_gemm<T>(c, 0, 1, M, N, K, batch, gt);
  ACR_CUDA(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), c.st));
  k_cmp_max<T><<<(int)std::min<size_t>((cn + 255) / 256, 152 * 16), 256, 0, c.st>>>(s1, s2, (long)cn, M, N,
                                                                                     g.sym ? 1 : 0, d);
  unsigned h[4];
  ACR_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c.st));
  ACR_CUDA(cudaStreamSynchronize(c.st));
  float md, mr;
  std::memcpy(&md, &h[0], 4);
  std::memcpy(&mr, &h[1], 4);
  const float rt = sizeof(T) == 4 ? 1e-3f : 1e-9f;
  if ((h[2] || !(md <= rt * mr)) && reported.fetch_add(1) < 200) {
    std::fprintf(stderr, "acr gemm verify MISMATCH %s M%d N%d K%d b%ld cfg %d split %d sym %d: max diff %g, max ref %g%s\n",
                 c.tag, M, N, K, batch, cfg, split, g.sym, md, mr, h[2] ? ", non-finite values" : "");
  }
  c.free(d, 4);
  c.free(s2, cn);
  c.free(s1, cn);
}

// Host check of the element range an operand touches over all batch entries.
template <class T>
static void check_op(const Ctx& c, const Op<T>& o, int nplanes, int nclus, int rows, int cols, const char* what) {
  if (rows <= 0 || cols <= 0) return;
  long lo = 0, hi = 0;
  bool first = true;
  int cs[4] = {0, 1, nclus - 2, nclus - 1};
  for (int pp : {0, nplanes - 1})
    for (int ci : cs) {
      if (ci < 0 || ci >= nclus) continue;
      int cc = o.sib ? (ci ^ 1) : ci;
      long off = (long)pp * o.ps + (long)(cc >> o.sh) * o.c1 + (long)(cc & 1) * o.c2;
      long top = off + (long)(rows - 1) * o.rs + (long)(cols - 1) * o.cs;
      long bot = off + std::min(0L, (long)(rows - 1) * o.rs) + std::min(0L, (long)(cols - 1) * o.cs);
      if (first || bot < lo) lo = bot;
      if (first || top > hi) hi = top;
      first = false;
    }
  c.check_range(o.p, lo, hi, sizeof(T), what);
}

template <class T>
static void gemm_impl(Ctx& c, int M, int N, int K, int nplanes, int nclus, T alpha, Op<T> A, Op<T> B, T beta, Op<T> C,
                      int sym) {
  long batch = (long)nplanes * nclus;
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (c.check_bounds) {
    if (K > 0) {
      check_op(c, A, nplanes, nclus, M, K, "gemm A");
      check_op(c, B, nplanes, nclus, K, N, "gemm B");
    }
    check_op(c, C, nplanes, nclus, M, N, "gemm C");
  }
  if (K <= 0) {
    // Empty inner dimension: C = beta * C.
    GArgs<T> g{M, N, 0, nclus, (int)batch, T(0), beta, A, B, C, 0, nullptr, 0};
    long tot = batch * (long)M * N;
    int nb = (int)std::min<long>((tot + 255) / 256, 152L * 16);
    c.kbegin();
    k_scale_c<T><<<nb, 256, 0, c.st>>>(g);
    c.kend(KC_COPY, 0, 2.0 * sizeof(T) * tot, "copy:scale_c");
    return;
  }
  if (batch > 0x7fffffffL) throw AcrError(1, "gemm batch too large");
  c.gemm_flops += (sym ? 1LL * M * (N + 1) : 2LL * M * N) * K * batch;
  GArgs<T> g{M, N, K, nclus, (int)batch, alpha, beta, A, B, C, K, nullptr, sym};
  const bool skinny = M <= 32 && B.cs == 1 && C.cs == 1;
  int cfg = heuristic_cfg(M, N, K, batch, (int)sizeof(T), c.tensor, skinny);
  int split = split_for(cfg, M, N, K, batch);
  if (c.force_cfg >= 0 && c.force_cfg < kNCfg && cfg_valid(c.force_cfg, (int)sizeof(T), c.tensor, skinny) &&
      grid_ok(c.force_cfg, M, N)) {
    cfg = c.force_cfg;
    split = split_for(cfg, M, N, K, batch);
  } else if (c.autotune) {
    const int layout =
        (A.cs == 1 ? 1 : 0) | (B.cs == 1 ? 2 : 0) | (C.cs == 1 ? 4 : 0) | (sym ? 8 : 0) | (skinny ? 16 : 0);
    unsigned long long key = shape_key(sizeof(T), c.tensor, M, N, K, batch, layout);
    int found = -1;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_cache_load();
      for (auto& kv : g_tuned)
        if (kv.first == key) { found = kv.second; break; }
    }
    if (found < 0) {
      // Time every candidate writing into a scratch C (beta = 0), keep the fastest.
      size_t cn = (size_t)batch * M * N;
      T* cs = c.alloc<T>(cn);
      GArgs<T> gt = g;
      gt.beta = T(0);
      gt.C.p = cs; gt.C.rs = N; gt.C.cs = 1; gt.C.ps = (long)nclus * M * N; gt.C.c1 = (long)M * N;
      gt.C.c2 = 0; gt.C.sh = 0; gt.C.sib = 0;
      cudaEvent_t e0, e1;
      ACR_CUDA(cudaEventCreate(&e0));
      ACR_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      int bestc = 0;
      for (int cand = 0; cand < 2 * kNCfg; ++cand) {
        int cf = cand % kNCfg;
        if (!cfg_valid(cf, (int)sizeof(T), c.tensor, skinny) || !grid_ok(cf, M, N)) continue;
        int sp = (cand / kNCfg) ? split_for(cf, M, N, K, batch) : 1;
        if ((cand / kNCfg) && sp == 1) continue;
        run_gemm<T>(c, cf, sp, M, N, K, batch, gt);  // warm
        ACR_CUDA(cudaEventRecord(e0, c.st));
        run_gemm<T>(c, cf, sp, M, N, K, batch, gt);
        ACR_CUDA(cudaEventRecord(e1, c.st));
        ACR_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        ACR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; bestc = cand; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      c.free(cs, cn);
      found = bestc;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned.push_back({key, found});
      tune_cache_append(key, found);
    }
    // a class shares one choice; it is valid for every member (the key holds the layouts and skinny)
    if (cfg_valid(found % kNCfg, (int)sizeof(T), c.tensor, skinny) && grid_ok(found % kNCfg, M, N)) {
      cfg = found % kNCfg;
      split = (found / kNCfg) ? split_for(cfg, M, N, K, batch) : 1;
    }
  }
  if (c.profile && c.site_detail) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%s M%d N%d K%d b%ld c%d s%d", c.tag, M, N, K, batch, cfg, split);
    c.tag = c.tagstore.insert(buf).first->c_str();
  }
  if (c.verify_gemm && cfg != 0) verify_choice<T>(c, cfg, split, M, N, K, batch, g);
  run_gemm<T>(c, cfg, split, M, N, K, batch, g);
  if (sym == 1) {
    long tot = batch * (long)M * N;
    int nb = (int)std::min<long>((tot + 255) / 256, 152L * 16);
    c.kbegin();
    k_mirror<T><<<nb, 256, 0, c.st>>>(g);
    c.kend(KC_COPY, 0, (double)sizeof(T) * tot, "copy:mirror");
  }
}

template <class T>
void gemm(Ctx& c, int M, int N, int K, int nplanes, int nclus, T alpha, Op<T> A, Op<T> B, T beta, Op<T> C) {
  gemm_impl<T>(c, M, N, K, nplanes, nclus, alpha, A, B, beta, C, 0);
}

template <class T>
void gemm_sym(Ctx& c, int M, int K, int nplanes, int nclus, T alpha, Op<T> A, Op<T> B, T beta, Op<T> C, bool mirror) {
  gemm_impl<T>(c, M, M, K, nplanes, nclus, alpha, A, B, beta, C, mirror ? 1 : 2);
}

// ---- fused multi-level expansion of a HODLR x panel product -------------------
// Y[rows of leaf] = alpha * ( leaf * W[rows]  +  sum_l U_l[rows] * C_l[sibling of the
// row's level-(l+1) cluster] ) + beta * Y[rows], where level l only reaches the
// first ncol_l columns:  the leaf product and every
// level's expansion in one pass over an inner dimension b + sum_l K_l, so Y is
// read and written once.  One CTA per (plane, leaf, 64 output columns).
template <class T>
__global__ void __launch_bounds__(256) k_hexpand(HexpArgs<T> a) {
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int nleaf = a.m / a.b;
  const int plane = blockIdx.x / nleaf, lf = blockIdx.x % nleaf;
  const int n0 = blockIdx.y * BN;
  const int row0 = lf * a.b;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  // segment -1: leaf; segments 0..nl-1: levels
  for (int sg = -1; sg < a.nl; ++sg) {
    const T* Ap;
    long ars, acs;
    const T* Bp;
    long brs;
    int K, nlim = a.w;
    if (sg < 0) {
      const T* lfp = a.leaf + plane * a.lps + (long)lf * a.b * a.b;
      Ap = lfp;
      ars = a.leaf_trans ? 1 : a.b;
      acs = a.leaf_trans ? a.b : 1;
      Bp = a.W + plane * a.wps + (long)row0 * a.wld;
      brs = a.wld;
      K = a.b;
    } else {
      K = a.K[sg];
      nlim = a.ncol[sg];
      if (n0 >= nlim) continue;  // uniform over the CTA
      const int s = a.s[sg];
      const int c = row0 / s;
      Ap = a.U[sg] + plane * a.ups[sg] + (long)row0 * K;
      ars = K;
      acs = 1;
      Bp = a.C[sg] + ((long)plane * a.nclus[sg] + (c ^ 1)) * (long)K * nlim;
      brs = nlim;
    }
    for (int k0 = 0; k0 < K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        int ii, kk;
        if (acs == 1) { ii = e / BK; kk = e % BK; } else { ii = e % BM; kk = e / BM; }
        int gk = k0 + kk;
        As[kk][ii] = (ii < a.b && gk < K) ? Ap[(long)ii * ars + (long)gk * acs] : T(0);
      }
      for (int e = tid; e < BK * BN; e += 256) {
        int kk = e / BN, jj = e % BN;
        int gk = k0 + kk, gj = n0 + jj;
        Bs[kk][jj] = (gk < K && gj < nlim) ? Bp[(long)gk * brs + gj] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  T* Yp = a.Y + plane * a.yps + (long)row0 * a.yld;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int r = ty * TM + i;
    if (r >= a.b) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int cj = n0 + tx * TN + j;
      if (cj >= a.w) continue;
      T* yp = Yp + (long)r * a.yld + cj;
      T v = a.alpha * acc[i][j];
      if (a.beta != T(0)) v += a.beta * *yp;
      *yp = v;
    }
  }
}

// ---- the fused expansion on the tcgen05 tensor cores (FP32 as 3xTF32) --------
// One CTA per (plane, pair of 64-row leaves 2t, 2t+1, 128 output columns): the
// 128 rows are one MMA tile.  The inner dimension is a list of segments, each
// starting on a 32-deep slice:
//   0: the two leaf blocks, block diagonal (K = 128), times the stacked W rows;
//   1: a level whose cluster holds both leaves (K = K_l): U_l rows times the
//      coefficients of the sibling cluster;
//   2: the last level, where the two leaves are siblings (K = 2 K_l):
//      [U(2t) 0; 0 U(2t+1)] times [C(2t+1); C(2t)].
// Loads, TF32 split, staging, MMA issue and epilogue follow k_gemm_tc05; the
// MMA N is the tile's column count rounded up to 16.
struct HexpSeg {
  int nseg = 0, nslice = 0;
  int type[MAXL + 1] = {}, lvl[MAXL + 1] = {}, slice0[MAXL + 1] = {};
};

__global__ void __launch_bounds__(tc::NT, 1) k_hexpand_tc(HexpArgs<float> a, HexpSeg sg, int* err) {
  constexpr int QT = (tc::BM * tc::BK / 4) / tc::NT;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t bars[tc::NSTAGE];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npair = a.m / 128;
  const int plane = blockIdx.x / npair, pr = blockIdx.x % npair;
  const int R0 = pr * 128;
  const int n0 = blockIdx.y * tc::BN;
  const int ncols = min(tc::BN, a.w - n0);
  const int nmma = (ncols + 15) / 16 * 16;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) |
                         ((uint32_t)(tc::BM >> 4) << 24);
  const int nk = sg.nslice;
  const uint32_t raw_s = smem_u32(tc_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;
  unsigned char* base = tc_raw + (base_s - raw_s);
  if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), tc::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < tc::NSTAGE; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const float* Wp = a.W + plane * a.wps;
  float ra0[QT][4], rb0[QT][4], ra1[QT][4], rb1[QT][4];
  // A: row i = e >> 3, quad q = e & 7 (k contiguous); B^T: column j = e & 127, quad e >> 7.
  auto load = [&](int kc, float (&ra)[QT][4], float (&rb)[QT][4]) {
    int si = 0;
    while (si + 1 < sg.nseg && kc >= sg.slice0[si + 1]) ++si;
    const int ty = sg.type[si], li = sg.lvl[si];
    const int k0 = (kc - sg.slice0[si]) * tc::BK;
    const int K = ty == 0 ? 64 : a.K[li];
    const int nc = ty == 0 ? a.w : a.ncol[li];
    const float* U = ty == 0 ? nullptr : a.U[li] + plane * a.ups[li];
#pragma unroll
    for (int it = 0; it < QT; ++it) {
      const int e = tid + tc::NT * it;
      const int i = e >> 3, q = e & 7, half = i >> 6;
      const int j = e & 127, qb = e >> 7, gj = n0 + j;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int k = k0 + 4 * q + jj;
        float va = 0.f;
        if (ty == 0) {
          if ((k >> 6) == half && k < 128) {
            const float* Lf = a.leaf + plane * a.lps + (long)(2 * pr + half) * 4096;
            const int ii = i & 63, kl = k & 63;
            va = a.leaf_trans ? Lf[kl * 64 + ii] : Lf[ii * 64 + kl];
          }
        } else if (ty == 1) {
          if (k < K) va = U[(long)(R0 + i) * K + k];
        } else {
          const int kk = k - half * K;
          if (kk >= 0 && kk < K) va = U[(long)(R0 + i) * K + kk];
        }
        ra[it][jj] = va;
        const int kb = k0 + 4 * qb + jj;
        float vb = 0.f;
        if (gj < nc) {
          if (ty == 0) {
            if (kb < 128) vb = Wp[(long)(R0 + kb) * a.wld + gj];
          } else if (ty == 1) {
            if (kb < K) {
              const int cl = R0 / a.s[li];
              vb = a.C[li][(((long)plane * a.nclus[li] + (cl ^ 1)) * K + kb) * nc + gj];
            }
          } else if (kb < 2 * K) {
            const int leafc = R0 / 64 + (kb < K ? 1 : 0);
            const int kk = kb < K ? kb : kb - K;
            vb = a.C[li][(((long)plane * a.nclus[li] + leafc) * K + kk) * nc + gj];
          }
        }
        rb[it][jj] = vb;
      }
    }
  };
  auto split4 = [](const float (&x)[4], float4& h, float4& l) {
    h.x = tf32_hi(x[0]); l.x = tf32_hi(x[0] - h.x);
    h.y = tf32_hi(x[1]); l.y = tf32_hi(x[1] - h.y);
    h.z = tf32_hi(x[2]); l.z = tf32_hi(x[2] - h.z);
    h.w = tf32_hi(x[3]); l.w = tf32_hi(x[3] - h.w);
  };
  auto store = [&](int s, const float (&ra)[QT][4], const float (&rb)[QT][4]) {
    unsigned char* st = base + s * tc::STAGE_BYTES;
#pragma unroll
    for (int it = 0; it < QT; ++it) {
      const int e = tid + tc::NT * it;
      const int i = e >> 3, q = e & 7, j = e & 127, qb = e >> 7;
      const uint32_t oa = i * 128 + ((q ^ (i & 7)) << 4), ob = j * 128 + ((qb ^ (j & 7)) << 4);
      float4 h, l;
      split4(ra[it], h, l);
      *reinterpret_cast<float4*>(st + oa) = h;
      *reinterpret_cast<float4*>(st + tc::TILE_BYTES + oa) = l;
      split4(rb[it], h, l);
      *reinterpret_cast<float4*>(st + 2 * tc::TILE_BYTES + ob) = h;
      *reinterpret_cast<float4*>(st + 3 * tc::TILE_BYTES + ob) = l;
    }
  };
  auto issue = [&](int kc, int s) {
    tc_fence_after();
    const uint32_t sa = base_s + s * tc::STAGE_BYTES;
#pragma unroll
    for (int kk = 0; kk < tc::BK / 8; ++kk) {
      const uint64_t ah = umma_desc_sw128(sa + kk * 32), al = umma_desc_sw128(sa + tc::TILE_BYTES + kk * 32);
      const uint64_t bh = umma_desc_sw128(sa + 2 * tc::TILE_BYTES + kk * 32),
                     bl = umma_desc_sw128(sa + 3 * tc::TILE_BYTES + kk * 32);
      umma_tf32(tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
      umma_tf32(tmem, ah, bl, idesc, 1u);
      umma_tf32(tmem, al, bh, idesc, 1u);
    }
    umma_commit(smem_u32(&bars[s]));
  };
  auto step = [&](int kc, float (&ra)[QT][4], float (&rb)[QT][4]) -> bool {
    const int s = kc % tc::NSTAGE;
    bool ok = true;
    if (kc >= tc::NSTAGE) ok = mbar_wait_bounded(smem_u32(&bars[s]), ((kc - tc::NSTAGE) / tc::NSTAGE) & 1);
    if (ok) store(s, ra, rb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) return false;
    if (kc + 2 < nk) load(kc + 2, ra, rb);
    if (tid == 0) issue(kc, s);
    return true;
  };
  bool ok = true;
  if (nk > 0) load(0, ra0, rb0);
  if (nk > 1) load(1, ra1, rb1);
  for (int kc = 0; kc < nk && ok; kc += 2) {
    ok = step(kc, ra0, rb0);
    if (ok && kc + 1 < nk) ok = step(kc + 1, ra1, rb1);
  }
  if (ok && nk > 0) ok = mbar_wait_bounded(smem_u32(&bars[(nk - 1) % tc::NSTAGE]), ((nk - 1) / tc::NSTAGE) & 1);
  if (!__syncthreads_and(ok)) s_ok = 0;
  __syncthreads();
  tc_fence_after();
  if (s_ok) {
    GArgs<float> g{};
    g.M = a.m; g.N = a.w; g.alpha = a.alpha; g.beta = a.beta;
    g.C = Op<float>{a.Y, a.yld, 1, a.yps, 0, 0, 0, 0};
    g.partial = nullptr;
    constexpr int CW = tc::BN / (tc::NT / 128);
    const int lb = (warp & 3) * 32, cb = (warp >> 2) * CW;
    float* stg = reinterpret_cast<float*>(base) + warp * 32 * 17;
#pragma unroll 1
    for (int ch = 0; ch < CW / 16; ++ch) {
      if (cb + ch * 16 >= nmma) break;  // uniform over the warp
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)(cb + ch * 16), r);
      store_chunk(g, stg, r, lane, R0 + lb, n0 + cb + ch * 16, plane, 0, 0);
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tc::TMEM_COLS);
}

template <class T>
void hexpand(Ctx& c, const HexpArgs<T>& a, int P) {
  if (P <= 0 || a.w <= 0) return;
  if (a.b > 64) throw AcrError(1, "fused expansion supports leaves of at most 64 rows");
  dim3 grid((unsigned)((long)P * (a.m / a.b)), (a.w + 63) / 64);
  double fl = 2.0 * a.b, by = 0;  // per output element
  for (int l = 0; l < a.nl; ++l) fl += 2.0 * a.K[l] * ((double)a.ncol[l] / a.w);
  fl *= (double)P * a.m * a.w;
  by = (double)sizeof(T) * P * a.m * (a.b + 2.0 * a.w);
  for (int l = 0; l < a.nl; ++l) by += (double)sizeof(T) * P * a.m * a.K[l];
  c.kbegin();
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (c.tensor && a.b == 64 && a.m % 128 == 0 && a.w > 64) {  // narrow panels (solve sweeps) stay on the FMA tiles
      HexpSeg sg;
      sg.type[0] = 0;
      sg.lvl[0] = 0;
      sg.slice0[0] = 0;
      int sl = 128 / tc::BK;
      sg.nseg = 1;
      for (int l = 0; l < a.nl; ++l) {
        const int ty = (a.s[l] == a.b) ? 2 : 1;
        const int kext = ty == 2 ? 2 * a.K[l] : a.K[l];
        sg.type[sg.nseg] = ty;
        sg.lvl[sg.nseg] = l;
        sg.slice0[sg.nseg] = sl;
        ++sg.nseg;
        sl += (kext + tc::BK - 1) / tc::BK;
      }
      sg.nslice = sl;
      ACR_CUDA(cudaFuncSetAttribute(k_hexpand_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
      dim3 g2((unsigned)((long)P * (a.m / 128)), (a.w + tc::BN - 1) / tc::BN);
      k_hexpand_tc<<<g2, tc::NT, tc::SMEM_BYTES, c.st>>>(a, sg, c.d_flag + 2);
      done = true;
    }
  }
  if (!done) k_hexpand<T><<<grid, 256, 0, c.st>>>(a);
  c.kend(KC_HEXPAND, fl, by);
  c.gemm_flops += (long long)fl;
}
template void hexpand<float>(Ctx&, const HexpArgs<float>&, int);
template void hexpand<double>(Ctx&, const HexpArgs<double>&, int);

template void gemm_sym<float>(Ctx&, int, int, int, int, float, Op<float>, Op<float>, float, Op<float>, bool);
template void gemm_sym<double>(Ctx&, int, int, int, int, double, Op<double>, Op<double>, double, Op<double>, bool);
template void gemm<float>(Ctx&, int, int, int, int, int, float, Op<float>, Op<float>, float, Op<float>);
template void gemm<double>(Ctx&, int, int, int, int, int, double, Op<double>, Op<double>, double,
                           Op<double>);

}  // namespace acr
