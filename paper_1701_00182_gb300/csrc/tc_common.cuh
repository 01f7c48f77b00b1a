// Shared pieces of the batched GEMM kernels: the argument block, operand
// addressing, and the tcgen05 / mbarrier building blocks (inline PTX) used by
// the tensor-core tilings.
#pragma once
#include <cstdint>

#include "acr_internal.h"

namespace acr {

template <class T>
struct GArgs {
  int M, N, K, nclus, batch;
  T alpha, beta;
  Op<T> A, B, C;
  int kchunk;
  T* partial;
  int sym;  // C is symmetric (A = B^T): only tiles touching the upper triangle are computed (2: no mirror pass)
};

template <class T>
__device__ __forceinline__ T* opaddr(const Op<T>& o, int plane, int c) {
  int cc = o.sib ? (c ^ 1) : c;
  return o.p + (long)plane * o.ps + (long)(cc >> o.sh) * o.c1 + (long)(cc & 1) * o.c2;
}

// FP32 GEMM with pre-split TF32 operand tiles fed by TMA (tma_gemm.cu).
void gemm_tma(Ctx& c, const GArgs<float>& g, long batch, int split, int* err);

// CUDA-core tilings for small batched products (gemm_small.cu): kind 0 = one
// warp per column slab (M <= 32, B and C row-major; grid computed inside),
// 1/2/3 = 64x64 / 64x128 / 128x64 tiles on the grid (batch, tiles, split).
template <class T>
void launch_gemm_small(int kind, const GArgs<T>& g, dim3 grid, long batch, int split, cudaStream_t st);

// Every mbarrier wait inside a kernel gives up after this long (ns).
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor: start address, leading byte offset 16 (not
// used by a swizzled K-major operand), stride byte offset 1024 (next 8-row
// atom), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = global_ns();
    else if ((it & 31) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// One arrival that also announces `bytes` of asynchronous copies completing on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

// TMA: the box at (x, y) of a 2D tensor map into shared memory, completion
// (bytes) signalled on the barrier.  x must be a multiple of 16 bytes / element.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TF32 high part rounded to nearest (ties away from zero: add half an ulp of
// bit 13 to the magnitude, clear the low 13 bits) and the rounded remainder.
__device__ __forceinline__ float tf32_hi(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// Epilogue of the tensor-core tiles: one 32-row x 16-column chunk of the
// accumulator, held one row per lane (r[j] = column j), goes through a per-warp
// shared-memory transpose (stg: 32 x 17 floats) so that each store
// instruction writes two 64-byte row segments instead of 32 scattered words.
// Rows row0.., columns col0.. of batch entry bi; split-K partials or
// C = alpha acc + beta C.
__device__ __forceinline__ void store_chunk(const GArgs<float>& g, float* stg, const uint32_t (&r)[16], int lane,
                                            int row0, int col0, int plane, int c, long bi) {
#pragma unroll
  for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = __uint_as_float(r[j]);
  __syncwarp();
  const bool part = g.partial != nullptr;
  float* Cb = part ? g.partial + ((long)blockIdx.z * g.batch + bi) * (long)g.M * g.N : opaddr(g.C, plane, c);
  const long crs = part ? (long)g.N : g.C.rs, ccs = part ? 1L : g.C.cs;
  const int jj = lane & 15;
#pragma unroll 4
  for (int it = 0; it < 16; ++it) {
    const int rr = 2 * it + (lane >> 4);
    const int gi = row0 + rr, gj = col0 + jj;
    if (gi < g.M && gj < g.N) {
      float* cp = Cb + (long)gi * crs + (long)gj * ccs;
      float v = stg[rr * 17 + jj];
      if (!part) {
        v *= g.alpha;
        if (g.beta != 0.f) v += g.beta * *cp;
      }
      *cp = v;
    }
  }
  __syncwarp();
}

}  // namespace acr
