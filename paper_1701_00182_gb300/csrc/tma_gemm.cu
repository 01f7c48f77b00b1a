// FP32 GEMM as 3xTF32 on the tcgen05 tensor cores with TMA-fed operands.
//
// Operands of the H-arithmetic are panels whose row strides are block ranks,
// so they cannot be read by the tensor memory accelerator directly (its global
// strides must be 16-byte multiples).  A memory-bound pre-pass therefore
// rewrites each operand once per call, for every (batch entry, 128-row tile,
// 32-deep K slice), as two dense 128 x 32 row-major tiles: the TF32 high part
// and the rounded remainder (16 KB each, tiles contiguous).  The GEMM kernel
// then streams those tiles with cp.async.bulk.tensor (128-byte swizzle, the
// layout the tensor core reads) into a three-stage shared-memory ring under a
// warp-specialised mbarrier pipeline:
//   thread 0   : producer, waits for a free stage and issues the four TMA loads
//                (A_hi, A_lo, B_hi, B_lo) that complete the stage's full barrier;
//   thread 32  : issues A_hi B_hi + A_hi B_lo + A_lo B_hi as 12 tcgen05.mma
//                (128 x 128 x 8) per stage and commits them to its empty barrier;
//   all 4 warps: after the last commit, read the 128 x 128 FP32 accumulator from
//                tensor memory (tcgen05.ld) and apply alpha / beta.
// A symmetric product (A = B^T) splits one operand and uses it for both.
// Every wait is bounded in time; on expiry a device flag is set, outstanding
// copies are waited for (bounded), the epilogue is skipped and TMEM is freed.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is fetched at run time)

#include <algorithm>
#include <mutex>

#include "acr_internal.h"
#include "tc_common.cuh"

namespace acr {

namespace tg {
constexpr int BM = 128, BN = 128, BK = 32;
constexpr int TILE_FLOATS = BM * BK;  // one 128 x 32 tile (16 KB)
constexpr int TILE_BYTES = TILE_FLOATS * 4;
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A_hi, A_lo, B_hi, B_lo
constexpr int NSTAGE = 3;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;  // + slack for the 1 KB alignment
constexpr int NT = 128;
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}  // namespace tg

// Pre-split of one operand X(row, k) (row < R, k < K) of batch entries
// b0 .. b0 + gridDim.x - 1: tile (entry, rt, ks) -> out[((lb * rtiles + rt) *
// ksl + ks) * 2 + {0: high, 1: remainder}], each 128 x 32 row major, zero
// outside the operand.
__global__ void __launch_bounds__(256) k_tf32_split(Op<float> X, int R, int K, int nclus, long b0, int rtiles,
                                                    int ksl, float* __restrict__ out) {
  __shared__ float t[128][33];
  const long lb = blockIdx.x, bi = b0 + lb;
  const int plane = (int)(bi / nclus), c = (int)(bi - (long)plane * nclus);
  const int rt = blockIdx.y, ks = blockIdx.z;
  const float* S = opaddr(X, plane, c);
  const long rs = X.rs, cs = X.cs;
  const int r0 = rt * 128, k0 = ks * 32, tid = threadIdx.x;
  if (cs == 1) {  // lanes along k
    for (int e = tid; e < 128 * 32; e += 256) {
      const int row = e >> 5, k = e & 31;
      t[row][k] = (r0 + row < R && k0 + k < K) ? S[(long)(r0 + row) * rs + (k0 + k)] : 0.f;
    }
  } else {  // lanes along rows
    for (int e = tid; e < 128 * 32; e += 256) {
      const int row = e & 127, k = e >> 7;
      t[row][k] = (r0 + row < R && k0 + k < K) ? S[(long)(r0 + row) * rs + (long)(k0 + k) * cs] : 0.f;
    }
  }
  __syncthreads();
  float* o = out + (((lb * rtiles + rt) * (long)ksl + ks) * 2) * tg::TILE_FLOATS;
  for (int e = tid; e < 1024; e += 256) {
    const int row = e >> 3, q = e & 7;
    float4 h, l;
    const float* v = &t[row][4 * q];
    h.x = tf32_hi(v[0]); l.x = tf32_hi(v[0] - h.x);
    h.y = tf32_hi(v[1]); l.y = tf32_hi(v[1] - h.y);
    h.z = tf32_hi(v[2]); l.z = tf32_hi(v[2] - h.z);
    h.w = tf32_hi(v[3]); l.w = tf32_hi(v[3] - h.w);
    *reinterpret_cast<float4*>(o + row * 32 + 4 * q) = h;
    *reinterpret_cast<float4*>(o + tg::TILE_FLOATS + row * 32 + 4 * q) = l;
  }
}

__global__ void __launch_bounds__(tg::NT, 1) k_gemm_tma(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB, GArgs<float> g,
                                                        long b0, int mtA, int ntB, int ksl, int* err) {
  extern __shared__ unsigned char tg_raw[];
  __shared__ __align__(8) uint64_t full[tg::NSTAGE], empty[tg::NSTAGE], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long lb = blockIdx.x, bi = b0 + lb;
  const int plane = (int)(bi / g.nclus), c = (int)(bi - (long)plane * g.nclus);
  const int tilesN = (g.N + tg::BN - 1) / tg::BN;
  const int mt = blockIdx.y / tilesN, nt = blockIdx.y % tilesN;
  const int m0 = mt * tg::BM, n0 = nt * tg::BN;
  if (g.sym && m0 >= n0 + tg::BN) return;  // tile strictly below the diagonal (uniform)
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const int ks0 = kbeg / tg::BK;
  const int nk = kend > kbeg ? (kend - kbeg + tg::BK - 1) / tg::BK : 0;
  const uint32_t raw_s = smem_u32(tg_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;

  if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), tg::TMEM_COLS);
  if (tid == 32) {
    for (int s = 0; s < tg::NSTAGE; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_err = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (tid == 0 && nk > 0) {
    // producer
    int issued = 0;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % tg::NSTAGE;
      if (kc >= tg::NSTAGE && !mbar_wait_bounded(smem_u32(&empty[s]), ((kc - tg::NSTAGE) / tg::NSTAGE) & 1)) {
        s_err = 1;
        break;
      }
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, tg::STAGE_BYTES);
      const uint32_t sa = base_s + s * tg::STAGE_BYTES;
      const int ya = (int)((((lb * mtA + mt) * (long)ksl + ks0 + kc) * 2) * tg::BM);
      const int yb = (int)((((lb * ntB + nt) * (long)ksl + ks0 + kc) * 2) * tg::BN);
      tma_load_2d(sa, &tmA, 0, ya, fb);
      tma_load_2d(sa + tg::TILE_BYTES, &tmA, 0, ya + tg::BM, fb);
      tma_load_2d(sa + 2 * tg::TILE_BYTES, &tmB, 0, yb, fb);
      tma_load_2d(sa + 3 * tg::TILE_BYTES, &tmB, 0, yb + tg::BN, fb);
      issued = kc + 1;
    }
    // none of this CTA's copies may still be in flight when it exits
    for (int kc = max(0, issued - tg::NSTAGE); kc < issued; ++kc)
      if (!mbar_wait_bounded(smem_u32(&full[kc % tg::NSTAGE]), (kc / tg::NSTAGE) & 1)) s_err = 1;
  } else if (tid == 32 && nk > 0) {
    // MMA issuer
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % tg::NSTAGE;
      if (!mbar_wait_bounded(smem_u32(&full[s]), (kc / tg::NSTAGE) & 1)) {
        s_err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = base_s + s * tg::STAGE_BYTES;
#pragma unroll
      for (int kk = 0; kk < tg::BK / 8; ++kk) {
        const uint64_t ah = umma_desc_sw128(sa + kk * 32), al = umma_desc_sw128(sa + tg::TILE_BYTES + kk * 32);
        const uint64_t bh = umma_desc_sw128(sa + 2 * tg::TILE_BYTES + kk * 32),
                       bl = umma_desc_sw128(sa + 3 * tg::TILE_BYTES + kk * 32);
        umma_tf32(tmem, ah, bh, tg::IDESC, (kc > 0 || kk > 0) ? 1u : 0u);
        umma_tf32(tmem, ah, bl, tg::IDESC, 1u);
        umma_tf32(tmem, al, bh, tg::IDESC, 1u);
      }
      umma_commit(smem_u32(&empty[s]));
    }
    umma_commit(smem_u32(&done));  // arrives once every MMA issued above has completed
  }
  bool ok = true;
  if (nk > 0) ok = mbar_wait_bounded(smem_u32(&done), 0);
  if (!__syncthreads_and(ok)) s_err = 1;
  __syncthreads();
  tc_fence_after();
  if (!s_err) {
    // the stage ring is free now: per-warp transpose buffers for the stores
    float* stg = reinterpret_cast<float*>(tg_raw + (base_s - raw_s)) + warp * 32 * 17;
    const int lbase = warp * 32;
#pragma unroll 1
    for (int ch = 0; ch < tg::BN / 16; ++ch) {
      uint32_t r[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)lbase << 16) + (uint32_t)(ch * 16), r);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      }
      store_chunk(g, stg, r, lane, m0 + lbase, n0 + ch * 16, plane, c, bi);
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tg::TMEM_COLS);
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  if (!fn) throw AcrError(5, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// rows x 32 FP32 row-major tile store, boxes of 128 rows, 128-byte swizzle.
CUtensorMap tile_map(float* base, long rows) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {32, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {32 * sizeof(float)};
  const cuuint32_t box[2] = {32, 128};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = tensor_map_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw AcrError(5, "cuTensorMapEncodeTiled rejected the split-operand layout");
  return m;
}

}  // namespace

// C (+)= alpha A B over `batch` entries (K already split into g.kchunk chunks,
// split > 1 writes g.partial).  Operand tiles are pre-split in chunks of batch
// entries whose tiles fit in about 2 GB.
void gemm_tma(Ctx& c, const GArgs<float>& g, long batch, int split, int* err) {
  const int mtA = (g.M + tg::BM - 1) / tg::BM, ntB = (g.N + tg::BN - 1) / tg::BN, ksl = (g.K + tg::BK - 1) / tg::BK;
  const bool share = g.sym != 0;  // B = A^T: B's tiles are A's
  const double tile2 = 2.0 * tg::TILE_BYTES;
  const double per_entry = tile2 * ksl * (mtA + (share ? 0 : ntB));
  long nb = std::max(1L, (long)(2.0e9 / per_entry));
  nb = std::min(nb, batch);
  const size_t na = (size_t)nb * mtA * ksl * 2 * tg::TILE_FLOATS, nbf = share ? 0 : (size_t)nb * ntB * ksl * 2 * tg::TILE_FLOATS;
  float* Ap = c.alloc<float>(na);
  float* Bp = share ? Ap : c.alloc<float>(nbf);
  const CUtensorMap tA = tile_map(Ap, (long)nb * mtA * ksl * 2 * tg::BM);
  const CUtensorMap tB = share ? tA : tile_map(Bp, (long)nb * ntB * ksl * 2 * tg::BN);
  Op<float> XB = g.B;  // B viewed as rows j, columns k
  XB.rs = g.B.cs;
  XB.cs = g.B.rs;
  ACR_CUDA(cudaFuncSetAttribute(k_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, tg::SMEM_BYTES));
  const int tiles = mtA * ntB;
  for (long b0 = 0; b0 < batch; b0 += nb) {
    const long nbc = std::min(nb, batch - b0);
    c.kbegin();
    k_tf32_split<<<dim3((unsigned)nbc, mtA, ksl), 256, 0, c.st>>>(g.A, g.M, g.K, g.nclus, b0, mtA, ksl, Ap);
    if (!share) k_tf32_split<<<dim3((unsigned)nbc, ntB, ksl), 256, 0, c.st>>>(XB, g.N, g.K, g.nclus, b0, ntB, ksl, Bp);
    c.kend(KC_TF32SPLIT, 0,
           (double)nbc * (4.0 + 8.0) * ((double)mtA * tg::BM * ksl * tg::BK + (share ? 0.0 : (double)ntB * tg::BN * ksl * tg::BK)),
           "tf32_split");
    if (!share) c.launches += 1;
    c.kbegin();
    k_gemm_tma<<<dim3((unsigned)nbc, tiles, split), tg::NT, tg::SMEM_BYTES, c.st>>>(tA, tB, g, b0, mtA,
                                                                                      share ? mtA : ntB, ksl, err);
    c.kend(KC_GEMM_TC, (g.sym ? 1.0 * g.M * (g.N + 1) : 2.0 * g.M * g.N) * g.K * nbc,
           4.0 * nbc * ((double)g.M * g.K + (double)g.K * g.N + (double)g.M * g.N * (split > 1 ? split : 1 + (g.beta != 0.f))));
  }
  if (!share) c.free(Bp, nbf);
  c.free(Ap, na);
}

}  // namespace acr
