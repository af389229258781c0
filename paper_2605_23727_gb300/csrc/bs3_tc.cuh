// Tensor-core (tcgen05) product for ensembles that share one coupling matrix:
//   C[M][Nc] = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// with A = A_hi + A_lo (M x K) and B = B_hi + B_lo (Nc x K) split into
// bfloat16 pairs (about 16 significant bits each), products accumulated in
// binary32 in tensor memory.  One CTA computes a 128 x 256 tile:
//   warp 0: TMA producer (2D tiles, 128-byte swizzle, two-stage ring);
//   warp 1: allocates tensor memory and issues tcgen05.mma (one thread);
//   warps 2 .. 2+EW-1: epilogue, tcgen05.ld of the accumulator rows (warp w
//   reads tensor-memory lanes 32*(w%4) .. +31; EW/4 warps share each lane
//   quarter and split its 32-column chunks).
// Every wait is bounded; a wait that runs out sets *err and the CTA winds down.
// gemm_persistent is the same pipeline over several tiles per CTA, with two
// accumulators in tensor memory (see there).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bs3 {
namespace tc {

constexpr int BM = 128, BK = 64, STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;                  // 16 KB per bf16 operand tile

// Tile of BM x BNT outputs (BNT = 256 or 128 accumulator columns in TMEM).
template <int BNT>
struct Tile {
  static_assert(BNT == 128 || BNT == 256, "tile width");
  static constexpr int BN = BNT;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = BN;
  // instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
  // K-major, N = BN, M = BM
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};

// the plain product's tile
constexpr int BN = 256;
constexpr int B_BYTES = Tile<BN>::B_BYTES;
constexpr int STAGE_BYTES = Tile<BN>::STAGE_BYTES;
constexpr int SMEM_BYTES = Tile<BN>::SMEM_BYTES;
constexpr int THREADS = 192;                      // plain product: four epilogue warps
constexpr int threads_for(int ew) { return 64 + 32 * ew; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(b, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile with 128-byte
// swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart (stride offset),
// descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Epilogue callback contract: store(row, col0, v[32]) for the 32 columns
// col0 .. col0+31 of one output row.
struct StoreRowMajor {
  float* C;
  long long ldc;
  __device__ __forceinline__ void operator()(int row, int col0, const float* v) const {
    float4* p = reinterpret_cast<float4*>(C + (size_t)row * ldc + col0);
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  }
};

template <int EW, int BNT, class Store>
__device__ __forceinline__ void gemm_tile(const CUtensorMap* mAh, const CUtensorMap* mAl, const CUtensorMap* mBh,
                                          const CUtensorMap* mBl, int m0, int n0, int K, const Store& store,
                                          int* err, long long spin) {
  using TL = Tile<BNT>;
  constexpr int BNL = TL::BN, B_BYTESL = TL::B_BYTES, STAGE_BYTESL = TL::STAGE_BYTES, TMEM_COLSL = TL::TMEM_COLS;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTESL);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_abort = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLSL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((kb / STAGES) & 1) ^ 1), spin)) {
        atomicExch(err, 1);
        *(volatile int*)s_abort = 1;
        break;
      }
      if (*(volatile int*)s_abort) break;
      unsigned char* st = base + s * STAGE_BYTESL;
      mbar_expect_tx(&full[s], STAGE_BYTESL);
      tma_load_2d(st, mAh, &full[s], kb * BK, m0);
      tma_load_2d(st + A_BYTES, mAl, &full[s], kb * BK, m0);
      tma_load_2d(st + 2 * A_BYTES, mBh, &full[s], kb * BK, n0);
      tma_load_2d(st + 2 * A_BYTES + B_BYTESL, mBl, &full[s], kb * BK, n0);
      issued = kb + 1;
    }
    // the copies of the last stages must land before the CTA ends
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1), spin);
  } else if (warp == 1 && lane == 0) {
    // --------------------------------------------------------------- MMA
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)((kb / STAGES) & 1), spin)) {
        atomicExch(err, 1);
        *(volatile int*)s_abort = 1;
        break;
      }
      fence_after();
      const unsigned char* st = base + s * STAGE_BYTESL;
      const uint64_t dAh = sw128_desc(smem_u32(st));
      const uint64_t dAl = sw128_desc(smem_u32(st + A_BYTES));
      const uint64_t dBh = sw128_desc(smem_u32(st + 2 * A_BYTES));
      const uint64_t dBl = sw128_desc(smem_u32(st + 2 * A_BYTES + B_BYTESL));
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 bf16 = 32 bytes further along K
        mma_bf16(tmem, dAh + o, dBh + o, TL::IDESC, (kb | kk) != 0);
        mma_bf16(tmem, dAh + o, dBl + o, TL::IDESC, 1);
        mma_bf16(tmem, dAl + o, dBh + o, TL::IDESC, 1);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);   // fires when every MMA issued above has completed
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    static_assert(EW % 4 == 0 && EW >= 4 && EW <= 32, "epilogue warps: a multiple of four");
    const bool ok = mbar_wait(done, 0, spin);
    fence_after();
    if (!ok) atomicExch(err, 1);
    if (ok && !*(volatile int*)s_abort) {
      const int quarter = warp & 3;   // tensor-memory lanes 32*quarter .. 32*quarter+31
      const int sub = (warp - 2) >> 2;   // which of the EW/4 warps of this quarter
      const int row = m0 + quarter * 32 + lane;
#pragma unroll 1
      for (int c = sub; c < BNL / 32; c += EW / 4) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c * 32), v);
        store(row, n0 + c * 32, v);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLSL) : "memory");
  }
}

// Persistent form: CTA b computes the tiles b, b + gridDim.x, b + 2 gridDim.x,
// ... of a tiles_m x tiles_n grid of BM x BNT tiles, numbered row block by row
// block (the column tiles of one row block are consecutive, so the CTAs that
// run together share the A rows in L2).  The operand ring runs on across
// tiles, and tensor memory holds two accumulators: the MMA thread fills one
// while the epilogue warps drain the other, so the epilogue of a tile overlaps
// the products of the next.  Barriers: full/empty (operand ring), acc_full
// (MMA -> epilogue, one commit per tile), acc_empty (epilogue -> MMA, one
// arrival per epilogue warp), mma_done (the last MMAs, before tensor memory
// is released).
template <int BNT>
struct PTile {
  static constexpr int S = BNT == 128 ? 3 : 2;   // ring stages
  static constexpr int SMEM_BYTES = S * Tile<BNT>::STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = 2 * BNT;
};

template <int EW, int BNT, class Store>
__device__ __forceinline__ void gemm_persistent(const CUtensorMap* mAh, const CUtensorMap* mAl,
                                                const CUtensorMap* mBh, const CUtensorMap* mBl, int tiles_m,
                                                int tiles_n, int K, const Store& store, int* err, long long spin) {
  using TL = Tile<BNT>;
  constexpr int S = PTile<BNT>::S;
  constexpr int BNL = TL::BN, B_BYTESL = TL::B_BYTES, STAGE_BYTESL = TL::STAGE_BYTES;
  constexpr int TMEM_COLSL = PTile<BNT>::TMEM_COLS;
  static_assert(EW % 4 == 0 && EW >= 4 && EW <= 32, "epilogue warps: a multiple of four");
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + S * STAGE_BYTESL);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  int* s_abort = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = K / BK;
  const int n_tiles = tiles_m * tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EW);
    }
    mbar_init(mma_done, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLSL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    int it = 0;   // operand stages issued so far (the ring position)
    bool stop = false;
    for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
      const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BNL;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = it % S;
        if (it >= S && !mbar_wait(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), spin)) {
          atomicExch(err, 1);
          *(volatile int*)s_abort = 1;
          stop = true;
          break;
        }
        if (*(volatile int*)s_abort) {
          stop = true;
          break;
        }
        unsigned char* st = base + s * STAGE_BYTESL;
        mbar_expect_tx(&full[s], STAGE_BYTESL);
        tma_load_2d(st, mAh, &full[s], kb * BK, m0);
        tma_load_2d(st + A_BYTES, mAl, &full[s], kb * BK, m0);
        tma_load_2d(st + 2 * A_BYTES, mBh, &full[s], kb * BK, n0);
        tma_load_2d(st + 2 * A_BYTES + B_BYTESL, mBl, &full[s], kb * BK, n0);
        ++it;
      }
    }
    // the copies of the last stages must land before the CTA ends
    for (int k = (it > S ? it - S : 0); k < it; ++k) mbar_wait(&full[k % S], (uint32_t)((k / S) & 1), spin);
  } else if (warp == 1 && lane == 0) {
    // --------------------------------------------------------------- MMA
    int it = 0, j = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x, ++j) {
      const int b = j & 1;
      // the epilogue has drained this accumulator (tile j - 2)
      if (j >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)(((j >> 1) & 1) ^ 1), spin)) {
        atomicExch(err, 1);
        *(volatile int*)s_abort = 1;
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(b * BNL);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = it % S;
        if (*(volatile int*)s_abort || !mbar_wait(&full[s], (uint32_t)((it / S) & 1), spin)) {
          atomicExch(err, 1);
          *(volatile int*)s_abort = 1;
          stop = true;
          break;
        }
        fence_after();
        const unsigned char* st = base + s * STAGE_BYTESL;
        const uint64_t dAh = sw128_desc(smem_u32(st));
        const uint64_t dAl = sw128_desc(smem_u32(st + A_BYTES));
        const uint64_t dBh = sw128_desc(smem_u32(st + 2 * A_BYTES));
        const uint64_t dBl = sw128_desc(smem_u32(st + 2 * A_BYTES + B_BYTESL));
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 bf16 = 32 bytes further along K
          mma_bf16(d, dAh + o, dBh + o, TL::IDESC, (kb | kk) != 0);
          mma_bf16(d, dAh + o, dBl + o, TL::IDESC, 1);
          mma_bf16(d, dAl + o, dBh + o, TL::IDESC, 1);
        }
        mma_commit(&empty[s]);
        ++it;
      }
      if (!stop) mma_commit(&acc_full[b]);   // fires when this tile's products are complete
    }
    // every MMA issued above has completed before tensor memory is released
    mma_commit(mma_done);
    mbar_wait(mma_done, 0, spin);
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int quarter = warp & 3;        // tensor-memory lanes 32*quarter .. 32*quarter+31
    const int sub = (warp - 2) >> 2;     // which of the EW/4 warps of this quarter
    int j = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
      const int b = j & 1;
      bool ok = !*(volatile int*)s_abort && mbar_wait(&acc_full[b], (uint32_t)((j >> 1) & 1), spin);
      fence_after();
      // one decision per warp: tcgen05.ld below is a warp-wide instruction
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          atomicExch(err, 1);
          *(volatile int*)s_abort = 1;
        }
        break;
      }
      const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BNL;
      const int row = m0 + quarter * 32 + lane;
#pragma unroll 1
      for (int c = sub; c < BNL / 32; c += EW / 4) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BNL + c * 32), v);
        store(row, n0 + c * 32, v);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLSL) : "memory");
  }
}

}  // namespace tc
}  // namespace bs3
