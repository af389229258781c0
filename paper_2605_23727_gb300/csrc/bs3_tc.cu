// Tensor-core split-bfloat16 product (bs3_tc.cuh) as a standalone entry point,
// and the shared helpers that build its operands and tensor maps.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/bs3.h"
#include "bs3_tc.cuh"
#include "bs3_tc_host.h"

namespace bs3 {

__global__ void split_bf16_kernel(const float* __restrict__ x, size_t n, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));   // v - h is exact in binary32
  }
}

__global__ void __launch_bounds__(tc::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                   const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, float* C,
                   long long ldc, int K, int* err, long long spin) {
  const tc::StoreRowMajor st{C, ldc};
  tc::gemm_tile<4, tc::BN>(&mAh, &mAl, &mBh, &mBl, blockIdx.x * tc::BM, blockIdx.y * tc::BN, K, st, err, spin);
}

// The product as the ensembles' stage products run it: persistent CTAs with
// two tensor-memory accumulators and 16 epilogue warps (gemm_persistent), the
// epilogue storing the binary32 accumulators row-major.
constexpr int kPersistEpiWarps = 16;

template <int BNT>
__global__ void __launch_bounds__(tc::threads_for(kPersistEpiWarps), 1)
    tc_gemm_persistent_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                              float* C, long long ldc, int tiles_m, int tiles_n, int K, int* err, long long spin) {
  const tc::StoreRowMajor st{C, ldc};
  tc::gemm_persistent<kPersistEpiWarps, BNT>(&mAh, &mAl, &mBh, &mBl, tiles_m, tiles_n, K, st, err, spin);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

int tc_encode_bf16_2d(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return BS3_ERR_CUDA;
  if (((uintptr_t)ptr & 15) != 0 || (cols * 2) % 16 != 0) return BS3_ERR_INVALID_ARG;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)tc::BK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BS3_OK : BS3_ERR_CUDA;
}

int tc_split(const float* x, size_t n, void* hi, void* lo, cudaStream_t stream) {
  const int blocks = (int)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32);
  split_bf16_kernel<<<blocks > 0 ? blocks : 1, 256, 0, stream>>>(x, n, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
  return cudaGetLastError() == cudaSuccess ? BS3_OK : BS3_ERR_CUDA;
}

}  // namespace bs3

using namespace bs3;

#define TC_CUDA(call)                             \
  do {                                            \
    if ((call) != cudaSuccess) { rc = BS3_ERR_CUDA; goto done; } \
  } while (0)
#define TC_RC(expr)                               \
  do {                                            \
    rc = (expr);                                  \
    if (rc != BS3_OK) goto done;                  \
  } while (0)

extern "C" int bs3_tc_gemm(int64_t M, int64_t Nc, int64_t K, const float* A, const float* B, float* C) {
  if (M < tc::BM || Nc < tc::BN || K < tc::BK || M % tc::BM || Nc % tc::BN || K % tc::BK || !A || !B || !C)
    return BS3_ERR_INVALID_ARG;
  if (K > (1 << 30) || M > (1 << 30) || Nc > (1 << 30)) return BS3_ERR_INVALID_ARG;
  int rc = BS3_OK;
  void *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  int* derr = nullptr;
  int herr = 0;
  CUtensorMap mAh, mAl, mBh, mBl;
  TC_CUDA(cudaMalloc(&ah, M * K * 2));
  TC_CUDA(cudaMalloc(&al, M * K * 2));
  TC_CUDA(cudaMalloc(&bh, Nc * K * 2));
  TC_CUDA(cudaMalloc(&bl, Nc * K * 2));
  TC_CUDA(cudaMalloc(&derr, sizeof(int)));
  TC_CUDA(cudaMemset(derr, 0, sizeof(int)));
  TC_RC(tc_split(A, (size_t)(M * K), ah, al, 0));
  TC_RC(tc_split(B, (size_t)(Nc * K), bh, bl, 0));
  TC_RC(tc_encode_bf16_2d(&mAh, ah, M, K, tc::BM));
  TC_RC(tc_encode_bf16_2d(&mAl, al, M, K, tc::BM));
  TC_RC(tc_encode_bf16_2d(&mBh, bh, Nc, K, tc::BN));
  TC_RC(tc_encode_bf16_2d(&mBl, bl, Nc, K, tc::BN));
  TC_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
  tc_gemm_kernel<<<dim3((unsigned)(M / tc::BM), (unsigned)(Nc / tc::BN)), tc::THREADS, tc::SMEM_BYTES>>>(
      mAh, mAl, mBh, mBl, C, (long long)Nc, (int)K, derr, (long long)1 << 22);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaDeviceSynchronize());
  TC_CUDA(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) rc = BS3_ERR_DEVICE_WAIT;
done:
  cudaFree(ah); cudaFree(al); cudaFree(bh); cudaFree(bl); cudaFree(derr);
  return rc;
}

template <int BNT>
static int tc_gemm_persistent_impl(int64_t M, int64_t Nc, int64_t K, const float* A, const float* B, float* C,
                                   int max_ctas) {
  using PT = tc::PTile<BNT>;
  int rc = BS3_OK;
  void *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  int* derr = nullptr;
  int herr = 0, dev = 0, sms = 0;
  int64_t tiles = 0;
  unsigned grid = 0;
  CUtensorMap mAh, mAl, mBh, mBl;
  TC_CUDA(cudaGetDevice(&dev));
  TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  tiles = (M / tc::BM) * (Nc / BNT);
  grid = (unsigned)std::min<int64_t>(tiles, max_ctas > 0 ? std::min(max_ctas, sms) : sms);
  TC_CUDA(cudaMalloc(&ah, M * K * 2));
  TC_CUDA(cudaMalloc(&al, M * K * 2));
  TC_CUDA(cudaMalloc(&bh, Nc * K * 2));
  TC_CUDA(cudaMalloc(&bl, Nc * K * 2));
  TC_CUDA(cudaMalloc(&derr, sizeof(int)));
  TC_CUDA(cudaMemset(derr, 0, sizeof(int)));
  TC_RC(tc_split(A, (size_t)(M * K), ah, al, 0));
  TC_RC(tc_split(B, (size_t)(Nc * K), bh, bl, 0));
  TC_RC(tc_encode_bf16_2d(&mAh, ah, M, K, tc::BM));
  TC_RC(tc_encode_bf16_2d(&mAl, al, M, K, tc::BM));
  TC_RC(tc_encode_bf16_2d(&mBh, bh, Nc, K, BNT));
  TC_RC(tc_encode_bf16_2d(&mBl, bl, Nc, K, BNT));
  TC_CUDA(cudaFuncSetAttribute(tc_gemm_persistent_kernel<BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               PT::SMEM_BYTES));
  tc_gemm_persistent_kernel<BNT><<<grid, tc::threads_for(kPersistEpiWarps), PT::SMEM_BYTES>>>(
      mAh, mAl, mBh, mBl, C, (long long)Nc, (int)(M / tc::BM), (int)(Nc / BNT), (int)K, derr, (long long)1 << 22);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaDeviceSynchronize());
  TC_CUDA(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) rc = BS3_ERR_DEVICE_WAIT;
done:
  cudaFree(ah); cudaFree(al); cudaFree(bh); cudaFree(bl); cudaFree(derr);
  return rc;
}

extern "C" int bs3_tc_gemm_persistent(int64_t M, int64_t Nc, int64_t K, const float* A, const float* B, float* C,
                                      int tile_n, int max_ctas) {
  if (tile_n != 128 && tile_n != 256) return BS3_ERR_INVALID_ARG;
  if (M < tc::BM || Nc < tile_n || K < tc::BK || M % tc::BM || Nc % tile_n || K % tc::BK || !A || !B || !C)
    return BS3_ERR_INVALID_ARG;
  if (K > (1 << 30) || M > (1 << 30) || Nc > (1 << 30) || max_ctas < 0) return BS3_ERR_INVALID_ARG;
  return tile_n == 128 ? tc_gemm_persistent_impl<128>(M, Nc, K, A, B, C, max_ctas)
                       : tc_gemm_persistent_impl<256>(M, Nc, K, A, B, C, max_ctas);
}
