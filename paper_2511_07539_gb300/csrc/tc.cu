// Self-test of the tensor-core helpers (tc.cuh): one CTA computes
// D = A B^T, A [128][32], B [N][32] (inputs rounded to TF32, nearest and ties
// away, or to BF16, nearest even; FP32 accumulation in TMEM), with the operand
// layout, descriptors, MMA issue, commit and TMEM loads that the batched LU's
// trailing updates use.
#include <cuda_runtime.h>

#include <string>

#include "tc.cuh"
#include "xt_internal.cuh"

namespace xt {

constexpr int kTcTestA = 48 * 1024;    // the A tile (16 KB) and room past it
constexpr int kTcTestB = 152 * 1024;   // the B tile (N * 128 B) and room past it
constexpr long long kTcSpin = 1ll << 24;

template <bool BF>
__global__ void __launch_bounds__(128) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ B,
                                                     int N, float* __restrict__ D, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tslot, 256);
  if (tid == 0) tc::bar_init(&bar, 1);
  unsigned char* As = tsm;
  unsigned char* Bs = tsm + kTcTestA;
  for (int e = tid; e < 128 * 32; e += blockDim.x) {
    const int r = e >> 5, k = e & 31;
    if constexpr (BF) *reinterpret_cast<uint16_t*>(As + tc::tile_off16(r, k, 128)) = tc::to_bf16(A[e]);
    else *reinterpret_cast<uint32_t*>(As + tc::tile_off(r, k, 128)) = tc::to_tf32(A[e]);
  }
  for (int e = tid; e < N * 32; e += blockDim.x) {
    const int r = e >> 5, k = e & 31;
    if constexpr (BF) *reinterpret_cast<uint16_t*>(Bs + tc::tile_off16(r, k, N)) = tc::to_bf16(B[e]);
    else *reinterpret_cast<uint32_t*>(Bs + tc::tile_off(r, k, N)) = tc::to_tf32(B[e]);
  }
  tc::fence_smem_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tslot;
  if (tid == 0) {
    const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
    // one MMA per 32 bytes of K (two chunks): 8 TF32 or 16 BF16 elements
    constexpr int nmma = BF ? 2 : 4;
    for (int k = 0; k < nmma; ++k) {
      const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(2 * k * (128 / 8) * 128), (128 / 8) * 128, 128);
      const uint64_t bd = tc::smem_desc(b0 + (uint32_t)(2 * k * (N / 8) * 128), (uint32_t)(N / 8) * 128, 128);
      if constexpr (BF) tc::mma_bf16(taddr, ad, bd, tc::idesc_bf16(128, N), k > 0);
      else tc::mma_tf32(taddr, ad, bd, tc::idesc_tf32(128, N), k > 0);
    }
    tc::commit(&bar);
  }
  const bool ok = tc::bar_wait(&bar, 0, kTcSpin);
  tc::fence_after();
  const int row = 32 * warp + lane;
  for (int c0 = 0; c0 < N; c0 += 16) {
    float v[16];
    tc::ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) D[(int64_t)row * N + c0 + q] = ok ? v[q] : __int_as_float(0x7FC00000);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 256);
  if (tid == 0) *status = ok ? 0 : 1;
}

}  // namespace xt

using namespace xt;

static int selftest(bool bf, int device, int N, const float* A, const float* B, float* D) {
  if (N < 16 || N > 256 || N % 16 || !A || !B || !D) return XT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return XT_ECUDA;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dS = nullptr;
  int st = 1, rc = XT_OK;
  const size_t smem = kTcTestA + kTcTestB;
  auto kern = bf ? k_tc_selftest<true> : k_tc_selftest<false>;
  if (cudaMalloc(&dA, 128 * 32 * 4) != cudaSuccess || cudaMalloc(&dB, (size_t)N * 32 * 4) != cudaSuccess ||
      cudaMalloc(&dD, (size_t)128 * N * 4) != cudaSuccess || cudaMalloc(&dS, 4) != cudaSuccess) {
    rc = XT_ENOMEM;
  } else if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
             cudaMemcpy(dA, A, 128 * 32 * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, B, (size_t)N * 32 * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = XT_ECUDA;
  } else {
    kern<<<1, 128, smem>>>(dA, dB, N, dD, dS);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(D, dD, (size_t)128 * N * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&st, dS, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = XT_ECUDA;
    else if (st != 0)
      rc = XT_ETIMEOUT;
  }
  cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dS);
  return rc;
}

extern "C" int xt_selftest_tc(int device, int N, const float* A, const float* B, float* D) {
  return selftest(false, device, N, A, B, D);
}

extern "C" int xt_selftest_tc_bf16(int device, int N, const float* A, const float* B, float* D) {
  return selftest(true, device, N, A, B, D);
}
