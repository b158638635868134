// The learned cost model: a BF16 MLP with FP32 accumulation on the
// tcgen05 tensor cores (no counterpart in the paper; a project addition that
// prunes the decompose search).
//
// k_gemm_tn: C[M x N] (FP32) = A[M x K] * B[N x K]^T with BF16 row-major
// (K-major) operands.  One CTA of 128 threads computes a 128 x NT tile: the
// K loop stages 64-wide chunks of A and B in shared memory with the 128-byte
// swizzle (double-buffered), one thread issues four K=16 MMAs per chunk into
// a tensor-memory accumulator and commits them to the chunk's mbarrier, and
// the four warps read the accumulator back (32 rows each) for the epilogue.
#include <algorithm>
#include <cstring>

#include "engine.h"
#include "tc.cuh"

namespace mp {

namespace {

constexpr uint32_t kWaitLimit = 1u << 26;   // mbarrier polls before a wait is abandoned

__device__ __forceinline__ void stage_rows(uint8_t* dst, const __nv_bfloat16* __restrict__ src, int rows,
                                           int ld, int k0) {
  // rows x 64 elements (8 chunks of 16 bytes per row) into the swizzled tile
  for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
    const int r = i >> 3, c = i & 7;
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(src + (size_t)r * ld + k0 + c * 8));
    *reinterpret_cast<uint4*>(dst + tc::sw128_offset(r, c * 8)) = v;
  }
}

template <int NT>
__global__ void __launch_bounds__(128) k_gemm_tn(const __nv_bfloat16* __restrict__ A,
                                                 const __nv_bfloat16* __restrict__ B, float* __restrict__ C,
                                                 int M, int N, int K, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  uint8_t* base = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
  constexpr int ABYTES = 128 * 128, BBYTES = NT * 128;
  uint8_t* bufA[2] = {base, base + ABYTES + BBYTES};
  uint8_t* bufB[2] = {base + ABYTES, base + 2 * ABYTES + BBYTES};
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, NT);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = tc::idesc_bf16(128, NT);
  bool ok = true;
  const int nk = K / 64;
  for (int kc = 0; kc < nk; ++kc) {
    const int b = kc & 1;
    if (kc >= 2) ok = ok && tc::mbar_wait(&bar[b], ((kc >> 1) - 1) & 1, kWaitLimit);
    stage_rows(bufA[b], A + (size_t)m0 * K, 128, K, kc * 64);
    stage_rows(bufB[b], B + (size_t)n0 * K, NT, K, kc * 64);
    tc::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(bufA[b]), b0 = tc::smem_u32(bufB[b]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_bf16(tmem, tc::sdesc_sw128(a0 + kk * 32), tc::sdesc_sw128(b0 + kk * 32), idesc,
                     (kc | kk) != 0);
      tc::mma_commit(&bar[b]);
    }
  }
  // the last commit covers every MMA issued before it
  const int last = nk - 1;
  ok = ok && tc::mbar_wait(&bar[last & 1], (last >> 1) & 1, kWaitLimit);
  tc::fence_after_sync();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < NT / 32; ++c) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c * 32, r);
      tc::tmem_ld_wait();
      float* dst = C + (size_t)row * N + n0 + c * 32;
#pragma unroll
      for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(dst + j) =
            make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                        __uint_as_float(r[j + 3]));
    }
  } else if (threadIdx.x == 0) {
    atomicExch(status, MP_ETIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NT);
}

size_t gemm_smem(int nt) { return 2 * (128 * 128 + (size_t)nt * 128) + 1024; }

template <int NT>
int launch_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int* status,
                cudaStream_t st) {
  const size_t sm = gemm_smem(NT);
  MP_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tn<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  dim3 grid(M / 128, N / NT);
  k_gemm_tn<NT><<<grid, 128, sm, st>>>(A, B, C, M, N, K, status);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

}  // namespace

int gemm_tn(const void* A, const void* B, float* C, int M, int N, int K, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || M % 128 || K % 64) return MP_EINVAL;
  const __nv_bfloat16* a = (const __nv_bfloat16*)A;
  const __nv_bfloat16* b = (const __nv_bfloat16*)B;
  if (N % 256 == 0) return launch_gemm<256>(a, b, C, M, N, K, status, st);
  if (N % 128 == 0) return launch_gemm<128>(a, b, C, M, N, K, status, st);
  if (N % 64 == 0) return launch_gemm<64>(a, b, C, M, N, K, status, st);
  return MP_EINVAL;
}

}  // namespace mp

extern "C" int mp_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, void* stream) {
  using namespace mp;
  if (!A || !B || !C) return MP_EINVAL;
  if (!is_device_pointer(A) || !is_device_pointer(B) || !is_device_pointer(C)) return MP_EINVAL;
  int* status = (int*)workspace(sizeof(int), 4);
  if (!status) return MP_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  MP_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  int rc = gemm_tn(A, B, C, M, N, K, status, st);
  if (rc) return rc;
  int h = 0;
  MP_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  return h;
}
