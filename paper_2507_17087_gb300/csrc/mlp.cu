// The learned cost model: a BF16 MLP with FP32 accumulation on the
// tcgen05 tensor cores (no counterpart in the paper; a project addition that
// prunes the decompose search).
//
// k_gemm_tn: C[M x N] (FP32) = A[M x K] * B[N x K]^T with BF16 row-major
// (K-major) operands.  One CTA of 128 threads computes a 128 x NT tile: TMA
// tensor copies bring 64-wide K chunks of A and B into shared memory in the
// 128-byte swizzled layout the MMA reads (three stages, mbarrier transaction
// counts), one thread issues four K=16 MMAs per chunk into a tensor-memory
// accumulator and commits them to the stage's mbarrier (which frees it for
// the chunk three ahead), and the four warps read the accumulator back (32
// rows each) for the epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "engine.h"
#include "mlp.cuh"
#include "tc.cuh"

namespace mp {

namespace {

constexpr uint32_t kWaitLimit = 1u << 26;   // mbarrier polls before a wait is abandoned

constexpr int kGemmStages = 3;

template <int NT>
__global__ void __launch_bounds__(128) k_gemm_tn(const __grid_constant__ CUtensorMap tmA,
                                                 const __grid_constant__ CUtensorMap tmB, float* __restrict__ C,
                                                 int M, int N, int K, int kcs, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kGemmStages], empty[kGemmStages], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  uint8_t* base = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
  constexpr uint32_t ABYTES = 128 * 128, BBYTES = NT * 128, SBYTES = ABYTES + BBYTES;   // multiples of 1024
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // split K: this CTA takes the 64-wide chunks [kc0, kc0 + nk) (kcs per split)
  const int kc0 = blockIdx.z * kcs;
  const int nk = min(kcs, K / 64 - kc0);

  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, NT);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kGemmStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = tc::idesc_bf16(128, NT);
  if (threadIdx.x == 0) {
    // chunk j uses stage j % 3 for the (j / 3)-th time: its full / empty
    // phases have parity (j / 3) & 1
    auto load = [&](int j) {
      const int s = j % kGemmStages;
      uint8_t* a = base + s * SBYTES;
      tc::mbar_expect_tx(&full[s], SBYTES);
      tc::tma_load_2d(a, &tmA, (kc0 + j) * 64, m0, &full[s]);
      tc::tma_load_2d(a + ABYTES, &tmB, (kc0 + j) * 64, n0, &full[s]);
    };
    int issued = 0, consumed = 0;
    bool ok = true;
    for (; issued < nk && issued < kGemmStages; ++issued) load(issued);
    for (int j = 0; j < nk && ok; ++j) {
      const int s = j % kGemmStages;
      if (!tc::mbar_wait(&full[s], (j / kGemmStages) & 1, kWaitLimit)) {
        ok = false;
        break;
      }
      consumed = j + 1;
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(base + s * SBYTES), b0 = a0 + ABYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_bf16(tmem, tc::sdesc_sw128(a0 + kk * 32), tc::sdesc_sw128(b0 + kk * 32), idesc, (j | kk) != 0);
      tc::mma_commit(&empty[s]);
      // refill the stage of chunk j - 1 (its MMAs queue ahead of chunk j's)
      if (j >= 1 && issued < nk) {
        const int sp = (j - 1) % kGemmStages;
        if (!tc::mbar_wait(&empty[sp], ((j - 1) / kGemmStages) & 1, kWaitLimit)) {
          ok = false;
          break;
        }
        load(issued++);
      }
    }
    tc::mma_commit(&done);   // every MMA issued so far
    if (!ok) {
      s_fail = 1;
      // copies still in flight land before the CTA goes on
      for (int c = consumed; c < issued; ++c) tc::mbar_wait(&full[c % kGemmStages], (c / kGemmStages) & 1, kWaitLimit);
    }
  }
  const bool mma_ok = tc::mbar_wait(&done, 0, kWaitLimit);
  const bool ok = __syncthreads_and(mma_ok && !s_fail) != 0;
  tc::fence_after_sync();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < NT / 32; ++c) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c * 32, r);
      tc::tmem_ld_wait();
      float* dst = C + (size_t)row * N + n0 + c * 32;
      if (gridDim.z > 1) {
        // partial sums of the splits meet in C (zeroed before the launch)
#pragma unroll
        for (int j = 0; j < 32; ++j) atomicAdd(dst + j, __uint_as_float(r[j]));
      } else {
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4*>(dst + j) =
              make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                          __uint_as_float(r[j + 3]));
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(status, MP_ETIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NT);
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

// Tensor map of a rows x K row-major BF16 matrix read in boxes of `box_rows`
// rows by 64 columns (128 bytes), 128-byte swizzled into shared memory.
int bf16_tile_map(CUtensorMap* map, const void* ptr, int rows, int K, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return MP_ECUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? MP_OK : MP_ECUDA;
}

size_t gemm_smem(int nt) { return kGemmStages * (128 * 128 + (size_t)nt * 128) + 1024; }

template <int NT>
int launch_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int* status,
                cudaStream_t st) {
  const size_t sm = gemm_smem(NT);
  MP_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tn<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  // few output tiles over a long K (the weight gradients: K = the batch):
  // split K over more CTAs, at least 8 chunks each, and add up in C
  const int tiles = (M / 128) * (N / NT), nk = K / 64;
  int splits = 1;
  if (tiles < 64 && nk >= 8) splits = std::min(nk / 8, std::max(1, 128 / tiles));
  const int kcs = (nk + splits - 1) / splits;
  splits = (nk + kcs - 1) / kcs;
  if (splits > 1) MP_CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), st));
  CUtensorMap tmA, tmB;
  int rc = bf16_tile_map(&tmA, A, M, K, 128);
  if (!rc) rc = bf16_tile_map(&tmB, B, N, K, NT);
  if (rc) return rc;
  dim3 grid(M / 128, N / NT, splits);
  k_gemm_tn<NT><<<grid, 128, sm, st>>>(tmA, tmB, C, M, N, K, kcs, status);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

}  // namespace

int gemm_tn(const void* A, const void* B, float* C, int M, int N, int K, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || M % 128 || K % 64) return MP_EINVAL;
  // operands are staged and results stored in 16-byte vectors
  if ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 15) return MP_EINVAL;
  const __nv_bfloat16* a = (const __nv_bfloat16*)A;
  const __nv_bfloat16* b = (const __nv_bfloat16*)B;
  // the widest tile that still gives about a wave of CTAs (the training
  // step's products are a few hundred MFLOP: 4096 x 256 at 128 x 256 tiles
  // would occupy 32 of the SMs)
  const int want = 128;
  if (N % 256 == 0 && (M / 128) * (N / 256) >= want) return launch_gemm<256>(a, b, C, M, N, K, status, st);
  if (N % 128 == 0 && (M / 128) * (N / 128) >= want) return launch_gemm<128>(a, b, C, M, N, K, status, st);
  if (N % 64 == 0) return launch_gemm<64>(a, b, C, M, N, K, status, st);
  if (N % 128 == 0) return launch_gemm<128>(a, b, C, M, N, K, status, st);
  if (N % 256 == 0) return launch_gemm<256>(a, b, C, M, N, K, status, st);
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

// ======================================================================
// Model parameters, training step and unfused forward
//
// Parameters (FP32 master copy, packed): W1[256x64] b1[256] W2[256x256]
// b2[256] W3[256x256] b3[256] w4[256] b4[1]; BF16 copies W1, W2, W3 feed the
// forward GEMMs and W2^T, W3^T the backward ones.  A training step on a
// batch X[B x 64] (BF16), targets t[B]:
//   Z1 = X W1^T, H1 = relu(Z1 + b1), Z2 = H1 W2^T, H2 = relu(Z2 + b2),
//   Z3 = H2 W3^T, y = relu(Z3 + b3) w4 + b4, loss = 0.5 mean (y - t)^2,
//   dZ3 = (dy w4^T) o [Z3 + b3 > 0], dW3 = dZ3^T H2, dZ2 = (dZ3 W3) o [..],
//   dW2 = dZ2^T H1, dZ1 = (dZ2 W2) o [..], dW1 = dZ1^T X, then Adam.
// Every product runs in k_gemm_tn (transposed operands are written by the
// elementwise kernels); elementwise work runs in FP32.

namespace mp {
namespace mlpk {



// 32 x 32 tiles: out[r][c] = f(in[r][c]) in BF16, optionally outT[c][r]
// (R x C row-major in, C x R row-major outT), column sums of the FP32
// values into colsum.
template <int KIND>
__global__ void __launch_bounds__(256) k_elem(const float* __restrict__ Z, const float* __restrict__ bias,
                                              const float* __restrict__ aux, const float* __restrict__ aux2,
                                              int R, int C, bf16* __restrict__ out, bf16* __restrict__ outT,
                                              float* __restrict__ colsum, float* __restrict__ colsum2) {
  // KIND 0: relu(Z + bias)                       (forward)
  // KIND 1: Z o [aux + bias > 0]                 (backward through relu; Z = dH, aux = pre-activation)
  // KIND 2: [Z + bias > 0] * dy[r] * w4[c]       (output layer backward; aux = dy, aux2 = w4),
  //         colsum2 += relu(Z + bias) * dy[r]    (gradient of w4)
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  float csum = 0.f, csum2 = 0.f;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    float v = 0.f;
    if (r < R && c < C) {
      const float z = Z[(size_t)r * C + c];
      const float b = bias ? bias[c] : 0.f;
      if (KIND == 0) {
        v = fmaxf(z + b, 0.f);
      } else if (KIND == 1) {
        v = (aux[(size_t)r * C + c] + b > 0.f) ? z : 0.f;
      } else {
        const float a = z + b;
        v = a > 0.f ? aux[r] * aux2[c] : 0.f;
        csum2 += fmaxf(a, 0.f) * aux[r];
      }
      if (out) out[(size_t)r * C + c] = __float2bfloat16(v);
    }
    tile[i][tx] = v;
    csum += v;
  }
  if (colsum) atomicAdd(colsum + c0 + tx, csum);
  if (KIND == 2 && colsum2) atomicAdd(colsum2 + c0 + tx, csum2);
  if (!outT) return;
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + tx;
    if (c < C && r < R) outT[(size_t)c * R + r] = __float2bfloat16(tile[tx][i]);
  }
}

// BF16 transpose: out[c][r] = in[r][c]
__global__ void __launch_bounds__(256) k_transpose_bf16(const bf16* __restrict__ in, int R, int C,
                                                        bf16* __restrict__ out) {
  __shared__ bf16 tile[32][34];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8)
    if (r0 + i < R && c0 + tx < C) tile[i][tx] = in[(size_t)(r0 + i) * C + c0 + tx];
  __syncthreads();
  for (int i = ty; i < 32; i += 8)
    if (c0 + i < C && r0 + tx < R) out[(size_t)(c0 + i) * R + r0 + tx] = tile[tx][i];
}

// y = relu(Z3 + b3) w4 + b4 per row (one warp per row); with targets:
// dy = (y - t) / B and the squared error into loss.
__global__ void __launch_bounds__(256) k_output(const float* __restrict__ Z3, const float* __restrict__ P, int B,
                                                const float* __restrict__ target, float* __restrict__ y,
                                                float* __restrict__ dy, float* __restrict__ loss) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  const float* z = Z3 + (size_t)warp * DH;
  float s = 0.f;
  for (int j = lane; j < DH; j += 32) s += fmaxf(z[j] + P[O_B3 + j], 0.f) * P[O_W4 + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) {
    const float out = s + P[O_B4];
    y[warp] = out;
    if (target) {
      const float d = out - target[warp];
      dy[warp] = d / B;
      atomicAdd(loss, 0.5f * d * d / B);
    }
  }
}

__global__ void k_sum(const float* __restrict__ v, int n, float* __restrict__ out) {
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out += t;
  }
}

// Adam (Kingma & Ba) with bias correction, then the BF16 copies.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_refresh(const float* __restrict__ P, bf16* __restrict__ W1b, bf16* __restrict__ W2b,
                          bf16* __restrict__ W3b, bf16* __restrict__ W2T, bf16* __restrict__ W3T,
                          unsigned char* __restrict__ Wimg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < DH * DH; i += gridDim.x * blockDim.x) {
    const int r = i / DH, c = i % DH;
    if (i < DH * DIN) {
      W1b[i] = __float2bfloat16(P[O_W1 + i]);
      *reinterpret_cast<bf16*>(Wimg + wimg_offset(1, i / DIN, i % DIN)) = W1b[i];
    }
    W2b[i] = __float2bfloat16(P[O_W2 + i]);
    W3b[i] = __float2bfloat16(P[O_W3 + i]);
    W2T[(size_t)c * DH + r] = __float2bfloat16(P[O_W2 + i]);
    W3T[(size_t)c * DH + r] = __float2bfloat16(P[O_W3 + i]);
    *reinterpret_cast<bf16*>(Wimg + wimg_offset(2, r, c)) = W2b[i];
    *reinterpret_cast<bf16*>(Wimg + wimg_offset(3, r, c)) = W3b[i];
  }
}

}  // namespace mlpk
}  // namespace mp



namespace mp {
namespace mlpk {

struct Bufs {
  float *Z1, *Z2, *Z3, *dH, *y, *dy;
  bf16 *XT, *H1, *H2, *H1T, *H2T, *dZ1, *dZ2, *dZ3, *dZ1T, *dZ2T, *dZ3T;
};

int ensure_ws(mp_mlp* h, int B, Bufs& b) {
  const size_t f32 = (size_t)B * DH * 4, b16 = (size_t)B * DH * 2;
  const size_t need = 4 * f32 + 2 * (size_t)B * 4 + (size_t)B * DIN * 2 + 11 * b16 + 64 * 256;
  if (h->ws_B < B) {
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_B = 0;
    if (cudaMalloc(&h->ws, need) != cudaSuccess) {
      cudaGetLastError();
      return MP_ENOMEM;
    }
    h->ws_B = B;
  }
  char* p = (char*)h->ws;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  b.Z1 = (float*)take(f32); b.Z2 = (float*)take(f32); b.Z3 = (float*)take(f32); b.dH = (float*)take(f32);
  b.y = (float*)take((size_t)B * 4); b.dy = (float*)take((size_t)B * 4);
  b.XT = (bf16*)take((size_t)B * DIN * 2);
  b.H1 = (bf16*)take(b16); b.H2 = (bf16*)take(b16); b.H1T = (bf16*)take(b16); b.H2T = (bf16*)take(b16);
  b.dZ1 = (bf16*)take(b16); b.dZ2 = (bf16*)take(b16); b.dZ3 = (bf16*)take(b16);
  b.dZ1T = (bf16*)take(b16); b.dZ2T = (bf16*)take(b16); b.dZ3T = (bf16*)take(b16);
  return MP_OK;
}

// 32 x 32 tiles of an R x C array: rows on x (up to 2^31 - 1 blocks, any
// batch), columns on y (C <= 256)
dim3 tiles(int R, int C) { return dim3((R + 31) / 32, (C + 31) / 32); }

// Forward through Z3 (and y); H1T / H2T only when training.  Every launch is
// checked at once: a launch that fails (a grid too large, say) must not
// leave the next kernels reading unwritten activations.
int forward(mp_mlp* h, const bf16* X, int B, Bufs& b, bool train, const float* target, cudaStream_t st) {
  int rc;
  if ((rc = gemm_tn(X, h->W1b, b.Z1, B, DH, DIN, h->status, st))) return rc;
  k_elem<0><<<tiles(B, DH), 256, 0, st>>>(b.Z1, h->P + O_B1, nullptr, nullptr, B, DH, b.H1, train ? b.H1T : nullptr,
                                          nullptr, nullptr);
  MP_CUDA_TRY(cudaGetLastError());
  if ((rc = gemm_tn(b.H1, h->W2b, b.Z2, B, DH, DH, h->status, st))) return rc;
  k_elem<0><<<tiles(B, DH), 256, 0, st>>>(b.Z2, h->P + O_B2, nullptr, nullptr, B, DH, b.H2, train ? b.H2T : nullptr,
                                          nullptr, nullptr);
  MP_CUDA_TRY(cudaGetLastError());
  if ((rc = gemm_tn(b.H2, h->W3b, b.Z3, B, DH, DH, h->status, st))) return rc;
  k_output<<<(B * 32 + 255) / 256, 256, 0, st>>>(b.Z3, h->P, B, target, b.y, b.dy, h->scalar);
  MP_CUDA_TRY(cudaGetLastError());
  count_launch(3);
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

int train_step(mp_mlp* h, const bf16* X, const float* target, int B, float lr, cudaStream_t st) {
  Bufs b;
  int rc = ensure_ws(h, B, b);
  if (rc) return rc;
  MP_CUDA_TRY(cudaMemsetAsync(h->G, 0, NPARAM * 4, st));
  MP_CUDA_TRY(cudaMemsetAsync(h->scalar, 0, 4, st));
  k_transpose_bf16<<<tiles(B, DIN), 256, 0, st>>>(X, B, DIN, b.XT);
  MP_CUDA_TRY(cudaGetLastError());
  count_launch();
  if ((rc = forward(h, X, B, b, true, target, st))) return rc;
  // output layer and layer 3
  k_sum<<<1, 256, 0, st>>>(b.dy, B, h->G + O_B4);
  MP_CUDA_TRY(cudaGetLastError());
  k_elem<2><<<tiles(B, DH), 256, 0, st>>>(b.Z3, h->P + O_B3, b.dy, h->P + O_W4, B, DH, b.dZ3, b.dZ3T, h->G + O_B3,
                                          h->G + O_W4);
  MP_CUDA_TRY(cudaGetLastError());
  count_launch(2);
  if ((rc = gemm_tn(b.dZ3T, b.H2T, h->G + O_W3, DH, DH, B, h->status, st))) return rc;
  if ((rc = gemm_tn(b.dZ3, h->W3T, b.dH, B, DH, DH, h->status, st))) return rc;
  k_elem<1><<<tiles(B, DH), 256, 0, st>>>(b.dH, h->P + O_B2, b.Z2, nullptr, B, DH, b.dZ2, b.dZ2T, h->G + O_B2, nullptr);
  MP_CUDA_TRY(cudaGetLastError());
  count_launch();
  if ((rc = gemm_tn(b.dZ2T, b.H1T, h->G + O_W2, DH, DH, B, h->status, st))) return rc;
  if ((rc = gemm_tn(b.dZ2, h->W2T, b.dH, B, DH, DH, h->status, st))) return rc;
  k_elem<1><<<tiles(B, DH), 256, 0, st>>>(b.dH, h->P + O_B1, b.Z1, nullptr, B, DH, b.dZ1, b.dZ1T, h->G + O_B1, nullptr);
  MP_CUDA_TRY(cudaGetLastError());
  count_launch();
  if ((rc = gemm_tn(b.dZ1T, b.XT, h->G + O_W1, DH, DIN, B, h->status, st))) return rc;
  if (lr > 0.f) {
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)h->step), c2 = 1.f - powf(b2, (float)h->step);
    k_adam<<<296, 256, 0, st>>>(h->P, h->G, h->M1, h->M2, NPARAM, lr, b1, b2, c1, c2, 1e-8f);
    MP_CUDA_TRY(cudaGetLastError());
    k_refresh<<<256, 256, 0, st>>>(h->P, h->W1b, h->W2b, h->W3b, h->W2T, h->W3T, h->Wimg);
    MP_CUDA_TRY(cudaGetLastError());
    count_launch(2);
  }
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

int upload_params(mp_mlp* h, const float* host, cudaStream_t st) {
  MP_CUDA_TRY(cudaMemcpyAsync(h->P, host, NPARAM * 4, cudaMemcpyHostToDevice, st));
  k_refresh<<<256, 256, 0, st>>>(h->P, h->W1b, h->W2b, h->W3b, h->W2T, h->W3T, h->Wimg);
  count_launch();
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  return MP_OK;
}

}  // namespace mlpk
}  // namespace mp

extern "C" int mp_mlp_create(uint64_t seed, mp_mlp** out) {
  using namespace mp::mlpk;
  if (!out) return MP_EINVAL;
  mp_mlp* h = new mp_mlp();
  cudaGetDevice(&h->device);
  // every region starts on a 256-byte boundary (NPARAM is odd; the GEMM
  // epilogue stores 16-byte vectors into the gradient blocks)
  const size_t preg = (NPARAM * 4 + 255) & ~size_t(255);
  size_t bytes = 4 * preg + 5 * (size_t)DH * DH * 2 + kWChunks * kWChunkBytes + 256 + 256;
  char* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return MP_ENOMEM;
  }
  cudaMemset(p, 0, bytes);
  h->P = (float*)p; p += preg;
  h->G = (float*)p; p += preg;
  h->M1 = (float*)p; p += preg;
  h->M2 = (float*)p; p += preg;
  h->W1b = (bf16*)p; p += (size_t)DH * DH * 2;
  h->W2b = (bf16*)p; p += (size_t)DH * DH * 2;
  h->W3b = (bf16*)p; p += (size_t)DH * DH * 2;
  h->W2T = (bf16*)p; p += (size_t)DH * DH * 2;
  h->W3T = (bf16*)p; p += (size_t)DH * DH * 2;
  h->Wimg = (unsigned char*)p; p += kWChunks * kWChunkBytes;
  h->status = (int*)p; p += 256;
  h->scalar = (float*)p;
  // He initialisation from splitmix64 + Box-Muller
  std::vector<float> host(NPARAM, 0.f);
  uint64_t s = seed;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto normal = [&]() {
    const double u1 = ((next() >> 11) + 1) * (1.0 / 9007199254740993.0);
    const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  for (size_t i = 0; i < (size_t)DH * DIN; ++i) host[O_W1 + i] = (float)(normal() * std::sqrt(2.0 / DIN));
  for (size_t i = 0; i < (size_t)DH * DH; ++i) host[O_W2 + i] = (float)(normal() * std::sqrt(2.0 / DH));
  for (size_t i = 0; i < (size_t)DH * DH; ++i) host[O_W3 + i] = (float)(normal() * std::sqrt(2.0 / DH));
  for (size_t i = 0; i < (size_t)DH; ++i) host[O_W4 + i] = (float)(normal() * std::sqrt(1.0 / DH));
  int rc = upload_params(h, host.data(), nullptr);
  if (rc) {
    mp_mlp_destroy(h);
    return rc;
  }
  *out = h;
  return MP_OK;
}

extern "C" int mp_mlp_destroy(mp_mlp* h) {
  if (!h) return MP_OK;
  if (h->ws) cudaFree(h->ws);
  if (h->P) cudaFree(h->P);
  delete h;
  return MP_OK;
}

extern "C" int mp_mlp_num_params(void) { return (int)mp::mlpk::NPARAM; }

extern "C" int mp_mlp_set_params(mp_mlp* h, const float* params) {
  if (!h || !params) return MP_EINVAL;
  return mp::mlpk::upload_params(h, params, nullptr);
}

extern "C" int mp_mlp_get_params(const mp_mlp* h, float* params, float* grads) {
  if (!h) return MP_EINVAL;
  if (params) MP_CUDA_TRY(cudaMemcpy(params, h->P, mp::mlpk::NPARAM * 4, cudaMemcpyDeviceToHost));
  if (grads) MP_CUDA_TRY(cudaMemcpy(grads, h->G, mp::mlpk::NPARAM * 4, cudaMemcpyDeviceToHost));
  return MP_OK;
}

extern "C" int mp_mlp_forward(mp_mlp* h, const void* X, float* y, int B, void* stream) {
  using namespace mp::mlpk;
  if (!h || !X || !y || B <= 0 || B % 128) return MP_EINVAL;
  if (B > kMaxRows) return MP_ENOTSUP;
  if (!mp::is_device_pointer(X) || !mp::is_device_pointer(y)) return MP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Bufs b;
  int rc = ensure_ws(h, B, b);
  if (rc) return rc;
  MP_CUDA_TRY(cudaMemsetAsync(h->status, 0, 4, st));
  if ((rc = forward(h, (const bf16*)X, B, b, false, nullptr, st))) return rc;
  MP_CUDA_TRY(cudaMemcpyAsync(y, b.y, (size_t)B * 4, cudaMemcpyDeviceToDevice, st));
  int s = 0;
  MP_CUDA_TRY(cudaMemcpyAsync(&s, h->status, 4, cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  return s;
}

extern "C" int mp_mlp_train_step(mp_mlp* h, const void* X, const float* target, int B, float lr, float* loss,
                                 void* stream) {
  using namespace mp::mlpk;
  if (!h || !X || !target || B <= 0 || B % 128) return MP_EINVAL;
  if (B > kMaxRows) return MP_ENOTSUP;
  if (!mp::is_device_pointer(X) || !mp::is_device_pointer(target)) return MP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  MP_CUDA_TRY(cudaMemsetAsync(h->status, 0, 4, st));
  int rc = train_step(h, (const bf16*)X, target, B, lr, st);
  if (rc) return rc;
  int s = 0;
  float l = 0.f;
  MP_CUDA_TRY(cudaMemcpyAsync(&s, h->status, 4, cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaMemcpyAsync(&l, h->scalar, 4, cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return s;
}

// ------------------------------------------------------------ checkpoint

namespace mp {
namespace mlpk {
namespace {

constexpr char kMagic[8] = {'M', 'A', 'P', 'L', 'E', 'M', 'L', 'P'};
constexpr uint32_t kFormat = 2;   // 2: the margin bound follows the header (1: none)

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t nparam;
  int64_t step;
};

// Waits on an mbarrier that nothing arrives on, as the tensor-core kernels
// wait on theirs: bounded polling, then MP_ETIMEOUT in the status word.
__global__ void k_wait_nobody(uint32_t limit, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  const bool done = tc::mbar_wait(&bar, 0, limit);
  if (!done && threadIdx.x == 0) atomicExch(status, MP_ETIMEOUT);
}

}  // namespace
}  // namespace mlpk
}  // namespace mp

extern "C" int mp_mlp_save(const mp_mlp* h, const char* path) {
  using namespace mp::mlpk;
  if (!h || !path) return MP_EINVAL;
  std::vector<float> buf(3 * NPARAM);
  MP_CUDA_TRY(cudaMemcpy(buf.data(), h->P, NPARAM * 4, cudaMemcpyDeviceToHost));
  MP_CUDA_TRY(cudaMemcpy(buf.data() + NPARAM, h->M1, NPARAM * 4, cudaMemcpyDeviceToHost));
  MP_CUDA_TRY(cudaMemcpy(buf.data() + 2 * NPARAM, h->M2, NPARAM * 4, cudaMemcpyDeviceToHost));
  CkptHeader hd;
  std::memcpy(hd.magic, kMagic, 8);
  hd.version = kFormat;
  hd.nparam = (uint32_t)NPARAM;
  hd.step = h->step;
  FILE* f = std::fopen(path, "wb");
  if (!f) return MP_EINVAL;
  const double bound = h->margin_bound;
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(&bound, 8, 1, f) == 1 &&
                  std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  return ok && closed ? MP_OK : MP_EINVAL;
}

extern "C" int mp_mlp_load(mp_mlp* h, const char* path) {
  using namespace mp::mlpk;
  if (!h || !path) return MP_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return MP_EINVAL;
  CkptHeader hd;
  std::vector<float> buf(3 * NPARAM);
  double bound = __builtin_inf();
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kMagic, 8) == 0 &&
            (hd.version == 1 || hd.version == kFormat) && hd.nparam == (uint32_t)NPARAM;
  if (ok && hd.version >= 2) ok = std::fread(&bound, 8, 1, f) == 1;
  ok = ok && std::fread(buf.data(), 4, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return MP_EINVAL;
  h->margin_bound = bound;
  MP_CUDA_TRY(cudaMemcpy(h->M1, buf.data() + NPARAM, NPARAM * 4, cudaMemcpyHostToDevice));
  MP_CUDA_TRY(cudaMemcpy(h->M2, buf.data() + 2 * NPARAM, NPARAM * 4, cudaMemcpyHostToDevice));
  h->step = (int)hd.step;
  return upload_params(h, buf.data(), nullptr);
}

extern "C" int mp_selftest_wait_timeout(uint32_t limit, void* stream) {
  using namespace mp;
  if (limit < 1 || limit > (1u << 26)) return MP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = (int*)workspace(sizeof(int), 6);
  if (!status) return MP_ENOMEM;
  MP_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  mlpk::k_wait_nobody<<<1, 32, 0, st>>>(limit, status);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  int h = 0;
  MP_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  return h;
}
