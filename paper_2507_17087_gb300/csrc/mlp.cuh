// The learned cost model's parameters and training entry points (shared by
// mlp.cu and learned.cu).
#pragma once

#include <cuda_bf16.h>

#include "engine.h"

namespace mp {
namespace mlpk {

constexpr int DIN = 64, DH = 256;
constexpr int kMaxRows = 1 << 26;   // rows of one forward / training batch (one warp per row in 32-bit indexing)
constexpr size_t O_W1 = 0, O_B1 = O_W1 + DH * DIN, O_W2 = O_B1 + DH, O_B2 = O_W2 + DH * DH, O_W3 = O_B2 + DH,
                 O_B3 = O_W3 + DH * DH, O_W4 = O_B3 + DH, O_B4 = O_W4 + DH, NPARAM = O_B4 + 1;

typedef __nv_bfloat16 bf16;

// The hidden-layer weights as the scoring kernel's shared-memory operand
// images: nine 256 x 64 BF16 chunks (W1; W2 by 64-column K chunks; W3 the
// same), each laid out K-major with the 128-byte swizzle, 32 KB apiece, so
// that one bulk copy moves a chunk into shared memory as is.
constexpr int kWChunks = 9;
constexpr size_t kWChunkBytes = 256 * 64 * 2;

// Byte offset of W element (row r, column c) of layer `layer` (1..3) in the
// chunk images.
__host__ __device__ inline size_t wimg_offset(int layer, int r, int c) {
  const int chunk = layer == 1 ? 0 : (layer == 2 ? 1 : 5) + c / 64;
  const int k = c % 64;
  return (size_t)chunk * kWChunkBytes + (size_t)r * 128 + (size_t)(((k >> 3) ^ (r & 7)) * 16) + (size_t)(k & 7) * 2;
}

int train_step(mp_mlp* h, const bf16* X, const float* target, int B, float lr, cudaStream_t st);

}  // namespace mlpk
}  // namespace mp

struct mp_mlp {
  int device = 0;
  float* P = nullptr;   // master parameters
  float* G = nullptr;   // gradients
  float* M1 = nullptr;  // Adam first moment
  float* M2 = nullptr;  // Adam second moment
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2T = nullptr, *W3T = nullptr;
  unsigned char* Wimg = nullptr;   // kWChunks swizzled chunk images (scoring)
  int* status = nullptr;
  float* scalar = nullptr;   // loss accumulator
  int step = 0;
  double margin_bound = __builtin_inf();   // calibrated overestimation bound of the margin rule (none yet)
  // per-batch work buffers
  int ws_B = 0;
  void* ws = nullptr;
};
