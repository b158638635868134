// The learned cost model's parameters and training entry points (shared by
// mlp.cu and learned.cu).
#pragma once

#include <cuda_bf16.h>

#include "engine.h"

namespace mp {
namespace mlpk {

constexpr int DIN = 64, DH = 256;
constexpr size_t O_W1 = 0, O_B1 = O_W1 + DH * DIN, O_W2 = O_B1 + DH, O_B2 = O_W2 + DH * DH, O_W3 = O_B2 + DH,
                 O_B3 = O_W3 + DH * DH, O_W4 = O_B3 + DH, O_B4 = O_W4 + DH, NPARAM = O_B4 + 1;

typedef __nv_bfloat16 bf16;

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
  int* status = nullptr;
  float* scalar = nullptr;   // loss accumulator
  int step = 0;
  // per-batch work buffers
  int ws_B = 0;
  void* ws = nullptr;
};
