// Internal declarations of the GB300 engine (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cstddef>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mapple.h"

#if defined(__CUDACC__)
#define MP_HD __host__ __device__ __forceinline__
#else
#define MP_HD inline
#endif

namespace mp {

constexpr int kMaxRank = MP_MAX_PROC_RANK;
constexpr int kMaxPrim = 200;

// ------------------------------------------------------------------ division
//
// Division by an invariant integer with a truncated reciprocal and one
// correction step (Granlund & Montgomery, PLDI 1994; Moller & Granlund,
// "Improved division by invariant integers", IEEE TC 2011).  With
// m = floor((2^W - 1) / d) we have n m / 2^W > n / d - 1 for every n < 2^W,
// so q0 = hi(n m) is either the quotient or one less; one compare fixes it.

MP_HD uint32_t umulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

MP_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

struct Div32 {
  uint32_t d, m;
};
struct Div64 {
  uint64_t d, m;
};

inline Div32 make_div32(uint32_t d) { return Div32{d, d ? 0xFFFFFFFFu / d : 0u}; }
inline Div64 make_div64(uint64_t d) { return Div64{d, d ? ~0ull / d : 0ull}; }

MP_HD uint32_t div32(uint32_t n, Div32 f) {
  uint32_t q = umulhi32(n, f.m);
  uint32_t r = n - q * f.d;
  return q + (r >= f.d ? 1u : 0u);
}
MP_HD void divmod32(uint32_t n, Div32 f, uint32_t& q, uint32_t& r) {
  q = umulhi32(n, f.m);
  r = n - q * f.d;
  if (r >= f.d) { q += 1; r -= f.d; }
}
MP_HD uint64_t div64(uint64_t n, Div64 f) {
  uint64_t q = umulhi64(n, f.m);
  uint64_t r = n - q * f.d;
  return q + (r >= f.d ? 1ull : 0ull);
}
MP_HD void divmod64(uint64_t n, Div64 f, uint64_t& q, uint64_t& r) {
  q = umulhi64(n, f.m);
  r = n - q * f.d;
  if (r >= f.d) { q += 1; r -= f.d; }
}

// ------------------------------------------------------------------ plan

enum PrimOp : int32_t { P_SPLIT = 0, P_MERGE = 1, P_SWAP = 2 };

// One primitive of the expanded chain, with what its inverse needs.
struct Prim {
  int32_t op;            // P_SPLIT / P_MERGE / P_SWAP
  int32_t p, q;          // split: p = i; merge / swap: p, q
  int32_t rank_before;   // rank of the space the primitive was applied to
  uint32_t d;            // split factor, or s_p of the merged space
  Div32 div;             // division by s_p (merge)
};

// A final-space coordinate as a function of one task coordinate x:
//   BLOCK  a = floor(x * s / L)
//   CYCLIC a = x mod s
//   BCYC   a = floor(x / b) mod s
enum CompKind : int32_t { C_BLOCK = 0, C_CYCLIC = 1, C_BCYC = 2 };

struct Comp {
  int32_t kind;
  uint32_t s;       // size of the final dimension
  uint32_t sigma;   // its stride in the flat final index F
  uint32_t b;       // block size (BCYC)
  uint64_t L;       // task extent along the owning dimension (L * s < 2^64)
  int32_t narrow;   // 1 when L * s < 2^32 (32-bit block arithmetic suffices)
  Div64 divL, divs64, divb64;
  Div32 divL32, divs, divb;
};

// Everything a kernel needs to map one index launch, except the primitive
// list.  The flat final index is F = sum_u a_u * sigma_u with dimension 0
// fastest (sigma_0 = 1).  Task dimension t drives the final coordinates of
// its components; their sub-index j_t = a_{c0} + s_{c0} * a_{c1} ranges over
// [0, J[t]) and indexes the per-dimension counts at Joff[t] + j_t.
struct MapCore {
  int32_t k;          // task rank
  int32_t lc;         // 1: linear-cyclic (F = lin mod P)
  int32_t rank;       // final processor-space rank
  int32_t nprim;
  uint32_t P, g;
  uint64_t npoints;
  uint64_t L[4];
  Div64 divL64[4];
  Div32 divL32[4];
  int32_t ncomp[4];
  Comp comp[4][2];
  uint32_t J[4], Joff[4], Jtotal;
  uint32_t s[kMaxRank];
  uint32_t sigma[kMaxRank];
  Div32 divs[kMaxRank];
  int32_t owner_dim[kMaxRank];
  int32_t owner_slot[kMaxRank];
  uint32_t lc_stride_mod[4];   // (prod_{u > t} L_u) mod P
  uint64_t lc_stride[4];       // prod_{u > t} L_u
  Div32 divP;
  Div64 divP64;
};

struct MapDesc : MapCore {
  Prim prim[kMaxPrim];
};

// Halo of the element-count mode for linear-cyclic launches (F = lin mod P):
// along dimension t the neighbours y + delta e_t, 1 <= |delta| <= w_t, of an
// element have flat indices F + delta * stride_t (mod P).  off[t][i] are the
// distinct non-zero offsets (delta stride_t mod P); pos / neg the smallest
// delta > 0 with +delta (resp. -delta) giving that offset, 0 if none.
constexpr int kMaxHaloWidth = MP_MAX_HALO_WIDTH;
struct LcHalo {
  uint32_t n[4];
  uint32_t off[4][2 * kMaxHaloWidth];
  uint8_t pos[4][2 * kMaxHaloWidth];
  uint8_t neg[4][2 * kMaxHaloWidth];
};

// Host-side plan: the descriptor plus the expanded primitive list.
struct HostPrim {
  int32_t op, p, q;
  int64_t d;
};

struct Plan {
  MapDesc desc;
  std::vector<HostPrim> prims;
  int rank;
  int64_t shape[kMaxRank];
};

// Build and validate a plan.  Returns MP_OK or an mp_status.
int build_plan(const mp_space* space, const mp_machine* machine, const mp_xform* chain, int n_xf,
               const mp_dist* dist, Plan& out);

// Ordered k-factorisations of d (lexicographic) and the decompose argmin.
std::vector<std::vector<int64_t>> ordered_factorisations(int64_t d, int k);
std::vector<int64_t> decompose_argmin(int64_t d, int k, const int64_t* l);
// With halo widths h (k values) and a transpose mask: the generalised
// objective; returns MP_EOVERFLOW when it does not fit in 127 bits.
int decompose_argmin_weighted(int64_t d, int k, const int64_t* l, const int64_t* h, int tmask,
                              std::vector<int64_t>& out);

// Canonical transform alphabet (split / merge / swap) of a shape.
struct CanonOp {
  int32_t op, p, q;
  int64_t d;
};
std::vector<CanonOp> canonical_alphabet(const std::vector<int64_t>& shape);
void apply_canon(std::vector<int64_t>& shape, const CanonOp& c);
std::vector<std::vector<CanonOp>> canonical_chains(int64_t nodes, int64_t ppn, int max_depth);

// C = A * B^T, BF16 operands (row-major, K contiguous), FP32 result (mlp.cu).
int gemm_tn(const void* A, const void* B, float* C, int M, int N, int K, int* status, cudaStream_t st);

// ------------------------------------------------------------------ runtime

// Grow-only per-device workspace; returns nullptr on allocation failure.
void* workspace(size_t bytes, int slot);
bool is_device_pointer(const void* p);
// Device address of a page-locked host allocation (written by kernels over
// the host link directly), or nullptr (also when MAPPLE_PINNED_DIRECT=0).
void* pinned_alias(const void* p);
void count_launch(uint64_t n = 1);
// One-shot events around the dominant kernel (mp_set_kernel_timer).
void timer_begin(cudaStream_t st);
void timer_end(cudaStream_t st);
// the same one-shot pair around the next launch of the learned scorer's layer kernel
void layer_timer_begin(cudaStream_t st);
void layer_timer_end(cudaStream_t st);

}  // namespace mp

namespace mp {
// Records where the last CUDA call failed (mp_last_error_detail).
void record_cuda_error(cudaError_t e, const char* file, int line);
}  // namespace mp

#define MP_CUDA_TRY(expr)                                      \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) {                                   \
      mp::record_cuda_error(_e, __FILE__, __LINE__);           \
      return MP_ECUDA;                                         \
    }                                                          \
  } while (0)
