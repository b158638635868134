// Learned pruning of the decompose search (no counterpart in the paper).
//
//   features   64 numbers per candidate (query shape, factorisation, its
//              closed-form primary cost relative to the best one, the
//              chain's transforms, where the chain's node boundaries fall
//              along each final dimension)
//   scoring    k_feat_img writes the candidates' features as swizzled BF16
//              operand tiles (full occupancy hides the feature arithmetic's
//              latency); k_mlp_img, one persistent CTA per SM, runs the three
//              hidden layers of two tiles at a time as tcgen05 MMAs with FP32
//              accumulators in 512 TMEM columns: a copy warp streams the
//              weights in 16 KB slices through a five-deep ring, one MMA
//              warp per tile issues, and 16 epilogue warps apply bias and
//              ReLU (and the output dot product) by halves of the columns,
//              each half's epilogue under the other half's (and the other
//              tile's) MMAs
//   top-K      65536-bin histogram of the order-preserving score keys, a
//              threshold bin, and a compaction of the candidates at or below
//   exact      the top-K are re-evaluated by the exact cost kernel; the
//              lexicographic argmin over them is returned when it is
//              certified (every candidate with a primary cost no higher than
//              the winner's was evaluated) or when the model's observed error
//              leaves a margin; otherwise the exhaustive search runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "mlp.cuh"
#include "search.cuh"
#include "tc.cuh"

namespace mp {
namespace lrn {

using mlpk::bf16;
using mlpk::DH;
using mlpk::DIN;

constexpr int kChainFeat = 32;
constexpr uint32_t kWaitLimit = 1u << 26;

struct QInfo {
  uint32_t E[3];
  uint32_t P, n, g;
  uint32_t nf;
  uint32_t nd;   // divisors of P (entries of the fibre-node table, per step j)
  unsigned long long nchains;
  unsigned long long pmin;
  unsigned long long tile_bytes;
  float qf[6];
};

__device__ __forceinline__ float lg2(float v) { return log2f(fmaxf(v, 1e-30f)); }

// Per chain: depth one-hot, each of three steps (split / merge / swap,
// log2 d, p, q) and whether the node changes between flat index 0 and 2^i.
__global__ void k_chain_feats(const ChainProg* __restrict__ progs, unsigned long long NC, uint32_t P,
                              float* __restrict__ out) {
  const unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= NC) return;
  const ChainProg cp = progs[c];
  float f[kChainFeat];
  for (int i = 0; i < kChainFeat; ++i) f[i] = 0.f;
  f[min(cp.depth, 3)] = 1.f;
  for (int s = 0; s < 3 && s < cp.depth; ++s) {
    const Prim& p = cp.prim[s];
    f[4 + 6 * s + p.op] = 1.f;
    f[4 + 6 * s + 3] = p.op == P_SPLIT ? lg2((float)p.d) / 12.f : 0.f;
    f[4 + 6 * s + 4] = p.p / 4.f;
    f[4 + 6 * s + 5] = p.op == P_SPLIT ? 0.f : p.q / 4.f;
  }
  const uint32_t n0 = resolve_node(cp, 0);
  for (int i = 0; i < 10; ++i) {
    const uint32_t b = 1u << i;
    f[22 + i] = (b < P && resolve_node(cp, b) != n0) ? 1.f : 0.f;
  }
  // feature-major (feature i of every chain contiguous): the candidates a
  // warp scores have consecutive chains, so each feature load is coalesced
  for (int i = 0; i < kChainFeat; ++i) out[(unsigned long long)i * NC + c] = f[i];
}

// Fibre-node table: the node of flat index b of each chain, for b = 0 and
// b = j * D[k] (j = 1, 2, 3; D the ascending divisors of P), which are the
// first points of every fibre the features look at (fibre strides are
// products of leading factors, so divisors of P).  Entry-major, entry
// e = 0 or 1 + (j - 1) nd + k of chain c at e * NC + c; 0xFFFF where b >= P.
// One warp per chain, so that its lanes walk the same chain program.
// gtab (may be null): every chain's node table (rows of Pp entries), read
// instead of walking the chain program.
__global__ void k_fibre_nodes(const ChainProg* __restrict__ progs, unsigned long long NC, uint32_t P,
                              const uint32_t* __restrict__ D, uint32_t nd, const uint16_t* __restrict__ gtab,
                              uint32_t Pp, uint16_t* __restrict__ out) {
  const unsigned long long c = (unsigned long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (c >= NC) return;
  const ChainProg& cp = progs[c];
  const uint32_t W = 1 + 3 * nd;
  for (uint32_t e = threadIdx.x & 31; e < W; e += 32) {
    uint32_t b = 0;
    if (e > 0) b = (1 + (e - 1) / nd) * D[(e - 1) % nd];
    uint16_t v = 0xFFFF;
    if (b < P) v = gtab ? __ldg(gtab + c * Pp + b) : (uint16_t)resolve_node(cp, b);
    out[(unsigned long long)e * NC + c] = v;
  }
}

// 64 features of candidate idx = fr * NC + c.  fnode: the fibre-node table;
// fdiv[fr]: the divisor indices of f0 (low half) and f0 f1 (high half).
__device__ __forceinline__ void candidate_features(const QInfo& Q, const uint16_t* __restrict__ fnode,
                                                   const uint32_t* __restrict__ fdiv, const Fact* __restrict__ facts,
                                                   const float* __restrict__ chainfeat, unsigned long long idx,
                                                   float x[64], unsigned long long* primary_out) {
  const unsigned long long fr = idx / Q.nchains, c = idx - fr * Q.nchains;
  const uint32_t f[3] = {facts[fr].f[0], facts[fr].f[1], facts[fr].f[2]};
  const unsigned long long p = primary_cost(Q.E, f);
  if (primary_out) *primary_out = p;
  const float pn = (float)((double)p / (double)max(Q.pmin, 1ull) - 1.0);
  for (int i = 0; i < 6; ++i) x[i] = Q.qf[i];
  for (int t = 0; t < 3; ++t) {
    const float ft = (float)f[t], Et = (float)Q.E[t];
    x[6 + t] = lg2(ft) / 12.f;
    x[9 + t] = lg2(fminf(ft, Et)) / 12.f;
    x[12 + t] = f[t] > Q.E[t] ? 1.f : 0.f;
    x[15 + t] = fminf(fmaxf(lg2(Et / ft), -8.f), 12.f) / 12.f;
  }
  x[18] = fminf(pn, 8.f) / 8.f;
  x[19] = log2f(1.f + pn) / 3.f;
  x[20] = p == Q.pmin ? 1.f : 0.f;
  for (int i = 0; i < kChainFeat; ++i) x[21 + i] = __ldg(chainfeat + (unsigned long long)i * Q.nchains + c);
  const uint32_t n0 = __ldg(fnode + c);
  const uint32_t stride[3] = {1u, f[0], f[0] * f[1]};
  const uint32_t dv = __ldg(fdiv + fr);
  const uint32_t di[3] = {0u, dv & 0xFFFFu, dv >> 16};
  for (int v = 0; v < 3; ++v) {
    float ch = 0.f, distinct = 1.f;
    if (f[v] > 1 && stride[v] < Q.P) {
      uint32_t seen[4] = {n0, 0, 0, 0};
      int ns = 1;
      for (uint32_t j = 1; j < 4 && j < f[v] && j * stride[v] < Q.P; ++j) {
        const uint32_t nd = __ldg(fnode + (unsigned long long)(1 + (j - 1) * Q.nd + di[v]) * Q.nchains + c);
        if (j == 1) ch = nd != n0 ? 1.f : 0.f;
        bool dup = false;
        for (int a = 0; a < ns; ++a) dup = dup || seen[a] == nd;
        if (!dup) seen[ns++] = nd;
      }
      distinct = (float)ns;
    }
    x[53 + v] = ch;
    x[56 + v] = distinct / 4.f;
  }
  x[59] = log2f(1.f + (float)p) / 40.f;
  x[60] = 1.f;
  x[61] = x[62] = x[63] = 0.f;
}

// Regression target: the primary cost relative to the least one, then the
// secondary on a log scale (within the candidates of least primary only the
// second term varies, over a range of a few units).
__device__ __forceinline__ float target_of(unsigned long long p_tiles, unsigned long long s_tiles,
                                           unsigned long long pmin) {
  const float sec = log2f(1.f + (float)s_tiles) / 8.f;
  if (p_tiles == pmin) return sec;   // the same value (2 * 0 + sec) without a double division
  const float pn = (float)((double)p_tiles / (double)max(pmin, 1ull) - 1.0);
  return 2.f * fminf(pn, 16.f) + sec;
}


// Features (BF16, row-major n x 64) of listed candidates; with exact costs
// (bytes) also the regression targets.
__global__ void k_features_idx(const __grid_constant__ QInfo Q, const uint16_t* __restrict__ fnode,
                               const uint32_t* __restrict__ fdiv, const Fact* __restrict__ facts,
                               const float* __restrict__ chainfeat,
                               const int64_t* __restrict__ idx, int64_t n, const uint64_t* __restrict__ pbytes,
                               const uint64_t* __restrict__ sbytes, bf16* __restrict__ X, float* __restrict__ target) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[64];
  candidate_features(Q, fnode, fdiv, facts, chainfeat, (unsigned long long)idx[i], x, nullptr);
  for (int j = 0; j < 64; j += 2)
    *reinterpret_cast<__nv_bfloat162*>(X + i * 64 + j) = __floats2bfloat162_rn(x[j], x[j + 1]);
  if (target) target[i] = target_of(pbytes[i] / Q.tile_bytes, sbytes[i] / Q.tile_bytes, Q.pmin);
}

// ------------------------------------------------------------ scoring in two kernels
//
// k_feat_img writes the features of a run of scored candidates as BF16
// operand images (one 16 KB K-major, 128-byte swizzled tile of 128 rows per
// 128 candidates; rows past the end are zero) at full occupancy, where the
// latency of the feature arithmetic (chain walks, table loads) hides behind
// many resident warps.  k_mlp_img then runs the three layers on those tiles,
// two per pass (256 candidates), in a persistent CTA per SM.

constexpr uint32_t kTileBytes = 128 * 128;   // 128 rows x 64 BF16

__global__ void __launch_bounds__(128) k_feat_img(const __grid_constant__ QInfo Q, const uint16_t* __restrict__ fnode,
                                                  const uint32_t* __restrict__ fdiv, const Fact* __restrict__ facts,
                                                  const float* __restrict__ chainfeat,
                                                  const uint32_t* __restrict__ flist, unsigned long long c0,
                                                  unsigned long long n, uint8_t* __restrict__ img) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;   // < padded n
  float x[64];
  if (i < n) {
    const unsigned long long cand = c0 + i;
    unsigned long long idx = cand;
    if (flist) {
      const unsigned long long j = cand / Q.nchains;
      idx = (unsigned long long)flist[j] * Q.nchains + (cand - j * Q.nchains);
    }
    candidate_features(Q, fnode, fdiv, facts, chainfeat, idx, x, nullptr);
  } else {
    for (int j = 0; j < 64; ++j) x[j] = 0.f;
  }
  uint8_t* tile = img + (i / 128) * kTileBytes;
  const uint32_t row = (uint32_t)(i % 128);
#pragma unroll
  for (int j = 0; j < 64; j += 8) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat162 h2 = __floats2bfloat162_rn(x[j + 2 * e], x[j + 2 * e + 1]);
      w[e] = *reinterpret_cast<uint32_t*>(&h2);
    }
    *reinterpret_cast<uint4*>(tile + tc::sw128_offset(row, j)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// The layer kernel streams the weights in slices of half a chunk (the 128
// output features of one half by 64 K): 18 per pass of two tiles, through a
// ring of kSlots 16 KB buffers.  Layer 1 is slices (chunk 0, half 0) and
// (chunk 0, half 1); layers 2 and 3 take K chunks 0 and 1 of half 0, the same
// of half 1, then K chunks 2 and 3 of half 0 and of half 1.  So the layer's
// reads of activation atoms 0 and 1 are done before half 0 is complete (its
// epilogue writes them at once), half 0's epilogue runs under half 1's last
// MMAs, and the next layer starts on atom 0 while half 1's epilogue runs.
constexpr int kSlots = 5;
constexpr uint32_t kSliceBytes = 16384;
constexpr int kSlices = 2 * mlpk::kWChunks;
constexpr size_t kMlpSmem = 2 * 65536 + kSlots * kSliceBytes + 1024;

// 16 epilogue warps (warp w: tile (w >> 2) & 1, TMEM lanes 32 (w & 3) .. + 31,
// activation atom w >> 3 of each half), one MMA warp per tile (their MMAs
// interleave on the tensor pipe, so one tile's waits hide behind the other
// tile's MMAs) and the copy warp.  19 warps put five on three of the SM's four
// register-file quarters: 96 registers a thread at most.
constexpr int kEpiWarps = 16;
constexpr int kMmaWarp = kEpiWarps, kCopyWarp = kEpiWarps + 2;   // MMA warps kMmaWarp + t
constexpr int kMlpThreads = (kEpiWarps + 3) * 32;

// Slice s (0 .. 17) of a pass: layer l (0 .. 2), K chunk k and half h.
__host__ __device__ __forceinline__ void slice_of(int s, int& l, int& k, int& h) {
  if (s < 2) {
    l = 0;
    k = 0;
    h = s;
    return;
  }
  l = 1 + (s - 2) / 8;
  const int r = (s - 2) % 8;
  h = (r >> 1) & 1;
  k = (r & 1) + 2 * (r >> 2);
}

// Per tile t, every barrier but the ring's completes once per pass (phase
// parity = pass parity): xfull[t] (tile t's features landed in its atom 0),
// accfull[t][l][h] (tile t's MMA warp commit: half h of layer l
// accumulated), infree[t] (commit: layer 3's MMAs that read atoms 0 and 1
// done), part[t * 4 + q] (32 threads: the output's second partial sum
// written).  A ring buffer is refilled once both MMA warps committed its slice
// (empty: two arrivals).  The MMA warps wait on counters instead (eight
// epilogue warps add one per pass to each of tile t's): landed (slices whose
// weights landed, published in order by the copy warp), tfree[t][l][h] (half h
// of layer l's accumulators read from TMEM), ready[t][l][k] (activation atom k
// of layer l written).
struct LayerBars {
  uint64_t full[kSlots], empty[kSlots];
  uint64_t xfull[2], drain[2];
  uint64_t accfull[2][3][2];
  uint64_t infree[2];
  uint64_t part[8];
};
struct LayerCounts {
  uint32_t landed;
  uint32_t tfree[2][3][2];
  uint32_t ready[2][2][4];
};

// A bounded wait that also gives up early once another role has failed.
__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, volatile int* fail) {
#pragma unroll 1
  for (int i = 0; i < 64; ++i) {
    if (tc::mbar_wait(bar, parity, kWaitLimit / 64)) return true;
    if (*fail) return false;
  }
  *fail = 1;
  return false;
}

// Packed FP32 pairs (one instruction for two lanes, each rounded as the
// scalar operation would round it) and the ReLU-clamping BF16 conversion.
__device__ __forceinline__ unsigned long long f2_pack(uint32_t lo, uint32_t hi) {
  unsigned long long v;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "r"(lo), "r"(hi));
  return v;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// BF16 pair of max(lo, 0) and max(hi, 0), lo in the low half
__device__ __forceinline__ uint32_t relu_bf16x2(unsigned long long v) {
  uint32_t d;
  asm("{\n\t.reg .b32 lo, hi;\n\t"
      "mov.b64 {lo, hi}, %1;\n\t"
      "cvt.rn.relu.bf16x2.f32 %0, hi, lo;\n\t}"
      : "=r"(d)
      : "l"(v));
  return d;
}
// Shared-memory event counters: a release add (or store) by the signalling
// thread; the waiting one polls with relaxed loads and fences once the count
// is reached.  A completed mbarrier phase takes
// about 200 cycles to observe, an acquire load of a counter a fraction of
// that, so the MMA warps, whose waits sit between the tensor pipe's work,
// wait on counters; the barriers stay where the hardware signals them (bulk
// copies, MMA commits).
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(tc::smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(tc::smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(tc::smem_u32(p)), "r"(v) : "memory");
}
// Waits (bounded) until the counter reaches target; gives up early once
// another role has failed.
__device__ __forceinline__ bool wait_count(const uint32_t* p, uint32_t target, volatile int* fail) {
#pragma unroll 1
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    if (ld_relaxed(p) >= target) {
      asm volatile("fence.acq_rel.cta;" ::: "memory");   // with the load: an acquire
      return true;
    }
    if ((i & 1023) == 1023 && *fail) return false;
  }
  *fail = 1;
  return false;
}

__device__ __forceinline__ unsigned long long f2_relu(unsigned long long v) {
  uint32_t lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(v));
  return f2_pack(__float_as_uint(fmaxf(__uint_as_float(lo), 0.f)), __float_as_uint(fmaxf(__uint_as_float(hi), 0.f)));
}

__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_img(const uint8_t* __restrict__ img, uint32_t ntiles,
                                                    const uint8_t* __restrict__ Wimg, const float* __restrict__ P,
                                                    unsigned long long n, float* __restrict__ scores,
                                                    int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ LayerBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  __shared__ LayerCounts cnt;
  __shared__ uint32_t s_xwaited[2];   // per MMA warp: feature tiles seen landed
  __shared__ __align__(16) float sb[4][256];   // b1, b2, b3, w4
  __shared__ float s_part[2][2][128];          // [pass parity][tile][row]: the output's second partial sum
  uint8_t* base = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
  // tile t's four 16 KB activation atoms at base + t * 65536 (atom 0 holds X in layer 1)
  uint8_t* ring = base + 131072;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t npass = ntiles > 2 * blockIdx.x ? (ntiles - 2 * blockIdx.x + 2 * gridDim.x - 1) / (2 * gridDim.x) : 0;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    sb[0][i] = __ldg(P + mlpk::O_B1 + i);
    sb[1][i] = __ldg(P + mlpk::O_B2 + i);
    sb[2][i] = __ldg(P + mlpk::O_B3 + i);
    sb[3][i] = __ldg(P + mlpk::O_W4 + i);
  }
  const float b4 = __ldg(P + mlpk::O_B4);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, 512);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < kSlots; ++i) {
      tc::mbar_init(&bars.full[i], 1);
      tc::mbar_init(&bars.empty[i], 2);
    }
    cnt.landed = 0;
    for (int t = 0; t < 2; ++t) {
      s_xwaited[t] = 0;
      tc::mbar_init(&bars.xfull[t], 1);
      tc::mbar_init(&bars.drain[t], 1);
      tc::mbar_init(&bars.infree[t], 1);
      for (int i = 0; i < 2; ++i) {
        for (int l = 0; l < 3; ++l) {
          tc::mbar_init(&bars.accfull[t][l][i], 1);
          cnt.tfree[t][l][i] = 0;
        }
        for (int k = 0; k < 4; ++k) cnt.ready[t][i][k] = 0;
      }
    }
    for (int i = 0; i < 8; ++i) tc::mbar_init(&bars.part[i], 32);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  // copy thread: feature tiles and slices whose copies were issued, slices published as landed
  uint32_t x_issued[2] = {0, 0}, issued = 0, pub = 0;
  if (warp == kCopyWarp) {
    if (lane == 0) {
      // slices are published (cnt.landed) in order as their copies land;
      // every wait of this thread keeps publishing meanwhile
      auto publish = [&]() {
        while (pub < issued && tc::mbar_test(&bars.full[pub % kSlots], (pub / kSlots) & 1)) st_release(&cnt.landed, ++pub);
      };
      auto wait_publishing = [&](uint64_t* bar, uint32_t parity) -> bool {
#pragma unroll 1
        for (uint32_t i = 0; i < kWaitLimit; ++i) {
          if (tc::mbar_test(bar, parity)) return true;
          publish();
          if ((i & 255) == 255 && s_fail) return false;
        }
        s_fail = 1;
        return false;
      };
      bool ok = true;
      for (uint32_t pass = 0; pass < npass && ok && !s_fail; ++pass) {
        // each feature tile goes into its atom 0 once the previous pass's
        // layer 3 has read it; a missing second tile (odd count, last pass)
        // completes its barrier with a plain arrival
        const uint32_t tA = 2 * (blockIdx.x + pass * gridDim.x);
        const uint32_t nt = tA + 1 < ntiles ? 2 : 1;
        for (uint32_t t = 0; t < 2 && ok; ++t) {
          if (pass > 0 && !(ok = wait_publishing(&bars.infree[t], (pass - 1) & 1))) break;
          if (t < nt) {
            tc::mbar_expect_tx(&bars.xfull[t], kTileBytes);
            tc::bulk_g2s(base + t * 65536, img + (size_t)(tA + t) * kTileBytes, kTileBytes, &bars.xfull[t]);
          } else {
            tc::mbar_arrive(&bars.xfull[t]);
          }
          ++x_issued[t];
        }
        for (int s = 0; s < kSlices && ok; ++s) {
          const uint32_t G = pass * kSlices + s, slot = G % kSlots, use = G / kSlots;
          if (use >= 1 && !(ok = wait_publishing(&bars.empty[slot], (use - 1) & 1))) break;
          int l, k, h;
          slice_of(s, l, k, h);
          const int chunk = l == 0 ? 0 : 1 + 4 * (l - 1) + k;
          tc::mbar_expect_tx(&bars.full[slot], kSliceBytes);
          tc::bulk_g2s(ring + slot * kSliceBytes, Wimg + (size_t)chunk * mlpk::kWChunkBytes + h * kSliceBytes,
                       kSliceBytes, &bars.full[slot]);
          ++issued;
          publish();
        }
      }
      // the last slices
#pragma unroll 1
      for (uint32_t i = 0; ok && pub < issued; ++i) {
        publish();
        if (i == kWaitLimit) s_fail = 1;
        if (s_fail) break;
      }
    }
  } else if (warp == kMmaWarp || warp == kMmaWarp + 1) {
    if (lane == 0) {
      const uint32_t t = warp - kMmaWarp;   // this warp's tile
      constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
      // operand descriptors of the tile's atom 0 and of ring buffer 0; the
      // others are byte offsets / 16 added to the start-address field
      const uint64_t adesc0 = tc::sdesc_sw128(tc::smem_u32(base + t * 65536));
      const uint64_t bdesc0 = tc::sdesc_sw128(tc::smem_u32(ring));
      const uint32_t dt = tmem + t * 256;
      uint32_t slot = 0;   // ring buffer of the next slice
      uint32_t consumed = 0, xwaited = 0;
      for (uint32_t pass = 0; pass < npass && !s_fail; ++pass) {
        const uint32_t ph = pass & 1;
        const uint32_t tA = 2 * (blockIdx.x + pass * gridDim.x);
        // a missing second tile still takes part in the barriers, without MMAs
        const bool live = tA + t < ntiles;
        if (!wait_or_fail(&bars.xfull[t], ph, &s_fail)) break;
        xwaited = pass + 1;
        bool ok = true;
        // the slice schedule unrolled: layer, K chunk and half are constants
#pragma unroll
        for (int s = 0; s < kSlices; ++s) {
          int l, k, h;
          slice_of(s, l, k, h);
          // layer 1 overwrites the accumulators the previous pass's output
          // layer read; in layers 2 and 3 half 0's slices wait for the atom
          // they read (atom 0's written after half 0's TMEM was read), half
          // 1's first slice for half 1's TMEM read
          if (l == 0 && pass > 0) ok = wait_count(&cnt.tfree[t][2][h], 8 * pass, &s_fail);
          if (ok && l >= 1 && h == 0) ok = wait_count(&cnt.ready[t][l - 1][k], 8 * (pass + 1), &s_fail);
          if (ok && l >= 1 && h == 1 && k == 0) ok = wait_count(&cnt.tfree[t][l - 1][1], 8 * (pass + 1), &s_fail);
          if (ok) ok = wait_count(&cnt.landed, consumed + 1, &s_fail);
          if (!ok) break;
          ++consumed;
          tc::fence_after_sync();
          if (live) {
            const uint64_t bd = bdesc0 + slot * (kSliceBytes >> 4);
            const uint64_t ad = adesc0 + ((k * 16384) >> 4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_bf16(dt + h * 128, ad + 2 * kk, bd + 2 * kk, idesc, (k == 0 && kk == 0) ? 0u : 1u);
          }
          tc::mma_commit(&bars.empty[slot]);
          if (l == 0 || k == 3) tc::mma_commit(&bars.accfull[t][l][h]);
          if (l == 2 && h == 1 && k == 1) tc::mma_commit(&bars.infree[t]);
          if (++slot == kSlots) slot = 0;
        }
        if (!ok) break;
      }
      s_xwaited[t] = xwaited;
      // every MMA issued has completed before the CTA goes on
      tc::mma_commit(&bars.drain[t]);
      if (!tc::mbar_wait(&bars.drain[t], 0, kWaitLimit)) s_fail = 1;
    }
  } else {
    const uint32_t t = ((uint32_t)warp >> 2) & 1, q = warp & 3, a = warp >> 3;
    const uint32_t row = q * 32 + lane;
    const uint32_t tq = tmem + ((q * 32) << 16) + t * 256;   // this warp's TMEM lanes, the tile's columns
    bool ok = true;
    for (uint32_t pass = 0; pass < npass && ok; ++pass) {
      const uint32_t ph = pass & 1;
      unsigned long long acc2 = 0;   // the output layer's partial dot product (even, odd columns)
      for (int l = 0; l < 3 && ok; ++l) {
        for (int h = 0; h < 2; ++h) {
          if (!(ok = wait_or_fail(&bars.accfull[t][l][h], ph, &s_fail))) break;
          tc::fence_after_sync();
          // this warp's columns of atoms 2h and 2h + 1 (warp a: columns
          // 32a .. 32a + 31 of each) are read from TMEM first, and the half's
          // TMEM is released; then each atom is finished and published
          uint32_t r0[32], r1[32];
          const int c0 = h * 128 + a * 32, c1 = c0 + 64;
          tc::tmem_ld32(tq + c0, r0);
          tc::tmem_ld32(tq + c1, r1);
          tc::tmem_ld_wait();
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) red_release_add(&cnt.tfree[t][l][h], 1);
          if (l == 2) {
            // relu(z + b3) . w4, even and odd columns in the two lanes of a
            // packed pair
            const unsigned long long* b3 = reinterpret_cast<const unsigned long long*>(sb[2]);
            const unsigned long long* w4 = reinterpret_cast<const unsigned long long*>(sb[3]);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              acc2 = f2_fma(f2_relu(f2_add(f2_pack(r0[2 * j], r0[2 * j + 1]), b3[c0 / 2 + j])), w4[c0 / 2 + j], acc2);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              acc2 = f2_fma(f2_relu(f2_add(f2_pack(r1[2 * j], r1[2 * j + 1]), b3[c1 / 2 + j])), w4[c1 / 2 + j], acc2);
            continue;
          }
          // layer 1's half 0 goes where its input (atom 0) is: wait for the
          // layer's last MMAs
          if (l == 0 && h == 0 && !(ok = wait_or_fail(&bars.accfull[t][0][1], ph, &s_fail))) break;
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            // bias, ReLU, BF16 pairs of the 32 columns
            const unsigned long long* bias = reinterpret_cast<const unsigned long long*>(sb[l] + (i ? c1 : c0));
            const uint32_t* r = i ? r1 : r0;
            uint32_t w[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = relu_bf16x2(f2_add(f2_pack(r[2 * j], r[2 * j + 1]), bias[j]));
            uint8_t* atom = base + t * 65536 + (2 * h + i) * 16384;
#pragma unroll
            for (int j = 0; j < 4; ++j)
              *reinterpret_cast<uint4*>(atom + tc::sw128_offset(row, 8 * (4 * a + j))) =
                  make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) red_release_add(&cnt.ready[t][l][2 * h + i], 1);
          }
        }
      }
      if (!ok) break;
      // the two warps of a (tile, lane quarter) add their halves of the dot
      // product; the second writes, the first adds and stores the score
      const uint32_t tA = 2 * (blockIdx.x + pass * gridDim.x);
      const uint32_t nt = tA + 1 < ntiles ? 2 : 1;
      uint32_t a_even, a_odd;
      asm("mov.b64 {%0, %1}, %2;" : "=r"(a_even), "=r"(a_odd) : "l"(acc2));
      const float acc = __uint_as_float(a_even) + __uint_as_float(a_odd);
      if (a == 1) {
        s_part[ph][t][row] = acc;
        tc::mbar_arrive(&bars.part[t * 4 + q]);
      } else {
        if (!(ok = wait_or_fail(&bars.part[t * 4 + q], ph, &s_fail))) break;
        const unsigned long long out = (unsigned long long)(tA + t) * 128 + row;
        if (t < nt && out < n) scores[out] = acc + s_part[ph][t][row] + b4;
      }
    }
  }
  __syncthreads();
  if (warp == kCopyWarp && lane == 0 && s_fail) {
    // copies issued but not seen landed (at most one per ring buffer, and
    // one feature tile each) complete before the CTA exits
    for (uint32_t G = pub; G < issued; ++G)
      tc::mbar_wait(&bars.full[G % kSlots], (G / kSlots) & 1, kWaitLimit);
    for (int t = 0; t < 2; ++t)
      if (x_issued[t] > s_xwaited[t]) tc::mbar_wait(&bars.xfull[t], (x_issued[t] - 1) & 1, kWaitLimit);
    atomicExch(status, MP_ETIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------ top-K

__device__ __forceinline__ uint32_t order_key(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The score of an order key: the inverse of order_key.
__device__ __forceinline__ float key_value(uint32_t key) {
  return __uint_as_float((key & 0x80000000u) ? (key ^ 0x80000000u) : ~key);
}

// Zeroes one selection's counters: the 65536 fine and 256 coarse bins of the
// score histogram and `words` more counter words after them.
__global__ void k_sel_init(unsigned* __restrict__ hist, unsigned words) {
  const unsigned n = 65536 + 256 + words;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) hist[i] = 0;
}

// 65536-bin histogram of the order keys' upper halves and a 256-bin coarse
// one of their top bytes (per CTA in shared memory, then added to the
// global one).  The scores crowd into few bins, so the lanes of a warp that
// share a bin add once; nonfinite counts the NaN / infinite scores (a model
// that produced one gets no margin).
__global__ void k_topk_hist(const float* __restrict__ s, unsigned long long n, unsigned* __restrict__ hist,
                            unsigned* __restrict__ coarse, unsigned* __restrict__ nonfinite) {
  __shared__ unsigned c[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) c[i] = 0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  unsigned bad = 0;
  for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x; i0 < n;
       i0 += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const bool in = i < n;
    const float v = in ? s[i] : 0.f;
    const uint32_t key = order_key(v);
    const unsigned fine = in ? key >> 16 : 0xFFFFFFFFu, top = in ? key >> 24 : 0xFFFFFFFFu;
    const unsigned pf = __match_any_sync(0xFFFFFFFFu, fine), pt = __match_any_sync(0xFFFFFFFFu, top);
    if (in && lane == (unsigned)(__ffs(pf) - 1)) atomicAdd(hist + fine, (unsigned)__popc(pf));
    if (in && lane == (unsigned)(__ffs(pt) - 1)) atomicAdd(c + top, (unsigned)__popc(pt));
    bad += in && !isfinite(v);
  }
  if (bad) atomicAdd(nonfinite, bad);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (c[i]) atomicAdd(coarse + i, c[i]);
}

// Inclusive prefix sum over a CTA of 256 threads (8 warps).
__device__ __forceinline__ unsigned block_scan256(unsigned v, unsigned* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  unsigned add = 0;
  for (int w = 0; w < warp; ++w) add += warp_tot[w];
  __syncthreads();
  return v + add;
}

// Smallest bin T whose cumulative count reaches K, through the coarse
// histogram (256 bins of 256 fine bins each) then the fine bins of the
// chosen coarse bin.  out[0] = T, out[1] = count below T; out[2] = the first
// bin not yet selected: 0, or with grow set one past the previous threshold
// (out[0] on entry).  Also resets the collection's counters (cnt[0], cnt[1])
// and its least left-out key (cnt[2]).  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_topk_threshold(const unsigned* __restrict__ hist,
                                                        const unsigned* __restrict__ coarse, unsigned K, int grow,
                                                        unsigned* __restrict__ out, unsigned* __restrict__ cnt) {
  __shared__ unsigned warp_tot[8];
  __shared__ unsigned pick[2];
  const unsigned t = threadIdx.x;
  const unsigned prev = out[0];
  if (t < 3) cnt[t] = t < 2 ? 0u : 0xFFFFFFFFu;   // the collection's counts and least left-out key
  const unsigned cc = coarse[t];
  const unsigned cum_c = block_scan256(cc, warp_tot);
  if (cum_c - cc < K && cum_c >= K) {
    pick[0] = t;
    pick[1] = cum_c - cc;
  }
  __syncthreads();
  const unsigned C = pick[0], base = pick[1];
  const unsigned h = hist[C * 256 + t];
  const unsigned cum = base + block_scan256(h, warp_tot);
  if (cum - h < K && cum >= K) {
    out[0] = C * 256 + t;
    out[1] = cum - h;
    out[2] = grow ? prev + 1 : 0;
  }
}

// positions whose bin b has lo <= b < T (below) and b == T (eq), with
// T = thr[0], lo = thr[2]: everything up to the threshold on the first
// selection, only what is new on a growth round; and the least order key
// among the positions left out (bins above T) into *key_out (one atomic per
// warp; *key_out starts at ~0)
__global__ void k_topk_collect(const float* __restrict__ s, unsigned long long n, const unsigned* __restrict__ thr,
                               int64_t* __restrict__ below, unsigned* __restrict__ nbelow,
                               int64_t* __restrict__ eq, unsigned* __restrict__ neq, unsigned cap_below,
                               unsigned cap_eq, unsigned* __restrict__ key_out) {
  const unsigned T = thr[0], lo = thr[2];
  unsigned least = 0xFFFFFFFFu;
  for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x; i0 < n;
       i0 += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    if (i >= n) break;
    const uint32_t key = order_key(s[i]);
    const unsigned b = key >> 16;
    if (b > T) least = min(least, key);
    if (b < lo || b > T) continue;
    if (b < T) {
      const unsigned k = atomicAdd(nbelow, 1u);
      if (k < cap_below) below[k] = (int64_t)i;
    } else {
      const unsigned k = atomicAdd(neq, 1u);
      if (k < cap_eq) eq[k] = (int64_t)i;
    }
  }
  least = __reduce_min_sync(0xFFFFFFFFu, least);
  if ((threadIdx.x & 31) == 0 && least != 0xFFFFFFFFu) atomicMin(key_out, least);
}


// Exact costs of a selection, one warp per selected candidate (warps stride
// over the selection).  Each warp holds its candidate's chain table (Pp
// uint16, copied from the space's cache) and its lanes' bitmaps (words x 32)
// in its own part of shared memory, so no barrier spans the CTA; the cost is
// the exhaustive search's warp routine.  The selection is the scored
// positions listed in list_a (count *cnt_a, at most cap_a) followed by those
// in list_b (*cnt_b, at most cap_b); with list_a null it is positions
// 0 .. n_identity - 1.  A position maps to a candidate through the scored
// factorisations (flist).  Outputs per entry, from entry out0 on (at most
// out_cap entries in all): candidate index, primary and secondary (tiles),
// score.
__global__ void k_sel_costs(const ChainProg* __restrict__ progs, const Fact* __restrict__ facts,
                            unsigned long long nchains, uint32_t P, uint32_t E0, uint32_t E1,
                            uint32_t E2, int words, const uint16_t* __restrict__ gtab, uint32_t Pp,
                            const uint32_t* __restrict__ flist, const int64_t* __restrict__ list_a,
                            const unsigned* __restrict__ cnt_a, unsigned cap_a, const int64_t* __restrict__ list_b,
                            const unsigned* __restrict__ cnt_b, unsigned cap_b, unsigned long long n_identity,
                            const float* __restrict__ scores, unsigned long long out0, unsigned long long out_cap,
                            int64_t* __restrict__ sel_idx, uint64_t* __restrict__ sel_p, uint64_t* __restrict__ sel_s,
                            float* __restrict__ sel_y, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t tab_bar[8];   // one per warp: its chain table's bulk copy
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = (size_t)Pp * 2 + (size_t)words * 32 * 4;   // Pp is a multiple of 8: 16-byte aligned
  uint16_t* tab = reinterpret_cast<uint16_t*>(smem_raw + wib * per_warp);
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw + wib * per_warp + (size_t)Pp * 2);
  uint64_t* bar = &tab_bar[wib];
  for (int w = 0; w < words; ++w) bm[w * 32 + lane] = 0;   // the routine leaves its bitmaps cleared
  if (lane == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  __syncwarp();
  uint32_t phase = 0;
  unsigned long long na, n;
  if (list_a) {
    na = min(*cnt_a, cap_a);
    n = na + min(*cnt_b, cap_b);
  } else {
    na = n = n_identity;
  }
  if (out0 >= out_cap) return;
  n = min(n, out_cap - out0);   // entries beyond the arrays are dropped (the reduction sees the selection incomplete)
  const uint32_t E[3] = {E0, E1, E2};
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  for (unsigned long long i = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib; i < n; i += nwarps) {
    const unsigned long long pos = !list_a ? i : (i < na ? (unsigned long long)list_a[i]
                                                         : (unsigned long long)list_b[i - na]);
    const unsigned long long j = pos / nchains, c = pos - j * nchains;
    const unsigned long long fr = flist[j];
    if (gtab) {
      // the chain's cached table in one bulk copy (Pp * 2 bytes, 16-byte aligned rows)
      if (lane == 0) {
        tc::fence_proxy_async();   // the previous candidate's reads of tab come first
        tc::mbar_expect_tx(bar, Pp * 2);
        tc::bulk_g2s(tab, gtab + c * Pp, Pp * 2, bar);
      }
      const bool ok = __all_sync(0xFFFFFFFFu, tc::mbar_wait(bar, phase, kWaitLimit));
      phase ^= 1;
      if (!ok) {
        if (lane == 0) atomicExch(status, MP_ETIMEOUT);
        tc::mbar_wait(bar, phase ^ 1, kWaitLimit);   // the copy may still land: let it, then stop
        return;
      }
    } else {   // the space's tables were too large to cache: resolve every flat index
      const ChainProg cp = progs[c];
      for (uint32_t b = lane; b < P; b += 32) tab[b] = (uint16_t)resolve_node(cp, b);
      __syncwarp();
    }
    const uint32_t f[3] = {facts[fr].f[0], facts[fr].f[1], facts[fr].f[2]};
    const unsigned long long sec = secondary_cost_warp<true, true>(tab, bm, 32, words, E, f, lane);
    if (lane == 0) {
      sel_idx[out0 + i] = (int64_t)(fr * nchains + c);
      sel_p[out0 + i] = primary_cost(E, f);
      sel_s[out0 + i] = sec;
      sel_y[out0 + i] = scores[pos];
    }
    __syncwarp();   // the next candidate's table overwrites this one
  }
}

// What the host reads back after a selection: the selection's argmin and
// the acceptance test, decided on the device.
struct SelResult {
  int64_t idx;                 // winner's candidate index
  unsigned long long p, s;     // winner's primary / secondary (tiles)
  unsigned n;                  // selection size
  int cert;                    // 0 none, 1 every threat evaluated, 2 lower bound, 3 margin rule
  float tau;                   // the least score left out (infinite: none)
  float y_best;                // the winner's regression target
  float over;                  // largest score - target on the selection
  float margin;                // tau - y_best - the calibrated bound (margin rule)
  int complete;                // every entry at or below the threshold bin was evaluated
  int pad;
};

// One CTA of 256 threads: argmin of (primary, secondary, index) over the
// selection (the n_prev entries of earlier rounds and this round's new
// ones), then the acceptance rule.  Certificates: (1) the selection
// holds every candidate of least primary (threats_pmin of them), or (2) the
// winner's secondary reaches min_lb, a lower bound on every least-primary
// candidate's secondary.  Margin rule (heuristic): every candidate left out
// scored at least tau; it can beat the winner only if the model
// overestimated it by more than tau - y_best, which the calibrated bound
// says does not happen (accepted when tau - y_best exceeds it).
__global__ void __launch_bounds__(256) k_sel_reduce(const unsigned* __restrict__ cnt, unsigned cap_a,
                                                      unsigned cap_b, unsigned n_prev, int prev_complete,
                                                      unsigned out_cap, const unsigned* __restrict__ thr,
                                                      const int64_t* __restrict__ sel_idx,
                                                      const uint64_t* __restrict__ sel_p,
                                                      const uint64_t* __restrict__ sel_s,
                                                      const float* __restrict__ sel_y, unsigned long long pmin,
                                                      unsigned long long min_lb, unsigned long long threats_pmin,
                                                      float rule_bound, const unsigned* __restrict__ nonfinite,
                                                      SelResult* __restrict__ out) {
  __shared__ Key redk[32];
  __shared__ float redo[32];
  __shared__ unsigned redn[32];
  const unsigned n_new = min(cnt[0], cap_a) + min(cnt[1], cap_b);
  const unsigned n = min(n_prev + n_new, out_cap);
  Key best{~0ull, ~0ull, ~0ull};
  float over = -INFINITY;
  unsigned n_pmin = 0;
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
    const Key k{sel_p[i], sel_s[i], (unsigned long long)sel_idx[i]};
    if (key_less(k, best)) best = k;
    over = fmaxf(over, sel_y[i] - target_of(k.p, k.s, pmin));
    n_pmin += k.p == pmin;
  }
  for (int o = 16; o > 0; o >>= 1) {
    over = fmaxf(over, __shfl_down_sync(0xFFFFFFFFu, over, o));
    n_pmin += __shfl_down_sync(0xFFFFFFFFu, n_pmin, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    redo[warp] = over;
    redn[warp] = n_pmin;
  }
  block_argmin(best, redk);   // synchronises the CTA; warp 0 holds the result
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      over = fmaxf(over, redo[w]);
      n_pmin += redn[w];
    }
    SelResult r;
    r.idx = (int64_t)best.idx;
    r.p = best.p;
    r.s = best.s;
    r.n = n;
    r.complete = prev_complete && cnt[0] <= cap_a && cnt[1] <= cap_b && n_prev + n_new <= out_cap;
    r.tau = cnt[2] == 0xFFFFFFFFu ? INFINITY : key_value(cnt[2]);   // the least score left out
    r.y_best = target_of(best.p, best.s, pmin);
    r.over = over;
    r.margin = r.tau - r.y_best - rule_bound;
    const bool at_pmin = n > 0 && best.p == pmin;
    r.cert = 0;
    if (at_pmin && n_pmin == threats_pmin) r.cert = 1;
    else if (at_pmin && best.s <= min_lb) r.cert = 2;
    else if (at_pmin && r.complete && *nonfinite == 0 && isfinite(rule_bound) && r.margin > 0.f) r.cert = 3;
    r.pad = 0;
    *out = r;
  }
}

// ------------------------------------------------------------ host side

int sm_count_l() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 132;
  }
  return n;
}

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

struct Pool {
  char* p = nullptr;
  size_t size = 0;
  ~Pool() {
    if (p) cudaFree(p);
  }
  char* get(size_t bytes) {
    if (size >= bytes) return p;
    if (p) cudaFree(p);
    p = nullptr;
    size = 0;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    size = bytes;
    return p;
  }
};

Pool g_pool_s;   // scores and selection

Pool g_pool_img;   // feature tile images of the scoring kernels

// Pinned host staging for the selection's small transfers (grows, never shrinks).
struct HostPool {
  char* p = nullptr;
  size_t size = 0;
  ~HostPool() {
    if (p) cudaFreeHost(p);
  }
  char* get(size_t bytes) {
    if (size >= bytes) return p;
    if (p) cudaFreeHost(p);
    p = nullptr;
    size = 0;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    size = bytes;
    return p;
  }
} g_host_stage;

// What the model reads of a candidate space besides the search's own copy,
// built once per space: chain features, the fibre-node table and each
// factorisation's divisor indices.  The 8 most recent spaces are kept.
struct LearnedSpace {
  std::shared_ptr<const SpaceCore> core;
  char* mem = nullptr;
  float* chainfeat = nullptr;
  uint16_t* fnode = nullptr;
  uint32_t* fdiv = nullptr;
  uint32_t nd = 0;
  int device = -1;
};
std::mutex g_lspace_mu;
std::vector<std::shared_ptr<LearnedSpace>> g_lspaces;

struct LearnedSpaceFree {
  ~LearnedSpaceFree() {
    for (auto& l : g_lspaces)
      if (l->mem) cudaFree(l->mem);
  }
} g_lspace_free;

int learned_space(const SearchSpace& S, const DeviceSpace& Dv, uint32_t P, cudaStream_t st,
                  std::shared_ptr<LearnedSpace>* out) {
  int device = 0;
  MP_CUDA_TRY(cudaGetDevice(&device));
  std::lock_guard<std::mutex> lk(g_lspace_mu);
  for (size_t i = 0; i < g_lspaces.size(); ++i)
    if (g_lspaces[i]->core == S.c) {
      if (g_lspaces[i]->device != device) return MP_ENOTSUP;
      auto hit = g_lspaces[i];
      g_lspaces.erase(g_lspaces.begin() + (long)i);
      g_lspaces.insert(g_lspaces.begin(), hit);
      *out = hit;
      return MP_OK;
    }
  const size_t NC = S.c->chains.size(), NF = S.c->facts.size();
  std::vector<uint32_t> D;
  for (uint32_t d = 1; d <= P; ++d)
    if (P % d == 0) D.push_back(d);
  const uint32_t nd = (uint32_t)D.size();
  std::vector<uint32_t> fdiv(NF);
  for (size_t i = 0; i < NF; ++i) {
    const uint32_t f0 = (uint32_t)S.c->facts[i][0], f01 = f0 * (uint32_t)S.c->facts[i][1];
    const uint32_t a = (uint32_t)(std::lower_bound(D.begin(), D.end(), f0) - D.begin());
    const uint32_t b = (uint32_t)(std::lower_bound(D.begin(), D.end(), f01) - D.begin());
    fdiv[i] = a | (b << 16);
  }
  const size_t W = 1 + 3 * (size_t)nd;
  const size_t o_cf = 0, o_fn = o_cf + a256(NC * kChainFeat * 4), o_fd = o_fn + a256(NC * W * 2),
               o_D = o_fd + a256(NF * 4), end = o_D + a256(nd * 4);
  auto ls = std::make_shared<LearnedSpace>();
  if (cudaMalloc(&ls->mem, end) != cudaSuccess) {
    cudaGetLastError();
    return MP_ENOMEM;
  }
  ls->core = S.c;
  ls->chainfeat = (float*)(ls->mem + o_cf);
  ls->fnode = (uint16_t*)(ls->mem + o_fn);
  ls->fdiv = (uint32_t*)(ls->mem + o_fd);
  ls->nd = nd;
  ls->device = device;
  uint32_t* d_D = (uint32_t*)(ls->mem + o_D);
  bool ok = cudaMemcpyAsync(ls->fdiv, fdiv.data(), NF * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(d_D, D.data(), nd * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok) {
    k_chain_feats<<<(unsigned)((NC + 127) / 128), 128, 0, st>>>(Dv.progs, NC, P, ls->chainfeat);
    k_fibre_nodes<<<(unsigned)((NC + 3) / 4), 128, 0, st>>>(Dv.progs, NC, P, d_D, nd, Dv.tab, Dv.Pp, ls->fnode);
    count_launch(2);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    cudaFree(ls->mem);
    return MP_ECUDA;
  }
  g_lspaces.insert(g_lspaces.begin(), ls);
  if (g_lspaces.size() > 8) {
    cudaFree(g_lspaces.back()->mem);   // waits for the device: no kernel still reads it
    g_lspaces.back()->mem = nullptr;
    g_lspaces.pop_back();
  }
  *out = ls;
  return MP_OK;
}

struct Prepared {
  SearchSpace S;
  QInfo Q;
  const DeviceSpace* D = nullptr;          // the space's device copy (chain programs, factorisations, node tables)
  std::shared_ptr<LearnedSpace> L;         // the space's model inputs (chain features, fibre nodes, divisors)
  const ChainProg* d_progs = nullptr;
  const Fact* d_facts = nullptr;
  const float* d_chainfeat = nullptr;
  const uint16_t* d_fnode = nullptr;   // fibre-node table (k_fibre_nodes)
  const uint32_t* d_fdiv = nullptr;    // per factorisation: divisor indices of f0 and f0 f1
  std::vector<unsigned long long> prim;   // primary (tiles) per factorisation
};

// Plans the query: the space's device copies (built on its first use) and
// the query's primaries per factorisation.
int prepare_query(const mp_search_query& q, Prepared& pq, cudaStream_t st) {
  int rc = prepare(q, pq.S);
  if (rc) return rc;
  const size_t NC = pq.S.c->chains.size(), NF = pq.S.c->facts.size();
  const uint32_t P = (uint32_t)q.procs;
  if ((rc = device_space(*pq.S.c, st, &pq.D))) return rc;
  if ((rc = learned_space(pq.S, *pq.D, P, st, &pq.L))) return rc;
  pq.d_progs = pq.D->progs;
  pq.d_facts = pq.D->facts;
  pq.d_chainfeat = pq.L->chainfeat;
  pq.d_fnode = pq.L->fnode;
  pq.d_fdiv = pq.L->fdiv;
  const uint32_t nd = pq.L->nd;
  // primaries in closed form on the host (no device round trip)
  const uint32_t E[3] = {(uint32_t)q.M, (uint32_t)q.N, (uint32_t)q.K};
  pq.prim.resize(NF);
  for (size_t fr = 0; fr < NF; ++fr) {
    const uint32_t f[3] = {(uint32_t)pq.S.c->facts[fr][0], (uint32_t)pq.S.c->facts[fr][1],
                           (uint32_t)pq.S.c->facts[fr][2]};
    pq.prim[fr] = primary_cost(E, f);
  }
  QInfo& Q = pq.Q;
  std::memset(&Q, 0, sizeof(Q));
  Q.E[0] = (uint32_t)q.M;
  Q.E[1] = (uint32_t)q.N;
  Q.E[2] = (uint32_t)q.K;
  Q.P = (uint32_t)q.procs;
  Q.g = (uint32_t)q.procs_per_node;
  Q.n = Q.P / Q.g;
  Q.nf = (uint32_t)NF;
  Q.nd = nd;
  Q.nchains = NC;
  Q.tile_bytes = q.tile_bytes;
  Q.pmin = *std::min_element(pq.prim.begin(), pq.prim.end());
  Q.qf[0] = std::log2((double)q.M) / 12.0;
  Q.qf[1] = std::log2((double)q.N) / 12.0;
  Q.qf[2] = std::log2((double)q.K) / 12.0;
  Q.qf[3] = std::log2((double)q.procs) / 14.0;
  Q.qf[4] = std::log2((double)Q.n) / 12.0;
  Q.qf[5] = std::log2((double)Q.g) / 3.0;
  return MP_OK;
}

uint64_t splitmix(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}


// Scores of the candidates at positions [0, ncand) of the scored list (flist
// maps positions to factorisation ranks; null = every candidate), in runs
// of 2^19 (64 MB of feature tiles, resident in L2 between the two kernels).
int score_candidates(mp_mlp* h, const Prepared& pq, const uint32_t* d_fl, uint64_t ncand, float* d_sc,
                     cudaStream_t st) {
  constexpr uint64_t kRun = uint64_t(1) << 19;
  const uint64_t run = std::min<uint64_t>(kRun, (ncand + 255) / 256 * 256);
  uint8_t* img = (uint8_t*)g_pool_img.get(run / 128 * kTileBytes);
  if (!img) return MP_ENOMEM;
  MP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_img, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem));
  for (uint64_t c0 = 0; c0 < ncand; c0 += kRun) {
    const uint64_t n = std::min<uint64_t>(kRun, ncand - c0);
    const uint32_t ntiles = (uint32_t)((n + 127) / 128);
    k_feat_img<<<ntiles, 128, 0, st>>>(pq.Q, pq.d_fnode, pq.d_fdiv, pq.d_facts, pq.d_chainfeat, d_fl, c0, n,
                                       img);
    const unsigned grid = (unsigned)std::min<uint64_t>((ntiles + 1) / 2, (uint64_t)sm_count_l());
    layer_timer_begin(st);
    k_mlp_img<<<grid, kMlpThreads, kMlpSmem, st>>>(img, ntiles, h->Wimg, h->P, n, d_sc + c0, h->status);
    layer_timer_end(st);
    count_launch(2);
    MP_CUDA_TRY(cudaGetLastError());
  }
  return MP_OK;
}


__global__ void k_gather(const bf16* __restrict__ X, const float* __restrict__ T, const int64_t* __restrict__ perm,
                         int B, bf16* __restrict__ Xb, float* __restrict__ Tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // one 16-byte chunk per thread
  if (i >= B * 8) return;
  const int r = i >> 3, c = i & 7;
  const int64_t src = perm[r];
  reinterpret_cast<uint4*>(Xb + (size_t)r * 64)[c] = reinterpret_cast<const uint4*>(X + (size_t)src * 64)[c];
  if (c == 0) Tb[r] = T[src];
}

void mlpk_gather(const bf16* X, const float* T, const int64_t* perm, int B, bf16* Xb, float* Tb, cudaStream_t st) {
  k_gather<<<(B * 8 + 255) / 256, 256, 0, st>>>(X, T, perm, B, Xb, Tb);
  count_launch();
}


float host_target(unsigned long long p, unsigned long long sc, unsigned long long pmin) {
  const float pn = (float)((double)p / (double)std::max(pmin, 1ull) - 1.0);
  return 2.f * std::min(pn, 16.f) + std::log2(1.f + (float)sc) / 8.f;
}

}  // namespace lrn
}  // namespace mp

// ------------------------------------------------------------ C ABI

extern "C" int mp_mlp_train_search(mp_mlp* h, const mp_search_query* queries, int n_queries, int samples_per_query,
                                   int epochs, int batch, float lr, uint64_t seed, float* final_loss, void* stream) {
  using namespace mp;
  using namespace mp::lrn;
  if (!h || !queries || n_queries < 1 || samples_per_query < 1 || epochs < 0 || batch < 128 || batch % 128)
    return MP_EINVAL;
  for (int i = 0; i < n_queries; ++i) {
    const int rc = validate_query(queries[i]);
    if (rc) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t total = (size_t)n_queries * samples_per_query;
  // dataset
  bf16* X = nullptr;
  float* T = nullptr;
  char* scratch = nullptr;
  int rc = MP_OK;
  const size_t per = (size_t)samples_per_query;
  if (cudaMalloc(&X, total * 64 * 2) != cudaSuccess || cudaMalloc(&T, total * 4) != cudaSuccess ||
      cudaMalloc(&scratch, a256(per * 8) * 3 + (size_t)batch * (64 * 2 + 4) + 1024) != cudaSuccess) {
    cudaGetLastError();
    if (X) cudaFree(X);
    if (T) cudaFree(T);
    return MP_ENOMEM;
  }
  int64_t* d_idx = (int64_t*)scratch;
  uint64_t* d_p = (uint64_t*)(scratch + a256(per * 8));
  uint64_t* d_s = (uint64_t*)(scratch + 2 * a256(per * 8));
  bf16* Xb = (bf16*)(scratch + 3 * a256(per * 8));
  float* Tb = (float*)((char*)Xb + (size_t)batch * 128);
  uint64_t rng = seed;
  std::vector<int64_t> idx(per);
  for (int qi = 0; qi < n_queries && !rc; ++qi) {
    const mp_search_query& q = queries[qi];
    Prepared pq;
    if ((rc = prepare_query(q, pq, st))) break;
    const uint64_t NC = pq.S.c->chains.size(), NF = pq.S.c->facts.size();
    std::vector<uint32_t> order(NF);
    std::iota(order.begin(), order.end(), 0u);
    std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return pq.prim[a] < pq.prim[b]; });
    // half on the factorisations of least primary cost (the learned search
    // ranks those), a quarter on the eight lowest primaries, a quarter uniform
    size_t nbest = 1;
    while (nbest < NF && pq.prim[order[nbest]] == pq.prim[order[0]]) ++nbest;
    for (size_t i = 0; i < per; ++i) {
      const uint64_t r = splitmix(rng);
      uint64_t fr;
      if (i % 4 < 2) fr = order[(r >> 20) % nbest];
      else if (i % 4 == 2) fr = order[(r >> 20) % std::min<uint64_t>(8, NF)];
      else fr = r % NF;
      idx[i] = (int64_t)(fr * NC + (splitmix(rng) % NC));
    }
    if (cudaMemcpyAsync(d_idx, idx.data(), per * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = MP_ECUDA; break; }
    if ((rc = candidate_costs_dev(q, pq.S, *pq.D, d_idx, (int64_t)per, d_p, d_s, st))) break;
    k_features_idx<<<(unsigned)((per + 127) / 128), 128, 0, st>>>(pq.Q, pq.d_fnode, pq.d_fdiv, pq.d_facts,
                                                                  pq.d_chainfeat, d_idx,
                                                                  (int64_t)per, d_p, d_s, X + (size_t)qi * per * 64,
                                                                  T + (size_t)qi * per);
    count_launch();
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = MP_ECUDA; break; }
  }
  // epochs of shuffled minibatches
  float loss = 0.f;
  std::vector<int64_t> perm(total);
  std::iota(perm.begin(), perm.end(), 0);
  int64_t* d_perm = nullptr;
  if (!rc && cudaMalloc(&d_perm, total * 8) != cudaSuccess) rc = MP_ENOMEM;
  // the step size follows a cosine from lr down to 5% of it over the run
  const double steps_total = (double)epochs * (double)(total / (size_t)batch);
  double step_i = 0.0;
  for (int e = 0; e < epochs && !rc; ++e) {
    for (size_t i = total - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(rng) % (i + 1)]);
    if (cudaMemcpyAsync(d_perm, perm.data(), total * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = MP_ECUDA; break; }
    for (size_t b0 = 0; b0 + batch <= total && !rc; b0 += batch) {
      mp::lrn::mlpk_gather(X, T, d_perm + b0, batch, Xb, Tb, st);
      MP_CUDA_TRY(cudaMemsetAsync(h->status, 0, 4, st));
      const double cosine = 0.5 * (1.0 + std::cos(3.141592653589793 * step_i / std::max(steps_total, 1.0)));
      step_i += 1.0;
      rc = mlpk::train_step(h, Xb, Tb, batch, (float)(lr * (0.05 + 0.95 * cosine)), st);
    }
    float l = 0.f;
    cudaMemcpyAsync(&l, h->scalar, 4, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    loss = l;
  }
  if (d_perm) cudaFree(d_perm);
  cudaFree(X);
  cudaFree(T);
  cudaFree(scratch);
  if (final_loss) *final_loss = loss;
  return rc;
}

namespace mp {
namespace lrn {

// Counter words after the histograms that k_sel_init clears: cnt (4), nonfinite (1).
constexpr unsigned kInitWords = 5;

// Entries of the selection arrays: a selection of up to cap_a + cap_b
// candidates plus the previous rounds' (at most as many again).
size_t sel_capacity(unsigned cap_a, unsigned cap_b) { return 2 * ((size_t)cap_a + cap_b); }

// Device buffers of one learned search (scores, histogram, selection).
struct SelBufs {
  float* sc;
  unsigned *hist, *coarse, *thr, *cnt, *nonfinite;
  int64_t *below, *eq, *sel_idx;
  uint64_t *sel_p, *sel_s;
  float* sel_y;
  uint32_t* fl;
  SelResult* res;
};

int sel_bufs(uint64_t ncand, unsigned cap_a, unsigned cap_b, size_t nfl, SelBufs& b) {
  const size_t cap = sel_capacity(cap_a, cap_b);
  // hist (65536 words), coarse (256 words), then the counters k_sel_init
  // also clears (cnt, nonfinite: kInitWords); thr is kept across rounds
  const size_t o_sc = 0, o_hist = a256(ncand * 4), o_coarse = o_hist + 65536 * 4, o_cnt = o_coarse + 256 * 4,
               o_nf = o_cnt + 16, o_thr = o_hist + a256((65536 + 256 + kInitWords) * 4), o_below = o_thr + 256,
               o_eq = o_below + a256((size_t)cap_a * 8),
               o_idx = o_eq + a256((size_t)cap_b * 8), o_p = o_idx + a256(cap * 8), o_s = o_p + a256(cap * 8),
               o_y = o_s + a256(cap * 8), o_fl = o_y + a256(cap * 4), o_res = o_fl + a256(nfl * 4),
               end = o_res + 256;
  char* w = g_pool_s.get(end);
  if (!w) return MP_ENOMEM;
  b.sc = (float*)(w + o_sc);
  b.hist = (unsigned*)(w + o_hist);
  b.coarse = (unsigned*)(w + o_coarse);
  b.thr = (unsigned*)(w + o_thr);
  b.cnt = (unsigned*)(w + o_cnt);
  b.nonfinite = (unsigned*)(w + o_nf);
  b.below = (int64_t*)(w + o_below);
  b.eq = (int64_t*)(w + o_eq);
  b.sel_idx = (int64_t*)(w + o_idx);
  b.sel_p = (uint64_t*)(w + o_p);
  b.sel_s = (uint64_t*)(w + o_s);
  b.sel_y = (float*)(w + o_y);
  b.fl = (uint32_t*)(w + o_fl);
  b.res = (SelResult*)(w + o_res);
  return MP_OK;
}

// Exact costs of the selection (or, with list_a null, of scored positions
// 0 .. n_identity - 1) into b.sel_*.
int launch_sel_costs(const mp_search_query& q, const Prepared& pq, const SelBufs& b, const int64_t* list_a,
                     const unsigned* cnt_a, unsigned cap_a, const int64_t* list_b, const unsigned* cnt_b,
                     unsigned cap_b, unsigned long long n_identity, unsigned long long out0,
                     unsigned long long out_cap, int* status, cudaStream_t st) {
  // one warp per candidate, each with its own chain table and bitmaps:
  // up to 4 warps per CTA within about 100 KB of shared memory
  const SearchSpace& S = pq.S;
  const uint32_t Pp = (uint32_t)((q.procs + 7) & ~7);
  const size_t per_warp = (size_t)Pp * 2 + (size_t)S.words * 32 * 4;
  const int wpc = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(100 * 1024) / per_warp));
  const size_t smem = per_warp * wpc;
  if (smem > 227 * 1024) return MP_ENOTSUP;
  if (smem > 40 * 1024)   // opt in with room for static shared memory
    MP_CUDA_TRY(cudaFuncSetAttribute(k_sel_costs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sel_costs, 32 * wpc, smem));
  const unsigned long long most = list_a ? (unsigned long long)cap_a + cap_b : n_identity;
  const unsigned grid = (unsigned)std::max<unsigned long long>(
      1, std::min<unsigned long long>((most + wpc - 1) / wpc,
                                      (unsigned long long)sm_count_l() * std::max(per_sm, 1)));
  k_sel_costs<<<grid, 32 * wpc, smem, st>>>(pq.d_progs, pq.d_facts, (unsigned long long)S.c->chains.size(),
                                            (uint32_t)q.procs, (uint32_t)q.M, (uint32_t)q.N, (uint32_t)q.K, S.words,
                                            pq.D->tab, Pp, b.fl, list_a,
                                            cnt_a, cap_a, list_b, cnt_b, cap_b, n_identity, b.sc, out0, out_cap,
                                            b.sel_idx, b.sel_p, b.sel_s, b.sel_y, status);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

// Factorisations of least primary cost (or every one) and the scored pool.
std::vector<uint32_t> pool_facts(const Prepared& pq, bool all) {
  std::vector<uint32_t> flist;
  for (uint64_t fr = 0; fr < pq.prim.size(); ++fr)
    if (all || pq.prim[fr] == pq.Q.pmin) flist.push_back((uint32_t)fr);
  return flist;
}

// Three timing events per host thread and device (created on first use).
cudaEvent_t* phase_events() {
  constexpr int kMaxDevices = 64;
  struct Ev {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    bool ok = false;
    ~Ev() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  };
  thread_local Ev per_device[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  Ev& v = per_device[dev];
  if (!v.ok) {
    v.ok = true;
    for (cudaEvent_t& x : v.e) v.ok = v.ok && cudaEventCreate(&x) == cudaSuccess;
    if (!v.ok) {
      cudaGetLastError();
      return nullptr;
    }
  }
  return v.e;
}

// Margin rule: accepted when tau - y_best exceeds the calibrated bound with
// this much head-room (relative, absolute).
constexpr float kMarginScale = 1.25f, kMarginSlack = 0.01f;

}  // namespace lrn
}  // namespace mp

extern "C" int mp_learned_search(mp_mlp* h, const mp_search_query* query, int K, int flags, mp_search_result* out,
                                 mp_learned_stats* stats, void* stream) {
  using namespace mp;
  using namespace mp::lrn;
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point a) { return std::chrono::duration<double, std::milli>(clk::now() - a).count(); };
  if (!h || !query || !out || K < 1 || K > 65536) return MP_EINVAL;
  int rc = validate_query(*query);
  if (rc) return rc;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  cudaStream_t st = (cudaStream_t)stream;
  const mp_search_query& q = *query;
  auto t_phase = clk::now();
  Prepared pq;
  if ((rc = prepare_query(q, pq, st))) return rc;
  const uint64_t NC = pq.S.c->chains.size(), NF = pq.S.c->facts.size();
  // the candidates that can win: every chain with a factorisation of least
  // primary cost (exact, closed form); MP_LEARNED_SCORE_ALL scores them all
  const bool all = (flags & MP_LEARNED_SCORE_ALL) != 0;
  const std::vector<uint32_t> flist = pool_facts(pq, all);
  const uint64_t ncand = NC * flist.size();
  uint64_t n_pmin_facts = 0;
  for (uint64_t fr = 0; fr < NF; ++fr) n_pmin_facts += pq.prim[fr] == pq.Q.pmin;
  // the selection grows by 8x (up to kMaxSel) while the acceptance rule fails
  const unsigned kMaxSel = 1u << 16;
  const unsigned cap_a = (unsigned)std::min<uint64_t>(std::max<unsigned>((unsigned)K, kMaxSel), ncand);
  const unsigned cap_b = 1u << 16;
  SelBufs b;
  if ((rc = sel_bufs(ncand, cap_a, cap_b, flist.size(), b))) return rc;
  // host staging (pinned): the result record, the status word, then the
  // scored factorisations (copied asynchronously from there)
  char* stage = g_host_stage.get(256 + flist.size() * 4);
  if (!stage) return MP_ENOMEM;
  std::memcpy(stage + 256, flist.data(), flist.size() * 4);
  MP_CUDA_TRY(cudaMemcpyAsync(b.fl, stage + 256, flist.size() * 4, cudaMemcpyHostToDevice, st));
  // a lower bound on the secondary of every candidate that can win (the
  // least-primary factorisations); reaching it certifies the winner
  uint64_t min_lb = ~0ull;
  std::vector<uint64_t> lb_of(NF, 0);
  for (uint64_t fr = 0; fr < NF; ++fr)
    if (pq.prim[fr] == pq.Q.pmin) {
      const uint32_t f[3] = {(uint32_t)pq.S.c->facts[fr][0], (uint32_t)pq.S.c->facts[fr][1],
                             (uint32_t)pq.S.c->facts[fr][2]};
      lb_of[fr] = secondary_lower_bound(pq.Q.E, f, pq.Q.n, pq.Q.g);
      min_lb = std::min(min_lb, lb_of[fr]);
    }
  SelResult* hres = (SelResult*)stage;
  int* hstatus = (int*)(stage + 128);
  if (stats) stats->ms_prepare = ms_since(t_phase);
  t_phase = clk::now();
  // phase boundaries on the stream (device time): scoring start, scores
  // ranked, last selection reduced
  cudaEvent_t* ev = stats ? phase_events() : nullptr;
  if (stats && !ev) return MP_ECUDA;
  if (ev) MP_CUDA_TRY(cudaEventRecord(ev[0], st));
  // ---- score every candidate of the pool, histogram of the scores
  MP_CUDA_TRY(cudaMemsetAsync(h->status, 0, 4, st));
  k_sel_init<<<64, 256, 0, st>>>(b.hist, kInitWords);
  count_launch();
  if ((rc = score_candidates(h, pq, b.fl, ncand, b.sc, st))) return rc;
  const unsigned gb = (unsigned)std::min<uint64_t>((ncand + 255) / 256, (uint64_t)sm_count_l() * 8);
  k_topk_hist<<<gb, 256, 0, st>>>(b.sc, ncand, b.hist, b.coarse, b.nonfinite);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  if (ev) MP_CUDA_TRY(cudaEventRecord(ev[1], st));
  if (stats) stats->n_scored = (int64_t)ncand;
  // ---- the Kc best scores (with the rest of the threshold bin), evaluated
  // exactly and reduced on the device; one round trip per selection
  const float rule_bound = std::isfinite(h->margin_bound) ? kMarginScale * std::max(0.f, (float)h->margin_bound) +
                                                                kMarginSlack
                                                          : INFINITY;
  unsigned Kc = (unsigned)std::min<uint64_t>((uint64_t)K, ncand);
  const unsigned long long out_cap = sel_capacity(cap_a, cap_b);
  SelResult r;
  std::memset(&r, 0, sizeof(r));
  r.complete = 1;
  int rounds = 0;
  for (;;) {
    // a growth round evaluates only the candidates it adds (the bins past
    // the previous threshold) and reduces them with the earlier ones
    const unsigned n_prev = rounds ? r.n : 0;
    const int prev_complete = r.complete;
    k_topk_threshold<<<1, 256, 0, st>>>(b.hist, b.coarse, Kc, rounds ? 1 : 0, b.thr, b.cnt);
    k_topk_collect<<<gb, 256, 0, st>>>(b.sc, ncand, b.thr, b.below, b.cnt, b.eq, b.cnt + 1, Kc, cap_b, b.cnt + 2);
    count_launch(2);
    MP_CUDA_TRY(cudaGetLastError());
    ++rounds;
    if ((rc = launch_sel_costs(q, pq, b, b.below, b.cnt, Kc, b.eq, b.cnt + 1, cap_b, 0, n_prev, out_cap, h->status,
                               st)))
      return rc;
    k_sel_reduce<<<1, 256, 0, st>>>(b.cnt, Kc, cap_b, n_prev, prev_complete, (unsigned)out_cap, b.thr, b.sel_idx,
                                     b.sel_p, b.sel_s, b.sel_y, pq.Q.pmin, min_lb, NC * n_pmin_facts, rule_bound,
                                     b.nonfinite, b.res);
    count_launch();
    MP_CUDA_TRY(cudaGetLastError());
    if (ev) MP_CUDA_TRY(cudaEventRecord(ev[2], st));
    MP_CUDA_TRY(cudaMemcpyAsync(hres, b.res, sizeof(SelResult), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaMemcpyAsync(hstatus, h->status, 4, cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (*hstatus) return *hstatus;
    r = *hres;
    if (r.n == 0) MP_CUDA_TRY(cudaErrorUnknown);   // the selection kernels produced nothing
    if (stats) stats->n_exact += r.n;
    if (r.cert || (flags & MP_LEARNED_NO_FALLBACK)) break;
    // grow 2x while the selection stays within half of the scored set and
    // complete; beyond that the exhaustive search (which shares each chain's
    // table over its factorisations) is the cheaper way to an exact answer
    const uint64_t next = (uint64_t)Kc * 2;
    if (!r.complete || next > kMaxSel || next * 2 > ncand) break;
    Kc = (unsigned)next;
  }
  if (stats) {
    float m = 0.f, e = 0.f;
    MP_CUDA_TRY(cudaEventElapsedTime(&m, ev[0], ev[1]));
    MP_CUDA_TRY(cudaEventElapsedTime(&e, ev[1], ev[2]));
    stats->ms_model = m;
    stats->ms_exact = e;
    stats->ms_wall = ms_since(t_phase);
    stats->certified = r.cert;
    stats->margin = r.margin;
    stats->max_overestimate = r.over;
    stats->margin_bound = rule_bound;
    stats->rounds = rounds;
    stats->n_selected = r.n;
  }
  if (!r.cert && !(flags & MP_LEARNED_NO_FALLBACK)) {
    t_phase = clk::now();
    mp_search_query qf = q;
    qf.flags = 0;
    // the selection's winner bounds the secondary the search must look for,
    // and factorisations whose lower bound lies above it need no scan
    const bool bounded = r.p == pq.Q.pmin;
    std::vector<uint8_t> skip(NF, 0);
    if (bounded)
      for (uint64_t fr = 0; fr < NF; ++fr) skip[fr] = pq.prim[fr] == pq.Q.pmin && lb_of[fr] > r.s;
    rc = exhaustive_search(qf, out, st, bounded ? r.s : ~0ull, bounded ? &skip : nullptr);
    if (stats) {
      stats->fallback = 1;
      stats->n_exact += out->n_candidates;
      stats->ms_fallback = ms_since(t_phase);
    }
    return rc;
  }
  // the winner of the selection
  std::memset(out, 0, sizeof(*out));
  const uint64_t idx = (uint64_t)r.idx, fr = idx / NC, c = idx % NC;
  out->index = (int64_t)idx;
  for (int t = 0; t < 3; ++t) out->f[t] = pq.S.c->facts[fr][t];
  out->chain_rank = (int64_t)c;
  out->chain_len = (int32_t)pq.S.c->chains[c].size();
  for (int o = 0; o < out->chain_len; ++o) {
    const CanonOp& op = pq.S.c->chains[c][o];
    mp_xform& x = out->chain[o];
    x.op = op.op == P_SPLIT ? MP_SPLIT : (op.op == P_MERGE ? MP_MERGE : MP_SWAP);
    x.i = op.p;
    x.j = op.op == P_SPLIT ? 0 : op.q;
    x.d = op.op == P_SPLIT ? op.d : 0;
  }
  out->primary_bytes = r.p * q.tile_bytes;
  out->secondary_bytes = r.s * q.tile_bytes;
  out->n_chains = (int64_t)NC;
  out->n_factorisations = (int64_t)NF;
  out->n_candidates = (int64_t)(NC * NF);
  return MP_OK;
}

// Calibration of the margin rule on queries held out of training: for each,
// every candidate of least primary cost is scored and evaluated exactly;
// the query's value is the model's overestimation of its best-scored optimal
// candidate (least score among the candidates of least secondary, minus
// their target).  A search misses the optimum under the margin rule only if
// that value exceeds tau - y_best, so the largest value over the queries is
// the bound the rule compares with.
extern "C" int mp_mlp_calibrate(mp_mlp* h, const mp_search_query* queries, int n_queries, double* bound_out,
                                void* stream) {
  using namespace mp;
  using namespace mp::lrn;
  if (!h || !queries || n_queries < 1) return MP_EINVAL;
  for (int i = 0; i < n_queries; ++i) {
    const int rc = validate_query(queries[i]);
    if (rc) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double bound = -INFINITY;
  std::vector<float> y;
  std::vector<uint64_t> sec;
  for (int qi = 0; qi < n_queries; ++qi) {
    const mp_search_query& q = queries[qi];
    Prepared pq;
    int rc = prepare_query(q, pq, st);
    if (rc) return rc;
    const std::vector<uint32_t> flist = pool_facts(pq, false);
    const uint64_t ncand = pq.S.c->chains.size() * flist.size();
    SelBufs b;
    if ((rc = sel_bufs(ncand, 1, (unsigned)std::min<uint64_t>(ncand, 0xFFFFFFFFull), flist.size(), b))) return rc;
    MP_CUDA_TRY(cudaMemcpyAsync(b.fl, flist.data(), flist.size() * 4, cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemsetAsync(h->status, 0, 4, st));
    if ((rc = score_candidates(h, pq, b.fl, ncand, b.sc, st))) return rc;
    if ((rc = launch_sel_costs(q, pq, b, nullptr, nullptr, 0, nullptr, nullptr, 0, ncand, 0, ncand, h->status, st)))
      return rc;
    y.resize(ncand);
    sec.resize(ncand);
    int status = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(y.data(), b.sel_y, ncand * 4, cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaMemcpyAsync(sec.data(), b.sel_s, ncand * 8, cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaMemcpyAsync(&status, h->status, 4, cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (status) return status;
    const uint64_t s_opt = *std::min_element(sec.begin(), sec.end());
    float best_score = INFINITY;
    for (uint64_t i = 0; i < ncand; ++i)
      if (sec[i] == s_opt) best_score = std::min(best_score, std::isnan(y[i]) ? INFINITY : y[i]);
    bound = std::max(bound, (double)best_score - (double)host_target(pq.Q.pmin, s_opt, pq.Q.pmin));
  }
  h->margin_bound = std::isnan(bound) ? INFINITY : bound;
  if (bound_out) *bound_out = h->margin_bound;
  return MP_OK;
}

extern "C" int mp_mlp_set_margin_bound(mp_mlp* h, double bound) {
  if (!h || std::isnan(bound)) return MP_EINVAL;
  h->margin_bound = bound;
  return MP_OK;
}

// Scores (and optionally features) of every candidate of a query, in index
// order: the fused scoring kernel as the learned search runs it.
extern "C" int mp_learned_scores(mp_mlp* h, const mp_search_query* query, float* scores, void* features,
                                 int64_t* n_out, void* stream) {
  using namespace mp;
  using namespace mp::lrn;
  if (!h || !query || !scores || !n_out) return MP_EINVAL;
  int rc = validate_query(*query);
  if (rc) return rc;
  if (!is_device_pointer(scores) || (features && !is_device_pointer(features))) return MP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Prepared pq;
  if ((rc = prepare_query(*query, pq, st))) return rc;
  const uint64_t ncand = (uint64_t)pq.S.c->chains.size() * pq.S.c->facts.size();
  *n_out = (int64_t)ncand;
  MP_CUDA_TRY(cudaMemsetAsync(h->status, 0, 4, st));
  if ((rc = score_candidates(h, pq, nullptr, ncand, scores, st))) return rc;
  if (features) {
    int64_t* d_idx = nullptr;
    if (cudaMalloc(&d_idx, ncand * 8) != cudaSuccess) return MP_ENOMEM;
    std::vector<int64_t> idx(ncand);
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    MP_CUDA_TRY(cudaMemcpyAsync(d_idx, idx.data(), ncand * 8, cudaMemcpyHostToDevice, st));
    k_features_idx<<<(unsigned)((ncand + 127) / 128), 128, 0, st>>>(pq.Q, pq.d_fnode, pq.d_fdiv, pq.d_facts,
                                                                     pq.d_chainfeat,
                                                                     d_idx, (int64_t)ncand, nullptr, nullptr,
                                                                     (bf16*)features, nullptr);
    count_launch();
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_idx);
  }
  int status = 0;
  MP_CUDA_TRY(cudaMemcpyAsync(&status, h->status, 4, cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  return status;
}
