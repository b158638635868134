// Device structures of the decompose search, shared by search.cu (exact
// evaluation) and mlp.cu (candidate features for the learned scorer).
#pragma once

#include <memory>
#include <mutex>
#include <vector>

#include "engine.h"

namespace mp {

constexpr int kMaxChainPrims = 12;

constexpr int kSearchMaxProcs = 16384;
constexpr int kSmemBudget = 200 * 1024;
constexpr uint32_t kPreMaxDiv = 256;   // full search: fibre counts precounted for divisors up to this
constexpr int kPreMaxN = 64;           // and for at most this many divisors

struct ChainProg {
  int32_t nprim;
  int32_t depth;   // transforms of the chain; the rest are the flattening merges
  Prim prim[kMaxChainPrims];
};

struct Fact {
  uint32_t f[3];
};

struct Key {
  unsigned long long p, s, idx;
};

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
  if (a.p != b.p) return a.p < b.p;
  if (a.s != b.s) return a.s < b.s;
  return a.idx < b.idx;
}

// Node of flat index b of the flattened chain space: apply the Fig. 4
// inverse of every primitive, last to first, starting from the 1-D index.
__device__ __forceinline__ uint32_t resolve_node(const ChainProg& cp, uint32_t b) {
  uint32_t a[kMaxChainPrims + 2];
  a[0] = b;
  int r = 1;
  for (int o = cp.nprim - 1; o >= 0; --o) {
    const Prim& p = cp.prim[o];
    if (p.op == P_SPLIT) {
      a[p.p] = a[p.p] + a[p.p + 1] * p.d;
      for (int t = p.p + 1; t < r - 1; ++t) a[t] = a[t + 1];
      r -= 1;
    } else if (p.op == P_MERGE) {
      uint32_t q, rem;
      divmod32(a[p.p], p.div, q, rem);
      for (int t = r; t > p.q; --t) a[t] = a[t - 1];
      a[p.q] = q;
      a[p.p] = rem;
      r += 1;
    } else {
      uint32_t tmp = a[p.p];
      a[p.p] = a[p.q];
      a[p.q] = tmp;
    }
  }
  return a[0];   // (node, proc) = (a[0], a[1])
}

// Iterates the distinct block coordinates of one dimension (extent E split
// into f blocks) with the number of tiles in each:
//   E >= f: rep = i, weight = ceil((i+1) E / f) - ceil(i E / f)
//   E <  f: rep = floor(i f / E), weight = 1
// using only additions (the quotient/remainder of E / f or f / E once).
struct BlockIter {
  uint32_t big;      // E >= f
  uint32_t A, B, m;  // quotient, remainder, modulus
  uint32_t r;        // running remainder
  uint32_t rep;
  __device__ __forceinline__ void init(uint32_t E, uint32_t f) {
    big = E >= f;
    if (big) { A = E / f; B = E % f; m = f; } else { A = f / E; B = f % E; m = E; }
    r = 0;
    rep = 0;
  }
  // positions the iterator at block index i (a few divisions, once; 32-bit
  // ones when the product fits)
  __device__ __forceinline__ void seek(uint32_t E, uint32_t f, uint32_t i) {
    big = E >= f;
    if (big) {
      A = E / f; B = E - A * f; m = f;
      // r = ceil(i E / f) f - i E = (f - (i E mod f)) mod f
      const unsigned long long ie = (unsigned long long)i * E;
      const uint32_t rem = (ie >> 32) ? (uint32_t)(ie % f) : (uint32_t)ie % f;
      r = rem ? f - rem : 0u;
      rep = i;
    } else {
      A = f / E; B = f - A * E; m = E;
      const unsigned long long iF = (unsigned long long)i * f;
      if (iF >> 32) {
        rep = (uint32_t)(iF / E);
        r = (uint32_t)(iF - (unsigned long long)rep * E);
      } else {
        rep = (uint32_t)iF / E;
        r = (uint32_t)iF - rep * E;
      }
    }
  }
  // returns the weight of the current representative and advances
  __device__ __forceinline__ uint32_t step() {
    uint32_t w;
    if (big) {
      const uint32_t borrow = r < B;
      w = A + borrow;
      r = r + (borrow ? m : 0) - B;
      rep += 1;
    } else {
      w = 1;
      r += B;
      const uint32_t carry = r >= m;
      r -= carry ? m : 0;
      rep += A + carry;
    }
    return w;
  }
};

// Distinct nodes along one fibre (count of nodes seen), bitmap per thread in
// shared memory (word w of thread t at bm[w * nthr + t]).
// ROT: the scan begins with element `start` (< n) and wraps round to it (the
// count does not depend on the order); threads that scan neighbouring fibres
// at power-of-two strides then start at different elements, so that their
// table reads fall into different shared-memory banks.
template <bool ROT = false>
__device__ __forceinline__ uint32_t fibre_distinct(const uint16_t* __restrict__ tab, uint32_t* bm, int nthr,
                                                   int words, uint32_t base, uint32_t stride, uint32_t E,
                                                   uint32_t f, uint32_t n, uint32_t start = 0) {
  if (E >= f) {
    // every block holds tiles: the fibre's blocks are 0 .. n - 1
    const uint16_t* p0 = tab + base;
    const uint16_t* p = ROT ? p0 + start * stride : p0;
    uint32_t j = start;
    uint32_t D = 0;
    for (uint32_t iv = 0; iv < n; ++iv) {
      const uint32_t node = *p;
      uint32_t* wp = bm + (node >> 5) * nthr;
      const uint32_t bit = 1u << (node & 31);
      const uint32_t word = *wp;
      if (!(word & bit)) {
        *wp = word | bit;
        ++D;
      }
      if (ROT && ++j == n) {
        j = 0;
        p = p0;
      } else {
        p += stride;
      }
    }
    if ((uint32_t)words <= n) {
      for (int w = 0; w < words; ++w) bm[w * nthr] = 0;
    } else {
      p = p0;
      for (uint32_t iv = 0; iv < n; ++iv, p += stride) bm[(*p >> 5) * nthr] = 0;
    }
    return D;
  }
  BlockIter it;
  it.init(E, f);
  uint32_t D = 0;
  for (uint32_t iv = 0; iv < n; ++iv) {
    const uint32_t node = tab[base + stride * it.rep];
    it.step();
    uint32_t* wp = bm + (node >> 5) * nthr;
    const uint32_t bit = 1u << (node & 31);
    const uint32_t word = *wp;
    if (!(word & bit)) {
      *wp = word | bit;
      ++D;
    }
  }
  if ((uint32_t)words <= n) {
    for (int w = 0; w < words; ++w) bm[w * nthr] = 0;
  } else {
    it.init(E, f);
    for (uint32_t iv = 0; iv < n; ++iv) {
      const uint32_t node = tab[base + stride * it.rep];
      it.step();
      bm[(node >> 5) * nthr] = 0;
    }
  }
  return D;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Secondary cost (tiles) of factorisation f for the chain tabulated in tab,
// computed by one warp.  Families with at least 32 fibres: lane l scans a
// contiguous share of them with its own bitmap (word w of lane l at
// bm[w * stride + l]).  Families with fewer fibres: the fibres are scanned
// one at a time, the lanes splitting the elements, each into its own bitmap;
// the distinct count is the population of the lanes' bitmaps ORed together.
// Every lane returns the total.
// ub: once the running total exceeds it the remaining families are skipped
// and ~0 is returned (the caller only needs costs up to ub).
// pre0 / pre2 (may be null): the distinct-node counts minus one (a byte: a
// precounted fibre has at most 256 points) of family 0's fibres
// (the blocks of f0 consecutive flat indices, by block) and of family 2's
// (the residue classes modulo P / f2, by residue), counted once per chain
// for every divisor and looked up here instead of scanned.
// UNROLL: the three families unrolled (their extents in registers rather
// than local memory); faster without the precounted tables, slower with them.
// ROT: each lane starts its fibre scans at element lane mod n (spreads the
// table reads over shared-memory banks when the lanes' fibres lie a power of
// two apart; measured faster for the learned search's one-candidate warps,
// slower in the full search, whose warps share one table).
template <bool UNROLL = false, bool ROT = false>
__device__ __forceinline__ unsigned long long secondary_cost_warp(const uint16_t* __restrict__ tab, uint32_t* bm,
                                                                  int stride, int words, const uint32_t E[3],
                                                                  const uint32_t f[3], int lane,
                                                                  unsigned long long ub = ~0ull,
                                                                  const uint8_t* __restrict__ pre0 = nullptr,
                                                                  const uint8_t* __restrict__ pre2 = nullptr) {
  const uint32_t fstride[3] = {1u, f[0], f[0] * f[1]};
  uint32_t n[3];
  for (int t = 0; t < 3; ++t) n[t] = E[t] < f[t] ? E[t] : f[t];
  unsigned long long sec = 0;
#pragma unroll(UNROLL ? 3 : 1)
  for (int v = 0; v < 3; ++v) {
    if (n[v] <= 1) continue;
    const int u = v == 0 ? 1 : 0;
    const int w = v == 2 ? 1 : 2;
    const uint32_t nfib = n[u] * n[w];
    const uint8_t* pre = v == 0 ? pre0 : (v == 2 ? pre2 : nullptr);
    if (nfib >= 32 || pre) {
      // the family's extents as scalars (not re-read from the arrays around
      // the fibre scans' shared-memory stores)
      const uint32_t Eu = E[u], fu = f[u], nu = n[u], su = fstride[u], sw = fstride[w];
      const uint32_t Ev = E[v], fv = f[v], nv = n[v], sv = fstride[v], f1 = f[1];
      const uint32_t rot = ROT ? (uint32_t)lane % nv : 0u;
      const uint32_t chunk = (nfib + 31) / 32;
      const uint32_t fb0 = lane * chunk, fb1 = min(nfib, fb0 + chunk);
      unsigned long long part = 0;
      if (fb0 < fb1 && pre && Eu >= fu && E[w] >= f[w]) {
        // precounted, every block of u and w holds tiles: fibre fb's count is
        // at pre[fb] (family 0: rep_u + f1 rep_w, family 2: rep_u + f0 rep_w,
        // and rep = block index), so the lane reads its bytes in order
        const uint32_t row0 = fb0 / nu;
        uint32_t iu = fb0 - row0 * nu;
        BlockIter itu, itw;
        itu.seek(Eu, fu, iu);
        itw.seek(E[w], f[w], row0);
        uint32_t wt_w = itw.step();
        for (uint32_t fb = fb0; fb < fb1; ++fb) {
          const uint32_t wt_u = itu.step();
          part += (unsigned long long)wt_u * wt_w * pre[fb];
          if (++iu == nu) {
            iu = 0;
            itu.r = 0;
            itu.rep = 0;
            wt_w = itw.step();
          }
        }
      } else if (fb0 < fb1) {
        const uint32_t row0 = fb0 / nu;
        uint32_t iu = fb0 - row0 * nu;
        BlockIter itu, itw;
        itu.seek(Eu, fu, iu);
        itw.seek(E[w], f[w], row0);
        uint32_t rep_w = itw.rep;
        uint32_t wt_w = itw.step();
        for (uint32_t fb = fb0; fb < fb1; ++fb) {
          const uint32_t rep_u = itu.rep;
          const uint32_t wt_u = itu.step();
          const uint32_t base = rep_u * su + rep_w * sw;
          const uint32_t D = pre ? (uint32_t)pre[v == 0 ? rep_u + rep_w * f1 : base] + 1u
                                 : fibre_distinct<ROT>(tab, bm + lane, stride, words, base, sv, Ev, fv, nv, rot);
          part += (unsigned long long)wt_u * wt_w * (D - 1);
          if (++iu == nu) {
            // back to block 0: the quotient and remainder stay, the running
            // remainder and the representative restart at 0
            iu = 0;
            itu.r = 0;
            itu.rep = 0;
            rep_w = itw.rep;
            wt_w = itw.step();
          }
        }
      }
      sec += warp_sum(part);
    } else {
      // few, long fibres: the lanes split each fibre's points, each marking
      // its own bitmap column, and the warp ORs the columns word by word
      const uint32_t Ev = E[v], fv = f[v], nv = n[v], sv = fstride[v], su = fstride[u], sw = fstride[w];
      // block coordinate of the lane's point iv = lane + 32 t: floor(iv fv / Ev)
      // when Ev < fv (iv when Ev >= fv), stepped by 32 points through its
      // remainder (iv fv < 2^19: P <= 2^14)
      const bool dense = Ev >= fv;
      const uint32_t Q = dense ? 32u : 32u * fv / Ev, R = dense ? 0u : 32u * fv % Ev;
      const uint32_t rep0 = dense ? (uint32_t)lane : (uint32_t)lane * fv / Ev;
      const uint32_t rem0 = dense ? 0u : (uint32_t)lane * fv % Ev;
      uint32_t* col = bm + lane;
      BlockIter itu, itw;
      itw.seek(E[w], f[w], 0);
      itu.seek(E[u], f[u], 0);
      for (uint32_t iw = 0; iw < n[w]; ++iw) {
        const uint32_t rep_w = itw.rep;
        const uint32_t wt_w = itw.step();
        itu.r = 0;
        itu.rep = 0;
        for (uint32_t iu = 0; iu < n[u]; ++iu) {
          const uint32_t rep_u = itu.rep;
          const uint32_t wt_u = itu.step();
          const uint32_t base = rep_u * su + rep_w * sw;
          uint32_t rep = rep0, rem = rem0;
          for (uint32_t iv = lane; iv < nv; iv += 32) {
            const uint32_t node = tab[base + rep * sv];
            uint32_t* wp = col + (node >> 5) * stride;
            const uint32_t bit = 1u << (node & 31);
            const uint32_t word = *wp;
            if (!(word & bit)) *wp = word | bit;
            rep += Q;
            rem += R;
            if (rem >= Ev) {
              rem -= Ev;
              ++rep;
            }
          }
          uint32_t D = 0;
          for (int k = 0; k < words; ++k) {
            D += __popc(__reduce_or_sync(0xFFFFFFFFu, col[k * stride]));
            col[k * stride] = 0;
          }
          sec += (unsigned long long)wt_u * wt_w * (D - 1);
        }
      }
    }
    if (sec > ub) return ~0ull;   // uniform across the warp
  }
  return sec;
}

__host__ __device__ __forceinline__ unsigned long long primary_cost(const uint32_t E[3], const uint32_t f[3]) {
  unsigned long long p = 0;
  for (int v = 0; v < 3; ++v) {
    const int u = v == 0 ? 1 : 0;
    const int w = v == 2 ? 1 : 2;
    const uint32_t nv = E[v] < f[v] ? E[v] : f[v];
    p += (unsigned long long)(nv - 1) * E[u] * E[w];
  }
  return p;
}

__device__ __forceinline__ void block_argmin(Key& k, Key* red) {
  for (int o = 16; o > 0; o >>= 1) {
    Key other;
    other.p = __shfl_down_sync(0xFFFFFFFFu, k.p, o);
    other.s = __shfl_down_sync(0xFFFFFFFFu, k.s, o);
    other.idx = __shfl_down_sync(0xFFFFFFFFu, k.idx, o);
    if (key_less(other, k)) k = other;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = k;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    k = lane < nw ? red[lane] : Key{~0ull, ~0ull, ~0ull};
    for (int o = 16; o > 0; o >>= 1) {
      Key other;
      other.p = __shfl_down_sync(0xFFFFFFFFu, k.p, o);
      other.s = __shfl_down_sync(0xFFFFFFFFu, k.s, o);
      other.idx = __shfl_down_sync(0xFFFFFFFFu, k.idx, o);
      if (key_less(other, k)) k = other;
    }
  }
}

__device__ __forceinline__ void build_table(const ChainProg& cp, uint16_t* tab, uint32_t P) {
  for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) tab[b] = (uint16_t)resolve_node(cp, b);
}

// The chain's node table from its cached copy (16-byte rows of Pp entries).
__device__ __forceinline__ void load_table(const uint16_t* __restrict__ row, uint16_t* tab, uint32_t Pp) {
  const uint4* src = reinterpret_cast<const uint4*>(row);
  uint4* dst = reinterpret_cast<uint4*>(tab);
  for (uint32_t i = threadIdx.x; i < Pp / 8; i += blockDim.x) dst[i] = __ldg(src + i);
}


// Secondary cost (tiles) of candidate (factorisation fr, chain c), computed
// by the whole CTA: the chain's node table in shared memory (copied from the
// space's cache, or built), the fibres of the three families spread over the
// threads, one bitmap per thread.  Every thread returns the total.
// smem_raw: words * blockDim.x bitmap words, then the table (Pp uint16);
// cp and red are the caller's __shared__ scratch.  Safe to call repeatedly
// from one CTA (it synchronises before reusing its scratch).
__device__ __forceinline__ unsigned long long candidate_secondary_block(
    const ChainProg* __restrict__ progs, const Fact* __restrict__ facts, unsigned long long fr, unsigned long long c,
    uint32_t P, const uint32_t E[3], int words, const uint16_t* __restrict__ gtab, uint32_t Pp,
    unsigned char* smem_raw, ChainProg& cp, unsigned long long* red) {
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw);
  uint16_t* tab = reinterpret_cast<uint16_t*>(smem_raw + (size_t)words * blockDim.x * 4);
  __syncthreads();
  if (threadIdx.x == 0) cp = progs[c];
  for (int w = 0; w < words; ++w) bm[w * blockDim.x + threadIdx.x] = 0;
  __syncthreads();
  if (gtab) load_table(gtab + (size_t)c * Pp, tab, Pp);
  else build_table(cp, tab, P);
  __syncthreads();
  const uint32_t f[3] = {facts[fr].f[0], facts[fr].f[1], facts[fr].f[2]};
  const uint32_t stride[3] = {1u, f[0], f[0] * f[1]};
  uint32_t n[3];
  for (int t = 0; t < 3; ++t) n[t] = E[t] < f[t] ? E[t] : f[t];
  unsigned long long sec = 0;
#pragma unroll   // constant family indices keep E, f, stride and n in registers
  for (int v = 0; v < 3; ++v) {
    if (n[v] <= 1) continue;
    const int u = v == 0 ? 1 : 0;
    const int w = v == 2 ? 1 : 2;
    const uint32_t nfib = n[u] * n[w];
    for (uint32_t fb = threadIdx.x; fb < nfib; fb += blockDim.x) {
      const uint32_t iu = fb % n[u], iw = fb / n[u];
      // representative and weight of block iu (iw) directly
      auto rep_wt = [&](int t, uint32_t i, uint32_t& rep, uint32_t& wt) {
        if (E[t] >= f[t]) {
          rep = i;
          const unsigned long long lo = ((unsigned long long)i * E[t] + f[t] - 1) / f[t];
          const unsigned long long hi = ((unsigned long long)(i + 1) * E[t] + f[t] - 1) / f[t];
          wt = (uint32_t)(hi - lo);
        } else {
          rep = (uint32_t)((unsigned long long)i * f[t] / E[t]);
          wt = 1;
        }
      };
      uint32_t ru, wu, rw, ww;
      rep_wt(u, iu, ru, wu);
      rep_wt(w, iw, rw, ww);
      const uint32_t base = ru * stride[u] + rw * stride[w];
      const uint32_t D = fibre_distinct(tab, bm + threadIdx.x, blockDim.x, words, base, stride[v], E[v], f[v], n[v]);
      sec += (unsigned long long)wu * ww * (D - 1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) sec += __shfl_down_sync(0xFFFFFFFFu, sec, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sec;
  __syncthreads();
  unsigned long long total = 0;
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) total += red[w];
  return total;
}

// ----------------------------------------------------------------- host side

// The candidate space of one machine shape and depth bound: factorisations,
// chains and their compiled programs.  Immutable once built and shared by
// every query on the same (processors, processors per node, depth).
// Its device copy (built on first use, kept with the space): the chain
// programs, the factorisations and, when it takes at most
// kNodeTableCacheBytes, every chain's node table (chain c's node of flat index
// b at tab[c * Pp + b], Pp = P rounded up to 8 so that each chain's row is
// 16-byte aligned), which the search kernels copy instead of rebuilding.
struct DeviceSpace {
  ChainProg* progs = nullptr;
  Fact* facts = nullptr;
  uint16_t* tab = nullptr;
  uint32_t Pp = 0;
  int device = -1;
};

struct SpaceCore {
  std::vector<std::vector<int64_t>> facts;
  std::vector<std::vector<CanonOp>> chains;
  std::vector<ChainProg> progs;
  std::vector<Fact> fdev;
  int64_t P = 0;
  mutable std::mutex dev_mu;
  mutable DeviceSpace dev;
  ~SpaceCore();
};

constexpr size_t kNodeTableCacheBytes = size_t(1) << 30;

// The space's device copy on the current device, built on st on first use
// (and synchronised then); MP_ENOTSUP when the space was first used on
// another device.
int device_space(const SpaceCore& c, cudaStream_t st, const DeviceSpace** out);

struct SearchSpace {
  std::shared_ptr<const SpaceCore> c;
  int words = 0;
  int threads = 0;
  size_t smem = 0;
};

ChainProg compile_chain(int64_t n, int64_t g, const std::vector<CanonOp>& ch);
int validate_query(const mp_search_query& q);
int prepare(const mp_search_query& q, SearchSpace& S);
// Exact costs (bytes) of n listed candidates, all buffers on the device
// (the space's device copy from device_space).
int candidate_costs_dev(const mp_search_query& q, const SearchSpace& S, const DeviceSpace& D, const int64_t* d_idx,
                        int64_t n, uint64_t* d_p, uint64_t* d_s, cudaStream_t st);
// Exhaustive argmin on the device; the result on the host.
// ub_secondary (tiles): a secondary cost some candidate of least primary is
// known to reach; candidates are scanned only as far as needed to show they
// exceed it (the result is the same as without it).
// skip (optional, one byte per factorisation): factorisations known not to
// hold the answer (a lower bound on their secondary above ub_secondary).
int exhaustive_search(const mp_search_query& q, mp_search_result* out, cudaStream_t st,
                      unsigned long long ub_secondary = ~0ull, const std::vector<uint8_t>* skip = nullptr);
// Lower bound (tiles) on the secondary cost of factorisation f over every
// chain; 0 when no bound applies (see search.cu).
uint64_t secondary_lower_bound(const uint32_t E[3], const uint32_t f[3], uint32_t nodes, uint32_t g);

}  // namespace mp
