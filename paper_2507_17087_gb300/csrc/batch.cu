// Batched mapping: thousands of index launches of uneven rank and size in
// one CUDA-graph replay.
//
// mp_batch_create plans every query once (validation, decompose expansion,
// rank fix-up), lays out one pool per kind of scratch (chain tables, c_t
// tables, per-dimension counts, linear-cyclic deficits) and uploads the
// per-query descriptors.  mp_batch_run replays a graph of these kernels:
//   k_b_resolve  chain table of every query          (sum P threads)
//   k_b_tables   c_t tables of every query           (sum of tabled L_t)
//   k_b_counts   closed-form per-dimension counts     (sum J)
//   k_b_slabs    linear-cyclic boundary deficits as residue ranges
//   k_b_defscan  their prefix sums
//   k_b_ids      persistent id writer: CTAs pull fixed-size tiles of 4-point
//                groups from an atomic work counter, stage the tile's chain
//                table (and its row contributions) in shared memory when the
//                query changes, and write the tile with k_ids's warp loops
//   k_b_reduce   histogram, received bytes, halo total per query
// The tile size is picked on the first run by timing the persistent kernel
// at a few sizes (autotune) and kept with the batch.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.cuh"

namespace mp {

namespace {

constexpr uint32_t kBatchMaxP = 16384;
constexpr uint64_t kBatchTableMax = 65536;   // tabled coordinates per dimension
constexpr uint64_t kFuseTarget = 2048;        // fused rows: at least this many points when the extents allow
constexpr uint64_t kFuseMax = 4096;           // fused rows staged in shared memory: at most this many points
constexpr uint64_t kShortRow = 512;          // fused rows shorter than this take the next dimension too

struct QDesc : MapCore {
  Tabs tabs;            // offsets relative to tab_base
  uint64_t tab_base;    // this query's tables in the table pool
  uint64_t ids_off;     // first id of this query (a multiple of 4)
  uint32_t p_off;       // chain table / hist / recv / deficits offset (prefix of P)
  uint32_t cnt_off;     // counts offset (prefix of Jtotal)
  uint32_t prim_off;    // primitives in the primitive pool
  int32_t mode;         // IdsMode
  uint64_t face[4];
  // M_FUSED: dimensions fuse_m..k-1 form rows of Lf points; rsrc (RowSrc)
  // says where a row offset's contribution comes from (a table at fuse_off,
  // relative to tab_base, or the last dimension's components).  R_TAB2: the
  // table at fuse_off fuses dimensions fuse_m+1..k-1 into Lin points
  int32_t fuse_m;
  uint32_t Lf;
  Div32 divLf;
  uint64_t fuse_off;
  int32_t rsrc;
  uint32_t Lin;
  Div32 divLin;
  uint64_t pad_;
};

// the fused table's first dimension and length (0 when rows have no table)
__host__ __device__ inline bool two_level(const QDesc& Q) { return Q.rsrc == R_TAB2 || Q.rsrc == R_TAB2A; }
__host__ __device__ inline int fused_first(const QDesc& Q) { return two_level(Q) ? Q.fuse_m + 1 : Q.fuse_m; }
__host__ __device__ inline uint32_t fused_len(const QDesc& Q) {
  if (Q.mode != M_FUSED) return 0;
  return two_level(Q) ? Q.Lin : (Q.rsrc <= R_TAB4 ? Q.Lf : 0);
}
static_assert(sizeof(QDesc) % 16 == 0, "QDesc is copied in 16-byte words");

struct Tile {
  uint32_t q;
  uint32_t gbeg, gend;   // 4-point groups of the query
};

// index of the query whose range [off[q], off[q+1]) holds e
template <typename T>
__device__ __forceinline__ uint32_t find_query(const T* __restrict__ off, uint32_t n, T e) {
  uint32_t lo = 0, hi = n;   // off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= e) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads) k_b_resolve(const QDesc* __restrict__ qd, const Prim* __restrict__ prims,
                                                        const uint32_t* __restrict__ p_pref, uint32_t n,
                                                        uint32_t total, uint32_t* __restrict__ Tpool) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const uint32_t q = find_query(p_pref, n, e);
    const QDesc& Q = qd[q];
    Tpool[e] = resolve_F(Q, prims + Q.prim_off, Q.nprim, e - Q.p_off);
  }
}

__global__ void __launch_bounds__(kThreads) k_b_tables(const QDesc* __restrict__ qd,
                                                       const uint64_t* __restrict__ tab_pref, uint32_t n,
                                                       uint64_t total, uint32_t* __restrict__ tabpool) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = find_query(tab_pref, n, e);
    const QDesc& Q = qd[q];
    const uint64_t r = e - Q.tab_base;
    if (fused_len(Q) && r >= Q.fuse_off) {
      // fused offset x -> coordinates of the fused dimensions (C order)
      uint64_t x = r - Q.fuse_off;
      if (x >= fused_len(Q)) continue;
      uint32_t c = 0;
      for (int t = Q.k - 1; t >= fused_first(Q); --t) {
        const uint64_t xt = x % Q.L[t];
        x /= Q.L[t];
        c += contrib(Q, t, xt);
      }
      tabpool[e] = c;
      continue;
    }
    int t = -1;
    for (int u = 0; u < Q.k; ++u)
      if (Q.tabs.has[u] && r >= Q.tabs.off[u]) t = u;
    if (t < 0) continue;
    const uint64_t x = r - Q.tabs.off[t];
    if (x < Q.L[t]) tabpool[e] = contrib(Q, t, x);
  }
}

__global__ void __launch_bounds__(kThreads) k_b_counts(const QDesc* __restrict__ qd,
                                                       const uint32_t* __restrict__ cnt_pref, uint32_t n,
                                                       uint32_t total, uint64_t* __restrict__ H,
                                                       uint64_t* __restrict__ X) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const uint32_t q = find_query(cnt_pref, n, e);
    const QDesc& Q = qd[q];
    const uint32_t r = e - Q.cnt_off;
    int t = 0;
    while (t < Q.k - 1 && r >= Q.Joff[t + 1]) ++t;
    uint64_t h, xc;
    dim_counts(Q, t, r - Q.Joff[t], h, xc);
    H[e] = h;
    if (X) X[e] = xc;
  }
}

// slab work list entry: query, dimension and the running offset
struct Slab {
  uint32_t q;
  int32_t t;
  uint64_t begin;   // first work index of this slab pair
};

// Linear-cyclic face deficits as residue ranges.  The points of slab x_t of
// dimension t are lin = hi * (L_t S_t) + x_t S_t + lo, lo < S_t (S_t the
// stride of t), hi < N / (L_t S_t): for each (slab, hi) their residues
// lin mod P form one cyclic run of S_t residues from r0.  Whole turns add to
// every residue (defall), the rest of the run goes into a difference array
// (deficit, prefix-summed by k_b_defscan).  Work: 2 N / (L_t S_t) entries
// per dimension instead of one per slab point.
__global__ void __launch_bounds__(kThreads) k_b_slabs(const QDesc* __restrict__ qd, const Slab* __restrict__ slabs,
                                                      const uint64_t* __restrict__ slab_pref, uint32_t nslabs,
                                                      uint64_t total, unsigned long long* __restrict__ deficit,
                                                      unsigned long long* __restrict__ defall) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = find_query(slab_pref, nslabs, e);
    const Slab sl = slabs[i];
    const QDesc& Q = qd[sl.q];
    const uint32_t t = (uint32_t)sl.t;
    const uint64_t S = Q.lc_stride[t], Lt = Q.L[t];
    const uint64_t H = Q.npoints / (Lt * S);
    const uint64_t local = e - sl.begin;
    const uint64_t side = local / H, hi = local - side * H;
    const uint64_t xt = side ? Lt - 1 : 0;
    const unsigned long long f = Q.face[t];
    uint64_t q0, r0;
    divmod64(hi * (Lt * S) + xt * S, Q.divP64, q0, r0);
    uint64_t full, rem;
    divmod64(S, Q.divP64, full, rem);
    if (full) atomicAdd(defall + sl.q, full * f);
    if (rem) {
      unsigned long long* D = deficit + Q.p_off;
      const uint64_t end = r0 + rem;
      atomicAdd(D + r0, f);
      if (end < Q.P) {
        atomicAdd(D + end, (unsigned long long)(-(long long)f));
      } else if (end > Q.P) {
        atomicAdd(D, f);
        atomicAdd(D + (end - Q.P), (unsigned long long)(-(long long)f));
      }
    }
  }
}

// Prefix sum of each linear-cyclic query's difference array, plus its whole
// turns: the deficit of every residue.  The last dimension's slabs (stride 1:
// points hi * L + x, hi < N / L) are counted per residue F instead, in closed
// form: hi * L = F - x (mod P) has solutions iff g = gcd(L mod P, P) divides
// F - x, and then hi = h0 (mod P / g).  One CTA per query.
__global__ void __launch_bounds__(kThreads) k_b_defscan(const QDesc* __restrict__ qd,
                                                        unsigned long long* __restrict__ deficit,
                                                        const unsigned long long* __restrict__ defall) {
  const QDesc& Q = qd[blockIdx.x];
  if (!Q.lc) return;
  __shared__ unsigned long long part[kThreads];
  __shared__ int64_t s_g, s_inv;
  const int last = Q.k - 1;
  const bool last_slabs = Q.lc_stride_mod[last] != 0 && Q.face[last] != 0;
  if (threadIdx.x == 0 && last_slabs) {
    int64_t g, inv;
    gcd_inverse((int64_t)(Q.L[last] % Q.P), (int64_t)Q.P, g, inv);
    s_g = g;
    s_inv = inv;
  }
  unsigned long long* D = deficit + Q.p_off;
  const uint32_t P = Q.P;
  const uint32_t per = (P + kThreads - 1) / kThreads;
  const uint32_t lo = min(P, threadIdx.x * per), hi = min(P, lo + per);
  unsigned long long sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += D[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < kThreads; o <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = (threadIdx.x ? part[threadIdx.x - 1] : 0) + defall[blockIdx.x];
  for (uint32_t i = lo; i < hi; ++i) {
    run += D[i];
    D[i] = run;
  }
  if (last_slabs) {
    const int64_t g = s_g, inv = s_inv, M = (int64_t)P / g;
    const uint64_t Lt = Q.L[last], H = Q.npoints / Lt;
    const unsigned long long f = Q.face[last];
    for (uint32_t i = lo; i < hi; ++i) {
      unsigned long long add = 0;
      for (int side = 0; side < 2; ++side) {
        const int64_t x = side ? (int64_t)((Lt - 1) % P) : 0;
        const int64_t c = ((int64_t)i - x + (int64_t)P) % (int64_t)P;
        if (c % g) continue;
        const int64_t h0 = M == 1 ? 0 : (int64_t)(((unsigned __int128)(c / g) * (uint64_t)inv) % (uint64_t)M);
        add += count_residue(H, (uint64_t)h0, (uint64_t)M);
      }
      D[i] += add * f;
    }
  }
}

// four resident blocks per SM: 64 registers and no spills, which the row
// paths (row bases kept a row ahead, two-level rows) need; the 48-register
// allocation without the bound spilled and ran the batch 5 % slower
__global__ void __launch_bounds__(kThreads, 4) k_b_ids(const QDesc* __restrict__ qd, const Tile* __restrict__ tiles,
                                                    uint32_t ntiles, const uint32_t* __restrict__ Tpool,
                                                    const uint32_t* __restrict__ tabpool, uint32_t smem_T,
                                                    int vec_ok, unsigned* __restrict__ counter,
                                                    int32_t* __restrict__ ids) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* Ts = smem;
  uint32_t* Cs = smem + smem_T;
  __shared__ uint32_t s_tile;
  // the current query's descriptor, staged in shared memory: the hot loop
  // reads its fields from there instead of re-loading global memory after
  // every store
  __shared__ __align__(16) QDesc sQ;
  uint32_t cur_q = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) break;
    const Tile tl = tiles[tile];
    const QDesc& Q = sQ;
    if (tl.q != cur_q) {
      const uint4* src = reinterpret_cast<const uint4*>(qd + tl.q);
      uint4* dst = reinterpret_cast<uint4*>(&sQ);
      for (uint32_t i = threadIdx.x; i < sizeof(QDesc) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < Q.P; i += blockDim.x) Ts[i] = __ldg(Tpool + Q.p_off + i);
      if (Q.mode == M_FAST_SMEM) {
        const int last = Q.k - 1;
        const uint32_t* cg = tabpool + Q.tab_base + Q.tabs.off[last];
        for (uint32_t i = threadIdx.x; i < (uint32_t)Q.L[last]; i += blockDim.x) Cs[i] = __ldg(cg + i);
      } else if (fused_len(Q)) {
        const uint32_t* cg = tabpool + Q.tab_base + Q.fuse_off;
        for (uint32_t i = threadIdx.x; i < fused_len(Q); i += blockDim.x) Cs[i] = __ldg(cg + i);
      }
      cur_q = tl.q;
      __syncthreads();
    }
    // the tile's groups, one contiguous sub-range per warp
    const uint32_t ng = tl.gend - tl.gbeg;
    const uint32_t per_warp = ((ng + kThreads / 32 - 1) / (kThreads / 32) + 31) / 32 * 32;
    const uint32_t wb = tl.gbeg + min(ng, (uint32_t)warp * per_warp);
    const uint32_t we = tl.gbeg + min(ng, (uint32_t)(warp + 1) * per_warp);
    int32_t* qids = ids + Q.ids_off;
    const uint32_t* ctab = tabpool + Q.tab_base;
    if (Q.lc) {
      ids_range_lc<uint32_t, true>(Q, Ts, wb, we, lane, vec_ok, qids);
    } else if (Q.mode == M_FUSED) {
      const RowAux aux{ctab + Q.tabs.off[Q.fuse_m], Q.Lin, Q.divLin};
#define MP_ROWS(SRC) \
  ids_range_rows<SRC>(Q, Q.tabs, Ts, Cs, ctab, aux, Q.fuse_m, Q.Lf, Q.divLf, wb, we, lane, vec_ok, qids)
      switch (Q.rsrc) {
        case R_TAB2: MP_ROWS(R_TAB2); break;
        case R_TAB2A: MP_ROWS(R_TAB2A); break;
        case R_TAB4: MP_ROWS(R_TAB4); break;
        case R_TAB: MP_ROWS(R_TAB); break;
        case R_BLOCK: MP_ROWS(R_BLOCK); break;
        case R_CYCLIC: MP_ROWS(R_CYCLIC); break;
        case R_BCYC: MP_ROWS(R_BCYC); break;
        default: MP_ROWS(R_HIER); break;
      }
#undef MP_ROWS
    } else if (Q.mode == M_FAST_SMEM) {
      ids_range<uint32_t, M_FAST_SMEM, true>(Q, Q.tabs, Ts, Cs, ctab, wb, we, lane, vec_ok, qids);
    } else if (Q.mode == M_FAST_GLOBAL) {
      ids_range<uint32_t, M_FAST_GLOBAL, true>(Q, Q.tabs, Ts, Cs, ctab, wb, we, lane, vec_ok, qids);
    } else {
      ids_range<uint32_t, M_GENERAL, true>(Q, Q.tabs, Ts, Cs, ctab, wb, we, lane, vec_ok, qids);
    }
    __syncthreads();   // smem and s_tile are rewritten next iteration
  }
}

__global__ void __launch_bounds__(kThreads) k_b_reduce(const QDesc* __restrict__ qd,
                                                       const uint32_t* __restrict__ p_pref, uint32_t n,
                                                       uint32_t total, const uint32_t* __restrict__ Tpool,
                                                       const uint64_t* __restrict__ H, const uint64_t* __restrict__ X,
                                                       const uint64_t* __restrict__ deficit,
                                                       uint64_t* __restrict__ hist, uint64_t* __restrict__ recv,
                                                       unsigned long long* __restrict__ halo) {
  const bool want_recv = recv || halo;
  for (uint32_t e0 = blockIdx.x * blockDim.x; e0 < total; e0 += gridDim.x * blockDim.x) {
    const uint32_t e = e0 + threadIdx.x;
    uint64_t r_F = 0;
    uint32_t q = 0xFFFFFFFFu;
    if (e < total) {
      q = find_query(p_pref, n, e);
      const QDesc& Q = qd[q];
      const uint32_t F = e - Q.p_off;
      uint64_t h_F;
      reduce_F(Q, H + Q.cnt_off, X ? X + Q.cnt_off : nullptr, deficit ? deficit + Q.p_off : nullptr, Q.face,
               want_recv, F, h_F, r_F);
      const uint32_t id = Tpool[e];
      if (hist) hist[Q.p_off + id] = h_F;
      if (recv) recv[Q.p_off + id] = r_F;
    }
    if (halo) {
      // lanes of one query add their bytes once
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, q);
      unsigned long long v = r_F;
      unsigned long long sum = 0;
      for (int l = 0; l < 32; ++l) {
        const unsigned long long o = __shfl_sync(0xFFFFFFFFu, v, l);
        if (grp & (1u << l)) sum += o;
      }
      if (q != 0xFFFFFFFFu && (threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1) && sum)
        atomicAdd(halo + q, sum);
    }
  }
}

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

int sm_count_b() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 132;
  }
  return n;
}

}  // namespace

}  // namespace mp

struct mp_batch {
  int n = 0;
  int device = 0;
  std::vector<mp::QDesc> qd;
  std::vector<mp::Prim> prims;
  std::vector<uint32_t> p_pref, cnt_pref;
  std::vector<uint64_t> tab_pref, ids_pref, slab_pref;
  std::vector<mp::Slab> slabs;
  uint32_t totalP = 0, totalJ = 0, maxP = 0, maxC = 0;
  uint64_t total_tab = 0, total_ids = 0, total_slab = 0;
  bool any_lc = false;
  // device state
  void* dmem = nullptr;
  size_t dbytes = 0;
  mp::QDesc* d_qd = nullptr;
  mp::Prim* d_prims = nullptr;
  uint32_t *d_p_pref = nullptr, *d_cnt_pref = nullptr, *d_T = nullptr, *d_tab = nullptr;
  uint64_t *d_tab_pref = nullptr, *d_slab_pref = nullptr, *d_H = nullptr, *d_X = nullptr, *d_def = nullptr,
           *d_defall = nullptr;
  mp::Slab* d_slabs = nullptr;
  unsigned* d_counter = nullptr;
  // tiles and the persistent id writer's launch shape
  uint32_t tile_groups = 0;
  mp::Tile* d_tiles = nullptr;
  uint32_t ntiles = 0;
  unsigned ids_blocks = 1;
  size_t ids_smem = 0;
  // graph
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;            // the reductions' stream beside the id writer
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* key[4] = {nullptr, nullptr, nullptr, nullptr};
  std::mutex mu;
};

namespace mp {
namespace {

std::vector<Tile> make_tiles(const mp_batch& b, uint32_t tile_groups) {
  std::vector<Tile> tiles;
  for (int q = 0; q < b.n; ++q) {
    const uint64_t groups = (b.qd[q].npoints + 3) / 4;
    for (uint64_t g = 0; g < groups; g += tile_groups)
      tiles.push_back(Tile{(uint32_t)q, (uint32_t)g, (uint32_t)std::min<uint64_t>(groups, g + tile_groups)});
  }
  return tiles;
}

int upload_tiles(mp_batch& b, uint32_t tile_groups) {
  std::vector<Tile> tiles = make_tiles(b, tile_groups);
  if (b.d_tiles) cudaFree(b.d_tiles);
  b.d_tiles = nullptr;
  if (cudaMalloc(&b.d_tiles, std::max<size_t>(1, tiles.size()) * sizeof(Tile)) != cudaSuccess) return MP_ENOMEM;
  MP_CUDA_TRY(cudaMemcpy(b.d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  b.ntiles = (uint32_t)tiles.size();
  b.tile_groups = tile_groups;
  // launch shape of the persistent id writer: every resident CTA slot
  b.ids_smem = (size_t)((b.maxP + 3) & ~3u) * 4 + (size_t)b.maxC * 4;
  if (b.ids_smem > 40 * 1024)   // opt in with room for static shared memory
    MP_CUDA_TRY(cudaFuncSetAttribute(k_b_ids, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.ids_smem));
  int per_sm = 0;
  MP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_ids, kThreads, b.ids_smem));
  if (per_sm < 1) per_sm = 1;
  b.ids_blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count_b() * per_sm, b.ntiles));
  return MP_OK;
}

int launch_ids(mp_batch& b, int32_t* ids, cudaStream_t st) {
  const int vec_ok = ((uintptr_t)ids & 15) == 0;
  MP_CUDA_TRY(cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned), st));
  k_b_ids<<<b.ids_blocks, kThreads, b.ids_smem, st>>>(b.d_qd, b.d_tiles, b.ntiles, b.d_T, b.d_tab,
                                                      (uint32_t)((b.maxP + 3) & ~3u), vec_ok, b.d_counter, ids);
  count_launch();
  return MP_OK;
}

// Enqueues the whole batch on st (used for capture).  The reductions read
// only the resolved chain table and the counts: when ids are wanted too they
// run on the batch's second stream beside the tables and the id writer, and
// st waits for them before the end.
int enqueue(mp_batch& b, int32_t* ids, uint64_t* hist, uint64_t* halo, uint64_t* recv, cudaStream_t st) {
  const unsigned big = (unsigned)sm_count_b() * 8;
  auto blocks_for = [&](uint64_t work) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + kThreads - 1) / kThreads, big));
  };
  const bool want_red = hist || halo || recv;
  const bool want_recv = halo || recv;
  k_b_resolve<<<blocks_for(b.totalP), kThreads, 0, st>>>(b.d_qd, b.d_prims, b.d_p_pref, (uint32_t)b.n, b.totalP,
                                                        b.d_T);
  count_launch();
  const bool fork = ids && want_red;
  cudaStream_t rs = st;
  if (fork) {
    MP_CUDA_TRY(cudaEventRecord(b.ev_fork, st));
    MP_CUDA_TRY(cudaStreamWaitEvent(b.side, b.ev_fork, 0));
    rs = b.side;
  }
  if (want_red && b.totalJ) {
    k_b_counts<<<blocks_for(b.totalJ), kThreads, 0, rs>>>(b.d_qd, b.d_cnt_pref, (uint32_t)b.n, b.totalJ, b.d_H,
                                                         want_recv ? b.d_X : nullptr);
    count_launch();
  }
  if (want_recv && b.any_lc) {
    MP_CUDA_TRY(cudaMemsetAsync(b.d_def, 0, (size_t)b.totalP * 8, rs));
    MP_CUDA_TRY(cudaMemsetAsync(b.d_defall, 0, (size_t)b.n * 8, rs));
    if (b.total_slab) {
      k_b_slabs<<<blocks_for(b.total_slab), kThreads, 0, rs>>>(b.d_qd, b.d_slabs, b.d_slab_pref,
                                                               (uint32_t)b.slabs.size(), b.total_slab,
                                                               (unsigned long long*)b.d_def,
                                                               (unsigned long long*)b.d_defall);
      count_launch();
    }
    k_b_defscan<<<(unsigned)b.n, kThreads, 0, rs>>>(b.d_qd, (unsigned long long*)b.d_def,
                                                   (const unsigned long long*)b.d_defall);
    count_launch();
  }
  if (want_red) {
    if (halo) MP_CUDA_TRY(cudaMemsetAsync(halo, 0, (size_t)b.n * 8, rs));
    k_b_reduce<<<blocks_for(b.totalP), kThreads, 0, rs>>>(b.d_qd, b.d_p_pref, (uint32_t)b.n, b.totalP, b.d_T, b.d_H,
                                                         want_recv ? b.d_X : nullptr, b.any_lc ? b.d_def : nullptr,
                                                         hist, recv, (unsigned long long*)halo);
    count_launch();
  }
  if (ids && b.total_tab) {
    k_b_tables<<<blocks_for(b.total_tab), kThreads, 0, st>>>(b.d_qd, b.d_tab_pref, (uint32_t)b.n, b.total_tab,
                                                            b.d_tab);
    count_launch();
  }
  if (ids) {
    int rc = launch_ids(b, ids, st);
    if (rc) return rc;
  }
  if (fork) {
    MP_CUDA_TRY(cudaEventRecord(b.ev_join, b.side));
    MP_CUDA_TRY(cudaStreamWaitEvent(st, b.ev_join, 0));
  }
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

// Times the persistent id writer at a few tile sizes and keeps the fastest.
int autotune(mp_batch& b, int32_t* ids, cudaStream_t st) {
  const uint32_t cand[] = {8192, 32768, 65536, 131072};
  float best_ms = 1e30f;
  uint32_t best = cand[1];
  cudaEvent_t e0, e1;
  MP_CUDA_TRY(cudaEventCreate(&e0));
  MP_CUDA_TRY(cudaEventCreate(&e1));
  int rc = enqueue(b, ids, nullptr, nullptr, nullptr, st);   // tables for the id writer
  for (uint32_t tg : cand) {
    if (rc) break;
    if ((rc = upload_tiles(b, tg))) break;
    if ((rc = launch_ids(b, ids, st))) break;   // warm
    cudaEventRecord(e0, st);
    if ((rc = launch_ids(b, ids, st))) break;
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = tg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  return upload_tiles(b, best);
}

}  // namespace
}  // namespace mp

extern "C" int mp_batch_create(const mp_query* queries, int n, mp_batch** out) {
  using namespace mp;
  if (!out || n < 1 || !queries) return MP_EINVAL;
  *out = nullptr;
  mp_batch* b = new mp_batch();
  b->n = n;
  cudaGetDevice(&b->device);
  b->qd.resize(n);
  b->p_pref.resize(n + 1);
  b->cnt_pref.resize(n + 1);
  b->tab_pref.resize(n + 1);
  b->ids_pref.resize(n + 1);
  // planning and the per-query choices are independent: host threads over
  // the queries; the offsets are assigned in order afterwards
  std::vector<std::vector<Prim>> qprims(n);
  std::vector<uint64_t> qtab(n, 0);
  std::vector<int> qrc(n, 0);
  auto plan_query = [&](int q) {
    const mp_query& Qh = queries[q];
    Plan pl;
    int rc = build_plan(&Qh.space, &Qh.machine, Qh.chain, Qh.n_xf, &Qh.dist, pl);
    if (!rc && (pl.desc.P > kBatchMaxP || pl.desc.npoints >= (uint64_t(1) << 31))) rc = MP_ENOTSUP;
    qrc[q] = rc;
    if (rc) return;
    QDesc& Q = b->qd[q];
    std::memset(&Q, 0, sizeof(Q));
    static_cast<MapCore&>(Q) = static_cast<const MapCore&>(pl.desc);
    qprims[q].assign(pl.desc.prim, pl.desc.prim + pl.desc.nprim);
    for (int t = 0; t < 4; ++t) Q.face[t] = t < Q.k ? Qh.face_bytes[t] : 0;
    uint64_t tabq = 0;
    for (int t = 0; t < Q.k; ++t) {
      Q.tabs.has[t] = !Q.lc && Q.L[t] <= kBatchTableMax;
      Q.tabs.off[t] = tabq;
      if (Q.tabs.has[t]) tabq += (Q.L[t] + 3) & ~uint64_t(3);
    }
    const int last = Q.k - 1;
    const bool aligned = !Q.lc && Q.L[last] % 4 == 0 && Q.tabs.has[last];
    Q.mode = M_GENERAL;
    if (aligned && Q.L[last] > kFuseMax) {
      Q.mode = M_FAST_GLOBAL;   // long aligned rows: 16-byte loads of the last table from L2
    } else if (!Q.lc) {
      // rows of the trailing dimensions fused into one table of at most
      // kFuseMax points (at least kFuseTarget when the extents allow), staged
      // in shared memory; rows longer than that (the last extent alone) take
      // their contribution from the last dimension's components in place
      int m = last;
      uint64_t Lf = Q.L[last];
      while (m > 0 && Lf < kFuseTarget && Lf * Q.L[m - 1] <= kFuseMax) Lf *= Q.L[--m];
      Q.mode = M_FUSED;
      Q.fuse_m = m;
      Q.Lf = (uint32_t)Lf;
      Q.divLf = make_div32((uint32_t)Lf);
      if (Lf < kShortRow && m > 0 && Q.tabs.has[m - 1]) {
        // rows this short would change their base every few groups: the
        // next dimension joins the row through its own table
        Q.rsrc = Lf % 4 == 0 ? R_TAB2A : R_TAB2;
        Q.Lin = (uint32_t)Lf;
        Q.divLin = make_div32((uint32_t)Lf);
        Q.fuse_m = m - 1;
        Q.Lf = (uint32_t)(Lf * Q.L[m - 1]);
        Q.divLf = make_div32(Q.Lf);
        Q.fuse_off = tabq;
        tabq += (Lf + 3) & ~uint64_t(3);
      } else if (Lf <= kFuseMax) {
        Q.rsrc = Lf % 4 == 0 ? R_TAB4 : R_TAB;
        Q.fuse_off = tabq;
        tabq += (Lf + 3) & ~uint64_t(3);
      } else if (Q.ncomp[last] == 2) {
        Q.rsrc = R_HIER;
      } else {
        const int kind = Q.comp[last][0].kind;
        Q.rsrc = kind == C_BLOCK ? R_BLOCK : (kind == C_CYCLIC ? R_CYCLIC : R_BCYC);
      }
    }
    qtab[q] = tabq;
  };
  {
    const int nthr = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto worker = [&]() {
      for (int q = next.fetch_add(64); q < n; q = next.fetch_add(64))
        for (int e = q; e < std::min(n, q + 64); ++e) plan_query(e);
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < nthr && i * 64 < n; ++i) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
  }
  for (int q = 0; q < n; ++q)
    if (qrc[q]) {
      const int rc = qrc[q];
      delete b;
      return rc;
    }
  uint64_t P_acc = 0, J_acc = 0, tab_acc = 0, ids_acc = 0, slab_acc = 0;
  for (int q = 0; q < n; ++q) {
    QDesc& Q = b->qd[q];
    const int last = Q.k - 1;
    const uint64_t tabq = qtab[q];
    Q.prim_off = (uint32_t)b->prims.size();
    b->prims.insert(b->prims.end(), qprims[q].begin(), qprims[q].end());
    if (Q.mode == M_FAST_SMEM) b->maxC = std::max<uint32_t>(b->maxC, (uint32_t)Q.L[last]);
    b->maxC = std::max<uint32_t>(b->maxC, fused_len(Q));
    b->maxP = std::max(b->maxP, Q.P);
    Q.p_off = (uint32_t)P_acc;
    Q.cnt_off = (uint32_t)J_acc;
    Q.tab_base = tab_acc;
    Q.ids_off = ids_acc;
    b->p_pref[q] = (uint32_t)P_acc;
    b->cnt_pref[q] = (uint32_t)J_acc;
    b->tab_pref[q] = tab_acc;
    b->ids_pref[q] = ids_acc;
    P_acc += Q.P;
    J_acc += Q.Jtotal;
    tab_acc += tabq;
    ids_acc += (Q.npoints + 3) & ~uint64_t(3);
    if (Q.lc) {
      b->any_lc = true;
      for (int t = 0; t + 1 < Q.k; ++t)   // the last dimension is counted in closed form
        if (Q.lc_stride_mod[t] != 0 && Q.face[t] != 0) {
          b->slabs.push_back(Slab{(uint32_t)q, t, slab_acc});
          b->slab_pref.push_back(slab_acc);
          slab_acc += 2 * (Q.npoints / (Q.L[t] * Q.lc_stride[t]));
        }
    }
    if (P_acc >= (uint64_t(1) << 31) || J_acc >= (uint64_t(1) << 31)) {
      delete b;
      return MP_ENOTSUP;
    }
  }
  b->p_pref[n] = (uint32_t)P_acc;
  b->cnt_pref[n] = (uint32_t)J_acc;
  b->tab_pref[n] = tab_acc;
  b->ids_pref[n] = ids_acc;
  b->slab_pref.push_back(slab_acc);
  b->totalP = (uint32_t)P_acc;
  b->totalJ = (uint32_t)J_acc;
  b->total_tab = tab_acc;
  b->total_ids = ids_acc;
  b->total_slab = slab_acc;
  // ------------------------------------------------ device pools
  const size_t o_qd = 0;
  const size_t o_prim = a256(o_qd + b->qd.size() * sizeof(QDesc));
  const size_t o_ppref = a256(o_prim + std::max<size_t>(1, b->prims.size()) * sizeof(Prim));
  const size_t o_cpref = a256(o_ppref + (n + 1) * 4);
  const size_t o_tpref = a256(o_cpref + (n + 1) * 4);
  const size_t o_spref = a256(o_tpref + (n + 1) * 8);
  const size_t o_slabs = a256(o_spref + b->slab_pref.size() * 8);
  const size_t o_T = a256(o_slabs + std::max<size_t>(1, b->slabs.size()) * sizeof(Slab));
  const size_t o_tab = a256(o_T + P_acc * 4);
  const size_t o_H = a256(o_tab + std::max<uint64_t>(1, tab_acc) * 4);
  const size_t o_X = a256(o_H + std::max<uint64_t>(1, J_acc) * 8);
  const size_t o_def = a256(o_X + std::max<uint64_t>(1, J_acc) * 8);
  const size_t o_defall = a256(o_def + (b->any_lc ? P_acc : 1) * 8);
  const size_t o_cnt = a256(o_defall + (size_t)n * 8);
  const size_t bytes = a256(o_cnt + 256);
  if (cudaMalloc(&b->dmem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return MP_ENOMEM;
  }
  b->dbytes = bytes;
  char* base = (char*)b->dmem;
  b->d_qd = (QDesc*)(base + o_qd);
  b->d_prims = (Prim*)(base + o_prim);
  b->d_p_pref = (uint32_t*)(base + o_ppref);
  b->d_cnt_pref = (uint32_t*)(base + o_cpref);
  b->d_tab_pref = (uint64_t*)(base + o_tpref);
  b->d_slab_pref = (uint64_t*)(base + o_spref);
  b->d_slabs = (Slab*)(base + o_slabs);
  b->d_T = (uint32_t*)(base + o_T);
  b->d_tab = (uint32_t*)(base + o_tab);
  b->d_H = (uint64_t*)(base + o_H);
  b->d_X = (uint64_t*)(base + o_X);
  b->d_def = (uint64_t*)(base + o_def);
  b->d_defall = (uint64_t*)(base + o_defall);
  b->d_counter = (unsigned*)(base + o_cnt);
  bool ok = cudaMemcpy(b->d_qd, b->qd.data(), b->qd.size() * sizeof(QDesc), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!b->prims.empty())
    ok = ok && cudaMemcpy(b->d_prims, b->prims.data(), b->prims.size() * sizeof(Prim), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
  ok = ok && cudaMemcpy(b->d_p_pref, b->p_pref.data(), (n + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(b->d_cnt_pref, b->cnt_pref.data(), (n + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(b->d_tab_pref, b->tab_pref.data(), (n + 1) * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(b->d_slab_pref, b->slab_pref.data(), b->slab_pref.size() * 8, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  if (!b->slabs.empty())
    ok = ok && cudaMemcpy(b->d_slabs, b->slabs.data(), b->slabs.size() * sizeof(Slab), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess;
  if (!ok || upload_tiles(*b, 8192) != MP_OK) {
    cudaGetLastError();
    mp_batch_destroy(b);
    return MP_ECUDA;
  }
  *out = b;
  return MP_OK;
}

extern "C" int mp_batch_info(const mp_batch* b, uint64_t* total_ids, uint64_t* total_procs, uint64_t* ids_offsets,
                             uint64_t* proc_offsets, int32_t* tile_groups) {
  if (!b) return MP_EINVAL;
  if (total_ids) *total_ids = b->total_ids;
  if (total_procs) *total_procs = b->totalP;
  if (ids_offsets)
    for (int q = 0; q <= b->n; ++q) ids_offsets[q] = b->ids_pref[q];
  if (proc_offsets)
    for (int q = 0; q <= b->n; ++q) proc_offsets[q] = b->p_pref[q];
  if (tile_groups) *tile_groups = (int32_t)b->tile_groups;
  return MP_OK;
}

extern "C" int mp_batch_run(mp_batch* b, int32_t* ids, uint64_t* hist, uint64_t* halo, uint64_t* recv, int flags,
                            void* stream) {
  using namespace mp;
  if (!b) return MP_EINVAL;
  std::lock_guard<std::mutex> lock(b->mu);
  for (void* p : {(void*)ids, (void*)hist, (void*)halo, (void*)recv})
    if (p && !is_device_pointer(p)) return MP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!(flags & MP_BATCH_NO_GRAPH) && (flags & MP_BATCH_AUTOTUNE) && ids) {
    int rc = autotune(*b, ids, st);
    if (rc) return rc;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  if (flags & MP_BATCH_NO_GRAPH) return enqueue(*b, ids, hist, halo, recv, st);
  void* key[4] = {ids, hist, halo, recv};
  if (!b->exec || std::memcmp(key, b->key, sizeof(key)) != 0) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // capture on the batch's private stream, then replay on the caller's
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    MP_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(*b, ids, hist, halo, recv, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return MP_ECUDA;
    ce = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      b->exec = nullptr;
      return MP_ECUDA;
    }
    std::memcpy(b->key, key, sizeof(key));
  }
  MP_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  return MP_OK;
}

extern "C" int mp_batch_set_tile(mp_batch* b, int32_t tile_groups) {
  using namespace mp;
  if (!b || tile_groups < 1) return MP_EINVAL;
  std::lock_guard<std::mutex> lock(b->mu);
  int rc = upload_tiles(*b, (uint32_t)tile_groups);
  if (rc) return rc;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return MP_OK;
}

extern "C" int mp_batch_destroy(mp_batch* b) {
  if (!b) return MP_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
  return MP_OK;
}
