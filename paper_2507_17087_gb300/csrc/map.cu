// map_points / comm_volume: kernels and C-ABI entry points.
//
// The five distributions are separable: every final processor-space
// coordinate a_u is a function of one task coordinate x_t (block, cyclic,
// block-cyclic per dimension; the hierarchical Cannon mapper of Appendix A.1
// drives two final coordinates from each task coordinate), and the
// linearised round robin of Fig. 5 is a function of the C-order linear index.
// With F = sum_u a_u sigma_u (dimension 0 fastest) the flat final index of a
// point is therefore F(x) = sum_t c_t(x_t), or lin(x) mod P.  The chain of
// transforms is a bijection from the final space onto Machine(GPU) (every
// primitive of Fig. 4 is invertible, Sec. 3.3), so
//   id(x) = T[F(x)],  T = chain resolution of every F in [0, P).
// Kernels:
//   k_resolve    T[F] for F < P: decode F, apply the Fig. 4 formulas of every
//                primitive from last to first                       (a3)
//   k_dimtables  c_t(x_t) for every coordinate of every dimension, and the
//                per-dimension counts H_t[c] (points with c_t = c) and
//                X_t[c] (neighbour pairs along t that cross) used by the
//                reductions                                         (a2)
//   k_ids        ids[lin] = T[base(row) + c_last(x_last)]; 16-byte stores,
//                persistent grid                                  (a1-a3)
//   k_reduce     hist and per-processor halo bytes from the per-dimension
//                counts: because the chain is a bijection, owner(x) !=
//                owner(y) iff F(x) != F(y), and for separable F a neighbour
//                along t crosses iff c_t changes                  (a4, a5)
//   k_lc_slabs   linear-cyclic only: boundary points that miss a neighbour.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "engine.h"

namespace mp {

namespace {

constexpr int kThreads = 256;
constexpr uint64_t kTableMax = uint64_t(1) << 22;   // per-dimension c_t tables kept in HBM/L2
constexpr uint32_t kSmemTMax = 16384;               // T staged in shared memory up to this P
constexpr uint32_t kSmemLastMax = 8192;             // c_last staged in shared memory

struct Tabs {
  uint64_t off[4];     // offset of dimension t's c_t table in ctab (if present)
  int32_t has[4];      // 1 if the table exists
};

__device__ __forceinline__ uint32_t comp_coord(const Comp& c, uint64_t x) {
  switch (c.kind) {
    case C_BLOCK:
      if (c.narrow) return div32((uint32_t)x * c.s, c.divL32);
      return (uint32_t)div64(x * (uint64_t)c.s, c.divL);
    case C_CYCLIC:
      if (x <= 0xFFFFFFFFull) {
        uint32_t q, r;
        divmod32((uint32_t)x, c.divs, q, r);
        return r;
      } else {
        uint64_t q, r;
        divmod64(x, c.divs64, q, r);
        return (uint32_t)r;
      }
    default: {  // block-cyclic
      uint64_t blk = x <= 0xFFFFFFFFull ? div32((uint32_t)x, c.divb) : div64(x, c.divb64);
      if (blk <= 0xFFFFFFFFull) {
        uint32_t q, r;
        divmod32((uint32_t)blk, c.divs, q, r);
        return r;
      }
      uint64_t q, r;
      divmod64(blk, c.divs64, q, r);
      return (uint32_t)r;
    }
  }
}

// c_t(x) = sum of the final coordinates driven by x times their strides
__device__ __forceinline__ uint32_t contrib(const MapDesc& D, int t, uint64_t x) {
  uint32_t v = comp_coord(D.comp[t][0], x) * D.comp[t][0].sigma;
  if (D.ncomp[t] > 1) v += comp_coord(D.comp[t][1], x) * D.comp[t][1].sigma;
  return v;
}

// ----------------------------------------------------------------- k_resolve

__global__ void __launch_bounds__(kThreads) k_resolve(const __grid_constant__ MapDesc D,
                                                      uint32_t* __restrict__ T) {
  const uint32_t F = blockIdx.x * blockDim.x + threadIdx.x;
  if (F >= D.P) return;
  uint32_t a[kMaxRank + 1];
  uint32_t rest = F;
  for (int u = 0; u < D.rank; ++u) {
    uint32_t q, r;
    divmod32(rest, D.divs[u], q, r);
    a[u] = r;
    rest = q;
  }
  int r = D.rank;
  for (int o = D.nprim - 1; o >= 0; --o) {
    const Prim& p = D.prim[o];
    if (p.op == P_SPLIT) {
      // Fig. 4 split: b_i = a_i + a_{i+1} d, b_t = a_{t+1} for t > i
      a[p.p] = a[p.p] + a[p.p + 1] * p.d;
      for (int t = p.p + 1; t < r - 1; ++t) a[t] = a[t + 1];
      r -= 1;
    } else if (p.op == P_MERGE) {
      // Fig. 4 merge: b_p = a_p mod s_p, b_q = floor(a_p / s_p), b_t = a_{t-1} for t > q
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
  T[F] = a[0] * D.g + a[1];
}

// ----------------------------------------------------------------- k_dimtables

// One thread per (t, x_t).  Counts are aggregated over the lanes of a warp
// that share (t, c) before the global atomics.
__global__ void __launch_bounds__(kThreads) k_dimtables(const __grid_constant__ MapDesc D, Tabs tabs,
                                                        uint64_t total, uint32_t* __restrict__ ctab,
                                                        unsigned long long* __restrict__ H,
                                                        unsigned long long* __restrict__ X) {
  uint64_t off[5];
  off[0] = 0;
  for (int t = 0; t < D.k; ++t) off[t + 1] = off[t] + D.L[t];
  const uint64_t lane = threadIdx.x & 31;
  // the trip count is uniform across a warp (e - lane is the warp's base)
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e - lane < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const bool live = e < total;
    int t = 0;
    while (t < D.k - 1 && e >= off[t + 1]) ++t;
    const uint64_t x = live ? e - off[t] : 0;
    uint32_t c = 0, cross = 0;
    if (live) {
      c = contrib(D, t, x);
      if (tabs.has[t]) ctab[tabs.off[t] + x] = c;
      if (X) {
        if (x > 0 && contrib(D, t, x - 1) != c) cross += 1;
        if (x + 1 < D.L[t] && contrib(D, t, x + 1) != c) cross += 1;
      }
    }
    if (H) {
      const unsigned active = __ballot_sync(0xFFFFFFFFu, live);
      if (live) {
        const uint32_t key = (uint32_t)t * D.P + c;
        const unsigned grp = __match_any_sync(active, key);
        const uint32_t xsum = __reduce_add_sync(grp, cross);
        if ((threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1)) {
          atomicAdd(H + (uint64_t)t * D.P + c, (unsigned long long)__popc(grp));
          if (X && xsum) atomicAdd(X + (uint64_t)t * D.P + c, (unsigned long long)xsum);
        }
      }
    }
  }
}

// ----------------------------------------------------------------- k_ids
//
// Each warp owns one contiguous range of 4-point groups; lane l takes groups
// start + l, start + l + 32, ... so that every store instruction of the warp
// writes 512 contiguous bytes.  Between two groups of a lane the linear index
// advances by 128 points: x_last advances by 128 and the row (the slow
// coordinates) only changes when x_last wraps, so the row's contribution
// base(row) = sum_{t < k-1} c_t(x_t) is recomputed once per row.

template <typename I>
__device__ __forceinline__ void split_lin(const MapDesc& D, I lin, I& row, I& x) {
  const int last = D.k - 1;
  if (sizeof(I) == 8) {
    uint64_t q, r;
    divmod64((uint64_t)lin, D.divL64[last], q, r);
    row = (I)q;
    x = (I)r;
  } else {
    uint32_t q, r;
    divmod32((uint32_t)lin, D.divL32[last], q, r);
    row = (I)q;
    x = (I)r;
  }
}

template <typename I>
__device__ __noinline__ uint32_t row_base(const MapDesc& D, const Tabs& tabs,
                                          const uint32_t* __restrict__ ctab, I row) {
  uint32_t base = 0;
  for (int t = D.k - 2; t >= 0; --t) {
    I q, xt;
    if (t == 0) {
      q = 0;
      xt = row;
    } else if (sizeof(I) == 8) {
      uint64_t q64, r64;
      divmod64((uint64_t)row, D.divL64[t], q64, r64);
      q = (I)q64;
      xt = (I)r64;
    } else {
      uint32_t q32, r32;
      divmod32((uint32_t)row, D.divL32[t], q32, r32);
      q = (I)q32;
      xt = (I)r32;
    }
    row = q;
    base += tabs.has[t] ? __ldg(ctab + tabs.off[t] + xt) : contrib(D, t, (uint64_t)xt);
  }
  return base;
}

enum IdsMode : int { M_FAST_SMEM = 0, M_FAST_GLOBAL = 1, M_GENERAL = 2 };

template <typename I, int MODE, bool TSMEM>
__global__ void __launch_bounds__(kThreads) k_ids(const __grid_constant__ MapDesc D,
                                                  const __grid_constant__ Tabs tabs,
                                                  const uint32_t* __restrict__ Tg,
                                                  const uint32_t* __restrict__ ctab, int vec_ok,
                                                  uint64_t groups_per_warp, int32_t* __restrict__ ids) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* Ts = smem;
  uint32_t* Cs = smem + (TSMEM ? ((D.P + 3) & ~3u) : 0);
  const int last = D.k - 1;
  const I Llast = (I)D.L[last];
  const uint32_t* __restrict__ cg = ctab + tabs.off[last];
  if (TSMEM)
    for (uint32_t i = threadIdx.x; i < D.P; i += blockDim.x) Ts[i] = __ldg(Tg + i);
  if (MODE == M_FAST_SMEM)
    for (uint32_t i = threadIdx.x; i < (uint32_t)Llast; i += blockDim.x) Cs[i] = __ldg(cg + i);
  __syncthreads();

  const I N = (I)D.npoints;
  const I groups = (N + 3) / 4;
  const I warp_id = (I)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const I gbeg = warp_id * (I)groups_per_warp;
  const I gend = min(groups, gbeg + (I)groups_per_warp);
  I g = gbeg + (threadIdx.x & 31);
  if (g >= gend) return;
  I lin0 = g * 4;
  I row, x;
  split_lin<I>(D, lin0, row, x);
  uint32_t base = row_base<I>(D, tabs, ctab, row);

  for (; g < gend; g += 32, lin0 += 128) {
    uint32_t v0, v1, v2, v3;
    int cnt = 4;
    if (MODE != M_GENERAL) {
      // Llast % 4 == 0: the group lies inside one row and x % 4 == 0
      const uint4 c = MODE == M_FAST_SMEM ? *reinterpret_cast<const uint4*>(Cs + x)
                                          : __ldg(reinterpret_cast<const uint4*>(cg + x));
      if (TSMEM) {
        v0 = Ts[base + c.x]; v1 = Ts[base + c.y]; v2 = Ts[base + c.z]; v3 = Ts[base + c.w];
      } else {
        v0 = __ldg(Tg + base + c.x); v1 = __ldg(Tg + base + c.y);
        v2 = __ldg(Tg + base + c.z); v3 = __ldg(Tg + base + c.w);
      }
    } else {
      // any shape: walk the four points, carrying into the next rows
      cnt = N - lin0 < 4 ? (int)(N - lin0) : 4;
      I xi = x, ri = row;
      uint32_t bi = base;
      uint32_t v[4] = {0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i < cnt) {
          if (xi == Llast) {
            xi = 0;
            ri += 1;
            bi = row_base<I>(D, tabs, ctab, ri);
          }
          const uint32_t c = tabs.has[last] ? __ldg(cg + xi) : contrib(D, last, (uint64_t)xi);
          v[i] = TSMEM ? Ts[bi + c] : __ldg(Tg + bi + c);
          ++xi;
        }
      }
      v0 = v[0]; v1 = v[1]; v2 = v[2]; v3 = v[3];
    }
    if (cnt == 4 && vec_ok) {
      __stcs(reinterpret_cast<int4*>(ids + lin0), make_int4((int)v0, (int)v1, (int)v2, (int)v3));
    } else {
      const uint32_t vv[4] = {v0, v1, v2, v3};
      for (int i = 0; i < cnt; ++i) ids[lin0 + i] = (int32_t)vv[i];
    }
    // next group of this lane: 128 points further
    x += 128;
    if (x >= Llast) {
      if (Llast >= 128) {
        x -= Llast;
        row += 1;
      } else {
        split_lin<I>(D, lin0 + 128, row, x);
      }
      base = row_base<I>(D, tabs, ctab, row);
    }
  }
}

// Linear-cyclic (Fig. 5): F = lin mod P; consecutive points advance F by 1
// and consecutive groups of a lane by 128 mod P.
template <typename I, bool TSMEM>
__global__ void __launch_bounds__(kThreads) k_ids_lc(const __grid_constant__ MapDesc D,
                                                     const uint32_t* __restrict__ Tg, int vec_ok,
                                                     uint64_t groups_per_warp, int32_t* __restrict__ ids) {
  extern __shared__ __align__(16) uint32_t smem[];
  if (TSMEM) {
    for (uint32_t i = threadIdx.x; i < D.P; i += blockDim.x) smem[i] = __ldg(Tg + i);
    __syncthreads();
  }
  const I N = (I)D.npoints;
  const I groups = (N + 3) / 4;
  const I warp_id = (I)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const I gbeg = warp_id * (I)groups_per_warp;
  const I gend = min(groups, gbeg + (I)groups_per_warp);
  I g = gbeg + (threadIdx.x & 31);
  if (g >= gend) return;
  I lin0 = g * 4;
  uint64_t q, F64;
  divmod64((uint64_t)lin0, D.divP64, q, F64);
  uint32_t F0 = (uint32_t)F64;
  const uint32_t inc = 128 % D.P;
  for (; g < gend; g += 32, lin0 += 128) {
    const int cnt = N - lin0 < 4 ? (int)(N - lin0) : 4;
    uint32_t v[4];
    uint32_t F = F0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      v[i] = TSMEM ? smem[F] : __ldg(Tg + F);
      F = (F + 1 == D.P) ? 0 : F + 1;
    }
    if (cnt == 4 && vec_ok) {
      __stcs(reinterpret_cast<int4*>(ids + lin0), make_int4((int)v[0], (int)v[1], (int)v[2], (int)v[3]));
    } else {
      for (int i = 0; i < cnt; ++i) ids[lin0 + i] = (int32_t)v[i];
    }
    F0 += inc;
    if (F0 >= D.P) F0 -= D.P;
  }
}

// ----------------------------------------------------------------- k_lc_slabs

// Linear-cyclic halo: along a dimension t whose linear stride is not a
// multiple of P every neighbour pair crosses, so a point receives
// face_t for each neighbour it has.  Each point of the slabs x_t = 0 and
// x_t = L_t - 1 lacks one neighbour; deficit[F] collects face_t for them.
__global__ void __launch_bounds__(kThreads) k_lc_slabs(const __grid_constant__ MapDesc D,
                                                       uint64_t f0, uint64_t f1, uint64_t f2,
                                                       uint64_t f3,
                                                       unsigned long long* __restrict__ deficit) {
  const uint64_t face[4] = {f0, f1, f2, f3};
  const uint64_t N = D.npoints;
  for (int t = 0; t < D.k; ++t) {
    if (D.lc_stride_mod[t] == 0 || face[t] == 0) continue;
    const uint64_t per_slab = N / D.L[t];
    const uint64_t stride = D.lc_stride[t];
    const Div64 dstride = Div64{stride, ~0ull / stride};
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * per_slab;
         e += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t side = e >= per_slab;
      const uint64_t s = e - side * per_slab;
      uint64_t hi, lo;
      divmod64(s, dstride, hi, lo);
      const uint64_t xt = side ? D.L[t] - 1 : 0;
      const uint64_t lin = hi * (D.L[t] * stride) + xt * stride + lo;
      uint64_t q, F;
      divmod64(lin, D.divP64, q, F);
      atomicAdd(deficit + F, (unsigned long long)face[t]);
    }
  }
}

// ----------------------------------------------------------------- k_reduce

__global__ void __launch_bounds__(kThreads) k_reduce(const __grid_constant__ MapDesc D,
                                                     const uint32_t* __restrict__ T,
                                                     const unsigned long long* __restrict__ H,
                                                     const unsigned long long* __restrict__ X,
                                                     const unsigned long long* __restrict__ deficit,
                                                     uint64_t f0, uint64_t f1, uint64_t f2, uint64_t f3,
                                                     uint64_t* __restrict__ hist,
                                                     uint64_t* __restrict__ recv,
                                                     unsigned long long* __restrict__ total) {
  const uint64_t face[4] = {f0, f1, f2, f3};
  const uint32_t F = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t r_F = 0;
  if (F < D.P) {
    uint64_t h_F;
    if (!D.lc) {
      uint32_t part[4] = {0, 0, 0, 0};
      uint32_t rest = F;
      for (int u = 0; u < D.rank; ++u) {
        uint32_t q, r;
        divmod32(rest, D.divs[u], q, r);
        rest = q;
        part[D.owner_dim[u]] += r * D.sigma[u];
      }
      uint64_t h[4], xc[4];
      h_F = 1;
      for (int t = 0; t < D.k; ++t) {
        h[t] = H[(uint64_t)t * D.P + part[t]];
        xc[t] = X ? X[(uint64_t)t * D.P + part[t]] : 0;
        h_F *= h[t];
      }
      if (X)
        for (int t = 0; t < D.k; ++t) {
          uint64_t v = face[t] * xc[t];
          for (int u = 0; u < D.k; ++u)
            if (u != t) v *= h[u];
          r_F += v;
        }
    } else {
      // C-order linear indices cover [0, N): lin = F (mod P) occurs
      // floor(N / P) times, once more when F < N mod P.
      uint64_t q, rem;
      divmod64(D.npoints, D.divP64, q, rem);
      h_F = q + (F < rem ? 1 : 0);
      if (deficit) {
        uint64_t G = 0;
        for (int t = 0; t < D.k; ++t)
          if (D.lc_stride_mod[t] != 0) G += 2 * face[t];
        r_F = G * h_F - deficit[F];
      }
    }
    const uint32_t id = T[F];
    if (hist) hist[id] = h_F;
    if (recv) recv[id] = r_F;
  }
  if (total) {
    __shared__ unsigned long long red[kThreads / 32];
    unsigned long long v = r_F;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      v = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
      if (threadIdx.x == 0 && v) atomicAdd(total, v);
    }
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 132;
  }
  return n;
}

struct Want {
  int32_t* ids;
  uint64_t* hist;
  uint64_t* recv;
  uint64_t* total;
  uint64_t face[4];
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Runs the kernels of one launch into device buffers.
// Device scratch of one launch: the chain table T, the per-dimension c_t
// tables, the per-dimension counts H / X and the linear-cyclic deficits.
struct Layout {
  Tabs tabs;
  uint64_t tab_total;
  size_t o_T, o_tab, o_H, o_X, o_def, nHX, n_def, bytes;
  bool need_red, need_X;
};

Layout make_layout(const MapDesc& D, const Want& w) {
  Layout ly;
  std::memset(&ly, 0, sizeof(ly));
  ly.need_red = w.hist || w.recv || w.total;
  ly.need_X = (w.recv || w.total) && !D.lc;
  for (int t = 0; t < D.k; ++t) {
    ly.tabs.has[t] = !D.lc && D.L[t] <= kTableMax;
    ly.tabs.off[t] = ly.tab_total;
    if (ly.tabs.has[t]) ly.tab_total += (D.L[t] + 3) & ~uint64_t(3);
  }
  ly.o_T = 0;
  ly.o_tab = align256(ly.o_T + (size_t)D.P * 4);
  ly.o_H = align256(ly.o_tab + ly.tab_total * 4);
  ly.nHX = ly.need_red && !D.lc ? (size_t)D.k * D.P : 0;
  ly.o_X = align256(ly.o_H + ly.nHX * 8);
  ly.o_def = align256(ly.o_X + (ly.need_X ? ly.nHX * 8 : 0));
  ly.n_def = D.lc && (w.recv || w.total) ? D.P : 0;
  ly.bytes = align256(ly.o_def + ly.n_def * 8);
  return ly;
}

// Runs the kernels of one launch into device buffers, with the scratch at ws
// (at least ly.bytes).
int run_launch_ws(const Plan& pl, const Want& w, const Layout& ly, char* ws, cudaStream_t st) {
  const MapDesc& D = pl.desc;
  const Tabs& tabs = ly.tabs;
  const uint64_t tab_total = ly.tab_total;
  const bool need_red = ly.need_red;
  const size_t nHX = ly.nHX, n_def = ly.n_def;
  uint32_t* T = (uint32_t*)(ws + ly.o_T);
  uint32_t* ctab = (uint32_t*)(ws + ly.o_tab);
  unsigned long long* H = nHX ? (unsigned long long*)(ws + ly.o_H) : nullptr;
  unsigned long long* X = ly.need_X ? (unsigned long long*)(ws + ly.o_X) : nullptr;
  unsigned long long* def = n_def ? (unsigned long long*)(ws + ly.o_def) : nullptr;

  // ------------------------------------------------ tables
  k_resolve<<<(D.P + kThreads - 1) / kThreads, kThreads, 0, st>>>(D, T);
  count_launch();
  if (H) MP_CUDA_TRY(cudaMemsetAsync(H, 0, nHX * 8, st));
  if (X) MP_CUDA_TRY(cudaMemsetAsync(X, 0, nHX * 8, st));
  uint64_t sumL = 0;
  for (int t = 0; t < D.k; ++t) sumL += D.L[t];
  const bool want_tabs = tab_total > 0 && w.ids;
  if (!D.lc && (want_tabs || H)) {
    uint64_t blocks = std::min<uint64_t>((sumL + kThreads - 1) / kThreads, (uint64_t)sm_count() * 16);
    k_dimtables<<<(unsigned)blocks, kThreads, 0, st>>>(D, tabs, sumL, ctab, H, X);
    count_launch();
  }
  // ------------------------------------------------ ids
  if (w.ids) {
    timer_begin(st);
    const int vec_ok = ((uintptr_t)w.ids & 15) == 0;
    const bool tsmem = D.P <= kSmemTMax;
    const int last = D.k - 1;
    const uint64_t groups = (D.npoints + 3) / 4;
    const bool wide = D.npoints > 0xFFFFFFFFull - 1024;
    const size_t tbytes = tsmem ? (size_t)((D.P + 3) & ~3u) * 4 : 0;
    auto grid_for = [&](const void* kern, size_t sm, uint64_t& gpw) {
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
      if (per_sm < 1) per_sm = 1;
      uint64_t blocks = (uint64_t)sm_count() * per_sm;
      const uint64_t warps_needed = (groups + 31) / 32;
      blocks = std::max<uint64_t>(1, std::min<uint64_t>(blocks, (warps_needed + 7) / 8));
      const uint64_t warps = blocks * (kThreads / 32);
      gpw = ((groups + warps - 1) / warps + 31) / 32 * 32;
      return (unsigned)blocks;
    };
    auto go = [&](const void* kern, size_t sm, auto launch) {
      if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      uint64_t gpw = 0;
      const unsigned blocks = grid_for(kern, sm, gpw);
      launch(blocks, gpw);
      count_launch();
    };
    if (D.lc) {
      const size_t sm = tbytes;
#define MP_LC(I, TS) go((const void*)k_ids_lc<I, TS>, sm, [&](unsigned b, uint64_t gpw) { \
        k_ids_lc<I, TS><<<b, kThreads, sm, st>>>(D, T, vec_ok, gpw, w.ids); })
      if (wide) { if (tsmem) MP_LC(uint64_t, true); else MP_LC(uint64_t, false); }
      else { if (tsmem) MP_LC(uint32_t, true); else MP_LC(uint32_t, false); }
#undef MP_LC
    } else {
      const bool aligned = D.L[last] % 4 == 0 && tabs.has[last];
      const int mode = !aligned ? M_GENERAL : (D.L[last] <= kSmemLastMax ? M_FAST_SMEM : M_FAST_GLOBAL);
      const size_t sm = tbytes + (mode == M_FAST_SMEM ? (size_t)D.L[last] * 4 : 0);
#define MP_IDS(I, MODE, TS) go((const void*)k_ids<I, MODE, TS>, sm, [&](unsigned b, uint64_t gpw) { \
        k_ids<I, MODE, TS><<<b, kThreads, sm, st>>>(D, tabs, T, ctab, vec_ok, gpw, w.ids); })
#define MP_IDS_T(I, MODE) do { if (tsmem) MP_IDS(I, MODE, true); else MP_IDS(I, MODE, false); } while (0)
#define MP_IDS_M(I) do { if (mode == M_FAST_SMEM) MP_IDS_T(I, M_FAST_SMEM); \
                         else if (mode == M_FAST_GLOBAL) MP_IDS_T(I, M_FAST_GLOBAL); \
                         else MP_IDS_T(I, M_GENERAL); } while (0)
      if (wide) MP_IDS_M(uint64_t); else MP_IDS_M(uint32_t);
#undef MP_IDS_M
#undef MP_IDS_T
#undef MP_IDS
    }
    timer_end(st);
    MP_CUDA_TRY(cudaGetLastError());
  }
  // ------------------------------------------------ reductions
  if (need_red) {
    if (w.total) MP_CUDA_TRY(cudaMemsetAsync(w.total, 0, 8, st));
    if (def) {
      MP_CUDA_TRY(cudaMemsetAsync(def, 0, n_def * 8, st));
      uint64_t work = 0;
      for (int t = 0; t < D.k; ++t) work += 2 * (D.npoints / D.L[t]);
      uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((work + kThreads - 1) / kThreads,
                                                                   (uint64_t)sm_count() * 8));
      k_lc_slabs<<<(unsigned)blocks, kThreads, 0, st>>>(D, w.face[0], w.face[1], w.face[2], w.face[3], def);
      count_launch();
    }
    k_reduce<<<(D.P + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        D, T, H, X, def, w.face[0], w.face[1], w.face[2], w.face[3], w.hist, w.recv,
        (unsigned long long*)w.total);
    count_launch();
  }
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

// Runs one launch with the scratch in the per-device workspace.
int run_launch(const Plan& pl, const Want& w, cudaStream_t st) {
  const Layout ly = make_layout(pl.desc, w);
  char* ws = (char*)workspace(ly.bytes, 0);
  if (!ws) return MP_ENOMEM;
  return run_launch_ws(pl, w, ly, ws, st);
}

// Resolves host/device outputs: device buffers are used directly, host
// buffers get a device staging area (workspace slot 1) and a copy back.
struct Staged {
  void* user;
  void* dev;
  size_t bytes;
};

int stage(void* user, size_t bytes, size_t& cursor, std::vector<Staged>& list, char* base,
          void** dev_out) {
  if (!user) {
    *dev_out = nullptr;
    return MP_OK;
  }
  if (is_device_pointer(user)) {
    *dev_out = user;
    return MP_OK;
  }
  *dev_out = base ? base + cursor : nullptr;
  list.push_back(Staged{user, *dev_out, bytes});
  cursor = align256(cursor + bytes);
  return MP_OK;
}

int run_with_staging(const Plan& pl, int32_t* ids, uint64_t* hist, uint64_t* recv, uint64_t* total,
                     const uint64_t* face, cudaStream_t st) {
  const MapDesc& D = pl.desc;
  size_t need = 0;
  auto host_bytes = [&](void* p, size_t b) {
    if (p && !is_device_pointer(p)) need = align256(need + b);
  };
  host_bytes(ids, D.npoints * 4);
  host_bytes(hist, (size_t)D.P * 8);
  host_bytes(recv, (size_t)D.P * 8);
  host_bytes(total, 8);
  char* base = nullptr;
  if (need) {
    base = (char*)workspace(need, 1);
    if (!base) return MP_ENOMEM;
  }
  std::vector<Staged> list;
  size_t cur = 0;
  Want w;
  std::memset(&w, 0, sizeof(w));
  void* p;
  stage(ids, D.npoints * 4, cur, list, base, &p); w.ids = (int32_t*)p;
  stage(hist, (size_t)D.P * 8, cur, list, base, &p); w.hist = (uint64_t*)p;
  stage(recv, (size_t)D.P * 8, cur, list, base, &p); w.recv = (uint64_t*)p;
  stage(total, 8, cur, list, base, &p); w.total = (uint64_t*)p;
  for (int t = 0; t < 4; ++t) w.face[t] = face && t < D.k ? face[t] : 0;
  int rc = run_launch(pl, w, st);
  if (rc) return rc;
  for (auto& s : list) MP_CUDA_TRY(cudaMemcpyAsync(s.user, s.dev, s.bytes, cudaMemcpyDeviceToHost, st));
  if (!list.empty()) MP_CUDA_TRY(cudaStreamSynchronize(st));
  return MP_OK;
}

}  // namespace

}  // namespace mp

extern "C" int mp_map_points(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                             int n_xf, const mp_dist* dist, int32_t* ids, uint64_t* hist,
                             void* stream) {
  mp::Plan pl;
  int rc = mp::build_plan(space, machine, chain, n_xf, dist, pl);
  if (rc) return rc;
  if (!ids && !hist) return MP_OK;
  return mp::run_with_staging(pl, ids, hist, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int mp_comm_volume(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                              int n_xf, const mp_dist* dist, const uint64_t* face_bytes,
                              uint64_t* total, uint64_t* recv, void* stream) {
  mp::Plan pl;
  int rc = mp::build_plan(space, machine, chain, n_xf, dist, pl);
  if (rc) return rc;
  if (!face_bytes || !total) return MP_EINVAL;
  return mp::run_with_staging(pl, nullptr, nullptr, recv, total, face_bytes, (cudaStream_t)stream);
}

// ------------------------------------------------------------ no-allocation variant
//
// mp_map_points_noalloc: the same launch as mp_map_points, with its scratch
// (chain table, per-dimension tables and counts) in one fixed array of this
// module's device memory instead of the grow-on-demand workspace.

namespace mp {
namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;   // 8 MiB on every device that loads the library

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// The array's name is a host-side stand-in in host code; its device address
// is looked up once per device, with that device current.
int noalloc_scratch(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MP_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return MP_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = (char*)g_noalloc_addr[dev];
  return MP_OK;
}

}  // namespace
}  // namespace mp

extern "C" int mp_map_points_noalloc(const mp_space* space, const mp_machine* machine,
                                     const mp_xform* chain, int n_xf, const mp_dist* dist, int32_t* ids,
                                     uint64_t* hist, void* stream) {
  mp::Plan pl;
  int rc = mp::build_plan(space, machine, chain, n_xf, dist, pl);
  if (rc) return rc;
  if (!ids && !hist) return MP_OK;
  if ((ids && !mp::is_device_pointer(ids)) || (hist && !mp::is_device_pointer(hist))) return MP_EINVAL;
  mp::Want w;
  std::memset(&w, 0, sizeof(w));
  w.ids = ids;
  w.hist = hist;
  const mp::Layout ly = mp::make_layout(pl.desc, w);
  if (ly.bytes > mp::kNoAllocBytes) return MP_ENOTSUP;
  char* ws = nullptr;
  rc = mp::noalloc_scratch(&ws);
  if (rc) return rc;
  return mp::run_launch_ws(pl, w, ly, ws, (cudaStream_t)stream);
}
