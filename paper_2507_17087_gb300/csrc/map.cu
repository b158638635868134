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
//   id(x) = T[F(x)],  T = chain resolution of every F in [0, P),
// and owner(x) != owner(y) iff F(x) != F(y).
// Kernels:
//   k_resolve   T[F] for F < P (Fig. 4 inverses, last to first)        (a3)
//   k_prep      T and c_t(x_t) for every coordinate of the tabled
//               dimensions in one launch (when ids want the tables) (a2-a3)
//   k_ids       ids[lin] = T[base(row) + c_last(x_last)], 16-byte
//               stores, one contiguous range per warp               (a1-a3)
//   k_counts    per-dimension counts in closed form: H_t[j] points whose
//               dimension-t sub-index is j, X_t[j] neighbour pairs along t
//               that leave such a point and change owner
//   k_reduce    hist[T[F]] = prod_t H_t, recv[T[F]] =
//               sum_t face_t X_t prod_{u != t} H_u, total = sum recv  (a4, a5)
//   k_lc_slabs  linear-cyclic only: boundary points missing a neighbour.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace mp {

namespace {

__global__ void __launch_bounds__(kThreads) k_resolve(const __grid_constant__ MapDesc D, uint32_t* __restrict__ T) {
  const uint32_t F = blockIdx.x * blockDim.x + threadIdx.x;
  if (F < D.P) T[F] = resolve_F(D, D.prim, D.nprim, F);
}

// The chain table and the c_t tables in one launch: flat final index e < P
// resolves the chain, the rest are table entries (c_t(x) for every
// coordinate x of the tabled dimensions).
__global__ void __launch_bounds__(kThreads) k_prep(const __grid_constant__ MapDesc D,
                                                   const __grid_constant__ Tabs tabs, uint64_t tab_total,
                                                   uint32_t* __restrict__ T, uint32_t* __restrict__ ctab) {
  const uint64_t total = (uint64_t)D.P + tab_total;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    if (e < D.P) {
      T[e] = resolve_F(D, D.prim, D.nprim, (uint32_t)e);
      continue;
    }
    const uint64_t r = e - D.P;
    int t = -1;
    for (int u = 0; u < D.k; ++u)
      if (tabs.has[u] && r >= tabs.off[u]) t = u;
    if (t < 0) continue;
    const uint64_t x = r - tabs.off[t];
    if (x < D.L[t]) ctab[r] = contrib(D, t, x);
  }
}

// elem_mode = 1: X holds the element counts (dim_elems) for halo widths w.
__global__ void __launch_bounds__(kThreads) k_counts(const __grid_constant__ MapDesc D, uint64_t* __restrict__ H,
                                                     uint64_t* __restrict__ X, int elem_mode, uint32_t w0,
                                                     uint32_t w1, uint32_t w2, uint32_t w3) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D.Jtotal) return;
  int t = 0;
  while (t < D.k - 1 && e >= D.Joff[t + 1]) ++t;
  uint64_t h, xc;
  dim_counts(D, t, e - D.Joff[t], h, xc);
  H[e] = h;
  if (X) {
    const uint32_t w[4] = {w0, w1, w2, w3};
    X[e] = elem_mode ? dim_elems(D, t, e - D.Joff[t], w[t]) : xc;
  }
}

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
  if (TSMEM)
    for (uint32_t i = threadIdx.x; i < D.P; i += blockDim.x) Ts[i] = __ldg(Tg + i);
  if (MODE == M_FAST_SMEM)
    for (uint32_t i = threadIdx.x; i < (uint32_t)D.L[last]; i += blockDim.x) Cs[i] = __ldg(ctab + tabs.off[last] + i);
  __syncthreads();
  const I groups = (I)((D.npoints + 3) / 4);
  const I warp_id = (I)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const I gbeg = warp_id * (I)groups_per_warp;
  const I gend = min(groups, gbeg + (I)groups_per_warp);
  ids_range<I, MODE, TSMEM>(D, tabs, TSMEM ? Ts : Tg, Cs, ctab, gbeg, gend, threadIdx.x & 31, vec_ok, ids);
}

// Rows of Lf points (the dimensions m..k-1; their contributions computed
// into shared memory by each CTA when SRC is a table source, or taken from
// the last dimension's components in place) for launches whose last extent
// is unaligned or untabled; 32-bit indices.
template <int SRC, bool TSMEM>
__global__ void __launch_bounds__(kThreads) k_ids_rows(const __grid_constant__ MapDesc D,
                                                       const __grid_constant__ Tabs tabs,
                                                       const uint32_t* __restrict__ Tg,
                                                       const uint32_t* __restrict__ ctab, int m, uint32_t Lf,
                                                       Div32 divLf, int vec_ok, uint64_t groups_per_warp,
                                                       int32_t* __restrict__ ids) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* Ts = smem;
  uint32_t* Cf = smem + (TSMEM ? ((D.P + 3) & ~3u) : 0);
  if (TSMEM)
    for (uint32_t i = threadIdx.x; i < D.P; i += blockDim.x) Ts[i] = __ldg(Tg + i);
  if (SRC == R_TAB || SRC == R_TAB4)
    for (uint32_t x = threadIdx.x; x < Lf; x += blockDim.x) {
      // row offset x -> coordinates of dimensions m..k-1 (C order)
      uint32_t rest = x, c = 0;
      for (int t = D.k - 1; t >= m; --t) {
        uint32_t q, r;
        divmod32(rest, D.divL32[t], q, r);
        c += contrib(D, t, r);
        rest = q;
      }
      Cf[x] = c;
    }
  __syncthreads();
  const uint32_t groups = (uint32_t)((D.npoints + 3) / 4);
  const uint32_t warp_id = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const uint64_t gb = (uint64_t)warp_id * groups_per_warp;
  if (gb >= groups) return;
  const uint32_t gbeg = (uint32_t)gb;
  const uint64_t ge = gb + groups_per_warp;
  const uint32_t gend = (uint32_t)(ge < groups ? ge : groups);
  ids_range_rows<SRC>(D, tabs, TSMEM ? Ts : Tg, Cf, ctab, RowAux{}, m, Lf, divLf, gbeg, gend, threadIdx.x & 31,
                      vec_ok, ids);
}

template <typename I, bool TSMEM>
__global__ void __launch_bounds__(kThreads) k_ids_lc(const __grid_constant__ MapDesc D,
                                                     const uint32_t* __restrict__ Tg, int vec_ok,
                                                     uint64_t groups_per_warp, int32_t* __restrict__ ids) {
  extern __shared__ __align__(16) uint32_t smem[];
  if (TSMEM) {
    for (uint32_t i = threadIdx.x; i < D.P; i += blockDim.x) smem[i] = __ldg(Tg + i);
    __syncthreads();
  }
  const I groups = (I)((D.npoints + 3) / 4);
  const I warp_id = (I)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const I gbeg = warp_id * (I)groups_per_warp;
  const I gend = min(groups, gbeg + (I)groups_per_warp);
  ids_range_lc<I, TSMEM>(D, TSMEM ? smem : Tg, gbeg, gend, threadIdx.x & 31, vec_ok, ids);
}

// Linear-cyclic halo: a point receives face_t for each neighbour it has
// along every dimension whose linear stride is not a multiple of P; the
// points of the slabs x_t = 0 and x_t = L_t - 1 each lack one.
__global__ void __launch_bounds__(kThreads) k_lc_slabs(const __grid_constant__ MapDesc D, uint64_t f0, uint64_t f1,
                                                       uint64_t f2, uint64_t f3,
                                                       unsigned long long* __restrict__ deficit) {
  const uint64_t face[4] = {f0, f1, f2, f3};
  for (int t = 0; t < D.k; ++t) {
    if (D.lc_stride_mod[t] == 0 || face[t] == 0) continue;
    const uint64_t n = 2 * (D.npoints / D.L[t]);
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x)
      atomicAdd(deficit + lc_slab_F(D, t, e), (unsigned long long)face[t]);
  }
}

// Element-count halo of a linear-cyclic launch: the points of the boundary
// slabs lack the offsets their cut window does not reach; each such offset
// comes off the receiving flat index F + offset.
__global__ void __launch_bounds__(kThreads) k_lc_wslabs(const __grid_constant__ MapDesc D,
                                                        const __grid_constant__ LcHalo lh, uint64_t f0,
                                                        uint64_t f1, uint64_t f2, uint64_t f3, uint32_t w0,
                                                        uint32_t w1, uint32_t w2, uint32_t w3,
                                                        unsigned long long* __restrict__ deficit) {
  const uint64_t face[4] = {f0, f1, f2, f3};
  const uint64_t wd[4] = {w0, w1, w2, w3};
  for (int t = 0; t < D.k; ++t) {
    if (lh.n[t] == 0 || face[t] == 0) continue;
    const uint64_t Lt = D.L[t];
    const uint64_t lo_n = wd[t] < Lt ? wd[t] : Lt;
    const uint64_t hi_n = wd[t] < Lt - lo_n ? wd[t] : Lt - lo_n;
    const uint64_t n = (lo_n + hi_n) * (D.npoints / Lt);
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (uint64_t)gridDim.x * blockDim.x) {
      uint64_t xt;
      const uint32_t F = lc_wslab_point(D, t, e, lo_n, xt);
      const uint64_t a = xt < wd[t] ? xt : wd[t];                     // reach towards 0
      const uint64_t b = Lt - 1 - xt < wd[t] ? Lt - 1 - xt : wd[t];   // reach towards L_t - 1
      for (uint32_t i = 0; i < lh.n[t]; ++i) {
        const bool reached = (lh.pos[t][i] && lh.pos[t][i] <= b) || (lh.neg[t][i] && lh.neg[t][i] <= a);
        if (reached) continue;
        uint32_t G = F + lh.off[t][i];
        if (G >= D.P) G -= D.P;
        atomicAdd(deficit + G, (unsigned long long)face[t]);
      }
    }
  }
}

// Linear-cyclic face deficits without one atomic per boundary point (the
// batched path does the same): the slab rows of every dimension but the last
// are cyclic runs of residues -- whole turns into defall, the rest into the
// difference array D (2 N / (L_t S_t) entries for dimension t); k_lc_scan
// prefix-sums D and counts the last dimension's slabs per residue in closed
// form.  Used when P <= kLcScanMax.
constexpr uint32_t kLcScanMax = 1u << 20;

struct LcRuns {
  uint64_t begin[5];   // work entries of dimensions 0 .. k-2, prefix
};

__global__ void __launch_bounds__(kThreads) k_lc_runs(const __grid_constant__ MapDesc D, const __grid_constant__ LcRuns R,
                                                      uint64_t f0, uint64_t f1, uint64_t f2, uint64_t f3,
                                                      unsigned long long* __restrict__ Dd,
                                                      unsigned long long* __restrict__ defall) {
  const uint64_t face[4] = {f0, f1, f2, f3};
  const uint64_t total = R.begin[D.k - 1];
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    int t = 0;
    while (e >= R.begin[t + 1]) ++t;
    const uint64_t S = D.lc_stride[t], Lt = D.L[t];
    const uint64_t H = D.npoints / (Lt * S);
    const uint64_t local = e - R.begin[t];
    const uint64_t side = local / H, hi = local - side * H;
    const uint64_t xt = side ? Lt - 1 : 0;
    const unsigned long long f = face[t];
    uint64_t q0, r0, full, rem;
    divmod64(hi * (Lt * S) + xt * S, D.divP64, q0, r0);
    divmod64(S, D.divP64, full, rem);
    if (full) atomicAdd(defall, full * f);
    if (rem) {
      const uint64_t end = r0 + rem;
      atomicAdd(Dd + r0, f);
      if (end < D.P) {
        atomicAdd(Dd + end, (unsigned long long)(-(long long)f));
      } else if (end > D.P) {
        atomicAdd(Dd, f);
        atomicAdd(Dd + (end - D.P), (unsigned long long)(-(long long)f));
      }
    }
  }
}

__global__ void __launch_bounds__(1024) k_lc_scan(const __grid_constant__ MapDesc D, uint64_t f_last,
                                                  unsigned long long* __restrict__ Dd,
                                                  const unsigned long long* __restrict__ defall) {
  __shared__ unsigned long long part[1024];
  __shared__ int64_t s_g, s_inv;
  const int last = D.k - 1;
  const bool last_slabs = D.lc_stride_mod[last] != 0 && f_last != 0;
  if (threadIdx.x == 0 && last_slabs) {
    int64_t g, inv;
    gcd_inverse((int64_t)(D.L[last] % D.P), (int64_t)D.P, g, inv);
    s_g = g;
    s_inv = inv;
  }
  const uint32_t P = D.P;
  const uint32_t per = (P + 1023) / 1024;
  const uint32_t lo = min(P, threadIdx.x * per), hi = min(P, lo + per);
  unsigned long long sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += Dd[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = (threadIdx.x ? part[threadIdx.x - 1] : 0) + *defall;
  const int64_t g = last_slabs ? s_g : 1, inv = last_slabs ? s_inv : 0, M = (int64_t)P / g;
  const uint64_t Lt = D.L[last], H = D.npoints / Lt;
  for (uint32_t i = lo; i < hi; ++i) {
    run += Dd[i];
    unsigned long long add = 0;
    if (last_slabs)
      for (int side = 0; side < 2; ++side) {
        const int64_t x = side ? (int64_t)((Lt - 1) % P) : 0;
        const int64_t c = ((int64_t)i - x + (int64_t)P) % (int64_t)P;
        if (c % g) continue;
        const int64_t h0 = M == 1 ? 0 : (int64_t)(((unsigned __int128)(c / g) * (uint64_t)inv) % (uint64_t)M);
        add += count_residue(H, (uint64_t)h0, (uint64_t)M);
      }
    Dd[i] = run + add * f_last;
  }
}

__global__ void __launch_bounds__(kThreads) k_reduce(const __grid_constant__ MapDesc D, const uint32_t* __restrict__ T,
                                                     const uint64_t* __restrict__ H, const uint64_t* __restrict__ X,
                                                     const uint64_t* __restrict__ deficit, uint64_t f0, uint64_t f1,
                                                     uint64_t f2, uint64_t f3, uint64_t* __restrict__ hist,
                                                     uint64_t* __restrict__ recv,
                                                     unsigned long long* __restrict__ total,
                                                     const __grid_constant__ LcHalo lh, int use_lh) {
  const uint64_t face[4] = {f0, f1, f2, f3};
  const uint32_t F = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t r_F = 0;
  if (F < D.P) {
    uint64_t h_F;
    reduce_F(D, H, X, deficit, face, recv || total, F, h_F, r_F, use_lh ? &lh : nullptr);
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
  uint64_t face[4];     // bytes per face (faces mode) or per element
  int elem_mode;        // 1: element-count halo with widths
  uint32_t width[4];
};

// Offsets of the element-count halo of a linear-cyclic launch (see LcHalo).
LcHalo make_lc_halo(const MapDesc& D, const Want& w) {
  LcHalo lh;
  std::memset(&lh, 0, sizeof(lh));
  for (int t = 0; t < D.k; ++t) {
    const uint64_t S = D.lc_stride_mod[t];
    for (uint32_t delta = 1; delta <= w.width[t] && delta < D.L[t]; ++delta) {
      const uint32_t plus = (uint32_t)(((unsigned __int128)delta * S) % D.P);
      const uint32_t minus = plus ? D.P - plus : 0;
      for (int side = 0; side < 2; ++side) {
        const uint32_t off = side ? minus : plus;
        if (off == 0) continue;
        uint32_t i = 0;
        while (i < lh.n[t] && lh.off[t][i] != off) ++i;
        if (i == lh.n[t]) lh.off[t][lh.n[t]++] = off;
        uint8_t& slot = side ? lh.neg[t][i] : lh.pos[t][i];
        if (!slot) slot = (uint8_t)delta;
      }
    }
  }
  return lh;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr uint64_t kIdsWarpGroups = 1024;   // single-launch id writers: 4-point groups per warp (target)
constexpr uint64_t kIdsMaxWaves = 32;       // and at most this many waves of CTAs

// A second stream (and its fork / join events) per host thread and device,
// for the reductions that run beside an id writer.  Null if it cannot be
// created (the reductions then run on the caller's stream).
struct ForkStreams {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool ok = false;
  ~ForkStreams() {
    if (side) cudaStreamDestroy(side);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
};

const ForkStreams* fork_streams() {
  constexpr int kMaxDevices = 64;
  thread_local ForkStreams per_device[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  ForkStreams& f = per_device[dev];
  if (!f.ok && !f.side) {
    f.ok = cudaStreamCreateWithFlags(&f.side, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming) == cudaSuccess;
    if (!f.ok) cudaGetLastError();
  }
  return f.ok ? &f : nullptr;
}

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
  if (w.ids)
    for (int t = 0; t < D.k; ++t) {
      ly.tabs.has[t] = !D.lc && D.L[t] <= kTableMax;
      ly.tabs.off[t] = ly.tab_total;
      if (ly.tabs.has[t]) ly.tab_total += (D.L[t] + 3) & ~uint64_t(3);
    }
  ly.o_T = 0;
  ly.o_tab = align256(ly.o_T + (size_t)D.P * 4);
  ly.o_H = align256(ly.o_tab + ly.tab_total * 4);
  ly.nHX = ly.need_red && !D.lc ? (size_t)D.Jtotal : 0;
  ly.o_X = align256(ly.o_H + ly.nHX * 8);
  ly.o_def = align256(ly.o_X + (ly.need_X ? ly.nHX * 8 : 0));
  ly.n_def = D.lc && (w.recv || w.total) ? D.P + 1 : 0;   // + the whole-turn word of the runs
  ly.bytes = align256(ly.o_def + ly.n_def * 8);
  return ly;
}

// Runs the kernels of one launch into device buffers, with the scratch at ws
// (at least ly.bytes).
int run_launch_ws(const Plan& pl, const Want& w, const Layout& ly, char* ws, cudaStream_t st, bool side_stream) {
  const MapDesc& D = pl.desc;
  const Tabs& tabs = ly.tabs;
  uint32_t* T = (uint32_t*)(ws + ly.o_T);
  uint32_t* ctab = (uint32_t*)(ws + ly.o_tab);
  uint64_t* H = ly.nHX ? (uint64_t*)(ws + ly.o_H) : nullptr;
  uint64_t* X = ly.need_X ? (uint64_t*)(ws + ly.o_X) : nullptr;
  unsigned long long* def = ly.n_def ? (unsigned long long*)(ws + ly.o_def) : nullptr;

  // ------------------------------------------------ tables
  if (ly.tab_total) {
    const uint64_t work = (uint64_t)D.P + ly.tab_total;
    const uint64_t blocks = std::min<uint64_t>((work + kThreads - 1) / kThreads, (uint64_t)sm_count() * 16);
    k_prep<<<(unsigned)blocks, kThreads, 0, st>>>(D, tabs, ly.tab_total, T, ctab);
  } else {
    k_resolve<<<(D.P + kThreads - 1) / kThreads, kThreads, 0, st>>>(D, T);
  }
  count_launch();
  // ------------------------------------------------ reductions (on rs)
  auto reductions = [&](cudaStream_t rs) -> int {
    if (ly.need_red) {
      if (w.total) MP_CUDA_TRY(cudaMemsetAsync(w.total, 0, 8, rs));
      const bool lc_elem = D.lc && w.elem_mode;
      LcHalo lh;
      std::memset(&lh, 0, sizeof(lh));
      if (lc_elem) lh = make_lc_halo(D, w);
      if (def) {
        MP_CUDA_TRY(cudaMemsetAsync(def, 0, ly.n_def * 8, rs));
        uint64_t work = 0;
        for (int t = 0; t < D.k; ++t) {
          const uint64_t lo_n = std::min<uint64_t>(lc_elem ? w.width[t] : 1, D.L[t]);
          const uint64_t hi_n = std::min<uint64_t>(lc_elem ? w.width[t] : 1, D.L[t] - lo_n);
          work += (lc_elem ? lo_n + hi_n : 2) * (D.npoints / D.L[t]);
        }
        const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((work + kThreads - 1) / kThreads,
                                                                           (uint64_t)sm_count() * 8));
        if (lc_elem) {
          k_lc_wslabs<<<(unsigned)blocks, kThreads, 0, rs>>>(D, lh, w.face[0], w.face[1], w.face[2], w.face[3],
                                                             w.width[0], w.width[1], w.width[2], w.width[3], def);
          count_launch();
        } else if (D.P <= kLcScanMax) {
          LcRuns R;
          std::memset(&R, 0, sizeof(R));
          for (int t = 0; t + 1 < D.k; ++t) {
            const bool crosses = D.lc_stride_mod[t] != 0 && w.face[t] != 0;
            R.begin[t + 1] = R.begin[t] + (crosses ? 2 * (D.npoints / (D.L[t] * D.lc_stride[t])) : 0);
          }
          unsigned long long* defall = def + D.P;   // one extra word after the deficits
          MP_CUDA_TRY(cudaMemsetAsync(defall, 0, 8, rs));
          const uint64_t runs = R.begin[D.k - 1];
          if (runs) {
            const uint64_t rb = std::max<uint64_t>(1, std::min<uint64_t>((runs + kThreads - 1) / kThreads,
                                                                         (uint64_t)sm_count() * 8));
            k_lc_runs<<<(unsigned)rb, kThreads, 0, rs>>>(D, R, w.face[0], w.face[1], w.face[2], w.face[3], def, defall);
            count_launch();
          }
          k_lc_scan<<<1, 1024, 0, rs>>>(D, w.face[D.k - 1], def, defall);
          count_launch();
        } else {
          k_lc_slabs<<<(unsigned)blocks, kThreads, 0, rs>>>(D, w.face[0], w.face[1], w.face[2], w.face[3], def);
          count_launch();
        }
      }
      k_reduce<<<(D.P + kThreads - 1) / kThreads, kThreads, 0, rs>>>(
          D, T, H, X, (const uint64_t*)def, w.face[0], w.face[1], w.face[2], w.face[3], w.hist, w.recv,
          (unsigned long long*)w.total, lh, lc_elem ? 1 : 0);
      count_launch();
    }
    return MP_OK;
  };
  // with ids wanted too, the counts and reductions (which read only the chain
  // table) run on a second stream beside the tables and the id writer
  const ForkStreams* fk = side_stream && w.ids && ly.need_red ? fork_streams() : nullptr;
  cudaStream_t rs = st;
  if (fk) {
    MP_CUDA_TRY(cudaEventRecord(fk->fork, st));
    MP_CUDA_TRY(cudaStreamWaitEvent(fk->side, fk->fork, 0));
    rs = fk->side;
  }
  if (H) {
    k_counts<<<(D.Jtotal + kThreads - 1) / kThreads, kThreads, 0, rs>>>(D, H, X, w.elem_mode, w.width[0],
                                                                         w.width[1], w.width[2], w.width[3]);
    count_launch();
  }
  // the caller's stream waits for the second stream on every way out of
  // this function, so that a capture on it never ends with a fork open
  struct Join {
    const ForkStreams* fk;
    cudaStream_t st;
    bool armed;
    ~Join() {
      if (armed) cudaStreamWaitEvent(st, fk->join, 0);
    }
  } join{fk, st, false};
  if (fk) {
    const int rc = reductions(rs);
    join.armed = cudaEventRecord(fk->join, rs) == cudaSuccess;
    if (rc) return rc;
    if (!join.armed) return MP_ECUDA;
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
    // Several waves of CTAs, each warp writing one contiguous range of about
    // kIdsWarpGroups 4-point groups: the warps writing at any moment then
    // cover one part of the output rather than all of it, which DRAM writes
    // faster (2 GiB of ids: 6.4 TB/s from one resident wave of long ranges,
    // 7.2 TB/s from 16-32 waves; shorter ranges than ~300 groups lose again)
    auto grid_for = [&](const void* kern, size_t sm, uint64_t& gpw) {
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
      if (per_sm < 1) per_sm = 1;
      const uint64_t wave = (uint64_t)sm_count() * per_sm;
      uint64_t blocks = (groups + (kThreads / 32) * kIdsWarpGroups - 1) / ((kThreads / 32) * kIdsWarpGroups);
      blocks = std::min<uint64_t>(std::max<uint64_t>(blocks, wave), wave * kIdsMaxWaves);
      const uint64_t warps_needed = (groups + 31) / 32;
      blocks = std::max<uint64_t>(1, std::min<uint64_t>(blocks, (warps_needed + 7) / 8));
      const uint64_t warps = blocks * (kThreads / 32);
      gpw = ((groups + warps - 1) / warps + 31) / 32 * 32;
      return (unsigned)blocks;
    };
    auto go = [&](const void* kern, size_t sm, auto launch) {
      if (sm > 40 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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
      if (mode == M_GENERAL && !wide) {
        // unaligned or untabled rows: fuse trailing dimensions into rows of
        // up to 4096 points with a table in shared memory, or compute the
        // last dimension's contribution in place
        int m = last;
        uint64_t Lf = D.L[last];
        while (m > 0 && Lf < 2048 && Lf * D.L[m - 1] <= 4096) Lf *= D.L[--m];
        int src;
        if (Lf <= 4096) src = Lf % 4 == 0 ? R_TAB4 : R_TAB;
        else if (D.ncomp[last] == 2) src = R_HIER;
        else src = D.comp[last][0].kind == C_BLOCK ? R_BLOCK : (D.comp[last][0].kind == C_CYCLIC ? R_CYCLIC : R_BCYC);
        const Div32 divLf = make_div32((uint32_t)Lf);
        const size_t sm = tbytes + (src <= R_TAB4 ? (size_t)((Lf + 3) & ~3ull) * 4 : 0);
#define MP_ROWS(SRC, TS) go((const void*)k_ids_rows<SRC, TS>, sm, [&](unsigned b, uint64_t gpw) { \
        k_ids_rows<SRC, TS><<<b, kThreads, sm, st>>>(D, tabs, T, ctab, m, (uint32_t)Lf, divLf, vec_ok, gpw, w.ids); })
#define MP_ROWS_T(SRC) do { if (tsmem) MP_ROWS(SRC, true); else MP_ROWS(SRC, false); } while (0)
        switch (src) {
          case R_TAB4: MP_ROWS_T(R_TAB4); break;
          case R_TAB: MP_ROWS_T(R_TAB); break;
          case R_BLOCK: MP_ROWS_T(R_BLOCK); break;
          case R_CYCLIC: MP_ROWS_T(R_CYCLIC); break;
          case R_BCYC: MP_ROWS_T(R_BCYC); break;
          default: MP_ROWS_T(R_HIER); break;
        }
#undef MP_ROWS_T
#undef MP_ROWS
        timer_end(st);
        MP_CUDA_TRY(cudaGetLastError());
        goto ids_done;
      }
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
ids_done:
  if (fk) {
    join.armed = false;
    MP_CUDA_TRY(cudaStreamWaitEvent(st, fk->join, 0));
  } else {
    int rc = reductions(st);
    if (rc) return rc;
  }
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

// Runs one launch with the scratch in the per-device workspace.
int run_launch(const Plan& pl, const Want& w, cudaStream_t st) {
  const Layout ly = make_layout(pl.desc, w);
  char* ws = (char*)workspace(ly.bytes, 0);
  if (!ws) return MP_ENOMEM;
  return run_launch_ws(pl, w, ly, ws, st, true);
}

// Resolves host/device outputs: device buffers are used directly, host
// buffers get a device staging area (workspace slot 1) and a copy back.
struct Staged {
  void* user;
  void* dev;
  size_t bytes;
};

int stage(void* user, size_t bytes, size_t& cursor, std::vector<Staged>& list, char* base,
          void** dev_out, bool direct_ok) {
  if (!user) {
    *dev_out = nullptr;
    return MP_OK;
  }
  if (is_device_pointer(user)) {
    *dev_out = user;
    return MP_OK;
  }
  void* alias = direct_ok ? pinned_alias(user) : nullptr;
  if (alias) {   // page-locked id array: the id writer stores into it directly
    *dev_out = alias;
    list.push_back(Staged{user, nullptr, 0});
    return MP_OK;
  }
  *dev_out = base ? base + cursor : nullptr;
  list.push_back(Staged{user, *dev_out, bytes});
  cursor = align256(cursor + bytes);
  return MP_OK;
}

int run_with_staging(const Plan& pl, int32_t* ids, uint64_t* hist, uint64_t* recv, uint64_t* total,
                     const uint64_t* face, cudaStream_t st, int elem_mode = 0, const int32_t* width = nullptr) {
  const MapDesc& D = pl.desc;
  size_t need = 0;
  auto host_bytes = [&](void* p, size_t b, bool direct_ok) {
    if (p && !is_device_pointer(p) && !(direct_ok && pinned_alias(p))) need = align256(need + b);
  };
  host_bytes(ids, D.npoints * 4, true);
  host_bytes(hist, (size_t)D.P * 8, false);
  host_bytes(recv, (size_t)D.P * 8, false);
  host_bytes(total, 8, false);
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
  stage(ids, D.npoints * 4, cur, list, base, &p, true); w.ids = (int32_t*)p;
  stage(hist, (size_t)D.P * 8, cur, list, base, &p, false); w.hist = (uint64_t*)p;
  stage(recv, (size_t)D.P * 8, cur, list, base, &p, false); w.recv = (uint64_t*)p;
  stage(total, 8, cur, list, base, &p, false); w.total = (uint64_t*)p;
  for (int t = 0; t < 4; ++t) w.face[t] = face && t < D.k ? face[t] : 0;
  w.elem_mode = elem_mode;
  for (int t = 0; t < 4; ++t) w.width[t] = width && t < D.k ? (uint32_t)width[t] : 0;
  int rc = run_launch(pl, w, st);
  if (rc) return rc;
  for (auto& s : list)
    if (s.bytes) MP_CUDA_TRY(cudaMemcpyAsync(s.user, s.dev, s.bytes, cudaMemcpyDeviceToHost, st));
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

extern "C" int mp_halo_volume(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                              int n_xf, const mp_dist* dist, const mp_halo* halo, uint64_t* total,
                              uint64_t* recv, void* stream) {
  mp::Plan pl;
  int rc = mp::build_plan(space, machine, chain, n_xf, dist, pl);
  if (rc) return rc;
  if (!halo || !total) return MP_EINVAL;
  if (halo->mode != MP_HALO_FACES && halo->mode != MP_HALO_ELEMENTS) return MP_EINVAL;
  if (halo->mode == MP_HALO_ELEMENTS)
    for (int t = 0; t < space->rank; ++t)
      if (halo->width[t] < 0 || halo->width[t] > MP_MAX_HALO_WIDTH) return MP_EINVAL;
  return mp::run_with_staging(pl, nullptr, nullptr, recv, total, halo->bytes, (cudaStream_t)stream,
                              halo->mode == MP_HALO_ELEMENTS ? 1 : 0, halo->width);
}

extern "C" int mp_map_launch(const mp_space* space, const mp_machine* machine, const mp_xform* chain, int n_xf,
                             const mp_dist* dist, const mp_halo* halo, int32_t* ids, uint64_t* hist,
                             uint64_t* total, uint64_t* recv, void* stream) {
  mp::Plan pl;
  int rc = mp::build_plan(space, machine, chain, n_xf, dist, pl);
  if (rc) return rc;
  if (!halo && (total || recv)) return MP_EINVAL;
  if (halo) {
    if (halo->mode != MP_HALO_FACES && halo->mode != MP_HALO_ELEMENTS) return MP_EINVAL;
    if (halo->mode == MP_HALO_ELEMENTS)
      for (int t = 0; t < space->rank; ++t)
        if (halo->width[t] < 0 || halo->width[t] > MP_MAX_HALO_WIDTH) return MP_EINVAL;
  }
  if (!ids && !hist && !total && !recv) return MP_OK;
  return mp::run_with_staging(pl, ids, hist, recv, total, halo ? halo->bytes : nullptr, (cudaStream_t)stream,
                              halo && halo->mode == MP_HALO_ELEMENTS ? 1 : 0, halo ? halo->width : nullptr);
}

// ------------------------------------------------------------ two-level search

namespace mp {
namespace {

// Chain realising a two-level candidate on Machine(n, g): the node dimension
// split by a, the processor dimension by b; for the block variant each
// (b_t, a_t) pair is brought together by swaps and merged with the GPU
// digit fastest, so that a block distribution over the product grid gives
// node floor(w_t / b_t) and GPU w_t mod b_t.
int hier_chain(int k, const int64_t* a, const int64_t* b, int variant, std::vector<mp_xform>& ch, mp_dist& dist) {
  ch.clear();
  auto op = [&](int o, int i, int j, int64_t d) {
    mp_xform x;
    std::memset(&x, 0, sizeof(x));
    x.op = o;
    x.i = i;
    x.j = j;
    x.d = d;
    ch.push_back(x);
  };
  for (int i = 0; i + 1 < k; ++i) op(MP_SPLIT, i, 0, a[i]);
  for (int j = 0; j + 1 < k; ++j) op(MP_SPLIT, k + j, 0, b[j]);
  dist.b = 1;
  if (variant == MP_HIER_CYCLIC) {
    dist.kind = MP_HIER;
    return MP_OK;
  }
  dist.kind = MP_BLOCK;
  // labels: node factor t = t, GPU factor t = k + t; wanted order
  // (gpu 0, node 0, gpu 1, node 1, ...)
  int lab[8];
  for (int t = 0; t < 2 * k; ++t) lab[t] = t;
  for (int pos = 0; pos < 2 * k; ++pos) {
    const int want = (pos & 1) ? pos / 2 : k + pos / 2;
    int j = pos;
    while (lab[j] != want) ++j;
    if (j != pos) {
      op(MP_SWAP, pos, j, 0);
      std::swap(lab[pos], lab[j]);
    }
  }
  for (int t = 0; t < k; ++t) op(MP_MERGE, t, t + 1, 0);
  return MP_OK;
}

}  // namespace
}  // namespace mp

extern "C" int mp_hier_chain(int32_t rank, const int64_t* a, const int64_t* b, int32_t variant, mp_xform* chain,
                             int32_t* n_xf, mp_dist* dist) {
  if (rank < 1 || rank > 4 || !a || !b || !chain || !n_xf || !dist) return MP_EINVAL;
  if (variant != MP_HIER_BLOCK && variant != MP_HIER_CYCLIC) return MP_EINVAL;
  std::vector<mp_xform> ch;
  int rc = mp::hier_chain(rank, a, b, variant, ch, *dist);
  if (rc) return rc;
  for (size_t o = 0; o < ch.size(); ++o) chain[o] = ch[o];
  *n_xf = (int32_t)ch.size();
  return MP_OK;
}

namespace mp {
namespace {

// Element-halo totals of many launch plans at once (the two-level search):
// the per-dimension counts of every plan, then one thread per flat final
// index F of every plan.  A plan's total needs neither its chain table nor
// its ids, only the counts (the owner changes exactly where a dimension's
// final coordinate does).
struct PlanHalo {
  MapCore c;
  uint64_t face[4];
  uint32_t width[4];
  uint32_t cnt_off, p_off;
};

// index q with pref[q] <= e < pref[q + 1]
__device__ __forceinline__ uint32_t find_plan(const uint32_t* __restrict__ pref, uint32_t n, uint32_t e) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pref[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads) k_plans_counts(const PlanHalo* __restrict__ plans,
                                                           const uint32_t* __restrict__ cnt_pref, uint32_t n,
                                                           uint32_t total, uint64_t* __restrict__ H,
                                                           uint64_t* __restrict__ X) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const PlanHalo& Q = plans[find_plan(cnt_pref, n, e)];
    const uint32_t r = e - Q.cnt_off;
    int t = 0;
    while (t < Q.c.k - 1 && r >= Q.c.Joff[t + 1]) ++t;
    uint64_t h, xc;
    dim_counts(Q.c, t, r - Q.c.Joff[t], h, xc);
    H[e] = h;
    X[e] = dim_elems(Q.c, t, r - Q.c.Joff[t], Q.width[t]);
  }
}

__global__ void __launch_bounds__(kThreads) k_plans_reduce(const PlanHalo* __restrict__ plans,
                                                           const uint32_t* __restrict__ p_pref, uint32_t n,
                                                           uint32_t total, const uint64_t* __restrict__ H,
                                                           const uint64_t* __restrict__ X,
                                                           unsigned long long* __restrict__ totals) {
  for (uint32_t e0 = blockIdx.x * blockDim.x; e0 < total; e0 += gridDim.x * blockDim.x) {
    const uint32_t e = e0 + threadIdx.x;
    uint32_t q = 0xFFFFFFFFu;
    unsigned long long r = 0;
    if (e < total) {
      q = find_plan(p_pref, n, e);
      const PlanHalo& Q = plans[q];
      uint64_t h_F, r_F;
      reduce_F(Q.c, H + Q.cnt_off, X + Q.cnt_off, nullptr, Q.face, true, e - Q.p_off, h_F, r_F);
      r = r_F;
    }
    // one atomic per group of lanes of the same plan
    const unsigned same = __match_any_sync(0xFFFFFFFFu, q);
    const int lane = threadIdx.x & 31;
    if (q != 0xFFFFFFFFu) {
      // the lowest lane of each group adds the group's sum
      unsigned long long s = 0;
      for (unsigned m = same; m; m &= m - 1) s += __shfl_sync(same, r, __ffs(m) - 1);
      if (lane == __ffs(same) - 1 && s) atomicAdd(totals + q, s);
    }
  }
}

}  // namespace
}  // namespace mp

extern "C" int mp_hier_search(const mp_hier_query* query, mp_hier_result* out, void* stream) {
  using namespace mp;
  if (!query || !out) return MP_EINVAL;
  const mp_hier_query& q = *query;
  const int k = q.space.rank;
  if (k < 1 || k > MP_MAX_TASK_RANK) return MP_EINVAL;
  if (q.variant != MP_HIER_BLOCK && q.variant != MP_HIER_CYCLIC) return MP_EINVAL;
  if (q.machine.nodes < 1 || q.machine.procs_per_node < 1) return MP_EINVAL;
  for (int t = 0; t < k; ++t)
    if (q.width[t] < 0 || q.width[t] > MP_MAX_HALO_WIDTH) return MP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const auto fa = ordered_factorisations(q.machine.nodes, k);
  const auto fb = ordered_factorisations(q.machine.procs_per_node, k);
  const size_t NA = fa.size(), NB = fb.size(), ncand = NA * NB;
  if (ncand > 65536) return MP_ENOTSUP;
  const mp_machine node_machine{q.machine.nodes, 1};
  // candidate plans: the node-level launch of node grid a (Machine(n, 1),
  // the node splits, the trailing size-1 dimension merged), and the
  // processor-level launch of (a, b)
  auto plan_node = [&](size_t i, Plan& pl) {
    std::vector<mp_xform> ch;
    mp_dist d;
    const int64_t ones[4] = {1, 1, 1, 1};
    hier_chain(k, fa[i].data(), ones, MP_HIER_BLOCK, ch, d);
    std::vector<mp_xform> nch(ch.begin(), ch.begin() + (k - 1));
    mp_xform m;
    std::memset(&m, 0, sizeof(m));
    m.op = MP_MERGE;
    m.i = k - 1;
    m.j = k;
    nch.push_back(m);
    const mp_dist blk{MP_BLOCK, 1};
    return build_plan(&q.space, &node_machine, nch.data(), (int)nch.size(), &blk, pl);
  };
  auto plan_proc = [&](size_t c, Plan& pl) {
    std::vector<mp_xform> ch;
    mp_dist d;
    hier_chain(k, fa[c / NB].data(), fb[c % NB].data(), q.variant, ch, d);
    return build_plan(&q.space, &q.machine, ch.data(), (int)ch.size(), &d, pl);
  };
  Plan pl;
  uint64_t* totals = (uint64_t*)workspace((NA + ncand) * 8, 5);
  if (!totals) return MP_ENOMEM;
  // every plan's total in two launches when no plan is linearised cyclic
  // (every plan built, so validated, before the launches)
  {
    std::vector<PlanHalo> ph(NA + ncand);
    std::vector<uint32_t> cnt_pref(NA + ncand + 1, 0), p_pref(NA + ncand + 1, 0);
    bool all_plain = true;
    for (size_t i = 0; i < NA + ncand && all_plain; ++i) {
      int rc = i < NA ? plan_node(i, pl) : plan_proc(i - NA, pl);
      if (rc) return rc;
      all_plain = !pl.desc.lc && (uint64_t)cnt_pref[i] + pl.desc.Jtotal < (1ull << 31) &&
                  (uint64_t)p_pref[i] + pl.desc.P < (1ull << 31);
      PlanHalo& h = ph[i];
      std::memset(&h, 0, sizeof(h));
      h.c = static_cast<const MapCore&>(pl.desc);
      for (int t = 0; t < 4; ++t) {
        h.face[t] = t < k ? q.bytes[t] : 0;
        h.width[t] = t < k ? (uint32_t)q.width[t] : 0;
      }
      h.cnt_off = cnt_pref[i];
      h.p_off = p_pref[i];
      cnt_pref[i + 1] = cnt_pref[i] + pl.desc.Jtotal;
      p_pref[i + 1] = p_pref[i] + pl.desc.P;
    }
    if (all_plain) {
      const size_t NP = NA + ncand, J = cnt_pref[NP], PT = p_pref[NP];
      auto align_up = [](size_t v) { return (v + 255) & ~size_t(255); };
      const size_t o_ph = 0, o_cp = align_up(NP * sizeof(PlanHalo)), o_pp = o_cp + align_up((NP + 1) * 4),
                   o_H = o_pp + align_up((NP + 1) * 4), o_X = o_H + align_up(J * 8), end = o_X + align_up(J * 8);
      char* ws = (char*)workspace(end, 7);
      if (!ws) return MP_ENOMEM;
      PlanHalo* d_ph = (PlanHalo*)(ws + o_ph);
      uint32_t* d_cp = (uint32_t*)(ws + o_cp);
      uint32_t* d_pp = (uint32_t*)(ws + o_pp);
      uint64_t* d_H = (uint64_t*)(ws + o_H);
      uint64_t* d_X = (uint64_t*)(ws + o_X);
      MP_CUDA_TRY(cudaMemcpyAsync(d_ph, ph.data(), NP * sizeof(PlanHalo), cudaMemcpyHostToDevice, st));
      MP_CUDA_TRY(cudaMemcpyAsync(d_cp, cnt_pref.data(), (NP + 1) * 4, cudaMemcpyHostToDevice, st));
      MP_CUDA_TRY(cudaMemcpyAsync(d_pp, p_pref.data(), (NP + 1) * 4, cudaMemcpyHostToDevice, st));
      MP_CUDA_TRY(cudaMemsetAsync(totals, 0, NP * 8, st));
      const unsigned big = (unsigned)sm_count() * 8;
      auto blocks_for = [&](uint64_t work) {
        return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + kThreads - 1) / kThreads, big));
      };
      if (J) {
        k_plans_counts<<<blocks_for(J), kThreads, 0, st>>>(d_ph, d_cp, (uint32_t)NP, (uint32_t)J, d_H, d_X);
        count_launch();
      }
      k_plans_reduce<<<blocks_for(PT), kThreads, 0, st>>>(d_ph, d_pp, (uint32_t)NP, (uint32_t)PT, d_H, d_X,
                                                          (unsigned long long*)totals);
      count_launch();
      MP_CUDA_TRY(cudaGetLastError());
    }
    if (all_plain) goto totals_ready;
  }
  {
  // every plan is validated before anything is launched
  for (size_t i = 0; i < NA; ++i) {
    int rc = plan_node(i, pl);
    if (rc) return rc;
  }
  for (size_t c = 0; c < ncand; ++c) {
    int rc = plan_proc(c, pl);
    if (rc) return rc;
  }
  auto run = [&](const Plan& p, uint64_t* total) {
    Want w;
    std::memset(&w, 0, sizeof(w));
    w.total = total;
    w.elem_mode = 1;
    for (int t = 0; t < 4; ++t) {
      w.face[t] = t < k ? q.bytes[t] : 0;
      w.width[t] = t < k ? (uint32_t)q.width[t] : 0;
    }
    return run_launch(p, w, st);
  };
  for (size_t i = 0; i < NA; ++i) {
    int rc = plan_node(i, pl);
    if (!rc) rc = run(pl, totals + i);
    if (rc) return rc;
  }
  for (size_t c = 0; c < ncand; ++c) {
    int rc = plan_proc(c, pl);
    if (!rc) rc = run(pl, totals + NA + c);
    if (rc) return rc;
  }
  }
totals_ready:
  std::vector<uint64_t> h(NA + ncand);
  MP_CUDA_TRY(cudaMemcpyAsync(h.data(), totals, h.size() * 8, cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  size_t best = 0;
  for (size_t c = 1; c < ncand; ++c) {
    const uint64_t p = h[c / NB], s = h[NA + c], bp = h[best / NB], bs = h[NA + best];
    if (p < bp || (p == bp && s < bs)) best = c;
  }
  std::memset(out, 0, sizeof(*out));
  out->index = (int64_t)best;
  for (int t = 0; t < k; ++t) {
    out->a[t] = fa[best / NB][t];
    out->b[t] = fb[best % NB][t];
  }
  out->primary_bytes = h[best / NB];
  out->secondary_bytes = h[NA + best];
  out->n_candidates = (int64_t)ncand;
  return MP_OK;
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
  // everything on the caller's stream: no second stream or events are created
  return mp::run_launch_ws(pl, w, ly, ws, (cudaStream_t)stream, false);
}
