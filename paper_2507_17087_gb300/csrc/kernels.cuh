// Device building blocks shared by the single-launch kernels (map.cu) and
// the batched persistent kernels (batch.cu).
#pragma once

#include "engine.h"

namespace mp {

constexpr int kThreads = 256;
constexpr uint64_t kTableMax = uint64_t(1) << 22;   // per-dimension c_t tables kept in HBM/L2
constexpr uint32_t kSmemTMax = 16384;               // T staged in shared memory up to this P
constexpr uint32_t kSmemLastMax = 8192;             // c_last staged in shared memory

// Where each dimension's c_t table lives inside the launch's table area.
struct Tabs {
  uint64_t off[4];     // offset of dimension t's table (a multiple of 4 entries)
  int32_t has[4];      // 1 if the table exists
};

// ------------------------------------------------------------ distribution

// Final coordinate of one component for task coordinate x:
//   BLOCK  floor(x s / L)   CYCLIC x mod s   BCYC floor(x / b) mod s
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
    default: {
      const uint64_t blk = x <= 0xFFFFFFFFull ? div32((uint32_t)x, c.divb) : div64(x, c.divb64);
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

// c_t(x): the flat-index contribution of the final coordinates driven by x.
__device__ __forceinline__ uint32_t contrib(const MapCore& D, int t, uint64_t x) {
  uint32_t v = comp_coord(D.comp[t][0], x) * D.comp[t][0].sigma;
  if (D.ncomp[t] > 1) v += comp_coord(D.comp[t][1], x) * D.comp[t][1].sigma;
  return v;
}

// ------------------------------------------------------------ chain resolve

// Processor id of flat final index F: decode F (dimension 0 fastest), then
// apply the Fig. 4 inverse formula of every primitive from last to first.
__device__ __forceinline__ uint32_t resolve_F(const MapCore& D, const Prim* __restrict__ prim, int nprim,
                                              uint32_t F) {
  uint32_t a[kMaxRank + 1];
  uint32_t rest = F;
  for (int u = 0; u < D.rank; ++u) {
    uint32_t q, r;
    divmod32(rest, D.divs[u], q, r);
    a[u] = r;
    rest = q;
  }
  int r = D.rank;
  for (int o = nprim - 1; o >= 0; --o) {
    const Prim p = prim[o];
    if (p.op == P_SPLIT) {
      // split: b_i = a_i + a_{i+1} d, b_t = a_{t+1} for t > i
      a[p.p] = a[p.p] + a[p.p + 1] * p.d;
      for (int t = p.p + 1; t < r - 1; ++t) a[t] = a[t + 1];
      r -= 1;
    } else if (p.op == P_MERGE) {
      // merge: b_p = a_p mod s_p, b_q = floor(a_p / s_p), b_t = a_{t-1} for t > q
      uint32_t q, rem;
      divmod32(a[p.p], p.div, q, rem);
      for (int t = r; t > p.q; --t) a[t] = a[t - 1];
      a[p.q] = q;
      a[p.p] = rem;
      r += 1;
    } else {
      const uint32_t tmp = a[p.p];
      a[p.p] = a[p.q];
      a[p.q] = tmp;
    }
  }
  return a[0] * D.g + a[1];
}

// ------------------------------------------------------------ counts

__device__ __forceinline__ uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// x in [0, n) with x = beta (mod m)
__device__ __forceinline__ uint64_t count_residue(uint64_t n, uint64_t beta, uint64_t m) {
  return beta < n ? (n - 1 - beta) / m + 1 : 0;
}

// Per-dimension counts of sub-index j of task dimension t, in closed form:
//   h = number of coordinates x in [0, L) whose final coordinates give j,
//   x = number of (x, x +- 1) neighbour pairs inside [0, L) leaving such an x
//       whose neighbour gives another sub-index.
__device__ __forceinline__ void dim_counts(const MapCore& D, int t, uint32_t j, uint64_t& h, uint64_t& xc) {
  const Comp& c0 = D.comp[t][0];
  const uint64_t L = D.L[t];
  const uint32_t alpha = j % c0.s;
  if (D.ncomp[t] == 1) {
    if (c0.kind == C_BLOCK) {
      // block alpha = [lo, hi); it changes owner at its ends only
      const uint64_t lo = ceil_div((uint64_t)alpha * L, c0.s);
      const uint64_t hi = ceil_div((uint64_t)(alpha + 1) * L, c0.s);
      h = hi - lo;
      xc = h ? (uint64_t)(lo > 0) + (uint64_t)(hi < L) : 0;
    } else if (c0.kind == C_CYCLIC) {
      // every neighbour has another residue when s >= 2
      h = count_residue(L, alpha, c0.s);
      xc = (c0.s >= 2 && h) ? 2 * h - (alpha == 0) - ((L - 1) % c0.s == alpha) : 0;
    } else {
      // blocks q = floor(x / b), q = alpha (mod s); owners change at block ends
      const uint64_t b = c0.b;
      const uint64_t Q = ceil_div(L, b);
      const uint64_t nq = count_residue(Q, alpha, c0.s);
      const bool last_here = nq && ((Q - 1) % c0.s == alpha);
      h = nq * b - (last_here ? Q * b - L : 0);
      xc = (c0.s >= 2 && nq) ? 2 * nq - (alpha == 0) - (last_here ? 1 : 0) : 0;
    }
  } else {
    // hierarchical: block alpha (s_u blocks) and residue beta mod s_l
    const Comp& c1 = D.comp[t][1];
    const uint32_t beta = j / c0.s;
    const uint64_t lo = ceil_div((uint64_t)alpha * L, c0.s);
    const uint64_t hi = ceil_div((uint64_t)(alpha + 1) * L, c0.s);
    h = count_residue(hi, beta, c1.s) - count_residue(lo, beta, c1.s);
    if (!h) {
      xc = 0;
    } else if (c1.s >= 2) {
      const bool has_first = lo == 0 && beta == 0;
      const bool has_last = hi == L && (L - 1) % c1.s == beta;
      xc = 2 * h - has_first - has_last;
    } else {
      xc = (uint64_t)(lo > 0) + (uint64_t)(hi < L);
    }
  }
}

// Element-count halo along one dimension (each element counted once per
// receiving owner and dimension within the halo width): the sub-index
// j occupies runs of positions (first run starts at a, last run ends at e,
// nq runs of `size` positions in all, consecutive runs `gap` apart); the
// positions outside them within distance w of one are
// |dilate(runs, w) \ runs|, clipped to [0, L).  Runs further apart than 2w
// dilate separately; otherwise the dilation is one interval.
__device__ __forceinline__ uint64_t run_dilation(uint64_t a, uint64_t e, uint64_t nq, uint64_t size,
                                                 uint64_t gap, uint64_t L, uint64_t w) {
  if (nq == 0 || w == 0) return 0;
  if (nq == 1 || 2 * w >= gap) {
    const uint64_t lo = a > w ? a - w : 0;
    const uint64_t hi = L - e > w ? e + w : L;
    return hi - lo - size;
  }
  const uint64_t cut_lo = w - (a < w ? a : w), cut_hi = w - (L - e < w ? L - e : w);
  return 2 * w * nq - cut_lo - cut_hi;
}

// Positions y of task dimension t outside sub-index j's positions and within
// distance w of one of them: the elements a processor with sub-index j along
// t receives per point of the other dimensions.
__device__ __forceinline__ uint64_t dim_elems(const MapCore& D, int t, uint32_t j, uint64_t w) {
  const Comp& c0 = D.comp[t][0];
  const uint64_t L = D.L[t];
  const uint32_t alpha = j % c0.s;
  if (D.ncomp[t] == 1) {
    if (c0.kind == C_BLOCK) {
      const uint64_t lo = ceil_div((uint64_t)alpha * L, c0.s);
      const uint64_t hi = ceil_div((uint64_t)(alpha + 1) * L, c0.s);
      return run_dilation(lo, hi, hi > lo ? 1 : 0, hi - lo, 0, L, w);
    }
    if (c0.kind == C_CYCLIC) {
      const uint64_t nq = count_residue(L, alpha, c0.s);
      if (!nq) return 0;
      return run_dilation(alpha, alpha + (nq - 1) * c0.s + 1, nq, nq, c0.s - 1, L, w);
    }
    const uint64_t b = c0.b;
    const uint64_t Q = ceil_div(L, b);
    const uint64_t nq = count_residue(Q, alpha, c0.s);
    if (!nq) return 0;
    const uint64_t qlast = alpha + (nq - 1) * c0.s;
    const uint64_t e = qlast * b + b < L ? qlast * b + b : L;
    const uint64_t size = nq * b - (qlast * b + b - e);
    return run_dilation((uint64_t)alpha * b, e, nq, size, (uint64_t)(c0.s - 1) * b, L, w);
  }
  // hierarchical: upper block alpha, lower residue beta (mod s_l) inside it
  const Comp& c1 = D.comp[t][1];
  const uint32_t beta = j / c0.s;
  const uint64_t sl = c1.s;
  const uint64_t lo = ceil_div((uint64_t)alpha * L, c0.s);
  const uint64_t hi = ceil_div((uint64_t)(alpha + 1) * L, c0.s);
  const uint64_t size = count_residue(hi, beta, sl) - count_residue(lo, beta, sl);
  if (!size) return 0;
  const uint64_t a = lo + (beta + sl - lo % sl) % sl;
  return run_dilation(a, a + (size - 1) * sl + 1, size, size, sl - 1, L, w);
}

// Points lin in [0, N) with lin = c (mod P).
__device__ __forceinline__ uint64_t lc_count(const MapCore& D, uint32_t c) {
  uint64_t q, rem;
  divmod64(D.npoints, D.divP64, q, rem);
  return q + (c < rem ? 1 : 0);
}

// hist and received bytes of flat final index F from the per-dimension
// counts (or, for linear-cyclic, from the closed form and the slab deficit).
// lh != nullptr selects the element-count halo for linear-cyclic launches.
__device__ __forceinline__ void reduce_F(const MapCore& D, const uint64_t* __restrict__ H,
                                         const uint64_t* __restrict__ X, const uint64_t* __restrict__ deficit,
                                         const uint64_t face[4], bool want_recv, uint32_t F, uint64_t& h_F,
                                         uint64_t& r_F, const LcHalo* lh = nullptr) {
  r_F = 0;
  if (!D.lc) {
    uint32_t j[4] = {0, 0, 0, 0};
    uint32_t rest = F;
    for (int u = 0; u < D.rank; ++u) {
      uint32_t q, r;
      divmod32(rest, D.divs[u], q, r);
      rest = q;
      const int t = D.owner_dim[u];
      j[t] += D.owner_slot[u] ? r * D.comp[t][0].s : r;
    }
    uint64_t h[4];
    h_F = 1;
    for (int t = 0; t < D.k; ++t) {
      h[t] = H[D.Joff[t] + j[t]];
      h_F *= h[t];
    }
    if (want_recv)
      for (int t = 0; t < D.k; ++t) {
        uint64_t v = face[t] * X[D.Joff[t] + j[t]];
        for (int u = 0; u < D.k; ++u)
          if (u != t) v *= h[u];
        r_F += v;
      }
  } else {
    // C-order linear indices cover [0, N): lin = F (mod P) occurs floor(N / P)
    // times, once more when F < N mod P; every neighbour along a dimension
    // whose linear stride is not a multiple of P crosses.
    uint64_t q, rem;
    divmod64(D.npoints, D.divP64, q, rem);
    h_F = q + (F < rem ? 1 : 0);
    if (want_recv && lh) {
      // every element within the halo width of one of F's points, once per
      // distinct offset; the boundary slabs' missing neighbours come off
      uint64_t r = 0;
      for (int t = 0; t < D.k; ++t)
        for (uint32_t i = 0; i < lh->n[t]; ++i) {
          const uint32_t off = lh->off[t][i];
          r += face[t] * lc_count(D, F >= off ? F - off : F + D.P - off);
        }
      r_F = r - deficit[F];
    } else if (want_recv) {
      uint64_t G = 0;
      for (int t = 0; t < D.k; ++t)
        if (D.lc_stride_mod[t] != 0) G += 2 * face[t];
      r_F = G * h_F - deficit[F];
    }
  }
}

// ------------------------------------------------------------ ids

template <typename I>
__device__ __forceinline__ void split_lin(const MapCore& D, I lin, I& row, I& x) {
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

// base(row) = sum_{t < k-1} c_t(x_t) of the slow coordinates of a row
template <typename I>
__device__ __noinline__ uint32_t row_base(const MapCore& D, const Tabs& tabs, const uint32_t* __restrict__ ctab,
                                          I row) {
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

enum IdsMode : int { M_FAST_SMEM = 0, M_FAST_GLOBAL = 1, M_GENERAL = 2, M_FUSED = 3 };

// base of a row when the dimensions m..k-1 are fused into one fast
// dimension: sum_{t < m} c_t(x_t) of the row's slow coordinates.
template <typename I>
__device__ __forceinline__ uint32_t row_base_inl(const MapCore& D, const Tabs& tabs,
                                                 const uint32_t* __restrict__ ctab, I row, int m) {
  uint32_t base = 0;
  for (int t = m - 1; t >= 0; --t) {
    I xt = row;
    if (t > 0) {
      uint32_t q32, r32;
      divmod32((uint32_t)row, D.divL32[t], q32, r32);
      row = (I)q32;
      xt = (I)r32;
    }
    base += tabs.has[t] ? __ldg(ctab + tabs.off[t] + xt) : contrib(D, t, (uint64_t)xt);
  }
  return base;
}

template <typename I>
__device__ __noinline__ uint32_t row_base_m(const MapCore& D, const Tabs& tabs, const uint32_t* __restrict__ ctab,
                                            I row, int m) {
  uint32_t base = 0;
  for (int t = m - 1; t >= 0; --t) {
    I xt = row;
    if (t > 0) {
      uint32_t q32, r32;
      divmod32((uint32_t)row, D.divL32[t], q32, r32);
      row = (I)q32;
      xt = (I)r32;
    }
    base += tabs.has[t] ? __ldg(ctab + tabs.off[t] + xt) : contrib(D, t, (uint64_t)xt);
  }
  return base;
}

// Where ids_range_rows finds the contribution of a row offset x:
//   R_TAB / R_TAB4  fused table Cf in shared memory (R_TAB4: Lf % 4 == 0, one
//                   16-byte load per group)
//   R_BLOCK, R_CYCLIC, R_BCYC, R_HIER  computed from the last dimension's
//                   components (rows = the last dimension, no table)
//   R_TAB2          two levels: rows are dimension m followed by the fused
//                   table's Lin points (dimensions m+1..k-1, too few for a
//                   row of their own); x -> C2[x / Lin] + Cf[x % Lin], with
//                   C2 dimension m's table in global memory
//   R_TAB2A         R_TAB2 with Lin % 4 == 0: every group lies inside one
//                   entry of C2 and reads its four Cf entries in one 16-byte load
enum RowSrc : int { R_TAB = 0, R_TAB4 = 1, R_BLOCK = 2, R_CYCLIC = 3, R_BCYC = 4, R_HIER = 5, R_TAB2 = 6, R_TAB2A = 7 };

// R_TAB2's second level (unused by the other row sources)
struct RowAux {
  const uint32_t* C2;
  uint32_t Lin;
  Div32 divLin;
};

template <int SRC>
__device__ __forceinline__ uint32_t row_contrib(const MapCore& D, const uint32_t* __restrict__ Cf, const RowAux& A,
                                                uint32_t x) {
  if (SRC == R_TAB || SRC == R_TAB4) return Cf[x];
  if (SRC == R_TAB2 || SRC == R_TAB2A) {
    uint32_t q, r;
    divmod32(x, A.divLin, q, r);
    return __ldg(A.C2 + q) + Cf[r];
  }
  const Comp& c0 = D.comp[D.k - 1][0];
  uint32_t a;
  if (SRC == R_BLOCK || SRC == R_HIER) {
    a = c0.narrow ? div32(x * c0.s, c0.divL32) : (uint32_t)div64((uint64_t)x * c0.s, c0.divL);
  } else if (SRC == R_CYCLIC) {
    uint32_t q;
    divmod32(x, c0.divs, q, a);
  } else {
    uint32_t q;
    divmod32(div32(x, c0.divb), c0.divs, q, a);
  }
  uint32_t v = a * c0.sigma;
  if (SRC == R_HIER) {
    const Comp& c1 = D.comp[D.k - 1][1];
    uint32_t q, r;
    divmod32(x, c1.divs, q, r);
    v += r * c1.sigma;
  }
  return v;
}

// ids for the 4-point groups [gbeg, gend) of one warp, row by row: the
// dimensions m..k-1 form rows of Lf points (fused into one table, or the last
// dimension alone with its contribution computed in place), the dimensions
// before m give the row base.  Groups inside a row take four contributions;
// a group that crosses a row end walks its points, and the next row's base
// it computes is kept for the wrap.  32-bit indices (launches below 2^31
// points).
template <int SRC>
__device__ __forceinline__ void ids_range_rows(const MapCore& D, const Tabs& tabs, const uint32_t* __restrict__ T,
                                               const uint32_t* __restrict__ Cf, const uint32_t* __restrict__ ctab,
                                               const RowAux& A, int m, uint32_t Lf, Div32 divLf, uint32_t gbeg,
                                               uint32_t gend, int lane, int vec_ok, int32_t* __restrict__ ids) {
  const uint32_t N = (uint32_t)D.npoints;
  uint32_t g = gbeg + (uint32_t)lane;
  if (g >= gend) return;
  uint32_t lin0 = g * 4;
  uint32_t row, x;
  divmod32(lin0, divLf, row, x);
  const uint32_t rows = N / Lf;
  uint32_t base = row_base_m<uint32_t>(D, tabs, ctab, row, m);
  // the next row's base, loaded a wrap ahead so that its latency overlaps
  // the groups in between
  uint32_t nbase = row + 1 < rows ? row_base_inl<uint32_t>(D, tabs, ctab, row + 1, m) : 0;
  // R_BLOCK / R_BCYC: the run [run_lo, run_hi) of the last dimension with
  // one final coordinate (block, or block of b points) that holds x, with
  // contribution rc; a group inside it has one id, looked up once
  // (only where runs can hold a group: blocks of at least 4 points)
  constexpr bool RUNS = SRC == R_BLOCK || SRC == R_BCYC;
  const Comp& cl = D.comp[D.k - 1][0];
  const bool use_runs = RUNS && (SRC == R_BCYC ? cl.b >= 4 : cl.L >= 4 * (uint64_t)cl.s);
  uint32_t rc = 0, run_lo = 1, run_hi = 0;
  for (; g < gend; g += 32, lin0 += 128) {
    const int cnt = N - lin0 < 4 ? (int)(N - lin0) : 4;
    uint32_t v[4] = {0, 0, 0, 0};
    if (use_runs && (x < run_lo || x >= run_hi)) {
      uint64_t lo, hi;
      if (SRC == R_BLOCK) {
        // block a of x: points [ceil(a L / s), ceil((a + 1) L / s))
        const uint32_t a = cl.narrow ? div32(x * cl.s, cl.divL32) : (uint32_t)div64((uint64_t)x * cl.s, cl.divL);
        rc = a * cl.sigma;
        lo = div64((uint64_t)a * cl.L + cl.s - 1, cl.divs64);
        hi = div64((uint64_t)(a + 1) * cl.L + cl.s - 1, cl.divs64);
      } else {
        rc = row_contrib<SRC>(D, Cf, A, x);
        lo = (uint64_t)div32(x, cl.divb) * cl.b;
        hi = lo + cl.b;
      }
      run_lo = (uint32_t)lo;
      run_hi = (uint32_t)(hi < Lf ? hi : Lf);
    }
    if (use_runs && x + 4 <= run_hi) {
      v[0] = v[1] = v[2] = v[3] = T[base + rc];
    } else if (SRC == R_TAB4) {
      const uint4 c = *reinterpret_cast<const uint4*>(Cf + x);
      v[0] = T[base + c.x]; v[1] = T[base + c.y]; v[2] = T[base + c.z]; v[3] = T[base + c.w];
    } else if (SRC == R_TAB2A && x + 4 <= Lf) {
      // x and Lin are multiples of 4: the group stays inside one entry of C2
      uint32_t q0, r0;
      divmod32(x, A.divLin, q0, r0);
      const uint32_t c = base + __ldg(A.C2 + q0);
      const uint4 f = *reinterpret_cast<const uint4*>(Cf + r0);
      v[0] = T[c + f.x]; v[1] = T[c + f.y]; v[2] = T[c + f.z]; v[3] = T[c + f.w];
    } else if (SRC == R_CYCLIC && x + 4 <= Lf) {
      // x mod s once, then one step per point
      const Comp& c0 = D.comp[D.k - 1][0];
      uint32_t q, a;
      divmod32(x, c0.divs, q, a);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[i] = T[base + a * c0.sigma];
        a = a + 1 == c0.s ? 0u : a + 1;
      }
    } else if (SRC == R_BCYC && x + 4 <= Lf) {
      // a group across blocks of b points: (x / b) mod s once, then the
      // position inside the block and the block's residue step along
      const Comp& c0 = D.comp[D.k - 1][0];
      uint32_t blk, rb, q, a;
      divmod32(x, c0.divb, blk, rb);
      divmod32(blk, c0.divs, q, a);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[i] = T[base + a * c0.sigma];
        if (++rb == c0.b) {
          rb = 0;
          a = a + 1 == c0.s ? 0u : a + 1;
        }
      }
    } else if (SRC == R_TAB2 && x + 4 <= Lf && A.Lin >= 4) {
      // the group meets at most two entries of C2 (q0 and, when it crosses
      // a boundary of the inner table, q0 + 1 < L[m], the row going on)
      uint32_t q0, r0;
      divmod32(x, A.divLin, q0, r0);
      const uint32_t lo = base + __ldg(A.C2 + q0);
      const uint32_t hi = r0 + 3 >= A.Lin ? base + __ldg(A.C2 + q0 + 1) : lo;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t r = r0 + i;
        const bool w = r >= A.Lin;
        v[i] = T[(w ? hi : lo) + Cf[w ? r - A.Lin : r]];
      }
    } else if (x + 4 <= Lf) {
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = T[base + row_contrib<SRC>(D, Cf, A, x + i)];
    } else if (Lf >= 4) {
      // the group crosses into the next row (at most once): select, do not
      // branch, so the lane does not hold its warp up (points past the end
      // of the launch are not stored)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t xi = x + i;
        const bool w = xi >= Lf;
        v[i] = T[(w ? nbase : base) + row_contrib<SRC>(D, Cf, A, w ? xi - Lf : xi)];
      }
    } else {
      uint32_t xi = x, ri = row, bi = base;
      for (int i = 0; i < cnt; ++i) {
        while (xi >= Lf) {
          xi -= Lf;
          ri += 1;
          bi = ri == row + 1 ? nbase : row_base_m<uint32_t>(D, tabs, ctab, ri, m);
        }
        v[i] = T[bi + row_contrib<SRC>(D, Cf, A, xi)];
        ++xi;
      }
    }
    if (cnt == 4 && vec_ok) {
      __stcs(reinterpret_cast<int4*>(ids + lin0), make_int4((int)v[0], (int)v[1], (int)v[2], (int)v[3]));
    } else {
      for (int i = 0; i < cnt; ++i) ids[lin0 + i] = (int32_t)v[i];
    }
    x += 128;
    if (x >= Lf) {
      if (Lf >= 128) {
        x -= Lf;
        row += 1;
        base = nbase;
      } else {
        uint32_t q, r;
        divmod32(x, divLf, q, r);
        row += q;
        x = r;
        base = row_base_m<uint32_t>(D, tabs, ctab, row, m);
      }
      nbase = row + 1 < rows ? row_base_inl<uint32_t>(D, tabs, ctab, row + 1, m) : 0;
    }
  }
}

// ids for the 4-point groups [gbeg, gend) of one warp: lane l takes groups
// gbeg + l, gbeg + l + 32, ... so each store instruction of the warp writes
// 512 contiguous bytes.  Between two groups of a lane the fastest
// coordinate advances by 128 and the row base is recomputed only on wrap.
//   T  : chain table (shared memory when TSMEM)
//   Cs : c_last in shared memory (M_FAST_SMEM)
template <typename I, int MODE, bool TSMEM>
__device__ __forceinline__ void ids_range(const MapCore& D, const Tabs& tabs, const uint32_t* __restrict__ T,
                                          const uint32_t* __restrict__ Cs, const uint32_t* __restrict__ ctab,
                                          I gbeg, I gend, int lane, int vec_ok, int32_t* __restrict__ ids) {
  const int last = D.k - 1;
  const I Llast = (I)D.L[last];
  const uint32_t* __restrict__ cg = ctab + tabs.off[last];
  const I N = (I)D.npoints;
  I g = gbeg + (I)lane;
  if (g >= gend) return;
  I lin0 = g * 4;
  I row, x;
  split_lin<I>(D, lin0, row, x);
  uint32_t base = row_base<I>(D, tabs, ctab, row);
  // fast rows of at least 128 points, 32-bit indices: the next row's base is
  // loaded a wrap ahead, so its latency overlaps the groups in between
  const bool ahead = MODE != M_GENERAL && sizeof(I) == 4 && Llast >= 128;
  const I rows = N / Llast;
  uint32_t nbase = ahead && row + 1 < rows ? row_base_inl<uint32_t>(D, tabs, ctab, (uint32_t)(row + 1), last) : 0;
  for (; g < gend; g += 32, lin0 += 128) {
    uint32_t v0, v1, v2, v3;
    int cnt = 4;
    if (MODE != M_GENERAL) {
      // Llast % 4 == 0: the group lies inside one row and x % 4 == 0
      const uint4 c = MODE == M_FAST_SMEM ? *reinterpret_cast<const uint4*>(Cs + x)
                                          : __ldg(reinterpret_cast<const uint4*>(cg + x));
      if (TSMEM) {
        v0 = T[base + c.x]; v1 = T[base + c.y]; v2 = T[base + c.z]; v3 = T[base + c.w];
      } else {
        v0 = __ldg(T + base + c.x); v1 = __ldg(T + base + c.y);
        v2 = __ldg(T + base + c.z); v3 = __ldg(T + base + c.w);
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
          v[i] = TSMEM ? T[bi + c] : __ldg(T + bi + c);
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
    x += 128;
    if (x >= Llast) {
      if (Llast >= 128) {
        x -= Llast;
        row += 1;
      } else {
        split_lin<I>(D, lin0 + 128, row, x);
      }
      if (ahead) {
        base = nbase;
        nbase = row + 1 < rows ? row_base_inl<uint32_t>(D, tabs, ctab, (uint32_t)(row + 1), last) : 0;
      } else {
        base = row_base<I>(D, tabs, ctab, row);
      }
    }
  }
}

// Linear-cyclic (Fig. 5): F = lin mod P; consecutive points advance F by 1
// and consecutive groups of a lane by 128 mod P.
template <typename I, bool TSMEM>
__device__ __forceinline__ void ids_range_lc(const MapCore& D, const uint32_t* __restrict__ T, I gbeg, I gend,
                                             int lane, int vec_ok, int32_t* __restrict__ ids) {
  const I N = (I)D.npoints;
  I g = gbeg + (I)lane;
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
      v[i] = TSMEM ? T[F] : __ldg(T + F);
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

// Linear-cyclic halo deficit of slab entry e (the slabs x_t = 0 and
// x_t = L_t - 1 of dimension t, 2 N / L_t points): the flat index F of that
// boundary point.
__device__ __forceinline__ uint32_t lc_slab_F(const MapCore& D, int t, uint64_t e) {
  const uint64_t per_slab = D.npoints / D.L[t];
  const uint64_t side = e >= per_slab;
  const uint64_t s = e - side * per_slab;
  const uint64_t stride = D.lc_stride[t];
  const uint64_t hi = s / stride, lo = s - hi * stride;
  const uint64_t xt = side ? D.L[t] - 1 : 0;
  const uint64_t lin = hi * (D.L[t] * stride) + xt * stride + lo;
  uint64_t q, F;
  divmod64(lin, D.divP64, q, F);
  return (uint32_t)F;
}

// Extended Euclid: g = gcd(a, m) and the inverse of a / g modulo m / g.
__device__ __forceinline__ void gcd_inverse(int64_t a, int64_t m, int64_t& g, int64_t& inv) {
  int64_t r0 = a, r1 = m, s0 = 1, s1 = 0;
  while (r1 != 0) {
    const int64_t q = r0 / r1;
    int64_t tmp = r0 - q * r1; r0 = r1; r1 = tmp;
    tmp = s0 - q * s1; s0 = s1; s1 = tmp;
  }
  g = r0;
  const int64_t mg = m / g;
  inv = mg == 1 ? 0 : ((s0 % mg) + mg) % mg;
}

// Element-count halo of a linear-cyclic launch, slab entry e of dimension t:
// the slabs are the positions x_t in [0, lo_n) and then L_t - 1, L_t - 2, ...
// (the positions whose halo window the boundary cuts).  Returns F of the
// point and its x_t.
__device__ __forceinline__ uint32_t lc_wslab_point(const MapCore& D, int t, uint64_t e, uint64_t lo_n,
                                                   uint64_t& xt) {
  const uint64_t per_slab = D.npoints / D.L[t];
  const uint64_t sidx = e / per_slab;
  const uint64_t s = e - sidx * per_slab;
  const uint64_t stride = D.lc_stride[t];
  const uint64_t hi = s / stride, lo = s - hi * stride;
  xt = sidx < lo_n ? sidx : D.L[t] - 1 - (sidx - lo_n);
  const uint64_t lin = hi * (D.L[t] * stride) + xt * stride + lo;
  uint64_t q, F;
  divmod64(lin, D.divP64, q, F);
  return (uint32_t)F;
}

}  // namespace mp
