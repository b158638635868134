// Host planner: validates a launch, expands decompose / balance_split into
// splits, applies the rank fix-up and compiles the result into the flat
// descriptor the kernels read.  Also the canonical transform alphabet used by
// the random-chain builder and the decompose search.
#include <algorithm>
#include <cstring>

#include "engine.h"

namespace mp {

namespace {

constexpr int64_t kMaxExtent = MP_MAX_EXTENT;   // keeps x * s below 2^64
constexpr int64_t kMaxPoints = int64_t(1) << 62;

std::vector<int64_t> divisors_ascending(int64_t v) {
  std::vector<int64_t> lo, hi;
  for (int64_t d = 1; d * d <= v; ++d)
    if (v % d == 0) {
      lo.push_back(d);
      if (d != v / d) hi.push_back(v / d);
    }
  std::reverse(hi.begin(), hi.end());
  lo.insert(lo.end(), hi.begin(), hi.end());
  return lo;
}

void factorise_rec(int64_t rest, int k, std::vector<int64_t>& cur,
                   std::vector<std::vector<int64_t>>& out) {
  if (k == 1) {
    cur.push_back(rest);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int64_t d : divisors_ascending(rest)) {
    cur.push_back(d);
    factorise_rec(rest / d, k - 1, cur, out);
    cur.pop_back();
  }
}

struct Builder {
  std::vector<int64_t> shape;
  std::vector<HostPrim> prims;
  std::vector<std::vector<int64_t>> before;   // shape before each primitive

  int split(int i, int64_t d) {
    int r = (int)shape.size();
    if (i < 0 || i >= r || d < 1 || shape[i] % d != 0) return MP_EINVAL;
    if (r + 1 > kMaxRank) return MP_ENOTSUP;
    if ((int)prims.size() >= kMaxPrim) return MP_ENOTSUP;
    before.push_back(shape);
    prims.push_back(HostPrim{P_SPLIT, i, -1, d});
    int64_t s = shape[i];
    shape[i] = d;
    shape.insert(shape.begin() + i + 1, s / d);
    return MP_OK;
  }
  int merge(int p, int q) {
    int r = (int)shape.size();
    if (!(0 <= p && p < q && q < r)) return MP_EINVAL;
    if ((int)prims.size() >= kMaxPrim) return MP_ENOTSUP;
    before.push_back(shape);
    prims.push_back(HostPrim{P_MERGE, p, q, 0});
    shape[p] *= shape[q];
    shape.erase(shape.begin() + q);
    return MP_OK;
  }
  int swap(int p, int q) {
    int r = (int)shape.size();
    if (p < 0 || q < 0 || p >= r || q >= r || p == q) return MP_EINVAL;
    if ((int)prims.size() >= kMaxPrim) return MP_ENOTSUP;
    before.push_back(shape);
    prims.push_back(HostPrim{P_SWAP, p, q, 0});
    std::swap(shape[p], shape[q]);
    return MP_OK;
  }
  // decompose(i, T): argmin factorisation of s_i, then k - 1 splits
  // split(i + n - 1, d_n), n = 1 .. k - 1 (Sec. 4.2).
  // h (may be null) and tmask select the generalised objective.
  int decompose(int i, int k, const int64_t* T, const int32_t* h = nullptr, int tmask = 0) {
    int r = (int)shape.size();
    if (i < 0 || i >= r || k < 1 || k > 4) return MP_EINVAL;
    unsigned __int128 prod = 1;
    for (int m = 0; m < k; ++m) {
      if (T[m] < 1) return MP_EINVAL;
      prod *= (uint64_t)T[m];
      if (prod >= (unsigned __int128)kMaxPoints) return MP_EINVAL;
    }
    if (tmask < 0 || tmask >= (1 << k)) return MP_EINVAL;
    bool weighted = tmask != 0;
    int64_t hw[4] = {1, 1, 1, 1};
    if (h) {
      bool any = false;
      for (int m = 0; m < k; ++m) {
        if (h[m] < 0) return MP_EINVAL;
        any = any || h[m] != 0;
      }
      if (any)
        for (int m = 0; m < k; ++m) hw[m] = h[m];
      weighted = weighted || any;
    }
    std::vector<int64_t> f;
    if (weighted) {
      int rc = decompose_argmin_weighted(shape[i], k, T, hw, tmask, f);
      if (rc) return rc;
    } else {
      f = decompose_argmin(shape[i], k, T);
    }
    for (int n = 1; n < k; ++n) {
      int rc = split(i + n - 1, f[n - 1]);
      if (rc) return rc;
    }
    return MP_OK;
  }
  int flatten() {
    while (shape.size() > 1) {
      int rc = merge(0, 1);
      if (rc) return rc;
    }
    return MP_OK;
  }
};

int target_rank(int kind, int k) {
  if (kind == MP_HIER) return 2 * k;
  if (kind == MP_LINEAR_CYCLIC) return 1;
  return k;
}

}  // namespace

std::vector<std::vector<int64_t>> ordered_factorisations(int64_t d, int k) {
  std::vector<std::vector<int64_t>> out;
  if (d < 1 || k < 1) return out;
  std::vector<int64_t> cur;
  factorise_rec(d, k, cur, out);
  return out;
}

// Objective of Sec. 4.2, sum_m d_m / l_m, compared exactly through the
// common denominator prod l; the first (lexicographically smallest) tuple
// wins ties.
std::vector<int64_t> decompose_argmin(int64_t d, int k, const int64_t* l) {
  std::vector<int64_t> best;
  unsigned __int128 best_v = 0;
  for (auto& f : ordered_factorisations(d, k)) {
    unsigned __int128 v = 0;
    for (int m = 0; m < k; ++m) {
      unsigned __int128 term = (uint64_t)f[m];
      for (int j = 0; j < k; ++j)
        if (j != m) term *= (uint64_t)l[j];
      v += term;
    }
    if (best.empty() || v < best_v) {
      best = f;
      best_v = v;
    }
  }
  return best;
}

// The appendix's generalised objective ("Generalization of the Decompose
// Primitive"): halo volume V = sum_m d_m h_m prod_{n != m} l_m plus
// (1 - 1/d_m) prod_n l_m for every transposed m.  Scaled by d (a constant of
// the argmin) every term is an integer: d V + prod l * sum_T (d_m - 1) d / d_m.
int decompose_argmin_weighted(int64_t d, int k, const int64_t* l, const int64_t* h, int tmask,
                              std::vector<int64_t>& out) {
  typedef unsigned __int128 u128;
  const u128 cap = ((u128)1) << 126;
  auto mul = [&](u128 a, u128 b, u128& r) {
    if (a != 0 && b > cap / a) return false;
    r = a * b;
    return true;
  };
  u128 Lambda = 1;
  for (int m = 0; m < k; ++m)
    if (!mul(Lambda, (uint64_t)l[m], Lambda)) return MP_EOVERFLOW;
  out.clear();
  u128 best_v = 0;
  for (auto& f : ordered_factorisations(d, k)) {
    u128 V = 0;
    for (int m = 0; m < k; ++m) {
      u128 term = (u128)(uint64_t)f[m] * (uint64_t)h[m];
      for (int n = 0; n < k; ++n)
        if (n != m && !mul(term, (uint64_t)l[n], term)) return MP_EOVERFLOW;
      V += term;
      if (V > cap) return MP_EOVERFLOW;
    }
    u128 v;
    if (!mul(V, (uint64_t)d, v)) return MP_EOVERFLOW;
    for (int m = 0; m < k; ++m) {
      if (!((tmask >> m) & 1)) continue;
      u128 add;
      if (!mul(Lambda, (u128)(uint64_t)(f[m] - 1) * (uint64_t)(d / f[m]), add)) return MP_EOVERFLOW;
      v += add;
      if (v > cap) return MP_EOVERFLOW;
    }
    if (out.empty() || v < best_v) {
      out = f;
      best_v = v;
    }
  }
  return MP_OK;
}

std::vector<CanonOp> canonical_alphabet(const std::vector<int64_t>& shape) {
  std::vector<CanonOp> out;
  int r = (int)shape.size();
  for (int i = 0; i < r; ++i)
    for (int64_t d : divisors_ascending(shape[i]))
      if (d > 1 && d < shape[i]) out.push_back(CanonOp{P_SPLIT, i, -1, d});
  for (int p = 0; p < r; ++p)
    for (int q = p + 1; q < r; ++q) out.push_back(CanonOp{P_MERGE, p, q, 0});
  for (int p = 0; p < r; ++p)
    for (int q = p + 1; q < r; ++q) out.push_back(CanonOp{P_SWAP, p, q, 0});
  return out;
}

void apply_canon(std::vector<int64_t>& shape, const CanonOp& c) {
  if (c.op == P_SPLIT) {
    int64_t s = shape[c.p];
    shape[c.p] = c.d;
    shape.insert(shape.begin() + c.p + 1, s / c.d);
  } else if (c.op == P_MERGE) {
    shape[c.p] *= shape[c.q];
    shape.erase(shape.begin() + c.q);
  } else {
    std::swap(shape[c.p], shape[c.q]);
  }
}

namespace {
void chains_rec(const std::vector<int64_t>& shape, int remaining, std::vector<CanonOp>& cur,
                std::vector<std::vector<CanonOp>>& out) {
  if (remaining == 0) {
    out.push_back(cur);
    return;
  }
  for (const CanonOp& c : canonical_alphabet(shape)) {
    std::vector<int64_t> next = shape;
    apply_canon(next, c);
    cur.push_back(c);
    chains_rec(next, remaining - 1, cur, out);
    cur.pop_back();
  }
}
}  // namespace

std::vector<std::vector<CanonOp>> canonical_chains(int64_t nodes, int64_t ppn, int max_depth) {
  std::vector<std::vector<CanonOp>> out;
  std::vector<int64_t> m0 = {nodes, ppn};
  for (int depth = 0; depth <= max_depth; ++depth) {
    std::vector<CanonOp> cur;
    chains_rec(m0, depth, cur, out);
  }
  return out;
}

int build_plan(const mp_space* space, const mp_machine* machine, const mp_xform* chain, int n_xf,
               const mp_dist* dist, Plan& out) {
  if (!space || !machine || !dist) return MP_EINVAL;
  const int k = space->rank;
  if (k < 1 || k > MP_MAX_TASK_RANK) return MP_EINVAL;
  unsigned __int128 npts = 1;
  for (int t = 0; t < k; ++t) {
    if (space->ext[t] < 1) return MP_EINVAL;
    if (space->ext[t] >= kMaxExtent) return MP_ENOTSUP;
    npts *= (uint64_t)space->ext[t];
    if (npts >= (unsigned __int128)kMaxPoints) return MP_EOVERFLOW;
  }
  if (machine->nodes < 1 || machine->procs_per_node < 1) return MP_EINVAL;
  const int64_t P = (int64_t)machine->nodes * machine->procs_per_node;
  if (P > MP_MAX_PROCS) return MP_ENOTSUP;
  if (dist->kind < MP_BLOCK || dist->kind > MP_LINEAR_CYCLIC) return MP_EINVAL;
  if (dist->kind == MP_BLOCK_CYCLIC && dist->b < 1) return MP_EINVAL;
  if (n_xf < 0 || n_xf > MP_MAX_XFORMS || (n_xf > 0 && !chain)) return MP_EINVAL;

  Builder B;
  B.shape = {machine->nodes, machine->procs_per_node};
  for (int o = 0; o < n_xf; ++o) {
    const mp_xform& x = chain[o];
    int rc;
    switch (x.op) {
      case MP_SPLIT: rc = B.split(x.i, x.d); break;
      case MP_MERGE: rc = B.merge(x.i, x.j); break;
      case MP_SWAP: rc = B.swap(x.i, x.j); break;
      case MP_DECOMPOSE: rc = B.decompose(x.i, x.k, x.T, x.h, x.transpose); break;
      case MP_BALANCE_SPLIT: {
        // balance_split(i, k) = decompose(i, (1, ..., 1))
        const int64_t ones[4] = {1, 1, 1, 1};
        rc = (x.k >= 1 && x.k <= 4) ? B.decompose(x.i, x.k, ones) : MP_EINVAL;
        break;
      }
      default: rc = MP_EINVAL;
    }
    if (rc) return rc;
  }

  int64_t L[4];
  for (int t = 0; t < k; ++t) L[t] = space->ext[t];
  const int tr = target_rank(dist->kind, k);
  if ((int)B.shape.size() != tr) {
    int rc = B.flatten();
    if (rc) return rc;
    if (dist->kind == MP_HIER) {
      // Appendix A.1: decompose the node dimension by the task space, then
      // the processor dimension by the task space / node factors (>= 1).
      if ((rc = B.split(0, machine->nodes))) return rc;
      if ((rc = B.decompose(0, k, L))) return rc;
      int64_t T2[4];
      for (int t = 0; t < k; ++t) T2[t] = std::max<int64_t>(1, L[t] / B.shape[t]);
      if ((rc = B.decompose(k, k, T2))) return rc;
    } else if (dist->kind != MP_LINEAR_CYCLIC) {
      if ((rc = B.decompose(0, k, L))) return rc;
    }
  }
  if ((int)B.shape.size() != tr) return MP_EINVAL;

  // ---------------------------------------------------------- descriptor
  MapDesc& D = out.desc;
  std::memset(&D, 0, sizeof(D));
  D.k = k;
  D.lc = dist->kind == MP_LINEAR_CYCLIC;
  D.rank = tr;
  D.P = (uint32_t)P;
  D.g = (uint32_t)machine->procs_per_node;
  D.npoints = (uint64_t)npts;
  D.divP = make_div32((uint32_t)P);
  D.divP64 = make_div64((uint64_t)P);
  for (int t = 0; t < k; ++t) {
    D.L[t] = (uint64_t)L[t];
    D.divL64[t] = make_div64((uint64_t)L[t]);
    D.divL32[t] = make_div32(L[t] <= 0xFFFFFFFFll ? (uint32_t)L[t] : 1u);
  }
  uint32_t sigma = 1;
  for (int u = 0; u < tr; ++u) {
    D.s[u] = (uint32_t)B.shape[u];
    D.sigma[u] = sigma;
    D.divs[u] = make_div32((uint32_t)B.shape[u]);
    sigma *= (uint32_t)B.shape[u];
  }
  auto comp = [&](int kind, int u, int t, int slot) {
    Comp c;
    std::memset(&c, 0, sizeof(c));
    c.kind = kind;
    c.s = D.s[u];
    c.sigma = D.sigma[u];
    c.b = (uint32_t)std::max(1, dist->b);
    c.L = (uint64_t)L[t];
    c.narrow = (unsigned __int128)(uint64_t)L[t] * c.s < ((unsigned __int128)1 << 32);
    c.divL = make_div64((uint64_t)L[t]);
    c.divs64 = make_div64(c.s);
    c.divb64 = make_div64(c.b);
    c.divL32 = make_div32(c.narrow ? (uint32_t)L[t] : 1u);
    c.divs = make_div32(c.s);
    c.divb = make_div32(c.b);
    D.owner_dim[u] = t;
    D.owner_slot[u] = slot;
    return c;
  };
  for (int t = 0; t < k; ++t) {
    switch (dist->kind) {
      case MP_BLOCK: D.ncomp[t] = 1; D.comp[t][0] = comp(C_BLOCK, t, t, 0); break;
      case MP_CYCLIC: D.ncomp[t] = 1; D.comp[t][0] = comp(C_CYCLIC, t, t, 0); break;
      case MP_BLOCK_CYCLIC: D.ncomp[t] = 1; D.comp[t][0] = comp(C_BCYC, t, t, 0); break;
      case MP_HIER:
        D.ncomp[t] = 2;
        D.comp[t][0] = comp(C_BLOCK, t, t, 0);
        D.comp[t][1] = comp(C_CYCLIC, k + t, t, 1);
        break;
      default: D.ncomp[t] = 0; break;
    }
    if (D.ncomp[t] > 0) {
      D.J[t] = D.comp[t][0].s * (D.ncomp[t] > 1 ? D.comp[t][1].s : 1u);
      D.Joff[t] = D.Jtotal;
      D.Jtotal += D.J[t];
    }
  }
  if (D.lc) {
    D.owner_dim[0] = 0;
    for (int t = 0; t < k; ++t) {
      unsigned __int128 stride = 1;
      for (int u = t + 1; u < k; ++u) stride *= (uint64_t)L[u];
      D.lc_stride_mod[t] = (uint32_t)(stride % (uint64_t)P);
      D.lc_stride[t] = (uint64_t)stride;
    }
  }
  D.nprim = (int)B.prims.size();
  for (int o = 0; o < D.nprim; ++o) {
    const HostPrim& h = B.prims[o];
    Prim& p = D.prim[o];
    p.op = h.op;
    p.p = h.p;
    p.q = h.q;
    p.rank_before = (int32_t)B.before[o].size();
    if (h.op == P_SPLIT) {
      p.d = (uint32_t)h.d;
    } else if (h.op == P_MERGE) {
      p.d = (uint32_t)B.before[o][h.p];
      p.div = make_div32(p.d);
    }
  }
  out.prims = B.prims;
  out.rank = tr;
  for (int u = 0; u < tr; ++u) out.shape[u] = B.shape[u];
  return MP_OK;
}

}  // namespace mp

// ------------------------------------------------------------ C ABI (host)

extern "C" int mp_plan(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                       int n_xf, const mp_dist* dist, int32_t* rank, int64_t* shape,
                       int32_t* n_prims, int64_t* prims, int32_t prims_cap) {
  mp::Plan pl;
  int rc = mp::build_plan(space, machine, chain, n_xf, dist, pl);
  if (rc) return rc;
  if (rank) *rank = pl.rank;
  if (shape)
    for (int u = 0; u < pl.rank; ++u) shape[u] = pl.shape[u];
  if (n_prims) *n_prims = (int32_t)pl.prims.size();
  if (prims)
    for (int o = 0; o < (int)pl.prims.size() && o < prims_cap; ++o) {
      prims[4 * o + 0] = pl.prims[o].op;
      prims[4 * o + 1] = pl.prims[o].p;
      prims[4 * o + 2] = pl.prims[o].q;
      prims[4 * o + 3] = pl.prims[o].d;
    }
  return MP_OK;
}

extern "C" int mp_chain_from_draws(int32_t nodes, int32_t procs_per_node, int32_t depth,
                                   const uint64_t* draws, mp_xform* out, int32_t* n_out) {
  if (nodes < 1 || procs_per_node < 1 || depth < 0 || depth > MP_MAX_XFORMS || !n_out ||
      (depth > 0 && (!draws || !out)))
    return MP_EINVAL;
  std::vector<int64_t> shape = {nodes, procs_per_node};
  int m = 0;
  for (int step = 0; step < depth; ++step) {
    auto A = mp::canonical_alphabet(shape);
    if (A.empty()) break;
    const mp::CanonOp& c = A[draws[step] % A.size()];
    mp::apply_canon(shape, c);
    mp_xform x;
    std::memset(&x, 0, sizeof(x));
    x.op = c.op == mp::P_SPLIT ? MP_SPLIT : (c.op == mp::P_MERGE ? MP_MERGE : MP_SWAP);
    x.i = c.p;
    x.j = c.op == mp::P_SPLIT ? 0 : c.q;
    x.d = c.op == mp::P_SPLIT ? c.d : 0;
    out[m++] = x;
  }
  *n_out = m;
  return MP_OK;
}

extern "C" int mp_search_space(int32_t procs, int32_t procs_per_node, int32_t max_depth,
                               int64_t* n_factorisations, int64_t* n_chains) {
  if (procs < 1 || procs_per_node < 1 || procs % procs_per_node || max_depth < 0 || max_depth > 4)
    return MP_EINVAL;
  if (n_factorisations) *n_factorisations = (int64_t)mp::ordered_factorisations(procs, 3).size();
  if (n_chains)
    *n_chains = (int64_t)mp::canonical_chains(procs / procs_per_node, procs_per_node, max_depth).size();
  return MP_OK;
}

// Algorithm A1: primes ascending, each into the smallest factor so far (the
// first on ties), factors sorted descending at the end.
extern "C" int mp_greedy_grid(int64_t d, int32_t k, int64_t* out) {
  if (d < 1 || k < 1 || k > 4 || !out) return MP_EINVAL;
  std::vector<int64_t> grid((size_t)k, 1);
  int64_t rest = d;
  auto place = [&](int64_t p) {
    size_t j = 0;
    for (size_t m = 1; m < grid.size(); ++m)
      if (grid[m] < grid[j]) j = m;
    grid[j] *= p;
  };
  for (int64_t p = 2; p <= rest / p; ++p)
    while (rest % p == 0) {
      place(p);
      rest /= p;
    }
  if (rest > 1) place(rest);
  std::sort(grid.begin(), grid.end(), [](int64_t a, int64_t b) { return a > b; });
  for (int m = 0; m < k; ++m) out[m] = grid[(size_t)m];
  return MP_OK;
}
