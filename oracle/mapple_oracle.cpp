// Plain, slow CPU oracle for the Mapple index-mapping hot path.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library.  It shares
// no code, header, table or helper with the CUDA engine.
//
// Every function evaluates the paper's definitions literally, one point and
// one transform at a time, on explicit coordinate vectors, with exact integer
// arithmetic (__int128 where a product can exceed 64 bits):
//
//   * transforms split / merge / swap: the index formulas of Fig. 4 (Sec. 3.3),
//     a point of the transformed space is resolved by applying each
//     transform's formula from the last transform to the first (Sec. 3.3,
//     "m''[a0,a1] = m'[...] = m[...]", and Sec. 5.2's block1D_x example);
//   * decompose(i, T): the optimisation problem of Sec. 4.2 (minimise
//     sum d_m / l_m subject to prod d_m = d_i), solved by the exhaustive
//     prime-exponent enumeration of Sec. 4.3, then expanded into k-1 splits
//     as Sec. 4.2 states;
//   * distributions: block (Fig. 1a / Fig. 3: idx = point * m.size / space),
//     cyclic (x mod s) and block-cyclic (floor(x / b) mod s, which the paper
//     names without a formula), the Cannon hierarchical block/cyclic mapper
//     (Appendix A.1), the linearised round-robin of Fig. 5 (C-order linear
//     index mod P; the figure itself is not available);
//   * halo volume: every directed nearest-neighbour face whose two endpoints
//     have different owners (Sec. 4.2, Fig. 10 surface formula; each face
//     counted once per direction, non-periodic); and the anisotropic element
//     count with per-dimension halo widths (the appendix's generalised
//     decompose): every element once per other owner that needs it along
//     each dimension;
//   * decompose with halo widths and all-to-all transposes: the appendix's
//     generalised objective V + sum_T V*_n, compared exactly;
//   * the greedy grid heuristic of Algorithm A1;
//   * the matmul moved-bytes cost of a candidate (per operand tile: distinct
//     processors - 1, distinct nodes - 1) and the exhaustive lexicographic
//     argmin over (factorisation, chain) candidates in canonical order;
//   * the two-level search over node grid x GPU grid (the Solomonik mapper
//     of Fig. 5b and the Cannon mapper of Appendix A.1 as search spaces):
//     inter-node then inter-processor element halo volume.
//
// Parity status: the Fig. 5 linearised cyclic distribution (its order is
// read as C order) and balance_split (read as decompose(i, (1, ..., 1))) are
// "parity unpinned" beyond the special cases the tests list (the paper gives
// no worked numbers for them).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

typedef int64_t i64;
typedef uint64_t u64;
typedef __int128 i128;

enum { OP_SPLIT = 0, OP_MERGE = 1, OP_SWAP = 2, OP_DECOMPOSE = 3, OP_BALANCE_SPLIT = 4 };
enum { D_BLOCK = 0, D_CYCLIC = 1, D_BLOCK_CYCLIC = 2, D_HIER = 3, D_LINEAR_CYCLIC = 4 };

const int MAXR = 32;   // processor-space rank bound inside the oracle

// A user transform as the oracle receives it: XF_W int64 per op
//   [op, i, j, k, d, T0, T1, T2, T3, h0, h1, h2, h3, transpose_mask]
// (h and the mask only matter to decompose; all-zero h means isotropic).
const int XF_W = 14;

// After decompose / balance_split are expanded only these remain.
struct Prim {
  int op;        // OP_SPLIT, OP_MERGE, OP_SWAP
  int p, q;      // split: p = i; merge/swap: p, q
  i64 d;         // split factor
  int rank_before;
  i64 before[MAXR];   // shape of the space the primitive is applied to
};

struct Plan {
  int n, g;                 // Machine(GPU) = (nodes, procs per node)
  int k;                    // task-space rank
  i64 L[4];                 // task-space extents
  int dist, b;              // distribution kind and block-cyclic block size
  std::vector<Prim> prims;  // chain + rank fix-up, in application order
  int rank;                 // final processor-space rank
  i64 s[MAXR];              // final processor-space shape
  i64 P;
  i64 npoints;
};

// ---------------------------------------------------------------- numbers

std::vector<std::pair<i64, int>> prime_factorise(i64 d) {
  std::vector<std::pair<i64, int>> out;
  for (i64 p = 2; p * p <= d; ++p) {
    int e = 0;
    while (d % p == 0) { d /= p; ++e; }
    if (e) out.push_back({p, e});
  }
  if (d > 1) out.push_back({d, 1});
  return out;
}

i64 ipow(i64 b, int e) { i64 r = 1; while (e--) r *= b; return r; }

// All non-negative integer solutions of z_1 + ... + z_k = a (Sec. 4.3), by
// recursion on the first coordinate.
void stars_and_bars(int a, int k, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  if ((int)cur.size() == k - 1) {
    cur.push_back(a);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int z = 0; z <= a; ++z) {
    cur.push_back(z);
    stars_and_bars(a - z, k, cur, out);
    cur.pop_back();
  }
}

// Every ordered k-factorisation of d (Sec. 4.3): per prime p_j distribute its
// exponent a_j over the k factors, then take the Cartesian product over the
// primes.  Returned sorted lexicographically ascending (the candidate order).
std::vector<std::vector<i64>> factorisations(i64 d, int k) {
  std::vector<std::vector<i64>> result;
  if (d < 1 || k < 1) return result;
  auto pf = prime_factorise(d);
  std::vector<std::vector<std::vector<int>>> per_prime;
  for (auto& pe : pf) {
    std::vector<std::vector<int>> sols;
    std::vector<int> cur;
    stars_and_bars(pe.second, k, cur, sols);
    per_prime.push_back(sols);
  }
  // Cartesian product
  std::vector<size_t> idx(per_prime.size(), 0);
  while (true) {
    std::vector<i64> f(k, 1);
    for (size_t j = 0; j < per_prime.size(); ++j)
      for (int m = 0; m < k; ++m) f[m] *= ipow(pf[j].first, per_prime[j][idx[j]][m]);
    result.push_back(f);
    size_t j = 0;
    while (j < per_prime.size()) {
      if (++idx[j] < per_prime[j].size()) break;
      idx[j] = 0;
      ++j;
    }
    if (j == per_prime.size()) break;
  }
  std::sort(result.begin(), result.end());
  return result;
}

// decompose objective (Sec. 4.2): sum_m d_m / l_m, compared exactly as the
// integer sum_m d_m * prod_{j != m} l_j (common denominator prod l).
i128 decompose_objective(const std::vector<i64>& f, const i64* l, int k) {
  i128 tot = 0;
  for (int m = 0; m < k; ++m) {
    i128 term = f[m];
    for (int j = 0; j < k; ++j)
      if (j != m) term *= l[j];
    tot += term;
  }
  return tot;
}

// Generalised objective of the appendix ("Generalization of the Decompose
// Primitive"): with halo width h_n along target dimension n the volume is
//   V = sum_n d_n h_n prod_{m != n} l_m,
// and an all-to-all transpose along dimension n adds
//   V*_n = (1 - 1/d_n) (prod_m w_m) d,   w_m = l_m / d_m,  d = prod_m d_m,
// i.e. (1 - 1/d_n) prod_m l_m.  The total V + sum_{n in T} V*_n is compared
// exactly after multiplying by the constant d:
//   d V + prod_m l_m * sum_{n in T} (d_n - 1) (d / d_n).
// Returns false when the value does not fit in 127 bits.
bool weighted_objective(const std::vector<i64>& f, const i64* l, const i64* h, int tmask, int k, i64 d,
                        i128& out) {
  const i128 lim = ((i128)1) << 125;
  i128 V = 0;
  for (int n = 0; n < k; ++n) {
    i128 term = (i128)f[n] * h[n];
    for (int m = 0; m < k; ++m) {
      if (m == n) continue;
      if (term > lim / l[m]) return false;
      term *= l[m];
    }
    V += term;
    if (V > lim) return false;
  }
  if (V > lim / d) return false;
  i128 tot = V * d;
  i128 Lambda = 1;
  for (int m = 0; m < k; ++m) {
    if (Lambda > lim / l[m]) return false;
    Lambda *= l[m];
  }
  for (int n = 0; n < k; ++n) {
    if (!((tmask >> n) & 1)) continue;
    const i128 c = (i128)(f[n] - 1) * (d / f[n]);
    if (c != 0 && Lambda > lim / c) return false;
    tot += Lambda * c;
    if (tot > lim) return false;
  }
  out = tot;
  return true;
}

// argmin over all factorisations; ties go to the lexicographically smallest
// tuple -- the enumeration is lexicographic and only a strictly
// smaller objective replaces the incumbent.  h == nullptr and tmask == 0 is
// the isotropic objective of Sec. 4.2.  Empty result: objective overflow.
std::vector<i64> decompose_factors(i64 d, int k, const i64* l, const i64* h = nullptr, int tmask = 0) {
  auto all = factorisations(d, k);
  std::vector<i64> best;
  i128 bestv = 0;
  for (auto& f : all) {
    i128 v;
    if (h == nullptr && tmask == 0) {
      v = decompose_objective(f, l, k);
    } else {
      i64 ones[4] = {1, 1, 1, 1};
      if (!weighted_objective(f, l, h ? h : ones, tmask, k, d, v)) return {};
    }
    if (best.empty() || v < bestv) { best = f; bestv = v; }
  }
  return best;
}

// ---------------------------------------------------------------- plan

struct Space {
  int r;
  i64 s[MAXR];
};

bool push_split(std::vector<Prim>& prims, Space& sp, int i, i64 d) {
  if (i < 0 || i >= sp.r || d < 1 || sp.r + 1 > MAXR) return false;
  if (sp.s[i] % d != 0) return false;
  Prim pr;
  pr.op = OP_SPLIT; pr.p = i; pr.q = -1; pr.d = d; pr.rank_before = sp.r;
  std::memcpy(pr.before, sp.s, sizeof(sp.s));
  prims.push_back(pr);
  // Fig. 4 / Sec. 3.3: (s_0, ..., d, s_i / d, ..., s_{n-1})
  Space nsp;
  nsp.r = sp.r + 1;
  for (int t = 0; t < i; ++t) nsp.s[t] = sp.s[t];
  nsp.s[i] = d;
  nsp.s[i + 1] = sp.s[i] / d;
  for (int t = i + 1; t < sp.r; ++t) nsp.s[t + 1] = sp.s[t];
  sp = nsp;
  return true;
}

bool push_merge(std::vector<Prim>& prims, Space& sp, int p, int q) {
  if (!(0 <= p && p < q && q < sp.r)) return false;
  Prim pr;
  pr.op = OP_MERGE; pr.p = p; pr.q = q; pr.d = 0; pr.rank_before = sp.r;
  std::memcpy(pr.before, sp.s, sizeof(sp.s));
  prims.push_back(pr);
  // Sec. 3.3: (s_0, ..., s_p * s_q, ..., s_{n-1}); dimension q removed
  Space nsp;
  nsp.r = sp.r - 1;
  int o = 0;
  for (int t = 0; t < sp.r; ++t) {
    if (t == q) continue;
    nsp.s[o++] = (t == p) ? sp.s[p] * sp.s[q] : sp.s[t];
  }
  sp = nsp;
  return true;
}

bool push_swap(std::vector<Prim>& prims, Space& sp, int p, int q) {
  if (p < 0 || q < 0 || p >= sp.r || q >= sp.r || p == q) return false;
  Prim pr;
  pr.op = OP_SWAP; pr.p = p; pr.q = q; pr.d = 0; pr.rank_before = sp.r;
  std::memcpy(pr.before, sp.s, sizeof(sp.s));
  prims.push_back(pr);
  std::swap(sp.s[p], sp.s[q]);
  return true;
}

// decompose(i, T) = k-1 splits split(i + n - 1, d_n), n = 1..k-1 (Sec. 4.2)
bool push_decompose(std::vector<Prim>& prims, Space& sp, int i, int k, const i64* T,
                    const i64* h = nullptr, int tmask = 0) {
  if (i < 0 || i >= sp.r || k < 1 || k > 4) return false;
  for (int m = 0; m < k; ++m)
    if (T[m] < 1) return false;
  // all-zero widths and no transposes: the isotropic objective
  bool weighted = tmask != 0;
  if (h)
    for (int m = 0; m < k; ++m) {
      if (h[m] < 0) return false;
      if (h[m] != 0) weighted = true;
    }
  if (tmask < 0 || tmask >= (1 << k)) return false;
  i64 hw[4] = {1, 1, 1, 1};
  if (h && weighted)
    for (int m = 0; m < k; ++m) hw[m] = h[m];
  std::vector<i64> f = weighted ? decompose_factors(sp.s[i], k, T, hw, tmask) : decompose_factors(sp.s[i], k, T);
  if ((int)f.size() != k) return false;
  for (int n = 1; n < k; ++n)
    if (!push_split(prims, sp, i + n - 1, f[n - 1])) return false;
  return true;
}

void flatten(std::vector<Prim>& prims, Space& sp) {
  while (sp.r > 1) push_merge(prims, sp, 0, 1);
}

int target_rank(int dist, int k) {
  if (dist == D_HIER) return 2 * k;
  if (dist == D_LINEAR_CYCLIC) return 1;
  return k;
}

// Returns 0 on success, 1 on an invalid chain or distribution.
int build_plan(Plan& pl, const i64* L, int k, int n, int g, const i64* xf, int nxf,
               int dist, int b) {
  if (k < 1 || k > 4 || n < 1 || g < 1) return 1;
  if (dist < 0 || dist > 4) return 1;
  if (dist == D_BLOCK_CYCLIC && b < 1) return 1;
  pl.n = n; pl.g = g; pl.k = k; pl.dist = dist; pl.b = b;
  pl.npoints = 1;
  for (int t = 0; t < k; ++t) {
    if (L[t] < 1) return 1;
    pl.L[t] = L[t];
    pl.npoints *= L[t];
  }
  pl.P = (i64)n * g;
  Space sp;
  sp.r = 2;
  sp.s[0] = n;
  sp.s[1] = g;
  pl.prims.clear();
  for (int o = 0; o < nxf; ++o) {
    const i64* e = xf + XF_W * o;
    int op = (int)e[0], i = (int)e[1], j = (int)e[2], kk = (int)e[3];
    i64 d = e[4];
    bool ok = false;
    if (op == OP_SPLIT) ok = push_split(pl.prims, sp, i, d);
    else if (op == OP_MERGE) ok = push_merge(pl.prims, sp, i, j);
    else if (op == OP_SWAP) ok = push_swap(pl.prims, sp, i, j);
    else if (op == OP_DECOMPOSE) ok = push_decompose(pl.prims, sp, i, kk, e + 5, e + 9, (int)e[13]);
    else if (op == OP_BALANCE_SPLIT) {
      // balance_split(i, k) is read as decompose(i, (1, ..., 1)): the paper
      // names it without a definition
      i64 ones[4] = {1, 1, 1, 1};
      ok = (kk >= 1 && kk <= 4) && push_decompose(pl.prims, sp, i, kk, ones);
    }
    if (!ok) return 1;
  }
  // rank fix-up so that the final space has the rank the distribution indexes
  int tr = target_rank(dist, k);
  if (sp.r != tr) {
    flatten(pl.prims, sp);
    if (dist == D_LINEAR_CYCLIC) {
      // already 1-D
    } else if (dist == D_HIER) {
      // Appendix A.1 pattern on the re-split machine (n, g): decompose the
      // node dimension by the task space, then the processor dimension by the
      // task space divided elementwise by the node factors (floor, at least 1).
      if (!push_split(pl.prims, sp, 0, n)) return 1;
      if (!push_decompose(pl.prims, sp, 0, k, pl.L)) return 1;
      i64 T2[4];
      for (int t = 0; t < k; ++t) {
        T2[t] = pl.L[t] / sp.s[t];
        if (T2[t] < 1) T2[t] = 1;
      }
      if (!push_decompose(pl.prims, sp, k, k, T2)) return 1;
    } else {
      if (!push_decompose(pl.prims, sp, 0, k, pl.L)) return 1;
    }
  }
  if (sp.r != tr) return 1;
  pl.rank = sp.r;
  std::memcpy(pl.s, sp.s, sizeof(sp.s));
  return 0;
}

// Resolve an index of the final space back to Machine(GPU) by applying each
// primitive's Fig. 4 formula from the last primitive to the first.
void resolve(const Plan& pl, const i64* a_final, i64& node, i64& proc) {
  i64 a[MAXR], bidx[MAXR];
  int r = pl.rank;
  for (int t = 0; t < r; ++t) a[t] = a_final[t];
  for (int o = (int)pl.prims.size() - 1; o >= 0; --o) {
    const Prim& pr = pl.prims[o];
    int n = pr.rank_before;   // rank of b (the space before the primitive)
    if (pr.op == OP_SPLIT) {
      int i = pr.p;
      for (int t = 0; t < n; ++t) {
        if (t < i) bidx[t] = a[t];
        else if (t == i) bidx[t] = a[i] + a[i + 1] * pr.d;
        else bidx[t] = a[t + 1];
      }
    } else if (pr.op == OP_MERGE) {
      int p = pr.p, q = pr.q;
      for (int t = 0; t < n; ++t) {
        if (t < p || (p < t && t < q)) bidx[t] = a[t];
        else if (t == p) bidx[t] = a[p] % pr.before[p];
        else if (t == q) bidx[t] = a[p] / pr.before[p];
        else bidx[t] = a[t - 1];
      }
    } else {  // swap
      for (int t = 0; t < n; ++t) bidx[t] = a[t];
      bidx[pr.p] = a[pr.q];
      bidx[pr.q] = a[pr.p];
    }
    for (int t = 0; t < n; ++t) a[t] = bidx[t];
    r = n;
  }
  node = a[0];
  proc = a[1];
}

// Distribution: task point -> index of the final processor space.
void distribute(const Plan& pl, const i64* x, i64* a) {
  int k = pl.k;
  switch (pl.dist) {
    case D_BLOCK:   // Fig. 1a: idx = point * m.size / space (floor, exact)
      for (int t = 0; t < k; ++t) a[t] = (i64)((i128)x[t] * pl.s[t] / pl.L[t]);
      break;
    case D_CYCLIC:
      for (int t = 0; t < k; ++t) a[t] = x[t] % pl.s[t];
      break;
    case D_BLOCK_CYCLIC:
      for (int t = 0; t < k; ++t) a[t] = (x[t] / pl.b) % pl.s[t];
      break;
    case D_HIER:    // Appendix A.1: upper = ip * m[:k] / is, lower = ip % m[k:]
      for (int t = 0; t < k; ++t) {
        a[t] = (i64)((i128)x[t] * pl.s[t] / pl.L[t]);
        a[k + t] = x[t] % pl.s[k + t];
      }
      break;
    case D_LINEAR_CYCLIC: {   // Fig. 5: C-order linearisation, round robin
      i128 lin = 0;
      for (int t = 0; t < k; ++t) lin = lin * pl.L[t] + x[t];
      a[0] = (i64)(lin % pl.s[0]);
      break;
    }
  }
}

i64 owner_of_point(const Plan& pl, const i64* x) {
  i64 a[MAXR];
  distribute(pl, x, a);
  i64 node, proc;
  resolve(pl, a, node, proc);
  return node * pl.g + proc;   // node-major processor id
}

void unravel(const Plan& pl, i64 lin, i64* x) {
  for (int t = pl.k - 1; t >= 0; --t) {
    x[t] = lin % pl.L[t];
    lin /= pl.L[t];
  }
}

// fn(lo, hi, worker) over [0, n) in `threads` contiguous chunks; serial
// below min_items (per-point loops: thread start-up outweighs small launches).
template <class F>
void parallel_for(i64 n, int threads, F fn, i64 min_items = 4096) {
  if (threads <= 1 || n < min_items) { fn(0, n, 0); return; }
  std::vector<std::thread> th;
  i64 chunk = (n + threads - 1) / threads;
  for (int w = 0; w < threads; ++w) {
    i64 lo = w * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back(fn, lo, hi, w);
  }
  for (auto& t : th) t.join();
}

// ------------------------------------------------- canonical op alphabet

struct COp { int op; int p; int q; i64 d; };

std::vector<i64> nontrivial_divisors(i64 s) {
  std::vector<i64> out;
  for (i64 d = 2; d < s; ++d)
    if (s % d == 0) out.push_back(d);
  return out;
}

// Canonical alphabet at shape s: split(i, d) for i ascending and
// d ascending over the divisors with 1 < d < s_i, then merge(p, q) for p < q
// lexicographic, then swap(p, q) for p < q lexicographic.
std::vector<COp> alphabet(const Space& sp) {
  std::vector<COp> out;
  for (int i = 0; i < sp.r; ++i)
    for (i64 d : nontrivial_divisors(sp.s[i])) out.push_back({OP_SPLIT, i, -1, d});
  for (int p = 0; p < sp.r; ++p)
    for (int q = p + 1; q < sp.r; ++q) out.push_back({OP_MERGE, p, q, 0});
  for (int p = 0; p < sp.r; ++p)
    for (int q = p + 1; q < sp.r; ++q) out.push_back({OP_SWAP, p, q, 0});
  return out;
}

bool apply_cop(std::vector<Prim>& prims, Space& sp, const COp& c) {
  if (c.op == OP_SPLIT) return push_split(prims, sp, c.p, c.d);
  if (c.op == OP_MERGE) return push_merge(prims, sp, c.p, c.q);
  return push_swap(prims, sp, c.p, c.q);
}

void enum_chains_rec(Space sp, int remaining, std::vector<COp>& cur,
                     std::vector<std::vector<COp>>& out) {
  if (remaining == 0) { out.push_back(cur); return; }
  auto A = alphabet(sp);
  for (auto& c : A) {
    Space nsp = sp;
    std::vector<Prim> dummy;
    apply_cop(dummy, nsp, c);
    cur.push_back(c);
    enum_chains_rec(nsp, remaining - 1, cur, out);
    cur.pop_back();
  }
}

// All chains of depth 0..max_depth over the canonical alphabet, ordered by
// depth, then lexicographically by the sequence of alphabet positions.
std::vector<std::vector<COp>> enum_chains(int n, int g, int max_depth) {
  std::vector<std::vector<COp>> out;
  Space sp;
  sp.r = 2; sp.s[0] = n; sp.s[1] = g;
  for (int depth = 0; depth <= max_depth; ++depth) {
    std::vector<COp> cur;
    enum_chains_rec(sp, depth, cur, out);
  }
  return out;
}

// ------------------------------------------------- matmul moved-bytes cost

// Owner (node, proc) of every flat index b of the 1-D space obtained by
// flattening chain(m0) with merge(0, 1) repeatedly.  This is the resolution
// of each b through the flatten merges and the chain; it does not depend on
// the factorisation, so it is tabulated once per chain.
struct ChainTable {
  std::vector<i64> node, proc;
};

ChainTable chain_table(int n, int g, const std::vector<COp>& chain) {
  Plan pl;
  pl.n = n; pl.g = g; pl.k = 1; pl.dist = D_LINEAR_CYCLIC; pl.b = 1;
  Space sp;
  sp.r = 2; sp.s[0] = n; sp.s[1] = g;
  for (auto& c : chain) apply_cop(pl.prims, sp, c);
  flatten(pl.prims, sp);
  pl.rank = 1;
  pl.s[0] = sp.s[0];
  i64 P = (i64)n * g;
  ChainTable tb;
  tb.node.resize(P);
  tb.proc.resize(P);
  for (i64 b = 0; b < P; ++b) {
    i64 a[1] = {b};
    resolve(pl, a, tb.node[b], tb.proc[b]);
  }
  return tb;
}

// Flat index of the decompose split of the flattened space into f = (f0, f1,
// f2): inverse of split(1, f1) then of split(0, f0) (dimension 0 fastest).
inline i64 flat_of(const i64* f, i64 a0, i64 a1, i64 a2) { return a0 + f[0] * (a1 + f[1] * a2); }

inline i64 blk(i64 x, i64 f, i64 L) { return (i64)((i128)x * f / L); }

// The moved-tile cost, literally, on the full tile grid: for every tile of A(i,k),
// B(k,j), C(i,j), count the distinct processors (and nodes) among the points
// (i,j,k) that touch it; the tile costs (distinct - 1) tile transfers.
// O(M N K) -- only for small grids (brute-force pin of the grouped form).
void matmul_cost_literal(i64 M, i64 N, i64 K, const ChainTable& tb, const i64* f,
                         i128& prim, i128& sec) {
  prim = 0; sec = 0;
  auto own = [&](i64 i, i64 j, i64 k) { return flat_of(f, blk(i, f[0], M), blk(j, f[1], N), blk(k, f[2], K)); };
  auto count = [&](std::vector<i64>& bs) {
    std::vector<i64> procs, nodes;
    for (i64 b : bs) { procs.push_back(tb.node[b] * 1000003 + tb.proc[b]); nodes.push_back(tb.node[b]); }
    std::sort(procs.begin(), procs.end());
    std::sort(nodes.begin(), nodes.end());
    i64 dp = std::unique(procs.begin(), procs.end()) - procs.begin();
    i64 dn = std::unique(nodes.begin(), nodes.end()) - nodes.begin();
    prim += dp - 1;
    sec += dn - 1;
  };
  std::vector<i64> bs;
  for (i64 i = 0; i < M; ++i)      // A(i,k): points (i, j, k) over j
    for (i64 k = 0; k < K; ++k) {
      bs.clear();
      for (i64 j = 0; j < N; ++j) bs.push_back(own(i, j, k));
      count(bs);
    }
  for (i64 k = 0; k < K; ++k)      // B(k,j): over i
    for (i64 j = 0; j < N; ++j) {
      bs.clear();
      for (i64 i = 0; i < M; ++i) bs.push_back(own(i, j, k));
      count(bs);
    }
  for (i64 i = 0; i < M; ++i)      // C(i,j): over k (reduction traffic)
    for (i64 j = 0; j < N; ++j) {
      bs.clear();
      for (i64 k = 0; k < K; ++k) bs.push_back(own(i, j, k));
      count(bs);
    }
}

// The same cost grouped by block coordinates: every tile whose two fixed
// coordinates fall in the same pair of blocks touches the same set of owners
// (the owner depends on a coordinate only through its block), so one fibre
// per block pair is evaluated and weighted by the number of tiles in it.
//
// The distinct block coordinates of each dimension and how many tiles fall in
// each depend on the factorisation and the extents only, so they are counted
// once per factorisation (BlockGroups) and shared by every chain.
struct BlockGroups {
  std::vector<std::vector<i64>> reps, wts;
};

BlockGroups block_groups(i64 M, i64 N, i64 K, const i64* f) {
  const i64 ext[3] = {M, N, K};
  BlockGroups bg;
  bg.reps.resize(3);
  bg.wts.resize(3);
  for (int t = 0; t < 3; ++t) {
    // distinct block coordinates of dimension t and how many tiles fall in each
    std::vector<i64> cnt(f[t], 0);
    for (i64 x = 0; x < ext[t]; ++x) cnt[blk(x, f[t], ext[t])]++;
    for (i64 a = 0; a < f[t]; ++a)
      if (cnt[a] > 0) { bg.reps[t].push_back(a); bg.wts[t].push_back(cnt[a]); }
  }
  return bg;
}

void matmul_cost_grouped(const BlockGroups& bg, const ChainTable& tb, const i64* f,
                         i64 n_nodes, i128& prim, i128& sec) {
  const std::vector<std::vector<i64>>& reps = bg.reps;
  const std::vector<std::vector<i64>>& wts = bg.wts;
  prim = 0; sec = 0;
  std::vector<char> seen_node(n_nodes, 0);
  std::vector<i64> touched;
  // family v: the fibre varies block coordinate v; u, w are the fixed ones
  for (int v = 0; v < 3; ++v) {
    int u = (v + 1) % 3, w = (v + 2) % 3;
    for (size_t iu = 0; iu < reps[u].size(); ++iu)
      for (size_t iw = 0; iw < reps[w].size(); ++iw) {
        i64 weight = wts[u][iu] * wts[w][iw];
        i64 distinct_nodes = 0;
        touched.clear();
        for (size_t iv = 0; iv < reps[v].size(); ++iv) {
          i64 a[3];
          a[u] = reps[u][iu]; a[w] = reps[w][iw]; a[v] = reps[v][iv];
          i64 b = flat_of(f, a[0], a[1], a[2]);
          i64 nd = tb.node[b];
          if (!seen_node[nd]) { seen_node[nd] = 1; touched.push_back(nd); ++distinct_nodes; }
        }
        for (i64 nd : touched) seen_node[nd] = 0;
        // distinct processors: the chain is a bijection, so distinct block
        // coordinates along the fibre are distinct processors
        prim += (i128)weight * (i64)(reps[v].size() - 1);
        sec += (i128)weight * (distinct_nodes - 1);
      }
  }
}

}  // namespace

// ====================================================================== C API

extern "C" {

// Final processor-space shape after chain + rank fix-up.  Returns 0 or 1 (invalid).
int or_final_shape(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist,
                   int b, int64_t* shape_out, int* rank_out) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  *rank_out = pl.rank;
  for (int t = 0; t < pl.rank; ++t) shape_out[t] = pl.s[t];
  return 0;
}

// Primitive list after expansion: 4 int64 per primitive [op, p, q, d]; returns count or -1.
int or_expand(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist, int b,
              int64_t* out, int cap) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return -1;
  int m = (int)pl.prims.size();
  for (int o = 0; o < m && o < cap; ++o) {
    out[4 * o + 0] = pl.prims[o].op;
    out[4 * o + 1] = pl.prims[o].p;
    out[4 * o + 2] = pl.prims[o].q;
    out[4 * o + 3] = pl.prims[o].d;
  }
  return m;
}

// Resolve final-space indices (rank r rows of `a`) to (node, proc).
int or_resolve(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist, int b,
               const int64_t* a, int64_t m, int64_t* node_out, int64_t* proc_out) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  for (int64_t e = 0; e < m; ++e) {
    i64 nd, pr;
    resolve(pl, a + e * pl.rank, nd, pr);
    node_out[e] = nd;
    proc_out[e] = pr;
  }
  return 0;
}

// ids[lin] for every point (C-order), hist[P]; either may be NULL.
int or_map_points(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist,
                  int b, int32_t* ids, uint64_t* hist, int threads) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  int T = threads < 1 ? 1 : threads;
  std::vector<std::vector<u64>> part(T, std::vector<u64>(hist ? pl.P : 0, 0));
  parallel_for(pl.npoints, T, [&](i64 lo, i64 hi, int w) {
    i64 x[4];
    for (i64 lin = lo; lin < hi; ++lin) {
      unravel(pl, lin, x);
      i64 id = owner_of_point(pl, x);
      if (ids) ids[lin] = (int32_t)id;
      if (hist) part[w][id]++;
    }
  });
  if (hist) {
    for (i64 p = 0; p < pl.P; ++p) {
      u64 s = 0;
      for (int w = 0; w < T; ++w) s += part[w][p];
      hist[p] = s;
    }
  }
  return 0;
}

// The per-point work of the hot path on the points [lo, lo + count): owner
// of the point and of each of its in-range nearest neighbours, and the
// halo bytes those neighbours send (used by the timed CPU baseline).
int or_map_range(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist, int b,
                 const uint64_t* face_bytes, int64_t lo, int64_t count, int threads,
                 int32_t* ids_out, uint64_t* halo_out) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  int T = threads < 1 ? 1 : threads;
  std::vector<u64> tot(T, 0);
  parallel_for(count, T, [&](i64 a, i64 z, int w) {
    i64 x[4], y[4];
    for (i64 e = a; e < z; ++e) {
      unravel(pl, lo + e, x);
      i64 me = owner_of_point(pl, x);
      ids_out[e] = (int32_t)me;
      for (int t = 0; t < pl.k; ++t)
        for (int delta = -1; delta <= 1; delta += 2) {
          for (int u = 0; u < pl.k; ++u) y[u] = x[u];
          y[t] += delta;
          if (y[t] < 0 || y[t] >= pl.L[t]) continue;
          if (owner_of_point(pl, y) != me) tot[w] += face_bytes[t];
        }
    }
  });
  u64 s = 0;
  for (int w = 0; w < T; ++w) s += tot[w];
  *halo_out = s;
  return 0;
}

// ids, histogram and halo of one launch: the owner of every point is
// evaluated once, as in or_map_points, and every directed pair (x, x + delta
// e_t), delta = +-1, both points inside the launch, compares the two owners
// from that array.  This is or_comm_volume's definition with the neighbour's
// owner looked up instead of evaluated again (seven owner evaluations per
// point are too slow for whole-batch checks).  ids may be NULL (kept
// internally); hist, total and recv may be NULL.
int or_map_launch(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist, int b,
                  const uint64_t* face_bytes, int32_t* ids, uint64_t* hist, uint64_t* total,
                  uint64_t* recv, int threads) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  int T = threads < 1 ? 1 : threads;
  std::vector<int32_t> own;
  if (!ids) {
    own.resize(pl.npoints);
    ids = own.data();
  }
  parallel_for(pl.npoints, T, [&](i64 lo, i64 hi, int) {
    i64 x[4];
    for (i64 lin = lo; lin < hi; ++lin) {
      unravel(pl, lin, x);
      ids[lin] = (int32_t)owner_of_point(pl, x);
    }
  });
  i64 stride[4];
  stride[pl.k - 1] = 1;
  for (int t = pl.k - 2; t >= 0; --t) stride[t] = stride[t + 1] * pl.L[t + 1];
  std::vector<u64> tot(T, 0);
  std::vector<std::vector<u64>> hpart(T), rpart(T);
  parallel_for(pl.npoints, T, [&](i64 lo, i64 hi, int w) {
    i64 x[4];
    u64 mine = 0;
    std::vector<u64> hv(hist ? pl.P : 0, 0), rv(recv ? pl.P : 0, 0);
    for (i64 lin = lo; lin < hi; ++lin) {
      const i64 me = ids[lin];
      if (hist) hv[me]++;
      unravel(pl, lin, x);
      for (int t = 0; t < pl.k; ++t)
        for (int delta = -1; delta <= 1; delta += 2) {
          const i64 y = x[t] + delta;
          if (y < 0 || y >= pl.L[t]) continue;
          if (ids[lin + delta * stride[t]] != me) {
            mine += face_bytes[t];
            if (recv) rv[me] += face_bytes[t];
          }
        }
    }
    tot[w] = mine;
    hpart[w] = std::move(hv);
    rpart[w] = std::move(rv);
  });
  if (total) {
    u64 s = 0;
    for (int w = 0; w < T; ++w) s += tot[w];
    *total = s;
  }
  for (i64 p = 0; p < pl.P; ++p) {
    u64 hs = 0, rs = 0;
    for (int w = 0; w < T; ++w) {
      if (hist && !hpart[w].empty()) hs += hpart[w][p];
      if (recv && !rpart[w].empty()) rs += rpart[w][p];
    }
    if (hist) hist[p] = hs;
    if (recv) recv[p] = rs;
  }
  return 0;
}

// Owner of each listed linear point index (C-order).
int or_owner_of(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist, int b,
                const int64_t* lins, int64_t m, int32_t* ids_out) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  i64 x[4];
  for (int64_t e = 0; e < m; ++e) {
    unravel(pl, lins[e], x);
    ids_out[e] = (int32_t)owner_of_point(pl, x);
  }
  return 0;
}

// Halo volume: every directed pair (x, x + delta e_t), delta =
// +-1, with both points inside the launch and different owners, adds
// face_bytes[t]; the receiver is the owner of x.  The neighbour's owner is
// evaluated independently for every pair.
int or_comm_volume(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist,
                   int b, const uint64_t* face_bytes, uint64_t* total, uint64_t* recv,
                   int threads) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  int T = threads < 1 ? 1 : threads;
  std::vector<u64> tot(T, 0);
  std::vector<std::vector<u64>> part(T, std::vector<u64>(recv ? pl.P : 0, 0));
  parallel_for(pl.npoints, T, [&](i64 lo, i64 hi, int w) {
    i64 x[4], y[4];
    u64 mine = 0;
    std::vector<u64> rv(recv ? pl.P : 0, 0);
    for (i64 lin = lo; lin < hi; ++lin) {
      unravel(pl, lin, x);
      i64 me = owner_of_point(pl, x);
      for (int t = 0; t < pl.k; ++t)
        for (int delta = -1; delta <= 1; delta += 2) {
          for (int u = 0; u < pl.k; ++u) y[u] = x[u];
          y[t] += delta;
          if (y[t] < 0 || y[t] >= pl.L[t]) continue;
          i64 other = owner_of_point(pl, y);
          if (other != me) {
            mine += face_bytes[t];
            if (recv) rv[me] += face_bytes[t];
          }
        }
    }
    tot[w] = mine;
    if (recv) part[w] = std::move(rv);
  });
  u64 s = 0;
  for (int w = 0; w < T; ++w) s += tot[w];
  *total = s;
  if (recv)
    for (i64 p = 0; p < pl.P; ++p) {
      u64 r = 0;
      for (int w = 0; w < T; ++w) r += part[w][p];
      recv[p] = r;
    }
  return 0;
}

// Halo volume in elements with per-dimension widths (the anisotropic halo
// of the appendix's "Generalization of the Decompose Primitive"; readings
// the element count).  A processor p that owns a point x needs every point
// y = x + delta e_t with 1 <= |delta| <= width[t] inside the launch; each
// element y it does not own is received once per dimension t along which it
// is needed, whichever of p's points need it:
//   total = sum_y sum_t bytes[t] * |{ owner(y + delta e_t) : 1 <= |delta| <= w_t,
//                                     in bounds } \ { owner(y) }|,
// and recv[p] gets bytes[t] for each such (p, y, t).
int or_halo_elements(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf, int dist,
                     int b, const int64_t* width, const uint64_t* bytes, uint64_t* total, uint64_t* recv,
                     int threads) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  for (int t = 0; t < k; ++t)
    if (width[t] < 0) return 1;
  int T = threads < 1 ? 1 : threads;
  std::vector<u64> tot(T, 0);
  std::vector<std::vector<u64>> part(T, std::vector<u64>(recv ? pl.P : 0, 0));
  parallel_for(pl.npoints, T, [&](i64 lo, i64 hi, int w) {
    i64 y[4], z[4];
    u64 mine = 0;
    std::vector<u64> rv(recv ? pl.P : 0, 0);
    std::vector<i64> seen;
    for (i64 lin = lo; lin < hi; ++lin) {
      unravel(pl, lin, y);
      const i64 me = owner_of_point(pl, y);
      for (int t = 0; t < pl.k; ++t) {
        seen.clear();
        for (i64 delta = -width[t]; delta <= width[t]; ++delta) {
          if (delta == 0) continue;
          for (int u = 0; u < pl.k; ++u) z[u] = y[u];
          z[t] += delta;
          if (z[t] < 0 || z[t] >= pl.L[t]) continue;
          const i64 p = owner_of_point(pl, z);
          if (p == me) continue;
          if (std::find(seen.begin(), seen.end(), p) == seen.end()) seen.push_back(p);
        }
        mine += bytes[t] * (u64)seen.size();
        if (recv)
          for (i64 p : seen) rv[p] += bytes[t];
      }
    }
    tot[w] = mine;
    if (recv) part[w] = std::move(rv);
  });
  u64 s = 0;
  for (int w = 0; w < T; ++w) s += tot[w];
  *total = s;
  if (recv)
    for (i64 p = 0; p < pl.P; ++p) {
      u64 r = 0;
      for (int w = 0; w < T; ++w) r += part[w][p];
      recv[p] = r;
    }
  return 0;
}

// Closed-form halo volume (derived from the surface formula of Sec. 4.2,
// Fig. 10, for the separable distributions): along dimension t the number of
// positions x_t in [0, L_t - 1) whose two sides differ in the distributed
// coordinate(s) is B_t, and every such position is a crossing for all
// prod_{u != t} L_u points, in both directions.
int or_halo_closed_form(const int64_t* L, int k, int n, int g, const int64_t* xf, int nxf,
                        int dist, int b, const uint64_t* face_bytes, uint64_t* total) {
  Plan pl;
  if (build_plan(pl, L, k, n, g, xf, nxf, dist, b)) return 1;
  u64 s = 0;
  for (int t = 0; t < k; ++t) {
    i64 Bt = 0;
    i64 Lt = pl.L[t];
    switch (dist) {
      case D_BLOCK: Bt = std::min(pl.s[t], Lt) - 1; break;
      case D_CYCLIC: Bt = pl.s[t] >= 2 ? Lt - 1 : 0; break;
      case D_BLOCK_CYCLIC: Bt = pl.s[t] >= 2 ? (Lt + b - 1) / b - 1 : 0; break;
      case D_HIER: Bt = pl.s[k + t] >= 2 ? Lt - 1 : std::min(pl.s[t], Lt) - 1; break;
      case D_LINEAR_CYCLIC: {
        i128 stride = 1;
        for (int u = t + 1; u < k; ++u) stride *= pl.L[u];
        Bt = (stride % pl.P != 0) ? Lt - 1 : 0;
        break;
      }
    }
    u64 others = 1;
    for (int u = 0; u < k; ++u)
      if (u != t) others *= (u64)pl.L[u];
    s += face_bytes[t] * 2 * (u64)Bt * others;
  }
  *total = s;
  return 0;
}

// Workload-balancing greedy of Sec. 4.3's counterexample: the primes of d
// (ascending, with multiplicity) are placed one at a time on the dimension
// that leaves the smallest spread max(w) - min(w) of the workload vector
// w_m = l_m / d_m (first dimension on ties).  Exact rational comparisons.
int or_greedy_workload(int64_t d, int k, const int64_t* l, int64_t* out) {
  if (d < 1 || k < 1 || k > 4) return 1;
  std::vector<i64> primes;
  for (auto& pe : prime_factorise(d))
    for (int e = 0; e < pe.second; ++e) primes.push_back(pe.first);
  std::vector<i64> fac(k, 1);
  // spread of w for factors f, as a fraction num/den (den > 0)
  auto spread = [&](const std::vector<i64>& f, i128& num, i128& den) {
    int imax = 0, imin = 0;   // w_a > w_b  <=>  l_a d_b > l_b d_a
    for (int m = 1; m < k; ++m) {
      if ((i128)l[m] * f[imax] > (i128)l[imax] * f[m]) imax = m;
      if ((i128)l[m] * f[imin] < (i128)l[imin] * f[m]) imin = m;
    }
    num = (i128)l[imax] * f[imin] - (i128)l[imin] * f[imax];
    den = (i128)f[imax] * f[imin];
  };
  for (i64 p : primes) {
    int bestj = -1;
    i128 bn = 0, bd = 1;
    for (int j = 0; j < k; ++j) {
      std::vector<i64> f = fac;
      f[j] *= p;
      i128 nn, dd;
      spread(f, nn, dd);
      if (bestj < 0 || nn * bd < bn * dd) { bestj = j; bn = nn; bd = dd; }
    }
    fac[bestj] *= p;
  }
  for (int m = 0; m < k; ++m) out[m] = fac[m];
  return 0;
}

// Ordered k-factorisations of d, lexicographic; writes up to cap tuples (k
// int64 each) and returns the total count.
int64_t or_factorisations(int64_t d, int k, int64_t* out, int64_t cap) {
  auto all = factorisations(d, k);
  for (int64_t e = 0; e < (int64_t)all.size() && e < cap; ++e)
    for (int m = 0; m < k; ++m) out[e * k + m] = all[e][m];
  return (int64_t)all.size();
}

int or_decompose(int64_t d, int k, const int64_t* l, int64_t* out) {
  if (d < 1 || k < 1 || k > 4) return 1;
  auto f = decompose_factors(d, k, l);
  for (int m = 0; m < k; ++m) out[m] = f[m];
  return 0;
}

// decompose with halo widths h (k values >= 1) and a transpose mask: the
// generalised objective of the appendix.  Returns 2 on objective overflow.
int or_decompose_weighted(int64_t d, int k, const int64_t* l, const int64_t* h, int tmask, int64_t* out) {
  if (d < 1 || k < 1 || k > 4 || tmask < 0 || tmask >= (1 << k)) return 1;
  for (int m = 0; m < k; ++m)
    if (l[m] < 1 || h[m] < 0) return 1;
  auto f = decompose_factors(d, k, l, h, tmask);
  if ((int)f.size() != k) return 2;
  for (int m = 0; m < k; ++m) out[m] = f[m];
  return 0;
}

// The generalised objective of one factorisation as the pair (d V, Lambda *
// sum_T (d_n - 1) d / d_n) in two int64 halves each (hi, lo) -- for tests.
int or_weighted_objective(int64_t d, int k, const int64_t* f, const int64_t* l, const int64_t* h, int tmask,
                          int64_t* out_hi_lo) {
  std::vector<i64> fv(f, f + k);
  i128 v;
  if (!weighted_objective(fv, l, h, tmask, k, d, v)) return 2;
  out_hi_lo[0] = (int64_t)(v >> 64);
  out_hi_lo[1] = (int64_t)(uint64_t)v;
  return 0;
}

// Algorithm A1: primes ascending; each goes to the currently smallest factor
// (the first index on ties); the factors are sorted descending.
int or_greedy(int64_t d, int k, int64_t* out) {
  if (d < 1 || k < 1) return 1;
  std::vector<i64> primes;
  for (auto& pe : prime_factorise(d))
    for (int e = 0; e < pe.second; ++e) primes.push_back(pe.first);
  std::vector<i64> fac(k, 1);
  for (i64 p : primes) {
    int j = 0;
    for (int m = 1; m < k; ++m)
      if (fac[m] < fac[j]) j = m;
    fac[j] *= p;
  }
  std::sort(fac.begin(), fac.end(), [](i64 a, i64 b) { return a > b; });
  for (int m = 0; m < k; ++m) out[m] = fac[m];
  return 0;
}

// Chains of depth <= max_depth on (n, g) in canonical order.  Each chain is
// written as max_depth ops of 4 int64 [op, p, q, d] (unused ops op = -1).
// Returns the total count; writes at most cap chains.
int64_t or_chains(int n, int g, int max_depth, int64_t* out, int64_t cap) {
  auto all = enum_chains(n, g, max_depth);
  for (int64_t c = 0; c < (int64_t)all.size() && c < cap; ++c)
    for (int o = 0; o < max_depth; ++o) {
      int64_t* e = out + (c * max_depth + o) * 4;
      if (o < (int)all[c].size()) {
        e[0] = all[c][o].op; e[1] = all[c][o].p; e[2] = all[c][o].q; e[3] = all[c][o].d;
      } else {
        e[0] = -1; e[1] = e[2] = e[3] = 0;
      }
    }
  return (int64_t)all.size();
}

// A chain drawn from random numbers: at each step the op is
// alphabet[draws[step] mod |alphabet|]; an empty alphabet ends the chain.
// Output: XF_W-int64 user ops.  Returns the number of ops.
int or_chain_from_draws(int n, int g, int depth, const uint64_t* draws, int64_t* xf_out) {
  Space sp;
  sp.r = 2; sp.s[0] = n; sp.s[1] = g;
  int m = 0;
  for (int step = 0; step < depth; ++step) {
    auto A = alphabet(sp);
    if (A.empty()) break;
    COp c = A[draws[step] % A.size()];
    std::vector<Prim> dummy;
    apply_cop(dummy, sp, c);
    int64_t* e = xf_out + XF_W * m;
    for (int z = 0; z < XF_W; ++z) e[z] = 0;
    e[0] = c.op;
    e[1] = c.p;
    e[2] = c.op == OP_SPLIT ? 0 : c.q;
    e[4] = c.op == OP_SPLIT ? c.d : 0;
    ++m;
  }
  return m;
}

// Matmul moved-tile cost of one candidate (chain = ops [op,p,q,d] x depth,
// op = -1 padding).  mode 0 = literal O(MNK), 1 = grouped.  Costs in tiles.
int or_matmul_cost(int64_t M, int64_t N, int64_t K, int n, int g, const int64_t* chain, int depth,
                   const int64_t* f, int mode, int64_t* primary, int64_t* secondary) {
  std::vector<COp> ch;
  for (int o = 0; o < depth; ++o) {
    const int64_t* e = chain + 4 * o;
    if (e[0] < 0) break;
    ch.push_back({(int)e[0], (int)e[1], (int)e[2], e[3]});
  }
  if (f[0] * f[1] * f[2] != (i64)n * g) return 1;
  ChainTable tb = chain_table(n, g, ch);
  i128 p, s;
  if (mode == 0) matmul_cost_literal(M, N, K, tb, f, p, s);
  else matmul_cost_grouped(block_groups(M, N, K, f), tb, f, n, p, s);
  *primary = (int64_t)p;
  *secondary = (int64_t)s;
  return 0;
}

// Exhaustive decompose search for one 3-D matmul query:
// candidates are (factorisation f of P into 3, chain c of depth <= max_depth
// on (P/g, g)), index = f_rank * n_chains + c_rank; the winner minimises
// (primary, secondary, index) lexicographically.  Costs are in tiles.
// out: [index, f0, f1, f2, c_rank, primary, secondary, n_candidates]
int or_search(int64_t M, int64_t N, int64_t K, int n, int g, int max_depth, int threads,
              int64_t* out) {
  auto fs = factorisations((i64)n * g, 3);
  auto chains = enum_chains(n, g, max_depth);
  i64 NC = (i64)chains.size();
  int T = threads < 1 ? 1 : threads;
  std::vector<BlockGroups> bgs(fs.size());
  parallel_for((i64)fs.size(), T, [&](i64 lo, i64 hi, int) {
    for (i64 fr = lo; fr < hi; ++fr) bgs[fr] = block_groups(M, N, K, fs[fr].data());
  }, 2);
  struct Best { i128 p, s; i64 idx; };
  std::vector<Best> best(T, Best{-1, -1, -1});
  parallel_for(NC, T, [&](i64 lo, i64 hi, int w) {
    for (i64 c = lo; c < hi; ++c) {
      ChainTable tb = chain_table(n, g, chains[c]);
      for (i64 fr = 0; fr < (i64)fs.size(); ++fr) {
        i128 p, s;
        matmul_cost_grouped(bgs[fr], tb, fs[fr].data(), n, p, s);
        i64 idx = fr * NC + c;
        Best& b = best[w];
        if (b.idx < 0 || p < b.p || (p == b.p && (s < b.s || (s == b.s && idx < b.idx))))
          b = Best{p, s, idx};
      }
    }
  }, 2);
  Best b = best[0];
  for (int w = 1; w < T; ++w) {
    const Best& o = best[w];
    if (o.idx < 0) continue;
    if (b.idx < 0 || o.p < b.p || (o.p == b.p && (o.s < b.s || (o.s == b.s && o.idx < b.idx)))) b = o;
  }
  i64 fr = b.idx / NC, c = b.idx % NC;
  out[0] = b.idx;
  out[1] = fs[fr][0]; out[2] = fs[fr][1]; out[3] = fs[fr][2];
  out[4] = c;
  out[5] = (int64_t)b.p;
  out[6] = (int64_t)b.s;
  out[7] = (int64_t)fs.size() * NC;
  return 0;
}

// ------------------------------------------------------------ hierarchical search
//
// Two-level mappings of a k-D launch on Machine(GPU) = (n, g):
// the node dimension split into a node grid a (prod a = n), the GPU dimension
// into a GPU grid b (prod b = g).  Node coordinate u_t = floor(x_t a_t / L_t)
// in both variants; GPU coordinate
//   variant 0 (block within the node, the Solomonik mapper of Fig. 5b):
//             v_t = floor(x_t a_t b_t / L_t) mod b_t
//   variant 1 (cyclic within the node, the Cannon mapper of Appendix A.1):
//             v_t = x_t mod b_t.
// Node index u_0 + a_0 (u_1 + a_1 (...)), GPU index v_0 + b_0 (v_1 + ...)
// (the split formula of Fig. 4, first factor fastest); id = node * g + gpu.
// Candidates: a over the ordered k-factorisations of n, b over those of g,
// both lexicographic; index = rank(a) * |F(g)| + rank(b).  Costs: primary =
// the element halo volume (as or_halo_elements) between nodes, secondary = the same
// between processors; the winner minimises (primary, secondary, index).

namespace {

struct Hier {
  int k;
  i64 L[4], a[4], b[4];
  int variant;
  int g;
};

void hier_owner(const Hier& h, const i64* x, i64& node, i64& proc) {
  i64 nd = 0, gp = 0, sa = 1, sb = 1;
  for (int t = 0; t < h.k; ++t) {
    const i64 u = (i64)((i128)x[t] * h.a[t] / h.L[t]);
    const i64 v = h.variant == 0 ? (i64)(((i128)x[t] * h.a[t] * h.b[t] / h.L[t]) % h.b[t]) : x[t] % h.b[t];
    nd += u * sa;
    gp += v * sb;
    sa *= h.a[t];
    sb *= h.b[t];
  }
  node = nd;
  proc = nd * h.g + gp;
}

// element halo volumes (node level, processor level) by brute force
void hier_costs(const Hier& h, const i64* width, const u64* bytes, int threads, u64& prim, u64& sec) {
  i64 N = 1;
  for (int t = 0; t < h.k; ++t) N *= h.L[t];
  int T = threads < 1 ? 1 : threads;
  std::vector<u64> pp(T, 0), ss(T, 0);
  parallel_for(N, T, [&](i64 lo, i64 hi, int w) {
    i64 y[4], z[4];
    std::vector<i64> sn, sp;
    for (i64 lin = lo; lin < hi; ++lin) {
      i64 rest = lin;
      for (int t = h.k - 1; t >= 0; --t) {
        y[t] = rest % h.L[t];
        rest /= h.L[t];
      }
      i64 n0, p0;
      hier_owner(h, y, n0, p0);
      for (int t = 0; t < h.k; ++t) {
        sn.clear();
        sp.clear();
        for (i64 d = -width[t]; d <= width[t]; ++d) {
          if (d == 0) continue;
          for (int u = 0; u < h.k; ++u) z[u] = y[u];
          z[t] += d;
          if (z[t] < 0 || z[t] >= h.L[t]) continue;
          i64 n1, p1;
          hier_owner(h, z, n1, p1);
          if (n1 != n0 && std::find(sn.begin(), sn.end(), n1) == sn.end()) sn.push_back(n1);
          if (p1 != p0 && std::find(sp.begin(), sp.end(), p1) == sp.end()) sp.push_back(p1);
        }
        pp[w] += bytes[t] * (u64)sn.size();
        ss[w] += bytes[t] * (u64)sp.size();
      }
    }
  });
  prim = sec = 0;
  for (int w = 0; w < T; ++w) {
    prim += pp[w];
    sec += ss[w];
  }
}

}  // namespace

// Costs of one hierarchical candidate (a, b).
int or_hier_costs(const int64_t* L, int k, int n, int g, const int64_t* a, const int64_t* b, int variant,
                  const int64_t* width, const uint64_t* bytes, int threads, uint64_t* primary, uint64_t* secondary) {
  if (k < 1 || k > 4 || n < 1 || g < 1 || variant < 0 || variant > 1) return 1;
  Hier h;
  h.k = k;
  h.variant = variant;
  h.g = g;
  i64 pa = 1, pb = 1;
  for (int t = 0; t < k; ++t) {
    if (L[t] < 1 || a[t] < 1 || b[t] < 1 || width[t] < 0) return 1;
    h.L[t] = L[t];
    h.a[t] = a[t];
    h.b[t] = b[t];
    pa *= a[t];
    pb *= b[t];
  }
  if (pa != n || pb != g) return 1;
  u64 p, s;
  hier_costs(h, width, bytes, threads, p, s);
  *primary = p;
  *secondary = s;
  return 0;
}

// Exhaustive hierarchical search.  out: [index, a0..a3, b0..b3, primary,
// secondary, n_candidates]
int or_hier_search(const int64_t* L, int k, int n, int g, int variant, const int64_t* width,
                   const uint64_t* bytes, int threads, int64_t* out) {
  if (k < 1 || k > 4 || n < 1 || g < 1 || variant < 0 || variant > 1) return 1;
  auto fa = factorisations(n, k);
  auto fb = factorisations(g, k);
  i64 best = -1;
  u64 bp = 0, bs = 0;
  for (size_t i = 0; i < fa.size(); ++i)
    for (size_t j = 0; j < fb.size(); ++j) {
      u64 p, s;
      if (or_hier_costs(L, k, n, g, fa[i].data(), fb[j].data(), variant, width, bytes, threads, &p, &s)) return 1;
      const i64 idx = (i64)(i * fb.size() + j);
      if (best < 0 || p < bp || (p == bp && s < bs)) {   // ties keep the lower index
        best = idx;
        bp = p;
        bs = s;
      }
    }
  const i64 i = best / (i64)fb.size(), j = best % (i64)fb.size();
  out[0] = best;
  for (int t = 0; t < 4; ++t) {
    out[1 + t] = t < k ? fa[i][t] : 0;
    out[5 + t] = t < k ? fb[j][t] : 0;
  }
  out[9] = (int64_t)bp;
  out[10] = (int64_t)bs;
  out[11] = (int64_t)(fa.size() * fb.size());
  return 0;
}

// Cost of an explicit list of candidate indices (for sampled checks).
int or_candidate_costs(int64_t M, int64_t N, int64_t K, int n, int g, int max_depth,
                       const int64_t* idx, int64_t m, int64_t* primary, int64_t* secondary,
                       int threads) {
  auto fs = factorisations((i64)n * g, 3);
  auto chains = enum_chains(n, g, max_depth);
  i64 NC = (i64)chains.size();
  std::vector<BlockGroups> bgs(fs.size());
  std::vector<char> have(fs.size(), 0);
  for (int64_t e = 0; e < m; ++e) {
    if (idx[e] < 0 || idx[e] / NC >= (i64)fs.size()) return 1;
    i64 fr = idx[e] / NC;
    if (!have[fr]) { bgs[fr] = block_groups(M, N, K, fs[fr].data()); have[fr] = 1; }
  }
  parallel_for(m, threads < 1 ? 1 : threads, [&](i64 lo, i64 hi, int) {
    for (i64 e = lo; e < hi; ++e) {
      i64 fr = idx[e] / NC, c = idx[e] % NC;
      ChainTable tb = chain_table(n, g, chains[c]);
      i128 p, s;
      matmul_cost_grouped(bgs[fr], tb, fs[fr].data(), n, p, s);
      primary[e] = (int64_t)p;
      secondary[e] = (int64_t)s;
    }
  }, 64);
  return 0;
}

}  // extern "C"
