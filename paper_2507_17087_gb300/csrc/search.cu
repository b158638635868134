// decompose_search: exhaustive argmin over (factorisation, chain) candidates
// for a 3-D matmul tile grid, and exact costs of listed candidates.
//
// Candidate (c, f): chain c over the canonical alphabet applied to
// Machine(GPU) = (n, g); the result is flattened with merge(0, 1) and split
// as f = (f0, f1, f2) with dimension 0 fastest (the splits decompose expands
// into, Sec. 4.2); tile (i, j, k) is block-mapped to a = (floor(i f0 / M),
// floor(j f1 / N), floor(k f2 / K)) and owned by the processor the chain
// resolves flat(a) = a0 + f0 (a1 + f1 a2) to.  The owner of a flat index does
// not depend on f, so each CTA tabulates node(b) for its chain once, in
// shared memory, and every thread then scores one factorisation at a time.
//
// Cost (in tiles): for each operand tile A(i,k), B(k,j), C(i,j) the number of
// distinct processors (primary) and nodes (secondary) among the points that
// touch it, minus one.  Tiles whose two fixed coordinates fall in the same
// pair of blocks touch the same owners, so one fibre per block pair is
// scanned and weighted by the tiles in it.  Distinct processors along a fibre
// equal distinct block coordinates (the chain is a bijection), which gives
// the primary in closed form: sum_v (min(E_v, f_v) - 1) E_u E_w.
#include <algorithm>
#include <array>
#include <cstring>
#include <mutex>

#include "search.cuh"

namespace mp {

namespace {

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// One CTA per chain; warp w scores factorisations w, w + W, ... with its 32
// lanes sharing each candidate's fibre scans.
// full = 1: every candidate's secondary is scanned.  full = 0: candidates
// whose (exact, closed-form) primary exceeds the minimum primary over all
// factorisations cannot win the lexicographic argmin and are not scanned.
// PRE: the precounted fibre tables (full search; one byte per fibre).  The
// full search runs three CTAs per SM at 80 registers (faster than four at 64,
// which spill); the primary-bound search, with few candidates per CTA, four.
template <bool PRE>
__global__ void __launch_bounds__(256, PRE ? 3 : 4) k_search(const ChainProg* __restrict__ progs, const Fact* __restrict__ facts, int nf,
                         uint32_t P, uint32_t E0, uint32_t E1, uint32_t E2, int words,
                         unsigned long long nchains, int full, unsigned long long ub,
                         const uint8_t* __restrict__ skip, const uint16_t* __restrict__ gtab, uint32_t Pp,
                         int npre, const uint32_t* __restrict__ pre_list, Key* __restrict__ chain_best) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Key red[32];
  __shared__ uint32_t s_pdiv[kPreMaxN], s_pm[kPreMaxN], s_poff[kPreMaxN + 1];
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw);
  uint16_t* tab = reinterpret_cast<uint16_t*>(smem_raw + (size_t)words * blockDim.x * 4);
  // npre > 0: after the table, the precounted fibre counts of every divisor
  // d = s_pdiv[k] <= kPreMaxDiv: the P / d blocks of d consecutive flat
  // indices at s_poff[k], then the P / d residue classes modulo P / d
  uint8_t* dtab = reinterpret_cast<uint8_t*>(smem_raw + (size_t)words * blockDim.x * 4 + (((size_t)P * 2 + 255) & ~(size_t)255));
  const uint32_t c = blockIdx.x;
  __shared__ ChainProg cp;
  if (threadIdx.x == 0) cp = progs[c];
  for (int i = threadIdx.x; i < npre; i += blockDim.x) {
    s_pdiv[i] = pre_list[i];
    s_pm[i] = pre_list[npre + i];
  }
  for (int i = threadIdx.x; i <= npre; i += blockDim.x) s_poff[i] = pre_list[2 * npre + i];
  for (int w = 0; w < words; ++w) bm[w * blockDim.x + threadIdx.x] = 0;
  __syncthreads();
  if (gtab) load_table(gtab + (size_t)c * Pp, tab, Pp);
  else build_table(cp, tab, P);
  __syncthreads();
  if (PRE && npre > 0) {
    const uint32_t nitems = s_poff[npre];
    for (uint32_t i = threadIdx.x; i < nitems; i += blockDim.x) {
      int lo = 0, hi = npre;   // s_poff[lo] <= i < s_poff[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_poff[mid] <= i) lo = mid;
        else hi = mid;
      }
      const uint32_t d = s_pdiv[lo], m = s_pm[lo], local = i - s_poff[lo];
      const bool blk = local < m;
      const uint32_t base = blk ? local * d : local - m, stride = blk ? 1u : m;
      dtab[i] = (uint8_t)(fibre_distinct(tab, bm + threadIdx.x, blockDim.x, words, base, stride, d, d, d) - 1);
    }
    __syncthreads();
  }
  // the precounted table of divisor v (null when v is not precounted)
  auto pre_of = [&](uint32_t v, bool res) -> const uint8_t* {
    if (!PRE || npre == 0 || v > kPreMaxDiv) return nullptr;
    int lo = 0, hi = npre;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_pdiv[mid] <= v) lo = mid;
      else hi = mid;
    }
    if (s_pdiv[lo] != v) return nullptr;
    return dtab + s_poff[lo] + (res ? s_pm[lo] : 0u);
  };
  const uint32_t E[3] = {E0, E1, E2};
  unsigned long long pmin = 0;
  if (!full) {
    Key m{~0ull, 0, 0};
    for (int fr = threadIdx.x; fr < nf; fr += blockDim.x) {
      const uint32_t f[3] = {facts[fr].f[0], facts[fr].f[1], facts[fr].f[2]};
      const unsigned long long p = primary_cost(E, f);
      if (p < m.p) m.p = p;
    }
    block_argmin(m, red);
    __shared__ unsigned long long s_pmin;
    if (threadIdx.x == 0) s_pmin = m.p;
    __syncthreads();
    pmin = s_pmin;
  }
  Key best{~0ull, ~0ull, ~0ull};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  uint32_t* wbm = bm + warp * 32;   // this warp's 32 bitmap columns
  for (int fr = warp; fr < nf; fr += nwarps) {
    const uint32_t f[3] = {facts[fr].f[0], facts[fr].f[1], facts[fr].f[2]};
    Key k;
    k.p = primary_cost(E, f);
    if (!full && k.p > pmin) continue;   // uniform across the warp
    if (skip && skip[fr]) continue;
    // families 0 and 2 from the precounted fibres where every block holds tiles
    const uint8_t* pre0 = E[0] >= f[0] ? pre_of(f[0], false) : nullptr;
    const uint8_t* pre2 = E[2] >= f[2] ? pre_of(f[2], true) : nullptr;
    k.s = secondary_cost_warp<!PRE>(tab, wbm, blockDim.x, words, E, f, lane, ub, pre0, pre2);
    k.idx = (unsigned long long)fr * nchains + c;
    if (key_less(k, best)) best = k;
  }
  block_argmin(best, red);
  if (threadIdx.x == 0) chain_best[c] = best;
}

// Every chain's node table (one CTA per chain), for the space's device copy.
__global__ void k_node_tables(const ChainProg* __restrict__ progs, uint32_t P, uint32_t Pp, uint16_t* __restrict__ tab) {
  __shared__ ChainProg cp;
  if (threadIdx.x == 0) cp = progs[blockIdx.x];
  __syncthreads();
  uint16_t* row = tab + (size_t)blockIdx.x * Pp;
  for (uint32_t b = threadIdx.x; b < Pp; b += blockDim.x) row[b] = b < P ? (uint16_t)resolve_node(cp, b) : (uint16_t)0;
}

__global__ void k_search_final(const Key* __restrict__ chain_best, unsigned long long n, Key* __restrict__ out) {
  __shared__ Key red[32];
  Key best{~0ull, ~0ull, ~0ull};
  for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) {
    const Key k = chain_best[i];
    if (key_less(k, best)) best = k;
  }
  block_argmin(best, red);
  if (threadIdx.x == 0) *out = best;
}

// One CTA per listed candidate: the chain's table in shared memory, the
// fibres of the three families spread over the threads.
__global__ void k_candidate_costs(const ChainProg* __restrict__ progs, const Fact* __restrict__ facts, int nf,
                                  const int64_t* __restrict__ idx, unsigned long long nchains, uint32_t P,
                                  uint32_t E0, uint32_t E1, uint32_t E2, int words,
                                  unsigned long long tile_bytes, const uint16_t* __restrict__ gtab, uint32_t Pp,
                                  uint64_t* __restrict__ prim_out, uint64_t* __restrict__ sec_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ChainProg cp;
  __shared__ unsigned long long red[32];
  const unsigned long long id = (unsigned long long)idx[blockIdx.x];
  if (idx[blockIdx.x] < 0 || id >= nchains * (unsigned long long)nf) {   // out of range: flag, no access
    if (threadIdx.x == 0) {
      prim_out[blockIdx.x] = ~0ull;
      sec_out[blockIdx.x] = ~0ull;
    }
    return;
  }
  const unsigned long long fr = id / nchains, c = id % nchains;
  const uint32_t E[3] = {E0, E1, E2};
  const unsigned long long s = candidate_secondary_block(progs, facts, fr, c, P, E, words, gtab, Pp, smem_raw, cp, red);
  if (threadIdx.x == 0) {
    const uint32_t f[3] = {facts[fr].f[0], facts[fr].f[1], facts[fr].f[2]};
    prim_out[blockIdx.x] = primary_cost(E, f) * tile_bytes;
    sec_out[blockIdx.x] = s * tile_bytes;
  }
}

}  // namespace

// The resolution program of chain c: the chain's primitives, then the
// flattening merges, with the shapes each one was applied to.
ChainProg compile_chain(int64_t n, int64_t g, const std::vector<CanonOp>& ch) {
  ChainProg cp;
  std::memset(&cp, 0, sizeof(cp));
  std::vector<int64_t> shape = {n, g};
  auto push = [&](int op, int p, int q, int64_t d) {
    Prim& pr = cp.prim[cp.nprim++];
    pr.op = op;
    pr.p = p;
    pr.q = q;
    pr.rank_before = (int32_t)shape.size();
    if (op == P_SPLIT) {
      pr.d = (uint32_t)d;
    } else if (op == P_MERGE) {
      pr.d = (uint32_t)shape[p];
      pr.div = make_div32(pr.d);
    }
  };
  for (const CanonOp& c : ch) {
    push(c.op, c.p, c.q, c.d);
    apply_canon(shape, c);
  }
  cp.depth = cp.nprim;
  while (shape.size() > 1) {
    push(P_MERGE, 0, 1, 0);
    shape[0] *= shape[1];
    shape.erase(shape.begin() + 1);
  }
  return cp;
}

int validate_query(const mp_search_query& q) {
  if (q.M < 1 || q.N < 1 || q.K < 1 || q.M > (1 << 20) || q.N > (1 << 20) || q.K > (1 << 20)) return MP_EINVAL;
  if (q.procs < 1 || q.procs_per_node < 1 || q.procs % q.procs_per_node) return MP_EINVAL;
  if (q.max_depth < 0 || q.max_depth > 4) return MP_EINVAL;
  if (q.procs > kSearchMaxProcs) return MP_ENOTSUP;
  const unsigned __int128 worst = ((unsigned __int128)q.M * q.K + (unsigned __int128)q.K * q.N +
                                   (unsigned __int128)q.M * q.N) * (uint64_t)q.procs * q.tile_bytes;
  if (worst >> 64) return MP_EOVERFLOW;
  return MP_OK;
}

namespace {

// Recently used candidate spaces, most recent first.  Building one enumerates
// every chain of the depth bound and compiles it (milliseconds for thousands
// of chains); a deployment queries the same machine over and over.
constexpr size_t kSpaceCache = 8;
std::mutex g_space_mu;
std::vector<std::pair<std::array<int64_t, 3>, std::shared_ptr<const SpaceCore>>> g_spaces;

std::shared_ptr<const SpaceCore> space_core(int64_t procs, int64_t g, int depth) {
  const std::array<int64_t, 3> key{procs, g, depth};
  {
    std::lock_guard<std::mutex> lk(g_space_mu);
    for (size_t i = 0; i < g_spaces.size(); ++i)
      if (g_spaces[i].first == key) {
        auto hit = g_spaces[i];
        g_spaces.erase(g_spaces.begin() + (long)i);
        g_spaces.insert(g_spaces.begin(), hit);
        return hit.second;
      }
  }
  auto core = std::make_shared<SpaceCore>();
  core->P = procs;
  const int64_t n = procs / g;
  core->facts = ordered_factorisations(procs, 3);
  core->chains = canonical_chains(n, g, depth);
  core->progs.resize(core->chains.size());
  for (size_t c = 0; c < core->chains.size(); ++c) core->progs[c] = compile_chain(n, g, core->chains[c]);
  core->fdev.resize(core->facts.size());
  for (size_t i = 0; i < core->facts.size(); ++i)
    for (int t = 0; t < 3; ++t) core->fdev[i].f[t] = (uint32_t)core->facts[i][t];
  std::lock_guard<std::mutex> lk(g_space_mu);
  g_spaces.insert(g_spaces.begin(), {key, core});
  if (g_spaces.size() > kSpaceCache) g_spaces.pop_back();
  return core;
}

}  // namespace

int prepare(const mp_search_query& q, SearchSpace& S) {
  const int64_t n = q.procs / q.procs_per_node;
  S.c = space_core(q.procs, q.procs_per_node, q.max_depth);
  S.words = (int)((n + 31) / 32);
  const size_t tab = align_up((size_t)q.procs * 2);
  int threads = 256;
  while (threads > 32 && tab + (size_t)S.words * 4 * threads > (size_t)kSmemBudget) threads -= 32;
  if (tab + (size_t)S.words * 4 * threads > (size_t)kSmemBudget) return MP_ENOTSUP;
  S.threads = threads;
  S.smem = (size_t)S.words * 4 * threads + tab;
  return MP_OK;
}

SpaceCore::~SpaceCore() {
  // cudaFree waits for the device, so no kernel still reads these
  if (dev.progs) cudaFree(dev.progs);
  if (dev.tab) cudaFree(dev.tab);
}

int device_space(const SpaceCore& c, cudaStream_t st, const DeviceSpace** out) {
  int device = 0;
  MP_CUDA_TRY(cudaGetDevice(&device));
  std::lock_guard<std::mutex> lk(c.dev_mu);
  DeviceSpace& D = c.dev;
  if (D.progs) {
    if (D.device != device) return MP_ENOTSUP;
    *out = &D;
    return MP_OK;
  }
  const size_t NC = c.progs.size(), NF = c.fdev.size();
  const size_t pb = align_up(NC * sizeof(ChainProg)), fb = align_up(NF * sizeof(Fact));
  char* mem = nullptr;
  if (cudaMalloc(&mem, pb + fb) != cudaSuccess) {
    cudaGetLastError();
    return MP_ENOMEM;
  }
  const uint32_t Pp = (uint32_t)((c.P + 7) & ~int64_t(7));
  uint16_t* tab = nullptr;
  if (NC * Pp * 2 <= kNodeTableCacheBytes && cudaMalloc(&tab, NC * Pp * 2) != cudaSuccess) {
    cudaGetLastError();
    tab = nullptr;   // the kernels build each chain's table themselves
  }
  bool ok = cudaMemcpyAsync(mem, c.progs.data(), NC * sizeof(ChainProg), cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(mem + pb, c.fdev.data(), NF * sizeof(Fact), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && tab && NC) {
    k_node_tables<<<(unsigned)NC, 256, 0, st>>>((const ChainProg*)mem, (uint32_t)c.P, Pp, tab);
    count_launch();
    ok = cudaGetLastError() == cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(mem);
    if (tab) cudaFree(tab);
    return MP_ECUDA;
  }
  D.progs = (ChainProg*)mem;
  D.facts = (Fact*)(mem + pb);
  D.tab = tab;
  D.Pp = Pp;
  D.device = device;
  *out = &D;
  return MP_OK;
}

namespace {

void fill_result(const mp_search_query& q, const SearchSpace& S, const Key& k, mp_search_result& r) {
  std::memset(&r, 0, sizeof(r));
  const uint64_t NC = S.c->chains.size();
  r.index = (int64_t)k.idx;
  const uint64_t fr = k.idx / NC, c = k.idx % NC;
  for (int t = 0; t < 3; ++t) r.f[t] = S.c->facts[fr][t];
  r.chain_rank = (int64_t)c;
  r.chain_len = (int32_t)S.c->chains[c].size();
  for (int o = 0; o < r.chain_len; ++o) {
    const CanonOp& op = S.c->chains[c][o];
    mp_xform& x = r.chain[o];
    x.op = op.op == P_SPLIT ? MP_SPLIT : (op.op == P_MERGE ? MP_MERGE : MP_SWAP);
    x.i = op.p;
    x.j = op.op == P_SPLIT ? 0 : op.q;
    x.d = op.op == P_SPLIT ? op.d : 0;
  }
  r.primary_bytes = k.p * q.tile_bytes;
  r.secondary_bytes = k.s * q.tile_bytes;
  r.n_chains = (int64_t)NC;
  r.n_factorisations = (int64_t)S.c->facts.size();
  r.n_candidates = r.n_chains * r.n_factorisations;
}

}  // namespace

int exhaustive_search(const mp_search_query& q, mp_search_result* out, cudaStream_t st,
                      unsigned long long ub_secondary, const std::vector<uint8_t>* skip) {
  SearchSpace S;
  int rc = prepare(q, S);
  if (rc) return rc;
  const uint64_t NC = S.c->chains.size(), NF = S.c->facts.size();
  if (skip && skip->size() != NF) return MP_EINVAL;
  const DeviceSpace* D = nullptr;
  if ((rc = device_space(*S.c, st, &D))) return rc;
  // full search: the fibre counts of families 0 and 2 precounted per chain
  // for the divisors up to kPreMaxDiv, when they fit in shared memory
  std::vector<uint32_t> pre;
  int npre = 0;
  size_t smem = S.smem;
  if (q.flags & MP_SEARCH_FULL) {
    std::vector<uint32_t> dv, mv, ov(1, 0);
    for (uint32_t d = 1; d <= (uint32_t)q.procs && d <= kPreMaxDiv; ++d)
      if (q.procs % d == 0) {
        dv.push_back(d);
        mv.push_back((uint32_t)q.procs / d);
        ov.push_back(ov.back() + 2 * ((uint32_t)q.procs / d));
      }
    const size_t need = S.smem + align_up((size_t)ov.back());
    if ((int)dv.size() <= kPreMaxN && need <= (size_t)kSmemBudget) {
      npre = (int)dv.size();
      smem = need;
      pre.insert(pre.end(), dv.begin(), dv.end());
      pre.insert(pre.end(), mv.begin(), mv.end());
      pre.insert(pre.end(), ov.begin(), ov.end());
    }
  }
  const size_t best_bytes = align_up(NC * sizeof(Key)) + align_up(sizeof(Key)) + align_up(NF) + align_up(pre.size() * 4 + 4);
  char* rest = (char*)workspace(best_bytes, 2);
  if (!rest) return MP_ENOMEM;
  uint32_t* d_pre = (uint32_t*)(rest + align_up(NC * sizeof(Key)) + align_up(sizeof(Key)) + align_up(NF));
  if (npre) MP_CUDA_TRY(cudaMemcpyAsync(d_pre, pre.data(), pre.size() * 4, cudaMemcpyHostToDevice, st));
  Key* chain_best = (Key*)rest;
  Key* d_out = (Key*)(rest + align_up(NC * sizeof(Key)));
  uint8_t* d_skip = nullptr;
  if (skip) {
    d_skip = (uint8_t*)(rest + align_up(NC * sizeof(Key)) + align_up(sizeof(Key)));
    MP_CUDA_TRY(cudaMemcpyAsync(d_skip, skip->data(), NF, cudaMemcpyHostToDevice, st));
  }
  const void* kern = npre ? (const void*)k_search<true> : (const void*)k_search<false>;
  // the opt-in also covers dynamic memory just under 48 KB that the kernel's
  // static shared memory takes past it
  if (smem > 32 * 1024)
    MP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  auto launch = npre ? k_search<true> : k_search<false>;
  launch<<<(unsigned)NC, S.threads, smem, st>>>(D->progs, D->facts, (int)S.c->facts.size(), (uint32_t)q.procs,
                                                    (uint32_t)q.M, (uint32_t)q.N, (uint32_t)q.K, S.words, NC,
                                                    (q.flags & MP_SEARCH_FULL) ? 1 : 0,
                                                    (q.flags & MP_SEARCH_FULL) ? ~0ull : ub_secondary,
                                                    (q.flags & MP_SEARCH_FULL) ? nullptr : d_skip, D->tab, D->Pp,
                                                    npre, d_pre, chain_best);
  count_launch();
  k_search_final<<<1, 1024, 0, st>>>(chain_best, NC, d_out);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  Key best;
  MP_CUDA_TRY(cudaMemcpyAsync(&best, d_out, sizeof(Key), cudaMemcpyDeviceToHost, st));
  MP_CUDA_TRY(cudaStreamSynchronize(st));
  fill_result(q, S, best, *out);
  return MP_OK;
}

int candidate_costs_dev(const mp_search_query& q, const SearchSpace& S, const DeviceSpace& D, const int64_t* d_idx,
                        int64_t n, uint64_t* d_p, uint64_t* d_s, cudaStream_t st) {
  if (n <= 0) return MP_OK;
  if (S.smem > 40 * 1024)   // opt in with room for static shared memory
    MP_CUDA_TRY(cudaFuncSetAttribute(k_candidate_costs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem));
  k_candidate_costs<<<(unsigned)n, S.threads, S.smem, st>>>(D.progs, D.facts, (int)S.c->facts.size(), d_idx,
                                                             (unsigned long long)S.c->chains.size(), (uint32_t)q.procs,
                                                             (uint32_t)q.M, (uint32_t)q.N, (uint32_t)q.K, S.words,
                                                             q.tile_bytes, D.tab, D.Pp, d_p, d_s);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  return MP_OK;
}

}  // namespace mp

extern "C" int mp_decompose_search(const mp_search_query* queries, int n_queries, mp_search_result* out,
                                   void* stream) {
  using namespace mp;
  if (n_queries < 0 || (n_queries > 0 && (!queries || !out))) return MP_EINVAL;
  for (int i = 0; i < n_queries; ++i) {
    int rc = validate_query(queries[i]);
    if (rc) return rc;
  }
  for (int i = 0; i < n_queries; ++i) {
    int rc = exhaustive_search(queries[i], &out[i], (cudaStream_t)stream);
    if (rc) return rc;
  }
  return MP_OK;
}

extern "C" int mp_candidate_costs(const mp_search_query* query, const int64_t* indices, int64_t n,
                                  uint64_t* primary, uint64_t* secondary, void* stream) {
  using namespace mp;
  if (!query || n < 0 || (n > 0 && (!indices || !primary || !secondary))) return MP_EINVAL;
  int rc = validate_query(*query);
  if (rc) return rc;
  if (n == 0) return MP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SearchSpace S;
  rc = prepare(*query, S);
  if (rc) return rc;
  const uint64_t NC = S.c->chains.size(), NF = S.c->facts.size();
  const bool idx_dev = is_device_pointer(indices);
  const bool p_dev = is_device_pointer(primary), s_dev = is_device_pointer(secondary);
  std::vector<int64_t> host_idx;
  if (!idx_dev) {
    host_idx.assign(indices, indices + n);
    for (int64_t v : host_idx)
      if (v < 0 || (uint64_t)v >= NC * NF) return MP_EINVAL;
  }
  const size_t ib = align_up((size_t)n * 8);
  const DeviceSpace* D = nullptr;
  if ((rc = device_space(*S.c, st, &D))) return rc;
  char* rest = (char*)workspace(3 * ib, 3);
  if (!rest) return MP_ENOMEM;
  int64_t* d_idx = idx_dev ? (int64_t*)indices : (int64_t*)rest;
  uint64_t* d_p = p_dev ? primary : (uint64_t*)(rest + ib);
  uint64_t* d_s = s_dev ? secondary : (uint64_t*)(rest + 2 * ib);
  if (!idx_dev) MP_CUDA_TRY(cudaMemcpyAsync(d_idx, host_idx.data(), n * 8, cudaMemcpyHostToDevice, st));
  if (S.smem > 40 * 1024)   // opt in with room for static shared memory
    MP_CUDA_TRY(cudaFuncSetAttribute(k_candidate_costs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem));
  k_candidate_costs<<<(unsigned)n, S.threads, S.smem, st>>>(D->progs, D->facts, (int)NF, d_idx, NC,
                                                             (uint32_t)query->procs, (uint32_t)query->M,
                                                             (uint32_t)query->N, (uint32_t)query->K, S.words,
                                                             query->tile_bytes, D->tab, D->Pp, d_p, d_s);
  count_launch();
  MP_CUDA_TRY(cudaGetLastError());
  if (!p_dev) MP_CUDA_TRY(cudaMemcpyAsync(primary, d_p, n * 8, cudaMemcpyDeviceToHost, st));
  if (!s_dev) MP_CUDA_TRY(cudaMemcpyAsync(secondary, d_s, n * 8, cudaMemcpyDeviceToHost, st));
  if (!p_dev || !s_dev) MP_CUDA_TRY(cudaStreamSynchronize(st));
  return MP_OK;
}

extern "C" int mp_search_candidate(const mp_search_query* query, int64_t index, int64_t* f, mp_xform* chain,
                                   int32_t* chain_len) {
  using namespace mp;
  if (!query || !f || !chain || !chain_len) return MP_EINVAL;
  int rc = validate_query(*query);
  if (rc) return rc;
  const int64_t n = query->procs / query->procs_per_node, g = query->procs_per_node;
  auto facts = ordered_factorisations(query->procs, 3);
  auto chains = canonical_chains(n, g, query->max_depth);
  const int64_t NC = (int64_t)chains.size();
  if (index < 0 || index >= NC * (int64_t)facts.size()) return MP_EINVAL;
  const int64_t fr = index / NC, c = index % NC;
  for (int t = 0; t < 3; ++t) f[t] = facts[fr][t];
  *chain_len = (int32_t)chains[c].size();
  for (int o = 0; o < *chain_len; ++o) {
    const CanonOp& op = chains[c][o];
    mp_xform& x = chain[o];
    std::memset(&x, 0, sizeof(x));
    x.op = op.op == P_SPLIT ? MP_SPLIT : (op.op == P_MERGE ? MP_MERGE : MP_SWAP);
    x.i = op.p;
    x.j = op.op == P_SPLIT ? 0 : op.q;
    x.d = op.op == P_SPLIT ? op.d : 0;
  }
  return MP_OK;
}

// ------------------------------------------------------------ secondary lower bound
//
// Every node owns g cells of the f0 x f1 x f2 block grid (the chain is a
// bijection).  For fibre family v (lines along v), sum over fibres of
// (distinct nodes - 1) x tiles per fibre >= w_v (sum over nodes of the number
// of v-lines the node's cells meet - number of v-lines), with w_v the
// smallest tile count of a v-fibre (floor(E_u / f_u) floor(E_w / f_w)).  The
// lines a cell set meets along v are its projection along v, and pushing
// the set towards the origin along any axis keeps that axis' projection and
// shrinks the other two (a line's count becomes the longest run over the
// merged lines), so the least weighted projection sum of g cells is reached
// by a down-set: heights h[i][j] non-increasing in i and j, summing to g.
// Its projections are sum_j h[0][j] (along dim 0), sum_i h[i][0] (dim 1) and
// the number of non-zero heights (dim 2).  Applies when E_t >= f_t (every
// block holds tiles) and g <= 32; 0 otherwise.

namespace mp {
namespace {

struct DownSet {
  uint32_t f0, f1, f2, g;
  uint64_t w[3];
  uint64_t best;
  uint32_t h[32][32];
  void rec(uint32_t i, uint32_t j, uint32_t rem) {
    if (rem == 0) {
      uint64_t p0 = 0, p1 = 0, p2 = 0;
      const uint32_t na = f0 < g ? f0 : g, nb = f1 < g ? f1 : g;
      for (uint32_t a = 0; a < na; ++a)
        for (uint32_t b = 0; b < nb; ++b) {
          if (!h[a][b]) continue;
          if (a == 0) p0 += h[a][b];
          if (b == 0) p1 += h[a][b];
          ++p2;
        }
      const uint64_t c = w[0] * p0 + w[1] * p1 + w[2] * p2;
      if (c < best) best = c;
      return;
    }
    if (i >= f0 || i >= g) return;
    if (j >= f1 || j >= g) {   // next row
      rec(i + 1, 0, rem);
      return;
    }
    const uint32_t up = i ? h[i - 1][j] : f2, left = j ? h[i][j - 1] : f2;
    uint32_t cap = up < left ? up : left;
    if (cap > rem) cap = rem;
    if (cap == 0) {   // the rest of this row is zero; a zero first cell ends the set
      if (j == 0) return;
      rec(i + 1, 0, rem);
      return;
    }
    for (uint32_t v = cap; v >= 1; --v) {
      h[i][j] = v;
      rec(i, j + 1, rem - v);
    }
    h[i][j] = 0;
    if (j > 0) rec(i + 1, 0, rem);   // row ends here
  }
};

}  // namespace

uint64_t secondary_lower_bound(const uint32_t E[3], const uint32_t f[3], uint32_t nodes, uint32_t g) {
  if (g == 0 || g > 32) return 0;
  for (int t = 0; t < 3; ++t)
    if (f[t] == 0 || E[t] < f[t]) return 0;
  DownSet ds;
  std::memset(&ds, 0, sizeof(ds));
  ds.f0 = f[0];
  ds.f1 = f[1];
  ds.f2 = f[2];
  ds.g = g;
  for (int v = 0; v < 3; ++v) {
    const int u = v == 0 ? 1 : 0, w = v == 2 ? 1 : 2;
    ds.w[v] = (uint64_t)(E[u] / f[u]) * (E[w] / f[w]);
  }
  ds.best = ~0ull;
  ds.rec(0, 0, g);
  if (ds.best == ~0ull) return 0;
  const uint64_t lines = ds.w[0] * f[1] * f[2] + ds.w[1] * f[0] * f[2] + ds.w[2] * f[0] * f[1];
  const unsigned __int128 tot = (unsigned __int128)ds.best * nodes;
  return tot > lines ? (uint64_t)(tot - lines) : 0;
}

}  // namespace mp

extern "C" int mp_secondary_lower_bound(const mp_search_query* query, const int64_t* f, uint64_t* lb_bytes) {
  using namespace mp;
  if (!query || !f || !lb_bytes) return MP_EINVAL;
  int rc = validate_query(*query);
  if (rc) return rc;
  if (f[0] < 1 || f[1] < 1 || f[2] < 1 || f[0] * f[1] * f[2] != query->procs) return MP_EINVAL;
  const uint32_t E[3] = {(uint32_t)query->M, (uint32_t)query->N, (uint32_t)query->K};
  const uint32_t ff[3] = {(uint32_t)f[0], (uint32_t)f[1], (uint32_t)f[2]};
  *lb_bytes = secondary_lower_bound(E, ff, (uint32_t)(query->procs / query->procs_per_node),
                                    (uint32_t)query->procs_per_node) * query->tile_bytes;
  return MP_OK;
}

