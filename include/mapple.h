/*
 * mapple.h -- C ABI of the GB300 engine for the Mapple index-mapping hot path
 * (Wei et al., "Mapple: A Domain-Specific Language for Mapping Distributed
 * Programs", arXiv 2507.17087).
 *
 * The engine evaluates an IndexTaskMap over a whole index launch: every point
 * of an N-D task space is sent through a distribution and a chain of
 * processor-space transforms to a (node, processor) id; the assignment is
 * reduced to a per-processor load histogram and an exact halo volume; and the
 * decompose search is run exhaustively over ordered factorisations and
 * transform chains.
 *
 * Conventions shared by every entry point
 *  - Return value: MP_OK (0) or one of the mp_status codes below.  Arguments
 *    are validated before anything is launched; on an error nothing has been
 *    written to any output.
 *  - Buffers are owned by the caller.  A buffer argument may point to device
 *    memory (cudaMalloc / torch) or to host memory (pinned or pageable); the
 *    engine looks the pointer up with cudaPointerGetAttributes.  With device
 *    buffers the call is asynchronous on `stream` (a cudaStream_t, NULL = the
 *    legacy default stream); with any host output buffer the call copies the
 *    result back (a page-locked id array is written by the id kernel directly
 *    through its device alias; MAPPLE_PINNED_DIRECT=0 stages it instead) and
 *    synchronises `stream` before returning.
 *  - The engine keeps a per-device workspace (tables, staging) that grows on
 *    demand and is reused by later calls; it is freed at process exit.  Calls
 *    that run concurrently on different streams of one device must be
 *    serialised by the caller (the workspace is shared).
 *  - A call that computes ids together with histograms or volumes runs the
 *    reductions on a second stream (one per host thread and device, created
 *    on first use) forked from `stream` after the chain table is built and
 *    joined back onto `stream` before the call's work ends, on every return
 *    path: the call stays ordered on `stream` and can be captured into a
 *    CUDA graph on it (allocate the workspace by one call before capturing).
 *  - Processor ids are node-major: id = node * procs_per_node + proc, where
 *    (node, proc) is the index of Machine(GPU) = (nodes, procs_per_node)
 *    (Sec. 3.2, Fig. 3).
 */
#ifndef MAPPLE_GB300_H
#define MAPPLE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
enum mp_status {
  MP_OK = 0,
  MP_EINVAL = 1,     /* invalid argument: bad transform, rank, extent, kind   */
  MP_EOVERFLOW = 2,  /* point count >= 2^62, or P too large for int32 ids     */
  MP_ENOMEM = 3,     /* device workspace allocation failed                    */
  MP_ECUDA = 4,      /* a CUDA runtime call failed                            */
  MP_ETIMEOUT = 5,   /* a bounded device-side wait gave up                    */
  MP_ENOTSUP = 6     /* size beyond what this engine supports (see limits)    */
};

/* ------------------------------------------------------------ limits */
#define MP_MAX_TASK_RANK 4        /* task-space rank (index launch)            */
#define MP_MAX_PROC_RANK 24       /* processor-space rank after transforms     */
#define MP_MAX_XFORMS 64          /* transforms in one chain                   */
#define MP_MAX_PROCS (1 << 26)    /* P = nodes * procs_per_node                */
#define MP_MAX_HALO_WIDTH 16      /* halo width per dimension (mp_halo_volume)  */
#define MP_MAX_EXTENT (1ll << 38) /* task extent bound: keeps the distributions'
                                     products x * s below 2^64 (MP_ENOTSUP)   */

/* ------------------------------------------------------------ data types */

/* Index launch (task space): rank 1..4, extents ext[0..rank), C order (last
 * dimension fastest), each extent 1 .. MP_MAX_EXTENT - 1 (an extent >=
 * MP_MAX_EXTENT is MP_ENOTSUP).  Point count prod(ext) must be < 2^62.  (Sec. 5.1's
 * ISpace / IPoint; Appendix A.1 task.ispace.) */
typedef struct mp_space {
  int32_t rank;
  int32_t reserved;
  int64_t ext[4];
} mp_space;

/* Machine(GPU): a 2-D processor space (nodes, processors per node),
 * Sec. 3.2. */
typedef struct mp_machine {
  int32_t nodes;
  int32_t procs_per_node;
} mp_machine;

/* Processor-space transforms (Fig. 4, Sec. 3.3; decompose Sec. 4.2). */
enum mp_op {
  MP_SPLIT = 0,          /* split(i, d): dim i of size s -> (d, s/d); d | s     */
  MP_MERGE = 1,          /* merge(i, j): i < j, dims fused at i, size s_i*s_j   */
  MP_SWAP = 2,           /* swap(i, j): exchange dims i and j, i != j           */
  MP_DECOMPOSE = 3,      /* decompose(i, T[0..k)): dim i -> k factors minimising
                            sum_m d_m / T_m, ties lexicographically smallest   */
  MP_BALANCE_SPLIT = 4   /* balance_split(i, k) = decompose(i, (1,...,1))      */
};

typedef struct mp_xform {
  int32_t op;         /* enum mp_op                                  */
  int32_t i;          /* dimension (split/merge/swap/decompose)      */
  int32_t j;          /* second dimension (merge/swap)               */
  int32_t k;          /* number of factors (decompose/balance_split) */
  int64_t d;          /* split factor                                */
  int64_t T[4];       /* decompose target extents T[0..k)            */
  int32_t h[4];       /* decompose: halo width along target dimension m
                         (0 everywhere = isotropic, width 1)         */
  int32_t transpose;  /* decompose: bit m set = all-to-all transpose
                         along target dimension m                    */
  int32_t reserved;
} mp_xform;
/* With halo widths h or transposes, decompose minimises the appendix's
 * generalised volume ("Generalization of the Decompose Primitive"):
 *   V = sum_m d_m h_m prod_{n != m} T_n  plus, for each transposed m,
 *   V*_m = (1 - 1/d_m) prod_n T_n,
 * compared exactly (MP_EOVERFLOW if s_i * V does not fit in 127 bits);
 * ties go to the lexicographically smallest factor tuple. */

/* Distributions: task point x -> index a of the final processor space. */
enum mp_dist_kind {
  MP_BLOCK = 0,          /* a_t = floor(x_t * s_t / L_t)  (Fig. 1a, Fig. 3)    */
  MP_CYCLIC = 1,         /* a_t = x_t mod s_t                                  */
  MP_BLOCK_CYCLIC = 2,   /* a_t = floor(x_t / b) mod s_t                       */
  MP_HIER = 3,           /* Appendix A.1 (Cannon): final rank 2k,
                            a_t = floor(x_t s_t / L_t), a_{k+t} = x_t mod s_{k+t} */
  MP_LINEAR_CYCLIC = 4   /* Fig. 5: a_0 = (C-order linear index of x) mod P    */
};

typedef struct mp_dist {
  int32_t kind;   /* enum mp_dist_kind                 */
  int32_t b;      /* block size of MP_BLOCK_CYCLIC     */
} mp_dist;

/* Rank fix-up.  The chain is applied to Machine(GPU) = (nodes, ppn).  If the
 * resulting rank differs from the rank the distribution indexes (k for
 * block / cyclic / block-cyclic, 2k for hier, 1 for linear-cyclic), the space
 * is flattened with merge(0,1) repeatedly and then: decompose(0, L) for the
 * rank-k kinds; split(0, nodes), decompose(0, L), decompose(k, L / node
 * factors) for hier (the Appendix A.1 pattern); nothing more for
 * linear-cyclic. */

/* ------------------------------------------------------------ entry points */

/* map_points: a1-a4 of the hot path.  For every point of `space` (C order)
 * writes ids[lin] = node * procs_per_node + proc, and hist[p] = number of
 * points mapped to processor p (p in [0, P)).
 *   chain / n_xf : transforms applied to Machine(GPU) in order (n_xf <= 64;
 *                  chain may be NULL when n_xf == 0)
 *   ids  : int32[prod(ext)] device or host, or NULL
 *   hist : uint64[P] device or host, or NULL (overwritten, not accumulated)
 * Errors: MP_EINVAL (invalid transform / distribution / extents),
 * MP_EOVERFLOW (prod(ext) >= 2^62), MP_ENOTSUP (P > MP_MAX_PROCS, or an
 * extent >= MP_MAX_EXTENT), MP_ENOMEM, MP_ECUDA. */
int mp_map_points(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                  int n_xf, const mp_dist* dist, int32_t* ids, uint64_t* hist, void* stream);

/* comm_volume: a5.  Nearest-neighbour (2k-point star) halo volume of the
 * launch under the mapping: every directed pair (x, x + delta e_t), delta =
 * +-1, with both points inside the launch and different owners, moves
 * face_bytes[t] bytes to the owner of x (Sec. 4.2's inter-processor surface,
 * Fig. 10; each face counted once per direction).
 *   face_bytes : host array of rank uint64 values (bytes per face along t)
 *   total      : uint64[1] device or host, required (overwritten)
 *   recv       : uint64[P] device or host, or NULL: bytes received per
 *                processor (overwritten)
 * Errors as mp_map_points. */
int mp_comm_volume(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                   int n_xf, const mp_dist* dist, const uint64_t* face_bytes, uint64_t* total,
                   uint64_t* recv, void* stream);

/* halo_volume: a5 with per-dimension halo widths.  Two counts:
 *  MP_HALO_FACES     the count of mp_comm_volume (width 1; width ignored):
 *                    bytes[t] per directed face (x, x +- e_t) across owners,
 *                    received by the owner of x;
 *  MP_HALO_ELEMENTS  de-duplicated elements (the appendix's anisotropic
 *                    halo, "Generalization of the Decompose Primitive"): a
 *                    processor p that owns a point x needs every
 *                    y = x + delta e_t, 1 <= |delta| <= width[t], inside the
 *                    launch; each such y that p does not own moves bytes[t]
 *                    to p once per dimension t, however many of p's points
 *                    need it.  For block layouts that divide the extents this
 *                    is sum_t 2 (d_t - 1) width[t] prod_{u != t} L_u.
 *   width : halo width per task dimension, 0..MP_MAX_HALO_WIDTH
 *   bytes : bytes per face / element along each task dimension
 *   total : uint64[1] device or host, required (overwritten)
 *   recv  : uint64[P] device or host, or NULL (bytes received per processor)
 * Errors as mp_map_points; MP_EINVAL for a width outside [0, 16] or an
 * unknown mode. */
enum mp_halo_mode { MP_HALO_FACES = 0, MP_HALO_ELEMENTS = 1 };
typedef struct mp_halo {
  int32_t mode;       /* enum mp_halo_mode            */
  int32_t width[4];   /* per task dimension           */
  int32_t reserved;
  uint64_t bytes[4];  /* per task dimension           */
} mp_halo;
int mp_halo_volume(const mp_space* space, const mp_machine* machine, const mp_xform* chain, int n_xf,
                   const mp_dist* dist, const mp_halo* halo, uint64_t* total, uint64_t* recv, void* stream);

/* Two-level search (the Solomonik mapper of Fig. 5b and the Cannon mapper of
 * Appendix A.1 as search spaces).  A candidate splits the node dimension of
 * Machine(GPU) into a node grid a (prod a = nodes) and the processor
 * dimension into a GPU grid b (prod b = procs_per_node), k = rank factors
 * each.  Node coordinate u_t = floor(x_t a_t / L_t); GPU coordinate
 *   MP_HIER_BLOCK   floor(x_t a_t b_t / L_t) mod b_t  (block within the node)
 *   MP_HIER_CYCLIC  x_t mod b_t                        (cyclic within the node)
 * node index u_0 + a_0 (u_1 + a_1 (...)), GPU index likewise, id = node *
 * procs_per_node + GPU.  Candidates: a over the ordered factorisations of
 * nodes, b over those of procs_per_node, both in lexicographic order; index =
 * rank(a) * |F(procs_per_node)| + rank(b).  Primary cost: the element halo
 * volume (mp_halo_volume, MP_HALO_ELEMENTS) between nodes; secondary: the
 * same between processors; the winner minimises (primary, secondary, index).
 * Every candidate's volumes are computed on the GPU.  Synchronous.
 * Errors: MP_EINVAL (rank, machine, widths, variant), MP_ENOTSUP (more than
 * 65536 candidates), as mp_halo_volume otherwise. */
enum mp_hier_variant { MP_HIER_BLOCK = 0, MP_HIER_CYCLIC = 1 };
typedef struct mp_hier_query {
  mp_space space;
  mp_machine machine;
  int32_t variant;    /* enum mp_hier_variant               */
  int32_t width[4];   /* halo width per task dimension      */
  uint64_t bytes[4];  /* bytes per element, per dimension   */
} mp_hier_query;
typedef struct mp_hier_result {
  int64_t index;
  int64_t a[4];               /* node grid (rank entries)            */
  int64_t b[4];               /* GPU grid                            */
  uint64_t primary_bytes;     /* inter-node halo bytes               */
  uint64_t secondary_bytes;   /* inter-processor halo bytes          */
  int64_t n_candidates;
} mp_hier_result;
int mp_hier_search(const mp_hier_query* query, mp_hier_result* out, void* stream);

/* The chain of a two-level candidate (for mp_map_points / mp_halo_volume):
 * splits of the node and GPU dimensions by a and b, then for MP_HIER_BLOCK
 * swaps and merges that pair each GPU factor (fastest) with its node factor,
 * to be used with the block distribution; for MP_HIER_CYCLIC the 2k-D space
 * of the hierarchical distribution.  Host only; writes at most 16 ops. */
int mp_hier_chain(int32_t rank, const int64_t* a, const int64_t* b, int32_t variant, mp_xform* chain,
                  int32_t* n_xf, mp_dist* dist);

/* The whole hot path of one launch in one call: ids and histogram as
 * mp_map_points, halo total and received bytes as mp_halo_volume (halo may
 * be NULL, then total and recv must be NULL too), sharing the chain table
 * and the per-dimension counts.  Any output may be NULL.  Errors as
 * mp_map_points / mp_halo_volume. */
int mp_map_launch(const mp_space* space, const mp_machine* machine, const mp_xform* chain, int n_xf,
                  const mp_dist* dist, const mp_halo* halo, int32_t* ids, uint64_t* hist, uint64_t* total,
                  uint64_t* recv, void* stream);

/* map_points without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * running under a memory manager that owns the device's whole budget (a
 * framework's caching allocator, or a pool sized once at start-up), and
 * latency-critical loops in which cudaMalloc's implicit device-wide
 * synchronisation would stall other streams.  It computes exactly what
 * mp_map_points computes and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   ids / hist : device memory only (a host buffer would need a staging
 *                area): MP_EINVAL otherwise; either may be NULL.
 *   scratch    : one 8 MiB array in this library's device memory, present on
 *                every GPU that loads the library until the process exits.  A
 *                launch whose scratch (4 P bytes of chain table, 4 bytes per
 *                coordinate of each tabled c_t, and, when hist is requested,
 *                8 bytes per sub-index of each dimension's counts -- at most
 *                8 * rank * P -- plus alignment) exceeds 8 MiB returns
 *                MP_ENOTSUP.  The scratch is rewritten (counts are cleared) by
 *                every call.
 *   set-up     : the first call on a device looks up the array's device
 *                address (cudaGetSymbolAddress, with that device current); make
 *                that first call before any stream capture.  The address is
 *                kept for the life of the process: a cudaDeviceReset between
 *                calls is not supported.
 *   streams    : every kernel runs on `stream`, the reductions after the id
 *                writer (mp_map_points would run them on a second stream); no
 *                stream or event is created.
 *   concurrency: every call shares the one array, so calls that overlap on
 *                the GPU (other streams, other host threads) race; serialise
 *                them. */
int mp_map_points_noalloc(const mp_space* space, const mp_machine* machine, const mp_xform* chain,
                          int n_xf, const mp_dist* dist, int32_t* ids, uint64_t* hist, void* stream);

/* decompose_search: a6-a8.  Exhaustive search for a 3-D matmul tile grid
 * (M, N, K) on Machine(GPU) = (P / procs_per_node, procs_per_node).  A
 * candidate is an ordered factorisation f = (f0, f1, f2) of P (Sec. 4.3) and
 * a transform chain c of depth <= max_depth over the canonical alphabet (at
 * shape s: split(i, d) for i ascending and 1 < d < s_i, d | s_i ascending;
 * merge(p, q) p < q lexicographic; swap(p, q) p < q lexicographic; chains
 * ordered by depth then by alphabet positions).  The candidate's mapping
 * flattens chain(Machine) with merge(0,1) repeatedly, splits it as f with
 * dimension 0 fastest (decompose's splits) and block-maps tile (i, j, k).
 * Its cost counts, for every tile of A(i,k), B(k,j) and C(i,j), the distinct
 * processors (primary) and distinct nodes (secondary) among the points
 * touching it, minus one, times tile_bytes.  The result minimises
 * (primary, secondary, index) lexicographically, index = f_rank * n_chains +
 * c_rank with f ranked in lexicographic order.  Synchronous; `out` is host. */
typedef struct mp_search_query {
  int64_t M, N, K;          /* tile-grid extents                        */
  int32_t procs;            /* P                                        */
  int32_t procs_per_node;   /* g (P % g == 0)                           */
  int32_t max_depth;        /* chain depth bound (0..4)                 */
  int32_t flags;            /* MP_SEARCH_* bits                         */
  uint64_t tile_bytes;      /* bytes per tile (512*512*4 for fp32)      */
} mp_search_query;

/* flags: MP_SEARCH_FULL scores the secondary cost of every candidate.
 * Without it, candidates whose primary cost (closed form in f) exceeds the
 * minimum primary are dismissed without scanning their secondary; the
 * argmin is the same.  Limits: M, N, K <= 2^20, P <= 16384. */
#define MP_SEARCH_FULL 1

typedef struct mp_search_result {
  int64_t index;            /* winning candidate index                  */
  int64_t f[3];             /* winning factorisation                    */
  int64_t chain_rank;       /* rank of the winning chain                */
  int32_t chain_len;        /* ops in the winning chain                 */
  int32_t reserved;
  mp_xform chain[4];        /* the winning chain                        */
  uint64_t primary_bytes;   /* primary cost in bytes                    */
  uint64_t secondary_bytes; /* secondary cost in bytes                  */
  int64_t n_candidates;     /* candidates evaluated                     */
  int64_t n_chains;         /* chains in the search space               */
  int64_t n_factorisations; /* factorisations in the search space       */
} mp_search_result;

int mp_decompose_search(const mp_search_query* queries, int n_queries, mp_search_result* out,
                        void* stream);

/* Exact costs of listed candidate indices of one query (device or host
 * arrays of n int64 indices; primary/secondary: uint64[n] in bytes).  Used to
 * re-evaluate sampled or proposed candidates.  MP_EINVAL on an index out of
 * range. */
int mp_candidate_costs(const mp_search_query* query, const int64_t* indices, int64_t n,
                       uint64_t* primary, uint64_t* secondary, void* stream);

/* ------------------------------------------------------------ batched launches */

/* One mapping query of a batch: a launch as mp_map_points / mp_comm_volume
 * take it, with its stencil face bytes. */
typedef struct mp_query {
  mp_space space;
  mp_machine machine;
  const mp_xform* chain;    /* read during mp_batch_create only            */
  int32_t n_xf;
  int32_t reserved;
  mp_dist dist;
  uint64_t face_bytes[4];
} mp_query;

typedef struct mp_batch mp_batch;   /* opaque planned batch */

/* Plans a batch once: validates and compiles every query (as mp_map_points),
 * lays out the output regions and uploads the descriptors to the current
 * device.  Limits per query: P <= 16384, fewer than 2^31 points.  Errors as
 * mp_map_points for the first bad query; MP_ENOMEM if the device pools
 * cannot be allocated.  The batch owns device memory until mp_batch_destroy. */
int mp_batch_create(const mp_query* queries, int n_queries, mp_batch** out);

/* Output layout: ids of query q start at ids_offsets[q] (a multiple of 4;
 * total_ids entries in all), hist / recv of query q at proc_offsets[q]
 * (total_procs entries in all; entry proc_offsets[q] + p is processor p of
 * query q).  Arrays of n + 1 entries, or NULL.  tile_groups: 4-point groups
 * per work tile of the persistent id writer (after autotuning). */
int mp_batch_info(const mp_batch* batch, uint64_t* total_ids, uint64_t* total_procs, uint64_t* ids_offsets,
                  uint64_t* proc_offsets, int32_t* tile_groups);

/* Runs the batch on `stream`: ids (int32[total_ids]), hist and recv
 * (uint64[total_procs]) and halo (uint64[n], total halo bytes per query) are
 * device buffers or NULL; results as mp_map_points / mp_comm_volume for every
 * query.  The kernels are captured into a CUDA graph on first use (and again
 * when the output pointers change) and replayed.  flags: MP_BATCH_AUTOTUNE
 * first times the persistent id writer at several tile sizes and keeps the
 * fastest (tiles of 8,192 to 131,072 four-point groups); MP_BATCH_NO_GRAPH
 * launches the kernels directly.  With ids and reductions both wanted, the
 * reductions run on the batch's own second stream beside the id writer and
 * join back onto `stream`.  Asynchronous.  Runs of one batch must not overlap
 * on the GPU (they share its pools). */
#define MP_BATCH_AUTOTUNE 1
#define MP_BATCH_NO_GRAPH 2
int mp_batch_run(mp_batch* batch, int32_t* ids, uint64_t* hist, uint64_t* halo, uint64_t* recv, int flags,
                 void* stream);

/* Sets the persistent id writer's tile size (4-point groups per tile, > 0),
 * e.g. one an earlier autotuning chose for the same batch: the persisted
 * autotune result.  The next run recaptures its graph.  Host side. */
int mp_batch_set_tile(mp_batch* batch, int32_t tile_groups);

int mp_batch_destroy(mp_batch* batch);

/* ------------------------------------------------------------ learned cost model */
/* The paper has no learned component; this is the project's surrogate that
 * prunes the decompose search (see mp_learned_search).  Its tensor-core
 * building block is exported for testing: */

/* C[M x N] (float32, row-major) = A[M x K] * B[N x K]^T with A, B bfloat16
 * row-major, FP32 accumulation on the tcgen05 tensor cores.  M % 128 == 0,
 * N % 64 == 0, K % 64 == 0; device buffers only.  Synchronous.  MP_ETIMEOUT
 * if a tensor-core completion wait gave up. */
int mp_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, void* stream);

/* The model: 64 candidate features -> 256 -> 256 -> 256 (ReLU) -> 1 score,
 * BF16 weights and activations, FP32 accumulation and FP32 master weights.
 * Parameters are packed as float32 W1[256x64] b1[256] W2[256x256] b2[256]
 * W3[256x256] b3[256] w4[256] b4[1] (mp_mlp_num_params() values). */
typedef struct mp_mlp mp_mlp;

int mp_mlp_create(uint64_t seed, mp_mlp** out);      /* He initialisation on the current device */
int mp_mlp_destroy(mp_mlp* model);
int mp_mlp_num_params(void);
int mp_mlp_set_params(mp_mlp* model, const float* params /* host */);
/* params / grads: host float32[mp_mlp_num_params()] or NULL; grads are those
 * of the last training step. */
int mp_mlp_get_params(const mp_mlp* model, float* params, float* grads);
/* y[B] = model(X[B x 64]) with X bfloat16; device buffers, B % 128 == 0,
 * B <= 2^26 (MP_ENOTSUP beyond). */
int mp_mlp_forward(mp_mlp* model, const void* X, float* y, int B, void* stream);
/* One Adam step (lr > 0) or gradients only (lr == 0) on the mean squared
 * error 0.5 mean (y - target)^2; *loss (host) receives the loss before the
 * step.  Device X (bfloat16 B x 64) and target (float32 B), B % 128 == 0,
 * B <= 2^26. */
int mp_mlp_train_step(mp_mlp* model, const void* X, const float* target, int B, float lr, float* loss,
                      void* stream);

/* Trains the model on exact costs: for each query, samples_per_query
 * candidates (half with the least primary cost, a quarter among the eight
 * lowest primaries, a quarter uniform) are evaluated exactly
 * (mp_candidate_costs), featurised, and the model takes `epochs` passes of
 * Adam over shuffled batches of `batch` (a multiple of 128), the step size
 * following a cosine from lr down to 0.05 lr over the run.  Regression
 * target: 2 min(p / p_min - 1, 16) + log2(1 + s) / 8 with p, s the
 * candidate's primary / secondary cost in tiles and p_min the query's least
 * primary.  *final_loss: last batch loss. */
int mp_mlp_train_search(mp_mlp* model, const mp_search_query* queries, int n_queries, int samples_per_query,
                        int epochs, int batch, float lr, uint64_t seed, float* final_loss, void* stream);

/* Learned decompose search.  Only candidates whose factorisation attains
 * the least primary cost can win the lexicographic argmin (the primary is
 * exact and closed-form), so the model scores those (fused tcgen05
 * inference; MP_LEARNED_SCORE_ALL scores every candidate).  The K best
 * scores, with the rest of the score-histogram bin the K-th falls in, are
 * evaluated exactly, and their argmin is found, on the device (one round
 * trip per selection).  It is returned when
 *   1 every candidate of least primary cost was evaluated (exact),
 *   2 its secondary reaches mp_secondary_lower_bound of every
 *     factorisation of least primary cost (exact), or
 *   3 the margin rule holds (a heuristic, calibrated by mp_mlp_calibrate):
 *     every candidate left out scored at least tau, and tau exceeds the
 *     winner's regression target by more than 1.25 x the calibrated
 *     overestimation bound + 0.01.  An uncalibrated model (or a model that
 *     produced a NaN / infinite score) gets no margin.
 * Otherwise the selection grows 2-fold in score order (while it stays
 * within 65536 candidates and half of those scored; each round evaluates
 * only the candidates it adds) and the rules are applied again; if they
 * still fail, the exhaustive search runs (exact).
 * So the returned costs are always the exact costs of the returned
 * candidate, and the candidate is the optimum under rules 1 and 2 and the
 * fallback; under rule 3 it is the optimum unless the model overestimated a
 * better candidate by more than its calibrated bound.
 * MP_LEARNED_NO_FALLBACK returns the argmin of the first selection without
 * growing or falling back.  K in [1, 65536].  Synchronous.
 * Phase times: ms_prepare and ms_fallback are host wall-clock; ms_model and
 * ms_exact are device time between events on the stream. */
typedef struct mp_learned_stats {
  int64_t n_scored;         /* candidates scored by the model                     */
  int64_t n_exact;          /* candidate evaluations, summed over the rounds      */
  int64_t n_selected;       /* size of the last selection                         */
  int32_t certified;        /* how the result was accepted: 0 not (fallback or
                               MP_LEARNED_NO_FALLBACK), 1 / 2 / 3 as above       */
  int32_t fallback;         /* 1: the exhaustive search ran                       */
  int32_t rounds;           /* selections evaluated (1 + growth steps)            */
  int32_t reserved;
  double margin;            /* tau - winner target - rule bound (last selection)  */
  double max_overestimate;  /* largest score - target on the last selection        */
  double margin_bound;      /* the rule bound used (infinite: not calibrated)     */
  double ms_prepare;        /* candidate space, pool, lower bounds (host)         */
  double ms_model;          /* fused scoring and the score histogram (device)     */
  double ms_exact;          /* selections, exact costs, argmin (device)           */
  double ms_wall;           /* scoring through the last selection (host)          */
  double ms_fallback;       /* the exhaustive search, when it ran (host)          */
} mp_learned_stats;
#define MP_LEARNED_NO_FALLBACK 1
#define MP_LEARNED_SCORE_ALL 2
int mp_learned_search(mp_mlp* model, const mp_search_query* query, int K, int flags, mp_search_result* out,
                      mp_learned_stats* stats, void* stream);

/* Calibrates the margin rule of mp_learned_search on queries held out of
 * training.  For each query every candidate of least primary cost is scored
 * and evaluated exactly, and the model's overestimation of its best-scored
 * optimal candidate (least score among the candidates of least secondary,
 * minus their regression target) is taken; the bound is the largest over
 * the queries (*bound_out, host).  The model keeps it (and checkpoints
 * carry it).  Synchronous. */
int mp_mlp_calibrate(mp_mlp* model, const mp_search_query* queries, int n_queries, double* bound_out,
                     void* stream);
/* Sets the bound directly (INFINITY: no margin rule). */
int mp_mlp_set_margin_bound(mp_mlp* model, double bound);

/* Scores of every candidate of a query in index order (the fused scoring
 * kernel of mp_learned_search), and optionally their features (bfloat16,
 * n x 64).  Device buffers sized by the search space (*n_out receives the
 * candidate count).  Synchronous. */
int mp_learned_scores(mp_mlp* model, const mp_search_query* query, float* scores, void* features, int64_t* n_out,
                      void* stream);

/* ------------------------------------------------------------ host helpers */

/* Plan only (no GPU work): final processor-space shape and the expanded
 * primitive list (split / merge / swap after decompose expansion and the rank
 * fix-up), 4 int64 per primitive [op, p, q, d].  rank/shape/prims may be
 * NULL.  Returns MP_OK or the validation error. */
int mp_plan(const mp_space* space, const mp_machine* machine, const mp_xform* chain, int n_xf,
            const mp_dist* dist, int32_t* rank, int64_t* shape, int32_t* n_prims,
            int64_t* prims, int32_t prims_cap);

/* A chain built from random numbers: at each step the op is the
 * (draws[step] mod |A|)-th entry of the canonical alphabet A of the current
 * shape; an empty alphabet ends the chain.  Writes *n_out <= depth ops. */
int mp_chain_from_draws(int32_t nodes, int32_t procs_per_node, int32_t depth,
                        const uint64_t* draws, mp_xform* out, int32_t* n_out);

/* Decodes candidate `index` of a search query: its factorisation f[3] and
 * its chain (chain_len <= 4 ops).  Host only; MP_EINVAL if out of range. */
int mp_search_candidate(const mp_search_query* query, int64_t index, int64_t* f, mp_xform* chain,
                        int32_t* chain_len);

/* A lower bound on the secondary cost (bytes) of factorisation f[3] of a
 * search query over every chain: each node owns procs_per_node cells of the
 * f0 x f1 x f2 block grid; the lines of a fibre family a node meets are its
 * projection, minimised over down-sets of that many cells (pushing a cell set
 * towards the origin along an axis never enlarges a projection), each line
 * weighted by the smallest tile count of its fibres.  0 when no bound
 * applies (an extent below its factor, or more than 32 processors per node).
 * Exact when the extents are divisible by f and an optimal chain gives every
 * node an optimal down-set.  Host only. */
int mp_secondary_lower_bound(const mp_search_query* query, const int64_t* f, uint64_t* lb_bytes);

/* Size of a decompose search space: number of factorisations of P into 3
 * ordered factors and number of canonical chains of depth <= max_depth. */
int mp_search_space(int32_t procs, int32_t procs_per_node, int32_t max_depth,
                    int64_t* n_factorisations, int64_t* n_chains);

/* The processor grid of Algorithm A1 (the greedy baseline the paper compares
 * decompose with, Sec. 4.3 and the appendix's "Baseline Greedy Algorithm"):
 * the prime factors of d in ascending order, each multiplied into the
 * currently smallest of k factors (first one on ties), then sorted in
 * descending order.  Host only; MP_EINVAL for d < 1 or k outside [1, 4]. */
int mp_greedy_grid(int64_t d, int32_t k, int64_t* out);

/* Measurement hook: the next launch of the dominant per-point kernel
 * (the id writer of mp_map_points) records `start_event` just before it and
 * `stop_event` just after it on the call's stream (both cudaEvent_t; one-shot,
 * cleared after use; NULL disables).  Lets a caller time that kernel alone
 * with CUDA events. */
int mp_set_kernel_timer(void* start_event, void* stop_event);

/* The same for the learned scorer's layer kernel (the three tcgen05 layers
 * and the output dot product, one launch per run of at most 2^19 scored
 * candidates): the next launch records `start_event` before it and
 * `stop_event` after it on the call's stream; one-shot; NULL disables. */
int mp_set_layer_timer(void* start_event, void* stop_event);

/* Bytes of launch description one kernel launch carries to the device as
 * parameters (the host-to-device input of a mapping call). */
uint64_t mp_descriptor_bytes(void);

/* ------------------------------------------------------------ checkpoint, self-tests */

/* Model checkpoint (training can resume from it): a binary file with a
 * versioned header -- 8 bytes "MAPLEMLP", uint32 format version (2), uint32
 * parameter count, int64 Adam step, float64 margin bound (mp_mlp_calibrate;
 * version 2 only) -- followed by the float32 parameters and the two float32
 * Adam moment arrays.  mp_mlp_load reads versions 1 and 2 (a version-1 file
 * leaves the model uncalibrated) and rejects another magic, version or
 * parameter count (MP_EINVAL) and a short file (MP_EINVAL); MP_ECUDA / file
 * errors otherwise.  Synchronous. */
int mp_mlp_save(const mp_mlp* model, const char* path);
int mp_mlp_load(mp_mlp* model, const char* path);

/* Device-side failure reporting without a fault: one CTA waits on an
 * mbarrier that nothing arrives on, with the same bounded polling the
 * tensor-core kernels use, `limit` polls (1 .. 2^26), and records
 * MP_ETIMEOUT in a status word; returns that status (MP_ETIMEOUT expected).
 * The context stays usable.  Synchronous. */
int mp_selftest_wait_timeout(uint32_t limit, void* stream);

/* Host-side fault injection: the next n requests for device workspace fail
 * as if the allocation had failed (the calls return MP_ENOMEM before
 * launching anything).  n = 0 clears it. */
int mp_debug_fail_allocations(int32_t n);

/* Human-readable text of a status code (static storage). */
const char* mp_strerror(int status);

/* Where the calling thread's last MP_ECUDA came from: source location and
 * the CUDA error name and text (empty if none). */
const char* mp_last_error_detail(void);

/* Number of kernel launches issued by this library in the calling process. */
uint64_t mp_kernel_launches(void);

/* Bytes of device workspace this library holds on the current device (the
 * grow-only per-device scratch of the mapping calls; 0 before the first
 * call).  Host only; lets a caller see whether a call allocated. */
uint64_t mp_workspace_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* MAPPLE_GB300_H */
