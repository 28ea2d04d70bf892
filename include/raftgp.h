/*
 * raftgp.h -- C ABI of the GB300 (sm_103a) RaftGP hot path.
 *
 * RaftGP (Gao et al., HPEC 2023) partitions an undirected graph in three stages:
 *   1. random feature extraction, Y = X Theta (Section III-A, Eq. 5), X one of
 *        M       = D^-1/2 A D^-1/2                      (NCut operator, Eq. 2)
 *        Q       = A - d d^T / 2e  (full modularity matrix, Eq. 4), applied as the sparse
 *                  product A Theta minus the rank-one term d (d^T Theta) / 2e
 *        Q-tilde = Q kept on the edges of G only       (reduced modularity, Section III-A);
 *   2. a randomly initialised, untrained GCN (Section III-B, Eq. 6):
 *        Z^(k) = rownorm(tanh(D-hat^-1/2 (A+I) D-hat^-1/2 Z^(k-1) W^(k))),  Z^(0) = Y;
 *   3. model selection: k-means for candidate block counts K, each partition scored by
 *      modularity (Eq. 3, evaluated as Eq. 7 with U = V) or NCut (Eq. 1); the best wins
 *      (Section III-C; the problem statement, Def. 1, leaves K unknown).
 *
 * Conventions for every entry point:
 *   - Graphs are symmetric CSR without self loops or duplicate entries (Section II:
 *     undirected, unweighted).  row_ptr has n+1 entries (int32 or int64), col has nnz int32
 *     entries, nnz = 2|E|.  All graph, feature and label arrays are DEVICE pointers owned by
 *     the caller; the library never allocates or frees device memory.  Scratch memory is a
 *     caller-owned device workspace whose size raftgp_workspace_size() returns (it may start
 *     at any address: the library aligns its pieces inside it).  A feature
 *     matrix Z (N x d, row-major, rows packed) must start on a 16-byte boundary; a Z that
 *     does not is rejected with RAFTGP_EINVAL (rows of 32 x elem bytes keep every row aligned).
 *   - Every call is ordered on the given CUDA stream.  Calls with host outputs synchronise
 *     that stream before returning; the others return as soon as the work is queued.
 *   - Every call returns a raftgp_status and never aborts.  Invalid arguments (null
 *     pointers, sizes out of range, a workspace that is too small) return RAFTGP_EINVAL or
 *     RAFTGP_ENOMEM before any work is queued.  Device-side checks (column index out of
 *     range, decreasing row_ptr, a self loop) set an error word that is read at the end of
 *     the call and reported as RAFTGP_EINVAL.  raftgp_last_error() gives a message.
 *   - Floating point: features are stored in FP32 or BF16 and always accumulated in FP32.
 *     Block edge counts and volumes are exact int64; modularity is one FP64 division of an
 *     exact integer numerator by an exact integer denominator; NCut is an FP64 sum in
 *     ascending block order.  k-means centroid sums are exact 2^-40 fixed point (int64),
 *     the means are formed in FP64.
 */
#ifndef RAFTGP_H
#define RAFTGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* raftgp_stream_t; /* a cudaStream_t; NULL is the legacy default stream */

typedef enum {
    RAFTGP_OK = 0,
    RAFTGP_EINVAL = 1,      /* bad argument or malformed graph */
    RAFTGP_ENOMEM = 2,      /* workspace too small */
    RAFTGP_ECUDA = 3,       /* a CUDA runtime call failed */
    RAFTGP_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    RAFTGP_EUNSUPPORTED = 5 /* a size or mode the library does not support */
} raftgp_status;

enum { RAFTGP_OP_NCUT = 0, RAFTGP_OP_MOD_FULL = 1, RAFTGP_OP_MOD_REDUCED = 2 };
enum { RAFTGP_F32 = 0, RAFTGP_BF16 = 1 };
enum { RAFTGP_CRIT_MOD = 0, RAFTGP_CRIT_NCUT = 1 };
/* k-means distance engine: plain FP32 FMA; or BF16 tcgen05 tensor cores with the centroids
 * split into BF16 hi + lo halves (~16-bit products) and an FP32 re-check of near ties in the
 * final assignment (RAFTGP_ASSIGN_TC); or the same with the hi half only in the Lloyd passes
 * (8-bit centroid products; the final assignment is still hi + lo with the FP32 re-check)
 * (RAFTGP_ASSIGN_TC8). */
enum { RAFTGP_ASSIGN_FFMA = 0, RAFTGP_ASSIGN_TC = 1, RAFTGP_ASSIGN_TC8 = 2 };
/* Re-check of near ties in the assignment whose labels are reported (the final assignment of
 * every candidate).  Its scores carry a bounded rounding error (the bound is derived in
 * assign_tc.cu and assign_ffma.cu from the operand splits and FP32 accumulation); every
 * (point, candidate) whose best two scores lie within twice that bound (plus a 25% margin) is
 * recomputed in the direct form sum_k (z_k - mu_k)^2 over ascending coordinates, each operation
 * rounded on its own:
 *   RAFTGP_RECHECK_NONE: no re-check (tensor cores: labels straight from the BF16 hi + lo scores);
 *   RAFTGP_RECHECK_FP32: in FP32 (tensor cores; the FP32 engine already reports the FP32 argmin);
 *   RAFTGP_RECHECK_FP64: in FP64 (both engines): every reported label is then the argmin of the
 *     FP64 direct-form distance from the stored z (BF16 or FP32) to the FP32 centroid, lowest
 *     index on ties, i.e. the same label an FP64 program evaluating that expression returns.
 * The FP32 engine needs one more assignment pass for RAFTGP_RECHECK_FP64. */
enum { RAFTGP_RECHECK_NONE = 0, RAFTGP_RECHECK_FP32 = 1, RAFTGP_RECHECK_FP64 = 2 };

#define RAFTGP_MAX_LAYERS 4
#define RAFTGP_MAX_BATCH_CAND 64 /* candidates evaluated together in one batch */

typedef struct {
    int64_t n;            /* number of nodes */
    int64_t nnz;          /* number of stored entries (2|E|) */
    const void* row_ptr;  /* device, n+1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
    int32_t row_ptr_bits; /* 32 or 64 */
    const int32_t* col;   /* device, nnz entries in [0, n) */
} raftgp_csr;

/* Embedding options (Section III-A/B). */
typedef struct {
    int32_t op;        /* RAFTGP_OP_*: the operator X of Eq. 5 */
    int32_t n_layers;  /* GCN layers, 0..RAFTGP_MAX_LAYERS; 0 = no GCN (Z = rownorm(Y)) */
    int32_t dims[RAFTGP_MAX_LAYERS + 1]; /* dims[0] = L, dims[k] = width of layer k;
                                            each one of 32, 64, 128 */
    int32_t dtype;     /* RAFTGP_F32 or RAFTGP_BF16: storage of Theta, hidden features, Z */
    uint64_t seed;     /* Philox4x32-10 key for Theta and W */
    const float* theta;                 /* optional device N x L FP32 row-major; NULL = draw */
    const float* W[RAFTGP_MAX_LAYERS];  /* optional device FP32 row-major L_{k-1} x L_k */
    void* stage_out[RAFTGP_MAX_LAYERS + 1]; /* optional device outputs in `dtype`: stage 0 =
                                               Y (N x L), stage k = Z^(k) (N x dims[k]) */
} raftgp_embed_opts;

/* Model-selection options (Section III-C). */
typedef struct {
    int32_t kmin, kmax; /* candidate range, 1 <= kmin <= kmax (kmax is clamped to n) */
    int32_t grid;       /* 0: every K in [kmin, kmax]; G > 0: a coarse grid of G values, then
                           G refined values between the neighbours of the best coarse K */
    int32_t iters;      /* maximum Lloyd assignment passes per candidate (>= 1) */
    int32_t criterion;  /* RAFTGP_CRIT_MOD (default) or RAFTGP_CRIT_NCUT */
    int32_t assign;     /* RAFTGP_ASSIGN_FFMA, RAFTGP_ASSIGN_TC or RAFTGP_ASSIGN_TC8 */
    int32_t batch;      /* candidates evaluated together (1 = one at a time, the plain form;
                           0 = as many as fit, at most RAFTGP_MAX_BATCH_CAND) */
    int32_t recheck;    /* RAFTGP_RECHECK_*: near-tie re-check of the reported labels */
    uint64_t seed;      /* Philox4x32-10 key for k-means++ */
} raftgp_select_opts;

/* Per-candidate report of raftgp_select / raftgp_partition (host memory). */
typedef struct {
    int32_t k_best;        /* out: chosen K */
    int32_t n_cand;        /* out: candidates evaluated */
    int32_t cand_cap;      /* in: capacity of the arrays below (they may be NULL if 0) */
    int32_t* cand_k;       /* out: K of each evaluated candidate, in evaluation order */
    double* cand_mod;      /* out: modularity (Eq. 3) */
    double* cand_ncut;     /* out: NCut (Eq. 1) */
    int32_t* cand_passes;  /* out: Lloyd assignment passes used */
} raftgp_select_result;

/* Bytes of device workspace the calls below need for this graph and these options.
 * Pass eopts = NULL for a selection-only call and sopts = NULL for an embedding-only call.
 * d (the embedding width) is used only when eopts is NULL.  Returns 0 on invalid input. */
size_t raftgp_workspace_size(const raftgp_csr* g, const raftgp_embed_opts* eopts,
                             const raftgp_select_opts* sopts, int32_t d);

/* Stages 1-2: Z = the normalised output of the last GCN layer (N x dims[n_layers], stored
 * in eopts->dtype, row-major) written to the device buffer Z.  Section III-A (Eq. 5) and
 * III-B (Eq. 6 and the row-wise l2 normalisation).  Asynchronous. */
raftgp_status raftgp_embed(const raftgp_csr* g, const raftgp_embed_opts* eopts, void* Z, void* ws,
                           size_t ws_bytes, raftgp_stream_t stream);

/* Stage 3: choose K and the partition for embeddings Z (device, N x d row-major, d one of
 * 32, 64, 128, stored as z_dtype).  Requires rows of norm <= 1 (the GCN output has unit
 * rows).  labels: device int32[N], the chosen partition, values in [0, k_best).  res: host
 * report (may be NULL).  Synchronises the stream. */
raftgp_status raftgp_select(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                            const raftgp_select_opts* sopts, int32_t* labels, raftgp_select_result* res,
                            void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* Stages 1-3 end to end: raftgp_embed followed by raftgp_select.  Synchronises the stream. */
raftgp_status raftgp_partition(const raftgp_csr* g, const raftgp_embed_opts* eopts,
                               const raftgp_select_opts* sopts, int32_t* labels, raftgp_select_result* res,
                               void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* Score a given partition: m[r] = number of undirected edges inside block r, vol[r] = sum of
 * the degrees in block r (both device int64[K], exact), *mod = Eq. 3 (via Eq. 7 with U = V,
 * exact integer numerator, one FP64 division) and *ncut = Eq. 1 (host doubles).
 * labels: device int32[N] with values in [0, K).  Synchronises the stream. */
raftgp_status raftgp_score(const raftgp_csr* g, const int32_t* labels, int32_t K, int64_t* m, int64_t* vol,
                           double* mod, double* ncut, void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* k-means++ seeding alone (the seeding step of stage 3): seeds (device int32[K]) receive K
 * point indices drawn by D^2 sampling from Z (device N x d, z_dtype).  D^2 is the FP32
 * direct-form squared distance summed over ascending coordinates, quantised to
 * floor(D^2 * 2^40) (uint64); draw t: r = Philox(seed; t, 0, 0, "Kmpp") words 0-1,
 * threshold floor(r * sum_q / 2^64), first index whose inclusive prefix exceeds it; if every
 * q is 0 the lowest-index unchosen point.  ws: at least 7 N + 8 max(ceil(N / 1024), 2048)
 * + 4 K + 2048 bytes.  All rounds usually run in one cooperative launch whose blocks meet at
 * bounded grid barriers; if a barrier gives up (2 s) the seeds not yet drawn are written as
 * -1.  Asynchronous. */
raftgp_status raftgp_kmeanspp(const void* Z, int64_t n, int32_t d, int32_t z_dtype, int32_t K, uint64_t seed,
                              int32_t* seeds, void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* Lloyd's k-means alone from given FP32 initial centroids mu0 (device K x d): at most
 * `iters` assignment passes, ties to the lowest centroid, stop when no label changes, an
 * empty cluster keeps its centroid.  labels: device int32[N], assigned against the returned
 * centroids; mu_out: device FP32 K x d (may be NULL); *passes (host): assignment passes
 * used.  `assign` picks the distance engine, `recheck` (RAFTGP_RECHECK_*) the near-tie
 * re-check of the reported labels; with iters = 1 and RAFTGP_RECHECK_FP64 the labels are the
 * FP64 direct-form argmin against mu0 itself.  ws: raftgp_lloyd_workspace_size(n, d, K)
 * bytes.  Synchronises the stream. */
size_t raftgp_lloyd_workspace_size(int64_t n, int32_t d, int32_t K);
raftgp_status raftgp_lloyd(const void* Z, int64_t n, int32_t d, int32_t z_dtype, const float* mu0, int32_t K,
                           int32_t iters, int32_t assign, int32_t recheck, int32_t* labels, float* mu_out,
                           int32_t* passes, void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* k-means++ seeding exactly as raftgp_kmeanspp, for callers that cannot allocate device
 * memory: for example a plugin running inside another program's CUDA context, whose device
 * memory that program's own allocator owns and budgets, or a process that reserves all the
 * device memory it may use before it starts partitioning.  The paper has no counterpart;
 * this is a deployment variant of the seeding step.
 * Its scratch (the D^2 array, nearest-seed indices, chosen-point flags, block sums and grid
 * barrier words, about 7 bytes per point) is a file-scope device array of
 * RAFTGP_NOALLOC_SCRATCH_BYTES.  Each CUDA context that runs the call holds its own copy until
 * the context ends.  With lazy module loading (CUDA_MODULE_LOADING=LAZY, the default) the
 * array's memory is committed by the first call in a context, not when the library is loaded:
 * a caller that reserves all the remaining device memory up front makes one call (any small
 * n) before reserving.  n above RAFTGP_NOALLOC_MAX_N (or K above 32767) is rejected with
 * RAFTGP_EUNSUPPORTED before any work is queued.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  The array's device address belongs to the context:
 * the first call in each context (the one current on the calling thread, else the device's
 * primary context) looks it up (cudaGetSymbolAddress) and caches it under the context's unique
 * id, so make that first call before any stream capture.  Every call in a context uses the same
 * array, which keeps the previous call's contents (the call clears what must start at zero):
 * calls whose work overlaps on the GPU (other streams, other host threads) race on it and must
 * not be issued.  Same arguments, results and status codes as raftgp_kmeanspp otherwise;
 * asynchronous. */
#define RAFTGP_NOALLOC_SCRATCH_BYTES (32u << 20) /* 32 MiB */
#define RAFTGP_NOALLOC_MAX_N 4500000
raftgp_status raftgp_kmeanspp_noalloc(const void* Z, int64_t n, int32_t d, int32_t z_dtype, int32_t K, uint64_t seed,
                                      int32_t* seeds, raftgp_stream_t stream);

/* ---- Instrumentation (the paper has no counterpart: its Table III times whole stages) ----
 * When enabled, each kernel family is bracketed by CUDA events recorded on the stream it is
 * launched on, and its launches are counted.  raftgp_profile_enable(1) clears the counters
 * and starts recording; raftgp_profile_enable(0) stops.  raftgp_profile_read synchronises the
 * device and writes up to `cap` entries (families with at least one launch); it returns the
 * number written.  Timing covers at most 32768 bracketed launch groups per enable; launches
 * beyond that are counted but not timed (timed < launches). */
typedef struct {
    const char* name;   /* kernel family, a static string */
    int64_t launches;   /* kernel launches since enable */
    int64_t timed;      /* launches covered by the timing */
    double ms;          /* summed device time of the timed launches */
} raftgp_prof_entry;

raftgp_status raftgp_profile_enable(int32_t on);
/* As raftgp_profile_enable(1), but only the named family (a name raftgp_profile_read reports,
 * e.g. "assign_tc") records events; the other families' launches are not counted.  NULL: every
 * family.  RAFTGP_EINVAL for an unknown name (profiling state unchanged). */
raftgp_status raftgp_profile_enable_family(const char* family);
int32_t raftgp_profile_read(raftgp_prof_entry* out, int32_t cap);

/* ---- Test hook (failure detection without a GPU fault) ----
 * From the next seeding on, block `block` of the persistent k-means++ kernel leaves at the
 * start of round 2 without arriving at the grid barrier.  The other blocks' bounded wait
 * (2 s) runs out: the kernel records a timeout, marks the unfinished seeds -1 and returns, and
 * raftgp_select / raftgp_partition report RAFTGP_ETIMEOUT; the context stays usable.  -1 (the
 * default) turns the hook off.  Not thread-safe; for tests only. */
void raftgp_debug_seed_skip_block(int32_t block);

/* Message for the last non-OK status returned on the calling thread. */
const char* raftgp_last_error(void);

/* Library version string. */
const char* raftgp_version(void);

/* ---- Algorithm 1: recursive bisection by local modularity ----
 * Partition(U): LMod(U; G) with U as one block (Definition 5, Eq. 7); K=2 k-means on U's
 * embeddings; LMod(U1, U2; G); U is a block if |U1| <= eps or |U2| <= eps or LMod(U) >
 * LMod(U1, U2) (compared exactly), otherwise U1 and U2 are partitioned.  `reading` chooses
 * e in Eq. 7: 0 = the G-degree sum of U over 2 (Definition 5 as printed), 1 = |E| of the
 * whole graph (a split is taken exactly when it raises the graph's modularity).  k-means++
 * draws Philox(seed; t, id_lo, id_hi, "Kmpp") with id the set's node in the recursion tree
 * (root 1, children 2 id, 2 id + 1); Lloyd as the FP32 engine, at most `iters` passes.  All
 * sets of one depth run together; the host reads the set count once per depth.  labels
 * (device int32[n]): blocks numbered by increasing smallest node; *k_out (host): the block
 * count.  Z: device N x d (32, 64 or 128), z_dtype F32 or BF16. */
typedef struct {
    int32_t eps;        /* size threshold, 5 in the paper */
    int32_t iters;      /* Lloyd pass cap */
    int32_t reading;    /* 0 literal, 1 global (see above) */
    uint64_t seed;
} raftgp_bisect_opts;
size_t raftgp_bisect_workspace_size(int64_t n, int32_t d, int32_t eps);
/* leaf (device uint64[n], may be NULL): each node's block as its node id in the recursion tree
 * (the input of a later raftgp_select_bisect_update). */
raftgp_status raftgp_select_bisect(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                                   const raftgp_bisect_opts* o, int32_t* labels, uint64_t* leaf, int32_t* k_out,
                                   void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* Streaming update of Algorithm 1 (Section III-D: the partition tree lets one update only the
 * tree paths of the nodes whose embedding changed).  g and Z are the new graph and embedding;
 * old_labels / old_k / old_leaf (device) are a previous run's labels, block count and leaf ids
 * (raftgp_select_bisect or this call) with the same options; changed (device uint8[n]) marks
 * every node whose embedding row or degree changed since (for an edge batch: at least both
 * endpoints of every new edge and every row the embedding recomputed).  A set of the recursion
 * that is the previous tree's node (every ancestor split as before) and holds no changed node
 * keeps its previous subtree without k-means; the others are partitioned again, and a changed
 * split rebuilds the subtree below it.  With reading 0 (2e = the G-degree sum of U) the
 * result equals raftgp_select_bisect on the new graph and embedding; with reading 1 every
 * decision also depends on |E|, and kept subtrees are not re-decided (the path update).
 * Outputs as raftgp_select_bisect; the same workspace size.  Synchronises the stream. */
raftgp_status raftgp_select_bisect_update(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                                          const raftgp_bisect_opts* o, const int32_t* old_labels, int32_t old_k,
                                          const uint64_t* old_leaf, const uint8_t* changed, int32_t* labels,
                                          uint64_t* leaf, int32_t* k_out, void* ws, size_t ws_bytes,
                                          raftgp_stream_t stream);

/* ---- Many graphs at once ----
 * The graphs arrive as one block-diagonal CSR: graph g owns the nodes graph_off[g] ..
 * graph_off[g+1]-1 (host int64[n_graphs + 1], graph_off[0] = 0, graph_off[n_graphs] = n) and
 * every column of its rows lies in that range (checked on the device).  Each graph is
 * partitioned as raftgp_partition would partition it alone with the k-means engine of
 * bo->assign: its own Eq. 5 projection (Philox rows by the node's index inside the graph;
 * eo->op the NCut operator, or with BF16 storage the full modularity operator, whose rank-one
 * term d (d^T Theta) / 2e is formed per graph from that graph's degrees and rows, in a fixed
 * order that differs from a single-graph run's, so its embedding may differ from it by FP32
 * rounding), the Eq. 6 layers, k-means++ and Lloyd for the candidates of its own coarse + refined
 * grid over [kmin, K_max(g)], K_max(g) = min(ceil(kmax_factor * N_g^0.35), 128, N_g), scored
 * by Eq. 3 / Eq. 1.  The embedding is one pass over the concatenation; the model selection
 * runs in persistent kernels over per-graph and per-candidate work queues; the whole
 * pipeline is captured once into a CUDA graph and replayed.  Embedding widths: final d of 32
 * or 64. */
typedef struct {
    int32_t kmin;          /* smallest K (>= 2) */
    float kmax_factor;     /* K_max(g) = min(ceil(kmax_factor * N_g^0.35), 128, N_g), e.g. 2 */
    int32_t grid;          /* coarse and refined grid size, 1..10 */
    int32_t iters;         /* Lloyd pass cap T */
    int32_t criterion;     /* RAFTGP_CRIT_MOD or RAFTGP_CRIT_NCUT */
    int32_t lloyd_variant; /* 0: autotune the Lloyd kernel; v in 1..7: use variant v - 1 of the
                              list raftgp_batch_plan_tuning reports (no timing) */
    int32_t embed_variant; /* BF16 embeddings: 0 autotunes the gathers' shape; v in 1..4 uses
                              shape v - 1 of raftgp_batch_plan_tuning_embed's list (no timing) */
    int32_t assign;        /* RAFTGP_ASSIGN_FFMA (default): the FP32 Lloyd kernels above, each
                              graph's result equal to a single-graph FP32 partition;
                              RAFTGP_ASSIGN_TC8 / RAFTGP_ASSIGN_TC: tensor-core Lloyd (BF16
                              embeddings only): Lloyd passes on the hi (TC8) or hi + lo (TC) BF16
                              centroid operand, the final assignment on hi + lo with the FP32
                              re-check of near ties, so every reported label is the FP32-nearest
                              centroid (the autotuner is not run) */
    uint64_t seed;         /* k-means++ seed (the same for every graph) */
} raftgp_batch_opts;

typedef struct raftgp_batch_plan raftgp_batch_plan;   /* opaque */

size_t raftgp_batch_workspace_size(const raftgp_csr* g, const int64_t* graph_off, int32_t n_graphs,
                                   const raftgp_embed_opts* eo, const raftgp_batch_opts* bo);

/* Validates the batch (synchronises), runs the autotuner (the Lloyd kernel's threads per CTA
 * and points per thread, timed on this batch; none of them changes a result) and captures the
 * whole partition into a CUDA graph.  labels (device int32[n]: each node's block inside its
 * graph), k_out (device int32[n_graphs]: K*), ws (device workspace) and any caller arrays the
 * options point at (eo->theta, eo->W) must stay valid for the plan's life.  *plan receives the
 * plan (NULL on failure). */
raftgp_status raftgp_batch_plan_create(const raftgp_csr* g, const int64_t* graph_off, int32_t n_graphs,
                                       const raftgp_embed_opts* eo, const raftgp_batch_opts* bo, int32_t* labels,
                                       int32_t* k_out, void* ws, size_t ws_bytes, raftgp_stream_t stream,
                                       raftgp_batch_plan** plan);
/* Replays the captured partition on `stream` (asynchronous). */
raftgp_status raftgp_batch_plan_run(raftgp_batch_plan* plan, raftgp_stream_t stream);
/* Host copies of every graph's candidates (n_graphs x 20 each; slots 0..9 coarse, 10..19
 * refined; unused slots have k = 0) after a run.  Synchronises. */
raftgp_status raftgp_batch_plan_candidates(raftgp_batch_plan* plan, int32_t* k, double* mod, double* ncut,
                                           int32_t* passes);
/* The autotuner's choice and its measured times (ms of the coarse Lloyd phase) for the seven
 * variants: the scalar Lloyd kernel at {128, 256, 512 threads} x {1, 2 points per thread}, in
 * that order, then the register-tiled kernel (256 threads, reported as 0 points per thread).
 * Every variant computes the same labels. */
raftgp_status raftgp_batch_plan_tuning(const raftgp_batch_plan* plan, int32_t* threads, int32_t* points_per_thread,
                                       float* ms);
/* The autotuner's choice for the BF16 embedding's gathers and its measured times (ms of one
 * embedding of the batch) for the four flat-stream shapes: {16, 32} entries per batch (at
 * width 128) x {2, 3} staging buffers, variant = 2 (batch 32) + (3 buffers); every shape gives
 * the same bits.  FP32 embeddings: variant 0 and times 0 (not tuned). */
raftgp_status raftgp_batch_plan_tuning_embed(const raftgp_batch_plan* plan, int32_t* variant, float* ms);
/* Waits for the device to finish and reports the last replay's device-side status: RAFTGP_OK,
 * or RAFTGP_ETIMEOUT if a bounded wait inside a kernel gave up (the labels are then
 * incomplete).  Synchronises. */
raftgp_status raftgp_batch_plan_check(const raftgp_batch_plan* plan);
/* The embedding of the last replay (n x d in the plan's dtype, row-major, the Z every graph's
 * model selection ran on) copied to the device buffer Z_out.  Synchronises. */
raftgp_status raftgp_batch_plan_embedding(const raftgp_batch_plan* plan, void* Z_out);
void raftgp_batch_plan_destroy(raftgp_batch_plan* plan);

/* One-shot: plan, run, synchronise, destroy. */
raftgp_status raftgp_partition_batched(const raftgp_csr* g, const int64_t* graph_off, int32_t n_graphs,
                                       const raftgp_embed_opts* eo, const raftgp_batch_opts* bo, int32_t* labels,
                                       int32_t* k_out, void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* ---- Differentiation form (the paper trains nothing: its GNN stays random, Section III-B;
 * these calls let the Eq. 6 weights be tuned against a relaxed modularity) ----
 * All arrays are device FP32, row-major; widths (lin, lout, d) are 32, 64 or 128; K <= 128.
 * H_in, H_out, dH_out, dH_in, Z and dZ start on 16-byte boundaries (RAFTGP_EINVAL otherwise).
 * Each call validates the graph on the device first (malformed graph: RAFTGP_EINVAL, nothing
 * else runs) and synchronises the stream once for that check.  `ws` is a device workspace
 * of at least raftgp_diff_workspace_size(n, width, K) bytes, width = the largest layer
 * width used, K = the largest centroid count; the caller owns every buffer. */
size_t raftgp_diff_workspace_size(int64_t n, int32_t width, int32_t K);

/* One Eq. 6 layer: H_out = rownorm(tanh(Ahat (H_in W))), Ahat = Dhat^-1/2 (A + I) Dhat^-1/2,
 * dhat = d + 1; H_in n x lin, W lin x lout, H_out n x lout; a zero row stays zero. */
raftgp_status raftgp_gcn_layer_forward(const raftgp_csr* g, const float* H_in, int32_t lin, const float* W,
                                       int32_t lout, float* H_out, void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* Gradients of that layer given dH_out = dL/dH_out (n x lout): dW (lin x lout) and, unless
 * dH_in is NULL, dH_in (n x lin).  Nothing from the forward is kept: P = H_in W and the
 * pre-activation are computed again here.  dW is summed over the points in FP64 in a fixed
 * order (deterministic). */
raftgp_status raftgp_gcn_layer_backward(const raftgp_csr* g, const float* H_in, int32_t lin, const float* W,
                                        int32_t lout, const float* dH_out, float* dH_in, float* dW, void* ws,
                                        size_t ws_bytes, raftgp_stream_t stream);

/* Relaxed modularity of the soft assignment S_i = softmax_c(-||z_i - mu_c||^2 / tau) against
 * fixed centroids mu (K x d): *loss (host) = -(tr(S^T A S) - ||d^T S||^2 / 2e) / 2e, which is
 * -Mod (Eq. 3) when S is one-hot.  Unless dZ is NULL, dZ = dL/dZ (n x d).  Synchronises. */
raftgp_status raftgp_softmod_loss(const raftgp_csr* g, const float* Z, int32_t d, const float* mu, int32_t K,
                                  float tau, double* loss, float* dZ, void* ws, size_t ws_bytes,
                                  raftgp_stream_t stream);

/* The same calls against a graph checked once.  A tuning loop makes these calls many times
 * per second: the one-shot calls above check the graph on the device and synchronise on
 * every call, the plan does so once, at creation.
 *
 * raftgp_diff_plan_create validates g (RAFTGP_EINVAL for a malformed graph, no plan made),
 * computes its degrees and the Eq. 6 normalisation into ws and synchronises the stream once.
 * width (32, 64 or 128) bounds every layer width and d of later calls, K (0..128) every
 * centroid count (0: no loss calls); ws holds at least raftgp_diff_workspace_size(n, width, K)
 * bytes.  The plan keeps copies of g's pointers and of ws: the graph's arrays and ws must
 * stay allocated and unchanged until raftgp_diff_plan_destroy.  The calls on a plan share
 * the scratch in ws, so they must be ordered on one stream (or the caller synchronises
 * between streams).  Each is asynchronous; argument errors are reported before any launch.
 *
 * raftgp_diff_plan_layer_forward / _layer_backward: as raftgp_gcn_layer_forward / _backward.
 * raftgp_diff_plan_softmod_loss: as raftgp_softmod_loss, except that `loss` is a DEVICE
 * pointer to one double, written on the stream (nothing is read back). */
typedef struct raftgp_diff_plan raftgp_diff_plan;   /* opaque */
raftgp_status raftgp_diff_plan_create(const raftgp_csr* g, int32_t width, int32_t K, void* ws, size_t ws_bytes,
                                      raftgp_stream_t stream, raftgp_diff_plan** plan);
raftgp_status raftgp_diff_plan_layer_forward(const raftgp_diff_plan* plan, const float* H_in, int32_t lin,
                                             const float* W, int32_t lout, float* H_out, raftgp_stream_t stream);
raftgp_status raftgp_diff_plan_layer_backward(const raftgp_diff_plan* plan, const float* H_in, int32_t lin,
                                              const float* W, int32_t lout, const float* dH_out, float* dH_in,
                                              float* dW, raftgp_stream_t stream);
raftgp_status raftgp_diff_plan_softmod_loss(const raftgp_diff_plan* plan, const float* Z, int32_t d,
                                            const float* mu, int32_t K, float tau, double* loss, float* dZ,
                                            raftgp_stream_t stream);
void raftgp_diff_plan_destroy(raftgp_diff_plan* plan);

/* Centroids of a labelling: mu (K x d) = the mean of the rows of each label (exact 2^-40
 * fixed-point sums, FP64 mean); an empty label gets a zero row.  labels: int32 in [0, K)
 * (RAFTGP_EINVAL otherwise).  Synchronises. */
raftgp_status raftgp_centroids(const float* Z, int64_t n, int32_t d, const int32_t* labels, int32_t K, float* mu,
                               void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* The Eq. 6 weights the embedding draws for layer `layer` (1-based) from `seed`: W (device,
 * lin x lout) = Xavier-normal, std sqrt(2 / (lin + lout)), from Philox counters (q, a, layer,
 * "Wgnn").  The starting point of a tuning run.  Asynchronous. */
raftgp_status raftgp_gcn_weights(int32_t layer, int32_t lin, int32_t lout, uint64_t seed, float* W,
                                 raftgp_stream_t stream);

/* One Adam step (Kingma and Ba, 2015) in place on count FP32 parameters: m, v are the moment
 * buffers (zero before step 1), step counts from 1.  Asynchronous. */
raftgp_status raftgp_adam_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr,
                               float beta1, float beta2, float eps, int32_t step, raftgp_stream_t stream);

/* ---- Algorithm 2 (Section IV): graphs drawn from the SBM of Definition 1 ----
 * A_ij ~ Pois(lambda_ij), lambda_ij = theta_i theta_j Omega_{c_i c_j}, for i < j (undirected,
 * no self loops); the drawn graph is the support of A (one edge per nonzero entry; its value
 * A_ij >= 1 is returned as a weight).  Each block pair r <= s has a virtual table of its
 * node pairs (row-major over the blocks' nodes in ascending order; the entries above the
 * diagonal when r = s), cut into segments of 2^16 consecutive entries; every segment runs the
 * paper's loop on its own (draw p, skip to the first entry t with RangeSum(m, t) > -ln p by
 * binary search over prefix sums of theta, draw the value Pois(lambda | >= 1), go on at t + 1).
 * Draw j of global segment g is Philox4x32-10(seed; g_lo, g_hi, j, "Sbm2").  All arrays are
 * device pointers; the caller owns them.
 *
 * raftgp_sbm_count checks the parameters (RAFTGP_EINVAL for a block outside [0, k), a
 * negative or non-finite theta or Omega), draws the graph's size and returns it in *m
 * (host); it synchronises.  raftgp_sbm_emit, called next with the same parameters and
 * workspace, writes the m edges (src[e], dst[e]: node ids; weight[e] may be NULL) in the order
 * (block pair, segment, draw); RAFTGP_EINVAL if m differs from the count's.  The workspace
 * grows as n^2 / 2^14 bytes (about 120 MB at n = 1M).
 *
 * raftgp_coo_to_csr builds the symmetric CSR of m undirected edges (both directions, every
 * row sorted): row_ptr int64[n + 1], col int32[2 m].  RAFTGP_EINVAL for an endpoint outside
 * [0, n) or a self loop, RAFTGP_EUNSUPPORTED for a row longer than 16384.  Synchronises. */
typedef struct {
    int64_t n;              /* nodes, 1 .. 2^31 - 2 */
    int32_t k;              /* blocks, >= 1 */
    const int32_t* block;   /* [n]: block c_i of node i, in [0, k) */
    const double* theta;    /* [n]: degree correction theta_i >= 0 */
    const double* omega;    /* [k * k], row-major: Omega_rs >= 0; entries with r <= s are read */
    uint64_t seed;
} raftgp_sbm;
size_t raftgp_sbm_workspace_size(int64_t n, int32_t k);
raftgp_status raftgp_sbm_count(const raftgp_sbm* p, int64_t* m, void* ws, size_t ws_bytes, raftgp_stream_t stream);
raftgp_status raftgp_sbm_emit(const raftgp_sbm* p, int32_t* src, int32_t* dst, int32_t* weight, int64_t m, void* ws,
                              size_t ws_bytes, raftgp_stream_t stream);
size_t raftgp_coo_to_csr_workspace_size(int64_t n);
raftgp_status raftgp_coo_to_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* row_ptr,
                                int32_t* col, void* ws, size_t ws_bytes, raftgp_stream_t stream);

/* ---- Streaming updates (Section III-D) ----
 * A stream owns a graph and the FP32 embedding of it with the NCut operator M (Eq. 5, Eq. 6):
 * Theta' = Theta_j d_j^-1/2, every GCN gather's input and Z, all inside the caller's workspace
 * (raftgp_stream_workspace_size; the CSR is double-buffered with room for nnz_cap stored
 * entries).  raftgp_stream_create embeds the graph in full (rows of g sorted, as everywhere).
 * raftgp_stream_add_edges adds m new undirected edges (src[e], dst[e], device int32): it
 * rejects (RAFTGP_EINVAL, stream unchanged) an endpoint outside [0, n), a self loop, an edge
 * already present or listed twice; RAFTGP_ENOMEM past nnz_cap.  It recomputes only the rows
 * whose values change -- S_0 = V' u N(V') for the projection (V' the endpoints of the new
 * edges), S_k = S_{k-1} u N(S_{k-1}) for GCN layer k -- with the same per-row kernels as a full
 * embedding, so Z equals raftgp_embed on the new graph bit for bit.  Synchronises.
 * raftgp_stream_info returns n, the stored-entry count and, per stage 0..n_layers, the rows
 * the last update recomputed (host; any pointer may be NULL).  raftgp_stream_copy copies the
 * current graph (row_ptr int64[n + 1], col int32[nnz]) and Z (FP32 n x d) into caller
 * buffers (device; any may be NULL), asynchronously on `stream`.  The modularity
 * operators and BF16 storage are not streamed (RAFTGP_EUNSUPPORTED): 2e and d^T Theta reach
 * every row. */
typedef struct raftgp_stream raftgp_stream;   /* opaque */
size_t raftgp_stream_workspace_size(int64_t n, int64_t nnz_cap, const raftgp_embed_opts* o);
raftgp_status raftgp_stream_create(const raftgp_csr* g, const raftgp_embed_opts* o, int64_t nnz_cap, void* ws,
                                   size_t ws_bytes, raftgp_stream** out, raftgp_stream_t stream);
raftgp_status raftgp_stream_add_edges(raftgp_stream* s, const int32_t* src, const int32_t* dst, int64_t m,
                                      raftgp_stream_t stream);
raftgp_status raftgp_stream_info(const raftgp_stream* s, int64_t* n, int64_t* nnz, int64_t* affected);
raftgp_status raftgp_stream_copy(const raftgp_stream* s, int64_t* row_ptr, int32_t* col, float* Z,
                                 raftgp_stream_t stream);
void raftgp_stream_destroy(raftgp_stream* s);

#ifdef __cplusplus
}
#endif

#endif /* RAFTGP_H */
