// internal.h -- declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "raftgp.h"

namespace raftgp {

int num_sms();

// Carves typed, 256-byte aligned arrays out of a caller-owned workspace; with a null base
// it only adds up the size.
// Carves a caller's workspace into 256-byte aligned pieces.  The base itself is rounded up
// to 256 bytes (every *_workspace_size() adds 256 bytes for this), so a workspace that starts
// anywhere still gives aligned pieces; bytes() is what the carve has used, counted from the
// caller's pointer.
struct Carver {
    char* base;
    size_t shift = 0;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {
        if (b) {
            shift = (size_t)((256 - ((uintptr_t)b & 255)) & 255);
            base += shift;
        }
    }
    size_t bytes() const { return shift + off; }
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};
// Records the message returned by raftgp_last_error() and returns st.
raftgp_status set_error(raftgp_status st, const char* fmt, ...);

// ---- instrumentation (prof.cu) ---------------------------------------------------------
enum ProfFamily {
    PF_DEGREES, PF_THETA, PF_SPMM_PROJ, PF_SPMM_GCN, PF_DENSE_TC, PF_SEED_UPDATE, PF_SEED_PICK, PF_BATCH_INIT, PF_ASSIGN_FFMA,
    PF_ASSIGN_TC, PF_ASSIGN_TC_FIRST, PF_ASSIGN_TC_FINAL, PF_RECHECK, PF_APPLY, PF_APPLY_FIRST, PF_LLOYD_UPDATE, PF_SCORE,
    PF_SELECT_BEST, PF_DIFF_SPMM, PF_DIFF_DENSE, PF_DIFF_LOSS, PF_DIFF, PF_OTHER, PF_ASSIGN_FFMA_FINAL, PF_COUNT
};
// Brackets the kernels launched in its lifetime with CUDA events when profiling is on.
class ProfScope {
  public:
    ProfScope(cudaStream_t s, int fam, int kernels);
    ~ProfScope();
  private:
    cudaStream_t s_;
    int fam_, kernels_;
    long long pair_;
};

// ---- embedding (embed.cu) -----------------------------------------------------------
enum { AGG_NCUT_ = 0, AGG_MOD_FULL_ = 1, AGG_MOD_REDUCED_ = 2, AGG_GCN_ = 3 };
// Degrees, scales and graph checks; if `heavy` is given, the rows gathered by a whole CTA
// (degree above 256) are listed there and counted in *heavy_count.
void launch_degrees(const raftgp_csr* g, int32_t* deg, float* rs, float* rsh, uint32_t* err, int32_t* heavy,
                    int* heavy_count, cudaStream_t s);
int theta_blocks(int64_t n);
// With `rows`, only the listed rows of Theta are written (nrows of them; no rank-one partials).
// Many graphs in one CSR (graph g owns rows off[g] .. off[g+1]-1): per graph d^T Theta from the
// stored Theta (g_graph, ng x L, FP64 sums in a fixed order, rounded to FP32) and 1 / 2e.
void launch_rank1_graphs(int ng, const int64_t* off, int L, int dtype, const void* theta, const int32_t* deg,
                         float* g_graph, double* inv_two_e_graph, cudaStream_t s);
void launch_theta(int64_t n, int L, int dtype, uint64_t seed, const float* user_theta, const float* colscale, const int32_t* local_row,
                  const int32_t* deg, void* theta, double* partial, float* gvec, cudaStream_t s,
                  const int32_t* rows = nullptr, int64_t nrows = 0);
void launch_weights(int layer, int lin, int lout, uint64_t seed, float* W, cudaStream_t s);
cudaError_t launch_layer(int agg, int dtype, const raftgp_csr* g, const int32_t* deg, const float* rowscale,
                         const float* gvec, int act, const float* W, int lin, int lout, const float* postscale,
                         const void* X, void* out, void* stage, const int32_t* heavy, const int* heavy_count,
                         cudaStream_t s, const int32_t* rows = nullptr, int64_t nrows = 0);
// BF16 gather-only layers (no fused W, not the reduced operator) as a flat stream of stored
// entries staged by cp.async (spmm_flat.cu).  `work` is a chunk counter the launch zeroes;
// nnz_g is the graph's stored-entry count (2e) for the modularity term.
bool spmm_flat_supported(int agg, int dtype, int lin);
cudaError_t launch_spmm_flat(int agg, int64_t n, int rp_bits, const void* row_ptr, const int32_t* col, int64_t nnz_g,
                             const int32_t* deg, const float* rowscale, const float* gvec, int act, int lin,
                             const void* X, void* out, void* stage, int* work, uint32_t* err, int variant,
                             cudaStream_t s, const int32_t* graph_of = nullptr, const float* g_graph = nullptr,
                             const double* inv_two_e_graph = nullptr, int ng = 0);
// CSR of A + I (row i: i, then its neighbours): rp_self has n + 1 entries, col_self nnz + n.
void launch_self_csr(const raftgp_csr* g, int64_t* rp_self, int32_t* col_self, cudaStream_t s);

// ---- device-wide inclusive scan of unsigned 64-bit values (bisect.cu) -------------------
// `tiles` holds ceil(n / SCAN_TILE) values; in and out may not overlap.
constexpr int64_t SCAN_TILE = 4096;
void scan_incl(const unsigned long long* in, int64_t n, unsigned long long* out, unsigned long long* tiles,
               cudaStream_t s);

// ---- Algorithm 2 SBM sampler and the CSR build of its output (sbm.cu) -------------------
struct SbmWs {
    uint32_t* err;
    unsigned long long *bcnt, *bincl;   // block sizes, inclusive scan
    int32_t* nodes;                     // nodes grouped by block (ascending in a block)
    double *th, *pre, *tri;             // theta in that order; per-block prefix sums
    unsigned long long *pseg, *pincl;   // segments per block pair, inclusive scan
    unsigned long long *seg_cnt, *seg_incl;   // edges per segment, inclusive scan
    uint32_t* seg_order;                      // the segments grouped by their expected draws
    uint8_t* seg_key;                         // each segment's group
    unsigned long long* bucket;               // group sizes, then their fill cursors
    unsigned long long* tiles;
};
int64_t sbm_max_segments(int64_t n, int K);
SbmWs carve_sbm(Carver& c, int64_t n, int K);
cudaError_t sbm_count(const raftgp_sbm* p, const SbmWs& w, int64_t* G_out, int64_t* m_out, cudaStream_t s);
cudaError_t sbm_emit(const raftgp_sbm* p, const SbmWs& w, int64_t G, int32_t* src, int32_t* dst, int32_t* weight,
                     cudaStream_t s);
struct CsrBuildWs {
    uint32_t* err;
    unsigned long long *deg, *incl, *fill, *tiles;
    int* long_rows;
    int* n_long;
};
CsrBuildWs carve_csr_build(Carver& c, int64_t n);
// Sorts every CSR row (or those with only[i] != 0) in place; long_rows holds n entries; a
// row longer than 16384 sets DERR_ROW_PTR in *err and stays unsorted.
cudaError_t sort_csr_rows(const int64_t* row_ptr, int64_t n, int32_t* col, const uint8_t* only, int* long_rows,
                          int* n_long, uint32_t* err, cudaStream_t s);
// Blocks for a grid-stride loop over `items` (at most 16 per SM).
int grid_for(int64_t items, int threads);
cudaError_t coo_to_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* row_ptr, int32_t* col,
                       const CsrBuildWs& w, uint32_t* herr, cudaStream_t s);

// ---- dense layer on tensor cores (dense_tc.cu) -----------------------------------------
void launch_w_split(const float* W, int lin, int lout, __nv_bfloat16* whi, __nv_bfloat16* wlo, cudaStream_t s);
cudaError_t launch_dense_tc(int lin, int lout, int64_t n, const void* X, const __nv_bfloat16* whi,
                            const __nv_bfloat16* wlo, const float* scale, void* out, uint32_t* err, cudaStream_t s);

// ---- k-means (kmeans.cu) --------------------------------------------------------------
constexpr int MAXC = RAFTGP_MAX_BATCH_CAND;

// One batch of candidates evaluated together; passed by value to every kernel.
struct CandBatch {
    int n;              // candidates in the batch
    int total_k;        // columns of the batch: the sum of the padded k[]
    int cs;             // label row stride (n rounded up to a multiple of 8)
    int k[MAXC];        // K of each candidate
    int off[MAXC];      // first centroid of each candidate (multiples of 64: candidates padded)
};

struct KmState {                 // device arrays of one batch (workspace)
    float* mu;                   // total_k x d FP32 centroids
    float* muT;                  // d x kpad: the same, k-major (row k holds coordinate k of every centroid)
    float* norm2;                // total_k, ||mu||^2 in FP32
    float* norm2p;               // kpad, ||mu||^2 + 4 (tensor-core epilogue: positive scores)
    long long* sums;             // total_k x d, 2^-40 fixed point
    int32_t* counts;             // total_k
    int16_t* labels;             // N x cs
    int16_t* labels_new;         // N x cs: tensor-core pass output before the changes are applied
    int32_t* active;             // MAXC
    int32_t* changed;            // 2 x MAXC (double-buffered by pass parity)
    int32_t* passes;             // MAXC
    __nv_bfloat16* bhi;          // kpad x d: BF16 rounding of -mu (tensor-core operand)
    __nv_bfloat16* blo;          // kpad x d: BF16 rounding of -mu - hi
    __nv_bfloat16* baug;         // kpad x 16: the norm slice [(||mu||^2+4)/2 hi, lo, 0...]
    int64_t bhi_rows;            // kpad (total_k rounded up, so chunk loads stay in bounds)
};

// k-means++ seeding scratch (carved from one region by carve_seed)
struct SeedState {
    float* D2;                     // n: squared distance to the nearest seed so far
    int16_t* nearest;              // n: index (into seeds) of that seed
    uint8_t* chosen;               // n: already a seed
    unsigned long long* blocksum;  // seed_nblocks(n): block sums of the quantised D^2
    float* cc2;                    // K: squared distance from each seed to the newest one
    unsigned* bar;                 // 4 words: grid barrier count, generation, abort; spare error word
    uint32_t* err;                 // device error word (DERR_TIMEOUT); bar + 3 unless the caller has one
    int32_t* seeds;                // K (caller's output)
    void* zs;                      // optional sector-major copy of Z (n x d elements), or null
};
int seed_nblocks(int64_t n);
size_t seed_scratch_bytes(int64_t n, int K);
SeedState carve_seed(void* base, int64_t n, int K, int32_t* seeds);
cudaError_t launch_seeding(const void* Z, int zdtype, int64_t n, int d, int K, uint64_t seed, SeedState ss,
                           cudaStream_t s);
void set_seed_skip_block(int block);   // test hook of the persistent seeding

void launch_batch_init(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, const int32_t* seeds,
                       const float* mu0, KmState st, cudaStream_t s);
cudaError_t launch_assign_ffma(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, KmState st, int pass,
                               int final_mode, int2* recheck, int* recheck_count, cudaStream_t s);
float ffma_tie_band(int d);
void launch_lloyd_update(const CandBatch& b, int d, KmState st, int pass, int last_pass, cudaStream_t s);
void launch_apply_changes(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, KmState st, int pass,
                          cudaStream_t s);
cudaError_t launch_assign_tc(const CandBatch& b, const void* Z, int64_t n, int d, KmState st, int pass, int final_mode,
                             int fast_lo, int2* recheck, int* recheck_count, uint32_t* err, cudaStream_t s);
void launch_recheck(const CandBatch& b, const void* Z, int zdtype, int d, KmState st, const int2* list,
                    const int* count, int fp64, cudaStream_t s);
float tc_tie_band(int d);

// ---- scoring (score.cu) ---------------------------------------------------------------
struct ScoreOut {                // per batch
    long long* m;                // total_k, directed intra-block entry counts
    long long* vol;              // total_k
    double* mod;                 // MAXC
    double* ncut;                // MAXC
};
struct BestState {               // across batches
    double mod, ncut;
    int32_t k;
    int32_t has;
    int32_t copy_from;           // batch candidate to copy labels from, or -1
};

void launch_score_batch(const CandBatch& b, const raftgp_csr* g, const int32_t* deg, const int16_t* labels,
                        ScoreOut so, uint32_t* err, cudaStream_t s);
void launch_select_best(const CandBatch& b, ScoreOut so, int criterion, BestState* best, const int16_t* labels,
                        int64_t n, int32_t* out_labels, cudaStream_t s);
cudaError_t launch_score_labels(const raftgp_csr* g, const int32_t* deg, const int32_t* labels, int K, long long* m,
                                long long* vol, double* out2, uint32_t* err, cudaStream_t s);

// ---- differentiation form (diff.cu) ----
cudaError_t launch_rowmm(int64_t n, const float* X, int lin, const float* W, int lout, bool trans, float* Y,
                         cudaStream_t s);
// mode: 0 GCN forward, 1 GCN backward (dA), 2 Ahat x, 3 A x
cudaError_t launch_spmm32(const raftgp_csr* g, int L, const float* rsh, const float* X, const float* G, float* out,
                          int mode, cudaStream_t s);
int wgrad_blocks(int64_t n);
cudaError_t launch_wgrad(int64_t n, const float* H, int lin, const float* dP, int lout, float* partial, float* dW,
                         cudaStream_t s);
int softmod_blocks(int64_t n);
cudaError_t launch_soft_assign(int64_t n, int d, const float* Z, const float* mu, int K, float tau, float* S,
                               cudaStream_t s);
cudaError_t launch_softmod_reduce(int64_t n, const int32_t* deg, const float* S, const float* AS, int K,
                                  double two_e, double* partial, double* red, cudaStream_t s);
cudaError_t launch_softmod_grad(int64_t n, int d, const float* Z, const float* mu, int K, float tau, const int32_t* deg,
                                const float* S, const float* AS, const double* red, double two_e, float* dZ,
                                cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s);
cudaError_t launch_centroids(int64_t n, int d, const float* Z, const int32_t* labels, int K, long long* sums,
                             int* counts, float* mu, uint32_t* err, cudaStream_t s);

// ---- many graphs at once (batched.cu) ----
constexpr int BATCH_COARSE = 10;   // candidate slots 0..9: the coarse grid
constexpr int BATCH_SLOTS = 20;    // slots 10..19: the refined grid
constexpr int BATCH_KMAX = 128;    // largest K of a graph in the batch
struct BatchDev {
    int ng;                        // graphs
    int64_t total_n;               // nodes of all graphs
    const int64_t* node_off;       // ng + 1
    const int32_t* kmax;           // ng
    const int32_t* seed_off;       // ng + 1: each graph's seeds in `seeds`
    const int32_t* order;          // ng: graphs by decreasing size (work order)
    int32_t* local_row;            // total_n: index of the node inside its graph
    int32_t* graph_of;             // total_n: the node's graph
    int32_t* seeds;                // sum of kmax
    int32_t* cand_k;               // ng x BATCH_SLOTS
    int32_t* n_coarse;             // ng
    int32_t* n_refine;             // ng
    double* cand_mod;              // ng x BATCH_SLOTS
    double* cand_ncut;             // ng x BATCH_SLOTS
    int32_t* cand_passes;          // ng x BATCH_SLOTS
    int16_t* labels;               // BATCH_SLOTS x total_n
    float* D2;                     // total_n (seeding)
    uint8_t* chosen;               // total_n (seeding)
    int* queue;                    // 4 work counters
};
size_t batch_lloyd_smem(int d);
void launch_batch_prologue(BatchDev b, int kmin, int G, cudaStream_t s);
cudaError_t launch_batch_seed(BatchDev b, const void* Z, int zdtype, int d, uint64_t seed, cudaStream_t s);
cudaError_t launch_batch_lloyd(BatchDev b, const void* Z, int zdtype, int d, int phase, int iters, const raftgp_csr* g,
                               int threads, int ppt, cudaStream_t s);
// tensor-core Lloyd of the batched form (BF16 embeddings, d = 32 or 64); stg: a device staging
// area of batch_tc_staging_bytes(d) for the centroid operands and the per-CTA centroid sums
size_t batch_tc_staging_bytes(int d);
cudaError_t launch_batch_lloyd_tc(BatchDev b, const void* Z, int d, int phase, int iters, int lo_fast,
                                  const raftgp_csr* g, void* stg, uint32_t* err, cudaStream_t s);
void launch_batch_refine(BatchDev b, int G, int criterion, cudaStream_t s);
void launch_batch_select(BatchDev b, int criterion, int32_t* labels_out, int32_t* k_out, cudaStream_t s);
void launch_batch_check(const raftgp_csr* g, int ng, const int64_t* node_off, uint32_t* err, cudaStream_t s);

// ---- Algorithm 1, recursive bisection (bisect.cu) ----
struct BisectDev {
    int eps, depth, cap_sets;
    // per position (current level)
    int32_t *perm, *perm_next, *pos_set;
    int8_t* lab;
    unsigned long long *q, *P, *F, *tiles;
    // per node
    int32_t *node_set, *node_lab, *block_of;
    // per set (current / next level)
    int64_t *set_off, *set_n, *nset_off, *nset_n;
    uint64_t *set_id, *nset_id;
    int64_t *s0, *child_pos;
    int32_t *active, *changed, *counts, *split, *block_id;
    float *mu, *norm2;
    long long* sums;
    unsigned long long *acc, *scan_in, *scan_out;
    int32_t* bmin;
    int* counters;
    long long* counters_ll;
    // tree ids of the final blocks (per node; may be null) and the streaming update's inputs:
    // the previous run's labels (k_old blocks) and leaf ids, and the nodes whose embedding or
    // degree changed (null in a full run)
    uint64_t* leaf_of;
    const int32_t* old_label;
    const uint64_t* old_leaf;
    const uint8_t* dirty;
    int k_old;
    // per set (current / next level): the set is the previous tree's node of the same id and
    // every ancestor split as before (1), or it is new (0); frozen: kept with its old subtree;
    // flag: a changed node inside (before the decision) or a changed split (after it)
    int32_t *set_keep, *nset_keep, *frozen, *flag;
};
cudaError_t launch_bisect(const raftgp_csr* g, const void* Z, int zdtype, int d, BisectDev b, int iters, uint64_t seed,
                          int reading, int32_t* labels, int32_t* k_out, cudaStream_t s);

}  // namespace raftgp
