// api.cu -- the C ABI (include/raftgp.h): argument checks, workspace layout and the order of
// kernel launches for each entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

static thread_local std::string g_last_error;

static raftgp_status fail(raftgp_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

raftgp_status set_error(raftgp_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

static raftgp_status cuda_fail(cudaError_t e, const char* where) {
    return fail(RAFTGP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Bump allocator over the caller's workspace (base == nullptr measures only).
static size_t elem_size(int dtype) { return dtype == RAFTGP_BF16 ? 2 : 4; }
static bool width_ok(int w) { return w == 32 || w == 64 || w == 128; }

static raftgp_status check_csr(const raftgp_csr* g) {
    if (!g) return fail(RAFTGP_EINVAL, "graph is NULL");
    if (g->n < 1) return fail(RAFTGP_EINVAL, "graph has n = %lld < 1", (long long)g->n);
    if (g->n > (int64_t)INT32_MAX - 1) return fail(RAFTGP_EUNSUPPORTED, "n above 2^31-2 is not supported");
    if (g->nnz < 0) return fail(RAFTGP_EINVAL, "nnz < 0");
    if (g->row_ptr_bits != 32 && g->row_ptr_bits != 64) return fail(RAFTGP_EINVAL, "row_ptr_bits must be 32 or 64");
    if (g->row_ptr_bits == 32 && g->nnz > (int64_t)INT32_MAX) return fail(RAFTGP_EINVAL, "nnz exceeds int32 row_ptr");
    if (!g->row_ptr || (g->nnz > 0 && !g->col)) return fail(RAFTGP_EINVAL, "graph arrays are NULL");
    if (g->nnz >= ((int64_t)1 << 31)) return fail(RAFTGP_EUNSUPPORTED, "nnz of 2^31 or more is not supported");
    return RAFTGP_OK;
}

static raftgp_status check_embed(const raftgp_embed_opts* o) {
    if (!o) return fail(RAFTGP_EINVAL, "embed options are NULL");
    if (o->op < RAFTGP_OP_NCUT || o->op > RAFTGP_OP_MOD_REDUCED) return fail(RAFTGP_EINVAL, "unknown operator %d", o->op);
    if (o->n_layers < 0 || o->n_layers > RAFTGP_MAX_LAYERS) return fail(RAFTGP_EINVAL, "n_layers out of range");
    for (int k = 0; k <= o->n_layers; ++k)
        if (!width_ok(o->dims[k])) return fail(RAFTGP_EUNSUPPORTED, "dims[%d] = %d: widths must be 32, 64 or 128", k, o->dims[k]);
    if (o->dtype != RAFTGP_F32 && o->dtype != RAFTGP_BF16) return fail(RAFTGP_EINVAL, "unknown dtype");
    return RAFTGP_OK;
}

static raftgp_status check_select(const raftgp_select_opts* o, int64_t n) {
    if (!o) return fail(RAFTGP_EINVAL, "select options are NULL");
    if (o->kmin < 1 || o->kmax < o->kmin) return fail(RAFTGP_EINVAL, "need 1 <= kmin <= kmax");
    if (std::min<int64_t>(o->kmax, n) < o->kmin) return fail(RAFTGP_EINVAL, "kmin exceeds the number of nodes");
    if (std::min<int64_t>(o->kmax, n) > 32767) return fail(RAFTGP_EUNSUPPORTED, "K above 32767 is not supported");
    if (o->grid < 0 || o->grid > RAFTGP_MAX_BATCH_CAND) return fail(RAFTGP_EINVAL, "grid out of range");
    if (o->iters < 1) return fail(RAFTGP_EINVAL, "iters must be >= 1");
    if (o->criterion != RAFTGP_CRIT_MOD && o->criterion != RAFTGP_CRIT_NCUT) return fail(RAFTGP_EINVAL, "unknown criterion");
    if (o->assign < RAFTGP_ASSIGN_FFMA || o->assign > RAFTGP_ASSIGN_TC8) return fail(RAFTGP_EINVAL, "unknown assign engine");
    if (o->recheck < RAFTGP_RECHECK_NONE || o->recheck > RAFTGP_RECHECK_FP64)
        return fail(RAFTGP_EINVAL, "unknown recheck mode");
    if (o->batch < 0) return fail(RAFTGP_EINVAL, "batch < 0");
    return RAFTGP_OK;
}

// ------------------------------------------------------------------------------------
// Workspace layouts
// ------------------------------------------------------------------------------------
struct EmbedWs {
    uint32_t* err;
    int32_t* deg;
    float* rs;
    float* rsh;
    int32_t* heavy;        // rows of degree above 256 (gathered by a whole CTA)
    int* heavy_count;
    int* work;             // chunk counters of the BF16 flat-stream gathers, one per layer
    int64_t* rp_self;      // BF16 GCN gathers: CSR of A + I (null otherwise)
    int32_t* col_self;
    float* W[RAFTGP_MAX_LAYERS];
    __nv_bfloat16* Whi[RAFTGP_MAX_LAYERS];  // BF16 form: W^T split into hi and lo for the tensor cores
    __nv_bfloat16* Wlo[RAFTGP_MAX_LAYERS];
    double* partial;
    float* gvec;
    void* bufA;
    void* bufB;
    const int32_t* local_row;   // many graphs in one CSR: each node's index inside its graph
    int flat_variant;           // shape of the BF16 flat-stream gathers (0: the default)
    // many graphs in one CSR with the full modularity operator: per-graph rank-one terms
    int ng;
    const int64_t* graph_off;   // ng + 1
    const int32_t* graph_of;    // n: each node's graph
    float* g_graph;             // ng x L: d^T Theta per graph
    double* inv_two_e_graph;    // ng
};

static int embed_maxw(const raftgp_embed_opts* o) {
    int w = o->dims[0];
    for (int k = 1; k <= o->n_layers; ++k) w = std::max(w, o->dims[k]);
    return w;
}

static EmbedWs carve_embed(Carver& c, int64_t n, int64_t nnz, const raftgp_embed_opts* o) {
    EmbedWs w{};
    w.err = c.take<uint32_t>(64);
    w.deg = c.take<int32_t>(n);
    w.rs = c.take<float>(n);
    w.rsh = c.take<float>(n);
    w.heavy = c.take<int32_t>(n);
    w.heavy_count = c.take<int>(64);
    w.work = c.take<int>(64);
    if (o->dtype == RAFTGP_BF16 && o->n_layers >= 1) {
        w.rp_self = c.take<int64_t>(n + 1);
        w.col_self = c.take<int32_t>(nnz + n);
    }
    for (int k = 1; k <= o->n_layers; ++k) {
        w.W[k - 1] = c.take<float>((size_t)o->dims[k - 1] * o->dims[k]);
        w.Whi[k - 1] = c.take<__nv_bfloat16>((size_t)o->dims[k - 1] * o->dims[k]);
        w.Wlo[k - 1] = c.take<__nv_bfloat16>((size_t)o->dims[k - 1] * o->dims[k]);
    }
    const int L = o->dims[0];
    w.partial = c.take<double>((size_t)theta_blocks(n) * L);
    w.gvec = c.take<float>(L);
    const size_t row = (size_t)embed_maxw(o) * elem_size(o->dtype);
    w.bufA = c.take<char>(row * (size_t)n);
    w.bufB = c.take<char>(row * (size_t)n);
    return w;
}

struct SelectWs {
    uint32_t* err;
    int32_t* deg;
    float* rs;
    float* rsh;
    SeedState seed;
    int32_t* seeds;
    KmState km;
    ScoreOut so;
    BestState* best;
    int2* recheck;
    int* recheck_count;
    int cmax;   // candidates per batch
    int kcap;   // centroids per batch
};

static int64_t kpad_of(int64_t k) { return (k + 255) / 256 * 256; }
static int pad64h(int k) { return (k + 63) / 64 * 64; }
// Most centroid columns one batch may hold (every candidate padded to a multiple of 64).
constexpr int kMaxBatchCols = 65536;

static void carve_km(Carver& c, KmState& km, int64_t kcap, int d, int64_t n, int cs) {
    const int64_t kp = kpad_of(kcap);
    km.mu = c.take<float>((size_t)kp * d);
    km.muT = c.take<float>((size_t)kp * d);
    km.norm2 = c.take<float>(kp + 64);
    km.norm2p = c.take<float>(kp + 64);
    km.sums = c.take<long long>((size_t)kp * d);
    km.counts = c.take<int32_t>(kp);
    km.labels = c.take<int16_t>((size_t)n * cs);
    km.labels_new = c.take<int16_t>((size_t)n * cs);
    km.active = c.take<int32_t>(MAXC);
    km.changed = c.take<int32_t>(2 * MAXC);
    km.passes = c.take<int32_t>(MAXC);
    km.bhi = c.take<__nv_bfloat16>((size_t)kp * d);
    km.blo = c.take<__nv_bfloat16>((size_t)kp * d);
    km.baug = c.take<__nv_bfloat16>((size_t)kp * 16);
    km.bhi_rows = kp;
}

static int batch_cap(const raftgp_select_opts* o, int kmax) {
    int span = o->grid > 0 ? o->grid : (kmax - o->kmin + 1);
    int c = o->batch == 0 ? RAFTGP_MAX_BATCH_CAND : std::min(o->batch, RAFTGP_MAX_BATCH_CAND);
    return std::max(1, std::min(c, span));
}

static SelectWs carve_select(Carver& c, int64_t n, int d, const raftgp_select_opts* o, uint32_t* err, int32_t* deg) {
    SelectWs w{};
    const int kmax = (int)std::min<int64_t>(o->kmax, n);
    w.err = err ? err : c.take<uint32_t>(64);
    if (deg) {
        w.deg = deg;
    } else {
        w.deg = c.take<int32_t>(n);
        w.rs = c.take<float>(n);
        w.rsh = c.take<float>(n);
    }
    w.seeds = c.take<int32_t>(kmax);
    w.seed = carve_seed(c.take<char>(seed_scratch_bytes(n, kmax)), n, kmax, w.seeds);
    w.seed.err = w.err;   // a seeding timeout is reported with the other device errors
    w.seed.zs = c.take<float>((size_t)n * d);   // the sector-major copy of Z for the seeding
    w.cmax = batch_cap(o, kmax);
    w.kcap = (int)std::min<int64_t>((int64_t)w.cmax * pad64h(kmax), kMaxBatchCols > pad64h(kmax) ? kMaxBatchCols : pad64h(kmax));
    const int cs = (w.cmax + 7) / 8 * 8;
    carve_km(c, w.km, w.kcap, d, n, cs);
    w.recheck = c.take<int2>((size_t)n * w.cmax);
    w.recheck_count = c.take<int>(64);
    w.so.m = c.take<long long>(w.kcap);
    w.so.vol = c.take<long long>(w.kcap);
    w.so.mod = c.take<double>(MAXC);
    w.so.ncut = c.take<double>(MAXC);
    w.best = c.take<BestState>(1);
    return w;
}

static raftgp_status read_error_word(const uint32_t* err, cudaStream_t s);

// ------------------------------------------------------------------------------------
// Embedding
// ------------------------------------------------------------------------------------
static raftgp_status run_embed(const raftgp_csr* g, const raftgp_embed_opts* o, void* Z, const EmbedWs& w,
                               bool degrees_done, cudaStream_t s) {
    const int64_t n = g->n;
    const int L = o->dims[0];
    if (!degrees_done) {
        launch_degrees(g, w.deg, w.rs, w.rsh, w.err, w.heavy, w.heavy_count, s);
        // no gather runs on a graph that failed the device checks
        raftgp_status st = read_error_word(w.err, s);
        if (st != RAFTGP_OK) return st;
    }
    for (int k = 1; k <= o->n_layers; ++k) {
        if (o->W[k - 1]) {
            cudaMemcpyAsync(w.W[k - 1], o->W[k - 1], sizeof(float) * (size_t)o->dims[k - 1] * o->dims[k],
                            cudaMemcpyDeviceToDevice, s);
        } else {
            launch_weights(k, o->dims[k - 1], o->dims[k], o->seed, w.W[k - 1], s);
        }
    }
    const bool rank1 = o->op == RAFTGP_OP_MOD_FULL;
    const bool per_graph = rank1 && w.graph_of;   // several graphs: a rank-one term per graph
    // Theta (prescaled by rs_j for the NCut operator) into bufB
    launch_theta(n, L, o->dtype, o->seed, o->theta, o->op == RAFTGP_OP_NCUT ? w.rs : nullptr, w.local_row, w.deg, w.bufB,
                 rank1 && !per_graph ? w.partial : nullptr, w.gvec, s);
    if (per_graph) launch_rank1_graphs(w.ng, w.graph_off, L, o->dtype, w.bufB, w.deg, w.g_graph, w.inv_two_e_graph, s);
    const int32_t* pg_of = per_graph ? w.graph_of : nullptr;
    const int agg0 = o->op == RAFTGP_OP_NCUT ? AGG_NCUT_ : (rank1 ? AGG_MOD_FULL_ : AGG_MOD_REDUCED_);
    cudaError_t e;
    // BF16 gathers without a fused weight product run as flat entry streams (spmm_flat.cu)
    const bool flat0 = spmm_flat_supported(agg0, o->dtype, L);
    if (o->n_layers == 0) {
        if (flat0)
            e = launch_spmm_flat(agg0, n, g->row_ptr_bits, g->row_ptr, g->col, g->nnz, w.deg, w.rs, w.gvec, 2, L,
                                 w.bufB, Z, o->stage_out[0], w.work, w.err, w.flat_variant, s, pg_of, w.g_graph,
                                 w.inv_two_e_graph, w.ng);
        else
            e = launch_layer(agg0, o->dtype, g, w.deg, w.rs, w.gvec, 2, nullptr, L, L, nullptr, w.bufB, Z,
                             o->stage_out[0], w.heavy, w.heavy_count, s);
        if (e != cudaSuccess) return cuda_fail(e, "projection");
        return RAFTGP_OK;
    }
    if (o->dtype == RAFTGP_BF16) {
        // BF16: every SpMM is a pure gather with its row epilogue; the weight products run as
        // tensor-core GEMMs (bufA / bufB alternate: the gather reads one, writes the other).
        // The GCN gathers walk the CSR of A + I, so the self loop is one more stored entry.
        for (int k = 1; k <= o->n_layers; ++k) launch_w_split(w.W[k - 1], o->dims[k - 1], o->dims[k], w.Whi[k - 1],
                                                              w.Wlo[k - 1], s);
        launch_self_csr(g, w.rp_self, w.col_self, s);
        if (flat0)
            e = launch_spmm_flat(agg0, n, g->row_ptr_bits, g->row_ptr, g->col, g->nnz, w.deg, w.rs, w.gvec, 0, L,
                                 w.bufB, w.bufA, o->stage_out[0], w.work, w.err, w.flat_variant, s, pg_of, w.g_graph,
                                 w.inv_two_e_graph, w.ng);
        else
            e = launch_layer(agg0, o->dtype, g, w.deg, w.rs, w.gvec, 0, nullptr, L, L, nullptr, w.bufB, w.bufA,
                             o->stage_out[0], w.heavy, w.heavy_count, s);
        if (e != cudaSuccess) return cuda_fail(e, "projection");
        e = launch_dense_tc(L, o->dims[1], n, w.bufA, w.Whi[0], w.Wlo[0], w.rsh, w.bufB, w.err, s);
        if (e != cudaSuccess) return cuda_fail(e, "dense layer");
        for (int k = 1; k <= o->n_layers; ++k) {
            const bool last = k == o->n_layers;
            if (spmm_flat_supported(AGG_GCN_, o->dtype, o->dims[k]))
                e = launch_spmm_flat(AGG_GCN_, n, 64, w.rp_self, w.col_self, g->nnz, w.deg, w.rsh, nullptr, 1,
                                     o->dims[k], w.bufB, last ? Z : w.bufA, o->stage_out[k], w.work + k, w.err, w.flat_variant, s);
            else
                e = launch_layer(AGG_GCN_, o->dtype, g, w.deg, w.rsh, nullptr, 1, nullptr, o->dims[k], o->dims[k],
                                 nullptr, w.bufB, last ? Z : w.bufA, o->stage_out[k], w.heavy, w.heavy_count, s);
            if (e != cudaSuccess) return cuda_fail(e, "gcn layer");
            if (!last) {
                e = launch_dense_tc(o->dims[k], o->dims[k + 1], n, w.bufA, w.Whi[k], w.Wlo[k], w.rsh, w.bufB, w.err, s);
                if (e != cudaSuccess) return cuda_fail(e, "dense layer");
            }
        }
        return RAFTGP_OK;
    }
    // FP32: layer 0 is the projection then x W1, prescaled by rsh for the first GCN gather
    e = launch_layer(agg0, o->dtype, g, w.deg, w.rs, w.gvec, 0, w.W[0], L, o->dims[1], w.rsh, w.bufB, w.bufA,
                     o->stage_out[0], w.heavy, w.heavy_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "projection");
    void* cur = w.bufA;
    void* nxt = w.bufB;
    for (int k = 1; k <= o->n_layers; ++k) {
        const bool last = k == o->n_layers;
        e = launch_layer(AGG_GCN_, o->dtype, g, w.deg, w.rsh, nullptr, 1, last ? nullptr : w.W[k], o->dims[k],
                         last ? o->dims[k] : o->dims[k + 1], last ? nullptr : w.rsh, cur, last ? Z : nxt,
                         o->stage_out[k], w.heavy, w.heavy_count, s);
        if (e != cudaSuccess) return cuda_fail(e, "gcn layer");
        std::swap(cur, nxt);
    }
    return RAFTGP_OK;
}

static raftgp_status read_error_word(const uint32_t* err, cudaStream_t s) {
    uint32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    if (h & (DERR_COL_RANGE | DERR_ROW_PTR | DERR_SELF_LOOP))
        return fail(RAFTGP_EINVAL, "malformed graph (device check flags 0x%x)", h);
    if (h & DERR_LABEL_RANGE) return fail(RAFTGP_EINVAL, "a label is outside [0, K)");
    if (h & DERR_NORM) return fail(RAFTGP_EINVAL, "an embedding row has norm above 1");
    if (h & DERR_TIMEOUT) return fail(RAFTGP_ETIMEOUT, "a bounded device wait timed out");
    if (h & DERR_BOUNDS) return fail(RAFTGP_ECUDA, "an internal index check failed (flags 0x%x)", h);
    return RAFTGP_OK;
}

// ------------------------------------------------------------------------------------
// Candidate grids (Section III-C model selection over K)
// ------------------------------------------------------------------------------------
static std::vector<int> coarse_grid(int kmin, int kmax, int G) {
    std::vector<int> out;
    if (G == 1) { out.push_back(kmin); return out; }
    for (int t = 0; t < G; ++t) {
        const int64_t num = 2 * (int64_t)(kmax - kmin) * t + (G - 1);
        const int k = kmin + (int)(num / (2 * (int64_t)(G - 1)));
        if (out.empty() || out.back() != k) out.push_back(k);
    }
    return out;
}

static std::vector<int> refine_grid(int lo, int hi, int G, const std::vector<int>& done) {
    std::vector<int> out;
    for (int t = 1; t <= G; ++t) {
        const int64_t num = 2 * (int64_t)(hi - lo) * t + (G + 1);
        const int k = lo + (int)(num / (2 * (int64_t)(G + 1)));
        if (std::find(done.begin(), done.end(), k) == done.end() && std::find(out.begin(), out.end(), k) == out.end())
            out.push_back(k);
    }
    return out;
}

struct CandRecord {
    int k;
    double mod, ncut;
    int passes;
};

static bool host_better(int criterion, const CandRecord& a, const CandRecord& b) {
    if (criterion == RAFTGP_CRIT_NCUT) {
        if (a.ncut != b.ncut) return a.ncut < b.ncut;
    } else {
        if (a.mod != b.mod) return a.mod > b.mod;
    }
    return a.k < b.k;
}

// Lloyd passes for one batch.  Tensor-core engine: FAST passes, then one FINAL assignment (the
// reported labels) whose near ties are re-checked in the direct form (FP32, or FP64 for
// recheck = 2).  FP32 engine: its passes already report the FP32 argmin; recheck = 2 adds a
// FINAL pass that lists its near ties for the FP64 re-check.
static raftgp_status run_lloyd(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, int iters, int engine,
                               int recheck, KmState km, int2* recheck_list, int* recheck_count, uint32_t* err,
                               cudaStream_t s) {
    const bool tc = engine != RAFTGP_ASSIGN_FFMA;
    for (int pass = 1; pass <= iters; ++pass) {
        cudaError_t e = tc ? launch_assign_tc(b, Z, n, d, km, pass, 0, engine == RAFTGP_ASSIGN_TC ? 1 : 0, nullptr,
                                              nullptr, err, s)
                           : launch_assign_ffma(b, Z, zdtype, n, d, km, pass, 0, nullptr, nullptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "assign");
        if (tc) launch_apply_changes(b, Z, zdtype, n, d, km, pass, s);
        launch_lloyd_update(b, d, km, pass, iters, s);
    }
    if (tc || recheck == RAFTGP_RECHECK_FP64) {
        cudaMemsetAsync(recheck_count, 0, sizeof(int), s);
        cudaError_t e = tc ? launch_assign_tc(b, Z, n, d, km, iters + 1, 1, 1, recheck_list, recheck_count, err, s)
                           : launch_assign_ffma(b, Z, zdtype, n, d, km, iters + 1, 1, recheck_list, recheck_count, s);
        if (e != cudaSuccess) return cuda_fail(e, "final assign");
        if (recheck != RAFTGP_RECHECK_NONE)
            launch_recheck(b, Z, zdtype, d, km, recheck_list, recheck_count, recheck == RAFTGP_RECHECK_FP64 ? 1 : 0, s);
    }
    return RAFTGP_OK;
}

// Evaluate a list of candidates in batches; appends their records.
static raftgp_status run_candidates(const raftgp_csr* g, const void* Z, int d, int zdtype,
                                    const raftgp_select_opts* o, const std::vector<int>& ks, const SelectWs& w,
                                    int32_t* labels, std::vector<CandRecord>& rec, cudaStream_t s) {
    const int64_t n = g->n;
    for (size_t b0 = 0; b0 < ks.size();) {
        // a batch: up to cmax candidates whose padded centroid ranges fit the workspace
        CandBatch b{};
        int off = 0;
        while (b.n < w.cmax && b0 + b.n < ks.size() && (b.n == 0 || off + pad64h(ks[b0 + b.n]) <= w.kcap)) {
            b.k[b.n] = ks[b0 + b.n];
            b.off[b.n] = off;
            off += pad64h(b.k[b.n]);
            ++b.n;
        }
        b0 += b.n;
        b.cs = (b.n + 7) / 8 * 8;
        b.total_k = off;
        launch_batch_init(b, Z, zdtype, n, d, w.seeds, nullptr, w.km, s);
        raftgp_status st = run_lloyd(b, Z, zdtype, n, d, o->iters, o->assign, o->recheck, w.km, w.recheck, w.recheck_count,
                                     w.err, s);
        if (st != RAFTGP_OK) return st;
        launch_score_batch(b, g, w.deg, w.km.labels, w.so, w.err, s);
        launch_select_best(b, w.so, o->criterion, w.best, w.km.labels, n, labels, s);
        double hm[MAXC], hn[MAXC];
        int32_t hp[MAXC];
        cudaMemcpyAsync(hm, w.so.mod, sizeof(double) * b.n, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hn, w.so.ncut, sizeof(double) * b.n, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hp, w.km.passes, sizeof(int32_t) * b.n, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "candidate batch");
        for (int c = 0; c < b.n; ++c) rec.push_back(CandRecord{b.k[c], hm[c], hn[c], hp[c]});
    }
    return RAFTGP_OK;
}

// Thread per 16-byte chunk of Z (coalesced); the G = d * elem / 16 lanes of a row (4 to 32,
// aligned groups of a warp) add their squares with shuffles.
__global__ void k_check_norms(const void* Z, int zdtype, int64_t n, int d, uint32_t* err) {
    const bool bf = zdtype == RAFTGP_BF16;
    const int G = d * (bf ? 2 : 4) / 16;
    const int64_t chunks = n * G;
    // unit rows stored in BF16 round to norms up to (1 + 2^-8)^2; FP32 to 1 + a few ulp
    const float lim = bf ? 1.02f : 1.0001f;
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x; q0 < chunks; q0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = q0 + threadIdx.x;
        float s = 0.f;
        if (q < chunks) {
            const uint4 v = reinterpret_cast<const uint4*>(Z)[q];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (bf) {
                    const float a = __uint_as_float(w[i] << 16), b = __uint_as_float(w[i] & 0xffff0000u);
                    s = fmaf(a, a, s);
                    s = fmaf(b, b, s);
                } else {
                    const float a = __uint_as_float(w[i]);
                    s = fmaf(a, a, s);
                }
            }
        }
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (q < chunks && q % G == 0 && !(s <= lim)) flag_error(err, DERR_NORM);
    }
}

static raftgp_status run_select(const raftgp_csr* g, const void* Z, int d, int zdtype, const raftgp_select_opts* o,
                                int32_t* labels, raftgp_select_result* res, const SelectWs& w, bool degrees_done,
                                cudaStream_t s) {
    const int64_t n = g->n;
    const int kmax = (int)std::min<int64_t>(o->kmax, n);
    if (!degrees_done) {
        cudaMemsetAsync(w.err, 0, sizeof(uint32_t), s);
        launch_degrees(g, w.deg, w.rs, w.rsh, w.err, nullptr, nullptr, s);
    }
    {
        const int64_t chunks = n * (int64_t)(d * (zdtype == RAFTGP_BF16 ? 2 : 4) / 16);
        int blocks = (int)std::min<int64_t>((chunks + 255) / 256, (int64_t)num_sms() * 8);
        ProfScope ps(s, PF_OTHER, 1);
        k_check_norms<<<std::max(blocks, 1), 256, 0, s>>>(Z, zdtype, n, d, w.err);
    }
    raftgp_status st = read_error_word(w.err, s);
    if (st != RAFTGP_OK) return st;
    // seeding for K_max, shared by every candidate
    {
        cudaError_t e = launch_seeding(Z, zdtype, n, d, kmax, o->seed, w.seed, s);
        if (e != cudaSuccess) return cuda_fail(e, "seeding");
    }
    cudaMemsetAsync(w.best, 0, sizeof(BestState), s);
    std::vector<CandRecord> rec;
    std::vector<int> ks;
    if (o->grid == 0) {
        for (int k = o->kmin; k <= kmax; ++k) ks.push_back(k);
        st = run_candidates(g, Z, d, zdtype, o, ks, w, labels, rec, s);
    } else {
        ks = coarse_grid(o->kmin, kmax, o->grid);
        st = run_candidates(g, Z, d, zdtype, o, ks, w, labels, rec, s);
        if (st == RAFTGP_OK) {
            int jb = 0;
            for (int j = 1; j < (int)rec.size(); ++j)
                if (host_better(o->criterion, rec[j], rec[jb])) jb = j;
            const int nc = (int)rec.size();
            const int lo = rec[jb > 0 ? jb - 1 : 0].k;
            const int hi = rec[jb < nc - 1 ? jb + 1 : nc - 1].k;
            std::vector<int> done;
            for (auto& r : rec) done.push_back(r.k);
            std::vector<int> ref = refine_grid(lo, hi, o->grid, done);
            if (!ref.empty()) st = run_candidates(g, Z, d, zdtype, o, ref, w, labels, rec, s);
        }
    }
    if (st != RAFTGP_OK) return st;
    st = read_error_word(w.err, s);
    if (st != RAFTGP_OK) return st;
    if (res) {
        int jb = 0;
        for (int j = 1; j < (int)rec.size(); ++j)
            if (host_better(o->criterion, rec[j], rec[jb])) jb = j;
        res->k_best = rec.empty() ? 0 : rec[jb].k;
        res->n_cand = (int)rec.size();
        for (int j = 0; j < (int)rec.size() && j < res->cand_cap; ++j) {
            if (res->cand_k) res->cand_k[j] = rec[j].k;
            if (res->cand_mod) res->cand_mod[j] = rec[j].mod;
            if (res->cand_ncut) res->cand_ncut[j] = rec[j].ncut;
            if (res->cand_passes) res->cand_passes[j] = rec[j].passes;
        }
    }
    return RAFTGP_OK;
}

}  // namespace raftgp

using namespace raftgp;

extern "C" {

size_t raftgp_workspace_size(const raftgp_csr* g, const raftgp_embed_opts* eopts, const raftgp_select_opts* sopts,
                             int32_t d) {
    if (!g || g->n < 1) return 0;
    Carver c(nullptr);
    uint32_t* err = nullptr;
    int32_t* deg = nullptr;
    if (eopts) {
        if (check_embed(eopts) != RAFTGP_OK) return 0;
        EmbedWs w = carve_embed(c, g->n, g->nnz, eopts);
        (void)w;
        err = reinterpret_cast<uint32_t*>(1);  // marks "shared with the embedding part"
        deg = reinterpret_cast<int32_t*>(1);
        d = eopts->dims[eopts->n_layers];
        if (sopts) c.take<char>((size_t)g->n * d * elem_size(eopts->dtype));  // Z of raftgp_partition
    }
    if (sopts) {
        if (check_select(sopts, g->n) != RAFTGP_OK || !width_ok(d)) return 0;
        carve_select(c, g->n, d, sopts, err, deg);
    }
    return c.off + 256;
}

raftgp_status raftgp_embed(const raftgp_csr* g, const raftgp_embed_opts* eopts, void* Z, void* ws, size_t ws_bytes,
                           raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((uintptr_t)Z & 15) return fail(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if ((st = check_embed(eopts))) return st;
    if (!Z || !ws) return fail(RAFTGP_EINVAL, "Z or workspace is NULL");
    if (ws_bytes < raftgp_workspace_size(g, eopts, nullptr, 0)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    EmbedWs w = carve_embed(c, g->n, g->nnz, eopts);
    cudaMemsetAsync(w.err, 0, sizeof(uint32_t), s);
    st = run_embed(g, eopts, Z, w, false, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "raftgp_embed");
    return RAFTGP_OK;
}

raftgp_status raftgp_select(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                            const raftgp_select_opts* sopts, int32_t* labels, raftgp_select_result* res, void* ws,
                            size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((uintptr_t)Z & 15) return fail(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if ((st = check_select(sopts, g->n))) return st;
    if (!width_ok(d)) return fail(RAFTGP_EUNSUPPORTED, "d = %d: must be 32, 64 or 128", d);
    if (z_dtype != RAFTGP_F32 && z_dtype != RAFTGP_BF16) return fail(RAFTGP_EINVAL, "unknown z_dtype");
    if (!Z || !labels || !ws) return fail(RAFTGP_EINVAL, "Z, labels or workspace is NULL");
    if (sopts->assign != RAFTGP_ASSIGN_FFMA && z_dtype != RAFTGP_BF16)
        return fail(RAFTGP_EINVAL, "tensor-core assignment needs BF16 embeddings");
    if (ws_bytes < raftgp_workspace_size(g, nullptr, sopts, d)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    SelectWs w = carve_select(c, g->n, d, sopts, nullptr, nullptr);
    st = run_select(g, Z, d, z_dtype, sopts, labels, res, w, false, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "raftgp_select");
    return RAFTGP_OK;
}

raftgp_status raftgp_partition(const raftgp_csr* g, const raftgp_embed_opts* eopts, const raftgp_select_opts* sopts,
                               int32_t* labels, raftgp_select_result* res, void* ws, size_t ws_bytes,
                               raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((st = check_embed(eopts))) return st;
    if ((st = check_select(sopts, g->n))) return st;
    if (!labels || !ws) return fail(RAFTGP_EINVAL, "labels or workspace is NULL");
    if (sopts->assign != RAFTGP_ASSIGN_FFMA && eopts->dtype != RAFTGP_BF16)
        return fail(RAFTGP_EINVAL, "tensor-core assignment needs BF16 embeddings");
    if (ws_bytes < raftgp_workspace_size(g, eopts, sopts, 0)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    const int d = eopts->dims[eopts->n_layers];
    Carver c(ws);
    EmbedWs ew = carve_embed(c, g->n, g->nnz, eopts);
    void* Z = c.take<char>((size_t)g->n * d * elem_size(eopts->dtype));
    SelectWs sw = carve_select(c, g->n, d, sopts, ew.err, ew.deg);
    cudaMemsetAsync(ew.err, 0, sizeof(uint32_t), s);
    st = run_embed(g, eopts, Z, ew, false, s);
    if (st) return st;
    st = run_select(g, Z, d, eopts->dtype, sopts, labels, res, sw, true, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "raftgp_partition");
    return RAFTGP_OK;
}

raftgp_status raftgp_score(const raftgp_csr* g, const int32_t* labels, int32_t K, int64_t* m, int64_t* vol,
                           double* mod, double* ncut, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if (K < 1) return fail(RAFTGP_EINVAL, "K must be >= 1");
    if (!labels || !m || !vol || !mod || !ncut || !ws) return fail(RAFTGP_EINVAL, "NULL argument");
    Carver c(ws);
    uint32_t* err = c.take<uint32_t>(64);
    int32_t* deg = c.take<int32_t>(g->n);
    float* rs = c.take<float>(g->n);
    float* rsh = c.take<float>(g->n);
    double* out2 = c.take<double>(2);
    if (ws_bytes < c.bytes()) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    launch_degrees(g, deg, rs, rsh, err, nullptr, nullptr, s);
    st = read_error_word(err, s);
    if (st) return st;
    cudaError_t e = launch_score_labels(g, deg, labels, K, reinterpret_cast<long long*>(m),
                                        reinterpret_cast<long long*>(vol), out2, err, s);
    if (e != cudaSuccess) return cuda_fail(e, "score");
    double h[2];
    e = cudaMemcpyAsync(h, out2, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "score copy");
    st = read_error_word(err, s);
    if (st) return st;
    *mod = h[0];
    *ncut = h[1];
    return RAFTGP_OK;
}

void raftgp_debug_seed_skip_block(int32_t block) { set_seed_skip_block(block); }

raftgp_status raftgp_kmeanspp(const void* Z, int64_t n, int32_t d, int32_t z_dtype, int32_t K, uint64_t seed,
                              int32_t* seeds, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    if (!Z || !seeds || !ws || n < 1) return fail(RAFTGP_EINVAL, "NULL argument or n < 1");
    if ((uintptr_t)Z & 15) return fail(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if (!width_ok(d)) return fail(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (K < 1 || K > n) return fail(RAFTGP_EINVAL, "need 1 <= K <= n");
    if (K > 32767) return fail(RAFTGP_EUNSUPPORTED, "K above 32767 is not supported");
    if (z_dtype != RAFTGP_F32 && z_dtype != RAFTGP_BF16) return fail(RAFTGP_EINVAL, "unknown z_dtype");
    Carver c(ws);
    char* region = c.take<char>(seed_scratch_bytes(n, K));
    if (ws_bytes < c.bytes()) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_seeding(Z, z_dtype, n, d, K, seed, carve_seed(region, n, K, seeds), s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kmeanspp");
    return RAFTGP_OK;
}

__global__ void k_labels_out(const int16_t* l16, int cs, int64_t n, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = l16[i * cs];
}

size_t raftgp_lloyd_workspace_size(int64_t n, int32_t d, int32_t K) {
    if (n < 1 || K < 1) return 0;
    Carver c(nullptr);
    KmState km{};
    carve_km(c, km, pad64h(K), d, n, 8);
    c.take<uint32_t>(64);
    c.take<int2>((size_t)n);
    c.take<int>(64);
    return c.off + 256;
}

raftgp_status raftgp_lloyd(const void* Z, int64_t n, int32_t d, int32_t z_dtype, const float* mu0, int32_t K,
                           int32_t iters, int32_t assign, int32_t recheck, int32_t* labels, float* mu_out,
                           int32_t* passes, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    if (!Z || !mu0 || !labels || !ws || n < 1) return fail(RAFTGP_EINVAL, "NULL argument or n < 1");
    if ((uintptr_t)Z & 15) return fail(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if (!width_ok(d)) return fail(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (K < 1 || K > 32767) return fail(RAFTGP_EINVAL, "need 1 <= K <= 32767");
    if (iters < 1) return fail(RAFTGP_EINVAL, "iters must be >= 1");
    if (assign < RAFTGP_ASSIGN_FFMA || assign > RAFTGP_ASSIGN_TC8) return fail(RAFTGP_EINVAL, "unknown assign engine");
    if (assign != RAFTGP_ASSIGN_FFMA && z_dtype != RAFTGP_BF16)
        return fail(RAFTGP_EINVAL, "tensor-core assignment needs BF16 embeddings");
    if (recheck < RAFTGP_RECHECK_NONE || recheck > RAFTGP_RECHECK_FP64) return fail(RAFTGP_EINVAL, "unknown recheck mode");
    Carver c(ws);
    KmState km{};
    carve_km(c, km, pad64h(K), d, n, 8);
    uint32_t* err = c.take<uint32_t>(64);
    int2* recheck_list = c.take<int2>((size_t)n);
    int* recheck_count = c.take<int>(64);
    if (ws_bytes < c.bytes()) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    CandBatch b{};
    b.n = 1;
    b.cs = 8;
    b.k[0] = K;
    b.off[0] = 0;
    b.total_k = pad64h(K);
    cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    launch_batch_init(b, Z, z_dtype, n, d, nullptr, mu0, km, s);
    raftgp_status st = run_lloyd(b, Z, z_dtype, n, d, iters, assign, recheck, km, recheck_list, recheck_count, err, s);
    if (st != RAFTGP_OK) return st;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    ProfScope ps(s, PF_OTHER, 1);
    k_labels_out<<<std::max(blocks, 1), 256, 0, s>>>(km.labels, 8, n, labels);
    if (mu_out) cudaMemcpyAsync(mu_out, km.mu, sizeof(float) * (size_t)K * d, cudaMemcpyDeviceToDevice, s);
    int32_t hp = 0;
    cudaMemcpyAsync(&hp, km.passes, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "lloyd");
    st = read_error_word(err, s);
    if (st != RAFTGP_OK) return st;
    if (passes) *passes = hp;
    return RAFTGP_OK;
}

const char* raftgp_last_error(void) { return g_last_error.c_str(); }

const char* raftgp_version(void) { return "raftgp-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ------------------------------------------------------------------------------------
// Differentiation form: one workspace layout for every call
// ------------------------------------------------------------------------------------
namespace {
struct DiffWs {
    int32_t* deg;
    float *rs, *rsh;
    uint32_t* err;
    float *P, *dA, *dP;     // n x width each
    float* wpart;           // wgrad partials
    float *S, *AS;          // n x 128 each
    double *spart, *red;    // loss partials, reduced sums
    long long* csums;       // K x width
    int* ccounts;           // K
};

DiffWs carve_diff(Carver& c, int64_t n, int width, int K) {
    DiffWs w{};
    w.deg = c.take<int32_t>(n);
    w.rs = c.take<float>(n);
    w.rsh = c.take<float>(n);
    w.err = c.take<uint32_t>(64);
    w.P = c.take<float>((size_t)n * width);
    w.dA = c.take<float>((size_t)n * width);
    w.dP = c.take<float>((size_t)n * width);
    w.wpart = c.take<float>((size_t)wgrad_blocks(n) * width * width);
    w.S = c.take<float>((size_t)n * 128);
    w.AS = c.take<float>((size_t)n * 128);
    w.spart = c.take<double>((size_t)softmod_blocks(n) * 129);
    w.red = c.take<double>(129 + 64);
    w.csums = c.take<long long>((size_t)(K > 0 ? K : 1) * width);
    w.ccounts = c.take<int>(K > 0 ? K : 1);
    return w;
}

// degrees, the normalisation and the device graph check (read back before any gather)
raftgp_status diff_prepare(const raftgp_csr* g, const DiffWs& w, cudaStream_t s) {
    cudaMemsetAsync(w.err, 0, sizeof(uint32_t), s);
    launch_degrees(g, w.deg, w.rs, w.rsh, w.err, nullptr, nullptr, s);
    return read_error_word(w.err, s);
}

// The steps of each call after the graph check; every launch is asynchronous.
raftgp_status layer_forward(const raftgp_csr* g, const DiffWs& w, const float* H_in, int lin, const float* W, int lout,
                            float* H_out, cudaStream_t s) {
    cudaError_t e = launch_rowmm(g->n, H_in, lin, W, lout, false, w.P, s);
    if (e == cudaSuccess) e = launch_spmm32(g, lout, w.rsh, w.P, nullptr, H_out, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "gcn layer forward");
    return RAFTGP_OK;
}

raftgp_status layer_backward(const raftgp_csr* g, const DiffWs& w, const float* H_in, int lin, const float* W,
                             int lout, const float* dH_out, float* dH_in, float* dW, cudaStream_t s) {
    // recompute P = H_in W; dA from the recomputed pre-activation and dH_out; dP = Ahat dA
    cudaError_t e = launch_rowmm(g->n, H_in, lin, W, lout, false, w.P, s);
    if (e == cudaSuccess) e = launch_spmm32(g, lout, w.rsh, w.P, dH_out, w.dA, 1, s);
    if (e == cudaSuccess) e = launch_spmm32(g, lout, w.rsh, w.dA, nullptr, w.dP, 2, s);
    if (e == cudaSuccess) e = launch_wgrad(g->n, H_in, lin, w.dP, lout, w.wpart, dW, s);
    if (e == cudaSuccess && dH_in) e = launch_rowmm(g->n, w.dP, lout, W, lin, true, dH_in, s);
    if (e != cudaSuccess) return cuda_fail(e, "gcn layer backward");
    return RAFTGP_OK;
}

// Leaves d^T S in red[0..128), sum S . AS in red[128] and the loss in red[129].
raftgp_status softmod(const raftgp_csr* g, const DiffWs& w, const float* Z, int d, const float* mu, int K, float tau,
                      float* dZ, cudaStream_t s) {
    const double two_e = (double)g->nnz;
    cudaError_t e = launch_soft_assign(g->n, d, Z, mu, K, tau, w.S, s);
    if (e == cudaSuccess) e = launch_spmm32(g, 128, w.rsh, w.S, nullptr, w.AS, 3, s);
    if (e == cudaSuccess) e = launch_softmod_reduce(g->n, w.deg, w.S, w.AS, K, two_e, w.spart, w.red, s);
    if (e == cudaSuccess && dZ) e = launch_softmod_grad(g->n, d, Z, mu, K, tau, w.deg, w.S, w.AS, w.red, two_e, dZ, s);
    if (e != cudaSuccess) return cuda_fail(e, "softmod loss");
    return RAFTGP_OK;
}

// H_in, the n x lout array (H_out or dH_out) and dH_in are read and written in 16-byte pieces.
raftgp_status layer_args(const float* H_in, int lin, const float* W, int lout, const void* H_out,
                         const void* dH_in = nullptr) {
    if (!H_in || !W || !H_out) return fail(RAFTGP_EINVAL, "NULL argument");
    if (((uintptr_t)H_in | (uintptr_t)H_out | (uintptr_t)dH_in) & 15)
        return fail(RAFTGP_EINVAL, "H_in, H_out, dH_out and dH_in must be 16-byte aligned");
    if (!width_ok(lin) || !width_ok(lout)) return fail(RAFTGP_EUNSUPPORTED, "widths must be 32, 64 or 128");
    return RAFTGP_OK;
}

// Z is read and dZ written in 16-byte pieces.
raftgp_status softmod_args(const raftgp_csr* g, const float* Z, int d, const float* mu, int K, float tau,
                           const void* loss, const float* dZ) {
    if (!Z || !mu || !loss) return fail(RAFTGP_EINVAL, "NULL argument");
    if (((uintptr_t)Z | (uintptr_t)dZ) & 15) return fail(RAFTGP_EINVAL, "Z and dZ must be 16-byte aligned");
    if (!width_ok(d)) return fail(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (K < 1 || K > 128) return fail(RAFTGP_EUNSUPPORTED, "K must be in [1, 128]");
    if (!(tau > 0.f)) return fail(RAFTGP_EINVAL, "tau must be positive");
    if (g->nnz == 0) return fail(RAFTGP_EINVAL, "the loss needs at least one edge");
    return RAFTGP_OK;
}
}  // namespace

struct raftgp_diff_plan {
    raftgp_csr g;
    int width = 0, K = 0;
    DiffWs w{};
};

extern "C" {

size_t raftgp_diff_workspace_size(int64_t n, int32_t width, int32_t K) {
    Carver c(nullptr);
    carve_diff(c, n, width, K);
    return c.off + 256;
}

raftgp_status raftgp_gcn_layer_forward(const raftgp_csr* g, const float* H_in, int32_t lin, const float* W,
                                       int32_t lout, float* H_out, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((st = layer_args(H_in, lin, W, lout, H_out))) return st;
    if (!ws) return fail(RAFTGP_EINVAL, "NULL argument");
    const int width = std::max(lin, lout);
    if (ws_bytes < raftgp_diff_workspace_size(g->n, width, 0)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    DiffWs w = carve_diff(c, g->n, width, 0);
    if ((st = diff_prepare(g, w, s))) return st;
    return layer_forward(g, w, H_in, lin, W, lout, H_out, s);
}

raftgp_status raftgp_gcn_layer_backward(const raftgp_csr* g, const float* H_in, int32_t lin, const float* W,
                                        int32_t lout, const float* dH_out, float* dH_in, float* dW, void* ws,
                                        size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((st = layer_args(H_in, lin, W, lout, dH_out, dH_in))) return st;
    if (!dW || !ws) return fail(RAFTGP_EINVAL, "NULL argument");
    const int width = std::max(lin, lout);
    if (ws_bytes < raftgp_diff_workspace_size(g->n, width, 0)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    DiffWs w = carve_diff(c, g->n, width, 0);
    if ((st = diff_prepare(g, w, s))) return st;
    return layer_backward(g, w, H_in, lin, W, lout, dH_out, dH_in, dW, s);
}

raftgp_status raftgp_softmod_loss(const raftgp_csr* g, const float* Z, int32_t d, const float* mu, int32_t K,
                                  float tau, double* loss, float* dZ, void* ws, size_t ws_bytes,
                                  raftgp_stream_t stream) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((st = softmod_args(g, Z, d, mu, K, tau, loss, dZ))) return st;
    if (!ws) return fail(RAFTGP_EINVAL, "NULL argument");
    if (ws_bytes < raftgp_diff_workspace_size(g->n, d, K)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    DiffWs w = carve_diff(c, g->n, d, K);
    if ((st = diff_prepare(g, w, s))) return st;
    if ((st = softmod(g, w, Z, d, mu, K, tau, dZ, s))) return st;
    cudaError_t e = cudaMemcpyAsync(loss, w.red + 129, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "softmod loss readback");
    return RAFTGP_OK;
}

raftgp_status raftgp_diff_plan_create(const raftgp_csr* g, int32_t width, int32_t K, void* ws, size_t ws_bytes,
                                      raftgp_stream_t stream, raftgp_diff_plan** plan) {
    if (!plan) return fail(RAFTGP_EINVAL, "NULL plan");
    *plan = nullptr;
    raftgp_status st = check_csr(g);
    if (st) return st;
    if (!ws) return fail(RAFTGP_EINVAL, "NULL argument");
    if (!width_ok(width)) return fail(RAFTGP_EUNSUPPORTED, "width must be 32, 64 or 128");
    if (K < 0 || K > 128) return fail(RAFTGP_EUNSUPPORTED, "K must be in [0, 128]");
    if (ws_bytes < raftgp_diff_workspace_size(g->n, width, K)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    raftgp_diff_plan* p = new raftgp_diff_plan();
    p->g = *g;
    p->width = width;
    p->K = K;
    Carver c(ws);
    p->w = carve_diff(c, g->n, width, K);
    if ((st = diff_prepare(&p->g, p->w, s))) {
        delete p;
        return st;
    }
    *plan = p;
    return RAFTGP_OK;
}

raftgp_status raftgp_diff_plan_layer_forward(const raftgp_diff_plan* p, const float* H_in, int32_t lin,
                                             const float* W, int32_t lout, float* H_out, raftgp_stream_t stream) {
    if (!p) return fail(RAFTGP_EINVAL, "NULL plan");
    raftgp_status st = layer_args(H_in, lin, W, lout, H_out);
    if (st) return st;
    if (std::max(lin, lout) > p->width) return fail(RAFTGP_EINVAL, "layer wider than the plan");
    return layer_forward(&p->g, p->w, H_in, lin, W, lout, H_out, (cudaStream_t)stream);
}

raftgp_status raftgp_diff_plan_layer_backward(const raftgp_diff_plan* p, const float* H_in, int32_t lin,
                                              const float* W, int32_t lout, const float* dH_out, float* dH_in,
                                              float* dW, raftgp_stream_t stream) {
    if (!p) return fail(RAFTGP_EINVAL, "NULL plan");
    raftgp_status st = layer_args(H_in, lin, W, lout, dH_out, dH_in);
    if (st) return st;
    if (!dW) return fail(RAFTGP_EINVAL, "NULL argument");
    if (std::max(lin, lout) > p->width) return fail(RAFTGP_EINVAL, "layer wider than the plan");
    return layer_backward(&p->g, p->w, H_in, lin, W, lout, dH_out, dH_in, dW, (cudaStream_t)stream);
}

raftgp_status raftgp_diff_plan_softmod_loss(const raftgp_diff_plan* p, const float* Z, int32_t d, const float* mu,
                                            int32_t K, float tau, double* loss, float* dZ, raftgp_stream_t stream) {
    if (!p) return fail(RAFTGP_EINVAL, "NULL plan");
    raftgp_status st = softmod_args(&p->g, Z, d, mu, K, tau, loss, dZ);
    if (st) return st;
    if (d > p->width || K > p->K) return fail(RAFTGP_EINVAL, "d or K larger than the plan's");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = softmod(&p->g, p->w, Z, d, mu, K, tau, dZ, s))) return st;
    cudaError_t e = cudaMemcpyAsync(loss, p->w.red + 129, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "softmod loss copy");
    return RAFTGP_OK;
}

void raftgp_diff_plan_destroy(raftgp_diff_plan* plan) { delete plan; }

raftgp_status raftgp_centroids(const float* Z, int64_t n, int32_t d, const int32_t* labels, int32_t K, float* mu,
                               void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    if (!Z || !labels || !mu || !ws || n < 1) return fail(RAFTGP_EINVAL, "NULL argument or n < 1");
    if ((uintptr_t)Z & 15) return fail(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if (!width_ok(d)) return fail(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (K < 1) return fail(RAFTGP_EINVAL, "K < 1");
    if (ws_bytes < raftgp_diff_workspace_size(n, d, K)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    DiffWs w = carve_diff(c, n, d, K);
    cudaMemsetAsync(w.err, 0, sizeof(uint32_t), s);
    cudaError_t e = launch_centroids(n, d, Z, labels, K, w.csums, w.ccounts, mu, w.err, s);
    if (e != cudaSuccess) return cuda_fail(e, "centroids");
    return read_error_word(w.err, s);
}

raftgp_status raftgp_gcn_weights(int32_t layer, int32_t lin, int32_t lout, uint64_t seed, float* W,
                                 raftgp_stream_t stream) {
    if (!W) return fail(RAFTGP_EINVAL, "W is NULL");
    if (layer < 1 || layer > RAFTGP_MAX_LAYERS) return fail(RAFTGP_EINVAL, "layer must be in [1, %d]", RAFTGP_MAX_LAYERS);
    if (!width_ok(lin) || !width_ok(lout)) return fail(RAFTGP_EUNSUPPORTED, "widths must be 32, 64 or 128");
    launch_weights(layer, lin, lout, seed, W, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gcn weights");
    return RAFTGP_OK;
}

raftgp_status raftgp_adam_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr,
                               float beta1, float beta2, float eps, int32_t step, raftgp_stream_t stream) {
    if (!param || !grad || !m || !v || count < 1) return fail(RAFTGP_EINVAL, "NULL argument or count < 1");
    if (step < 1) return fail(RAFTGP_EINVAL, "step counts from 1");
    cudaError_t e = launch_adam(param, grad, m, v, count, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "adam");
    return RAFTGP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Many graphs at once: plan (validation, autotuning, CUDA-graph capture) and replay
// ------------------------------------------------------------------------------------
struct raftgp_batch_plan {
    raftgp_csr g;
    raftgp_embed_opts eo;
    raftgp_batch_opts bo;
    int ng = 0, d = 0;
    int64_t total_n = 0;
    std::vector<int64_t> h_off;
    std::vector<int32_t> h_kmax, h_seed_off, h_order;
    EmbedWs ew{};
    void* Z = nullptr;
    BatchDev bd{};
    uint32_t* err = nullptr;
    int32_t* labels = nullptr;
    int32_t* k_out = nullptr;
    int threads = 256, ppt = 1;
    float tune_ms[7] = {};
    void* stg = nullptr;   // tensor-core Lloyd: staging of the centroid operands
    float flat_ms[4] = {};  // BF16 embedding: one embedding per flat-stream gather shape
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;   // the plan's own stream, on which the graph is captured
};

namespace {
const int kTuneThreads[3] = {128, 256, 512};

raftgp_status batch_layout(const raftgp_csr* g, const int64_t* off, int ng, const raftgp_embed_opts* eo,
                           const raftgp_batch_opts* bo, raftgp_batch_plan& p) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((st = check_embed(eo))) return st;
    if (!off || ng < 1 || !bo) return fail(RAFTGP_EINVAL, "NULL argument or n_graphs < 1");
    if (eo->op != RAFTGP_OP_NCUT && !(eo->op == RAFTGP_OP_MOD_FULL && eo->dtype == RAFTGP_BF16))
        return fail(RAFTGP_EUNSUPPORTED,
                    "the batched form supports the NCut operator, and the full modularity operator with BF16 storage");
    const int d = eo->dims[eo->n_layers];
    if (d != 32 && d != 64) return fail(RAFTGP_EUNSUPPORTED, "the batched form needs a final width of 32 or 64");
    if (bo->kmin < 2) return fail(RAFTGP_EINVAL, "kmin must be >= 2");
    if (bo->grid < 1 || bo->grid > BATCH_COARSE) return fail(RAFTGP_EINVAL, "grid must be in [1, %d]", BATCH_COARSE);
    if (bo->iters < 1) return fail(RAFTGP_EINVAL, "iters must be >= 1");
    if (!(bo->kmax_factor > 0.f)) return fail(RAFTGP_EINVAL, "kmax_factor must be positive");
    if (bo->lloyd_variant < 0 || bo->lloyd_variant > 7) return fail(RAFTGP_EINVAL, "lloyd_variant must be in [0, 7]");
    if (bo->embed_variant < 0 || bo->embed_variant > 4) return fail(RAFTGP_EINVAL, "embed_variant must be in [0, 4]");
    if (bo->assign < RAFTGP_ASSIGN_FFMA || bo->assign > RAFTGP_ASSIGN_TC8) return fail(RAFTGP_EINVAL, "unknown assign engine");
    if (bo->assign != RAFTGP_ASSIGN_FFMA && eo->dtype != RAFTGP_BF16)
        return fail(RAFTGP_EINVAL, "tensor-core assignment needs BF16 embeddings");
    if (off[0] != 0 || off[ng] != g->n) return fail(RAFTGP_EINVAL, "graph_off must run from 0 to n");
    p.g = *g;
    p.eo = *eo;
    p.bo = *bo;
    p.ng = ng;
    p.d = d;
    p.total_n = g->n;
    p.h_off.assign(off, off + ng + 1);
    p.h_kmax.resize(ng);
    p.h_seed_off.resize(ng + 1);
    p.h_seed_off[0] = 0;
    for (int i = 0; i < ng; ++i) {
        const int64_t n = off[i + 1] - off[i];
        if (n < 2) return fail(RAFTGP_EINVAL, "graph %d has fewer than 2 nodes", i);
        int64_t km = (int64_t)std::ceil((double)bo->kmax_factor * std::pow((double)n, 0.35));
        km = std::min<int64_t>(std::min<int64_t>(km, BATCH_KMAX), n);
        if (km < bo->kmin) return fail(RAFTGP_EINVAL, "graph %d: K_max %lld is below kmin", i, (long long)km);
        p.h_kmax[i] = (int32_t)km;
        p.h_seed_off[i + 1] = p.h_seed_off[i] + (int32_t)km;
    }
    p.h_order.resize(ng);
    for (int i = 0; i < ng; ++i) p.h_order[i] = i;
    std::stable_sort(p.h_order.begin(), p.h_order.end(),
                     [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    return RAFTGP_OK;
}

void carve_batch(Carver& c, raftgp_batch_plan& p) {
    const int64_t n = p.total_n;
    p.ew = carve_embed(c, n, p.g.nnz, &p.eo);
    p.Z = c.take<char>((size_t)n * p.d * elem_size(p.eo.dtype));
    p.err = c.take<uint32_t>(64);
    BatchDev& b = p.bd;
    b.ng = p.ng;
    b.total_n = n;
    b.node_off = c.take<int64_t>(p.ng + 1);
    b.kmax = c.take<int32_t>(p.ng);
    b.seed_off = c.take<int32_t>(p.ng + 1);
    b.order = c.take<int32_t>(p.ng);
    b.local_row = c.take<int32_t>(n);
    b.graph_of = c.take<int32_t>(n);
    b.seeds = c.take<int32_t>(p.h_seed_off.empty() ? 1 : p.h_seed_off.back());
    b.cand_k = c.take<int32_t>((size_t)p.ng * BATCH_SLOTS);
    b.n_coarse = c.take<int32_t>(p.ng);
    b.n_refine = c.take<int32_t>(p.ng);
    b.cand_mod = c.take<double>((size_t)p.ng * BATCH_SLOTS);
    b.cand_ncut = c.take<double>((size_t)p.ng * BATCH_SLOTS);
    b.cand_passes = c.take<int32_t>((size_t)p.ng * BATCH_SLOTS);
    b.labels = c.take<int16_t>((size_t)BATCH_SLOTS * n);
    b.D2 = c.take<float>(n);
    b.chosen = c.take<uint8_t>(n);
    b.queue = c.take<int>(64);
    p.ew.local_row = b.local_row;
    if (p.eo.op == RAFTGP_OP_MOD_FULL) {
        p.ew.ng = p.ng;
        p.ew.graph_off = b.node_off;
        p.ew.graph_of = b.graph_of;
        p.ew.g_graph = c.take<float>((size_t)p.ng * p.eo.dims[0]);
        p.ew.inv_two_e_graph = c.take<double>(p.ng);
    }
    p.stg = p.bo.assign != RAFTGP_ASSIGN_FFMA ? c.take<char>(batch_tc_staging_bytes(p.d)) : nullptr;
}

// everything after validation: embedding, grids, seeding, both Lloyd phases, selection
raftgp_status batch_enqueue(raftgp_batch_plan& p, cudaStream_t s) {
    const int zdtype = p.eo.dtype;
    cudaMemsetAsync(p.err, 0, sizeof(uint32_t), s);   // device error word of this replay
    cudaMemsetAsync(p.bd.cand_k, 0, sizeof(int32_t) * (size_t)p.ng * BATCH_SLOTS, s);
    launch_batch_prologue(p.bd, p.bo.kmin, p.bo.grid, s);   // work counters, local rows, coarse grids
    raftgp_status st = run_embed(&p.g, &p.eo, p.Z, p.ew, true, s);
    if (st) return st;
    cudaError_t e = launch_batch_seed(p.bd, p.Z, zdtype, p.d, p.bo.seed, s);
    auto lloyd = [&](int phase) {
        return p.bo.assign != RAFTGP_ASSIGN_FFMA
                   ? launch_batch_lloyd_tc(p.bd, p.Z, p.d, phase, p.bo.iters, p.bo.assign == RAFTGP_ASSIGN_TC ? 1 : 0,
                                           &p.g, p.stg, p.err, s)
                   : launch_batch_lloyd(p.bd, p.Z, zdtype, p.d, phase, p.bo.iters, &p.g, p.threads, p.ppt, s);
    };
    if (e == cudaSuccess) e = lloyd(0);
    if (e != cudaSuccess) return cuda_fail(e, "batched selection");
    if (p.bo.grid > 1) {
        launch_batch_refine(p.bd, p.bo.grid, p.bo.criterion, s);
        e = lloyd(1);
        if (e != cudaSuccess) return cuda_fail(e, "batched selection");
    }
    launch_batch_select(p.bd, p.bo.criterion, p.labels, p.k_out, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batched selection");
    return RAFTGP_OK;
}
}  // namespace

extern "C" {

size_t raftgp_batch_workspace_size(const raftgp_csr* g, const int64_t* graph_off, int32_t n_graphs,
                                   const raftgp_embed_opts* eo, const raftgp_batch_opts* bo) {
    raftgp_batch_plan p;
    if (batch_layout(g, graph_off, n_graphs, eo, bo, p) != RAFTGP_OK) return 0;
    Carver c(nullptr);
    carve_batch(c, p);
    return c.off + 256;
}

raftgp_status raftgp_batch_plan_create(const raftgp_csr* g, const int64_t* graph_off, int32_t n_graphs,
                                       const raftgp_embed_opts* eo, const raftgp_batch_opts* bo, int32_t* labels,
                                       int32_t* k_out, void* ws, size_t ws_bytes, raftgp_stream_t stream,
                                       raftgp_batch_plan** plan) {
    if (!plan) return fail(RAFTGP_EINVAL, "plan is NULL");
    *plan = nullptr;
    if (!labels || !k_out || !ws) return fail(RAFTGP_EINVAL, "labels, k_out or workspace is NULL");
    std::unique_ptr<raftgp_batch_plan> p(new raftgp_batch_plan());
    raftgp_status st = batch_layout(g, graph_off, n_graphs, eo, bo, *p);
    if (st) return st;
    if (ws_bytes < raftgp_batch_workspace_size(g, graph_off, n_graphs, eo, bo))
        return fail(RAFTGP_ENOMEM, "workspace too small");
    Carver c(ws);
    carve_batch(c, *p);
    p->labels = labels;
    p->k_out = k_out;
    cudaStream_t s = (cudaStream_t)stream;
    BatchDev& b = p->bd;
    cudaMemcpyAsync((void*)b.node_off, p->h_off.data(), sizeof(int64_t) * (p->ng + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)b.kmax, p->h_kmax.data(), sizeof(int32_t) * p->ng, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)b.seed_off, p->h_seed_off.data(), sizeof(int32_t) * (p->ng + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((void*)b.order, p->h_order.data(), sizeof(int32_t) * p->ng, cudaMemcpyHostToDevice, s);
    // the graph checks (CSR, block-diagonal), degrees and the heavy-row list, once
    cudaMemsetAsync(p->ew.err, 0, sizeof(uint32_t), s);
    launch_degrees(&p->g, p->ew.deg, p->ew.rs, p->ew.rsh, p->ew.err, p->ew.heavy, p->ew.heavy_count, s);
    launch_batch_check(&p->g, p->ng, b.node_off, p->ew.err, s);
    if ((st = read_error_word(p->ew.err, s))) return st;
    // local rows and each node's graph, which the embedding reads (Philox counters, the
    // per-graph rank-one term), before its first run
    launch_batch_prologue(b, p->bo.kmin, p->bo.grid, s);
    // autotuning of the BF16 embedding's gathers: one embedding timed per flat-stream shape
    // (batch size and staging depth; every shape gives the same bits)
    if (p->eo.dtype == RAFTGP_BF16) {
        cudaEvent_t f0, f1;
        cudaEventCreate(&f0);
        cudaEventCreate(&f1);
        float fbest = INFINITY;
        int fv = 0;
        for (int v = 0; v < 4; ++v) {
            if (p->bo.embed_variant > 0 && v != p->bo.embed_variant - 1) continue;   // a forced shape
            p->ew.flat_variant = v;
            cudaEventRecord(f0, s);
            raftgp_status est = run_embed(&p->g, &p->eo, p->Z, p->ew, true, s);
            cudaEventRecord(f1, s);
            float ms = INFINITY;
            if (est == RAFTGP_OK && cudaEventSynchronize(f1) == cudaSuccess) cudaEventElapsedTime(&ms, f0, f1);
            p->flat_ms[v] = ms;
            if (ms < fbest) {
                fbest = ms;
                fv = v;
            }
        }
        cudaEventDestroy(f0);
        cudaEventDestroy(f1);
        p->ew.flat_variant = fv;
        if (!(fbest < INFINITY)) return fail(RAFTGP_ECUDA, "no embedding gather shape could run");
    }
    // autotuning: the coarse Lloyd phase timed for every variant on this batch (results are
    // the same for all of them)
    p->threads = 256;
    p->ppt = 1;
    if ((st = batch_enqueue(*p, s))) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = INFINITY;
    for (int v = 0; v < 7; ++v) {
        if (p->bo.assign != RAFTGP_ASSIGN_FFMA) {   // the tensor-core Lloyd kernel has one shape
            best = 0.f;
            p->threads = 192;
            p->ppt = -1;
            break;
        }
        if (p->bo.lloyd_variant > 0 && v != p->bo.lloyd_variant - 1) continue;   // a forced variant
        // six shapes of the scalar kernel, then the register-tiled kernel (ppt 0)
        const int th = v < 6 ? kTuneThreads[v / 2] : 256, pp = v < 6 ? 1 + v % 2 : 0;
        cudaMemsetAsync(b.queue + 1, 0, sizeof(int), s);
        cudaEventRecord(e0, s);
        cudaError_t e = launch_batch_lloyd(b, p->Z, p->eo.dtype, p->d, 0, p->bo.iters, &p->g, th, pp, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = INFINITY;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        else cudaGetLastError();
        p->tune_ms[v] = ms;
        if (ms < best) {
            best = ms;
            p->threads = th;
            p->ppt = pp;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!(best < INFINITY)) return fail(RAFTGP_ECUDA, "no Lloyd variant could run");
    // capture the whole partition on the plan's own stream (the caller's stream may be the
    // legacy default stream, which cannot be captured); the graph is launched on any stream
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "plan stream");
    e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(p->cap);
        return cuda_fail(e, "begin capture");
    }
    st = batch_enqueue(*p, p->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->cap, &graph);
    if (st || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(p->cap);
        return st ? st : cuda_fail(e, "end capture");
    }
    p->graph = graph;
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaStreamDestroy(p->cap);
        return cuda_fail(e, "graph instantiate");
    }
    *plan = p.release();
    return RAFTGP_OK;
}

raftgp_status raftgp_batch_plan_run(raftgp_batch_plan* plan, raftgp_stream_t stream) {
    if (!plan || !plan->exec) return fail(RAFTGP_EINVAL, "plan is NULL");
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return RAFTGP_OK;
}

raftgp_status raftgp_batch_plan_candidates(raftgp_batch_plan* plan, int32_t* k, double* mod, double* ncut,
                                           int32_t* passes) {
    if (!plan) return fail(RAFTGP_EINVAL, "plan is NULL");
    const size_t cnt = (size_t)plan->ng * BATCH_SLOTS;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && k) e = cudaMemcpy(k, plan->bd.cand_k, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mod) e = cudaMemcpy(mod, plan->bd.cand_mod, cnt * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ncut) e = cudaMemcpy(ncut, plan->bd.cand_ncut, cnt * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && passes)
        e = cudaMemcpy(passes, plan->bd.cand_passes, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "candidates");
    return RAFTGP_OK;
}

raftgp_status raftgp_batch_plan_tuning(const raftgp_batch_plan* plan, int32_t* threads, int32_t* points_per_thread,
                                       float* ms) {
    if (!plan) return fail(RAFTGP_EINVAL, "plan is NULL");
    if (threads) *threads = plan->threads;
    if (points_per_thread) *points_per_thread = plan->ppt;
    if (ms)
        for (int v = 0; v < 7; ++v) ms[v] = plan->tune_ms[v];
    return RAFTGP_OK;
}

raftgp_status raftgp_batch_plan_tuning_embed(const raftgp_batch_plan* plan, int32_t* variant, float* ms) {
    if (!plan) return fail(RAFTGP_EINVAL, "plan is NULL");
    if (variant) *variant = plan->ew.flat_variant;
    if (ms)
        for (int v = 0; v < 4; ++v) ms[v] = plan->flat_ms[v];
    return RAFTGP_OK;
}

raftgp_status raftgp_batch_plan_check(const raftgp_batch_plan* plan) {
    if (!plan) return fail(RAFTGP_EINVAL, "plan is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "batched partition");
    raftgp_status st = read_error_word(plan->err, nullptr);
    return st ? st : read_error_word(plan->ew.err, nullptr);
}

raftgp_status raftgp_batch_plan_embedding(const raftgp_batch_plan* plan, void* Z_out) {
    if (!plan || !Z_out) return fail(RAFTGP_EINVAL, "plan or Z_out is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(Z_out, plan->Z, (size_t)plan->total_n * plan->d * elem_size(plan->eo.dtype),
                       cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "embedding");
    return RAFTGP_OK;
}

void raftgp_batch_plan_destroy(raftgp_batch_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->cap) cudaStreamDestroy(plan->cap);
    delete plan;
}

raftgp_status raftgp_partition_batched(const raftgp_csr* g, const int64_t* graph_off, int32_t n_graphs,
                                       const raftgp_embed_opts* eo, const raftgp_batch_opts* bo, int32_t* labels,
                                       int32_t* k_out, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_batch_plan* plan = nullptr;
    raftgp_status st = raftgp_batch_plan_create(g, graph_off, n_graphs, eo, bo, labels, k_out, ws, ws_bytes, stream,
                                                &plan);
    if (st) return st;
    st = raftgp_batch_plan_run(plan, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (!st && e == cudaSuccess) st = raftgp_batch_plan_check(plan);
    raftgp_batch_plan_destroy(plan);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "batched partition");
    return RAFTGP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Algorithm 1
// ------------------------------------------------------------------------------------
namespace {
BisectDev carve_bisect(Carver& c, int64_t n, int d, int eps) {
    BisectDev b{};
    b.eps = eps;
    const int64_t cap = n / (eps + 1) + 2;
    b.cap_sets = (int)cap;
    b.perm = c.take<int32_t>(n);
    b.perm_next = c.take<int32_t>(n);
    b.pos_set = c.take<int32_t>(n);
    b.lab = c.take<int8_t>(n);
    b.q = c.take<unsigned long long>(n);
    b.P = c.take<unsigned long long>(n);
    b.F = c.take<unsigned long long>(n);
    b.tiles = c.take<unsigned long long>(n / 4096 + 64);
    b.node_set = c.take<int32_t>(n);
    b.node_lab = c.take<int32_t>(n);
    b.block_of = c.take<int32_t>(n);
    b.set_off = c.take<int64_t>(cap);
    b.set_n = c.take<int64_t>(cap);
    b.nset_off = c.take<int64_t>(cap);
    b.nset_n = c.take<int64_t>(cap);
    b.set_id = c.take<uint64_t>(cap);
    b.nset_id = c.take<uint64_t>(cap);
    b.s0 = c.take<int64_t>(cap);
    b.child_pos = c.take<int64_t>(cap);
    b.active = c.take<int32_t>(cap);
    b.changed = c.take<int32_t>(2 * cap);
    b.counts = c.take<int32_t>(2 * cap);
    b.split = c.take<int32_t>(cap);
    b.block_id = c.take<int32_t>(cap);
    b.mu = c.take<float>((size_t)cap * 2 * d);
    b.norm2 = c.take<float>(2 * cap);
    b.sums = c.take<long long>((size_t)cap * 2 * d);
    b.acc = c.take<unsigned long long>(5 * cap);
    b.scan_in = c.take<unsigned long long>(3 * cap);
    b.scan_out = c.take<unsigned long long>(3 * cap);
    b.bmin = c.take<int32_t>(n + cap);   // block indices: the previous run's (up to n) + this run's
    b.counters = c.take<int>(64);
    b.counters_ll = c.take<long long>(8);
    b.set_keep = c.take<int32_t>(cap);
    b.nset_keep = c.take<int32_t>(cap);
    b.frozen = c.take<int32_t>(cap);
    b.flag = c.take<int32_t>(cap);
    return b;
}

__global__ void k_iota(int32_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
}  // namespace

extern "C" {

size_t raftgp_bisect_workspace_size(int64_t n, int32_t d, int32_t eps) {
    Carver c(nullptr);
    c.take<uint32_t>(64);
    c.take<int32_t>(n);
    c.take<float>(n);
    c.take<float>(n);
    carve_bisect(c, n, d, eps < 1 ? 1 : eps);
    return c.off + 256;
}

static raftgp_status bisect_common(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                                   const raftgp_bisect_opts* o, const int32_t* old_labels, int32_t old_k,
                                   const uint64_t* old_leaf, const uint8_t* dirty, int32_t* labels, uint64_t* leaf,
                                   int32_t* k_out, void* ws, size_t ws_bytes, cudaStream_t s) {
    raftgp_status st = check_csr(g);
    if (st) return st;
    if ((uintptr_t)Z & 15) return fail(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if (!Z || !o || !labels || !k_out || !ws) return fail(RAFTGP_EINVAL, "NULL argument");
    if (!width_ok(d)) return fail(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (z_dtype != RAFTGP_F32 && z_dtype != RAFTGP_BF16) return fail(RAFTGP_EINVAL, "unknown z_dtype");
    if (o->eps < 1) return fail(RAFTGP_EINVAL, "eps must be >= 1");
    if (o->iters < 1) return fail(RAFTGP_EINVAL, "iters must be >= 1");
    if (o->reading != 0 && o->reading != 1) return fail(RAFTGP_EINVAL, "reading must be 0 or 1");
    if (dirty && (!old_labels || !old_leaf || old_k < 1 || old_k > g->n))
        return fail(RAFTGP_EINVAL, "the update needs the previous labels (1 <= old_k <= n) and leaf ids");
    if (ws_bytes < raftgp_bisect_workspace_size(g->n, d, o->eps)) return fail(RAFTGP_ENOMEM, "workspace too small");
    Carver c(ws);
    uint32_t* err = c.take<uint32_t>(64);
    int32_t* deg = c.take<int32_t>(g->n);
    float* rs = c.take<float>(g->n);
    float* rsh = c.take<float>(g->n);
    BisectDev b = carve_bisect(c, g->n, d, o->eps);
    b.leaf_of = leaf;
    b.old_label = old_labels;
    b.old_leaf = old_leaf;
    b.dirty = dirty;
    b.k_old = dirty ? old_k : 0;
    cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    launch_degrees(g, deg, rs, rsh, err, nullptr, nullptr, s);
    if ((st = read_error_word(err, s))) return st;
    k_iota<<<(unsigned)std::min<int64_t>((g->n + 255) / 256, 4096), 256, 0, s>>>(b.perm, g->n);
    cudaError_t e = launch_bisect(g, Z, z_dtype, d, b, o->iters, o->seed, o->reading, labels, k_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "bisect");
    return RAFTGP_OK;
}

raftgp_status raftgp_select_bisect(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                                   const raftgp_bisect_opts* o, int32_t* labels, uint64_t* leaf, int32_t* k_out,
                                   void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    return bisect_common(g, Z, d, z_dtype, o, nullptr, 0, nullptr, nullptr, labels, leaf, k_out, ws, ws_bytes,
                         (cudaStream_t)stream);
}

raftgp_status raftgp_select_bisect_update(const raftgp_csr* g, const void* Z, int32_t d, int32_t z_dtype,
                                          const raftgp_bisect_opts* o, const int32_t* old_labels, int32_t old_k,
                                          const uint64_t* old_leaf, const uint8_t* changed, int32_t* labels,
                                          uint64_t* leaf, int32_t* k_out, void* ws, size_t ws_bytes,
                                          raftgp_stream_t stream) {
    if (!changed) return fail(RAFTGP_EINVAL, "changed is NULL");
    return bisect_common(g, Z, d, z_dtype, o, old_labels, old_k, old_leaf, changed, labels, leaf, k_out, ws,
                         ws_bytes, (cudaStream_t)stream);
}

// ---- Algorithm 2 sampler and the CSR build ----
static raftgp_status check_sbm(const raftgp_sbm* p) {
    if (!p) return fail(RAFTGP_EINVAL, "sbm parameters are NULL");
    if (p->n < 1) return fail(RAFTGP_EINVAL, "sbm n must be >= 1");
    if (p->n > (int64_t)INT32_MAX - 1) return fail(RAFTGP_EUNSUPPORTED, "n above 2^31-2 is not supported");
    if (p->k < 1 || p->k > 65535) return fail(RAFTGP_EINVAL, "sbm k must be in 1..65535");
    if (!p->block || !p->theta || !p->omega) return fail(RAFTGP_EINVAL, "sbm arrays are NULL");
    return RAFTGP_OK;
}

size_t raftgp_sbm_workspace_size(int64_t n, int32_t k) {
    Carver c(nullptr);
    carve_sbm(c, n < 1 ? 1 : n, k < 1 ? 1 : k);
    return c.off + 256;
}

raftgp_status raftgp_sbm_count(const raftgp_sbm* p, int64_t* m, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_status st = check_sbm(p);
    if (st) return st;
    if (!m || !ws) return fail(RAFTGP_EINVAL, "NULL argument");
    if (ws_bytes < raftgp_sbm_workspace_size(p->n, p->k)) return fail(RAFTGP_ENOMEM, "workspace too small");
    Carver c(ws);
    SbmWs w = carve_sbm(c, p->n, p->k);
    int64_t G = 0;
    cudaError_t e = sbm_count(p, w, &G, m, (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return fail(RAFTGP_EINVAL, "sbm: a block outside [0, k) or a negative theta/Omega");
    if (e != cudaSuccess) return cuda_fail(e, "sbm count");
    return RAFTGP_OK;
}

raftgp_status raftgp_sbm_emit(const raftgp_sbm* p, int32_t* src, int32_t* dst, int32_t* weight, int64_t m, void* ws,
                              size_t ws_bytes, raftgp_stream_t stream) {
    raftgp_status st = check_sbm(p);
    if (st) return st;
    if ((m > 0 && (!src || !dst)) || !ws) return fail(RAFTGP_EINVAL, "NULL argument");
    if (ws_bytes < raftgp_sbm_workspace_size(p->n, p->k)) return fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    SbmWs w = carve_sbm(c, p->n, p->k);
    // the segment and edge counts the count pass left in the workspace
    const int64_t npairs = (int64_t)p->k * (p->k + 1) / 2;
    unsigned long long G = 0, mm = 0;
    cudaMemcpyAsync(&G, w.pincl + (npairs - 1), sizeof(G), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sbm emit");
    if ((int64_t)G > sbm_max_segments(p->n, p->k)) return fail(RAFTGP_EINVAL, "sbm emit without a count pass");
    if (G > 0) {
        cudaMemcpyAsync(&mm, w.seg_incl + (G - 1), sizeof(mm), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sbm emit");
    }
    if ((int64_t)mm != m) return fail(RAFTGP_EINVAL, "m = %lld differs from the count pass (%lld)", (long long)m,
                                      (long long)mm);
    e = sbm_emit(p, w, (int64_t)G, src, dst, weight, s);
    if (e != cudaSuccess) return cuda_fail(e, "sbm emit");
    return RAFTGP_OK;
}

size_t raftgp_coo_to_csr_workspace_size(int64_t n) {
    Carver c(nullptr);
    carve_csr_build(c, n < 1 ? 1 : n);
    return c.off + 256;
}

raftgp_status raftgp_coo_to_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* row_ptr,
                                int32_t* col, void* ws, size_t ws_bytes, raftgp_stream_t stream) {
    if (n < 1 || n > (int64_t)INT32_MAX - 1) return fail(RAFTGP_EINVAL, "n must be in 1..2^31-2");
    if (m < 0 || 2 * m >= ((int64_t)1 << 31)) return fail(RAFTGP_EUNSUPPORTED, "2 m must be below 2^31");
    if (!row_ptr || !ws || (m > 0 && (!src || !dst || !col))) return fail(RAFTGP_EINVAL, "NULL argument");
    if (ws_bytes < raftgp_coo_to_csr_workspace_size(n)) return fail(RAFTGP_ENOMEM, "workspace too small");
    Carver c(ws);
    CsrBuildWs w = carve_csr_build(c, n);
    uint32_t herr = 0;
    cudaError_t e = coo_to_csr(n, m, src, dst, row_ptr, col, w, &herr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "coo to csr");
    if (herr & (DERR_COL_RANGE | DERR_SELF_LOOP)) return fail(RAFTGP_EINVAL, "an endpoint outside [0, n) or a self loop");
    if (herr & DERR_ROW_PTR) return fail(RAFTGP_EUNSUPPORTED, "a row longer than 16384");
    return RAFTGP_OK;
}

}  // extern "C"
