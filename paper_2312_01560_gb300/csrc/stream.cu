// stream.cu -- the streaming extension of Section III-D: edges arrive, the embedding follows.
//
// A stream keeps the graph (a double-buffered CSR with room for nnz_cap stored entries) and
// every intermediate of the FP32 embedding with the NCut operator M = D^-1/2 A D^-1/2:
// Theta' (Theta_j d_j^-1/2), the inputs P_k = (d+1)^-1/2 (Z^(k-1) W_k) of each GCN gather and
// the output Z.  Adding a set E' of new edges:
//   1. checks E' (endpoints in range, no self loop, no edge already present or repeated) and
//      merges it into the other CSR buffer (old rows copied, new entries appended, the rows
//      of V' -- the endpoints of E' -- sorted again);
//   2. recomputes degrees and scales, and Theta' for the rows of V' (their d_j changed);
//   3. recomputes only the rows whose value changes: S_0 = V' u N(V') for the projection
//      (row i of M Theta' involves d_i, its neighbours and their d_j), then
//      S_k = S_{k-1} u N(S_{k-1}) for GCN layer k (Eq. 6 mixes each row with its neighbours;
//      the rows of V' also change their own scale (d+1)^-1/2 and lie in every S_k).
// The recomputed rows run through the same per-row kernels as a full embedding (rows above
// 256 neighbours by the CTA-per-row kernel), every other row keeps its stored value, so the
// result equals a full embedding of the new graph bit for bit.
//
// The modularity operators are not streamed: their 2e and d^T Theta reach every row.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

namespace {

__global__ void k_st_mark_edges(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, uint8_t* mask,
                                uint32_t* err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        if (u < 0 || u >= n || v < 0 || v >= n) {
            flag_error(err, DERR_COL_RANGE);
            continue;
        }
        if (u == v) {
            flag_error(err, DERR_SELF_LOOP);
            continue;
        }
        mask[u] = 1;
        mask[v] = 1;
    }
}

// An edge already in the (sorted) old graph is an error: binary search of v in row u.
__global__ void k_st_present(const int64_t* rp, const int32_t* col, const int32_t* src, const int32_t* dst,
                             int64_t m, int64_t n, uint32_t* err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
        int64_t lo = rp[u], hi = rp[u + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        if (lo < rp[u + 1] && col[lo] == v) flag_error(err, DERR_ROW_PTR);
    }
}

__global__ void k_st_degree(const int64_t* rp, int64_t n, const int32_t* src, const int32_t* dst, int64_t m,
                            unsigned long long* deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        deg[i] = (unsigned long long)(rp[i + 1] - rp[i]);
}

__global__ void k_st_degree_add(const int32_t* src, const int32_t* dst, int64_t m, unsigned long long* deg) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(deg + src[e], 1ull);
        atomicAdd(deg + dst[e], 1ull);
    }
}

__global__ void k_st_rowptr(const unsigned long long* incl, int64_t n, int64_t* rp_new) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        rp_new[i] = i == 0 ? 0 : (int64_t)incl[i - 1];
}

// warp per row: the old entries to their new place; fill = where the row's new entries go
__global__ void k_st_copy_rows(const int64_t* rp, const int32_t* col, int64_t n, const int64_t* rp_new,
                               int32_t* col_new, unsigned long long* fill) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t b = rp[i], len = rp[i + 1] - b, nb = rp_new[i];
        for (int64_t k = lane; k < len; k += 32) col_new[nb + k] = col[b + k];
        if (lane == 0) fill[i] = (unsigned long long)(nb + len);
    }
}

__global__ void k_st_scatter(const int32_t* src, const int32_t* dst, int64_t m, unsigned long long* fill,
                             int32_t* col_new) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        col_new[atomicAdd(fill + u, 1ull)] = v;
        col_new[atomicAdd(fill + v, 1ull)] = u;
    }
}

// a repeated entry in a sorted row of V' means E' listed an edge twice
__global__ void k_st_repeats(const int64_t* rp, int64_t n, const int32_t* col, const uint8_t* only, uint32_t* err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!only[i]) continue;
        for (int64_t p = rp[i] + 1; p < rp[i + 1]; ++p)
            if (col[p] == col[p - 1]) flag_error(err, DERR_ROW_PTR);
    }
}

// out = in u N(in): warp per marked row
__global__ void k_st_expand(const int64_t* rp, const int32_t* col, int64_t n, const uint8_t* in, uint8_t* out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        if (!in[i]) continue;
        if (lane == 0) out[i] = 1;
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) out[col[p]] = 1;
    }
}

// marked rows into a light list (degree <= 256) and a heavy list; counts[0], counts[1]
__global__ void k_st_lists(const uint8_t* mask, const int32_t* deg, int64_t n, int32_t* light, int32_t* heavy,
                           int* counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[i]) continue;
        if (deg[i] > 256) heavy[atomicAdd(counts + 1, 1)] = (int32_t)i;   // as launch_degrees classifies
        else light[atomicAdd(counts, 1)] = (int32_t)i;
    }
}

}  // namespace
}  // namespace raftgp

using namespace raftgp;

struct raftgp_stream {
    raftgp_embed_opts eo{};
    int64_t n = 0, nnz = 0, cap = 0;
    int cur = 0;
    int64_t* rp[2] = {nullptr, nullptr};
    int32_t* col[2] = {nullptr, nullptr};
    uint32_t* err = nullptr;
    int32_t* deg = nullptr;
    float *rs = nullptr, *rsh = nullptr;
    int32_t* heavy_all = nullptr;
    int* heavy_all_count = nullptr;
    float* W[RAFTGP_MAX_LAYERS] = {};
    float* theta = nullptr;
    float* P[RAFTGP_MAX_LAYERS + 1] = {};   // P[k]: the input of GCN gather k (1..L)
    float* Z = nullptr;
    uint8_t *mask_a = nullptr, *mask_b = nullptr, *mask_v = nullptr;
    int32_t *light = nullptr, *heavy = nullptr;
    int* counts = nullptr;
    unsigned long long *deg64 = nullptr, *incl = nullptr, *fill = nullptr, *tiles = nullptr;
    int* long_rows = nullptr;
    int* n_long = nullptr;
    int64_t affected[RAFTGP_MAX_LAYERS + 1] = {};
};

static raftgp_status st_fail(raftgp_status st, const char* what) { return set_error(st, "%s", what); }
static raftgp_status st_cuda(cudaError_t e, const char* where) {
    return set_error(RAFTGP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

static void carve_stream(Carver& c, raftgp_stream& s, int64_t n, int64_t cap, const raftgp_embed_opts* o) {
    for (int b = 0; b < 2; ++b) {
        s.rp[b] = c.take<int64_t>(n + 1);
        s.col[b] = c.take<int32_t>(cap);
    }
    s.err = c.take<uint32_t>(64);
    s.deg = c.take<int32_t>(n);
    s.rs = c.take<float>(n);
    s.rsh = c.take<float>(n);
    s.heavy_all = c.take<int32_t>(n);
    s.heavy_all_count = c.take<int>(64);
    for (int k = 1; k <= o->n_layers; ++k) s.W[k - 1] = c.take<float>((size_t)o->dims[k - 1] * o->dims[k]);
    s.theta = c.take<float>((size_t)n * o->dims[0]);
    for (int k = 1; k <= o->n_layers; ++k) s.P[k] = c.take<float>((size_t)n * o->dims[k]);
    s.Z = c.take<float>((size_t)n * o->dims[o->n_layers]);
    s.mask_a = c.take<uint8_t>(n);
    s.mask_b = c.take<uint8_t>(n);
    s.mask_v = c.take<uint8_t>(n);
    s.light = c.take<int32_t>(n);
    s.heavy = c.take<int32_t>(n);
    s.counts = c.take<int>(64);
    s.deg64 = c.take<unsigned long long>(n + 1);
    s.incl = c.take<unsigned long long>(n + 1);
    s.fill = c.take<unsigned long long>(n + 1);
    s.tiles = c.take<unsigned long long>((n + SCAN_TILE - 1) / SCAN_TILE + 1);
    s.long_rows = c.take<int>(n + 1);
    s.n_long = c.take<int>(64);
}

static raftgp_csr st_graph(const raftgp_stream& s) {
    raftgp_csr g;
    g.n = s.n;
    g.nnz = s.nnz;
    g.row_ptr = s.rp[s.cur];
    g.row_ptr_bits = 64;
    g.col = s.col[s.cur];
    return g;
}

static cudaError_t st_read_err(raftgp_stream& s, uint32_t* h, cudaStream_t cs) {
    cudaMemcpyAsync(h, s.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs);
    return cudaStreamSynchronize(cs);
}

// The gather of stage k (0: the projection, k >= 1: GCN layer k) for the listed rows, or
// for every row when rows == null.
static cudaError_t st_stage(raftgp_stream& s, int k, const raftgp_csr& g, const int32_t* light, int64_t nlight,
                            const int32_t* heavy, const int* heavy_count, cudaStream_t cs) {
    const raftgp_embed_opts* o = &s.eo;
    const int L = o->n_layers;
    if (k == 0)
        return launch_layer(AGG_NCUT_, RAFTGP_F32, &g, s.deg, s.rs, nullptr, 0, s.W[0], o->dims[0], o->dims[1], s.rsh,
                            s.theta, s.P[1], nullptr, heavy, heavy_count, cs, light, nlight);
    const bool last = k == L;
    return launch_layer(AGG_GCN_, RAFTGP_F32, &g, s.deg, s.rsh, nullptr, 1, last ? nullptr : s.W[k], o->dims[k],
                        last ? o->dims[k] : o->dims[k + 1], last ? nullptr : s.rsh, s.P[k], last ? (void*)s.Z : s.P[k + 1],
                        nullptr, heavy, heavy_count, cs, light, nlight);
}

extern "C" {

size_t raftgp_stream_workspace_size(int64_t n, int64_t nnz_cap, const raftgp_embed_opts* o) {
    if (!o || n < 1 || nnz_cap < 0 || o->n_layers < 1 || o->n_layers > RAFTGP_MAX_LAYERS) return 0;
    Carver c(nullptr);
    raftgp_stream s;
    carve_stream(c, s, n, nnz_cap, o);
    return c.off + 256;
}

raftgp_status raftgp_stream_create(const raftgp_csr* g, const raftgp_embed_opts* o, int64_t nnz_cap, void* ws,
                                   size_t ws_bytes, raftgp_stream** out, raftgp_stream_t stream) {
    if (!g || !o || !ws || !out) return st_fail(RAFTGP_EINVAL, "NULL argument");
    if (g->n < 1 || g->n > (int64_t)INT32_MAX - 1 || g->nnz < 0 || !g->row_ptr || (g->nnz > 0 && !g->col))
        return st_fail(RAFTGP_EINVAL, "malformed graph descriptor");
    if (g->row_ptr_bits != 32 && g->row_ptr_bits != 64) return st_fail(RAFTGP_EINVAL, "row_ptr_bits must be 32 or 64");
    if (o->op != RAFTGP_OP_NCUT)
        return st_fail(RAFTGP_EUNSUPPORTED, "streaming updates need the NCut operator (2e reaches every row otherwise)");
    if (o->dtype != RAFTGP_F32) return st_fail(RAFTGP_EUNSUPPORTED, "streaming updates keep FP32 state");
    if (o->n_layers < 1 || o->n_layers > RAFTGP_MAX_LAYERS) return st_fail(RAFTGP_EINVAL, "n_layers must be 1..4");
    for (int k = 0; k <= o->n_layers; ++k)
        if (o->dims[k] != 32 && o->dims[k] != 64 && o->dims[k] != 128)
            return st_fail(RAFTGP_EUNSUPPORTED, "widths must be 32, 64 or 128");
    if (o->theta) return st_fail(RAFTGP_EUNSUPPORTED, "a caller-supplied Theta is not streamed");
    if (nnz_cap < g->nnz || nnz_cap >= ((int64_t)1 << 31)) return st_fail(RAFTGP_EINVAL, "nnz_cap must be in [nnz, 2^31)");
    if (ws_bytes < raftgp_stream_workspace_size(g->n, nnz_cap, o)) return st_fail(RAFTGP_ENOMEM, "workspace too small");
    cudaStream_t cs = (cudaStream_t)stream;
    raftgp_stream* s = new (std::nothrow) raftgp_stream();
    if (!s) return st_fail(RAFTGP_ENOMEM, "host allocation");
    s->eo = *o;
    s->n = g->n;
    s->nnz = g->nnz;
    s->cap = nnz_cap;
    Carver c(ws);
    carve_stream(c, *s, g->n, nnz_cap, o);
    // the graph as int64 row pointers in buffer 0
    if (g->row_ptr_bits == 64) {
        cudaMemcpyAsync(s->rp[0], g->row_ptr, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToDevice, cs);
    } else {
        std::vector<int32_t> h(g->n + 1);
        std::vector<int64_t> h64(g->n + 1);
        cudaMemcpyAsync(h.data(), g->row_ptr, sizeof(int32_t) * (g->n + 1), cudaMemcpyDeviceToHost, cs);
        cudaStreamSynchronize(cs);
        for (int64_t i = 0; i <= g->n; ++i) h64[i] = h[i];
        cudaMemcpyAsync(s->rp[0], h64.data(), sizeof(int64_t) * (g->n + 1), cudaMemcpyHostToDevice, cs);
    }
    if (g->nnz > 0) cudaMemcpyAsync(s->col[0], g->col, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToDevice, cs);
    s->cur = 0;
    raftgp_csr cg = st_graph(*s);
    cudaMemsetAsync(s->err, 0, sizeof(uint32_t), cs);
    cudaMemsetAsync(s->heavy_all_count, 0, sizeof(int), cs);
    launch_degrees(&cg, s->deg, s->rs, s->rsh, s->err, s->heavy_all, s->heavy_all_count, cs);
    uint32_t h = 0;
    cudaError_t e = st_read_err(*s, &h, cs);
    if (e != cudaSuccess) { delete s; return st_cuda(e, "stream create"); }
    if (h) { delete s; return st_fail(RAFTGP_EINVAL, "malformed graph (device check flags)"); }
    for (int k = 1; k <= o->n_layers; ++k) {
        if (o->W[k - 1])
            cudaMemcpyAsync(s->W[k - 1], o->W[k - 1], sizeof(float) * (size_t)o->dims[k - 1] * o->dims[k],
                            cudaMemcpyDeviceToDevice, cs);
        else
            launch_weights(k, o->dims[k - 1], o->dims[k], o->seed, s->W[k - 1], cs);
    }
    launch_theta(g->n, o->dims[0], RAFTGP_F32, o->seed, nullptr, s->rs, nullptr, s->deg, s->theta, nullptr, nullptr, cs);
    for (int k = 0; k <= o->n_layers && e == cudaSuccess; ++k)
        e = st_stage(*s, k, cg, nullptr, 0, s->heavy_all, s->heavy_all_count, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) { delete s; return st_cuda(e, "stream create"); }
    for (int k = 0; k <= o->n_layers; ++k) s->affected[k] = g->n;
    *out = s;
    return RAFTGP_OK;
}

raftgp_status raftgp_stream_add_edges(raftgp_stream* s, const int32_t* src, const int32_t* dst, int64_t m,
                                      raftgp_stream_t stream) {
    if (!s) return st_fail(RAFTGP_EINVAL, "NULL stream");
    if (m < 0 || (m > 0 && (!src || !dst))) return st_fail(RAFTGP_EINVAL, "bad edge list");
    if (m == 0) {
        for (int k = 0; k <= s->eo.n_layers; ++k) s->affected[k] = 0;
        return RAFTGP_OK;
    }
    if (s->nnz + 2 * m > s->cap) return st_fail(RAFTGP_ENOMEM, "nnz_cap exceeded");
    cudaStream_t cs = (cudaStream_t)stream;
    const int64_t n = s->n;
    const int o = s->cur, t = 1 - s->cur;
    // 1. check E' and build the merged CSR in the other buffer
    cudaMemsetAsync(s->err, 0, sizeof(uint32_t), cs);
    cudaMemsetAsync(s->mask_v, 0, n, cs);
    k_st_mark_edges<<<grid_for(m, 256), 256, 0, cs>>>(src, dst, m, n, s->mask_v, s->err);
    k_st_present<<<grid_for(m, 256), 256, 0, cs>>>(s->rp[o], s->col[o], src, dst, m, n, s->err);
    uint32_t h = 0;
    cudaError_t e = st_read_err(*s, &h, cs);
    if (e != cudaSuccess) return st_cuda(e, "stream update");
    if (h & (DERR_COL_RANGE | DERR_SELF_LOOP)) return st_fail(RAFTGP_EINVAL, "an endpoint outside [0, n) or a self loop");
    if (h) return st_fail(RAFTGP_EINVAL, "an edge already in the graph");
    k_st_degree<<<grid_for(n, 256), 256, 0, cs>>>(s->rp[o], n, src, dst, m, s->deg64);
    k_st_degree_add<<<grid_for(m, 256), 256, 0, cs>>>(src, dst, m, s->deg64);
    scan_incl(s->deg64, n, s->incl, s->tiles, cs);
    k_st_rowptr<<<grid_for(n + 1, 256), 256, 0, cs>>>(s->incl, n, s->rp[t]);
    k_st_copy_rows<<<grid_for(n * 32, 256), 256, 0, cs>>>(s->rp[o], s->col[o], n, s->rp[t], s->col[t], s->fill);
    k_st_scatter<<<grid_for(m, 256), 256, 0, cs>>>(src, dst, m, s->fill, s->col[t]);
    e = sort_csr_rows(s->rp[t], n, s->col[t], s->mask_v, s->long_rows, s->n_long, s->err, cs);
    if (e != cudaSuccess) return st_cuda(e, "stream update");
    k_st_repeats<<<grid_for(n, 256), 256, 0, cs>>>(s->rp[t], n, s->col[t], s->mask_v, s->err);
    if ((e = st_read_err(*s, &h, cs)) != cudaSuccess) return st_cuda(e, "stream update");
    if (h) return st_fail(RAFTGP_EINVAL, "an edge listed twice, or a row longer than 16384");
    // 2. the new graph: degrees and scales, Theta' of V'
    s->cur = t;
    s->nnz += 2 * m;
    raftgp_csr g = st_graph(*s);
    cudaMemsetAsync(s->heavy_all_count, 0, sizeof(int), cs);
    launch_degrees(&g, s->deg, s->rs, s->rsh, s->err, s->heavy_all, s->heavy_all_count, cs);
    int hc[2] = {0, 0};
    cudaMemsetAsync(s->counts, 0, 2 * sizeof(int), cs);
    k_st_lists<<<grid_for(n, 256), 256, 0, cs>>>(s->mask_v, s->deg, n, s->light, s->heavy, s->counts);
    cudaMemcpyAsync(hc, s->counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, cs);
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return st_cuda(e, "stream update");
    launch_theta(hc[0], s->eo.dims[0], RAFTGP_F32, s->eo.seed, nullptr, s->rs, nullptr, s->deg, s->theta, nullptr,
                 nullptr, cs, s->light, hc[0]);
    launch_theta(hc[1], s->eo.dims[0], RAFTGP_F32, s->eo.seed, nullptr, s->rs, nullptr, s->deg, s->theta, nullptr,
                 nullptr, cs, s->heavy, hc[1]);
    // 3. the rows of every stage whose value changes: S_0 = V' u N(V'), S_k = S_{k-1} u N(S_{k-1})
    uint8_t* in = s->mask_v;
    uint8_t* bufs[2] = {s->mask_a, s->mask_b};
    for (int k = 0; k <= s->eo.n_layers; ++k) {
        uint8_t* outm = bufs[k & 1];
        cudaMemcpyAsync(outm, in, n, cudaMemcpyDeviceToDevice, cs);
        k_st_expand<<<grid_for(n * 32, 256), 256, 0, cs>>>(s->rp[t], s->col[t], n, in, outm);
        cudaMemsetAsync(s->counts, 0, 2 * sizeof(int), cs);
        k_st_lists<<<grid_for(n, 256), 256, 0, cs>>>(outm, s->deg, n, s->light, s->heavy, s->counts);
        cudaMemcpyAsync(hc, s->counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, cs);
        if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return st_cuda(e, "stream update");
        s->affected[k] = (int64_t)hc[0] + hc[1];
        e = st_stage(*s, k, g, s->light, hc[0], s->heavy, s->counts + 1, cs);
        if (e != cudaSuccess) return st_cuda(e, "stream update");
        in = outm;
    }
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return st_cuda(e, "stream update");
    return RAFTGP_OK;
}

raftgp_status raftgp_stream_info(const raftgp_stream* s, int64_t* n, int64_t* nnz, int64_t* affected) {
    if (!s) return st_fail(RAFTGP_EINVAL, "NULL stream");
    if (n) *n = s->n;
    if (nnz) *nnz = s->nnz;
    if (affected)
        for (int k = 0; k <= s->eo.n_layers; ++k) affected[k] = s->affected[k];
    return RAFTGP_OK;
}

raftgp_status raftgp_stream_copy(const raftgp_stream* s, int64_t* row_ptr, int32_t* col, float* Z,
                                 raftgp_stream_t stream) {
    if (!s) return st_fail(RAFTGP_EINVAL, "NULL stream");
    cudaStream_t cs = (cudaStream_t)stream;
    if (row_ptr) cudaMemcpyAsync(row_ptr, s->rp[s->cur], sizeof(int64_t) * (s->n + 1), cudaMemcpyDeviceToDevice, cs);
    if (col && s->nnz > 0) cudaMemcpyAsync(col, s->col[s->cur], sizeof(int32_t) * s->nnz, cudaMemcpyDeviceToDevice, cs);
    if (Z)
        cudaMemcpyAsync(Z, s->Z, sizeof(float) * (size_t)s->n * s->eo.dims[s->eo.n_layers], cudaMemcpyDeviceToDevice,
                        cs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return st_cuda(e, "stream copy");
    return RAFTGP_OK;
}

void raftgp_stream_destroy(raftgp_stream* s) { delete s; }

}  // extern "C"
