// embed.cu -- stages 1 and 2 of RaftGP (Section III-A, Eq. 5; Section III-B, Eq. 6).
//
// Data flow for n_layers >= 1 (all feature matrices row-major, storage type T = float or bf16,
// FP32 accumulation):
//   degrees:   d_i, rs_i = d_i^-1/2 (0 if isolated), rsh_i = (d_i + 1)^-1/2
//   Theta':    Theta_j * (rs_j for M, 1 otherwise)                (Philox, N x L)
//   g:         d^T Theta (FP64, only for the full modularity matrix)
//   layer 0:   Y_i = sum_j Theta'_j, then the operator's row epilogue (x rs_i, or minus the
//              rank-one term, or the Q-tilde weights), then P1'_i = rsh_i * (Y_i W1)
//   layer k:   H_i = rsh_i * (P'_i + sum_j P'_j)  ( = (D-hat^-1/2 (A+I) D-hat^-1/2 Z W)_i ),
//              Z^(k)_i = rownorm(tanh(H_i)), then P'_{k+1} = rsh_i * (Z^(k)_i W_{k+1})
// The weight product is applied before the aggregation (Z W, then aggregate): the same
// matrix product as Eq. 6, cheaper when W narrows the width.  Prescaling the gathered
// rows by their column weight (rs_j or rsh_j) makes every SpMM an unweighted gather-sum.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

// ------------------------------------------------------------------------------------
// Degrees, reciprocal square roots and graph checks (8 lanes per row, 4 rows per warp).
// ------------------------------------------------------------------------------------
__global__ void k_degrees(int64_t n, int64_t nnz, const int32_t* rp32, const int64_t* rp64, const int32_t* col,
                          int32_t* deg, float* rs, float* rsh, uint32_t* err, int32_t* heavy, int* heavy_count) {
    const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (warp == 0 && lane == 0) {
        const int64_t first = rp64 ? rp64[0] : rp32[0];
        const int64_t last = rp64 ? rp64[n] : rp32[n];
        if (first != 0 || last != nnz) flag_error(err, DERR_ROW_PTR);
    }
    const unsigned gmask = 0xffu << (8 * grp);   // this row's lanes
    for (int64_t i0 = warp * 4; i0 < n; i0 += nwarps * 4) {
        const int64_t i = i0 + grp;
        const bool valid = i < n;
        int64_t b = 0, e = 0;
        bool bad_rp = false;
        if (valid) {
            b = rp64 ? rp64[i] : rp32[i];
            e = rp64 ? rp64[i + 1] : rp32[i + 1];
            bad_rp = e < b || b < 0 || e > nnz;
        }
        bool bad_range = false, bad_loop = false;
        if (valid && !bad_rp) {
            for (int64_t p = b + sub; p < e; p += 8) {
                const int32_t j = __ldg(col + p);
                bad_range |= (j < 0 || (int64_t)j >= n);
                bad_loop |= ((int64_t)j == i);
            }
        }
        const unsigned mr = __ballot_sync(0xffffffffu, bad_range), ml = __ballot_sync(0xffffffffu, bad_loop);
        if (valid && sub == 0) {
            if (bad_rp) {
                flag_error(err, DERR_ROW_PTR);
            } else {
                if (mr & gmask) flag_error(err, DERR_COL_RANGE);
                if (ml & gmask) flag_error(err, DERR_SELF_LOOP);
                const int64_t d = e - b;
                deg[i] = (int32_t)d;
                rs[i] = d > 0 ? rsqrtf((float)d) : 0.0f;
                rsh[i] = rsqrtf((float)(d + 1));
                if (heavy && d > 256) heavy[atomicAdd(heavy_count, 1)] = (int32_t)i;   // HEAVY_DEG
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Theta (Eq. 5): Theta_jr ~ N(0, 1/L), four columns per Philox block with counter
// (q, j_lo, j_hi, "Thet").  Stored prescaled by `colscale_j` (rs_j for M).  For the full
// modularity matrix the same kernel forms per-block FP32 partials of d_j * Theta_jr
// (from the stored, rounded values), reduced over blocks in FP64 by k_rank1_finish.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_theta(int64_t n, int L, uint64_t seed, const float* user_theta, const float* colscale,
                        const int32_t* deg, T* theta, double* partial, const int32_t* local_row,
                        const int32_t* rows) {
    const int tpr = L / 4;                       // threads per row
    const int slots = blockDim.x / tpr;          // rows per block iteration
    const int q = threadIdx.x % tpr;
    const int slot = threadIdx.x / tpr;
    const float sigma = rsqrtf((float)L);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t jq = (int64_t)blockIdx.x * slots + slot; jq < n; jq += (int64_t)gridDim.x * slots) {
        const int64_t j = rows ? (int64_t)rows[jq] : jq;   // with a row list, n counts its entries
        float g[4];
        if (user_theta) {
#pragma unroll
            for (int s = 0; s < 4; ++s) g[s] = user_theta[j * L + 4 * q + s];
        } else {
            // the row counter is the node's index inside its own graph when several graphs share
            // one concatenated CSR
            const int64_t jr = local_row ? (int64_t)local_row[j] : j;
            const U32x4 x = philox4x32_10((uint32_t)q, (uint32_t)jr, (uint32_t)((uint64_t)jr >> 32), STREAM_THETA, seed);
            box_muller(x.x, x.y, g[0], g[1]);
            box_muller(x.z, x.w, g[2], g[3]);
#pragma unroll
            for (int s = 0; s < 4; ++s) g[s] *= sigma;
        }
        const float cs = colscale ? colscale[j] : 1.0f;
        T out[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) out[s] = Vec<T>::from_float(g[s] * cs);
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4*>(theta + j * L + 4 * q) =
                make_float4(Vec<T>::to_float(out[0]), Vec<T>::to_float(out[1]), Vec<T>::to_float(out[2]),
                            Vec<T>::to_float(out[3]));
        } else {
#pragma unroll
            for (int s = 0; s < 4; ++s) theta[j * L + 4 * q + s] = out[s];
        }
        if (partial) {
            const float dj = (float)deg[j];
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[s] += dj * Vec<T>::to_float(out[s]);
        }
    }
    if (!partial) return;
    extern __shared__ float sred[];  // [slots][L]
#pragma unroll
    for (int s = 0; s < 4; ++s) sred[slot * L + 4 * q + s] = acc[s];
    __syncthreads();
    for (int c = threadIdx.x; c < L; c += blockDim.x) {
        double t = 0.0;
        for (int r = 0; r < slots; ++r) t += (double)sred[r * L + c];
        partial[(int64_t)blockIdx.x * L + c] = t;
    }
}

__global__ void k_rank1_finish(int nblocks, int L, const double* partial, float* g) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * L + c];
    g[c] = (float)t;
}

// Per-graph rank-one term of the full modularity matrix when several graphs share one CSR: a
// block per graph; thread (slot, q) sums d_j Theta_j,4q..4q+3 over the graph's rows slot,
// slot + slots, ... in FP64, the slots are added in ascending order, and 2e = sum_j d_j (exact).
template <typename T>
__global__ void k_rank1_graphs(int ng, const int64_t* __restrict__ off, int L, const T* __restrict__ theta,
                               const int32_t* __restrict__ deg, float* g_graph, double* inv_two_e_graph) {
    extern __shared__ double sr[];   // [slots][L]
    const int tpr = L / 4, slots = blockDim.x / tpr;
    const int q = threadIdx.x % tpr, slot = threadIdx.x / tpr;
    __shared__ long long s_two_e;
    for (int g = blockIdx.x; g < ng; g += gridDim.x) {
        const int64_t a = off[g], b = off[g + 1];
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        long long te = 0;
        // U of this slot's rows loaded before any is added (a graph of 50k rows is otherwise 6k
        // dependent round trips for its block); the additions keep the row order
        constexpr int U = 8;
        if (slot < slots)
            for (int64_t j0 = a + slot; j0 < b; j0 += (int64_t)slots * U) {
                int dj[U];
                float th[U][4];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t j = j0 + (int64_t)u * slots;
                    dj[u] = j < b ? deg[j] : 0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) th[u][c] = j < b ? Vec<T>::to_float(theta[j * L + 4 * q + c]) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (j0 + (int64_t)u * slots >= b) break;
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[c] += (double)dj[u] * (double)th[u][c];
                    if (q == 0) te += dj[u];
                }
            }
        if (threadIdx.x == 0) s_two_e = 0;
        __syncthreads();
        if (slot < slots) {
#pragma unroll
            for (int c = 0; c < 4; ++c) sr[slot * L + 4 * q + c] = acc[c];
            if (q == 0 && te) atomicAdd(reinterpret_cast<unsigned long long*>(&s_two_e), (unsigned long long)te);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < L; c += blockDim.x) {
            double t = 0.0;
            for (int r = 0; r < slots; ++r) t += sr[r * L + c];
            g_graph[(int64_t)g * L + c] = (float)t;
        }
        if (threadIdx.x == 0) inv_two_e_graph[g] = s_two_e > 0 ? 1.0 / (double)s_two_e : 0.0;
        __syncthreads();
    }
}

void launch_rank1_graphs(int ng, const int64_t* off, int L, int dtype, const void* theta, const int32_t* deg,
                         float* g_graph, double* inv_two_e_graph, cudaStream_t s) {
    const int threads = 256;
    const size_t sm = (size_t)(threads / (L / 4)) * L * sizeof(double);
    const int blocks = ng < num_sms() * 4 ? ng : num_sms() * 4;
    ProfScope ps(s, PF_THETA, 1);
    if (dtype == RAFTGP_BF16)
        k_rank1_graphs<__nv_bfloat16><<<blocks, threads, sm, s>>>(ng, off, L, (const __nv_bfloat16*)theta, deg, g_graph,
                                                                  inv_two_e_graph);
    else
        k_rank1_graphs<float><<<blocks, threads, sm, s>>>(ng, off, L, (const float*)theta, deg, g_graph, inv_two_e_graph);
}

// GCN weights W^(k), Xavier-normal, entry (a, 4q+s) from Philox block (q, a, k, "Wgnn").
__global__ void k_weights(int layer, int lin, int lout, uint64_t seed, float* W) {
    const int qn = lout / 4;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= lin * qn) return;
    const int a = t / qn, q = t % qn;
    const float s = sqrtf(2.0f / (float)(lin + lout));
    const U32x4 x = philox4x32_10((uint32_t)q, (uint32_t)a, (uint32_t)layer, STREAM_W, seed);
    float g[4];
    box_muller(x.x, x.y, g[0], g[1]);
    box_muller(x.z, x.w, g[2], g[3]);
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) W[a * lout + 4 * q + s2] = s * g[s2];
}

// ------------------------------------------------------------------------------------
// The SpMM layer: warp per row, lanes split the 16-byte chunks of a gathered row, several
// neighbour rows in flight per warp, FP32 accumulation, fused row epilogue.
// ------------------------------------------------------------------------------------
enum Agg { AGG_NCUT = 0, AGG_MOD_FULL = 1, AGG_MOD_REDUCED = 2, AGG_GCN = 3 };

struct LayerArgs {
    int64_t n;
    const int32_t* rp32;
    const int64_t* rp64;
    const int32_t* col;
    const int32_t* deg;
    const float* rowscale;   // rs (M) or rsh (GCN): multiplies the aggregate
    const float* g;          // d^T Theta for the full modularity matrix
    double inv_two_e;        // 1 / 2e
    int act;                 // 0: none, 1: tanh then row l2-normalisation, 2: normalisation only
    const float* W;          // LIN x lout FP32, or null
    int lout;
    const float* postscale;  // multiplies the W product (rsh for the next GCN gather), or null
    void* out;               // N x (W ? lout : LIN) in T
    void* stage;             // optional N x LIN in T: the activated row before W
    const int32_t* heavy;    // rows gathered by k_spmm_heavy (null: every row by k_spmm_layer)
    const int* heavy_count;
    const int32_t* rows;     // the rows k_spmm_layer gathers (null: 0 .. n-1)
    int64_t nrows;
};

// Rows with more neighbours than this are gathered by a whole CTA (k_spmm_heavy) instead of
// one warp: on power-law graphs they carry a large share of the entries.
constexpr int HEAVY_DEG = 256;

template <typename T, int LIN>
struct Lanes {
    static constexpr int E = Vec<T>::E;   // elements per lane chunk (16 bytes)
    static constexpr int LPR = LIN / E;   // lanes per gathered row
    static constexpr int GPW = 32 / LPR;  // rows gathered concurrently per warp
    static constexpr int U = 8;           // unrolled gathers per lane
    static_assert(LPR >= 1 && LPR <= 32 && (32 % LPR) == 0, "bad width");
};

// Issues this lane's U gathers of chunk positions t + u GPW + grp (column indices held one per
// lane in my_col, cnt of them valid); rows are kept as raw 16-byte words until added.
template <int AGG, typename T, int LIN>
__device__ __forceinline__ void gather_issue(const T* __restrict__ X, int32_t my_col, float my_d, int cnt, int t,
                                             int grp, int sub, uint4 (&r)[Lanes<T, LIN>::U],
                                             float (&dj)[Lanes<T, LIN>::U]) {
    using Ln = Lanes<T, LIN>;
#pragma unroll
    for (int u = 0; u < Ln::U; ++u) {
        const int idx = t + u * Ln::GPW + grp;
        const int src = idx < cnt ? idx : 0;
        const int32_t j = __shfl_sync(0xffffffffu, my_col, src);
        if constexpr (AGG == AGG_MOD_REDUCED) dj[u] = __shfl_sync(0xffffffffu, my_d, src);
        if (idx < cnt) {
            r[u] = Vec<T>::load_raw(X + (int64_t)j * LIN + sub * Ln::E);
        } else {
            r[u] = make_uint4(0u, 0u, 0u, 0u);
            dj[u] = 0.f;
        }
    }
}

template <int AGG, typename T, int LIN>
__device__ __forceinline__ void gather_add(const uint4 (&r)[Lanes<T, LIN>::U], const float (&dj)[Lanes<T, LIN>::U],
                                           float* acc, float* accd) {
    using Ln = Lanes<T, LIN>;
#pragma unroll
    for (int u = 0; u < Ln::U; ++u) {
        float v[Ln::E];
        Vec<T>::unpack(r[u], v);
#pragma unroll
        for (int e = 0; e < Ln::E; ++e) {
            acc[e] += v[e];
            if constexpr (AGG == AGG_MOD_REDUCED) accd[e] += dj[u] * v[e];
        }
    }
}

// Gathers chunk positions [t0, cnt) of one chunk of at most 32 neighbours.
template <int AGG, typename T, int LIN>
__device__ __forceinline__ void gather_chunk(const T* __restrict__ X, int32_t my_col, float my_d, int cnt, int t0,
                                             int grp, int sub, float* acc, float* accd) {
    using Ln = Lanes<T, LIN>;
    for (int t = t0; t < cnt; t += Ln::GPW * Ln::U) {
        uint4 r[Ln::U];
        float dj[Ln::U];
        gather_issue<AGG, T, LIN>(X, my_col, my_d, cnt, t, grp, sub, r, dj);
        gather_add<AGG, T, LIN>(r, dj, acc, accd);
    }
}

// Adds X[col[p]] for p in [beg, end) to this lane's chunk of the row sum (and, for the
// reduced modularity operator, the d_j-weighted sum).  Lane groups take different neighbours;
// the caller combines the groups.
template <int AGG, typename T, int LIN>
__device__ __forceinline__ void gather_range(const LayerArgs& a, const T* __restrict__ X, int64_t beg, int64_t end,
                                             int lane, float* acc, float* accd) {
    using Ln = Lanes<T, LIN>;
    const int grp = lane / Ln::LPR, sub = lane % Ln::LPR;
    for (int64_t base = beg; base < end; base += 32) {
        const int cnt = (int)((end - base) < 32 ? (end - base) : 32);
        const int32_t my_col = lane < cnt ? __ldg(a.col + base + lane) : 0;
        float my_d = 0.f;
        if constexpr (AGG == AGG_MOD_REDUCED) my_d = lane < cnt ? (float)__ldg(a.deg + my_col) : 0.f;
        gather_chunk<AGG, T, LIN>(X, my_col, my_d, cnt, 0, grp, sub, acc, accd);
    }
}

// Combines the lane groups of a warp: afterwards every group holds the warp's row sum.
template <int AGG, typename T, int LIN>
__device__ __forceinline__ void combine_groups(float* acc, float* accd) {
    using Ln = Lanes<T, LIN>;
#pragma unroll
    for (int o = 16; o >= Ln::LPR; o >>= 1) {
#pragma unroll
        for (int e = 0; e < Ln::E; ++e) {
            acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
            if constexpr (AGG == AGG_MOD_REDUCED) accd[e] += __shfl_xor_sync(0xffffffffu, accd[e], o);
        }
    }
}

// Row epilogue of row i from its full neighbour sum (held by every lane group): the operator's
// row term, the activation, the optional stage output, then either the plain output row or
// the dense layer out_i = postscale_i * (y W).  Executed by one full warp.
template <int AGG, typename T, int LIN>
__device__ __forceinline__ void row_epilogue(const LayerArgs& a, int64_t i, const float* acc, const float* accd,
                                             int lane, float* vbuf, const float* Ws) {
    using Ln = Lanes<T, LIN>;
    constexpr int E = Ln::E, LPR = Ln::LPR;
    const int grp = lane / LPR, sub = lane % LPR;
    float y[E];
    if constexpr (AGG == AGG_NCUT || AGG == AGG_GCN) {
        const float s = a.rowscale[i];
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = s * acc[e];
    } else if constexpr (AGG == AGG_MOD_FULL) {
        const float c = (float)((double)a.deg[i] * a.inv_two_e);
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = acc[e] - c * a.g[sub * E + e];
    } else {
        const float c = (float)((double)a.deg[i] * a.inv_two_e);
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = acc[e] - c * accd[e];
    }
    if (a.act != 0) {
        float ss = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (a.act == 1) y[e] = tanhf(y[e]);
            ss += y[e] * y[e];
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] *= inv;
    }
    if (a.stage && grp == 0) Vec<T>::store(reinterpret_cast<T*>(a.stage) + i * LIN + sub * E, y);
    if (!a.W) {
        if (grp == 0) Vec<T>::store(reinterpret_cast<T*>(a.out) + i * LIN + sub * E, y);
        return;
    }
    // dense layer: lane computes lout/32 adjacent columns from W in shared memory
    if (grp == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) vbuf[sub * E + e] = y[e];
    }
    __syncwarp();
    const float ps = a.postscale ? a.postscale[i] : 1.0f;
    T* orow = reinterpret_cast<T*>(a.out) + i * a.lout;
    if (a.lout == 128) {
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int k = 0; k < LIN; ++k) {
            const float yk = vbuf[k];
            const float4 w = *reinterpret_cast<const float4*>(Ws + k * 128 + 4 * lane);
            o[0] += yk * w.x; o[1] += yk * w.y; o[2] += yk * w.z; o[3] += yk * w.w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) orow[4 * lane + c] = Vec<T>::from_float(o[c] * ps);
    } else if (a.lout == 64) {
        float o[2] = {0.f, 0.f};
#pragma unroll 8
        for (int k = 0; k < LIN; ++k) {
            const float yk = vbuf[k];
            const float2 w = *reinterpret_cast<const float2*>(Ws + k * 64 + 2 * lane);
            o[0] += yk * w.x; o[1] += yk * w.y;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) orow[2 * lane + c] = Vec<T>::from_float(o[c] * ps);
    } else {
        float o = 0.f;
#pragma unroll 8
        for (int k = 0; k < LIN; ++k) o += vbuf[k] * Ws[k * 32 + lane];
        orow[lane] = Vec<T>::from_float(o * ps);
    }
    __syncwarp();
}

// Light rows: one warp per row (grid-stride), FP32 accumulation, fused row epilogue.
template <int AGG, typename T, int LIN>
__global__ void __launch_bounds__(256, 4) k_spmm_layer(LayerArgs a, const T* __restrict__ X) {
    constexpr int E = Lanes<T, LIN>::E;
    extern __shared__ float smem[];
    float* Ws = smem;                                       // LIN x lout
    float* vbuf = smem + (a.W ? LIN * a.lout : 0) + (threadIdx.x >> 5) * LIN;
    if (a.W) {
        for (int t = threadIdx.x; t < LIN * a.lout; t += blockDim.x) Ws[t] = a.W[t];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int grp = lane / Lanes<T, LIN>::LPR, sub = lane % Lanes<T, LIN>::LPR;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // Software pipeline over the warp's rows: the next row's bounds and first 32 column indices
    // are loaded while this row's first gathers are in flight.
    // rows are visited by index q (row a.rows[q] with a list, else q)
    const int64_t count = a.rows ? a.nrows : a.n;
    int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t beg = 0, end = 0;
    int32_t my_col = 0;
    if (q < count) {
        const int64_t r0 = a.rows ? (int64_t)a.rows[q] : q;
        beg = a.rp64 ? a.rp64[r0] : a.rp32[r0];
        end = a.rp64 ? a.rp64[r0 + 1] : a.rp32[r0 + 1];
        const int c0 = (a.heavy && end - beg > HEAVY_DEG) ? 0 : (int)(end - beg < 32 ? end - beg : 32);
        my_col = lane < c0 ? __ldg(a.col + beg + lane) : 0;
    }
    for (; q < count; q += nwarps) {
        const int64_t i = a.rows ? (int64_t)a.rows[q] : q;
        const int64_t qnext = q + nwarps;
        int64_t nbeg = 0, nend = 0;
        if (qnext < count) {
            const int64_t inext = a.rows ? (int64_t)a.rows[qnext] : qnext;
            nbeg = a.rp64 ? a.rp64[inext] : a.rp32[inext];
            nend = a.rp64 ? a.rp64[inext + 1] : a.rp32[inext + 1];
        }
        const bool heavy_row = a.heavy && end - beg > HEAVY_DEG;   // gathered by k_spmm_heavy
        const int cnt = heavy_row ? 0 : (int)(end - beg < 32 ? end - beg : 32);
        float my_d = 0.f;
        if constexpr (AGG == AGG_MOD_REDUCED) my_d = lane < cnt ? (float)__ldg(a.deg + my_col) : 0.f;
        float acc[E];
        float accd[AGG == AGG_MOD_REDUCED ? E : 1];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        if constexpr (AGG == AGG_MOD_REDUCED) {
#pragma unroll
            for (int e = 0; e < E; ++e) accd[e] = 0.f;
        }
        uint4 r[Lanes<T, LIN>::U];
        float dj[Lanes<T, LIN>::U];
        gather_issue<AGG, T, LIN>(X, my_col, my_d, cnt, 0, grp, sub, r, dj);
        if constexpr (AGG == AGG_GCN) {
            if (grp == 0 && !heavy_row) Vec<T>::load(X + i * LIN + sub * E, acc);   // the self loop of A + I
        }
        const int ncnt = (a.heavy && nend - nbeg > HEAVY_DEG) ? 0 : (int)(nend - nbeg < 32 ? nend - nbeg : 32);
        const int32_t ncol = lane < ncnt ? __ldg(a.col + nbeg + lane) : 0;
        if (!heavy_row) {
            gather_add<AGG, T, LIN>(r, dj, acc, accd);
            gather_chunk<AGG, T, LIN>(X, my_col, my_d, cnt, Lanes<T, LIN>::GPW * Lanes<T, LIN>::U, grp, sub, acc,
                                      accd);
            if (end - beg > 32) gather_range<AGG, T, LIN>(a, X, beg + 32, end, lane, acc, accd);
            combine_groups<AGG, T, LIN>(acc, accd);
            row_epilogue<AGG, T, LIN>(a, i, acc, accd, lane, vbuf, a.W ? Ws : nullptr);
        }
        beg = nbeg;
        end = nend;
        my_col = ncol;
    }
}

// Heavy rows: one CTA of 8 warps per row; each warp gathers a fixed slice of the neighbour
// list, the slices are added in warp order (deterministic), then warp 0 runs the epilogue.
template <int AGG, typename T, int LIN>
__global__ void __launch_bounds__(256) k_spmm_heavy(LayerArgs a, const T* __restrict__ X) {
    constexpr int E = Lanes<T, LIN>::E, LPR = Lanes<T, LIN>::LPR;
    constexpr int NW = 8;
    extern __shared__ float smem[];
    float* Ws = smem;                                       // LIN x lout
    float* vbuf = smem + (a.W ? LIN * a.lout : 0);          // LIN
    float* part = vbuf + LIN;                               // NW x LIN (and NW x LIN for accd)
    if (a.W) {
        for (int t = threadIdx.x; t < LIN * a.lout; t += blockDim.x) Ws[t] = a.W[t];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / LPR, sub = lane % LPR;
    const int nheavy = *a.heavy_count;
    for (int h = blockIdx.x; h < nheavy; h += gridDim.x) {
        const int64_t i = a.heavy[h];
        const int64_t beg = a.rp64 ? a.rp64[i] : a.rp32[i];
        const int64_t end = a.rp64 ? a.rp64[i + 1] : a.rp32[i + 1];
        const int64_t chunk = ((end - beg + NW - 1) / NW + 31) / 32 * 32;
        const int64_t b0 = beg + w * chunk;
        const int64_t b1 = b0 + chunk < end ? b0 + chunk : end;
        float acc[E];
        float accd[AGG == AGG_MOD_REDUCED ? E : 1];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        if constexpr (AGG == AGG_MOD_REDUCED) {
#pragma unroll
            for (int e = 0; e < E; ++e) accd[e] = 0.f;
        }
        if constexpr (AGG == AGG_GCN) {
            if (w == 0 && grp == 0) Vec<T>::load(X + i * LIN + sub * E, acc);   // the self loop of A + I
        }
        if (b0 < b1) gather_range<AGG, T, LIN>(a, X, b0, b1, lane, acc, accd);
        combine_groups<AGG, T, LIN>(acc, accd);
        __syncthreads();   // previous row's epilogue is done with part[]
        if (grp == 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                part[w * LIN + sub * E + e] = acc[e];
                if constexpr (AGG == AGG_MOD_REDUCED) part[(NW + w) * LIN + sub * E + e] = accd[e];
            }
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                float s = 0.f, sd = 0.f;
                for (int q = 0; q < NW; ++q) {
                    s += part[q * LIN + sub * E + e];
                    if constexpr (AGG == AGG_MOD_REDUCED) sd += part[(NW + q) * LIN + sub * E + e];
                }
                acc[e] = s;
                if constexpr (AGG == AGG_MOD_REDUCED) accd[e] = sd;
            }
            row_epilogue<AGG, T, LIN>(a, i, acc, accd, lane, vbuf, a.W ? Ws : nullptr);
        }
    }
}

// ------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------
static int g_num_sms = 0;
int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

void launch_degrees(const raftgp_csr* g, int32_t* deg, float* rs, float* rsh, uint32_t* err, int32_t* heavy,
                    int* heavy_count, cudaStream_t s) {
    if (heavy) cudaMemsetAsync(heavy_count, 0, sizeof(int), s);
    const int threads = 256;
    int64_t blocks = (g->n * 32 + threads - 1) / threads;
    blocks = blocks < 1 ? 1 : (blocks > (int64_t)num_sms() * 16 ? (int64_t)num_sms() * 16 : blocks);
    ProfScope ps(s, PF_DEGREES, 1);
    k_degrees<<<(unsigned)blocks, threads, 0, s>>>(
        g->n, g->nnz, g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr,
        g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr, g->col, deg, rs, rsh, err, heavy, heavy_count);
}

int theta_blocks(int64_t n) {
    int64_t b = (n + 31) / 32;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

void launch_theta(int64_t n, int L, int dtype, uint64_t seed, const float* user_theta, const float* colscale, const int32_t* local_row,
                  const int32_t* deg, void* theta, double* partial, float* gvec, cudaStream_t s, const int32_t* rows,
                  int64_t nrows) {
    const int threads = 256;
    if (rows) {
        n = nrows;          // the listed rows only (no rank-one partials)
        partial = nullptr;
        if (n == 0) return;
    }
    const int blocks = theta_blocks(n);
    const size_t sm = partial ? (size_t)(threads / (L / 4)) * L * sizeof(float) : 0;
    ProfScope ps(s, PF_THETA, partial ? 2 : 1);
    if (dtype == RAFTGP_BF16)
        k_theta<__nv_bfloat16><<<blocks, threads, sm, s>>>(n, L, seed, user_theta, colscale, deg,
                                                           (__nv_bfloat16*)theta, partial, local_row, rows);
    else
        k_theta<float><<<blocks, threads, sm, s>>>(n, L, seed, user_theta, colscale, deg, (float*)theta, partial,
                                                   local_row, rows);
    if (partial) k_rank1_finish<<<(L + 127) / 128, 128, 0, s>>>(blocks, L, partial, gvec);
}

void launch_weights(int layer, int lin, int lout, uint64_t seed, float* W, cudaStream_t s) {
    const int total = lin * (lout / 4);
    ProfScope ps(s, PF_OTHER, 1);
    k_weights<<<(total + 255) / 256, 256, 0, s>>>(layer, lin, lout, seed, W);
}

template <int AGG, typename T, int LIN>
static cudaError_t launch_layer_t(const LayerArgs& a, const void* X, cudaStream_t s) {
    const int threads = 256;
    const size_t smem = (size_t)((a.W ? LIN * a.lout : 0) + (threads / 32) * LIN) * sizeof(float);
    auto kern = k_spmm_layer<AGG, T, LIN>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t count = a.rows ? a.nrows : a.n;
    int64_t blocks = (count + (threads / 32) - 1) / (threads / 32);
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    ProfScope ps(s, AGG == AGG_GCN ? PF_SPMM_GCN : PF_SPMM_PROJ, a.heavy ? 2 : 1);
    if (count > 0) kern<<<(unsigned)blocks, threads, smem, s>>>(a, reinterpret_cast<const T*>(X));
    if (a.heavy) {
        const size_t hsmem = (size_t)((a.W ? LIN * a.lout : 0) + LIN + 2 * 8 * LIN) * sizeof(float);
        auto hk = k_spmm_heavy<AGG, T, LIN>;
        if (hsmem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
            if (e != cudaSuccess) return e;
        }
        hk<<<(unsigned)(num_sms() * 4), 256, hsmem, s>>>(a, reinterpret_cast<const T*>(X));
    }
    return cudaGetLastError();
}

template <int AGG, typename T>
static cudaError_t launch_layer_w(const LayerArgs& a, int lin, const void* X, cudaStream_t s) {
    switch (lin) {
        case 32: return launch_layer_t<AGG, T, 32>(a, X, s);
        case 64: return launch_layer_t<AGG, T, 64>(a, X, s);
        case 128: return launch_layer_t<AGG, T, 128>(a, X, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t launch_layer_a(int agg, const LayerArgs& a, int lin, const void* X, cudaStream_t s) {
    switch (agg) {
        case AGG_NCUT: return launch_layer_w<AGG_NCUT, T>(a, lin, X, s);
        case AGG_MOD_FULL: return launch_layer_w<AGG_MOD_FULL, T>(a, lin, X, s);
        case AGG_MOD_REDUCED: return launch_layer_w<AGG_MOD_REDUCED, T>(a, lin, X, s);
        case AGG_GCN: return launch_layer_w<AGG_GCN, T>(a, lin, X, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_layer(int agg, int dtype, const raftgp_csr* g, const int32_t* deg, const float* rowscale,
                         const float* gvec, int act, const float* W, int lin, int lout, const float* postscale,
                         const void* X, void* out, void* stage, const int32_t* heavy, const int* heavy_count,
                         cudaStream_t s, const int32_t* rows, int64_t nrows) {
    LayerArgs a;
    a.heavy = heavy;
    a.heavy_count = heavy_count;
    a.rows = rows;
    a.nrows = nrows;
    a.n = g->n;
    a.rp32 = g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr;
    a.rp64 = g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr;
    a.col = g->col;
    a.deg = deg;
    a.rowscale = rowscale;
    a.g = gvec;
    a.inv_two_e = g->nnz > 0 ? 1.0 / (double)g->nnz : 0.0;
    a.act = act;
    a.W = W;
    a.lout = lout;
    a.postscale = postscale;
    a.out = out;
    a.stage = stage;
    if (dtype == RAFTGP_BF16) return launch_layer_a<__nv_bfloat16>(agg, a, lin, X, s);
    return launch_layer_a<float>(agg, a, lin, X, s);
}

}  // namespace raftgp
