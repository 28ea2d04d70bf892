// batched.cu -- many graphs of uneven size partitioned together.
//
// The graphs arrive as one block-diagonal CSR (global node ids, graph g owning the rows
// node_off[g] .. node_off[g+1]).  The embedding (Eq. 5 with the NCut operator, Eq. 6) is one
// pass over the concatenation: every step of it is per node, and the projection draws its
// Philox rows by the node's index inside its own graph, so each graph gets the embedding it
// would get alone.  Model selection then runs per graph, in persistent kernels that take
// work from queues (heaviest first):
//   seeding  one CTA per graph: k-means++ for the graph's K_max (D^2 in FP32 direct form,
//            quantised floor(D^2 2^40), the same Philox draws as a single graph)
//   lloyd    one CTA per (graph, candidate K): Lloyd passes with the centroids, their norms,
//            the 2^-40 fixed-point sums and the counts in shared memory, then the partition's
//            intra-block edges and volumes (exact integers) and its modularity / NCut
//   grids    the coarse grid per graph before, the refined grid from the coarse scores between
//            the two Lloyd phases, the best candidate per graph at the end -- all on the device
// The arithmetic of every decision (distances, ties to the lowest index, the fixed-point sums,
// the FP64 means and the order of the norm sums, the integer scores, the grid rules) is the
// same as the single-graph FP32 engine's, so each graph's labels equal the ones a single-graph
// partition with the same embedding and options returns.
#include <cuda_runtime.h>

#include "batch_score.cuh"
#include "common.cuh"
#include "internal.h"

namespace raftgp {

// ------------------------------------------------------------------------------------
// Block-wide exclusive scan of one unsigned 64-bit value per thread (any block size that is a
// multiple of 32, at most 1024); returns the thread's exclusive prefix and the total.
// ------------------------------------------------------------------------------------
__device__ unsigned long long bscan(unsigned long long v, unsigned long long* total, unsigned long long* ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < nw ? ws[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) ws[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = (w > 0 ? ws[w - 1] : 0ull) + x - v;
    *total = ws[nw - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ uint64_t bk_draw(uint64_t seed, int t) {
    const U32x4 x = philox4x32_10((uint32_t)t, 0u, 0u, STREAM_KMPP, seed);
    return (uint64_t)x.x | ((uint64_t)x.y << 32);
}
__device__ __forceinline__ unsigned long long bk_quant(float d2) { return __float2ull_rz(d2 * FIXED_SCALE_F); }

// ------------------------------------------------------------------------------------
// Per-node index inside its graph (Philox row counters) and per-node graph ids.
// ------------------------------------------------------------------------------------
__global__ void k_batch_local_rows(int ng, const int64_t* __restrict__ node_off, int32_t* __restrict__ local_row,
                                   int32_t* __restrict__ graph_of) {
    for (int g = blockIdx.x; g < ng; g += gridDim.x) {
        const int64_t a = node_off[g], b = node_off[g + 1];
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            local_row[i] = (int32_t)(i - a);
            graph_of[i] = g;
        }
    }
}

// Every column of a graph's rows must lie inside the graph (block-diagonal batch).
__global__ void k_batch_check(int ng, const int64_t* __restrict__ node_off, const int64_t* __restrict__ rp64,
                              const int32_t* __restrict__ rp32, const int32_t* __restrict__ col, uint32_t* err) {
    for (int g = blockIdx.x; g < ng; g += gridDim.x) {
        const int64_t a = node_off[g], b = node_off[g + 1];
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            const int64_t e0 = rp64 ? rp64[i] : (int64_t)rp32[i], e1 = rp64 ? rp64[i + 1] : (int64_t)rp32[i + 1];
            for (int64_t q = e0; q < e1; ++q)
                if (col[q] < a || col[q] >= b) {
                    flag_error(err, DERR_COL_RANGE);
                    break;
                }
        }
    }
}

// Coarse grid per graph: kmin + round((kmax - kmin) t / (G - 1)), t = 0..G-1, round half up,
// duplicates dropped (slots 0..9, ascending).
__global__ void k_batch_coarse(BatchDev b, int kmin, int G) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < b.ng; g += gridDim.x * blockDim.x) {
        const int kmax = b.kmax[g];
        int nc = 0, last = -1;
        if (G == 1) {
            b.cand_k[g * BATCH_SLOTS] = kmin;
            nc = 1;
        } else {
            for (int t = 0; t < G; ++t) {
                const int64_t num = 2 * (int64_t)(kmax - kmin) * t + (G - 1);
                const int k = kmin + (int)(num / (2 * (int64_t)(G - 1)));
                if (k != last) b.cand_k[g * BATCH_SLOTS + nc++] = k;
                last = k;
            }
        }
        b.n_coarse[g] = nc;
        b.n_refine[g] = 0;
    }
}

__device__ __forceinline__ bool bk_better(int criterion, double ma, double na, int ka, double mb, double nb, int kb) {
    if (criterion == RAFTGP_CRIT_NCUT) {
        if (na != nb) return na < nb;
    } else {
        if (ma != mb) return ma > mb;
    }
    return ka < kb;
}

// Refined grid between the coarse neighbours of the best coarse candidate:
// lo + round((hi - lo) t / (G + 1)), t = 1..G, minus the values already evaluated (slots 10..).
__global__ void k_batch_refine(BatchDev b, int G, int criterion) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < b.ng; g += gridDim.x * blockDim.x) {
        const int nc = b.n_coarse[g];
        const int* ks = b.cand_k + g * BATCH_SLOTS;
        const double* md = b.cand_mod + g * BATCH_SLOTS;
        const double* nd = b.cand_ncut + g * BATCH_SLOTS;
        int jb = 0;
        for (int j = 1; j < nc; ++j)
            if (bk_better(criterion, md[j], nd[j], ks[j], md[jb], nd[jb], ks[jb])) jb = j;
        const int lo = ks[jb > 0 ? jb - 1 : 0], hi = ks[jb < nc - 1 ? jb + 1 : nc - 1];
        int nr = 0;
        for (int t = 1; t <= G && nr < BATCH_SLOTS - BATCH_COARSE; ++t) {
            const int64_t num = 2 * (int64_t)(hi - lo) * t + (G + 1);
            const int k = lo + (int)(num / (2 * (int64_t)(G + 1)));
            bool seen = false;
            for (int j = 0; j < nc; ++j) seen |= ks[j] == k;
            for (int j = 0; j < nr; ++j) seen |= ks[BATCH_COARSE + j] == k;
            if (!seen) b.cand_k[g * BATCH_SLOTS + BATCH_COARSE + nr++] = k;
        }
        b.n_refine[g] = nr;
    }
}

// ------------------------------------------------------------------------------------
// Seeding: persistent, one CTA of 1024 threads per graph (heaviest first).
// ------------------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(1024) k_batch_seed(BatchDev b, const T* __restrict__ Z, uint64_t seed) {
    __shared__ float c[D];
    __shared__ unsigned long long ws[32];
    __shared__ int s_g;
    __shared__ long long s_pick;
    for (;;) {
        if (threadIdx.x == 0) {
            const int u = atomicAdd(b.queue + 0, 1);
            s_g = u < b.ng ? b.order[u] : -1;
        }
        __syncthreads();
        const int g = s_g;
        if (g < 0) return;
        const int64_t o = b.node_off[g];
        const int64_t n = b.node_off[g + 1] - o;
        const int K = b.kmax[g];
        int32_t* seeds = b.seeds + b.seed_off[g];
        float* D2 = b.D2 + o;
        uint8_t* chosen = b.chosen + o;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) chosen[i] = 0;
        long long p = (long long)mulhi64(bk_draw(seed, 0), (uint64_t)n);
        __syncthreads();
        if (threadIdx.x == 0) {
            seeds[0] = (int32_t)p;
            chosen[p] = 1;
        }
        for (int t = 1; t < K; ++t) {
            for (int k = threadIdx.x; k < D; k += blockDim.x) c[k] = load_elem(Z, (o + p) * D + k);
            __syncthreads();
            // D^2 update (FP32 direct form, ascending coordinates)
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                float s = 0.0f;
                const T* zi = Z + (o + i) * D;
#pragma unroll
                for (int v = 0; v < D / Vec<T>::E; ++v) {
                    float x[Vec<T>::E];
                    Vec<T>::load(zi + v * Vec<T>::E, x);
#pragma unroll
                    for (int e = 0; e < Vec<T>::E; ++e) {
                        const float dl = __fsub_rn(x[e], c[v * Vec<T>::E + e]);
                        s = __fadd_rn(s, __fmul_rn(dl, dl));
                    }
                }
                if (t == 1 || s < D2[i]) D2[i] = s;
            }
            __syncthreads();
            // contiguous segments in index order, one per thread
            const int64_t L = (n + blockDim.x - 1) / blockDim.x;
            const int64_t r0 = (int64_t)threadIdx.x * L;
            const int64_t r1 = r0 + L < n ? r0 + L : n;
            unsigned long long v = 0;
            for (int64_t i = r0; i < r1; ++i) v += bk_quant(D2[i]);
            unsigned long long tot;
            const unsigned long long ex = bscan(v, &tot, ws);
            if (threadIdx.x == 0) s_pick = -1;
            __syncthreads();
            if (tot > 0) {
                const unsigned long long thr = mulhi64(bk_draw(seed, t), tot);
                if (r0 < r1 && ex + v > thr && ex <= thr) {
                    unsigned long long run = ex;
                    for (int64_t i = r0; i < r1; ++i) {
                        run += bk_quant(D2[i]);
                        if (run > thr) {
                            s_pick = i;
                            break;
                        }
                    }
                }
            } else if (threadIdx.x == 0) {
                // every remaining point coincides with a seed: the lowest-index unchosen one
                for (int64_t i = 0; i < n; ++i)
                    if (!chosen[i]) {
                        s_pick = i;
                        break;
                    }
            }
            __syncthreads();
            p = s_pick < 0 ? 0 : s_pick;   // unreachable fallback keeps indices in range
            if (threadIdx.x == 0) {
                seeds[t] = (int32_t)p;
                chosen[p] = 1;
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Lloyd + score: persistent, one CTA per (graph, candidate).  PHASE 0: coarse slots, 1: refined.
// PPT points per thread share each centroid load.
// ------------------------------------------------------------------------------------
template <typename T, int D, int PPT>
__global__ void k_batch_lloyd(BatchDev b, const T* __restrict__ Z, int phase, int iters, const int64_t* __restrict__ rp64,
                              const int32_t* __restrict__ rp32, const int32_t* __restrict__ col) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long* sums = reinterpret_cast<long long*>(smraw);              // BATCH_KMAX x D
    float* mu = reinterpret_cast<float*>(sums + BATCH_KMAX * D);        // BATCH_KMAX x D
    float* nrm = mu + BATCH_KMAX * D;                                    // BATCH_KMAX
    int* cnt = reinterpret_cast<int*>(nrm + BATCH_KMAX);                 // BATCH_KMAX
    __shared__ int s_item, s_changed;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int per_graph = phase == 0 ? BATCH_COARSE : BATCH_SLOTS - BATCH_COARSE;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.queue + 1 + phase, 1);
        __syncthreads();
        const int u = s_item;
        if (u >= b.ng * per_graph) return;
        const int g = b.order[u / per_graph];
        const int j = u % per_graph;
        const int slot = (phase == 0 ? 0 : BATCH_COARSE) + j;
        if (j >= (phase == 0 ? b.n_coarse[g] : b.n_refine[g])) {
            __syncthreads();
            continue;
        }
        const int K = b.cand_k[g * BATCH_SLOTS + slot];
        const int64_t o = b.node_off[g];
        const int64_t n = b.node_off[g + 1] - o;
        int16_t* lab = b.labels + (int64_t)slot * b.total_n + o;
        const int32_t* seeds = b.seeds + b.seed_off[g];
        // centroids from the first K seeds; norms in ascending coordinates
        for (int t = threadIdx.x; t < K * D; t += blockDim.x) {
            mu[t] = load_elem(Z, (o + seeds[t / D]) * D + (t % D));
            sums[t] = 0;
        }
        for (int t = threadIdx.x; t < K; t += blockDim.x) cnt[t] = 0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) lab[i] = -1;
        __syncthreads();
        for (int c = threadIdx.x; c < K; c += blockDim.x) {
            float s = 0.f;
            for (int k = 0; k < D; ++k) s = fmaf(mu[c * D + k], mu[c * D + k], s);
            nrm[c] = s;
        }
        __syncthreads();
        int passes = iters;
        for (int pass = 1; pass <= iters; ++pass) {
            if (threadIdx.x == 0) s_changed = 0;
            __syncthreads();
            int nch = 0;
            for (int64_t i0 = (int64_t)threadIdx.x * PPT; i0 < n; i0 += (int64_t)blockDim.x * PPT) {
                float z[PPT][D];
#pragma unroll
                for (int r = 0; r < PPT; ++r)
#pragma unroll
                    for (int k = 0; k < D; ++k) z[r][k] = i0 + r < n ? load_elem(Z, (o + i0 + r) * D + k) : 0.f;
                float bv[PPT];
                int bi[PPT];
#pragma unroll
                for (int r = 0; r < PPT; ++r) { bv[r] = INFINITY; bi[r] = 0x7fffffff; }
                for (int c = 0; c < K; ++c) {
                    float acc[PPT];
#pragma unroll
                    for (int r = 0; r < PPT; ++r) acc[r] = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float m = mu[c * D + k];
#pragma unroll
                        for (int r = 0; r < PPT; ++r) acc[r] = fmaf(z[r][k], m, acc[r]);
                    }
                    const float nc = nrm[c];
#pragma unroll
                    for (int r = 0; r < PPT; ++r) {
                        const float s = fmaf(-2.0f, acc[r], nc);
                        if (s < bv[r]) { bv[r] = s; bi[r] = c; }
                    }
                }
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    const int64_t i = i0 + r;
                    if (i >= n) continue;
                    int nl = bi[r];
                    if (nl < 0 || nl >= K) nl = 0;   // every score NaN (non-finite input): keep indices in range
                    const int ol = lab[i];
                    if (nl == ol) continue;
                    lab[i] = (int16_t)nl;
                    ++nch;
                    atomicAdd(cnt + nl, 1);
                    if (ol >= 0) atomicSub(cnt + ol, 1);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const long long v = __float2ll_rn(z[r][k] * FIXED_SCALE_F);
                        atomicAdd(reinterpret_cast<unsigned long long*>(sums + nl * D + k), (unsigned long long)v);
                        if (ol >= 0)
                            atomicAdd(reinterpret_cast<unsigned long long*>(sums + ol * D + k), (unsigned long long)(-v));
                    }
                }
            }
            nch = __reduce_add_sync(0xffffffffu, nch);
            if (lane == 0 && nch) atomicAdd(&s_changed, nch);
            __syncthreads();
            if (s_changed == 0) {
                passes = pass;
                break;
            }
            if (pass == iters) break;       // no update after the last pass
            // FP64 means of the fixed-point sums, norms in lane order then a warp sum
            for (int cc = warp; cc < K; cc += nwarps) {
                const int ct = cnt[cc];
                if (ct <= 0) continue;
                const double inv = 1.0 / ((double)ct * FIXED_SCALE);
                float s = 0.f;
                for (int k = lane; k < D; k += 32) {
                    const float v = (float)((double)sums[cc * D + k] * inv);
                    mu[cc * D + k] = v;
                    s = fmaf(v, v, s);
                }
                s = warp_sum(s);
                if (lane == 0) nrm[cc] = s;
            }
            __syncthreads();
        }
        batch_score_item(b, g, slot, K, o, n, lab, passes, reinterpret_cast<unsigned long long*>(sums), rp64, rp32, col);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Lloyd + score, register-tiled: persistent, one CTA of 256 threads per (graph, candidate).
// The centroids live in shared memory k-major (muT[k][c], BATCH_KMAX columns, unused columns
// zero with an infinite norm).  Each pass walks the graph's points in tiles of 256, staged
// transposed (zT[k][p]); warp w scores points 32w..32w+31 against the centroids in column
// groups: lane (pr, cr) = (lane / 8, lane % 8) holds 8 points {4pr..4pr+3, 16+4pr..16+4pr+3}
// and NC centroids of a group of 8 NC columns (NC = 8: {4cr..4cr+3, 32+4cr..32+4cr+3};
// NC = 4: {4cr..4cr+3}; NC = 2: {2cr, 2cr+1}), the group width chosen by how many real
// centroids remain.  Scores, tie rule, fixed-point sums, FP64 means and norm order are the
// scalar kernel's (and the single-graph engine's), so the labels are the same.
// ------------------------------------------------------------------------------------
constexpr int BT_THREADS = 256;
constexpr int BT_PTS = 256;

size_t batch_lloyd_tiled_smem(int d) {
    return (size_t)BATCH_KMAX * d * sizeof(long long) + (size_t)d * BATCH_KMAX * sizeof(float) +
           BATCH_KMAX * (sizeof(float) + sizeof(int)) + (size_t)d * BT_PTS * sizeof(float);
}

template <int D, int NC>
__device__ __forceinline__ void bt_group(const float* __restrict__ zw, const float* __restrict__ muT,
                                         const float* __restrict__ nrm, int c0, int pr, int cr, float* bv, int* bi) {
    float acc[8][NC];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[r][j] = 0.f;
#pragma unroll 4
    for (int k = 0; k < D; ++k) {
        const float4 za = *reinterpret_cast<const float4*>(zw + k * BT_PTS + 4 * pr);
        const float4 zb = *reinterpret_cast<const float4*>(zw + k * BT_PTS + 16 + 4 * pr);
        const float z[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
        float m[NC];
        const float* mk = muT + k * BATCH_KMAX + c0;
        if constexpr (NC == 8) {
            const float4 ma = *reinterpret_cast<const float4*>(mk + 4 * cr);
            const float4 mb = *reinterpret_cast<const float4*>(mk + 32 + 4 * cr);
            m[0] = ma.x; m[1] = ma.y; m[2] = ma.z; m[3] = ma.w;
            m[4] = mb.x; m[5] = mb.y; m[6] = mb.z; m[7] = mb.w;
        } else if constexpr (NC == 4) {
            const float4 ma = *reinterpret_cast<const float4*>(mk + 4 * cr);
            m[0] = ma.x; m[1] = ma.y; m[2] = ma.z; m[3] = ma.w;
        } else {
            const float2 ma = *reinterpret_cast<const float2*>(mk + 2 * cr);
            m[0] = ma.x; m[1] = ma.y;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int j = 0; j < NC; ++j) acc[r][j] = fmaf(z[r], m[j], acc[r][j]);
    }
    // this lane's columns in ascending order
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int col = c0 + (NC == 8 ? (j < 4 ? 4 * cr + j : 32 + 4 * cr + (j - 4)) : NC == 4 ? 4 * cr + j : 2 * cr + j);
        const float nq = nrm[col];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float s = fmaf(-2.0f, acc[r][j], nq);
            if (s < bv[r]) { bv[r] = s; bi[r] = col; }
        }
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(BT_THREADS, 1)
    k_batch_lloyd_tiled(BatchDev b, const T* __restrict__ Z, int phase, int iters, const int64_t* __restrict__ rp64,
                        const int32_t* __restrict__ rp32, const int32_t* __restrict__ col) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long* sums = reinterpret_cast<long long*>(smraw);              // BATCH_KMAX x D
    float* muT = reinterpret_cast<float*>(sums + BATCH_KMAX * D);       // D x BATCH_KMAX
    float* nrm = muT + D * BATCH_KMAX;                                   // BATCH_KMAX
    int* cnt = reinterpret_cast<int*>(nrm + BATCH_KMAX);                 // BATCH_KMAX
    float* zT = reinterpret_cast<float*>(cnt + BATCH_KMAX);              // D x BT_PTS
    __shared__ int s_item, s_changed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = BT_THREADS >> 5;
    const int pr = lane >> 3, cr = lane & 7;
    const int per_graph = phase == 0 ? BATCH_COARSE : BATCH_SLOTS - BATCH_COARSE;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(b.queue + 1 + phase, 1);
        __syncthreads();
        const int u = s_item;
        if (u >= b.ng * per_graph) return;
        const int g = b.order[u / per_graph];
        const int j = u % per_graph;
        const int slot = (phase == 0 ? 0 : BATCH_COARSE) + j;
        if (j >= (phase == 0 ? b.n_coarse[g] : b.n_refine[g])) {
            __syncthreads();
            continue;
        }
        const int K = b.cand_k[g * BATCH_SLOTS + slot];
        const int64_t o = b.node_off[g];
        const int64_t n = b.node_off[g + 1] - o;
        int16_t* lab = b.labels + (int64_t)slot * b.total_n + o;
        const int32_t* seeds = b.seeds + b.seed_off[g];
        // centroids from the first K seeds (unused columns zero); norms in ascending coordinates
        for (int t = tid; t < BATCH_KMAX * D; t += BT_THREADS) {
            const int c = t / D, k = t % D;
            muT[k * BATCH_KMAX + c] = c < K ? load_elem(Z, (o + seeds[c]) * D + k) : 0.f;
            sums[t] = 0;
        }
        for (int t = tid; t < BATCH_KMAX; t += BT_THREADS) cnt[t] = 0;
        for (int64_t i = tid; i < n; i += BT_THREADS) lab[i] = -1;
        __syncthreads();
        for (int c = tid; c < BATCH_KMAX; c += BT_THREADS) {
            float s = 0.f;
            for (int k = 0; k < D; ++k) s = fmaf(muT[k * BATCH_KMAX + c], muT[k * BATCH_KMAX + c], s);
            nrm[c] = c < K ? s : INFINITY;
        }
        __syncthreads();
        int passes = iters;
        for (int pass = 1; pass <= iters; ++pass) {
            if (tid == 0) s_changed = 0;
            int nch = 0;
            for (int64_t p0 = 0; p0 < n; p0 += BT_PTS) {
                __syncthreads();   // the previous tile's reads (and s_changed's reset) are done
                {
                    constexpr int E = Vec<T>::E;
                    for (int t = tid; t < BT_PTS * (D / E); t += BT_THREADS) {
                        const int p = t % BT_PTS, k0 = (t / BT_PTS) * E;
                        float v[E];
                        if (p0 + p < n) {
                            Vec<T>::load(Z + (o + p0 + p) * D + k0, v);
                        } else {
#pragma unroll
                            for (int e = 0; e < E; ++e) v[e] = 0.f;
                        }
#pragma unroll
                        for (int e = 0; e < E; ++e) zT[(k0 + e) * BT_PTS + p] = v[e];
                    }
                }
                __syncthreads();
                float bv[8];
                int bi[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) { bv[r] = INFINITY; bi[r] = 0x7fffffff; }
                const float* zw = zT + 32 * warp;
                for (int c0 = 0; c0 < K; c0 += 64) {
                    const int left = K - c0;
                    if (left > 32) bt_group<D, 8>(zw, muT, nrm, c0, pr, cr, bv, bi);
                    else if (left > 16) bt_group<D, 4>(zw, muT, nrm, c0, pr, cr, bv, bi);
                    else bt_group<D, 2>(zw, muT, nrm, c0, pr, cr, bv, bi);
                }
                // combine the 8 lanes of a point group (ties to the lowest column); lane cr
                // reports point cr of its group
#pragma unroll
                for (int ofs = 1; ofs < 8; ofs <<= 1) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const float ov = __shfl_xor_sync(0xffffffffu, bv[r], ofs);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi[r], ofs);
                        if (ov < bv[r] || (ov == bv[r] && oi < bi[r])) { bv[r] = ov; bi[r] = oi; }
                    }
                }
                int mi = 0x7fffffff;
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    if (r == cr) mi = bi[r];
                const int p = 32 * warp + (cr < 4 ? 4 * pr + cr : 16 + 4 * pr + (cr - 4));
                const int64_t i = p0 + p;
                if (i < n) {
                    int nl = mi;
                    if (nl < 0 || nl >= K) nl = 0;   // every score NaN (non-finite input): keep indices in range
                    const int ol = lab[i];
                    if (nl != ol) {
                        lab[i] = (int16_t)nl;
                        ++nch;
                        atomicAdd(cnt + nl, 1);
                        if (ol >= 0) atomicSub(cnt + ol, 1);
#pragma unroll 4
                        for (int k = 0; k < D; ++k) {
                            const long long v = __float2ll_rn(zT[k * BT_PTS + p] * FIXED_SCALE_F);
                            atomicAdd(reinterpret_cast<unsigned long long*>(sums + nl * D + k), (unsigned long long)v);
                            if (ol >= 0)
                                atomicAdd(reinterpret_cast<unsigned long long*>(sums + ol * D + k),
                                          (unsigned long long)(-v));
                        }
                    }
                }
            }
            nch = __reduce_add_sync(0xffffffffu, nch);
            if (lane == 0 && nch) atomicAdd(&s_changed, nch);
            __syncthreads();
            if (s_changed == 0) {
                passes = pass;
                break;
            }
            if (pass == iters) break;       // no update after the last pass
            // FP64 means of the fixed-point sums, norms in lane order then a warp sum
            for (int cc = warp; cc < K; cc += nwarps) {
                const int ct = cnt[cc];
                if (ct <= 0) continue;
                const double inv = 1.0 / ((double)ct * FIXED_SCALE);
                float s = 0.f;
                for (int k = lane; k < D; k += 32) {
                    const float v = (float)((double)sums[cc * D + k] * inv);
                    muT[k * BATCH_KMAX + cc] = v;
                    s = fmaf(v, v, s);
                }
                s = warp_sum(s);
                if (lane == 0) nrm[cc] = s;
            }
            __syncthreads();
        }
        batch_score_item(b, g, slot, K, o, n, lab, passes, reinterpret_cast<unsigned long long*>(sums), rp64, rp32, col);
        __syncthreads();
    }
}

// Best candidate per graph (criterion; exact ties to the smaller K): its labels (int32, as the
// index inside the graph's partition) and K.
__global__ void k_batch_select(BatchDev b, int criterion, int32_t* __restrict__ labels_out, int32_t* __restrict__ k_out) {
    __shared__ int s_slot;
    for (int g = blockIdx.x; g < b.ng; g += gridDim.x) {
        if (threadIdx.x == 0) {
            const int nc = b.n_coarse[g], nr = b.n_refine[g];
            int best = 0;
            for (int jj = 1; jj < nc + nr; ++jj) {
                const int j = jj < nc ? jj : BATCH_COARSE + jj - nc;
                const int bs = best;
                if (bk_better(criterion, b.cand_mod[g * BATCH_SLOTS + j], b.cand_ncut[g * BATCH_SLOTS + j],
                              b.cand_k[g * BATCH_SLOTS + j], b.cand_mod[g * BATCH_SLOTS + bs],
                              b.cand_ncut[g * BATCH_SLOTS + bs], b.cand_k[g * BATCH_SLOTS + bs]))
                    best = j;
            }
            s_slot = best;
            k_out[g] = b.cand_k[g * BATCH_SLOTS + best];
        }
        __syncthreads();
        const int64_t o = b.node_off[g], e = b.node_off[g + 1];
        const int16_t* lab = b.labels + (int64_t)s_slot * b.total_n;
        for (int64_t i = o + threadIdx.x; i < e; i += blockDim.x) labels_out[i] = lab[i];
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
void launch_batch_check(const raftgp_csr* g, int ng, const int64_t* node_off, uint32_t* err, cudaStream_t s) {
    k_batch_check<<<ng < 4096 ? ng : 4096, 256, 0, s>>>(ng, node_off,
                                                        g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr,
                                                        g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr,
                                                        g->col, err);
}

size_t batch_lloyd_smem(int d) {
    return (size_t)BATCH_KMAX * d * (sizeof(long long) + sizeof(float)) + BATCH_KMAX * (sizeof(float) + sizeof(int));
}

void launch_batch_prologue(BatchDev b, int kmin, int G, cudaStream_t s) {
    ProfScope ps(s, PF_BATCH_INIT, 2);
    cudaMemsetAsync(b.queue, 0, 4 * sizeof(int), s);
    k_batch_local_rows<<<b.ng < 4096 ? b.ng : 4096, 256, 0, s>>>(b.ng, b.node_off, b.local_row, b.graph_of);
    k_batch_coarse<<<(b.ng + 127) / 128, 128, 0, s>>>(b, kmin, G);
}

cudaError_t launch_batch_seed(BatchDev b, const void* Z, int zdtype, int d, uint64_t seed, cudaStream_t s) {
    ProfScope ps(s, PF_SEED_UPDATE, 1);
    const int blocks = b.ng < num_sms() ? b.ng : num_sms();
#define RAFTGP_BS(T, DD) k_batch_seed<T, DD><<<blocks, 1024, 0, s>>>(b, (const T*)Z, seed)
    if (zdtype == RAFTGP_BF16) {
        if (d == 32) RAFTGP_BS(__nv_bfloat16, 32); else if (d == 64) RAFTGP_BS(__nv_bfloat16, 64); else return cudaErrorInvalidValue;
    } else {
        if (d == 32) RAFTGP_BS(float, 32); else if (d == 64) RAFTGP_BS(float, 64); else return cudaErrorInvalidValue;
    }
#undef RAFTGP_BS
    return cudaGetLastError();
}

template <typename T, int D, int PPT>
static cudaError_t batch_lloyd_t(BatchDev b, const T* Z, int phase, int iters, const raftgp_csr* g, int threads,
                                 cudaStream_t s) {
    const size_t smem = batch_lloyd_smem(D);
    auto kern = k_batch_lloyd<T, D, PPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = num_sms() * per_sm;
    kern<<<blocks, threads, smem, s>>>(b, Z, phase, iters, g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr,
                                       g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr, g->col);
    return cudaGetLastError();
}

template <typename T, int D>
static cudaError_t batch_lloyd_tiled_t(BatchDev b, const T* Z, int phase, int iters, const raftgp_csr* g,
                                       cudaStream_t s) {
    const size_t smem = batch_lloyd_tiled_smem(D);
    auto kern = k_batch_lloyd_tiled<T, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<num_sms() * per_sm, BT_THREADS, smem, s>>>(b, Z, phase, iters,
                                                      g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr,
                                                      g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr,
                                                      g->col);
    return cudaGetLastError();
}

// threads / ppt pick the scalar kernel's shape; ppt == 0 picks the register-tiled kernel
cudaError_t launch_batch_lloyd(BatchDev b, const void* Z, int zdtype, int d, int phase, int iters, const raftgp_csr* g,
                               int threads, int ppt, cudaStream_t s) {
    ProfScope ps(s, PF_ASSIGN_FFMA, 1);
    if (ppt == 0) {
        if (zdtype == RAFTGP_BF16) {
            if (d == 32) return batch_lloyd_tiled_t<__nv_bfloat16, 32>(b, (const __nv_bfloat16*)Z, phase, iters, g, s);
            if (d == 64) return batch_lloyd_tiled_t<__nv_bfloat16, 64>(b, (const __nv_bfloat16*)Z, phase, iters, g, s);
        } else {
            if (d == 32) return batch_lloyd_tiled_t<float, 32>(b, (const float*)Z, phase, iters, g, s);
            if (d == 64) return batch_lloyd_tiled_t<float, 64>(b, (const float*)Z, phase, iters, g, s);
        }
        return cudaErrorInvalidValue;
    }
#define RAFTGP_BL(T, DD, P) return batch_lloyd_t<T, DD, P>(b, (const T*)Z, phase, iters, g, threads, s)
    if (zdtype == RAFTGP_BF16) {
        if (d == 32) { if (ppt == 2) RAFTGP_BL(__nv_bfloat16, 32, 2); RAFTGP_BL(__nv_bfloat16, 32, 1); }
        if (d == 64) { if (ppt == 2) RAFTGP_BL(__nv_bfloat16, 64, 2); RAFTGP_BL(__nv_bfloat16, 64, 1); }
    } else {
        if (d == 32) { if (ppt == 2) RAFTGP_BL(float, 32, 2); RAFTGP_BL(float, 32, 1); }
        if (d == 64) { if (ppt == 2) RAFTGP_BL(float, 64, 2); RAFTGP_BL(float, 64, 1); }
    }
#undef RAFTGP_BL
    return cudaErrorInvalidValue;
}

void launch_batch_refine(BatchDev b, int G, int criterion, cudaStream_t s) {
    ProfScope ps(s, PF_SELECT_BEST, 1);
    k_batch_refine<<<(b.ng + 127) / 128, 128, 0, s>>>(b, G, criterion);
}

void launch_batch_select(BatchDev b, int criterion, int32_t* labels_out, int32_t* k_out, cudaStream_t s) {
    ProfScope ps(s, PF_SELECT_BEST, 1);
    k_batch_select<<<b.ng < 4096 ? b.ng : 4096, 256, 0, s>>>(b, criterion, labels_out, k_out);
}

}  // namespace raftgp
