// bisect.cu -- Algorithm 1 (hierarchical model selection): recursive 2-way splits accepted by
// local modularity (Definition 5 / Eq. 7), level-synchronous on the device.
//
// Every set of one depth is a contiguous range of a node permutation (ascending node order
// inside a set).  One level:
//   1. k-means++ for K=2 per set: the first seed at floor(r_0 n / 2^64), the FP32 direct-form
//      D^2 to it quantised to floor(D^2 2^40), a device-wide scan, the second seed where the
//      set's prefix first exceeds floor(r_1 sum / 2^64) (r_t = Philox(seed; t, id_lo, id_hi,
//      "Kmpp"), id = the set's node in the recursion tree, root 1);
//   2. Lloyd passes for all sets at once (the FP32 engine's arithmetic: ascending FMA dot
//      products, score fma(-2, dot, ||mu||^2), ties to cluster 0), the changes applied to
//      2^-40 fixed-point sums, aggregated per CTA for the sets its positions cover;
//   3. per set the intra-set and intra-half edges and the G-degree sums of the halves (exact
//      integers), the stopping rule (|U1| or |U2| <= eps, or LMod(U) > LMod(U1, U2) compared
//      as 128-bit integers, with 2e the G-degree sum of U or of all of V);
//   4. scans number the children and the finished blocks deterministically; a stable scatter
//      builds the next level's permutation.
// Sets of at most 2 eps + 1 nodes are blocks without k-means (one half would have at most eps
// nodes), and so is a set at depth 62.  At the end the blocks are numbered by their smallest
// node index.
//
// Streaming update (Section III-D: "update only a tree path" once embeddings change).  Given
// the previous run's labels and per-node leaf ids (the tree id of each node's block) and the
// nodes whose embedding or degree changed, a set is kept as the previous tree node when it is
// that node (every ancestor split exactly as before) and holds no changed node: its old
// subtree's blocks are reused without any k-means.  A set holding a changed node is
// partitioned again; if its new decision and every node's side equal the old ones, its
// children may be kept in turn, otherwise its subtree is rebuilt.  With 2e the G-degree sum of
// U (the literal reading) a kept subtree's inputs (its nodes' embeddings, degrees and inner
// edges, and its tree ids) are those of the previous run, so the result equals a full run on
// the new graph; with the global reading every decision also depends on |E|, which a new edge
// changes, and the kept subtrees are the paper's path-update approximation.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

constexpr int BS_WIN = 8;   // sets a CTA aggregates in shared memory

__device__ __forceinline__ uint64_t bs_draw(uint64_t seed, int t, uint64_t id) {
    const U32x4 x = philox4x32_10((uint32_t)t, (uint32_t)id, (uint32_t)(id >> 32), STREAM_KMPP, seed);
    return (uint64_t)x.x | ((uint64_t)x.y << 32);
}

// ------------------------------------------------------------------------------------
// Device-wide inclusive scan of unsigned 64-bit values (three launches).
// ------------------------------------------------------------------------------------
constexpr int SC_T = 1024, SC_ITEMS = 4, SC_TILE = SC_T * SC_ITEMS;
static_assert(SC_TILE == SCAN_TILE, "the tile count callers reserve");

__device__ unsigned long long sc_block_incl(unsigned long long v, unsigned long long* ws, unsigned long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const unsigned long long r = x + (w > 0 ? ws[w - 1] : 0ull);
    *total = ws[31];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_T) k_scan_tiles(const unsigned long long* in, int64_t n, unsigned long long* out,
                                                     unsigned long long* tile_tot) {
    __shared__ unsigned long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    unsigned long long v[SC_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0ull;
        s += v[k];
    }
    unsigned long long tot;
    const unsigned long long incl = sc_block_incl(s, ws, &tot);
    unsigned long long run = incl - s;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        run += v[k];
        if (base + k < n) out[base + k] = run;
    }
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

// exclusive prefix of the tile totals, in place (one block, any count)
__global__ void __launch_bounds__(SC_T) k_scan_totals(unsigned long long* tot, int64_t tiles) {
    __shared__ unsigned long long ws[32];
    const int64_t per = (tiles + SC_T - 1) / SC_T;
    const int64_t a = (int64_t)threadIdx.x * per, b = a + per < tiles ? a + per : tiles;
    unsigned long long s = 0;
    for (int64_t i = a; i < b; ++i) s += tot[i];
    unsigned long long total;
    unsigned long long run = sc_block_incl(s, ws, &total) - s;
    for (int64_t i = a; i < b; ++i) {
        const unsigned long long v = tot[i];
        tot[i] = run;
        run += v;
    }
}

__global__ void k_scan_add(unsigned long long* out, int64_t n, const unsigned long long* tile_off) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] += tile_off[i / SC_TILE];
}

void scan_incl(const unsigned long long* in, int64_t n, unsigned long long* out, unsigned long long* tiles,
               cudaStream_t s) {
    if (n <= 0) return;
    const int64_t nt = (n + SC_TILE - 1) / SC_TILE;
    k_scan_tiles<<<(unsigned)nt, SC_T, 0, s>>>(in, n, out, tiles);
    k_scan_totals<<<1, SC_T, 0, s>>>(tiles, nt);
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    k_scan_add<<<(unsigned)blocks, 256, 0, s>>>(out, n, tiles);
}

// ------------------------------------------------------------------------------------
// Level kernels
// ------------------------------------------------------------------------------------
__device__ __forceinline__ bool bs_small(const BisectDev& b, int s) { return b.set_n[s] <= 2 * b.eps + 1 || b.depth >= 62; }

// positions -> set, nodes -> set, labels cleared
// Thread per position (the sets of a level are ascending ranges of positions; one set can hold
// every node, so the work is spread over positions, not sets): the position's set by binary
// search over the set offsets.
__global__ void k_bs_setup(BisectDev b, int S, int64_t M) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = S - 1;
        while (lo < hi) {   // the last set starting at or before p
            const int mid = (lo + hi + 1) >> 1;
            if (b.set_off[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        if (S < 1 || p < b.set_off[lo] || p >= b.set_off[lo] + b.set_n[lo]) continue;
        b.pos_set[p] = lo;
        b.node_set[b.perm[p]] = lo;
        b.node_lab[b.perm[p]] = -1;
        b.lab[p] = -1;
    }
}

__global__ void k_bs_seed0(BisectDev b, int S, uint64_t seed) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        b.s0[s] = b.set_off[s] + (int64_t)mulhi64(bs_draw(seed, 0, b.set_id[s]), (uint64_t)b.set_n[s]);
        b.changed[s] = 0;
        b.changed[b.cap_sets + s] = 0;
        // streaming update: the previous tree node without a changed node keeps its subtree
        const int fz = b.dirty ? (b.set_keep[s] && b.flag[s] == 0) : 0;
        b.frozen[s] = fz;
        if (b.dirty) b.flag[s] = 0;   // reused below for "the split changed"
        b.active[s] = (bs_small(b, s) || fz) ? 0 : 1;
    }
}

// Streaming update: flag the kept sets that hold a changed node.
__global__ void k_bs_dirty(BisectDev b, int64_t M) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const int s = b.pos_set[p];
        if (b.set_keep[s] && b.dirty[b.perm[p]]) b.flag[s] = 1;
    }
}

// Streaming update: does a kept, re-partitioned set split as before?  The old side of node i
// under the set's tree id u is the bit below u on the path to i's old leaf; a set that was a
// leaf before (old leaf == u) and splits now has changed too.
__device__ __forceinline__ int bs_bitlen(uint64_t x) { return 64 - __clzll((long long)x); }
__global__ void k_bs_sides(BisectDev b, int64_t M) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const int s = b.pos_set[p];
        if (!b.set_keep[s] || b.frozen[s] || !b.split[s]) continue;
        const uint64_t u = b.set_id[s], leaf = b.old_leaf[b.perm[p]];
        const int lu = bs_bitlen(u), ll = bs_bitlen(leaf);
        bool same = false;
        if (ll > lu && (leaf >> (ll - lu)) == u) same = (int)((leaf >> (ll - lu - 1)) & 1ull) == (int)b.lab[p];
        if (!same) b.flag[s] = 1;
    }
}

template <typename T, int D>
__global__ void k_bs_d2(BisectDev b, const T* __restrict__ Z, int64_t M) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const int s = b.pos_set[p];
        unsigned long long q = 0;
        if (b.active[s]) {
            const T* zi = Z + (int64_t)b.perm[p] * D;
            const T* zc = Z + (int64_t)b.perm[b.s0[s]] * D;
            float acc = 0.0f;
            for (int k = 0; k < D; ++k) {
                const float t = __fsub_rn(load_elem(zi, k), load_elem(zc, k));
                acc = __fadd_rn(acc, __fmul_rn(t, t));
            }
            q = __float2ull_rz(acc * FIXED_SCALE_F);
        }
        b.q[p] = q;
    }
}

template <typename T, int D>
__global__ void k_bs_seed1(BisectDev b, const T* __restrict__ Z, int S, uint64_t seed) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        if (!b.active[s]) continue;
        const int64_t off = b.set_off[s], n = b.set_n[s];
        const unsigned long long base = off > 0 ? b.P[off - 1] : 0ull;
        const unsigned long long tot = b.P[off + n - 1] - base;
        int64_t s1;
        if (tot == 0) {
            s1 = b.s0[s] == off ? off + 1 : off;   // the lowest-index unchosen point
        } else {
            const unsigned long long thr = mulhi64(bs_draw(seed, 1, b.set_id[s]), tot);
            int64_t lo = off, hi = off + n - 1;   // first p with P[p] - base > thr
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (b.P[mid] - base > thr) hi = mid; else lo = mid + 1;
            }
            s1 = lo;
        }
        const int64_t src[2] = {(int64_t)b.perm[b.s0[s]], (int64_t)b.perm[s1]};
        for (int c = 0; c < 2; ++c) {
            float nrm = 0.f;
            for (int k = 0; k < D; ++k) {
                const float v = load_elem(Z, src[c] * D + k);
                b.mu[((int64_t)s * 2 + c) * D + k] = v;
                b.sums[((int64_t)s * 2 + c) * D + k] = 0;
                nrm = fmaf(v, v, nrm);
            }
            b.norm2[s * 2 + c] = nrm;
            b.counts[s * 2 + c] = 0;
        }
    }
}

// One Lloyd pass over every position of the active sets.  A CTA aggregates the fixed-point
// changes of the first BS_WIN sets its positions cover in shared memory; positions of later
// sets use global atomics directly.
template <typename T, int D>
__global__ void __launch_bounds__(256, 6) k_bs_assign(BisectDev b, const T* __restrict__ Z, int64_t M, int pass) {
    __shared__ long long ssum[BS_WIN][2][D];
    __shared__ float smu[BS_WIN][2 * D];   // the window's centroids
    __shared__ int scnt[BS_WIN][2], sch[BS_WIN];
    __shared__ int s_first;
    constexpr int E = Vec<T>::E;           // elements per 16-byte load
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < M; p0 += (int64_t)gridDim.x * blockDim.x) {
        __syncthreads();
        const int sf = b.pos_set[p0];
        if (threadIdx.x == 0) s_first = sf;
        for (int t = threadIdx.x; t < BS_WIN * 2 * D; t += blockDim.x) (&ssum[0][0][0])[t] = 0;
        for (int t = threadIdx.x; t < BS_WIN * 2 * D; t += blockDim.x)
            (&smu[0][0])[t] = sf + t / (2 * D) < b.cap_sets ? b.mu[(int64_t)sf * 2 * D + t] : 0.f;
        for (int t = threadIdx.x; t < BS_WIN * 2; t += blockDim.x) (&scnt[0][0])[t] = 0;
        for (int t = threadIdx.x; t < BS_WIN; t += blockDim.x) sch[t] = 0;
        __syncthreads();
        const int64_t p = p0 + threadIdx.x;
        if (p < M) {
            const int s = b.pos_set[p];
            if (b.active[s]) {
                // the point's row in 16-byte loads, the centroids of the window's sets from
                // shared memory; products added over ascending coordinates
                const T* zi = Z + (int64_t)b.perm[p] * D;
                const int ws = s - sf;
                const float* m0 = ws >= 0 && ws < BS_WIN ? smu[ws] : b.mu + (int64_t)s * 2 * D;
                float d0 = 0.f, d1 = 0.f;
#pragma unroll 2
                for (int k0 = 0; k0 < D; k0 += E) {
                    float v[E];
                    Vec<T>::load(zi + k0, v);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        d0 = fmaf(v[e], m0[k0 + e], d0);
                        d1 = fmaf(v[e], m0[D + k0 + e], d1);
                    }
                }
                // the FP32 engine's selection: ascending centroids, strict improvement
                float bv = INFINITY;
                int bi = 0x7fffffff;
                const float sc0 = fmaf(-2.0f, d0, b.norm2[s * 2]), sc1 = fmaf(-2.0f, d1, b.norm2[s * 2 + 1]);
                if (sc0 < bv) { bv = sc0; bi = 0; }
                if (sc1 < bv) { bv = sc1; bi = 1; }
                const int nl = (bi < 0 || bi > 1) ? 0 : bi;
                const int ol = b.lab[p];
                if (nl != ol) {
                    b.lab[p] = (int8_t)nl;
                    const int w = s - s_first;
                    if (w < BS_WIN) {
                        atomicAdd(&sch[w], 1);
                        atomicAdd(&scnt[w][nl], 1);
                        if (ol >= 0) atomicSub(&scnt[w][ol], 1);
                        for (int k0 = 0; k0 < D; k0 += E) {
                            float zv[E];
                            Vec<T>::load(zi + k0, zv);
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                const int k = k0 + e;
                                const long long v = __float2ll_rn(zv[e] * FIXED_SCALE_F);
                                atomicAdd(reinterpret_cast<unsigned long long*>(&ssum[w][nl][k]), (unsigned long long)v);
                                if (ol >= 0)
                                    atomicAdd(reinterpret_cast<unsigned long long*>(&ssum[w][ol][k]), (unsigned long long)(-v));
                            }
                        }
                    } else {
                        atomicAdd(b.changed + (pass & 1) * b.cap_sets + s, 1);
                        atomicAdd(b.counts + s * 2 + nl, 1);
                        if (ol >= 0) atomicSub(b.counts + s * 2 + ol, 1);
                        for (int k = 0; k < D; ++k) {
                            const long long v = __float2ll_rn(load_elem(zi, k) * FIXED_SCALE_F);
                            atomicAdd(reinterpret_cast<unsigned long long*>(b.sums + ((int64_t)s * 2 + nl) * D + k),
                                      (unsigned long long)v);
                            if (ol >= 0)
                                atomicAdd(reinterpret_cast<unsigned long long*>(b.sums + ((int64_t)s * 2 + ol) * D + k),
                                          (unsigned long long)(-v));
                        }
                    }
                }
            }
        }
        __syncthreads();
        // flush the window
        for (int t = threadIdx.x; t < BS_WIN * 2 * D; t += blockDim.x) {
            const int w = t / (2 * D), c = (t / D) % 2, k = t % D;
            const long long v = ssum[w][c][k];
            if (v) atomicAdd(reinterpret_cast<unsigned long long*>(b.sums + ((int64_t)(s_first + w) * 2 + c) * D + k),
                             (unsigned long long)v);
        }
        for (int t = threadIdx.x; t < BS_WIN * 2; t += blockDim.x) {
            const int w = t / 2, c = t % 2;
            if (scnt[w][c]) atomicAdd(b.counts + (s_first + w) * 2 + c, scnt[w][c]);
        }
        for (int t = threadIdx.x; t < BS_WIN; t += blockDim.x)
            if (sch[t]) atomicAdd(b.changed + (pass & 1) * b.cap_sets + s_first + t, sch[t]);
    }
}

// After a pass: a set without changes has converged; otherwise the FP64 means of the sums
// (empty halves keep their centroid), the norms in lane order then a warp sum.
template <int D>
__global__ void k_bs_update(BisectDev b, int S, int pass, int last_pass) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < 2 * (int64_t)S; u += warps) {
        const int s = (int)(u >> 1), c = (int)(u & 1);
        if (!b.active[s]) continue;
        const int ch = b.changed[(pass & 1) * b.cap_sets + s];
        __syncwarp();
        if (ch == 0) {
            if (c == 0 && lane == 0) b.active[s] = 0;
            continue;
        }
        if (c == 0 && lane == 0) b.changed[((pass + 1) & 1) * b.cap_sets + s] = 0;
        if (pass >= last_pass) continue;
        const int cnt = b.counts[s * 2 + c];
        if (cnt <= 0) continue;
        const double inv = 1.0 / ((double)cnt * FIXED_SCALE);
        float nrm = 0.f;
        for (int k = lane; k < D; k += 32) {
            const float v = (float)((double)b.sums[((int64_t)s * 2 + c) * D + k] * inv);
            b.mu[((int64_t)s * 2 + c) * D + k] = v;
            nrm = fmaf(v, v, nrm);
        }
        nrm = warp_sum(nrm);
        if (lane == 0) b.norm2[s * 2 + c] = nrm;
    }
}

__global__ void k_bs_nodelab(BisectDev b, int64_t M) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x)
        b.node_lab[b.perm[p]] = b.lab[p];
}

// Intra-set and intra-half edge ends and the G-degree sums of the halves, per set (window
// aggregation as in the assignment).
template <typename OffT>
__global__ void __launch_bounds__(256) k_bs_lmod(BisectDev b, Csr<OffT> g, int64_t M) {
    __shared__ unsigned long long sv[BS_WIN][5];   // mU2, mC2[0], mC2[1], vol[0], vol[1]
    __shared__ int s_first;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < M; p0 += (int64_t)gridDim.x * blockDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) s_first = b.pos_set[p0];
        for (int t = threadIdx.x; t < BS_WIN * 5; t += blockDim.x) (&sv[0][0])[t] = 0;
        __syncthreads();
        // a warp per position of the chunk, its lanes over the node's neighbours (a power-law
        // graph's hubs have thousands)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int r = wid; r < (int)blockDim.x; r += (int)(blockDim.x >> 5)) {
            const int64_t p = p0 + r;
            if (p >= M) break;
            const int s = b.pos_set[p];
            const int c = b.lab[p];
            if (c < 0) continue;
            const int i = b.perm[p];
            const int64_t e0 = g.begin(i), e1 = g.end(i);
            unsigned long long mu2 = 0, mc2 = 0;
            for (int64_t q = e0 + lane; q < e1; q += 32) {
                const int j = g.col[q];
                if (b.node_set[j] == s) {
                    ++mu2;
                    if (b.node_lab[j] == c) ++mc2;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mu2 += __shfl_xor_sync(0xffffffffu, mu2, o);
                mc2 += __shfl_xor_sync(0xffffffffu, mc2, o);
            }
            if (lane == 0) {
                const unsigned long long deg = (unsigned long long)(e1 - e0);
                const int w = s - s_first;
                if (w < BS_WIN) {
                    atomicAdd(&sv[w][0], mu2);
                    atomicAdd(&sv[w][1 + c], mc2);
                    atomicAdd(&sv[w][3 + c], deg);
                } else {
                    atomicAdd(b.acc + (int64_t)s * 5, mu2);
                    atomicAdd(b.acc + (int64_t)s * 5 + 1 + c, mc2);
                    atomicAdd(b.acc + (int64_t)s * 5 + 3 + c, deg);
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < BS_WIN * 5; t += blockDim.x) {
            const unsigned long long v = (&sv[0][0])[t];
            if (v) atomicAdd(b.acc + (int64_t)(s_first + t / 5) * 5 + t % 5, v);
        }
    }
}

// Stopping rule per set; split[s] = 1 (two children) or 0 (a block).
__global__ void k_bs_decide(BisectDev b, int S, int64_t two_e_global) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        int split = 0;
        if (!bs_small(b, s) && !b.frozen[s]) {
            const long long n0 = b.counts[s * 2], n1 = b.counts[s * 2 + 1];
            const unsigned long long* a = b.acc + (int64_t)s * 5;
            const long long mU = (long long)(a[0] / 2), m0 = (long long)(a[1] / 2), m1c = (long long)(a[2] / 2);
            const long long v0 = (long long)a[3], v1 = (long long)a[4];
            const long long two_e = two_e_global > 0 ? two_e_global : v0 + v1;
            const __int128 num1 = (__int128)2 * two_e * mU - (__int128)(v0 + v1) * (v0 + v1);
            const __int128 num2 = (__int128)2 * two_e * (m0 + m1c) - ((__int128)v0 * v0 + (__int128)v1 * v1);
            const bool keep = n0 <= b.eps || n1 <= b.eps || (two_e > 0 && num1 > num2);
            split = keep ? 0 : 1;
        }
        b.split[s] = split;
        b.scan_in[s] = (unsigned long long)split;                             // children rank
        b.scan_in[b.cap_sets + s] = split ? (unsigned long long)b.set_n[s] : 0ull;   // child positions
        b.scan_in[2 * (int64_t)b.cap_sets + s] = split ? 0ull : 1ull;        // block rank
    }
}

// Next level's sets, this level's blocks.
__global__ void k_bs_emit(BisectDev b, int S, int block_base) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        const unsigned long long rank = b.scan_out[s] - (unsigned long long)b.split[s];
        const unsigned long long pos = b.scan_out[b.cap_sets + s] - (b.split[s] ? (unsigned long long)b.set_n[s] : 0ull);
        if (b.split[s]) {
            const int c0 = (int)(2 * rank), c1 = c0 + 1;
            const int64_t n0 = b.counts[s * 2];
            b.nset_off[c0] = (int64_t)pos;
            b.nset_n[c0] = n0;
            b.nset_id[c0] = b.set_id[s] * 2;
            b.nset_off[c1] = (int64_t)pos + n0;
            b.nset_n[c1] = b.set_n[s] - n0;
            b.nset_id[c1] = b.set_id[s] * 2 + 1;
            b.child_pos[s] = (int64_t)pos;
            if (b.dirty) {
                const int keep = b.set_keep[s] && !b.flag[s];   // split exactly as before
                b.nset_keep[c0] = keep;
                b.nset_keep[c1] = keep;
            }
        } else {
            b.block_id[s] = block_base + (int)(b.scan_out[2 * (int64_t)b.cap_sets + s] - 1);
        }
        if (s == S - 1) {
            b.counters[0] = (int)(2 * (b.scan_out[s]));                         // next sets
            b.counters[1] = (int)(b.scan_out[2 * (int64_t)b.cap_sets + s]);      // blocks here
            b.counters_ll[0] = (long long)b.scan_out[b.cap_sets + s];            // next positions
        }
    }
}

// Stable scatter of the splitting sets' positions (half 0 first), block ids of the others.
// f = inclusive prefix over positions of (label == 0) flags.
__global__ void k_bs_scatter(BisectDev b, int64_t M, int64_t n) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const int s = b.pos_set[p];
        const int node = b.perm[p];
        if (b.split[s]) {
            const int64_t off = b.set_off[s];
            const unsigned long long before = off > 0 ? b.F[off - 1] : 0ull;
            const int64_t zeros_upto = (int64_t)(b.F[p] - before);    // label-0 positions in [off, p]
            const int64_t n0 = b.counts[s * 2];
            int64_t np;
            if (b.lab[p] == 0) np = b.child_pos[s] + zeros_upto - 1;
            else np = b.child_pos[s] + n0 + ((p - off + 1) - zeros_upto) - 1;
            if (np >= 0 && np < n) b.perm_next[np] = node;
            else atomicAdd(b.counters + 2, 1);       // inconsistent counts: reported, never written
        } else if (b.frozen[s]) {
            // a kept subtree: the node stays in its previous block
            b.block_of[node] = b.old_label[node];
            if (b.leaf_of) b.leaf_of[node] = b.old_leaf[node];
            b.node_set[node] = -1;
        } else {
            b.block_of[node] = b.k_old + b.block_id[s];
            if (b.leaf_of) b.leaf_of[node] = b.set_id[s];
            b.node_set[node] = -1;
        }
    }
}

__global__ void k_bs_flags(BisectDev b, int64_t M) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x)
        b.q[p] = b.lab[p] == 0 ? 1ull : 0ull;
}

// canonical numbering: blocks by increasing smallest node
__global__ void k_bs_min(BisectDev b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicMin(b.bmin + b.block_of[i], (int)i);
}
__global__ void k_bs_mark(BisectDev b, int nblocks, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b.q[i] = 0;
}
__global__ void k_bs_mark2(BisectDev b, int nblocks, int64_t n) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nblocks; r += gridDim.x * blockDim.x)
        if (b.bmin[r] >= 0 && b.bmin[r] < n) b.q[b.bmin[r]] = 1;
}
__global__ void k_bs_label(BisectDev b, int64_t n, int32_t* labels) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        labels[i] = (int32_t)(b.P[b.bmin[b.block_of[i]]] - 1);
}

// ------------------------------------------------------------------------------------
// Host driver
// ------------------------------------------------------------------------------------
static int grid1(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T, int D>
static cudaError_t bisect_t(const raftgp_csr* g, const T* Z, BisectDev b, int iters, uint64_t seed, int reading,
                            int32_t* labels, int32_t* k_out, cudaStream_t s) {
    const int64_t n = g->n;
    // level 0: one set holding every node
    int S = 1;
    int64_t M = n;
    cudaMemsetAsync(b.counters, 0, 3 * sizeof(int), s);
    int block_base = 0;
    {
        const int64_t off0 = 0;
        const uint64_t id1 = 1;
        cudaMemcpyAsync(b.set_off, &off0, sizeof(int64_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(b.set_n, &n, sizeof(int64_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(b.set_id, &id1, sizeof(uint64_t), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    if (b.dirty) {
        const int32_t one = 1;
        cudaMemcpyAsync(b.set_keep, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s);   // the root is the old root
        cudaStreamSynchronize(s);
    }
    const int64_t two_e_global = reading == 1 ? g->nnz : 0;
    Csr<int64_t> c64{g->n, g->nnz, (const int64_t*)g->row_ptr, g->col};
    Csr<int32_t> c32{g->n, g->nnz, (const int32_t*)g->row_ptr, g->col};
    for (int depth = 0; S > 0; ++depth) {
        b.depth = depth;
        k_bs_setup<<<grid1(M), 256, 0, s>>>(b, S, M);
        if (b.dirty) {
            cudaMemsetAsync(b.flag, 0, sizeof(int32_t) * (size_t)S, s);
            k_bs_dirty<<<grid1(M), 256, 0, s>>>(b, M);
        }
        k_bs_seed0<<<grid1(S), 256, 0, s>>>(b, S, seed);
        k_bs_d2<T, D><<<grid1(M), 256, 0, s>>>(b, Z, M);
        scan_incl(b.q, M, b.P, b.tiles, s);
        k_bs_seed1<T, D><<<grid1(S), 256, 0, s>>>(b, Z, S, seed);
        for (int pass = 1; pass <= iters; ++pass) {
            k_bs_assign<T, D><<<grid1(M), 256, 0, s>>>(b, Z, M, pass);
            k_bs_update<D><<<grid1(2 * (int64_t)S * 32), 256, 0, s>>>(b, S, pass, iters);
        }
        k_bs_nodelab<<<grid1(M), 256, 0, s>>>(b, M);
        cudaMemsetAsync(b.acc, 0, sizeof(unsigned long long) * 5 * (size_t)S, s);
        if (g->row_ptr_bits == 64) k_bs_lmod<int64_t><<<grid1(M), 256, 0, s>>>(b, c64, M);
        else k_bs_lmod<int32_t><<<grid1(M), 256, 0, s>>>(b, c32, M);
        k_bs_decide<<<grid1(S), 256, 0, s>>>(b, S, two_e_global);
        if (b.dirty) k_bs_sides<<<grid1(M), 256, 0, s>>>(b, M);
        for (int part = 0; part < 3; ++part)
            scan_incl(b.scan_in + (int64_t)part * b.cap_sets, S, b.scan_out + (int64_t)part * b.cap_sets, b.tiles, s);
        k_bs_emit<<<grid1(S), 256, 0, s>>>(b, S, block_base);
        k_bs_flags<<<grid1(M), 256, 0, s>>>(b, M);
        scan_incl(b.q, M, b.F, b.tiles, s);
        k_bs_scatter<<<grid1(M), 256, 0, s>>>(b, M, n);
        int hc[3];
        long long hm = 0;
        cudaMemcpyAsync(hc, b.counters, sizeof(hc), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hm, b.counters_ll, sizeof(hm), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (hc[2] != 0) return cudaErrorIllegalState;   // never expected: counts and labels disagree
        block_base += hc[1];
        S = hc[0];
        M = hm;
        std::swap(b.perm, b.perm_next);
        std::swap(b.set_off, b.nset_off);
        std::swap(b.set_n, b.nset_n);
        std::swap(b.set_id, b.nset_id);
        std::swap(b.set_keep, b.nset_keep);
    }
    // numbering by smallest node (block indices: the previous run's for kept subtrees, then
    // this run's new blocks)
    const int nb = b.k_old + block_base;
    cudaMemsetAsync(b.bmin, 0x7f, sizeof(int) * (size_t)nb, s);
    k_bs_min<<<grid1(n), 256, 0, s>>>(b, n);
    k_bs_mark<<<grid1(n), 256, 0, s>>>(b, nb, n);
    k_bs_mark2<<<grid1(nb), 256, 0, s>>>(b, nb, n);
    scan_incl(b.q, n, b.P, b.tiles, s);
    k_bs_label<<<grid1(n), 256, 0, s>>>(b, n, labels);
    unsigned long long blocks = 0;   // the blocks that hold nodes (kept subtrees may leave gaps)
    cudaMemcpyAsync(&blocks, b.P + (n - 1), sizeof(blocks), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *k_out = (int32_t)blocks;
    return cudaGetLastError();
}

cudaError_t launch_bisect(const raftgp_csr* g, const void* Z, int zdtype, int d, BisectDev b, int iters, uint64_t seed,
                          int reading, int32_t* labels, int32_t* k_out, cudaStream_t s) {
    ProfScope ps(s, PF_OTHER, 1);
#define RAFTGP_BS(T, DD) return bisect_t<T, DD>(g, (const T*)Z, b, iters, seed, reading, labels, k_out, s)
    if (zdtype == RAFTGP_BF16) {
        if (d == 32) RAFTGP_BS(__nv_bfloat16, 32);
        if (d == 64) RAFTGP_BS(__nv_bfloat16, 64);
        if (d == 128) RAFTGP_BS(__nv_bfloat16, 128);
    } else {
        if (d == 32) RAFTGP_BS(float, 32);
        if (d == 64) RAFTGP_BS(float, 64);
        if (d == 128) RAFTGP_BS(float, 128);
    }
#undef RAFTGP_BS
    return cudaErrorInvalidValue;
}

}  // namespace raftgp
