// kmeans.cu -- k-means for model selection (Section III-C: "apply KMeans" to the
// embeddings for each candidate K), FP32 engine.
//
//   seeding   k-means++ (D^2 sampling) once for K_max; candidate K starts from the first K
//             seeds.  D^2 is the FP32 direct-form squared distance (ascending coordinates,
//             every subtract/multiply/add rounded separately), quantised to
//             floor(D^2 * 2^40) so the cumulative sums are exact integers.
//   assign    label_i = argmin_c ||z_i - mu_c||^2 over every candidate of a batch, evaluated
//             as ||mu_c||^2 - 2 z_i.mu_c (the ||z_i||^2 term is common), ties to the lowest c.
//   update    centroid sums kept in exact 2^-40 fixed point (int64) and updated incrementally:
//             a point whose label changes is subtracted from its old cluster and added to its
//             new one, so the sums equal the from-scratch sums bit for bit in any order.  The
//             mean is formed in FP64; an empty cluster keeps its centroid.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace raftgp {

template <typename T>
__device__ __forceinline__ float zval(const T* Z, int64_t i) {
    return load_elem(Z, i);
}

__device__ __forceinline__ uint64_t kmpp_draw(uint64_t seed, int t) {
    const U32x4 x = philox4x32_10((uint32_t)t, 0u, 0u, STREAM_KMPP, seed);
    return (uint64_t)x.x | ((uint64_t)x.y << 32);
}

// floor(D^2 * 2^40): the FP32 product by a power of two is exact, the conversion truncates.
__device__ __forceinline__ unsigned long long quantise(float d2) { return __float2ull_rz(d2 * FIXED_SCALE_F); }

constexpr int SEED_THREADS = 256;
constexpr int SEED_PPT = 4;                               // points per thread
constexpr int SEED_PPB = SEED_THREADS * SEED_PPT;         // points per block partial

// FP32 direct-form squared distance of one row against the centre in shared memory:
// ascending coordinates, 16-byte vector loads, every subtract/multiply/add rounded separately.
template <typename T, int D>
__device__ __forceinline__ float row_sqdist(const T* __restrict__ zi, const float* __restrict__ c) {
    constexpr int E = Vec<T>::E;
    float s = 0.0f;
#pragma unroll
    for (int v = 0; v < D / E; ++v) {
        float x[E];
        Vec<T>::load(zi + v * E, x);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float t = __fsub_rn(x[e], c[v * E + e]);
            s = __fadd_rn(s, __fmul_rn(t, t));
        }
    }
    return s;
}

__global__ void k_seed_first(int64_t n, uint64_t seed, SeedState ss) {
    const int64_t i = (int64_t)mulhi64(kmpp_draw(seed, 0), (uint64_t)n);
    ss.seeds[0] = (int32_t)i;
    ss.chosen[i] = 1;
}

// Round t: D^2_i = min(D^2_i, dist(z_i, c)) for the newest seed c = seeds[t-1], and per-block
// sums of the quantised D^2.  A point whose nearest seed c_j satisfies
// |c_j - c|^2 >= 4 D^2_i (1 + 1e-4) cannot get closer (triangle inequality, with a margin that
// covers the FP32 rounding of both sides), so its row is not read: the result is identical to
// evaluating every distance.
template <typename T, int D>
__global__ void __launch_bounds__(SEED_THREADS) k_seed_update(const T* __restrict__ Z, int64_t n, int t,
                                                              SeedState ss) {
    __shared__ float c[D];
    __shared__ unsigned long long wsum[SEED_THREADS / 32];
    const int64_t ci = ss.seeds[t - 1];
    for (int k = threadIdx.x; k < D; k += blockDim.x) c[k] = load_elem(Z, ci * D + k);
    __syncthreads();
    unsigned long long q = 0;
    const int64_t base = (int64_t)blockIdx.x * SEED_PPB + threadIdx.x;
    if (t == 1) {
        for (int r = 0; r < SEED_PPT; ++r) {
            const int64_t i = base + (int64_t)r * SEED_THREADS;
            if (i >= n) break;
            const float cur = row_sqdist<T, D>(Z + i * D, c);
            ss.D2[i] = cur;
            ss.nearest[i] = 0;
            q += quantise(cur);
        }
    } else {
        // independent loads first: current D^2, nearest seed, and that seed's distance to c
        float cur[SEED_PPT], bound[SEED_PPT];
#pragma unroll
        for (int r = 0; r < SEED_PPT; ++r) {
            const int64_t i = base + (int64_t)r * SEED_THREADS;
            cur[r] = i < n ? ss.D2[i] : 0.f;
            bound[r] = i < n ? __ldg(ss.cc2 + ss.nearest[i]) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < SEED_PPT; ++r) {
            const int64_t i = base + (int64_t)r * SEED_THREADS;
            if (i < n && !(bound[r] >= 4.0f * cur[r] * 1.0001f)) {
                const float nd = row_sqdist<T, D>(Z + i * D, c);
                if (nd < cur[r]) {
                    cur[r] = nd;
                    ss.D2[i] = nd;
                    ss.nearest[i] = (int16_t)(t - 1);
                }
            }
            if (i < n) q += quantise(cur[r]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sum = 0;
        for (int w = 0; w < SEED_THREADS / 32; ++w) sum += wsum[w];
        ss.blocksum[blockIdx.x] = sum;
    }
}

// Exclusive scan of 1024 values held one per thread; returns this thread's exclusive prefix
// and the block total.
__device__ unsigned long long block_scan_1024(unsigned long long v, unsigned long long* total) {
    __shared__ unsigned long long ws[32];
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
        ws[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const unsigned long long before = (w > 0 ? ws[w - 1] : 0ull) + x - v;
    *total = ws[31];
    __syncthreads();
    return before;
}

// Pick seed t: threshold floor(r_t * sum q / 2^64), first point whose inclusive prefix of q
// exceeds it (the lowest-index unchosen point if every q is 0).  Then the squared distances
// from every earlier seed to the new one, for the next round's skip test.  One block of 1024.
template <typename T, int D>
__global__ void __launch_bounds__(1024) k_seed_pick(const T* __restrict__ Z, int64_t n, int nblocks, uint64_t seed,
                                                    int t, SeedState ss) {
    __shared__ unsigned long long s_thr, s_base;
    __shared__ int s_block;
    __shared__ long long s_pick;
    __shared__ long long wmin[32];
    unsigned long long run = 0;  // running prefix of completed chunks
    unsigned long long tot = 0;
    for (int b0 = 0; b0 < nblocks; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        unsigned long long v = b < nblocks ? ss.blocksum[b] : 0ull, ct;
        block_scan_1024(v, &ct);
        tot += ct;
    }
    if (threadIdx.x == 0) {
        s_pick = -1;
        s_block = -1;
        s_thr = tot > 0 ? mulhi64(kmpp_draw(seed, t), tot) : 0ull;
    }
    __syncthreads();
    if (tot == 0) {
        // every remaining point coincides with a seed: lowest-index unchosen point
        for (int64_t base = 0; base < n; base += 1024) {
            const int64_t i = base + threadIdx.x;
            const bool cand = i < n && !ss.chosen[i];
            const unsigned mask = __ballot_sync(0xffffffffu, cand);
            if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = mask ? base + (threadIdx.x & ~31) + __ffs(mask) - 1 : -1;
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 0; w < 32; ++w)
                    if (wmin[w] >= 0) { s_pick = wmin[w]; break; }
            }
            __syncthreads();
            if (s_pick >= 0) break;
        }
    } else {
        const unsigned long long thr = s_thr;
        for (int b0 = 0; b0 < nblocks; b0 += 1024) {
            const int b = b0 + threadIdx.x;
            const unsigned long long v = b < nblocks ? ss.blocksum[b] : 0ull;
            unsigned long long ct;
            const unsigned long long ex = block_scan_1024(v, &ct);
            if (b < nblocks && run + ex + v > thr && run + ex <= thr) {
                s_block = b;
                s_base = run + ex;
            }
            __syncthreads();
            if (s_block >= 0) break;
            run += ct;
        }
        const int b = s_block < 0 ? 0 : s_block;   // always found: thr < total
        // inside the block: SEED_PPB points, 2 per thread in index order
        unsigned long long base = s_base;
        for (int h = 0; h < SEED_PPB / 1024; ++h) {
            const int64_t i = (int64_t)b * SEED_PPB + h * 1024 + threadIdx.x;
            const unsigned long long v = i < n ? quantise(ss.D2[i]) : 0ull;
            unsigned long long ct;
            const unsigned long long ex = block_scan_1024(v, &ct);
            if (i < n && base + ex + v > thr && base + ex <= thr) s_pick = i;
            __syncthreads();
            if (s_pick >= 0) break;
            base += ct;
        }
    }
    __syncthreads();
    const long long p = s_pick < 0 ? 0 : s_pick;     // unreachable fallback keeps indices in range
    if (threadIdx.x == 0) {
        ss.seeds[t] = (int32_t)p;
        ss.chosen[p] = 1;
    }
    // |c_j - c_t|^2 for j < t (FP32; used only as a conservative bound): a warp per seed,
    // lanes over coordinates
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x >> 5; j < t; j += blockDim.x >> 5) {
        const int64_t sj = ss.seeds[j];
        float acc = 0.f;
        for (int k = lane; k < D; k += 32) {
            const float dlt = load_elem(Z, sj * D + k) - load_elem(Z, p * D + k);
            acc = fmaf(dlt, dlt, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) ss.cc2[j] = acc;
    }
}

int seed_nblocks(int64_t n) { return (int)((n + SEED_PPB - 1) / SEED_PPB); }

// ------------------------------------------------------------------------------------
// Persistent seeding: every round in one cooperative launch (all blocks resident), one block
// per SM.  A block owns a contiguous range of points whose D^2 and nearest seed stay in
// shared memory for all K rounds, together with a copy of every seed row (for the skip
// bound).  Per round:
//   1. each block loads the newest seed, computes its squared distance to every earlier
//      seed, and updates its points.  A row is read one 32-byte sector at a time in ascending
//      coordinates; the FP32 partial sums never decrease (every term is >= 0 and rounding is
//      monotone), so once a partial sum reaches the current D^2 the row cannot lower it and
//      the rest of the row is not read.  The rows that do lower D^2 are summed in full, so
//      every D^2 is the same as the plain evaluation.  Each warp applies the skip bound to
//      its rows, lists the rest, and reads them in sector passes: pass s reads sector s of
//      every listed row (lanes on consecutive entries, two entries per lane in flight) and
//      keeps, compacted, the rows whose partial sum is still below their D^2.  When a block
//      owns more points than the lists can hold, a warp works through its rows in chunks.  When the
//      caller provides a sector-major copy of Z (plane s = sector s of every row), the lanes
//      of a pass read consecutive sectors.
//   2. block partial sums of the quantised D^2 are published; grid barrier.
//   3. every block finds the owner of the threshold from the partial sums (the same integer
//      arithmetic in every block); the owner scans its points in index order and publishes
//      the seed; the other blocks wait for that one word.
// The waits spin with a 2 s limit; on a timeout the kernel records DERR_TIMEOUT, raises
// an abort word that releases the other blocks, marks the unfinished seeds -1 and returns.
// ------------------------------------------------------------------------------------
constexpr int SP_THREADS = 1024;
constexpr int SP_MAX_SMEM = 200 * 1024;

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) { return *(volatile const unsigned*)p; }

// bar[0] counts arrivals and never resets: the barrier of round t completes when it reaches
// t x gridDim.x, so the last block to arrive releases the others with its one atomic.
// bar[2] is the abort word.  Returns false in every thread of the block if the wait gave up
// (2 s limit: records DERR_TIMEOUT and raises the abort word) or another block aborted.
__device__ bool grid_barrier(unsigned* bar, unsigned target, uint32_t* err, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        if (atomicAdd(bar, 1u) + 1u != target) {
            const uint64_t t0 = global_ns();
            unsigned it = 0;
            while (ld_volatile(bar) < target) {
                if (ld_volatile(bar + 2)) { ok = 0; break; }
                if ((++it & 63) == 0 && global_ns() - t0 > TC_WAIT_NS) {
                    atomicOr(err, (uint32_t)DERR_TIMEOUT);
                    atomicExch(bar + 2, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Waits until the owner block of round t has published seeds[t] (the seeds start at -1).
// Same 2 s limit and abort word as grid_barrier.
__device__ bool wait_seed(const int32_t* seeds, int t, unsigned* bar, uint32_t* err, int* s_ok, long long* s_seed) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = global_ns();
        unsigned it = 0;
        int v;
        while ((v = (int)ld_volatile(reinterpret_cast<const unsigned*>(seeds + t))) < 0) {
            if (ld_volatile(bar + 2)) { ok = 0; break; }
            if ((++it & 63) == 0 && global_ns() - t0 > TC_WAIT_NS) {
                atomicOr(err, (uint32_t)DERR_TIMEOUT);
                atomicExch(bar + 2, 1u);
                ok = 0;
                break;
            }
        }
        __threadfence();
        *s_seed = v;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Row loads that ask L2 to keep the lines (evict_last): the rows are read again every round,
// and Z is about the size of L2.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint4 ld_keep16(const void* p, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
// One 32-byte sector per lane in a single request (a 256-bit load, sm_100 and later).
__device__ __forceinline__ void ld_keep32(const void* p, uint64_t pol, uint4& lo, uint4& hi) {
    asm volatile("ld.global.nc.L2::cache_hint.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
                 : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
                 : "l"(p), "l"(pol));
}

template <typename T, int D>
__global__ void __launch_bounds__(SP_THREADS, 1)
    k_seed_persistent(const T* __restrict__ Z, const T* __restrict__ ZS, int64_t n, int K, uint64_t seed,
                      SeedState ss, int per_block, int off_near, int off_rows, int off_cc2, int off_list,
                      int off_acc, int list_per_warp, int skip_block) {
    extern __shared__ __align__(16) uint8_t sp_smem[];
    float* sD2 = reinterpret_cast<float*>(sp_smem);
    int16_t* sNear = reinterpret_cast<int16_t*>(sp_smem + off_near);
    T* srow = reinterpret_cast<T*>(sp_smem + off_rows);
    float* scc2 = reinterpret_cast<float*>(sp_smem + off_cc2);
    uint16_t* sList = reinterpret_cast<uint16_t*>(sp_smem + off_list);   // rows to read, per warp
    float* sAcc = reinterpret_cast<float*>(sp_smem + off_acc);           // their partial sums
    __shared__ float c[D];
    __shared__ unsigned long long wsum[SP_THREADS / 32];
    __shared__ unsigned long long s_thr, s_base;
    __shared__ long long s_pick, s_seed;
    __shared__ int s_owner, s_ok;
    __shared__ unsigned long long s_part[1024];
    constexpr int E = Vec<T>::E;                    // elements per 16-byte load
    constexpr int SEC = 32 / (int)sizeof(T);        // elements per 32-byte sector
    constexpr int NSEC = D / SEC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t lo = (int64_t)blockIdx.x * per_block;
    const int cnt = (int)(n - lo < per_block ? (n - lo > 0 ? n - lo : 0) : per_block);
    const int G = gridDim.x;
    const uint64_t pol = l2_keep_policy();
    // rows are a multiple of 32 bytes, so the sectors are 32-byte aligned when Z is; the
    // sector-major copy ZS (plane s holds sector s of every row) is 256-byte aligned
    const bool a32 = ZS || ((uintptr_t)Z & 31) == 0;

    long long p = (long long)mulhi64(kmpp_draw(seed, 0), (uint64_t)n);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ss.seeds[0] = (int32_t)p;
        ss.chosen[p] = 1;
    }
    int t = 1;
    for (; t < K; ++t) {
        if (t == 2 && (int)blockIdx.x == skip_block) break;   // test hook: leave without arriving
        // ---- 1. the newest seed, its distance to the earlier ones, the update ----
        for (int k = threadIdx.x; k < D; k += SP_THREADS) {
            const T v = Z[p * D + k];
            c[k] = Vec<T>::to_float(v);
            srow[(int64_t)(t - 1) * D + k] = v;
        }
        __syncthreads();
        // the new seed's squared distance to every earlier seed: 8-lane groups, four seeds
        // per warp at a time
        for (int jb = warp * 4; jb < t - 1; jb += SP_THREADS / 8) {
            const int j = jb + (lane >> 3), sub = lane & 7;
            float acc = 0.f;
            if (j < t - 1) {
#pragma unroll
                for (int k = sub; k < D; k += 8) {
                    const float dl = Vec<T>::to_float(srow[(int64_t)j * D + k]) - c[k];
                    acc = fmaf(dl, dl, acc);
                }
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            if (j < t - 1 && sub == 0) scc2[j] = acc;
        }
        __syncthreads();
        unsigned long long q = 0;
        // the warp's rows (warp * 32 + lane + 1024 k) in chunks of list_per_warp / 32 groups of
        // 32: the skip bound over a chunk; the rows that need their distance are listed in the
        // warp's slice of sList
        uint16_t* wl = sList + warp * list_per_warp;
        float* wacc = sAcc + warp * list_per_warp;
        const int chunk_rows = SP_THREADS * (list_per_warp / 32);
        for (int kc = warp * 32; kc < cnt; kc += chunk_rows) {
            int nl = 0;
            for (int k0 = kc; k0 < cnt && k0 < kc + chunk_rows; k0 += SP_THREADS) {
                const int rr = k0 + lane;
                bool need = false;
                if (rr < cnt) {
                    if (t == 1) {
                        need = true;
                    } else {
                        const float c0 = sD2[rr];
                        if (scc2[sNear[rr]] >= 4.0f * c0 * 1.0001f) q += quantise(c0);
                        else need = true;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, need);
                if (need) wl[nl + __popc(m & ((1u << lane) - 1u))] = (uint16_t)rr;
                nl += __popc(m);
            }
            __syncwarp();
            // Sector passes over the list: pass s reads sector s of every listed row (lanes on
            // consecutive entries, 2 entries per lane in flight), and keeps in the list, compacted
            // in place with its partial sum, each row whose sum is still below its D^2.
            constexpr int U = 2;
            int len = nl;
            for (int sec = 0; sec < NSEC && len > 0; ++sec) {
                int out = 0;
                for (int j0 = 0; j0 < len; j0 += 32 * U) {
                    int rr[U];
                    float acc[U];
                    uint4 rw[U][2];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = j0 + 32 * u + lane;
                        rr[u] = j < len ? (int)wl[j] : -1;
                        acc[u] = (j < len && sec > 0) ? wacc[j] : 0.f;
                        if (rr[u] >= 0) {
                            const T* zs = ZS ? ZS + ((int64_t)sec * n + lo + rr[u]) * SEC : Z + (lo + rr[u]) * D + sec * SEC;
                            if (a32) {
                                ld_keep32(zs, pol, rw[u][0], rw[u][1]);
                            } else {
                                rw[u][0] = ld_keep16(zs, pol);
                                rw[u][1] = ld_keep16(zs + E, pol);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        bool keep = false;
                        if (rr[u] >= 0) {
                            float a = acc[u];
#pragma unroll
                            for (int v = 0; v < SEC / E; ++v) {
                                float x[E];
                                Vec<T>::unpack(rw[u][v], x);
#pragma unroll
                                for (int e = 0; e < E; ++e) {
                                    const float dl = __fsub_rn(x[e], c[sec * SEC + v * E + e]);
                                    a = __fadd_rn(a, __fmul_rn(dl, dl));
                                }
                            }
                            acc[u] = a;
                            float cur = t > 1 ? sD2[rr[u]] : INFINITY;
                            if (sec + 1 == NSEC) {
                                // round 1 reads every row in full and always stores it, so the shared
                                // state is initialised whatever the data (a non-finite sum included)
                                if (t == 1 || a < cur) {
                                    cur = a;
                                    sD2[rr[u]] = a;
                                    sNear[rr[u]] = (int16_t)(t - 1);
                                }
                                q += quantise(cur);
                            } else if (t > 1 && a >= cur) {
                                q += quantise(cur);
                            } else {
                                keep = true;
                            }
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, keep);
                        if (keep) {
                            const int pos = out + __popc(m & ((1u << lane) - 1u));
                            wl[pos] = (uint16_t)rr[u];
                            wacc[pos] = acc[u];
                        }
                        out += __popc(m);
                    }
                }
                __syncwarp();
                len = out;
            }
            __syncwarp();   // the list slice is rewritten by the next chunk
        }
        // ---- 2. block partial sum; barrier ----
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (lane == 0) wsum[warp] = q;
        __syncthreads();
        unsigned long long* part = ss.blocksum + (size_t)(t & 1) * G;
        if (warp == 0) {
            unsigned long long sum = wsum[lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) part[blockIdx.x] = sum;
        }
        if (!grid_barrier(ss.bar, (unsigned)t * (unsigned)G, ss.err, &s_ok)) break;
        // ---- 3. the owner of the threshold picks and publishes the seed ----
        if (warp == 0) {
            for (int b = lane; b < G; b += 32) s_part[b] = __ldcg(part + b);
            __syncwarp();
            unsigned long long tot = 0;
            for (int b = lane; b < G; b += 32) tot += s_part[b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            const unsigned long long thr = tot > 0 ? mulhi64(kmpp_draw(seed, t), tot) : 0ull;
            int owner = -1;
            unsigned long long run = 0, base = 0;
            for (int b0 = 0; b0 < G && owner < 0 && tot > 0; b0 += 32) {
                const unsigned long long v = b0 + lane < G ? s_part[b0 + lane] : 0ull;
                unsigned long long x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const unsigned hit = __ballot_sync(0xffffffffu, b0 + lane < G && run + x > thr && run + x - v <= thr);
                if (hit) {
                    const int l = __ffs(hit) - 1;
                    owner = b0 + l;
                    base = run + __shfl_sync(0xffffffffu, x - v, l);
                }
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) {
                s_owner = tot > 0 ? owner : -2;
                s_thr = thr;
                s_base = base;
                s_pick = -1;
            }
        }
        __syncthreads();
        if (s_owner == -2 && blockIdx.x == 0) {
            // every remaining point coincides with a seed: the lowest-index unchosen point
            for (int64_t b0 = 0; b0 < n; b0 += SP_THREADS) {
                const int64_t i = b0 + threadIdx.x;
                const bool cand = i < n && !__ldcg(ss.chosen + i);
                const unsigned m = __ballot_sync(0xffffffffu, cand);
                if (lane == 0) wsum[warp] = m ? (unsigned long long)(b0 + warp * 32 + __ffs(m) - 1) : ~0ull;
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int w = 0; w < SP_THREADS / 32; ++w)
                        if (wsum[w] != ~0ull) { s_pick = (long long)wsum[w]; break; }
                }
                __syncthreads();
                if (s_pick >= 0) break;
            }
        } else if (s_owner == (int)blockIdx.x) {
            // contiguous segments in index order, one per thread
            const unsigned long long thr = s_thr - s_base;
            const int L = (cnt + SP_THREADS - 1) / SP_THREADS;
            const int r0 = threadIdx.x * L;
            const int r1 = r0 + L < cnt ? r0 + L : cnt;
            unsigned long long v = 0;
            for (int rr = r0; rr < r1; ++rr) v += quantise(sD2[rr]);
            unsigned long long ct;
            const unsigned long long ex = block_scan_1024(v, &ct);
            if (r0 < r1 && ex + v > thr && ex <= thr) {
                unsigned long long run = ex;
                for (int rr = r0; rr < r1; ++rr) {
                    run += quantise(sD2[rr]);
                    if (run > thr) {
                        s_pick = lo + rr;
                        break;
                    }
                }
            }
            __syncthreads();
        }
        if ((s_owner == -2 && blockIdx.x == 0) || s_owner == (int)blockIdx.x) {
            if (threadIdx.x == 0) {
                const long long pk = s_pick < 0 ? 0 : s_pick;   // unreachable fallback keeps indices in range
                ss.chosen[pk] = 1;
                __threadfence();   // chosen before the seed: a block that sees the seed sees the mark
                atomicExch(reinterpret_cast<unsigned*>(ss.seeds + t), (unsigned)pk);
            }
        }
        // the other blocks only need the new seed: wait for it instead of a second barrier (the
        // block sums are double-buffered, and the next round's barrier orders everything else)
        if (!wait_seed(ss.seeds, t, ss.bar, ss.err, &s_ok, &s_seed)) break;
        p = s_seed;
    }
    if (t < K && threadIdx.x == 0) {
        for (int j = t; j < K; ++j) ss.seeds[j] = -1;   // aborted: the unfinished seeds are invalid
    }
}

// Shared-memory layout of the persistent kernel; false if it does not fit.
template <typename T, int D>
static bool persistent_layout(int per_block, int K, int* off_near, int* off_rows, int* off_cc2, int* off_list,
                              int* off_acc, int* list_per_warp, int* bytes) {
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    if (per_block > 65535) return false;   // row lists hold 16-bit indices
    const size_t near = a16((size_t)per_block * 4);
    const size_t rows = near + a16((size_t)per_block * 2);
    const size_t cc2 = rows + a16((size_t)K * D * sizeof(T));
    const size_t list = cc2 + a16((size_t)K * 4);
    // the row lists cover all of a warp's rows at once when they fit, else chunks of fewer
    // 32-row groups (lpw entries per warp)
    int lpw = (per_block + SP_THREADS - 1) / SP_THREADS * 32;
    size_t acc = 0, total = 0;
    for (; lpw >= 32; lpw -= 32) {
        acc = list + a16((size_t)(SP_THREADS / 32) * lpw * 2);
        total = acc + a16((size_t)(SP_THREADS / 32) * lpw * 4);
        if (total <= (size_t)SP_MAX_SMEM) break;
    }
    if (lpw < 32) return false;
    *off_near = (int)near;
    *off_rows = (int)rows;
    *off_cc2 = (int)cc2;
    *off_list = (int)list;
    *off_acc = (int)acc;
    *list_per_warp = lpw;
    *bytes = (int)total;
    return true;
}

// The sector-major copy of Z: plane s (n x 32 bytes) holds the s-th 32-byte sector of every
// row, so lanes on consecutive rows read consecutive sectors.
template <typename T, int D>
__global__ void k_sector_planes(const T* __restrict__ Z, int64_t n, T* __restrict__ ZS) {
    constexpr int SEC = 32 / (int)sizeof(T), NSEC = D / SEC;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * n * NSEC;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / (2 * NSEC);
        const int sec = (int)(q / 2 % NSEC), h = (int)(q & 1);
        reinterpret_cast<uint4*>(ZS + ((int64_t)sec * n + i) * SEC)[h] =
            reinterpret_cast<const uint4*>(Z + i * D + sec * SEC)[h];
    }
}

// Test hook (raftgp_debug_seed_skip_block): this block of the persistent kernel leaves at the
// start of round 2 without arriving at the grid barrier, so the other blocks' bounded wait
// runs out; -1 (the default) turns it off.
static int g_seed_skip_block = -1;
void set_seed_skip_block(int block) { g_seed_skip_block = block; }

// Launches the persistent kernel; returns false (nothing launched) if the state does not fit
// shared memory or the device cannot hold one resident block per SM.
template <typename T, int D>
static bool seed_persistent_t(const T* Z, int64_t n, int K, uint64_t seed, SeedState ss, cudaStream_t s) {
    int G = num_sms();
    if (G > 1024) G = 1024;
    if ((int64_t)G > n) G = (int)n;
    const int per_block = (int)((n + G - 1) / G);
    int off_near, off_rows, off_cc2, off_list, off_acc, list_per_warp, bytes;
    if (!persistent_layout<T, D>(per_block, K, &off_near, &off_rows, &off_cc2, &off_list, &off_acc, &list_per_warp,
                                 &bytes))
        return false;
    auto kern = k_seed_persistent<T, D>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SP_THREADS, bytes) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    cudaMemsetAsync(ss.chosen, 0, (size_t)n, s);
    cudaMemsetAsync(ss.bar, 0, 3 * sizeof(unsigned), s);
    cudaMemsetAsync(ss.seeds, 0xff, (size_t)K * sizeof(int32_t), s);   // -1: not published yet
    const T* ZS = reinterpret_cast<const T*>(ss.zs);
    void* args[] = {(void*)&Z, (void*)&ZS, (void*)&n, (void*)&K, (void*)&seed, (void*)&ss, (void*)&per_block,
                    (void*)&off_near, (void*)&off_rows, (void*)&off_cc2, (void*)&off_list, (void*)&off_acc,
                    (void*)&list_per_warp,
                    (void*)&g_seed_skip_block};
    ProfScope ps(s, PF_SEED_UPDATE, ZS ? 2 : 1);
    if (ZS) {
        int64_t blocks = (2 * n * (D * (int64_t)sizeof(T) / 32) + 255) / 256;
        if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
        k_sector_planes<T, D><<<(unsigned)blocks, 256, 0, s>>>(Z, n, reinterpret_cast<T*>(ss.zs));
    }
    if (cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(SP_THREADS), args, (size_t)bytes, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}


// the partial sums hold seed_nblocks(n) entries for the per-round kernels, or two rounds of
// one per SM for the persistent kernel (at most 2 x 1024 blocks)
static size_t seed_partials(int64_t n) {
    const size_t nb = (size_t)seed_nblocks(n);
    return nb > 2048 ? nb : 2048;
}

size_t seed_scratch_bytes(int64_t n, int K) {
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return a((size_t)n * 4) + a((size_t)n * 2) + a((size_t)n) + a(seed_partials(n) * 8) + a((size_t)K * 4) + a(16);
}

SeedState carve_seed(void* base, int64_t n, int K, int32_t* seeds) {
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* p = (char*)base;
    SeedState ss;
    ss.D2 = (float*)p;
    p += a((size_t)n * 4);
    ss.nearest = (int16_t*)p;
    p += a((size_t)n * 2);
    ss.chosen = (uint8_t*)p;
    p += a((size_t)n);
    ss.blocksum = (unsigned long long*)p;
    p += a(seed_partials(n) * 8);
    ss.cc2 = (float*)p;
    p += a((size_t)K * 4);
    ss.bar = (unsigned*)p;
    ss.err = ss.bar + 3;
    ss.seeds = seeds;
    ss.zs = nullptr;
    return ss;
}

template <typename T, int D>
static void seed_run_t(const T* Z, int64_t n, int K, uint64_t seed, SeedState ss, cudaStream_t s) {
    if (seed_persistent_t<T, D>(Z, n, K, seed, ss, s)) return;
    // one launch per round for the update and one for the pick
    const int nb = seed_nblocks(n);
    cudaMemsetAsync(ss.chosen, 0, (size_t)n, s);
    {
        ProfScope ps(s, PF_SEED_PICK, 1);
        k_seed_first<<<1, 1, 0, s>>>(n, seed, ss);
    }
    for (int t = 1; t < K; ++t) {
        {
            ProfScope ps(s, PF_SEED_UPDATE, 1);
            k_seed_update<T, D><<<nb, SEED_THREADS, 0, s>>>(Z, n, t, ss);
        }
        ProfScope ps(s, PF_SEED_PICK, 1);
        k_seed_pick<T, D><<<1, 1024, 0, s>>>(Z, n, nb, seed, t, ss);
    }
}

cudaError_t launch_seeding(const void* Z, int zdtype, int64_t n, int d, int K, uint64_t seed, SeedState ss,
                           cudaStream_t s) {
    if (zdtype == RAFTGP_BF16) {
        const __nv_bfloat16* z = (const __nv_bfloat16*)Z;
        switch (d) {
            case 32: seed_run_t<__nv_bfloat16, 32>(z, n, K, seed, ss, s); break;
            case 64: seed_run_t<__nv_bfloat16, 64>(z, n, K, seed, ss, s); break;
            case 128: seed_run_t<__nv_bfloat16, 128>(z, n, K, seed, ss, s); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        const float* z = (const float*)Z;
        switch (d) {
            case 32: seed_run_t<float, 32>(z, n, K, seed, ss, s); break;
            case 64: seed_run_t<float, 64>(z, n, K, seed, ss, s); break;
            case 128: seed_run_t<float, 128>(z, n, K, seed, ss, s); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Batch set-up: centroids from seeds (or given mu0), zero sums/counts, labels = -1.
// ------------------------------------------------------------------------------------
// v = hi + lo with hi = bf16(v), lo = bf16(v - hi): two BF16 operands that carry ~16 bits.
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *hi = h;
    *lo = __float2bfloat16_rn(v - __bfloat162float(h));
}

__host__ __device__ __forceinline__ int pad64(int k) { return (k + 63) / 64 * 64; }

// Everything derived from one FP32 centroid row: ||mu||^2 (ascending coordinates), the
// +4-shifted copy, the tensor-core operands -mu = hi + lo, and the norm slice
// [(||mu||^2 + 4)/2 as hi, lo, then 128, then zeros] (the 128 puts every score of the
// tensor-core Lloyd pass in [128, 256)).  A padding row (no centroid) gets an infinite norm
// and the norm slice [127, 0, 128]: its score is 255, above every real one (below 132), so
// it never wins an argmin.
__device__ void write_row_operands(KmState st, int64_t row, int d, bool padding) {
    float* mu = st.mu + row * d;
    __nv_bfloat16* aug = st.baug + row * 16;
    if (padding) {
        for (int k = 0; k < d; ++k) {
            mu[k] = 0.f;
            st.muT[(int64_t)k * st.bhi_rows + row] = 0.f;
            st.bhi[row * d + k] = __float2bfloat16_rn(0.f);
            st.blo[row * d + k] = __float2bfloat16_rn(0.f);
        }
        st.norm2[row] = INFINITY;
        st.norm2p[row] = INFINITY;
        aug[0] = __float2bfloat16_rn(127.0f);
        aug[1] = __float2bfloat16_rn(0.f);
        aug[2] = __float2bfloat16_rn(128.0f);
        for (int k = 3; k < 16; ++k) aug[k] = __float2bfloat16_rn(0.f);
        return;
    }
    float s = 0.f;
    for (int k = 0; k < d; ++k) {
        const float v = mu[k];
        s = fmaf(v, v, s);
        st.muT[(int64_t)k * st.bhi_rows + row] = v;
        split_bf16(-v, st.bhi + row * d + k, st.blo + row * d + k);
    }
    st.norm2[row] = s;
    st.norm2p[row] = s + 4.0f;
    split_bf16(0.5f * (s + 4.0f), aug, aug + 1);
    aug[2] = __float2bfloat16_rn(128.0f);
    for (int k = 3; k < 16; ++k) aug[k] = __float2bfloat16_rn(0.f);
}

// The same for one real centroid row by a whole warp (lanes over coordinates; the norm is a
// fixed-order warp reduction).
__device__ void warp_row_operands(KmState st, int64_t row, int d) {
    const int lane = threadIdx.x & 31;
    float s = 0.f;
    for (int k = lane; k < d; k += 32) {
        const float v = st.mu[row * d + k];
        s = fmaf(v, v, s);
        st.muT[(int64_t)k * st.bhi_rows + row] = v;
        split_bf16(-v, st.bhi + row * d + k, st.blo + row * d + k);
    }
    s = warp_sum(s);
    if (lane == 0) {
        st.norm2[row] = s;
        st.norm2p[row] = s + 4.0f;
    }
    if (lane < 16) {
        __nv_bfloat16* aug = st.baug + row * 16;
        const __nv_bfloat16 h = __float2bfloat16_rn(0.5f * (s + 4.0f));
        aug[lane] = lane == 0 ? h
                  : lane == 1 ? __float2bfloat16_rn(0.5f * (s + 4.0f) - __bfloat162float(h))
                  : lane == 2 ? __float2bfloat16_rn(128.0f)
                              : __float2bfloat16_rn(0.f);
    }
}

template <typename T>
__global__ void k_batch_init_mu(CandBatch b, const T* Z, int64_t n, int d, const int32_t* seeds, const float* mu0,
                                KmState st) {
    const int c = blockIdx.y;
    if (c >= b.n) return;
    const int K = b.k[c], off = b.off[c];
    for (int j = blockIdx.x; j < pad64(K); j += gridDim.x) {
        int64_t src = (seeds && j < K) ? (int64_t)seeds[j] : -1;
        if (src >= n) src = -1;   // an aborted seeding leaves -1: such a centroid starts at 0
        for (int k = threadIdx.x; k < d; k += blockDim.x) {
            float v = 0.f;
            if (j < K) v = mu0 ? mu0[(int64_t)j * d + k] : (src >= 0 ? zval(Z, src * d + k) : 0.f);
            st.mu[(int64_t)(off + j) * d + k] = v;
            st.sums[(int64_t)(off + j) * d + k] = 0;
        }
        if (threadIdx.x == 0) st.counts[off + j] = 0;
    }
    if (c == b.n - 1) {
        // zero the rows after the batch (read by full-size chunk loads)
        const int64_t first = (int64_t)b.total_k, last = st.bhi_rows;
        for (int64_t t = first * d + blockIdx.x * blockDim.x + threadIdx.x; t < last * d; t += gridDim.x * blockDim.x) {
            st.bhi[t] = __float2bfloat16_rn(0.f);
            st.blo[t] = __float2bfloat16_rn(0.f);
        }
        for (int64_t t = first * 16 + blockIdx.x * blockDim.x + threadIdx.x; t < last * 16; t += gridDim.x * blockDim.x)
            st.baug[t] = __float2bfloat16_rn(0.f);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st.active[c] = 1;
        st.changed[c] = 0;
        st.changed[MAXC + c] = 0;
        st.passes[c] = 0;
    }
}

// Operands of every row of the batch, one thread per row.
__global__ void k_operands(CandBatch b, int d, KmState st) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= b.total_k) return;
    int c = 0;
    while (c + 1 < b.n && b.off[c + 1] <= row) ++c;
    write_row_operands(st, row, d, row - b.off[c] >= b.k[c]);
}

__global__ void k_fill_labels(int16_t* labels, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        labels[i] = -1;
}

void launch_batch_init(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, const int32_t* seeds,
                       const float* mu0, KmState st, cudaStream_t s) {
    ProfScope ps(s, PF_BATCH_INIT, 3);
    dim3 grid(64, b.n);
    if (zdtype == RAFTGP_BF16)
        k_batch_init_mu<__nv_bfloat16><<<grid, 128, 0, s>>>(b, (const __nv_bfloat16*)Z, n, d, seeds, mu0, st);
    else
        k_batch_init_mu<float><<<grid, 128, 0, s>>>(b, (const float*)Z, n, d, seeds, mu0, st);
    k_operands<<<(b.total_k + 127) / 128, 128, 0, s>>>(b, d, st);
    const int64_t cnt = n * (int64_t)b.cs;
    int blocks = (int)((cnt + 255) / 256);
    if (blocks > num_sms() * 8) blocks = num_sms() * 8;
    if (blocks < 1) blocks = 1;
    k_fill_labels<<<blocks, 256, 0, s>>>(st.labels, cnt);
}

// ------------------------------------------------------------------------------------
// After a tensor-core pass: compare the new labels with the previous ones (coalesced: a warp
// reads 32 consecutive (point, candidate) pairs), count the changes, move each changed point
// between the fixed-point sums of its old and new cluster (lanes over coordinates), and keep
// the new labels.  Inactive candidates were not reassigned and are skipped.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_apply_changes(CandBatch b, const T* __restrict__ Z, int64_t n, int d,
                                                       KmState st, int pass) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long act = 0;   // candidates reassigned in this pass
    for (int c = 0; c < b.n; ++c)
        if (st.active[c]) act |= 1ull << c;
    // changes per candidate, counted in shared memory and added to the global counter once per
    // block (one global atomic per warp would serialise every warp on the same few words)
    __shared__ int s_changed[MAXC];
    for (int c = threadIdx.x; c < MAXC; c += blockDim.x) s_changed[c] = 0;
    __syncthreads();
    // thread per point; its label row (cs int16 = whole 16-byte vectors) is read once
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        for (int g0 = 0; g0 < b.n; g0 += 8) {
            uint4 nv = make_uint4(0, 0, 0, 0), ov = make_uint4(0, 0, 0, 0);
            if (valid) {
                nv = *reinterpret_cast<const uint4*>(st.labels_new + i * b.cs + g0);
                ov = *reinterpret_cast<const uint4*>(st.labels + i * b.cs + g0);
            }
            const uint32_t nw[4] = {nv.x, nv.y, nv.z, nv.w}, ow[4] = {ov.x, ov.y, ov.z, ov.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int c = g0 + h;
                const int nl = (int16_t)(nw[h >> 1] >> (16 * (h & 1)));
                const int ol = (int16_t)(ow[h >> 1] >> (16 * (h & 1)));
                const bool ch = valid && c < b.n && ((act >> c) & 1ull) && nl != ol;
                if (ch) {
                    st.labels[i * b.cs + c] = (int16_t)nl;
                    atomicAdd(st.counts + b.off[c] + nl, 1);
                    if (ol >= 0) atomicSub(st.counts + b.off[c] + ol, 1);
                }
                unsigned mask = __ballot_sync(0xffffffffu, ch);
                if (lane == 0 && mask) atomicAdd(&s_changed[c], __popc(mask));
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int64_t pi = __shfl_sync(0xffffffffu, i, src);
                    const int pn = __shfl_sync(0xffffffffu, nl, src);
                    const int po = __shfl_sync(0xffffffffu, ol, src);
                    const int off = b.off[c];
                    for (int k = lane; k < d; k += 32) {
                        const long long v = __float2ll_rn(zval(Z, pi * d + k) * FIXED_SCALE_F);
                        atomicAdd(reinterpret_cast<unsigned long long*>(st.sums + (int64_t)(off + pn) * d + k),
                                  (unsigned long long)v);
                        if (po >= 0)
                            atomicAdd(reinterpret_cast<unsigned long long*>(st.sums + (int64_t)(off + po) * d + k),
                                      (unsigned long long)(-v));
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < b.n; c += blockDim.x)
        if (s_changed[c]) atomicAdd(st.changed + (pass & 1) * MAXC + c, s_changed[c]);
}

void launch_apply_changes(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, KmState st, int pass,
                          cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    ProfScope ps(s, pass == 1 ? PF_APPLY_FIRST : PF_APPLY, 1);
    if (zdtype == RAFTGP_BF16)
        k_apply_changes<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(b, (const __nv_bfloat16*)Z, n, d, st, pass);
    else
        k_apply_changes<float><<<(unsigned)blocks, 256, 0, s>>>(b, (const float*)Z, n, d, st, pass);
}

// ------------------------------------------------------------------------------------
// After a pass: a candidate with no label change is converged (inactive); otherwise its
// centroids become the FP64 means of the fixed-point sums (empty clusters keep theirs).
// ------------------------------------------------------------------------------------
__global__ void k_lloyd_update(CandBatch b, int d, KmState st, int pass, int last_pass) {
    const int c = blockIdx.y;
    if (c >= b.n || !st.active[c]) return;
    const int changed = st.changed[(pass & 1) * MAXC + c];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st.passes[c] = pass;
        st.changed[((pass + 1) & 1) * MAXC + c] = 0;
    }
    if (changed == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st.active[c] = 0;
        return;
    }
    // after the last allowed pass the centroids stay those the final labels were assigned against
    if (pass >= last_pass) return;
    const int K = b.k[c], off = b.off[c];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < K; j += gridDim.x * wpb) {
        const int cnt = st.counts[off + j];
        if (cnt <= 0) continue;
        const double inv = 1.0 / ((double)cnt * FIXED_SCALE);
        for (int k = lane; k < d; k += 32)
            st.mu[(int64_t)(off + j) * d + k] = (float)((double)st.sums[(int64_t)(off + j) * d + k] * inv);
        __syncwarp();
        warp_row_operands(st, off + j, d);
    }
}

void launch_lloyd_update(const CandBatch& b, int d, KmState st, int pass, int last_pass, cudaStream_t s) {
    dim3 grid(64, b.n);
    ProfScope ps(s, PF_LLOYD_UPDATE, 1);
    k_lloyd_update<<<grid, 256, 0, s>>>(b, d, st, pass, last_pass);
}

}  // namespace raftgp
