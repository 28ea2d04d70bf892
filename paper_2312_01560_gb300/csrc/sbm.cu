// sbm.cu -- Algorithm 2 (Section IV): graphs drawn from the degree-corrected SBM of
// Definition 1, A_ij ~ Pois(lambda_ij), lambda_ij = theta_i theta_j Omega_{c_i c_j}, and
// the device CSR build of the drawn graph.
//
// The virtual table of each block pair r <= s (row-major over the blocks' nodes in ascending
// order; for r = s only the entries above the diagonal) is cut into segments of 2^16
// consecutive entries, and each segment runs Algorithm 2's loop on its own: draw p, skip to
// the smallest entry t with RangeSum(m, t) > -ln p by binary search over a closed form of the
// prefix mass (block prefix sums of theta), emit it with its weight Pois(lambda | >= 1), and
// continue at t + 1.  The entries are independent, so the cut leaves the distribution
// unchanged; it makes the segments independent work items (one thread each) and fixes which
// draws each uses: draw j of global segment g is Philox4x32-10(seed; g_lo, g_hi, j, "Sbm2").
// The prefix mass is formed with explicitly rounded FP64 operations (no contraction), so
// the same draws give the same graph as a plain sequential evaluation of the same formulas.
//
// Two passes over the segments (count, then emit at the scanned offsets) give the edges in
// the order (pair, segment, draw).  The CSR build counts degrees, scatters both directions
// and sorts every row (bitonic in shared memory), so its result is canonical.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

namespace {

constexpr int64_t SBM_SEG = 65536;
constexpr uint32_t STREAM_SBM = 0x53626d32u;   // "Sbm2"
constexpr double TWO_M53 = 1.0 / 9007199254740992.0;

__device__ __forceinline__ int64_t pair_start(int64_t K, int64_t r) { return r * K - r * (r - 1) / 2; }

// (r, s) of pair p in the order r-major, s >= r.
__device__ __forceinline__ void pair_rs(int64_t K, int64_t p, int& r, int& s) {
    int64_t lo = 0, hi = K - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (pair_start(K, mid) <= p) lo = mid;
        else hi = mid - 1;
    }
    r = (int)lo;
    s = (int)(lo + (p - pair_start(K, lo)));
}

struct SbmPairDev {
    bool tri;
    int64_t nr, ns;
    float inv_ns;         // 1 / ns: the row estimate of a rectangular table (corrected exactly)
    const int32_t* nodes_r;
    const int32_t* nodes_s;
    const double* th_r;
    const double* th_s;
    const double* pre_r;
    const double* pre_s;
    const double* tri_r;
    double tot_s, om;
};

__device__ __forceinline__ int64_t tri_row_start(int64_t n, int64_t a) { return a * n - a * (a + 1) / 2; }

// Row a and column b of linear index t.  Both are exact integers: an FP32 estimate of the row
// (FP64 runs at a small fraction of the FP32 rate here, and the prefix-mass probes that call
// this made the sampler FP64-bound), then exact integer steps to the row that holds t.
__device__ __forceinline__ void table_entry(const SbmPairDev& P, int64_t t, int64_t& a, int64_t& b) {
    if (!P.tri) {
        int64_t r = (int64_t)__fmul_rn((float)t, P.inv_ns);
        if (r < 0) r = 0;
        while (r > 0 && r * P.ns > t) --r;
        while ((r + 1) * P.ns <= t) ++r;
        a = r;
        b = t - r * P.ns;
        return;
    }
    const int64_t n = P.nr;
    const int64_t size = n * (n - 1) / 2;
    if (t >= size) {
        a = n - 1;
        b = n;
        return;
    }
    // row a solves a^2 - (2n - 1) a + 2t = 0; the discriminant in exact unsigned arithmetic
    const uint64_t q = (uint64_t)(2 * n - 1);
    const uint64_t disc = q * q - 8ull * (uint64_t)t;
    int64_t r = (int64_t)__fmul_rn(__fsub_rn((float)q, __fsqrt_rn((float)disc)), 0.5f);
    if (r < 0) r = 0;
    if (r > n - 2) r = n - 2;
    while (r > 0 && tri_row_start(n, r) > t) --r;
    while (r + 1 <= n - 2 && tri_row_start(n, r + 1) <= t) ++r;
    a = r;
    b = r + 1 + (t - tri_row_start(n, r));
}

// Sum of lambda over the table entries before linear index t.
__device__ __forceinline__ double prefix_mass(const SbmPairDev& P, int64_t t) {
    int64_t a, b;
    table_entry(P, t, a, b);
    if (!P.tri) {
        if (a >= P.nr) return __dmul_rn(P.om, __dmul_rn(P.pre_r[P.nr], P.tot_s));
        const double rowpart = __dmul_rn(P.om, __dmul_rn(P.pre_r[a], P.tot_s));
        const double colpart = __dmul_rn(P.om, __dmul_rn(P.th_r[a], P.pre_s[b]));
        return __dadd_rn(rowpart, colpart);
    }
    const double rowpart = __dmul_rn(P.om, P.tri_r[a]);
    const double colpart = __dmul_rn(P.om, __dmul_rn(P.th_r[a], __dsub_rn(P.pre_r[b], P.pre_r[a + 1])));
    return __dadd_rn(rowpart, colpart);
}

__device__ __forceinline__ int pois_ge1(double lam, uint64_t y) {
    const double u = __dmul_rn((double)(y >> 11), TWO_M53);
    double term = __ddiv_rn(lam, expm1(lam));
    double c = term;
    int k = 1;
    while (u >= c && k < (1 << 20)) {
        ++k;
        term = __dmul_rn(term, __ddiv_rn(lam, (double)k));
        c = __dadd_rn(c, term);
    }
    return k;
}

struct SbmDev {
    int64_t n;
    int K;
    uint64_t seed;
    const double* omega;
    const unsigned long long* bincl;   // inclusive block sizes
    const int32_t* nodes;               // nodes grouped by block, ascending inside a block
    const double* th;                   // theta in that order
    const double* pre;                  // per block r: n_r + 1 prefix sums at offset boff_r + r
    const double* tri;
    const unsigned long long* pincl;    // inclusive segment counts per pair
    int64_t npairs;
};

__device__ __forceinline__ int64_t boff(const SbmDev& d, int r) { return r == 0 ? 0 : (int64_t)d.bincl[r - 1]; }

// Grouping: warp per block r collects its nodes in ascending order (ballot compaction).
__global__ void k_sbm_count_blocks(const int32_t* block, const double* theta, int64_t n, int K,
                                   unsigned long long* bcnt, uint32_t* err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = block[i];
        const double t = theta[i];
        if (!(t >= 0.0) || isinf(t)) flag_error(err, DERR_NORM);
        if (c < 0 || c >= K) {
            flag_error(err, DERR_COL_RANGE);
            continue;
        }
        atomicAdd(bcnt + c, 1ull);
    }
}

__global__ void k_sbm_fill(const int32_t* block, const double* theta, int64_t n, int K,
                           const unsigned long long* bincl, int32_t* nodes, double* th) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < K; r += warps) {
        int64_t pos = r == 0 ? 0 : (int64_t)bincl[r - 1];
        for (int64_t base = 0; base < n; base += 1024) {
            int32_t c[32];   // 32 independent loads in flight, then the ballots in order
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int64_t i = base + 32 * k + lane;
                c[k] = i < n ? __ldg(block + i) : -1;
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int64_t i = base + 32 * k + lane;
                const bool mine = c[k] == r;
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (mine) {
                    const int64_t q = pos + __popc(m & ((1u << lane) - 1u));
                    nodes[q] = (int32_t)i;
                    th[q] = theta[i];
                }
                pos += __popc(m);
            }
        }
    }
}

// Per block, a warp each, left to right: Pre_r[k] = sum_{q<k} theta, and
// Tri_r[a] = sum_{a'<a} theta_a' (Tot_r - Pre_r[a'+1]).  The lanes load (or form) 32 terms at
// a time into shared memory; lane 0 alone adds them in order and stores the running sums, so
// the chain of FP64 additions is one lane's (FP64 runs at a small fraction of the FP32 rate
// here) and no term waits on a round trip through global memory.
__global__ void __launch_bounds__(128) k_sbm_prefix(int K, const unsigned long long* __restrict__ bincl,
                                                    const double* __restrict__ th, double* __restrict__ pre,
                                                    double* __restrict__ tri) {
    __shared__ double sv[4][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < K; r += warps) {
        const int64_t o = r == 0 ? 0 : (int64_t)bincl[r - 1];
        const int64_t nr = (int64_t)bincl[r] - o;
        double* P = pre + o + r;
        double* T = tri + o + r;
        double run = 0.0;
        for (int64_t base = 0; base < nr; base += 32) {
            const int cnt = nr - base < 32 ? (int)(nr - base) : 32;
            sv[wl][lane] = lane < cnt ? th[o + base + lane] : 0.0;
            __syncwarp();
            if (lane == 0)
                for (int j = 0; j < cnt; ++j) {
                    run = __dadd_rn(run, sv[wl][j]);
                    P[base + j + 1] = run;
                }
            __syncwarp();
        }
        if (lane == 0) P[0] = 0.0;
        const double tot = __shfl_sync(0xffffffffu, run, 0);
        __syncwarp();
        run = 0.0;
        for (int64_t base = 0; base < nr; base += 32) {
            const int cnt = nr - base < 32 ? (int)(nr - base) : 32;
            sv[wl][lane] = lane < cnt ? __dmul_rn(th[o + base + lane], __dsub_rn(tot, P[base + lane + 1])) : 0.0;
            __syncwarp();
            if (lane == 0)
                for (int j = 0; j < cnt; ++j) {
                    run = __dadd_rn(run, sv[wl][j]);
                    T[base + j + 1] = run;
                }
            __syncwarp();
        }
        if (lane == 0) T[0] = 0.0;
    }
}

__device__ __forceinline__ int64_t table_size(bool tri, int64_t nr, int64_t ns) {
    return tri ? nr * (nr - 1) / 2 : nr * ns;
}

__global__ void k_sbm_pair_segs(SbmDev d, unsigned long long* pseg, uint32_t* err) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < d.npairs; p += (int64_t)gridDim.x * blockDim.x) {
        int r, s;
        pair_rs(d.K, p, r, s);
        const double om = d.omega[(int64_t)r * d.K + s];
        if (!(om >= 0.0) || isinf(om)) flag_error(err, DERR_NORM);
        const int64_t nr = (int64_t)d.bincl[r] - boff(d, r), ns = (int64_t)d.bincl[s] - boff(d, s);
        const int64_t size = table_size(r == s, nr, ns);
        pseg[p] = (unsigned long long)((size + SBM_SEG - 1) / SBM_SEG);
    }
}

// Segment g: its block pair's table and its entry range [t0, t1).
__device__ __forceinline__ void seg_setup(const SbmDev& d, int64_t g, SbmPairDev& P, int64_t& t0, int64_t& t1) {
    // pair of segment g: the first p with pincl[p] > g
    int64_t lo = 0, hi = d.npairs - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (d.pincl[mid] > (unsigned long long)g) hi = mid;
        else lo = mid + 1;
    }
    const int64_t p = lo;
    const int64_t sg = g - (p == 0 ? 0 : (int64_t)d.pincl[p - 1]);
    int r, s;
    pair_rs(d.K, p, r, s);
    P.tri = r == s;
    const int64_t orr = boff(d, r), os = boff(d, s);
    P.nr = (int64_t)d.bincl[r] - orr;
    P.ns = (int64_t)d.bincl[s] - os;
    P.nodes_r = d.nodes + orr;
    P.nodes_s = d.nodes + os;
    P.th_r = d.th + orr;
    P.th_s = d.th + os;
    P.pre_r = d.pre + orr + r;
    P.pre_s = d.pre + os + s;
    P.tri_r = d.tri + orr + r;
    P.tot_s = P.pre_s[P.ns];
    P.inv_ns = P.ns > 0 ? __frcp_rn((float)P.ns) : 0.f;
    P.om = d.omega[(int64_t)r * d.K + s];
    const int64_t size = table_size(P.tri, P.nr, P.ns);
    t0 = sg * SBM_SEG;
    t1 = t0 + SBM_SEG < size ? t0 + SBM_SEG : size;
}

// Work order of the segments: grouped by their expected number of draws (the lambda mass of
// their entries, on a log scale in SBM_BUCKETS buckets), so that the 32 segments of a warp run
// loops of similar length.  Which thread runs a segment changes nothing in its draws or in
// where its edges go.
constexpr int SBM_BUCKETS = 32;
// Buckets from here on (about 255 expected draws and more) run a warp per segment.
constexpr int SBM_HEAVY = 16;
__device__ __forceinline__ int seg_bucket(double w) {
    if (!(w > 0.0)) return 0;                       // zero (and NaN: never sampled, flagged before)
    if (!(w < 1.0e9)) return SBM_BUCKETS - 1;       // huge or infinite
    const int b = (int)floor(2.0 * log2(1.0 + w));
    return b < SBM_BUCKETS - 1 ? b : SBM_BUCKETS - 1;
}

// Pass 1: each segment's bucket, and the buckets' sizes (block histograms added once per block).
__global__ void __launch_bounds__(256) k_sbm_seg_bucket(SbmDev d, int64_t G, uint8_t* key, unsigned long long* bcount) {
    __shared__ unsigned int h[SBM_BUCKETS];
    for (int b = threadIdx.x; b < SBM_BUCKETS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
        SbmPairDev P;
        int64_t t0, t1;
        seg_setup(d, g, P, t0, t1);
        const int b = seg_bucket(__dsub_rn(prefix_mass(P, t1), prefix_mass(P, t0)));
        key[g] = (uint8_t)b;
        atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < SBM_BUCKETS; b += blockDim.x)
        if (h[b]) atomicAdd(bcount + b, (unsigned long long)h[b]);
}

// The buckets' starts (exclusive scan, one thread) and their fill cursors.
__global__ void k_sbm_seg_starts(const unsigned long long* bcount, unsigned long long* cursor) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (int b = 0; b < SBM_BUCKETS; ++b) {
        cursor[b] = run;
        run += bcount[b];
    }
}

// Pass 2: each block reserves its segments' places bucket by bucket (one global atomic per
// bucket and block) and writes them there.
__global__ void __launch_bounds__(256) k_sbm_seg_scatter(int64_t G, const uint8_t* key, unsigned long long* cursor,
                                                         uint32_t* order) {
    __shared__ unsigned int h[SBM_BUCKETS];
    __shared__ unsigned long long base[SBM_BUCKETS];
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < G; g0 += (int64_t)gridDim.x * blockDim.x) {
        for (int b = threadIdx.x; b < SBM_BUCKETS; b += blockDim.x) h[b] = 0;
        __syncthreads();
        const int64_t g = g0 + threadIdx.x;
        const int b = g < G ? (int)key[g] : -1;
        unsigned int rank = 0;
        if (b >= 0) rank = atomicAdd(&h[b], 1u);
        __syncthreads();
        for (int q = threadIdx.x; q < SBM_BUCKETS; q += blockDim.x)
            base[q] = h[q] ? atomicAdd(cursor + q, (unsigned long long)h[q]) : 0ull;
        __syncthreads();
        if (b >= 0) order[base[b] + rank] = (uint32_t)g;
        __syncthreads();
    }
}

// One thread per global segment: Algorithm 2's loop on the segment.  The segments are taken
// from `order` positions [0, *split) (all G without an order), heaviest bucket first.  COUNT
// mode stores the number of edges; EMIT mode writes them at the segment's offset.
template <bool EMIT>
__global__ void __launch_bounds__(128) k_sbm_segments(SbmDev d, int64_t G, const uint32_t* order,
                                                      const unsigned long long* split, unsigned long long* seg_cnt,
                                                      const unsigned long long* seg_incl, int32_t* src, int32_t* dst,
                                                      int32_t* weight) {
    const int64_t end = split ? (int64_t)*split : G;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < end; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = end - 1 - k;
        const int64_t g = order ? (int64_t)order[idx] : idx;
        SbmPairDev P;
        int64_t t0, t1;
        seg_setup(d, g, P, t0, t1);
        const double Fend = prefix_mass(P, t1);
        int64_t out = EMIT ? (int64_t)seg_incl[g] - (int64_t)seg_cnt[g] : 0;
        const int64_t cap = EMIT ? (int64_t)seg_cnt[g] : 0;   // the count pass's edges of this segment
        int64_t count = 0;
        int64_t m = t0;
        uint32_t j = 0;
        while (m < t1) {
            const U32x4 x = philox4x32_10((uint32_t)g, (uint32_t)((uint64_t)g >> 32), j, STREAM_SBM, d.seed);
            ++j;
            const uint64_t w01 = (uint64_t)x.x | ((uint64_t)x.y << 32);
            const uint64_t w23 = (uint64_t)x.z | ((uint64_t)x.w << 32);
            const double pu = __dmul_rn((double)((w01 >> 11) + 1), TWO_M53);
            const double V = __dadd_rn(prefix_mass(P, m), -log(pu));
            if (!(Fend > V)) break;
            int64_t a0 = m, a1 = t1 - 1;
            while (a0 < a1) {
                const int64_t mid = a0 + (a1 - a0) / 2;
                if (prefix_mass(P, mid + 1) > V) a1 = mid;
                else a0 = mid + 1;
            }
            if (EMIT && count < cap) {
                int64_t a, b;
                table_entry(P, a0, a, b);
                src[out] = P.nodes_r[a];
                dst[out] = P.nodes_s[b];
                if (weight) weight[out] = pois_ge1(__dmul_rn(P.om, __dmul_rn(P.th_r[a], P.th_s[b])), w23);
                ++out;
            }
            ++count;
            m = a0 + 1;
        }
        if (!EMIT) seg_cnt[g] = (unsigned long long)count;
    }
}

// The binary search of Algorithm 2's skip (the first entry a in [a0, a1] with F(a + 1) > V),
// five levels per round: lane L < 31 evaluates node L + 1 of the next five levels' decision
// tree (heap order; node h's children are 2h, taken when the probe is true, and 2h + 1) at the
// range the one-thread search would hold there, then the warp follows the actual outcomes.  It
// reaches the same entry as the one-thread search through the same probes, so the result does
// not depend on F being monotone in its rounding.
__device__ __forceinline__ void warp_skip_search(const SbmPairDev& P, double V, int64_t& a0, int64_t& a1, int lane) {
    while (a0 < a1) {
        const int h = lane + 1;
        const int depth = 31 - __clz(h);
        int64_t lo = a0, hi = a1;
        bool live = lane < 31;
        for (int dd = depth - 1; dd >= 0 && live; --dd) {
            if (lo >= hi) {
                live = false;
                break;
            }
            const int64_t mid = lo + (hi - lo) / 2;
            if (((h >> dd) & 1) == 0) hi = mid;
            else lo = mid + 1;
        }
        bool pr = false;
        if (live && lo < hi) pr = prefix_mass(P, lo + (hi - lo) / 2 + 1) > V;
        const unsigned res = __ballot_sync(0xffffffffu, pr);
        int node = 1;
        for (int step = 0; step < 5 && a0 < a1; ++step) {
            const int64_t mid = a0 + (a1 - a0) / 2;
            if ((res >> (node - 1)) & 1u) {
                a1 = mid;
                node = 2 * node;
            } else {
                a0 = mid + 1;
                node = 2 * node + 1;
            }
        }
    }
}

// A warp per segment for order positions [*split, G), the heaviest buckets (a segment there
// holds hundreds to thousands of edges, and one thread's chain of dependent probes through the
// heaviest set the length of the whole pass), heaviest first.  Every lane draws the same
// numbers; lane 0 writes.
template <bool EMIT>
__global__ void __launch_bounds__(256) k_sbm_segments_warp(SbmDev d, int64_t G, const uint32_t* __restrict__ order,
                                                           const unsigned long long* __restrict__ split,
                                                           unsigned long long* seg_cnt,
                                                           const unsigned long long* seg_incl, int32_t* src,
                                                           int32_t* dst, int32_t* weight) {
    const int lane = threadIdx.x & 31;
    const int64_t begin = (int64_t)*split;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; begin + k < G; k += nw) {
        const int64_t g = (int64_t)order[G - 1 - k];
        SbmPairDev P;
        int64_t t0, t1;
        seg_setup(d, g, P, t0, t1);
        const double Fend = prefix_mass(P, t1);
        int64_t out = EMIT ? (int64_t)seg_incl[g] - (int64_t)seg_cnt[g] : 0;
        const int64_t cap = EMIT ? (int64_t)seg_cnt[g] : 0;
        int64_t count = 0;
        int64_t m = t0;
        uint32_t j = 0;
        while (m < t1) {
            // the draw and its target mass by lane 0 alone, then shared with the warp
            double V = 0.0;
            uint64_t w23 = 0;
            if (lane == 0) {
                const U32x4 x = philox4x32_10((uint32_t)g, (uint32_t)((uint64_t)g >> 32), j, STREAM_SBM, d.seed);
                const uint64_t w01 = (uint64_t)x.x | ((uint64_t)x.y << 32);
                w23 = (uint64_t)x.z | ((uint64_t)x.w << 32);
                const double pu = __dmul_rn((double)((w01 >> 11) + 1), TWO_M53);
                V = __dadd_rn(prefix_mass(P, m), -log(pu));
            }
            ++j;
            V = __shfl_sync(0xffffffffu, V, 0);
            if (!(Fend > V)) break;
            int64_t a0 = m, a1 = t1 - 1;
            warp_skip_search(P, V, a0, a1, lane);
            if (EMIT && count < cap && lane == 0) {
                int64_t a, b;
                table_entry(P, a0, a, b);
                src[out] = P.nodes_r[a];
                dst[out] = P.nodes_s[b];
                if (weight) weight[out] = pois_ge1(__dmul_rn(P.om, __dmul_rn(P.th_r[a], P.th_s[b])), w23);
            }
            if (EMIT && count < cap) ++out;
            ++count;
            m = a0 + 1;
        }
        if (!EMIT && lane == 0) seg_cnt[g] = (unsigned long long)count;
    }
}

// ---- CSR build --------------------------------------------------------------------------
__global__ void k_csr_degree(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, unsigned long long* deg,
                             uint32_t* err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) {
            flag_error(err, u == v ? DERR_SELF_LOOP : DERR_COL_RANGE);
            continue;
        }
        atomicAdd(deg + u, 1ull);
        atomicAdd(deg + v, 1ull);
    }
}

__global__ void k_csr_rowptr(const unsigned long long* incl, int64_t n, int64_t* row_ptr, unsigned long long* fill) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i == 0 ? 0 : (int64_t)incl[i - 1];
        row_ptr[i] = v;
        if (i < n) fill[i] = (unsigned long long)v;
    }
}

__global__ void k_csr_scatter(const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                              unsigned long long* fill, int32_t* col) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
        col[atomicAdd(fill + u, 1ull)] = v;
        col[atomicAdd(fill + v, 1ull)] = u;
    }
}

// Bitonic sort of one row in shared memory by `threads` threads (the row padded with INT_MAX
// to the power of two P).
__device__ __forceinline__ void bitonic_row(int32_t* sm, int P, int tid, int threads, bool block_sync) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += threads) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t x = sm[i], y = sm[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        sm[i] = y;
                        sm[l] = x;
                    }
                }
            }
            if (block_sync) __syncthreads();
            else __syncwarp();
        }
    }
}

constexpr int CSR_WARP_MAX = 256;     // rows up to this length: one warp each
constexpr int CSR_BLOCK_MAX = 16384;  // longer rows: one block each, up to this length

__global__ void __launch_bounds__(256) k_csr_sort_short(const int64_t* row_ptr, int64_t n, int32_t* col,
                                                        const uint8_t* only, int* long_rows, int* n_long,
                                                        uint32_t* err) {
    __shared__ int32_t sm[8][CSR_WARP_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        if (only && !only[i]) continue;
        const int64_t b = row_ptr[i], e = row_ptr[i + 1], len = e - b;
        if (len <= 1) continue;
        if (len > CSR_WARP_MAX) {
            if (lane == 0) {
                if (len > CSR_BLOCK_MAX) flag_error(err, DERR_ROW_PTR);
                else long_rows[atomicAdd(n_long, 1)] = (int)i;
            }
            continue;
        }
        int P = 2;
        while (P < len) P <<= 1;
        for (int k = lane; k < P; k += 32) sm[w][k] = k < len ? col[b + k] : 0x7fffffff;
        __syncwarp();
        bitonic_row(sm[w], P, lane, 32, false);
        for (int k = lane; k < len; k += 32) col[b + k] = sm[w][k];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(1024) k_csr_sort_long(const int64_t* row_ptr, int32_t* col, const int* long_rows,
                                                        const int* n_long) {
    extern __shared__ int32_t smem_rows[];
    for (int q = blockIdx.x; q < *n_long; q += gridDim.x) {
        const int64_t i = long_rows[q];
        const int64_t b = row_ptr[i], len = row_ptr[i + 1] - b;
        int P = 2;
        while (P < len) P <<= 1;
        for (int k = threadIdx.x; k < P; k += blockDim.x) smem_rows[k] = k < len ? col[b + k] : 0x7fffffff;
        __syncthreads();
        bitonic_row(smem_rows, P, threadIdx.x, blockDim.x, true);
        for (int k = threadIdx.x; k < len; k += blockDim.x) col[b + k] = smem_rows[k];
        __syncthreads();
    }
}

}  // namespace

int grid_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// One resident wave of the warp-per-segment kernel (its CTAs per SM from the occupancy API).
template <bool EMIT>
int sbm_warp_grid() {
    static int per_sm = 0;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sbm_segments_warp<EMIT>, 256, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    return num_sms() * per_sm;
}

// ---- workspace ---------------------------------------------------------------------------
int64_t sbm_max_segments(int64_t n, int K) {
    const int64_t npairs = (int64_t)K * (K + 1) / 2;
    return n * (n - 1) / 2 / SBM_SEG + npairs + 1;
}

SbmWs carve_sbm(Carver& c, int64_t n, int K) {
    SbmWs w{};
    const int64_t npairs = (int64_t)K * (K + 1) / 2;
    const int64_t G = sbm_max_segments(n, K);
    const int64_t most = std::max<int64_t>(std::max<int64_t>(n, npairs), std::max<int64_t>(G, K));
    w.err = c.take<uint32_t>(64);
    w.bcnt = c.take<unsigned long long>(K);
    w.bincl = c.take<unsigned long long>(K);
    w.nodes = c.take<int32_t>(n + 1);
    w.th = c.take<double>(n + 1);
    w.pre = c.take<double>(n + K);
    w.tri = c.take<double>(n + K);
    w.pseg = c.take<unsigned long long>(npairs);
    w.pincl = c.take<unsigned long long>(npairs);
    w.seg_cnt = c.take<unsigned long long>(G);
    w.seg_incl = c.take<unsigned long long>(G);
    w.seg_order = c.take<uint32_t>(G);
    w.seg_key = c.take<uint8_t>(G);
    w.bucket = c.take<unsigned long long>(2 * SBM_BUCKETS);
    w.tiles = c.take<unsigned long long>((most + SCAN_TILE - 1) / SCAN_TILE + 1);
    return w;
}

// Count pass: groups the blocks, builds the prefix sums and the segment table, counts every
// segment's edges and scans them.  Returns the number of segments and of edges (host).
cudaError_t sbm_count(const raftgp_sbm* p, const SbmWs& w, int64_t* G_out, int64_t* m_out, cudaStream_t s) {
    const int64_t n = p->n;
    const int K = p->k;
    const int64_t npairs = (int64_t)K * (K + 1) / 2;
    ProfScope ps(s, PF_OTHER, 7);
    cudaMemsetAsync(w.err, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(w.bcnt, 0, sizeof(unsigned long long) * K, s);
    k_sbm_count_blocks<<<grid_for(n, 256), 256, 0, s>>>(p->block, p->theta, n, K, w.bcnt, w.err);
    scan_incl(w.bcnt, K, w.bincl, w.tiles, s);
    k_sbm_fill<<<grid_for((int64_t)K * 32, 256), 256, 0, s>>>(p->block, p->theta, n, K, w.bincl, w.nodes, w.th);
    k_sbm_prefix<<<grid_for((int64_t)K * 32, 128), 128, 0, s>>>(K, w.bincl, w.th, w.pre, w.tri);
    SbmDev d{n, K, p->seed, p->omega, w.bincl, w.nodes, w.th, w.pre, w.tri, w.pincl, npairs};
    k_sbm_pair_segs<<<grid_for(npairs, 256), 256, 0, s>>>(d, w.pseg, w.err);
    scan_incl(w.pseg, npairs, w.pincl, w.tiles, s);
    unsigned long long G = 0;
    uint32_t herr = 0;
    cudaMemcpyAsync(&G, w.pincl + (npairs - 1), sizeof(G), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&herr, w.err, sizeof(herr), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (herr) return cudaErrorInvalidValue;
    if ((int64_t)G > sbm_max_segments(n, K)) return cudaErrorInvalidValue;
    if (G > 0) {
        // segment indices in the work order fit 32 bits up to 2^32 segments; beyond, the
        // segments run in index order
        const uint32_t* order = G < (1ull << 32) ? w.seg_order : nullptr;
        if (order) {
            cudaMemsetAsync(w.bucket, 0, sizeof(unsigned long long) * SBM_BUCKETS, s);
            k_sbm_seg_bucket<<<grid_for((int64_t)G, 256), 256, 0, s>>>(d, (int64_t)G, w.seg_key, w.bucket);
            k_sbm_seg_starts<<<1, 32, 0, s>>>(w.bucket, w.bucket + SBM_BUCKETS);
            k_sbm_seg_scatter<<<grid_for((int64_t)G, 256), 256, 0, s>>>((int64_t)G, w.seg_key, w.bucket + SBM_BUCKETS,
                                                                         w.seg_order);
        }
        const unsigned long long* split = order ? w.bucket + SBM_BUCKETS + (SBM_HEAVY - 1) : nullptr;
        k_sbm_segments<false><<<grid_for((int64_t)G, 128), 128, 0, s>>>(d, (int64_t)G, order, split, w.seg_cnt,
                                                                         nullptr, nullptr, nullptr, nullptr);
        if (order)
            k_sbm_segments_warp<false><<<sbm_warp_grid<false>(), 256, 0, s>>>(d, (int64_t)G, order, split, w.seg_cnt,
                                                                               nullptr, nullptr, nullptr, nullptr);
        scan_incl(w.seg_cnt, (int64_t)G, w.seg_incl, w.tiles, s);
    }
    unsigned long long m = 0;
    if (G > 0) cudaMemcpyAsync(&m, w.seg_incl + (G - 1), sizeof(m), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *G_out = (int64_t)G;
    *m_out = (int64_t)m;
    return cudaSuccess;
}

cudaError_t sbm_emit(const raftgp_sbm* p, const SbmWs& w, int64_t G, int32_t* src, int32_t* dst, int32_t* weight,
                     cudaStream_t s) {
    const int K = p->k;
    const int64_t npairs = (int64_t)K * (K + 1) / 2;
    if (G <= 0) return cudaSuccess;
    SbmDev d{p->n, K, p->seed, p->omega, w.bincl, w.nodes, w.th, w.pre, w.tri, w.pincl, npairs};
    ProfScope ps(s, PF_OTHER, 1);
    const uint32_t* order = (unsigned long long)G < (1ull << 32) ? w.seg_order : nullptr;
    const unsigned long long* split = order ? w.bucket + SBM_BUCKETS + (SBM_HEAVY - 1) : nullptr;
    k_sbm_segments<true><<<grid_for(G, 128), 128, 0, s>>>(d, G, order, split, w.seg_cnt, w.seg_incl, src, dst, weight);
    if (order)
        k_sbm_segments_warp<true><<<sbm_warp_grid<true>(), 256, 0, s>>>(d, G, order, split, w.seg_cnt, w.seg_incl, src,
                                                                         dst, weight);
    return cudaGetLastError();
}

// ---- CSR rows sorted in place --------------------------------------------------------------
cudaError_t sort_csr_rows(const int64_t* row_ptr, int64_t n, int32_t* col, const uint8_t* only, int* long_rows,
                          int* n_long, uint32_t* err, cudaStream_t s) {
    cudaMemsetAsync(n_long, 0, sizeof(int), s);
    k_csr_sort_short<<<grid_for(n * 32, 256), 256, 0, s>>>(row_ptr, n, col, only, long_rows, n_long, err);
    const size_t smem = CSR_BLOCK_MAX * sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_csr_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_csr_sort_long<<<num_sms() * 2, 1024, smem, s>>>(row_ptr, col, long_rows, n_long);
    return cudaGetLastError();
}

// ---- CSR of the drawn graph ---------------------------------------------------------------
CsrBuildWs carve_csr_build(Carver& c, int64_t n) {
    CsrBuildWs w{};
    w.err = c.take<uint32_t>(64);
    w.deg = c.take<unsigned long long>(n + 1);
    w.incl = c.take<unsigned long long>(n + 1);
    w.fill = c.take<unsigned long long>(n + 1);
    w.tiles = c.take<unsigned long long>((n + SCAN_TILE - 1) / SCAN_TILE + 1);
    w.long_rows = c.take<int>(n + 1);
    w.n_long = c.take<int>(64);
    return w;
}

cudaError_t coo_to_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* row_ptr, int32_t* col,
                       const CsrBuildWs& w, uint32_t* herr, cudaStream_t s) {
    ProfScope ps(s, PF_OTHER, 6);
    cudaMemsetAsync(w.err, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(w.n_long, 0, sizeof(int), s);
    cudaMemsetAsync(w.deg, 0, sizeof(unsigned long long) * (n + 1), s);
    if (m > 0) k_csr_degree<<<grid_for(m, 256), 256, 0, s>>>(src, dst, m, n, w.deg, w.err);
    if (n > 0) scan_incl(w.deg, n, w.incl, w.tiles, s);
    k_csr_rowptr<<<grid_for(n + 1, 256), 256, 0, s>>>(w.incl, n, row_ptr, w.fill);
    if (m > 0) k_csr_scatter<<<grid_for(m, 256), 256, 0, s>>>(src, dst, m, n, w.fill, col);
    if (n > 0) {
        cudaError_t e = sort_csr_rows(row_ptr, n, col, nullptr, w.long_rows, w.n_long, w.err, s);
        if (e != cudaSuccess) return e;
    }
    cudaMemcpyAsync(herr, w.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    return cudaStreamSynchronize(s);
}

}  // namespace raftgp
