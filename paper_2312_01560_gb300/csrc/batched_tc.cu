// batched_tc.cu -- the batched form's Lloyd k-means on the 5th-generation tensor cores.
//
// Persistent CTAs (two per SM) taking (graph, candidate K) work items from a queue, as the FP32
// batched kernel, but each assignment pass is a tcgen05 GEMM of the graph's points against its
// K <= 128 centroids:
//   - the centroid operand (BF16 split of -mu into hi and lo, and the K=16 norm slice
//     [(||mu||^2 + 4)/2 hi, lo, 128, 0...] of the tensor-core k-means) is rebuilt from the FP32
//     centroids in shared memory at the start of every pass, written to this CTA's rows of a
//     global staging area and brought into shared memory by TMA (which applies the operand
//     swizzle);
//   - warp 0 loads the graph's 128-point tiles by TMA into two buffers, warp 1 issues the MMAs
//     (M = 128, N = K rounded up to 32, K = 16 steps) into two 128-column tensor-memory
//     accumulators, warps 2-5 read them back (thread = point) and take the argmin;
//   - Lloyd passes multiply the hi half only plus the norm slice, so the accumulator is
//     128 + (||z - mu||^2 - ||z||^2 + 4) / 2 and the integer-key argmin of the single-graph
//     engine applies (ties to the lowest column); a changed label moves the point's 2^-40
//     fixed-point row between the clusters' sums (this CTA's slice of a global area, 64-bit
//     reductions in L2);
//   - the final assignment multiplies hi + lo, keeps the exact best and second-best FP32
//     scores and re-checks every point whose two best lie within the derived band in the FP32
//     direct form over all K centroids, so every reported label is the FP32-nearest centroid;
//   - means in FP64 from the fixed-point sums, norms in the single-graph engine's order, empty
//     clusters keep their centroid, the pass cap and the stop rule as there; then the
//     partition's exact integer score.
// Every mbarrier wait is bounded: on timeout the CTA records DERR_TIMEOUT, stops issuing, lets
// its copies and MMAs drain (bounded), frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "batch_score.cuh"
#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace raftgp {

constexpr int BTC_ROWS = 128;         // centroid rows of the operand (BATCH_KMAX)
constexpr int BTC_THREADS = 192;      // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
// Two CTAs per SM (2 x 256 tensor-memory columns; shared memory 62 KB at d = 32, 107 KB at
// d = 64): an item's passes are a chain of dependent steps on few tiles, so a second item on
// the SM fills the gaps.
constexpr int BTC_MAX_CTAS_PER_SM = 2;
static_assert(BTC_ROWS == BATCH_KMAX, "one operand row per possible centroid");

template <int D>
struct BtcCfg {
    static constexpr int ATOM = D < 64 ? D : 64;           // K elements per swizzle-atom row
    static constexpr int ATOM_BYTES = ATOM * 2;            // 64 or 128
    static constexpr int NATOM = D / ATOM;                 // 1 for D <= 64
    static constexpr int TILE = 128 * ATOM_BYTES * NATOM;  // a 128-row operand tile (A or one B half)
    static constexpr int AUG = 128 * 32;                   // a 128-row K=16 slice
    static constexpr int LAYOUT = ATOM_BYTES == 128 ? 2 : 4;   // 128B or 64B swizzle
    static constexpr int SBO = 8 * ATOM_BYTES;
    // dynamic shared memory, 1024-aligned regions
    static constexpr int OFF_A = 0;                        // two point tiles
    static constexpr int OFF_AUGA = OFF_A + 2 * TILE;      // the constant slice of a point tile
    static constexpr int OFF_BHI = OFF_AUGA + AUG;
    static constexpr int OFF_BLO = OFF_BHI + TILE;
    static constexpr int OFF_BAUG = OFF_BLO + TILE;
    static constexpr int OFF_MU = OFF_BAUG + AUG;          // FP32 centroids, 128 x D
    static constexpr int OFF_NRM = OFF_MU + 128 * D * 4;   // ||mu||^2 + 4 (infinite on padding rows)
    static constexpr int OFF_SCORE = OFF_NRM + 128 * 4;    // the scorer's 2 x 128 counters (u64)
    static constexpr int OFF_CNT = OFF_SCORE + 2 * 128 * 8;
    static constexpr int BYTES = OFF_CNT + 128 * 4;
    static constexpr int SMEM = BYTES + 1024;              // + alignment slack
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

struct BtcCtl {
    uint64_t a_full[2], a_empty[2], acc_full[2], acc_empty[2], b_full, drain;
    uint32_t tmem_base;
    int abort;
    int item, changed;
    int epi_abort;           // an epilogue wait gave up (read by all epilogue threads after a barrier)
    int nchg[2];             // label changes of the tile being applied (two lists, by tile parity)
    int4 chg[2][128];        // (point, old label, new label)
};

// Coordinate k of row r of a point tile as TMA wrote it into shared memory: 16-byte chunk c of
// the row sits at chunk c ^ (r & 7) (128-byte rows, 128B swizzle, D = 64) or c ^ ((r >> 1) & 3)
// (64-byte rows, 64B swizzle, D = 32).
template <int D>
__device__ __forceinline__ float tile_coord(const uint8_t* tile, int r, int k) {
    constexpr int RB = D * 2;
    const int c = k >> 3;
    const int pc = RB == 128 ? (c ^ (r & 7)) : (c ^ ((r >> 1) & 3));
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tile + r * RB + pc * 16 + (k & 7) * 2));
}

// Barrier of the 128 epilogue threads (warps 2-5) only.
__device__ __forceinline__ void btc_epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

struct BtcArgs {
    BatchDev b;
    const __nv_bfloat16* Z;
    int phase, iters, lo_fast;
    const int64_t* rp64;
    const int32_t* rp32;
    const int32_t* col;
    __nv_bfloat16* stg_hi;    // gridDim.x x 128 x D
    __nv_bfloat16* stg_lo;
    __nv_bfloat16* stg_aug;   // gridDim.x x 128 x 16
    long long* gsums;         // gridDim.x x 128 x D: each CTA's 2^-40 fixed-point centroid sums
    float band;               // near-tie band of the final assignment (tc_tie_band(D))
    uint32_t* err;
};

__device__ __forceinline__ void btc_split(float v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *hi = h;
    *lo = __float2bfloat16_rn(v - __bfloat162float(h));
}

// The operand rows of this pass from the FP32 centroids in shared memory (every thread of the
// CTA): row c < K gets the BF16 split of -mu_c and its norm slice, rows K..127 are padding
// (zero operand, slice [127, 0, 128]: score 255, above every real one; infinite norm).  Norms
// as the single-graph engine forms them: before the first update with sequential fused
// multiply-adds over ascending coordinates, afterwards lane-strided then a warp sum.
template <int D>
__device__ void btc_build(const BtcArgs& a, const float* mu, float* nrm4, int K, bool seq_norm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = BTC_THREADS / 32;
    __nv_bfloat16* hi = a.stg_hi + (size_t)blockIdx.x * 128 * D;
    __nv_bfloat16* lo = a.stg_lo + (size_t)blockIdx.x * 128 * D;
    __nv_bfloat16* aug = a.stg_aug + (size_t)blockIdx.x * 128 * 16;
    for (int c = warp; c < 128; c += NW) {
        if (c >= K) {
            for (int k = lane; k < D; k += 32) {
                hi[c * D + k] = __float2bfloat16_rn(0.f);
                lo[c * D + k] = __float2bfloat16_rn(0.f);
            }
            if (lane < 16)
                aug[c * 16 + lane] = __float2bfloat16_rn(lane == 0 ? 127.0f : lane == 2 ? 128.0f : 0.0f);
            if (lane == 0) nrm4[c] = INFINITY;
            continue;
        }
        float s = 0.f;
        if (seq_norm) {
            if (lane == 0)
                for (int k = 0; k < D; ++k) s = fmaf(mu[c * D + k], mu[c * D + k], s);
            s = __shfl_sync(0xffffffffu, s, 0);
        } else {
            for (int k = lane; k < D; k += 32) s = fmaf(mu[c * D + k], mu[c * D + k], s);
            s = warp_sum(s);
        }
        for (int k = lane; k < D; k += 32) btc_split(-mu[c * D + k], hi + c * D + k, lo + c * D + k);
        if (lane < 16) {
            const float half = 0.5f * (s + 4.0f);
            const __nv_bfloat16 h = __float2bfloat16_rn(half);
            aug[c * 16 + lane] = lane == 0 ? h
                               : lane == 1 ? __float2bfloat16_rn(half - __bfloat162float(h))
                               : lane == 2 ? __float2bfloat16_rn(128.0f)
                                           : __float2bfloat16_rn(0.f);
        }
        if (lane == 0) nrm4[c] = s + 4.0f;
    }
    // the rows are read next by TMA (the async proxy)
    asm volatile("fence.proxy.async;" ::: "memory");
}

template <int D>
__global__ void __launch_bounds__(BTC_THREADS, BTC_MAX_CTAS_PER_SM)
    k_batch_lloyd_tc(const __grid_constant__ BtcArgs a, const __grid_constant__ CUtensorMap tmZ,
                     const __grid_constant__ CUtensorMap tmHi, const __grid_constant__ CUtensorMap tmLo,
                     const __grid_constant__ CUtensorMap tmAug) {
    using C = BtcCfg<D>;
    static_assert(C::NATOM == 1, "rows of at most 64 BF16 values (d = 32 or 64)");
    extern __shared__ uint8_t btc_dyn[];
    __shared__ BtcCtl ctl;
    uint8_t* base = (uint8_t*)(((uintptr_t)btc_dyn + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base + C::OFF_A;
    uint8_t* sAugA = base + C::OFF_AUGA;
    uint8_t* sBhi = base + C::OFF_BHI;
    uint8_t* sBlo = base + C::OFF_BLO;
    uint8_t* sBaug = base + C::OFF_BAUG;
    float* mu = reinterpret_cast<float*>(base + C::OFF_MU);
    float* nrm4 = reinterpret_cast<float*>(base + C::OFF_NRM);
    // the centroid sums live in global memory (L2), this CTA's slice: in shared memory they
    // would take 64 KB at d = 64 and leave room for one CTA per SM; updated with 64-bit
    // reductions, read back through L2 (ld.global.cg)
    long long* sums = a.gsums + (size_t)blockIdx.x * 128 * D;
    unsigned long long* score_scratch = reinterpret_cast<unsigned long long*>(base + C::OFF_SCORE);
    int* cnt = reinterpret_cast<int*>(base + C::OFF_CNT);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const BatchDev& b = a.b;

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&ctl.a_full[q], 1);
            mbar_init(&ctl.a_empty[q], 2);   // the tile's MMAs, and the epilogue's change application
            mbar_init(&ctl.acc_full[q], 1);
            mbar_init(&ctl.acc_empty[q], 128);
        }
        mbar_init(&ctl.b_full, 1);
        mbar_init(&ctl.drain, 1);
        ctl.abort = 0;
        ctl.epi_abort = 0;
        ctl.nchg[0] = ctl.nchg[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // constant K=16 slice of a point tile: every row reads 1, 1, 1 at K = 0, 1, 2 (and at 8, 9,
    // 10, so the row is the same under the 32-byte swizzle)
    for (int t = threadIdx.x; t < C::AUG / 16; t += BTC_THREADS)
        reinterpret_cast<uint4*>(sAugA)[t] = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(&ctl.tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem_base;

    // running counts, the same in every role: point tiles through the two A buffers and the
    // two accumulators (n_a) and operand loads (n_b); the last tiles the producer issued
    uint32_t n_a = 0, n_b = 0;
    uint32_t issued_a = 0;
    bool issued_b = false;
    const int per_graph = a.phase == 0 ? BATCH_COARSE : BATCH_SLOTS - BATCH_COARSE;
    for (;;) {
        if (threadIdx.x == 0) ctl.item = atomicAdd(b.queue + 1 + a.phase, 1);
        __syncthreads();
        const int u = ctl.item;
        if (u >= b.ng * per_graph || *(volatile int*)&ctl.abort) break;
        const int g = b.order[u / per_graph];
        const int jj = u % per_graph;
        const int slot = (a.phase == 0 ? 0 : BATCH_COARSE) + jj;
        if (jj >= (a.phase == 0 ? b.n_coarse[g] : b.n_refine[g])) {
            __syncthreads();
            continue;
        }
        const int K = b.cand_k[g * BATCH_SLOTS + slot];
        const int64_t o = b.node_off[g];
        const int64_t n = b.node_off[g + 1] - o;
        int16_t* lab = b.labels + (int64_t)slot * b.total_n + o;
        const int32_t* seeds = b.seeds + b.seed_off[g];
        const int T = (int)((n + 127) / 128);
        const int Np = (K + 31) / 32 * 32;    // MMA N: the real centroids rounded up to 32
        // centroids from the first K seeds (BF16 rows widened), zero sums and counts
        for (int t = threadIdx.x; t < 128 * D; t += BTC_THREADS) {
            const int c = t / D, k = t % D;
            int64_t src = c < K ? (int64_t)seeds[c] : -1;
            if (src >= n) src = -1;   // an aborted seeding leaves -1: such a centroid starts at 0
            mu[t] = src >= 0 ? __bfloat162float(a.Z[(o + src) * D + k]) : 0.f;
            sums[t] = 0;
        }
        for (int t = threadIdx.x; t < 128; t += BTC_THREADS) cnt[t] = 0;
        for (int64_t i = threadIdx.x; i < n; i += BTC_THREADS) lab[i] = -1;
        __syncthreads();
        int passes = a.iters;
        bool fin = false, updated = false;
        for (int pass = 1;; ++pass) {
            btc_build<D>(a, mu, nrm4, K, !updated);
            if (threadIdx.x == 0) ctl.changed = 0;
            __syncthreads();
            const bool use_lo = fin || a.lo_fast;
            if (warp == 0) {
                // ---------------- TMA producer ----------------
                if (lane == 0) {
                    mbar_expect_tx(&ctl.b_full, (uint32_t)((use_lo ? 2 : 1) * C::TILE + C::AUG));
                    tma_load_2d(sBhi, &tmHi, &ctl.b_full, 0, (int)blockIdx.x * 128);
                    if (use_lo) tma_load_2d(sBlo, &tmLo, &ctl.b_full, 0, (int)blockIdx.x * 128);
                    tma_load_2d(sBaug, &tmAug, &ctl.b_full, 0, (int)blockIdx.x * 128);
                    issued_b = true;
                    for (int t = 0; t < T; ++t) {
                        const uint32_t q = n_a + t;
                        const int buf = q & 1;
                        if (!mbar_wait(&ctl.a_empty[buf], ((q >> 1) & 1) ^ 1, &ctl, a.err)) break;
                        mbar_expect_tx(&ctl.a_full[buf], (uint32_t)C::TILE);
                        tma_load_2d(sA + buf * C::TILE, &tmZ, &ctl.a_full[buf], 0, (int)(o + 128 * (int64_t)t));
                        issued_a = q + 1;
                    }
                }
            } else if (warp == 1) {
                // ---------------- MMA issuer ----------------
                if (lane == 0) {
                    const uint32_t idesc = instr_desc(Np);
                    const uint64_t dA = smem_desc(smem_addr(sA), C::LAYOUT, C::SBO);
                    const uint64_t dBhi = smem_desc(smem_addr(sBhi), C::LAYOUT, C::SBO);
                    const uint64_t dBlo = smem_desc(smem_addr(sBlo), C::LAYOUT, C::SBO);
                    const uint64_t dAugA = smem_desc(smem_addr(sAugA), 6, 256);
                    const uint64_t dAugB = smem_desc(smem_addr(sBaug), 6, 256);
                    bool ok = mbar_wait(&ctl.b_full, n_b & 1, &ctl, a.err);
                    tc_fence_after();
                    for (int t = 0; t < T && ok; ++t) {
                        const uint32_t q = n_a + t;
                        const int buf = q & 1;
                        if (!(ok = mbar_wait(&ctl.a_full[buf], (q >> 1) & 1, &ctl, a.err))) break;
                        if (!(ok = mbar_wait(&ctl.acc_empty[buf], ((q >> 1) & 1) ^ 1, &ctl, a.err))) break;
                        tc_fence_after();
                        const uint32_t dcol = tmem + (uint32_t)(buf * 128);
                        const uint64_t dAt = dA + (uint64_t)((buf * C::TILE) >> 4);
                        // -z.mu from the BF16 hi (and lo) halves of -mu
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            if (half == 1 && !use_lo) break;
#pragma unroll
                            for (int k = 0; k < C::ATOM / 16; ++k)
                                mma_bf16(dcol, dAt + (uint64_t)((k * 32) >> 4),
                                         (half ? dBlo : dBhi) + (uint64_t)((k * 32) >> 4), idesc, (half | k) ? 1 : 0);
                        }
                        // Lloyd pass: + (||mu||^2 + 4)/2 + 128 from the constant slice
                        if (!fin) mma_bf16(dcol, dAugA, dAugB, idesc, 1);
                        mma_commit(&ctl.acc_full[buf]);
                        mma_commit(&ctl.a_empty[buf]);
                    }
                }
            } else {
                // ---------------- epilogue: thread = point ----------------
                // Every epilogue thread reaches both named barriers of every tile, so the exit
                // after a failed wait is taken by all of them together.
                const int quarter = warp & 3;
                const int row = quarter * 32 + lane;
                const int ew = warp - 2;                 // epilogue warp 0..3
                const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
                for (int t = 0; t < T; ++t) {
                    const uint32_t q = n_a + t;
                    const int buf = q & 1;
                    const int64_t i = 128 * (int64_t)t + row;
                    // the point's previous label, loaded before the wait (only this thread
                    // writes it, one pass earlier)
                    const int ol_pre = (!fin && i < n) ? (int)lab[i] : -1;
                    const bool ok = __all_sync(0xffffffffu, mbar_wait(&ctl.acc_full[buf], (q >> 1) & 1, &ctl, a.err));
                    float bv = INFINITY, b2 = INFINITY;
                    int bi = -1;
                    if (ok) {
                        tc_fence_after();
                        if (!fin) {
                            // keys: accumulator bits x 64 + (0x48000000 + column in its 64-column slice)
                            // a 64-column slice per tensor-memory load (one wait), a last slice of 32
                            // columns alone
                            for (int h = 0; 64 * h < Np; ++h) {
                                float m0 = INFINITY, m1 = INFINITY;
                                uint32_t r[64];
                                const int w = Np - 64 * h >= 64 ? 64 : 32;
                                if (w == 64) tmem_ld64(lane_base + (uint32_t)(buf * 128 + 64 * h), r);
                                else tmem_ld32(lane_base + (uint32_t)(buf * 128 + 64 * h), *reinterpret_cast<uint32_t(*)[32]>(r));
#pragma unroll
                                for (int k = 0; k < 64; k += 4) {
                                    if (k < w) {
                                        m0 = min3f(m0, __uint_as_float(r[k] * 64u + (0x48000000u + k)),
                                                   __uint_as_float(r[k + 1] * 64u + (0x48000000u + k + 1)));
                                        m1 = min3f(m1, __uint_as_float(r[k + 2] * 64u + (0x48000000u + k + 2)),
                                                   __uint_as_float(r[k + 3] * 64u + (0x48000000u + k + 3)));
                                    }
                                }
                                const uint32_t kb = __float_as_uint(fminf(m0, m1));
                                const float v = __uint_as_float(kb & 0xFFFFFFC0u);
                                if (v < bv) { bv = v; bi = 64 * h + (int)(kb & 63u); }
                            }
                        } else {
                            // exact best and second best of ||mu||^2 + 4 - 2 z.mu
                            for (int pc = 0; pc < Np / 32; ++pc) {
                                uint32_t r[32];
                                tmem_ld32(lane_base + (uint32_t)(buf * 128 + 32 * pc), r);
#pragma unroll
                                for (int k = 0; k < 32; ++k) {
                                    const float sc = fmaf(2.0f, __uint_as_float(r[k]), nrm4[32 * pc + k]);
                                    if (sc < bv) { b2 = bv; bv = sc; bi = 32 * pc + k; } else { b2 = fminf(b2, sc); }
                                }
                            }
                        }
                        tc_fence_before();
                        mbar_arrive(&ctl.acc_empty[buf]);   // every column read: the accumulator is free
                        if (i < n) {
                            int nl = bi;
                            if (nl < 0 || nl >= K) nl = 0;   // non-finite scores: keep indices in range
                            if (fin) {
                                if (!(b2 - bv > a.band)) {
                                    // near tie: FP32 direct form over every centroid, ties to the lowest
                                    const __nv_bfloat16* zi = a.Z + (o + i) * D;
                                    float best = INFINITY;
                                    int bj = 0;
                                    for (int c = 0; c < K; ++c) {
                                        float sd = 0.f;
                                        for (int k = 0; k < D; ++k) {
                                            const float dd = __fsub_rn(__bfloat162float(zi[k]), mu[c * D + k]);
                                            sd = __fadd_rn(sd, __fmul_rn(dd, dd));
                                        }
                                        if (sd < best) { best = sd; bj = c; }
                                    }
                                    nl = bj;
                                }
                                lab[i] = (int16_t)nl;
                            } else {
                                int ol = ol_pre;
                                if (ol < -1 || ol >= K) {   // never expected: reported, taken as unassigned
                                    flag_error(a.err, DERR_BOUNDS);
                                    ol = -1;
                                }
                                if (nl != ol) {
                                    lab[i] = (int16_t)nl;
                                    const int slot_c = atomicAdd(&ctl.nchg[t & 1], 1);
                                    if (slot_c < 128) ctl.chg[t & 1][slot_c] = make_int4((int)i, ol, nl, 0);
                                    else flag_error(a.err, DERR_BOUNDS);
                                }
                            }
                        }
                    } else if (lane == 0) {
                        ctl.epi_abort = 1;
                    }
                    btc_epi_sync();
                    if (*(volatile int*)&ctl.epi_abort) break;
                    if (!fin) {
                        // the tile's changes: a warp per change, lanes over coordinates, each moving
                        // the point's 2^-40 fixed-point row from its old cluster's sum to its new one
                        // Eight of the warp's changes at a time, their rows read from the point tile
                        // in shared memory (kept until this application is done) before any of
                        // their reductions is issued.
                        const int nch = ctl.nchg[t & 1] < 128 ? ctl.nchg[t & 1] : 128;
                        constexpr int GCH = 8, KPL = D / 32;   // changes per group, coordinates per lane
                        for (int e0 = ew; e0 < nch; e0 += 4 * GCH) {
                            int4 r[GCH];
                            float zv[GCH][KPL];
#pragma unroll
                            for (int gq = 0; gq < GCH; ++gq) {
                                const int e = e0 + 4 * gq;
                                r[gq] = e < nch ? ctl.chg[t & 1][e] : make_int4(-1, -1, -1, 0);
                                const bool okr = e < nch && r[gq].x >= 0 && r[gq].x < n && r[gq].y >= -1 && r[gq].y < K &&
                                                 r[gq].z >= 0 && r[gq].z < K;
                                if (e < nch && !okr && lane == 0) flag_error(a.err, DERR_BOUNDS);
                                if (!okr) r[gq].x = -1;
#pragma unroll
                                for (int kk = 0; kk < KPL; ++kk)
                                    zv[gq][kk] = okr ? tile_coord<D>(sA + buf * C::TILE, (int)(r[gq].x - 128 * (int64_t)t),
                                                                  lane + 32 * kk)
                                                     : 0.f;
                            }
#pragma unroll
                            for (int gq = 0; gq < GCH; ++gq) {
                                if (r[gq].x < 0) continue;
                                if (lane == 0) {
                                    atomicAdd(cnt + r[gq].z, 1);
                                    if (r[gq].y >= 0) atomicSub(cnt + r[gq].y, 1);
                                }
#pragma unroll
                                for (int kk = 0; kk < KPL; ++kk) {
                                    const int k = lane + 32 * kk;
                                    const long long v = __float2ll_rn(zv[gq][kk] * FIXED_SCALE_F);
                                    atomicAdd(reinterpret_cast<unsigned long long*>(sums + r[gq].z * D + k),
                                              (unsigned long long)v);
                                    if (r[gq].y >= 0)
                                        atomicAdd(reinterpret_cast<unsigned long long*>(sums + r[gq].y * D + k),
                                                  (unsigned long long)(-v));
                                }
                            }
                        }
                    }
                    btc_epi_sync();
                    if (threadIdx.x == 64) mbar_arrive(&ctl.a_empty[buf]);   // the point tile may be refilled
                    if (!fin && threadIdx.x == 64) {
                        ctl.changed += ctl.nchg[t & 1];
                        ctl.nchg[t & 1] = 0;
                    }
                }
            }
            n_a += (uint32_t)T;
            n_b += 1;
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (*(volatile int*)&ctl.abort) break;
            if (fin) break;
            if (ctl.changed == 0) {           // converged: the final assignment against these centroids
                passes = pass;
                fin = true;
                continue;
            }
            if (pass == a.iters) {            // no update after the last pass
                fin = true;
                continue;
            }
            // FP64 means of the fixed-point sums; empty clusters keep their centroid
            {
                // four of the warp's clusters at a time: their sums are read (through L2) before
                // any mean is formed
                constexpr int NW = BTC_THREADS / 32, UC = 4, KPL = D / 32;
                for (int cc0 = warp; cc0 < K; cc0 += NW * UC) {
                    int ct[UC];
                    long long sv[UC][KPL];
#pragma unroll
                    for (int u = 0; u < UC; ++u) {
                        const int cc = cc0 + NW * u;
                        ct[u] = cc < K ? cnt[cc] : 0;
#pragma unroll
                        for (int kk = 0; kk < KPL; ++kk) sv[u][kk] = ct[u] > 0 ? __ldcg(sums + cc * D + lane + 32 * kk) : 0;
                    }
#pragma unroll
                    for (int u = 0; u < UC; ++u) {
                        if (ct[u] <= 0) continue;
                        const int cc = cc0 + NW * u;
                        const double inv = 1.0 / ((double)ct[u] * FIXED_SCALE);
#pragma unroll
                        for (int kk = 0; kk < KPL; ++kk) mu[cc * D + lane + 32 * kk] = (float)((double)sv[u][kk] * inv);
                    }
                }
            }
            updated = true;
            __syncthreads();
        }
        if (*(volatile int*)&ctl.abort) break;
        batch_score_item(b, g, slot, K, o, n, lab, passes, score_scratch, a.rp64, a.rp32, a.col);
        __syncthreads();
    }
    // exit: the producer lets its last copies land, the MMA issuer waits for its last MMAs
    // (both bounded), then tensor memory is freed
    if (warp == 0 && lane == 0) {
        if (issued_b) mbar_drain(&ctl.b_full, (n_b - 1) & 1);
        for (uint32_t q = issued_a > 2 ? issued_a - 2 : 0; q < issued_a; ++q) mbar_drain(&ctl.a_full[q & 1], (q >> 1) & 1);
    }
    if (warp == 1 && lane == 0) {
        mma_commit(&ctl.drain);
        mbar_drain(&ctl.drain, 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
// operand rows (hi, lo, norm slice) and centroid sums of up to BTC_MAX_CTAS_PER_SM CTAs per SM
size_t batch_tc_staging_bytes(int d) {
    const size_t rows = (size_t)num_sms() * BTC_MAX_CTAS_PER_SM * 128;
    const size_t ops = (rows * (2 * (size_t)d + 16) * sizeof(__nv_bfloat16) + 255) / 256 * 256;
    return ops + rows * (size_t)d * sizeof(long long);
}

template <int D>
static cudaError_t launch_btc_t(BatchDev b, const __nv_bfloat16* Z, int phase, int iters, int lo_fast,
                                const raftgp_csr* g, void* stg, uint32_t* err, cudaStream_t s) {
    using C = BtcCfg<D>;
    auto kern = k_batch_lloyd_tc<D>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // the CTAs that can be resident at once (at most BTC_MAX_CTAS_PER_SM per SM, which the
    // staging area is sized for)
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BTC_THREADS, C::SMEM)) != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (per_sm > BTC_MAX_CTAS_PER_SM) per_sm = BTC_MAX_CTAS_PER_SM;
    const int grid = num_sms() * per_sm;
    BtcArgs a;
    a.b = b;
    a.Z = Z;
    a.phase = phase;
    a.iters = iters;
    a.lo_fast = lo_fast;
    a.rp64 = g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr;
    a.rp32 = g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr;
    a.col = g->col;
    a.stg_hi = reinterpret_cast<__nv_bfloat16*>(stg);
    a.stg_lo = a.stg_hi + (size_t)grid * 128 * D;
    a.stg_aug = a.stg_lo + (size_t)grid * 128 * D;
    {
        const size_t rows = (size_t)num_sms() * BTC_MAX_CTAS_PER_SM * 128;   // as batch_tc_staging_bytes
        const size_t ops = (rows * (2 * (size_t)D + 16) * sizeof(__nv_bfloat16) + 255) / 256 * 256;
        a.gsums = reinterpret_cast<long long*>(reinterpret_cast<char*>(stg) + ops);
    }
    a.band = tc_tie_band(D);
    a.err = err;
    const CUtensorMapSwizzle swz = C::ATOM_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap tz, th, tl, tg;
    if ((e = make_map_bf16(&tz, Z, D, b.total_n, C::ATOM, 128, swz)) != cudaSuccess) return e;
    if ((e = make_map_bf16(&th, a.stg_hi, D, (int64_t)grid * 128, C::ATOM, 128, swz)) != cudaSuccess) return e;
    if ((e = make_map_bf16(&tl, a.stg_lo, D, (int64_t)grid * 128, C::ATOM, 128, swz)) != cudaSuccess) return e;
    if ((e = make_map_bf16(&tg, a.stg_aug, 16, (int64_t)grid * 128, 16, 128, CU_TENSOR_MAP_SWIZZLE_32B)) != cudaSuccess)
        return e;
    kern<<<grid, BTC_THREADS, C::SMEM, s>>>(a, tz, th, tl, tg);
    return cudaGetLastError();
}

cudaError_t launch_batch_lloyd_tc(BatchDev b, const void* Z, int d, int phase, int iters, int lo_fast,
                                  const raftgp_csr* g, void* stg, uint32_t* err, cudaStream_t s) {
    ProfScope ps(s, PF_ASSIGN_TC, 1);
    const __nv_bfloat16* z = reinterpret_cast<const __nv_bfloat16*>(Z);
    if (d == 32) return launch_btc_t<32>(b, z, phase, iters, lo_fast, g, stg, err, s);
    if (d == 64) return launch_btc_t<64>(b, z, phase, iters, lo_fast, g, stg, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace raftgp
