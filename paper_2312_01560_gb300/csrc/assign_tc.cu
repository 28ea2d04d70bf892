// assign_tc.cu -- k-means assignment on the 5th-generation tensor cores (sm_103a).
//
// For a tile of 128 points and a chunk of NCH = 256 centroids the distance GEMM
//     D[p][c] = z_p . mu_c
// runs as tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor memory).  The
// centroids are split into two BF16 halves, mu = hi + lo (lo = the rounded residual), and
// both halves are multiplied into the same accumulator, so the dot product carries about 16
// significant bits of mu instead of 8.  The epilogue reads the accumulator with tcgen05.ld
// (thread t owns TMEM lane t = point t) and keeps, per candidate K, the argmin of
//     ||mu_c||^2 - 2 D[p][c]        (= ||z_p - mu_c||^2 - ||z_p||^2, ties to the lowest c).
// In the Lloyd passes a constant K=16 slice adds (||mu_c||^2 + 4)/2 + 128 to the product, so
// the accumulator is 128 + (||z_p - mu_c||^2 - ||z_p||^2 + 4)/2, inside [128, 256) for unit
// rows: there its FP32 bit pattern is 0x43000000 + m with m the score on a 2^-16 grid, and one
// integer multiply-add turns it into the key 64 m + column, whose minimum gives score and
// column at once.
//
// Warp roles in a persistent CTA (one per SM): warp 0 issues TMA loads (two point tiles per
// step, centroid chunks of NCH = 256 columns through a ring of stages), warp 1 allocates
// tensor memory and issues the MMAs (M = 128, N = 256, K = 16), warps 2-9 are two epilogue
// groups of 4 warps, each owning one point tile of the step and one 256-column accumulator
// (2 x 256 columns fill tensor memory).  N = 256 halves the shared-memory operand bytes per
// FLOP against N = 128 with four groups (6% faster at 1M points, 10 candidates); 64-column
// chunks with two buffers per group measured slower still.
// Every mbarrier wait is bounded: on timeout the CTA raises an abort flag, records
// DERR_TIMEOUT, drains its in-flight copies and MMAs (again bounded), frees its tensor memory
// and returns.
//
// Modes: FAST (Lloyd passes; the lo half is optional there) writes the new labels (k_apply_changes then counts the changes
// and applies them to the 2^-40 fixed-point centroid sums); FINAL (the assignment whose labels
// are reported) also tracks the second-best score and lists every (point, candidate) whose best
// two scores lie within the error band of the BF16 product, for an exact FP32 re-check.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace raftgp {

constexpr int TC_NCH = 256;                            // centroids per chunk = MMA N
constexpr int TC_GROUPS = 512 / TC_NCH;               // epilogue warpgroups = point tiles per step

// LO: the centroid chunks carry the lo half too (FINAL always; FAST optionally).  Without it a
// ring stage is smaller, so the ring gets deeper.
template <int D, bool LO = true>
struct TcCfg {
    static constexpr int ATOM = D < 64 ? D : 64;          // K elements per swizzle-atom row
    static constexpr int ATOM_BYTES = ATOM * 2;           // 64 or 128
    static constexpr int NATOM = D / ATOM;
    static constexpr int NCH = TC_NCH;                    // centroids per chunk = MMA N
    static constexpr int SLICES = NCH / 64;               // 64-column slices per chunk
    static constexpr int GROUPS = TC_GROUPS;              // point tiles per CTA step, one per epilogue group
    static constexpr int ACC_BUFS = 512 / (GROUPS * NCH); // accumulator buffers per group
    static constexpr int A_BUFS = D == 128 ? 1 : 2;       // point-tile groups in flight
    static constexpr int A_ATOM_BYTES = 128 * ATOM_BYTES;
    static constexpr int A_TILE_BYTES = NATOM * A_ATOM_BYTES;     // one 128-point tile
    static constexpr int A_BYTES = GROUPS * A_TILE_BYTES;         // one group of tiles
    static constexpr int AUG_A_BYTES = 128 * 32;          // the constant K=16 slice of a point tile
    static constexpr int B_ATOM_BYTES = NCH * ATOM_BYTES;
    static constexpr int B_BYTES = NATOM * B_ATOM_BYTES;  // one half (hi or lo) of a chunk
    static constexpr int AUG_B_BYTES = NCH * 32;          // the K=16 norm slice of a chunk
    static constexpr int NHALF = LO ? 2 : 1;              // hi (and lo) halves per ring stage
    static constexpr int STAGE_BYTES = NHALF * B_BYTES + AUG_B_BYTES;
    static constexpr int LAYOUT = ATOM_BYTES == 128 ? 2 : 4;  // descriptor swizzle: 128B or 64B
    static constexpr int SBO = 8 * ATOM_BYTES;                 // stride between 8-row groups
    static constexpr int FIXED = 1024 + A_BUFS * A_BYTES + AUG_A_BYTES;
    // ring depth: what the budget (227 KB less the static control block) leaves, at most 8
    static constexpr int STAGES_FIT = (218 * 1024 - FIXED) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT < 8 ? STAGES_FIT : 8;
    static_assert(STAGES >= 1, "the centroid ring needs a stage");
    static constexpr int SMEM = FIXED + STAGES * STAGE_BYTES;
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
    static_assert(GROUPS * ACC_BUFS * NCH <= 512, "the accumulator buffers must fit tensor memory");
};

constexpr int TC_MAX_CHUNKS = 1024;
constexpr int TC_THREADS = 64 + TC_GROUPS * 128;      // warp 0 TMA, warp 1 MMA, then the epilogue groups

struct TcCtl {
    uint64_t a_full[2], a_empty[2];
    uint64_t b_full[8], b_empty[8];
    uint64_t acc_full[TC_GROUPS][2], acc_empty[TC_GROUPS][2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    int nchunks;
    int chunk_col[TC_MAX_CHUNKS];
    // per 64-column slice (two per chunk): candidate + 128 if the candidate's padded range ends
    // with the slice, or -1 (inactive candidate / beyond the batch)
    int16_t slice_info[(TC_NCH / 64) * TC_MAX_CHUNKS];   // SLICES per chunk
};

// ---------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------
struct TcArgs {
    CandBatch b;
    int64_t n;
    const __nv_bfloat16* Z;   // N x D
    KmState st;
    int pass;                 // FAST: pass number (parity selects the change counter)
    uint32_t key_mul;         // 64 (a run-time operand, so the key is one integer multiply-add)
    float tie_band;           // FINAL: second-best within this band -> re-check
    int2* recheck;            // FINAL: list of (point, candidate)
    int* recheck_count;
    uint32_t* err;
};

// FINAL: the reported assignment (hi + lo, exact top two, near-tie list); otherwise a Lloyd
// pass.  One CTA of 576 threads per SM (at most 96 registers per thread).
template <int D, bool LO, bool FINAL>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_assign_tc(const __grid_constant__ TcArgs a, const __grid_constant__ CUtensorMap tmA,
                const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                const __grid_constant__ CUtensorMap tmAug) {
    using C = TcCfg<D, LO>;
    static_assert(LO || !FINAL, "the final assignment multiplies both halves");
    extern __shared__ uint8_t dyn_smem[];
    __shared__ TcCtl ctl;
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;                                   // A_BUFS groups of GROUPS point tiles
    uint8_t* sAug = base + C::A_BUFS * C::A_BYTES;        // 128 rows x 32 B, constant
    uint8_t* sB = sAug + C::AUG_A_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const CandBatch& b = a.b;
    constexpr bool use_lo = LO;

    if (threadIdx.x == 0) {
        ctl.abort = 0;
        for (int q = 0; q < C::A_BUFS; ++q) {
            mbar_init(&ctl.a_full[q], 1);
            mbar_init(&ctl.a_empty[q], 1);
        }
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&ctl.b_full[s], 1);
            mbar_init(&ctl.b_empty[s], 1);
        }
        for (int g = 0; g < TC_GROUPS; ++g)
            for (int q = 0; q < 2; ++q) {
                mbar_init(&ctl.acc_full[g][q], 1);
                mbar_init(&ctl.acc_empty[g][q], 128);
            }
        mbar_init(&ctl.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // NCH-column chunks holding columns of an active candidate (FINAL: every candidate), with
        // the candidate of each 64-column slice; candidates are padded to whole slices
        int nch = 0, c = 0;
        const int total_chunks = (b.total_k + C::NCH - 1) / C::NCH;
        for (int q = 0; q < total_chunks && nch < TC_MAX_CHUNKS; ++q) {
            const int lo = q * C::NCH;
            int info[C::SLICES];
            for (int h = 0; h < C::SLICES; ++h) info[h] = -1;
            bool need = false;
            for (int h = 0; h < C::SLICES; ++h) {
                const int col0 = lo + 64 * h;
                if (col0 >= b.total_k) break;
                while (c + 1 < b.n && b.off[c + 1] <= col0) ++c;
                const int pad_end = c + 1 < b.n ? b.off[c + 1] : b.total_k;
                if (col0 < b.off[c] + b.k[c] && (FINAL || a.st.active[c])) {
                    info[h] = c + (col0 + 64 >= pad_end ? 128 : 0);
                    need = true;
                }
            }
            if (need) {
                ctl.chunk_col[nch] = lo;
                for (int h = 0; h < C::SLICES; ++h) ctl.slice_info[C::SLICES * nch + h] = (int16_t)info[h];
                ++nch;
            }
        }
        ctl.nchunks = nch;
    }
    // constant K=16 slice of a point tile: every row reads 1, 1, 1 at K = 0, 1, 2 (and again at
    // 8, 9, 10, so the row is the same under the 32-byte swizzle, which may exchange its halves)
    for (int t = threadIdx.x; t < C::AUG_A_BYTES / 16; t += blockDim.x)
        reinterpret_cast<uint4*>(sAug)[t] = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(&ctl.tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem_base;
    const int nchunks = ctl.nchunks;
    const int64_t nsteps = (a.n + 128 * C::GROUPS - 1) / (128 * C::GROUPS);   // groups of 4 tiles

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0 && nchunks > 0) {
            int it = 0, tl = 0;
            bool ok = true;
            for (int64_t step = blockIdx.x; step < nsteps && ok; step += gridDim.x, ++tl) {
                const int ab = tl % C::A_BUFS;
                if (!(ok = mbar_wait(&ctl.a_empty[ab], ((tl / C::A_BUFS) & 1) ^ 1, &ctl, a.err))) break;
                mbar_expect_tx(&ctl.a_full[ab], C::A_BYTES);
                for (int g = 0; g < C::GROUPS; ++g)
                    for (int t = 0; t < C::NATOM; ++t)
                        tma_load_2d(sA + ab * C::A_BYTES + g * C::A_TILE_BYTES + t * C::A_ATOM_BYTES, &tmA,
                                    &ctl.a_full[ab], t * C::ATOM, (int)((step * C::GROUPS + g) * 128));
                for (int q = 0; q < nchunks; ++q, ++it) {
                    const int s = it % C::STAGES;
                    if (!(ok = mbar_wait(&ctl.b_empty[s], ((it / C::STAGES) & 1) ^ 1, &ctl, a.err))) break;
                    uint8_t* dst = sB + s * C::STAGE_BYTES;
                    mbar_expect_tx(&ctl.b_full[s], C::STAGE_BYTES);
                    for (int t = 0; t < C::NATOM; ++t) {
                        tma_load_2d(dst + t * C::B_ATOM_BYTES, &tmBhi, &ctl.b_full[s], t * C::ATOM, ctl.chunk_col[q]);
                        if (use_lo)
                            tma_load_2d(dst + C::B_BYTES + t * C::B_ATOM_BYTES, &tmBlo, &ctl.b_full[s], t * C::ATOM,
                                        ctl.chunk_col[q]);
                    }
                    tma_load_2d(dst + C::NHALF * C::B_BYTES, &tmAug, &ctl.b_full[s], 0, ctl.chunk_col[q]);
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA can exit
                for (int k = (it > C::STAGES ? it - C::STAGES : 0); k < it; ++k)
                    mbar_drain(&ctl.b_full[k % C::STAGES], (k / C::STAGES) & 1);
                for (int k = (tl > C::A_BUFS ? tl - C::A_BUFS : 0); k <= tl; ++k)
                    mbar_drain(&ctl.a_full[k % C::A_BUFS], (k / C::A_BUFS) & 1);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0 && nchunks > 0) {
            const uint32_t idesc = instr_desc(C::NCH);
            // descriptors of the region bases; each operand adds its byte offset / 16 to the start
            // address field (every address stays below 256 KB, so the field never overflows)
            const uint64_t dA = smem_desc(smem_addr(sA), C::LAYOUT, C::SBO);
            const uint64_t dB = smem_desc(smem_addr(sB), C::LAYOUT, C::SBO);
            const uint64_t dAugA = smem_desc(smem_addr(sAug), 6, 256);
            const uint64_t dAugB = smem_desc(smem_addr(sB + C::NHALF * C::B_BYTES), 6, 256);
            int it = 0, tl = 0;
            bool ok = true;
            for (int64_t step = blockIdx.x; step < nsteps && ok; step += gridDim.x, ++tl) {
                const int ab = tl % C::A_BUFS;
                if (!(ok = mbar_wait(&ctl.a_full[ab], (tl / C::A_BUFS) & 1, &ctl, a.err))) break;
                tc_fence_after();
                const uint64_t dAgrp = dA + (uint64_t)((ab * C::A_BYTES) >> 4);
                for (int q = 0; q < nchunks && ok; ++q, ++it) {
                    const int s = it % C::STAGES;
                    const int buf = it % C::ACC_BUFS;
                    const uint32_t acc_par = (uint32_t)((it / C::ACC_BUFS) & 1);
                    if (!(ok = mbar_wait(&ctl.b_full[s], (it / C::STAGES) & 1, &ctl, a.err))) break;
                    const uint64_t dBst = dB + (uint64_t)((s * C::STAGE_BYTES) >> 4);
                    const uint64_t dAugBst = dAugB + (uint64_t)((s * C::STAGE_BYTES) >> 4);
#pragma unroll
                    for (int g = 0; g < C::GROUPS; ++g) {
                        if (!(ok = mbar_wait(&ctl.acc_empty[g][buf], acc_par ^ 1, &ctl, a.err))) break;
                        tc_fence_after();
                        const uint32_t dcol = tmem + (uint32_t)((g * C::ACC_BUFS + buf) * C::NCH);
                        const uint64_t dAg = dAgrp + (uint64_t)((g * C::A_TILE_BYTES) >> 4);
                        // -z.mu from the BF16 hi (and lo) halves of -mu
#pragma unroll
                        for (int half = 0; half < 2; ++half)
                            if (half < C::NHALF)
#pragma unroll
                            for (int t = 0; t < C::NATOM; ++t)
#pragma unroll
                                for (int k = 0; k < C::ATOM / 16; ++k) {
                                    const uint64_t ad = dAg + (uint64_t)((t * C::A_ATOM_BYTES + k * 32) >> 4);
                                    const uint64_t bd =
                                        dBst + (uint64_t)((half * C::B_BYTES + t * C::B_ATOM_BYTES + k * 32) >> 4);
                                    mma_bf16(dcol, ad, bd, idesc, (half | t | k) ? 1 : 0);
                                }
                        // FAST: + (||mu||^2 + 4)/2 + 128 from the constant slice, so the accumulator
                        // is 128 + (||z - mu||^2 - ||z||^2 + 4)/2
                        if (!FINAL) mma_bf16(dcol, dAugA, dAugBst, idesc, 1);
                        mma_commit(&ctl.acc_full[g][buf]);  // this group's accumulator is ready
                    }
                    if (ok) mma_commit(&ctl.b_empty[s]);  // the stage is free once these MMAs retire
                }
                if (ok) mma_commit(&ctl.a_empty[ab]);     // the point tiles are free after the last chunk
            }
            // wait for every MMA issued by this thread before tensor memory is released
            mma_commit(&ctl.drain);
            mbar_drain(&ctl.drain, 0);
        }
    } else {
        // ---------------- epilogue: group wg owns point tile wg of each step ----------------
        const int wg = (warp - 2) >> 2;               // epilogue group
        const int quarter = warp & 3;                 // TMEM lanes this warp may access
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(wg * C::ACC_BUFS * C::NCH);
        int it = 0;
        bool ok = nchunks > 0;
        for (int64_t step = blockIdx.x; step < nsteps && ok; step += gridDim.x) {
            const int64_t i = (step * C::GROUPS + wg) * 128 + row;
            const bool valid = i < a.n;
            float bv = INFINITY, b2 = INFINITY;
            int bi = -1;
            for (int q = 0; q < nchunks; ++q, ++it) {
                const int buf = it % C::ACC_BUFS;
                if (!(ok = mbar_wait(&ctl.acc_full[wg][buf], (it / C::ACC_BUFS) & 1, &ctl, a.err))) break;
                tc_fence_after();
                const int col_q = ctl.chunk_col[q];
                // the candidate of slice h ends here: write its label for this point
                auto finish = [&](int info) {
                    const int cand = info & 127;
                    const int K = b.k[cand], off = b.off[cand];
                    int nl = bi - off;
                    if (nl < 0 || nl >= K) nl = 0;       // non-finite scores: keep indices in range
                    if (FINAL) {
                        if (valid) {
                            a.st.labels[i * b.cs + cand] = (int16_t)nl;
                            if (!(b2 - bv > a.tie_band)) {
                                const int slot = atomicAdd(a.recheck_count, 1);
                                a.recheck[slot] = make_int2((int)i, cand);
                            }
                        }
                    } else if (valid) {
                        // the change against the previous pass is applied by k_apply_changes, so
                        // this epilogue never waits on a load
                        a.st.labels_new[i * b.cs + cand] = (int16_t)nl;
                    }
                    bv = INFINITY;
                    b2 = INFINITY;
                    bi = -1;
                };
                if (FINAL) {
#pragma unroll 1
                    for (int h = 0; h < C::SLICES; ++h) {
                        const int info = ctl.slice_info[C::SLICES * q + h];
                        uint32_t r[1][64];
                        if (info >= 0) tmem_ld64(lane_base + (uint32_t)(buf * C::NCH + 64 * h), r[0]);
                        if (h == C::SLICES - 1) {
                            tc_fence_before();
                            mbar_arrive(&ctl.acc_empty[wg][buf]);   // every slice read: the buffer is free
                        }
                        if (info < 0) continue;
                        const int col0 = col_q + 64 * h;
                        // exact best and second best of ||mu||^2 + 4 - 2 z.mu (FP32 norms; padding
                        // columns carry an infinite norm and never win)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            float np4[16];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float4 t4 = __ldg(reinterpret_cast<const float4*>(a.st.norm2p + col0) + 4 * v + u);
                                np4[4 * u] = t4.x; np4[4 * u + 1] = t4.y; np4[4 * u + 2] = t4.z; np4[4 * u + 3] = t4.w;
                            }
#pragma unroll
                            for (int k = 0; k < 16; ++k) {
                                const float sc = fmaf(2.0f, __uint_as_float(r[0][16 * v + k]), np4[k]);
                                if (sc < bv) { b2 = bv; bv = sc; bi = col0 + 16 * v + k; } else { b2 = fminf(b2, sc); }
                            }
                        }
                        if (info >= 128) finish(info);
                    }
                } else {
                    // Lloyd pass: the chunk in two 128-column tensor-memory loads (one wait each),
                    // reduced in 32-column pieces; the buffer is released as soon as the second
                    // load has landed, before its columns are reduced.  Keys: accumulator bits x 64 + (0x48000000 + column)
                    // wraps to 0x08000000 + 64 m + column, a positive normal float, so a float
                    // minimum gives the (score, column) minimum (four independent chains).  An
                    // accumulator outside [128, 256) (a non-finite row) gives a meaningless
                    // key; the label stays in range in finish().
                    const uint32_t mul = a.key_mul;
                    const uint32_t cbase = lane_base + (uint32_t)(buf * C::NCH);
                    uint32_t r[128];
                    float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
#pragma unroll
                    for (int hh = 0; hh < C::NCH / 128; ++hh) {
                        tmem_ld128_issue(cbase + 128u * hh, r);
                        tmem_wait_ld128(r);
                        if (hh + 1 == C::NCH / 128) {
                            tc_fence_before();
                            mbar_arrive(&ctl.acc_empty[wg][buf]);   // every column read: the buffer is free
                        }
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp) {
                            const int pc = 4 * hh + pp;           // 32-column piece of the chunk
                            const uint32_t* x = r + 32 * pp;
                            const uint32_t c0 = 0x48000000u + 32u * (pc & 1);
#pragma unroll
                            for (int k = 0; k < 32; k += 8) {
                                m0 = min3f(m0, __uint_as_float(x[k] * mul + (c0 + k)), __uint_as_float(x[k + 1] * mul + (c0 + k + 1)));
                                m1 = min3f(m1, __uint_as_float(x[k + 2] * mul + (c0 + k + 2)), __uint_as_float(x[k + 3] * mul + (c0 + k + 3)));
                                m2 = min3f(m2, __uint_as_float(x[k + 4] * mul + (c0 + k + 4)), __uint_as_float(x[k + 5] * mul + (c0 + k + 5)));
                                m3 = min3f(m3, __uint_as_float(x[k + 6] * mul + (c0 + k + 6)), __uint_as_float(x[k + 7] * mul + (c0 + k + 7)));
                            }
                            if (pc & 1) {
                                // end of 64-column slice h
                                const int h = pc >> 1;
                                const int info = ctl.slice_info[C::SLICES * q + h];
                                if (info >= 0) {
                                    const float kmin = fminf(min3f(m0, m1, m2), m3);
                                    const uint32_t kb = __float_as_uint(kmin);
                                    const float v = __uint_as_float(kb & 0xFFFFFFC0u);
                                    if (v < bv) { bv = v; bi = col_q + 64 * h + (int)(kb & 63u); }
                                    if (info >= 128) finish(info);
                                }
                                m0 = m1 = m2 = m3 = INFINITY;
                            }
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// Direct-form re-check of the listed (point, candidate) pairs: one warp per pair, lanes split
// the candidate's centroids, ||z - mu_c||^2 summed over ascending coordinates with every
// subtract, multiply and add rounded on its own (no contraction), ties to the lowest index.
// F64: in FP64 from the stored values (BF16 or FP32 z, FP32 mu, widened exactly), the same
// expression as the FP64 oracle's, so the re-checked labels are the FP64 argmin bit for bit;
// otherwise in FP32.
template <typename T, int D, bool F64>
__global__ void __launch_bounds__(256) k_recheck(CandBatch b, const T* __restrict__ Z, KmState st, const int2* list,
                                                 const int* count) {
    using R = typename std::conditional<F64, double, float>::type;
    const int lane = threadIdx.x & 31;
    const int total = *count;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += (gridDim.x * blockDim.x) >> 5) {
        const int2 pc = list[e];
        const int64_t i = pc.x;
        const int c = pc.y;
        R z[D];
#pragma unroll
        for (int k = 0; k < D; ++k) z[k] = (R)Vec<T>::to_float(Z[i * D + k]);
        const int K = b.k[c], off = b.off[c];
        R bv = (R)INFINITY;
        int bi = 0x7fffffff;
        for (int j = lane; j < K; j += 32) {
            const float* mu = st.mu + (int64_t)(off + j) * D;
            R s = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (F64) {
                    const double t = __dsub_rn((double)z[k], (double)mu[k]);
                    s = (R)__dadd_rn((double)s, __dmul_rn(t, t));
                } else {
                    const float t = __fsub_rn((float)z[k], mu[k]);
                    s = (R)__fadd_rn((float)s, __fmul_rn(t, t));
                }
            }
            if (s < bv) { bv = s; bi = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const R ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0 && bi >= 0 && bi < K) st.labels[i * b.cs + c] = (int16_t)bi;
    }
}

// Error band of the final tensor-core assignment's scores.  Each score is
//   s_c = fmaf(2, a_c, n_c),  a_c = the tensor-core sum of z_k hi_k and z_k lo_k (k < d),
//   n_c = fl(fl(||mu_c||^2) + 4),  hi + lo = the two-term BF16 split of -mu_c,
// and approximates t_c = ||mu_c||^2 + 4 - 2 z.mu_c from the stored z (BF16) and mu_c (FP32).
// With BF16 unit roundoff 2^-8, FP32 unit roundoff u = 2^-24, ||z|| <= 1, ||mu_c|| <= 1:
//   split:  hi = RN(-mu), lo = RN(-mu - hi) (the subtraction is exact), so
//           |hi_k + lo_k + mu_k| <= 2^-16 |mu_k| and |z.(hi + lo) + z.mu| <= 2^-16;
//   sum:    every product z_k hi_k, z_k lo_k is exact in FP32 (8-bit significands); the 2d
//           products enter the FP32 accumulator 16 per MMA.  Modelled as each MMA rounding or
//           truncating its 16 aligned products and the accumulator with an error of at most
//           2^-23 of the largest magnitude per term: at most 17 * 2^-23 * S per MMA, d/8 MMAs,
//           S = sum |z_k| (|hi_k| + |lo_k|) <= (1 + 2^-8)^2 < 1.01;
//   norm:   ||mu||^2 as d fused multiply-adds: <= d u 1.01; the +4: <= 5 u;
//   score:  the final fmaf, |s_c| <= 8: <= 8 u;
//   E = 2 (2^-16 + (d/8) 17 2^-23 1.01) + 1.01 d u + 13 u.
// Two scores whose exact order differs from their computed order lie within 2E; the band is
// 2E with a 25% margin (also covering the FP64 re-check's own rounding, below 1e-13).
float tc_tie_band(int d) {
    const double u = 1.0 / 16777216.0;
    const double E = 2.0 * (1.0 / 65536.0 + (d / 8.0) * 17.0 * (2.0 * u) * 1.01) + 1.01 * d * u + 13.0 * u;
    return (float)(2.5 * E);
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cudaError_t get_encoder() {
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

cudaError_t make_map_bf16(CUtensorMap* m, const void* base, int width, int64_t rows, int box_width, int box_rows,
                          CUtensorMapSwizzle swz) {
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)width * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_width, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static cudaError_t make_map_w(CUtensorMap* m, const void* base, int width, int64_t rows, int box_width, int box_rows,
                              CUtensorMapSwizzle swz) {
    return make_map_bf16(m, base, width, rows, box_width, box_rows, swz);
}

template <int D>
static cudaError_t make_map(CUtensorMap* m, const void* base, int64_t rows, int box_rows) {
    using C = TcCfg<D>;
    return make_map_w(m, base, D, rows, C::ATOM, box_rows,
                      C::ATOM_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
}

template <int D, bool LO, bool FINAL>
static cudaError_t launch_tc_t(const CandBatch& b, const __nv_bfloat16* Z, int64_t n, KmState st, int pass,
                               int2* recheck, int* recheck_count, uint32_t* err, cudaStream_t s) {
    using C = TcCfg<D, LO>;
    static_assert(C::SMEM + sizeof(TcCtl) <= 227 * 1024, "dynamic + static shared memory budget");
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    CUtensorMap ta, th, tl, tg;
    if ((e = make_map<D>(&ta, Z, n, 128)) != cudaSuccess) return e;
    if ((e = make_map<D>(&th, st.bhi, st.bhi_rows, C::NCH)) != cudaSuccess) return e;
    if ((e = make_map<D>(&tl, st.blo, st.bhi_rows, C::NCH)) != cudaSuccess) return e;
    if ((e = make_map_w(&tg, st.baug, 16, st.bhi_rows, 16, C::NCH, CU_TENSOR_MAP_SWIZZLE_32B)) != cudaSuccess) return e;
    TcArgs a;
    a.b = b;
    a.n = n;
    a.Z = Z;
    a.st = st;
    a.pass = pass;
    a.key_mul = 64u;
    a.tie_band = tc_tie_band(D);
    a.recheck = recheck;
    a.recheck_count = recheck_count;
    a.err = err;
    const int smem = C::SMEM;
    auto kern = k_assign_tc<D, LO, FINAL>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    const int64_t nsteps = (n + 128 * C::GROUPS - 1) / (128 * C::GROUPS);
    const int grid = (int)(nsteps < num_sms() ? nsteps : num_sms());
    {
        ProfScope ps(s, FINAL ? PF_ASSIGN_TC_FINAL : (pass == 1 ? PF_ASSIGN_TC_FIRST : PF_ASSIGN_TC), 1);
        kern<<<grid, TC_THREADS, smem, s>>>(a, ta, th, tl, tg);
    }
    return cudaGetLastError();
}

cudaError_t launch_assign_tc(const CandBatch& b, const void* Z, int64_t n, int d, KmState st, int pass, int final_mode,
                             int fast_lo, int2* recheck, int* recheck_count, uint32_t* err, cudaStream_t s) {
    // the chunk table holds every chunk of the batch
    if (b.total_k > TC_MAX_CHUNKS * TcCfg<64>::NCH) return cudaErrorInvalidValue;
    const __nv_bfloat16* z = (const __nv_bfloat16*)Z;
    const bool lo = final_mode || fast_lo;     // FINAL always multiplies both halves
#define RAFTGP_TC_CASE(DD)                                                                         \
    case DD:                                                                                     \
        return final_mode ? launch_tc_t<DD, true, true>(b, z, n, st, pass, recheck, recheck_count, err, s)   \
               : lo       ? launch_tc_t<DD, true, false>(b, z, n, st, pass, recheck, recheck_count, err, s)  \
                          : launch_tc_t<DD, false, false>(b, z, n, st, pass, recheck, recheck_count, err, s);
    switch (d) {
        RAFTGP_TC_CASE(32)
        RAFTGP_TC_CASE(64)
        RAFTGP_TC_CASE(128)
    }
#undef RAFTGP_TC_CASE
    return cudaErrorInvalidValue;
}

void launch_recheck(const CandBatch& b, const void* Z, int zdtype, int d, KmState st, const int2* list,
                    const int* count, int fp64, cudaStream_t s) {
    const int blocks = num_sms() * 4;
    ProfScope ps(s, PF_RECHECK, 1);
#define RAFTGP_RC(TT, DD)                                                                                  \
    case DD:                                                                                               \
        if (fp64) k_recheck<TT, DD, true><<<blocks, 256, 0, s>>>(b, (const TT*)Z, st, list, count);       \
        else k_recheck<TT, DD, false><<<blocks, 256, 0, s>>>(b, (const TT*)Z, st, list, count);           \
        break;
    if (zdtype == RAFTGP_BF16) {
        switch (d) { RAFTGP_RC(__nv_bfloat16, 32) RAFTGP_RC(__nv_bfloat16, 64) RAFTGP_RC(__nv_bfloat16, 128) }
    } else {
        switch (d) { RAFTGP_RC(float, 32) RAFTGP_RC(float, 64) RAFTGP_RC(float, 128) }
    }
#undef RAFTGP_RC
}

}  // namespace raftgp
