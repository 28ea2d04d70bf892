// spmm_flat.cu -- the BF16 gather SpMM of the projection (Eq. 5) and of the GCN layers (Eq. 6)
// as a flat stream of stored entries.
//
// A random-graph gather is bound by how many row reads stay in flight.  Here a warp walks a
// chunk of 64 consecutive rows as one stream of stored entries (CSR order) in batches of
// B = GPW x U entries: lane group g of the GPW groups (LPR lanes, 16 bytes each, per gathered
// row) loads entries u GPW + g of the batch, so every batch issues B row reads whatever the
// row boundaries are; the column indices of the next batch are loaded while the current
// batch's rows are in flight (across the chunk boundary too).  Each lane group adds its
// entries to its own FP32 accumulator; when the stream passes a row end the groups are
// combined and the row is finished (operator term, tanh, row l2-normalisation) by the whole
// warp, lane group g finishing columns [g EG, (g+1) EG) of its lane's chunk.
//
// The GCN gathers run on the CSR of A + I built once per embedding (k_self_csr: each row's
// own index first, then its neighbours), so the self loop is one more stream entry.
// Chunks come from an atomic counter; the next chunk's row pointers and row scales are
// loaded one chunk ahead.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

// Row staging: 0 = every lane copies 16 bytes of a gathered row with cp.async; 1 = TMA
// tile::gather4 (four indexed rows of the feature matrix per instruction, completion on a
// per-buffer mbarrier).  Both give the same bits.
#ifndef RAFTGP_FLAT_G4
#define RAFTGP_FLAT_G4 0
#endif

namespace raftgp {

namespace {

constexpr int FL_CH = 64;   // rows per chunk

struct FlatArgs {
    int64_t n;
    const int32_t* rp32;
    const int64_t* rp64;
    const int32_t* col;
    const int32_t* deg;
    const float* rowscale;   // rs (projection with M) or rsh (GCN)
    const float* g;          // d^T Theta (full modularity matrix)
    double inv_two_e;
    int act;                 // 0 none, 1 tanh + row l2-normalisation, 2 normalisation only
    __nv_bfloat16* out;
    __nv_bfloat16* stage;    // optional copy of the finished rows
    int* work;               // chunk counter (zeroed before the launch)
    uint32_t* err;           // device error word (a bounded wait that gave up: DERR_TIMEOUT)
    // many graphs in one CSR (full modularity operator): each row's graph, and per graph its
    // d^T Theta (ng x L) and 1 / 2e; null for one graph (then g and inv_two_e above)
    const int32_t* graph_of;
    const float* g_graph;
    const double* inv_two_e_graph;
    int ng;
};

// A row's graph, checked against the graph count (an inconsistent index is reported and
// graph 0 used instead).
__device__ __forceinline__ int fl_graph(const FlatArgs& a, int64_t i) {
    const int g = a.graph_of[i];
    if (g < 0 || g >= a.ng) {
        flag_error(a.err, DERR_BOUNDS);
        return 0;
    }
    return g;
}

// Four rows (y0..y3) of the 2D tensor map, the whole row width from x = 0, into dst (4 boxes
// one after another); completion counted on bar.
__device__ __forceinline__ void tma_gather4(void* dst, const CUtensorMap* map, uint64_t* bar, int y0, int y1, int y2,
                                            int y3) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(0), "r"(y0), "r"(y1), "r"(y2), "r"(y3)
        : "memory");
}

// Bounded wait on a staging buffer's mbarrier (2 s); false (and DERR_TIMEOUT) if it gave up.
__device__ __forceinline__ bool fl_wait(uint64_t* bar, uint32_t parity, uint32_t* err) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 255) == 255 && global_ns() - t0 > TC_WAIT_NS) {
            if (err) atomicOr(err, DERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ int64_t rp_at(const FlatArgs& a, int64_t r) {
    r = r < a.n ? r : a.n;
    return a.rp64 ? a.rp64[r] : (int64_t)a.rp32[r];
}

// A chunk's data: per lane the row pointers of rows lane, lane + 32 and 64 of the chunk
// (clamped at n) and the row scales of rows lane and lane + 32.
struct Chunk {
    int64_t id;
    int64_t rpA, rpB, rpC;
    float scA, scB;
};

template <int AGG>
__device__ __forceinline__ void fetch_chunk(const FlatArgs& a, int lane, int64_t nchunks, Chunk& c) {
    int id = 0;
    if (lane == 0) id = atomicAdd(a.work, 1);
    c.id = __shfl_sync(0xffffffffu, id, 0);
    if (c.id >= nchunks) return;
    const int64_t r0 = c.id * FL_CH;
    c.rpA = rp_at(a, r0 + lane);
    c.rpB = rp_at(a, r0 + 32 + lane);
    c.rpC = rp_at(a, r0 + FL_CH);
    const int64_t ra = r0 + lane, rb = r0 + 32 + lane;
    if constexpr (AGG == AGG_MOD_FULL_) {
        if (a.graph_of) {
            c.scA = ra < a.n ? (float)((double)a.deg[ra] * a.inv_two_e_graph[fl_graph(a, ra)]) : 0.f;
            c.scB = rb < a.n ? (float)((double)a.deg[rb] * a.inv_two_e_graph[fl_graph(a, rb)]) : 0.f;
        } else {
            c.scA = ra < a.n ? (float)((double)a.deg[ra] * a.inv_two_e) : 0.f;
            c.scB = rb < a.n ? (float)((double)a.deg[rb] * a.inv_two_e) : 0.f;
        }
    } else {
        c.scA = ra < a.n ? a.rowscale[ra] : 0.f;
        c.scB = rb < a.n ? a.rowscale[rb] : 0.f;
    }
}

// Stream position (relative to the chunk start) where row k (0 <= k <= 64) of the chunk starts.
__device__ __forceinline__ int64_t chunk_bound(const Chunk& c, int k, int64_t rp0) {
    int64_t v;
    if (k < 32) v = __shfl_sync(0xffffffffu, c.rpA, k);
    else if (k < 64) v = __shfl_sync(0xffffffffu, c.rpB, k - 32);
    else v = c.rpC;
    return v - rp0;
}

template <int N>
__device__ __forceinline__ void store_vals(__nv_bfloat16* p, const float* y) {
    if constexpr (N == 1) {
        p[0] = __float2bfloat16_rn(y[0]);
    } else {
        uint32_t w[N / 2];
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(y[2 * k], y[2 * k + 1]);
            w[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        if constexpr (N == 8) *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        else if constexpr (N == 4) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        else *reinterpret_cast<uint32_t*>(p) = w[0];
    }
}

// Widen 8 BF16 values and add them into 8 FP32 accumulators, two per packed f32x2 add (the same
// two round-to-nearest additions as scalar code).
__device__ __forceinline__ void add_raw(const uint4& v, float* acc) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint64_t p, q;
        asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(acc[2 * i]), "f"(acc[2 * i + 1]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(q) : "r"(w[i] << 16), "r"(w[i] & 0xffff0000u));
        asm("add.rn.f32x2 %0, %0, %1;" : "+l"(p) : "l"(q));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * i]), "=f"(acc[2 * i + 1]) : "l"(p));
    }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

#ifndef RAFTGP_FLAT_WARPS
#define RAFTGP_FLAT_WARPS 8
#endif
#ifndef RAFTGP_FLAT_B128
#define RAFTGP_FLAT_B128 16
#endif
constexpr int FL_WARPS = RAFTGP_FLAT_WARPS;   // warps per block

template <int LIN, int B128 = RAFTGP_FLAT_B128>
struct FlCfg {
    static constexpr int E = 8;                 // BF16 elements per 16-byte lane chunk
    static constexpr int LPR = LIN / E;         // lanes per gathered row
    static constexpr int GPW = 32 / LPR;        // lane groups
    static constexpr int B = LIN == 128 ? B128 : 32;   // entries per batch
    static constexpr int U = B / GPW;           // copies per lane per batch
    static constexpr int ROWB = LIN * 2;
    static constexpr int EG = E / GPW;          // columns each lane finishes
    static_assert(B <= 32 && B % GPW == 0 && E % GPW == 0, "lane layout");
};

template <int AGG, int LIN, int NBUF, bool G4, int B128>
__global__ void __launch_bounds__(FL_WARPS * 32) k_spmm_flat(FlatArgs a, const __nv_bfloat16* __restrict__ X,
                                                             const __grid_constant__ CUtensorMap tmX) {
    using C = FlCfg<LIN, B128>;
    constexpr int E = C::E, LPR = C::LPR, GPW = C::GPW, B = C::B, U = C::U, ROWB = C::ROWB, EG = C::EG;
    extern __shared__ __align__(1024) unsigned char fl_smem[];
    __shared__ uint64_t fl_bar[FL_WARPS][NBUF];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int grp = lane / LPR, sub = lane % LPR;
    const int c0 = sub * E + grp * EG;   // first column this lane finishes
    unsigned char* wbuf = fl_smem + wid * (NBUF * B * ROWB);
    const __nv_bfloat16* Xl = X + sub * E;
    if constexpr (G4) {
        if (lane == 0)
            for (int q = 0; q < NBUF; ++q) mbar_init(&fl_bar[wid][q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
    }
    bool ok = true;

    float gl[EG];
#pragma unroll
    for (int e = 0; e < EG; ++e) {
        if constexpr (AGG == AGG_MOD_FULL_) gl[e] = a.graph_of ? 0.f : a.g[c0 + e];
        else gl[e] = 0.f;
    }

    const int64_t nchunks = (a.n + FL_CH - 1) / FL_CH;
    Chunk cur, nxt;
    fetch_chunk<AGG>(a, lane, nchunks, nxt);

    // Batches are issued NBUF - 1 ahead of the one being added: bi / ba count issued / added
    // batches (buffer = count % NBUF).  The issue side walks (ichunk, iq): the chunk and stream
    // position of the next batch to issue; my_col holds that batch's column indices.
    long long bi = 0, ba = 0;
    int32_t my_col = 0;
    int ich = 0;            // 0: the issue side is in `cur`, 1: in `nxt`
    int64_t iq = 0;         // next stream position to issue in that chunk
    bool mc_next = false;   // my_col holds nxt's first batch (loaded when cur ran out)
    auto chunk_items = [&](const Chunk& c, int64_t& rp0) {
        rp0 = __shfl_sync(0xffffffffu, c.rpA, 0);
        return c.rpC - rp0;
    };
    // Loads the column indices of the batch at stream position q of chunk c.
    auto load_cols = [&](const Chunk& c, int64_t q) {
        int64_t rp0;
        const int64_t items = chunk_items(c, rp0);
        my_col = (lane < B && q + lane < items) ? __ldg(a.col + rp0 + q + lane) : 0;
    };
    // Issues the next batch (if any is left on the issue side) and advances it.
    auto issue = [&]() -> bool {
        for (;;) {
            const Chunk& c = ich == 0 ? cur : nxt;
            if (c.id >= nchunks) return false;
            int64_t rp0;
            const int64_t items = chunk_items(c, rp0);
            if (iq < items) {
                const int cnt = (items - iq) < B ? (int)(items - iq) : B;
                unsigned char* buf = wbuf + (int)(bi % NBUF) * (B * ROWB);
                __syncwarp();
                if constexpr (G4) {
                    // lane L < ceil(cnt / 4) gathers entries 4L .. 4L+3 (past cnt: entry 0 again)
                    int32_t j[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int t = 4 * lane + q;
                        j[q] = __shfl_sync(0xffffffffu, my_col, t < cnt ? t : 0);
                    }
                    const int ninst = (cnt + 3) / 4;
                    uint64_t* bar = &fl_bar[wid][(int)(bi % NBUF)];
                    // the buffer's previous contents were read by every lane (generic proxy)
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(ninst * 4 * ROWB));
                    __syncwarp();
                    if (lane < ninst) tma_gather4(buf + 4 * lane * ROWB, &tmX, bar, j[0], j[1], j[2], j[3]);
                } else {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int t = u * GPW + grp;
                        const int32_t j = __shfl_sync(0xffffffffu, my_col, t < cnt ? t : 0);
                        if (t < cnt) cp_async16(buf + t * ROWB + sub * 16, Xl + (int64_t)j * LIN);
                    }
                    cp_async_commit();
                }
                ++bi;
                iq += cnt;
                if (iq < items) {
                    load_cols(c, iq);
                } else if (ich == 0 && nxt.id < nchunks) {
                    load_cols(nxt, 0);
                    mc_next = true;
                }
                return true;
            }
            if (ich == 1) return false;   // never run two chunks ahead
            ich = 1;
            iq = 0;
            // the next chunk's first indices, unless loaded when cur's last batch was issued
            if (!mc_next && nxt.id < nchunks) {
                load_cols(nxt, 0);
                mc_next = true;
            }
        }
    };

    float acc[E];
    while (ok && nxt.id < nchunks) {
        cur = nxt;
        fetch_chunk<AGG>(a, lane, nchunks, nxt);
        if (ich == 1) {   // the issue side had moved into this chunk: iq and my_col are current
            ich = 0;
        } else {          // nothing of this chunk issued yet
            iq = 0;
            if (!mc_next) load_cols(cur, 0);
        }
        mc_next = false;
        const int64_t row0 = cur.id * FL_CH;
        const int nrows = (int)((a.n - row0) < FL_CH ? (a.n - row0) : FL_CH);
        int64_t rp0;
        const int64_t items = chunk_items(cur, rp0);
        int cr = 0;
        int64_t cb = chunk_bound(cur, 1, rp0);
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;

        auto finish = [&]() {
#pragma unroll
            for (int o = 16; o >= LPR; o >>= 1) {
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
            }
            const float sc = __shfl_sync(0xffffffffu, cr < 32 ? cur.scA : cur.scB, cr & 31);
            float y[EG];
#pragma unroll
            for (int e = 0; e < EG; ++e) {
                float v = acc[e];
#pragma unroll
                for (int q = 1; q < GPW; ++q)
                    if (grp == q) v = acc[q * EG + e];
                if constexpr (AGG == AGG_MOD_FULL_) {
                    // the row's own graph's d^T Theta when several graphs share the CSR
                    const float ge = a.graph_of ? a.g_graph[(int64_t)fl_graph(a, row0 + cr) * LIN + c0 + e] : gl[e];
                    y[e] = v - sc * ge;
                } else {
                    y[e] = sc * v;
                }
            }
            if (a.act != 0) {
                float ss = 0.f;
#pragma unroll
                for (int e = 0; e < EG; ++e) {
                    if (a.act == 1) y[e] = tanhf(y[e]);
                    ss += y[e] * y[e];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                const float inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
#pragma unroll
                for (int e = 0; e < EG; ++e) y[e] *= inv;
            }
            const int64_t i = row0 + cr;
            if (a.stage) store_vals<EG>(a.stage + i * LIN + c0, y);
            store_vals<EG>(a.out + i * LIN + c0, y);
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0.f;
            ++cr;
            cb = cr < nrows ? chunk_bound(cur, cr + 1, rp0) : items;
        };

        for (int64_t q0 = 0; q0 < items; q0 += B) {
            // keep NBUF - 1 batches in flight beyond the one about to be added
            while (bi - ba < NBUF && issue()) {
            }
            static_assert(NBUF >= 2 && NBUF <= 4, "pipeline depth");
            if constexpr (G4) {
                if (!fl_wait(&fl_bar[wid][(int)(ba % NBUF)], (uint32_t)((ba / NBUF) & 1), a.err)) {
                    ok = false;
                    break;
                }
            } else {
                const long long ahead = bi - ba - 1;   // batches issued after this one
                if (ahead >= NBUF - 1) cp_async_wait<NBUF - 1>();
                else if (ahead == 2) cp_async_wait<2>();
                else if (ahead == 1) cp_async_wait<1>();
                else cp_async_wait<0>();
            }
            __syncwarp();
            const unsigned char* buf = wbuf + (int)(ba % NBUF) * (B * ROWB) + sub * 16;
            const int cnt = (items - q0) < B ? (int)(items - q0) : B;
            const int64_t end = q0 + cnt;
            int64_t s_lo = q0;
            for (;;) {
                const int64_t s_hi = cb < end ? cb : end;   // entries of row cr in this batch
                const int t0 = (int)(s_lo - q0);
                int t = t0 + ((grp - t0 % GPW) + GPW) % GPW;
                const int tend = (int)(s_hi - q0);
#pragma unroll 4
                for (; t < tend; t += GPW) {
                    const uint4 v = *reinterpret_cast<const uint4*>(buf + t * ROWB);
                    add_raw(v, acc);
                }
                if (cb > end || cr >= nrows) break;   // row cr continues in the next batch
                finish();
                s_lo = s_hi;
                if (cr >= nrows) break;
            }
            ++ba;
        }
        if (!ok) break;
        while (cr < nrows) finish();   // the last row and any empty rows at the end
    }
    if constexpr (G4) {
        // a wait gave up: let the copies still in flight land before the warp exits (bounded)
        for (long long k = ba; k < bi; ++k) mbar_drain(&fl_bar[wid][(int)(k % NBUF)], (uint32_t)((k / NBUF) & 1));
    } else {
        cp_async_wait<0>();
    }
}

// CSR of A + I: row i holds i first, then its neighbours in their stored order.
__global__ void k_self_csr(int64_t n, const int32_t* rp32, const int64_t* rp64, const int32_t* col, int64_t* rp_self,
                           int32_t* col_self) {
    // 8 lanes per row, 4 rows per warp in flight
    const int sub = threadIdx.x & 7;
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) >> 3;
    for (int64_t i = grp; i < n; i += ngrp) {
        const int64_t b = rp64 ? rp64[i] : rp32[i];
        const int64_t e = rp64 ? rp64[i + 1] : rp32[i + 1];
        const int64_t o = b + i;
        if (sub == 0) {
            rp_self[i] = o;
            col_self[o] = (int32_t)i;
            if (i == n - 1) rp_self[n] = e + n;
        }
        for (int64_t p = b + sub; p < e; p += 8) col_self[o + 1 + (p - b)] = __ldg(col + p);
    }
}

template <int AGG, int LIN, int NBUF, int B128 = RAFTGP_FLAT_B128>
cudaError_t launch_flat_t(const FlatArgs& a, const void* X, cudaStream_t s) {
    using C = FlCfg<LIN, B128>;
    constexpr bool G4 = RAFTGP_FLAT_G4 != 0;
    auto kern = k_spmm_flat<AGG, LIN, NBUF, G4, B128>;
    const int smem = FL_WARPS * NBUF * C::B * C::ROWB;
    CUtensorMap tmX;
    memset(&tmX, 0, sizeof(tmX));
    if (G4) {
        // rows of X, one box = one whole row (the gather's boxes are one row high)
        cudaError_t me = make_map_bf16(&tmX, X, LIN, a.n, LIN, 1, CU_TENSOR_MAP_SWIZZLE_NONE);
        if (me != cudaSuccess) return me;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FL_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t nchunks = (a.n + FL_CH - 1) / FL_CH;
    const int64_t want = (nchunks + FL_WARPS - 1) / FL_WARPS;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    const int blocks = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    ProfScope ps(s, AGG == AGG_GCN_ ? PF_SPMM_GCN : PF_SPMM_PROJ, 1);
    kern<<<blocks, FL_WARPS * 32, smem, s>>>(a, reinterpret_cast<const __nv_bfloat16*>(X), tmX);
    return cudaGetLastError();
}

#ifndef RAFTGP_FLAT_NBUF
#define RAFTGP_FLAT_NBUF 2
#endif

// Shape variants (the same sums in the same order, so the same bits): 0 = the default (16
// entries per batch at width 128, two staging buffers), 1 = 16 entries and three buffers,
// 2 = 32 entries and two buffers, 3 = 32 entries and three buffers.
template <int AGG>
cudaError_t launch_flat_w(const FlatArgs& a, int lin, const void* X, int variant, cudaStream_t s) {
    switch (lin) {
        case 32:
            return variant & 1 ? launch_flat_t<AGG, 32, 3>(a, X, s) : launch_flat_t<AGG, 32, RAFTGP_FLAT_NBUF>(a, X, s);
        case 64:
            return variant & 1 ? launch_flat_t<AGG, 64, 3>(a, X, s) : launch_flat_t<AGG, 64, RAFTGP_FLAT_NBUF>(a, X, s);
        case 128:
            switch (variant) {
                case 1: return launch_flat_t<AGG, 128, 3, 16>(a, X, s);
                case 2: return launch_flat_t<AGG, 128, 2, 32>(a, X, s);
                case 3: return launch_flat_t<AGG, 128, 3, 32>(a, X, s);
                default: return launch_flat_t<AGG, 128, RAFTGP_FLAT_NBUF>(a, X, s);
            }
        default: return cudaErrorNotSupported;
    }
}

}  // namespace

bool spmm_flat_supported(int agg, int dtype, int lin) {
    return dtype == RAFTGP_BF16 && agg != AGG_MOD_REDUCED_ && (lin == 32 || lin == 64 || lin == 128);
}

void launch_self_csr(const raftgp_csr* g, int64_t* rp_self, int32_t* col_self, cudaStream_t s) {
    if (g->n == 0) {
        cudaMemsetAsync(rp_self, 0, sizeof(int64_t), s);
        return;
    }
    const int threads = 256;
    int64_t blocks = (g->n * 32 + threads - 1) / threads;
    blocks = blocks > (int64_t)num_sms() * 16 ? (int64_t)num_sms() * 16 : blocks;
    ProfScope ps(s, PF_OTHER, 1);
    k_self_csr<<<(unsigned)blocks, threads, 0, s>>>(g->n, g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr,
                                                    g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr, g->col,
                                                    rp_self, col_self);
}

cudaError_t launch_spmm_flat(int agg, int64_t n, int rp_bits, const void* row_ptr, const int32_t* col, int64_t nnz_g,
                             const int32_t* deg, const float* rowscale, const float* gvec, int act, int lin,
                             const void* X, void* out, void* stage, int* work, uint32_t* err, int variant,
                             cudaStream_t s, const int32_t* graph_of, const float* g_graph,
                             const double* inv_two_e_graph, int ng) {
    FlatArgs a;
    a.ng = ng;
    a.graph_of = graph_of;
    a.g_graph = g_graph;
    a.inv_two_e_graph = inv_two_e_graph;
    a.n = n;
    a.rp32 = rp_bits == 32 ? (const int32_t*)row_ptr : nullptr;
    a.rp64 = rp_bits == 64 ? (const int64_t*)row_ptr : nullptr;
    a.col = col;
    a.deg = deg;
    a.rowscale = rowscale;
    a.g = gvec;
    a.inv_two_e = nnz_g > 0 ? 1.0 / (double)nnz_g : 0.0;
    a.act = act;
    a.out = reinterpret_cast<__nv_bfloat16*>(out);
    a.stage = reinterpret_cast<__nv_bfloat16*>(stage);
    a.work = work;
    a.err = err;
    if (n == 0) return cudaSuccess;
    switch (agg) {
        case AGG_NCUT_: return launch_flat_w<AGG_NCUT_>(a, lin, X, variant, s);
        case AGG_MOD_FULL_: return launch_flat_w<AGG_MOD_FULL_>(a, lin, X, variant, s);
        case AGG_GCN_: return launch_flat_w<AGG_GCN_>(a, lin, X, variant, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace raftgp
