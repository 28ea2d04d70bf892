// assign_ffma.cu -- plain FP32 k-means assignment (Section III-C, "apply KMeans") on the FMA
// pipes, register-tiled.
//
// One CTA of 256 threads owns a tile of 256 points and walks every candidate of the batch (the
// active ones in a Lloyd pass, all of them in the final assignment), 64 centroids at a time:
//   - the point tile is staged once, transposed (zT[k][p], FP32), so every candidate reuses it;
//   - a chunk of 64 centroids comes from the k-major copy of the centroids (muT[k][col], kept by
//     the centroid update) with 16-byte cp.async copies, double-buffered, with its 64 norms;
//   - warp w computes points 32w..32w+31 against the whole chunk: lane (pr, cr) = (lane / 8,
//     lane % 8) holds points {4pr..4pr+3, 16+4pr..16+4pr+3} and centroids {4cr..4cr+3,
//     32+4cr..32+4cr+3} in an 8 x 8 register tile, so per coordinate it issues four 16-byte
//     shared loads (each served in one shared-memory wavefront: the z loads are shared by the 8
//     lanes of a point group, the centroid loads are 128 contiguous bytes) for 64 FMAs;
//   - score s = fmaf(-2, z.mu, ||mu||^2) with z.mu accumulated by fmaf over ascending
//     coordinates (= ||z - mu||^2 - ||z||^2); each lane keeps its own minimum over ascending
//     columns, and at the end of a candidate the 8 lanes of a point group combine theirs (ties
//     to the lowest column), so the label is the lowest-index minimum of the FP32 scores.
// Lloyd pass: a changed label moves the point's 2^-40 fixed-point row between the two clusters'
// sums (64-bit reductions), the counts follow, and one change counter per candidate and warp.
// Final assignment: labels only, and every (point, candidate) whose best two scores lie within
// the error band of this FP32 evaluation is listed for the FP64 re-check.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

constexpr int FF_THREADS = 256;
constexpr int FF_PTS = 256;   // points per CTA (8 warps x 32)
constexpr int FF_CH = 64;     // centroids per chunk (every candidate is padded to 64 columns)

template <int D>
struct FfCfg {
    static constexpr int ZT = D * FF_PTS;            // floats of the point tile
    static constexpr int CHUNK = D * FF_CH + FF_CH;  // floats of one chunk buffer (+ its norms)
    // chunk buffers: three where they fit (two CTAs per SM at d <= 64: 2 x 115,456 bytes plus
    // the per-CTA reserve stay within the SM's 233,472), so one barrier per chunk suffices
    static constexpr int BUFS = D <= 64 ? 3 : 2;
    static constexpr int SMEM = (ZT + BUFS * CHUNK) * (int)sizeof(float);
    static constexpr int MIN_BLOCKS = D <= 64 ? 2 : 1;
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

// Packed FP32 pairs (Blackwell f32x2): two independent IEEE fused multiply-adds per
// instruction, each rounded exactly as fmaf, on 64-bit register pairs (low half first).
__device__ __forceinline__ uint64_t ff_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void ff_unpack(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void ff_fma2(uint64_t& acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

__device__ __forceinline__ void ff_cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void ff_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void ff_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void ff_wait_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Advances (c, q) to the next chunk: the next 64 columns of candidate c that hold a real
// centroid, else the first chunk of the next candidate taken (every one if `all`, else the
// active ones).  Returns false past the last.
__device__ __forceinline__ bool ff_next(const CandBatch& b, const int32_t* active, bool all, int& c, int& q) {
    if (c >= 0 && (q + 1) * FF_CH < b.k[c]) {
        ++q;
        return true;
    }
    q = 0;
    for (++c; c < b.n; ++c)
        if (all || active[c]) return true;
    return false;
}

template <int D>
__device__ __forceinline__ void ff_load_chunk(float* buf, const KmState& st, int col0, int tid) {
    constexpr int ROW16 = FF_CH / 4;   // 16-byte pieces per coordinate row of the chunk
    for (int t = tid; t < D * ROW16 + ROW16; t += FF_THREADS) {
        if (t < D * ROW16) {
            const int k = t / ROW16, j4 = t % ROW16;
            ff_cp16(buf + k * FF_CH + 4 * j4, st.muT + (int64_t)k * st.bhi_rows + col0 + 4 * j4);
        } else {
            const int j4 = t - D * ROW16;
            ff_cp16(buf + D * FF_CH + 4 * j4, st.norm2 + col0 + 4 * j4);
        }
    }
    ff_commit();
}

// One chunk against the warp's 32 points: lane (pr, cr) accumulates its 8 points against NJ
// centroids (NJ = 8: columns {4cr..4cr+3, 32+4cr..32+4cr+3}; NJ = 4: {4cr..4cr+3}, for a
// chunk whose real centroids all lie in its first 32 columns), then folds the scores into its
// running minimum (and second minimum, FINAL) per point, columns ascending.
template <int D, bool FINAL, int NJ>
__device__ __forceinline__ void ff_chunk(const float* __restrict__ zw, const float* __restrict__ mT, int pr, int cr,
                                         int q, float* bv, float* b2, int* bi) {
    constexpr int NB = NJ / 2;   // centroid pairs
    // the accumulators as packed pairs: dg[a][b] = (z_2a m_2b, z_2a+1 m_2b+1) and
    // an[a][b] = (z_2a m_2b+1, z_2a+1 m_2b), each summed over ascending coordinates
    uint64_t dg[4][NB], an[4][NB];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2i = 0; b2i < NB; ++b2i) { dg[a][b2i] = 0ull; an[a][b2i] = 0ull; }
#pragma unroll 4
    for (int k = 0; k < D; ++k) {
        const float4 za = *reinterpret_cast<const float4*>(zw + k * FF_PTS + 4 * pr);
        const float4 zb = *reinterpret_cast<const float4*>(zw + k * FF_PTS + 16 + 4 * pr);
        const float4 ma = *reinterpret_cast<const float4*>(mT + k * FF_CH + 4 * cr);
        const uint64_t zp[4] = {ff_pack(za.x, za.y), ff_pack(za.z, za.w), ff_pack(zb.x, zb.y), ff_pack(zb.z, zb.w)};
        uint64_t mp[NB], ms[NB];
        mp[0] = ff_pack(ma.x, ma.y); mp[1] = ff_pack(ma.z, ma.w);
        ms[0] = ff_pack(ma.y, ma.x); ms[1] = ff_pack(ma.w, ma.z);
        if constexpr (NJ == 8) {
            const float4 mb = *reinterpret_cast<const float4*>(mT + k * FF_CH + 32 + 4 * cr);
            mp[2] = ff_pack(mb.x, mb.y); mp[3] = ff_pack(mb.z, mb.w);
            ms[2] = ff_pack(mb.y, mb.x); ms[3] = ff_pack(mb.w, mb.z);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b2i = 0; b2i < NB; ++b2i) {
                ff_fma2(dg[a][b2i], zp[a], mp[b2i]);
                ff_fma2(an[a][b2i], zp[a], ms[b2i]);
            }
    }
    float acc[8][NJ];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2i = 0; b2i < NB; ++b2i) {
            ff_unpack(dg[a][b2i], acc[2 * a][2 * b2i], acc[2 * a + 1][2 * b2i + 1]);
            ff_unpack(an[a][b2i], acc[2 * a][2 * b2i + 1], acc[2 * a + 1][2 * b2i]);
        }
    // this lane's columns, ascending: 4cr..4cr+3, then 32+4cr..32+4cr+3
    const float* nrm = mT + D * FF_CH;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int jc = j < 4 ? 4 * cr + j : 32 + 4 * cr + (j - 4);
        const float nq = nrm[jc];
        const int col = q * FF_CH + jc;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float sc = fmaf(-2.0f, acc[r][j], nq);
            if (FINAL) {
                if (sc < bv[r]) { b2[r] = bv[r]; bv[r] = sc; bi[r] = col; } else { b2[r] = fminf(b2[r], sc); }
            } else if (sc < bv[r]) {
                bv[r] = sc;
                bi[r] = col;
            }
        }
    }
}

template <typename T, int D, bool FINAL>
__global__ void __launch_bounds__(FF_THREADS, FfCfg<D>::MIN_BLOCKS)
    k_assign_ffma(CandBatch b, const T* __restrict__ Z, int64_t n, KmState st, int pass, float band, int2* recheck,
                  int* recheck_count) {
    using C = FfCfg<D>;
    extern __shared__ float4 ff_smem4[];
    float* zT = reinterpret_cast<float*>(ff_smem4);
    float* chunk0 = zT + C::ZT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pr = lane >> 3, cr = lane & 7;
    const int64_t p0 = (int64_t)blockIdx.x * FF_PTS;

    int c = -1, q = 0;
    bool has = ff_next(b, st.active, FINAL, c, q);
    if (!has) return;
    ff_load_chunk<D>(chunk0, st, b.off[c], tid);

    // the point tile, transposed: thread t reads 16 bytes of row p and writes 4 or 8 coordinates
    {
        constexpr int E = Vec<T>::E;   // elements per 16 bytes
        for (int t = tid; t < FF_PTS * (D / E); t += FF_THREADS) {
            const int p = t % FF_PTS, k0 = (t / FF_PTS) * E;
            float v[E];
            if (p0 + p < n) {
                Vec<T>::load(Z + (p0 + p) * D + k0, v);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = 0.f;
            }
#pragma unroll
            for (int e = 0; e < E; ++e) zT[(k0 + e) * FF_PTS + p] = v[e];
        }
    }

    float bv[8], b2[8];
    int bi[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) { bv[r] = INFINITY; b2[r] = INFINITY; bi[r] = 0x7fffffff; }
    const float* zw = zT + 32 * warp;
    int buf = 0;
    while (has) {
        int cn = c, qn = q;
        const bool hn = ff_next(b, st.active, FINAL, cn, qn);
        const int nbuf = buf + 1 == C::BUFS ? 0 : buf + 1;
        if (hn) {
            // three buffers: the one refilled here was last read two chunks ago, before the
            // previous barrier; two buffers: the barrier at the end of the previous chunk
            ff_load_chunk<D>(chunk0 + nbuf * C::CHUNK, st, b.off[cn] + qn * FF_CH, tid);
            ff_wait_but_one();
        } else {
            ff_wait_all();
        }
        __syncthreads();   // this chunk's copies, issued by every thread, have landed
        const float* mT = chunk0 + buf * C::CHUNK;
        // a candidate's last chunk with at most 32 real centroids: only the first half
        if (b.k[c] - q * FF_CH > 32) ff_chunk<D, FINAL, 8>(zw, mT, pr, cr, q, bv, b2, bi);
        else ff_chunk<D, FINAL, 4>(zw, mT, pr, cr, q, bv, b2, bi);
        if (!hn || cn != c) {
            // candidate c is complete: combine the 8 lanes of each point group (ties to the
            // lowest column), then lane cr reports point cr of the group
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float ov = __shfl_xor_sync(0xffffffffu, bv[r], o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi[r], o);
                    if (FINAL) {
                        const float o2 = __shfl_xor_sync(0xffffffffu, b2[r], o);
                        b2[r] = fminf(fminf(b2[r], o2), fmaxf(bv[r], ov));
                    }
                    if (ov < bv[r] || (ov == bv[r] && oi < bi[r])) { bv[r] = ov; bi[r] = oi; }
                }
            }
            float mv = INFINITY, m2 = INFINITY;
            int mi = 0x7fffffff;
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (r == cr) { mv = bv[r]; m2 = b2[r]; mi = bi[r]; }
            const int p = 32 * warp + (cr < 4 ? 4 * pr + cr : 16 + 4 * pr + (cr - 4));
            const int64_t i = p0 + p;
            const int K = b.k[c], off = b.off[c];
            int nl = mi;
            if (nl < 0 || nl >= K) nl = 0;   // every score NaN (non-finite input): keep indices in range
            bool changed = false;
            if (i < n) {
                int16_t* lp = st.labels + i * b.cs + c;
                if (FINAL) {
                    *lp = (int16_t)nl;
                    if (!(m2 - mv > band)) {
                        const int slot = atomicAdd(recheck_count, 1);
                        recheck[slot] = make_int2((int)i, c);
                    }
                } else {
                    const int ol = *lp;
                    if (nl != ol) {
                        changed = true;
                        *lp = (int16_t)nl;
                        atomicAdd(st.counts + off + nl, 1);
                        if (ol >= 0) atomicSub(st.counts + off + ol, 1);
                        long long* sn = st.sums + (int64_t)(off + nl) * D;
                        long long* so = ol >= 0 ? st.sums + (int64_t)(off + ol) * D : nullptr;
#pragma unroll 4
                        for (int k = 0; k < D; ++k) {
                            const long long v = __float2ll_rn(zT[k * FF_PTS + p] * FIXED_SCALE_F);
                            atomicAdd(reinterpret_cast<unsigned long long*>(sn + k), (unsigned long long)v);
                            if (so) atomicAdd(reinterpret_cast<unsigned long long*>(so + k), (unsigned long long)(-v));
                        }
                    }
                }
            }
            if (!FINAL) {
                const int cnt = __popc(__ballot_sync(0xffffffffu, changed));
                if (lane == 0 && cnt) atomicAdd(st.changed + (pass & 1) * MAXC + c, cnt);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) { bv[r] = INFINITY; b2[r] = INFINITY; bi[r] = 0x7fffffff; }
        }
        if (C::BUFS == 2) __syncthreads();   // every warp is done with this buffer before it is refilled
        c = cn;
        q = qn;
        has = hn;
        buf = nbuf;
    }
}

template <typename T, int D, bool FINAL>
static cudaError_t launch_ff_t(const CandBatch& b, const T* Z, int64_t n, KmState st, int pass, float band,
                               int2* recheck, int* recheck_count, cudaStream_t s) {
    using C = FfCfg<D>;
    auto kern = k_assign_ffma<T, D, FINAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + FF_PTS - 1) / FF_PTS;
    ProfScope ps(s, FINAL ? PF_ASSIGN_FFMA_FINAL : PF_ASSIGN_FFMA, 1);
    kern<<<(unsigned)tiles, FF_THREADS, C::SMEM, s>>>(b, Z, n, st, pass, band, recheck, recheck_count);
    return cudaGetLastError();
}

// Error band of the final assignment's scores (near ties inside it are re-checked in FP64).
// Each score s_c = fmaf(-2, a_c, n_c) approximates t_c = ||mu_c||^2 - 2 z.mu_c from the FP32
// inputs (exact: z and mu_c are the stored values).  With u = 2^-24, unit rows (||z|| <= 1) and
// centroids of norm <= 1 (means of such rows):
//   a_c, d fused multiply-adds in sequence:      |a_c - z.mu_c|       <= d u (1 + d u)
//   n_c, d fused multiply-adds of squares:       |n_c - ||mu_c||^2|   <= d u (1 + d u)
//   the final fmaf, |s_c| <= 4:                   one rounding         <= 4 u
// so |s_c - t_c| <= 3 d u (1 + d u) + 4 u =: E, and two scores whose exact order differs from
// their computed order lie within 2E.  The band is 2E with a 25% margin (which also covers the
// FP64 re-check's own rounding, below 1e-13).
float ffma_tie_band(int d) {
    const double u = 1.0 / 16777216.0;
    const double E = 3.0 * d * u * (1.0 + d * u) + 4.0 * u;
    return (float)(2.5 * E);
}

cudaError_t launch_assign_ffma(const CandBatch& b, const void* Z, int zdtype, int64_t n, int d, KmState st, int pass,
                               int final_mode, int2* recheck, int* recheck_count, cudaStream_t s) {
    const float band = ffma_tie_band(d);
#define RAFTGP_FF_CASE(TT, DD)                                                                                 \
    case DD:                                                                                                   \
        return final_mode ? launch_ff_t<TT, DD, true>(b, (const TT*)Z, n, st, pass, band, recheck, recheck_count, s) \
                          : launch_ff_t<TT, DD, false>(b, (const TT*)Z, n, st, pass, band, recheck, recheck_count, s);
    if (zdtype == RAFTGP_BF16) {
        switch (d) {
            RAFTGP_FF_CASE(__nv_bfloat16, 32)
            RAFTGP_FF_CASE(__nv_bfloat16, 64)
            RAFTGP_FF_CASE(__nv_bfloat16, 128)
        }
    } else {
        switch (d) {
            RAFTGP_FF_CASE(float, 32)
            RAFTGP_FF_CASE(float, 64)
            RAFTGP_FF_CASE(float, 128)
        }
    }
#undef RAFTGP_FF_CASE
    return cudaErrorInvalidValue;
}

}  // namespace raftgp
