// diff.cu -- the differentiation form: forward and backward of one Eq. 6 GCN layer, a relaxed
// soft-assignment modularity loss with its gradient, an Adam step, and centroids from labels.
//
// Layer (FP32 storage, FP32 arithmetic; sums over many points end in FP64: the weight
// gradient's block partials are added in FP64, the loss adds FP32 sums of eight rows in FP64):
//     P = H W,  A = Ahat P,  T = tanh(A),  H' = T / ||T||_row          (a zero row stays 0)
//     Ahat = Dhat^-1/2 (A + I) Dhat^-1/2, dhat = d + 1
// Backward with recomputation (only the layer input is kept): P and A are computed again,
//     dT = (dH' - H' (H' . dH')) / ||T||,  dA = dT (1 - T^2),  dP = Ahat dA  (Ahat symmetric),
//     dW = H^T dP,  dH = dP W^T.
// Loss against fixed centroids mu (K <= 128), temperature tau:
//     S_i = softmax_c(-||z_i - mu_c||^2 / tau),  L = -(tr(S^T A S) - ||d^T S||^2 / 2e) / 2e,
//     dL/dS = -(A S - d (d^T S) / 2e) / e,  dL/dD = -S (dL/dS - rowsum(S dL/dS)) / tau,
//     dL/dz_i = 2 (sum_c G_ic) z_i - 2 sum_c G_ic mu_c.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

// ------------------------------------------------------------------------------------
// Y = X W (TRANS: X W^T), X: n x LIN (16-byte aligned), W: LIN x LOUT (TRANS: LOUT x LIN),
// row-major.  W stays in shared memory, k-major; X comes in tiles of TR rows, KC columns at a
// time, by cp.async into two buffers (rows padded to KC + 4 floats).  Thread (ty, tx) owns
// rows ty + TYN i (i < 8) and columns 4 tx + 4 TXN g + q (g < 2, q < 4), reading X two
// columns at a time: a warp's 8- and 16-byte shared reads fall in distinct banks.  Every
// output is fmaf over ascending k from zero.
// ------------------------------------------------------------------------------------
template <int LIN, int LOUT>
struct RmCfg {
    static constexpr int TXN = LOUT / 8;   // column threads: 16, 8, 4
    static constexpr int TYN = 256 / TXN;  // row threads: 16, 32, 64
    static constexpr int TR = 8 * TYN;     // rows per tile: 128, 256, 512
    static constexpr int KC = 4096 / TR;   // X columns per stage: 32, 16, 8
    static constexpr int KCP = KC + 4;     // padded stage row, floats
    static constexpr int NCH = LIN / KC;   // stages per tile
    static constexpr int BUF = TR * KCP;   // floats per stage buffer
    static constexpr int SMEM = (LIN * LOUT + 2 * BUF) * (int)sizeof(float);
    static_assert(KC <= LIN && LIN % KC == 0, "stage width");
    static_assert((TR * KC / 4) % 256 == 0, "stage pieces per thread");
};

__device__ __forceinline__ void rm_cp16(float* dst, const float* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}

// Stage (rows r0.., columns k0..k0+KC) of X into buf; rows at or past n are zero-filled.
template <int LIN, int LOUT>
__device__ __forceinline__ void rm_stage(float* buf, const float* __restrict__ X, int64_t n, int64_t r0, int k0) {
    using C = RmCfg<LIN, LOUT>;
    constexpr int P = C::KC / 4;   // 16-byte pieces per stage row
#pragma unroll
    for (int u = 0; u < C::TR * P / 256; ++u) {
        const int t = threadIdx.x + 256 * u;
        const int r = t / P, j = t % P;
        const bool ok = r0 + r < n;
        rm_cp16(buf + r * C::KCP + 4 * j, ok ? X + (r0 + r) * LIN + k0 + 4 * j : X, ok ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int LIN, int LOUT, bool TRANS>
__global__ void __launch_bounds__(256, 2) k_rowmm(int64_t n, const float* __restrict__ X, const float* __restrict__ W,
                                                  float* __restrict__ Y) {
    using C = RmCfg<LIN, LOUT>;
    extern __shared__ __align__(16) float sm[];
    float* sW = sm;                    // LIN x LOUT, k-major
    float* sX = sm + LIN * LOUT;       // two stage buffers
    const int64_t tiles = (n + C::TR - 1) / C::TR;
    if ((int64_t)blockIdx.x >= tiles) return;
    const int64_t steps = (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x * C::NCH;
    rm_stage<LIN, LOUT>(sX, X, n, (int64_t)blockIdx.x * C::TR, 0);
    for (int t = threadIdx.x; t < LIN * LOUT; t += 256) {
        const int k = t / LOUT, c = t % LOUT;
        sW[t] = TRANS ? W[(int64_t)c * LIN + k] : W[t];
    }
    const int ty = threadIdx.x / C::TXN, tx = threadIdx.x % C::TXN;
    float acc[8][8];
    for (int64_t s = 0; s < steps; ++s) {
        const int ch = (int)(s % C::NCH);
        const int64_t r0 = ((int64_t)blockIdx.x + (s / C::NCH) * gridDim.x) * C::TR;
        if (s + 1 < steps) {
            const int64_t s1 = s + 1;
            rm_stage<LIN, LOUT>(sX + (s1 & 1) * C::BUF, X, n,
                                ((int64_t)blockIdx.x + (s1 / C::NCH) * gridDim.x) * C::TR, (int)(s1 % C::NCH) * C::KC);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        if (ch == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        }
        const float* xb = sX + (s & 1) * C::BUF;
        for (int kk = 0; kk < C::KC; kk += 2) {
            float2 xa[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) xa[i] = *reinterpret_cast<const float2*>(xb + (ty + C::TYN * i) * C::KCP + kk);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float* wr = sW + (ch * C::KC + kk + q) * LOUT + 4 * tx;
                const float4 w0 = *reinterpret_cast<const float4*>(wr);
                const float4 w1 = *reinterpret_cast<const float4*>(wr + 4 * C::TXN);
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float xv = q == 0 ? xa[i].x : xa[i].y;
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv, wv[j], acc[i][j]);
                }
            }
        }
        if (ch == C::NCH - 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t r = r0 + ty + C::TYN * i;
                if (r < n) {
                    float* o = Y + r * LOUT + 4 * tx;
                    *reinterpret_cast<float4*>(o) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                    *reinterpret_cast<float4*>(o + 4 * C::TXN) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
                }
            }
        }
        __syncthreads();   // this buffer is free before the stage two steps on is copied into it
    }
}

// ------------------------------------------------------------------------------------
// Warp-per-row SpMM over FP32 rows of width L (a multiple of 32; each lane VW = L/32
// consecutive columns), eight neighbour rows in flight per lane.  Modes:
//   SP_GCN_FWD  out = rownorm(tanh(rsh_i (rsh_i x_i + sum_j rsh_j x_j)))
//   SP_GCN_BWD  the same T, r, H' recomputed, then with g = dH'_i:
//               out = (g - H' (H'.g)) / r * (1 - T^2)            (dA of the layer)
//   SP_LINEAR   out = rsh_i (rsh_i x_i + sum_j rsh_j x_j)       (Ahat x)
//   SP_ADJ      out = sum_j x_j                                  (A x)
// ------------------------------------------------------------------------------------
enum SpMode { SP_GCN_FWD = 0, SP_GCN_BWD = 1, SP_LINEAR = 2, SP_ADJ = 3 };

// VW consecutive floats of one row as a single 4-, 8- or 16-byte access.
template <int VW>
struct RowPiece {
    __device__ __forceinline__ static void load(const float* p, float* o) {
        if constexpr (VW == 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p));
            o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
        } else if constexpr (VW == 2) {
            const float2 v = __ldg(reinterpret_cast<const float2*>(p));
            o[0] = v.x; o[1] = v.y;
        } else {
            o[0] = __ldg(p);
        }
    }
    // read once: evict first
    __device__ __forceinline__ static void load_once(const float* p, float* o) {
        if constexpr (VW == 4) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
            o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
        } else if constexpr (VW == 2) {
            const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
            o[0] = v.x; o[1] = v.y;
        } else {
            o[0] = __ldcs(p);
        }
    }
    // STREAM: evict-first store, for outputs that no later pass gathers from
    template <bool STREAM>
    __device__ __forceinline__ static void store(float* p, const float* v) {
        if constexpr (VW == 4) {
            const float4 x = make_float4(v[0], v[1], v[2], v[3]);
            if constexpr (STREAM) __stcs(reinterpret_cast<float4*>(p), x); else *reinterpret_cast<float4*>(p) = x;
        } else if constexpr (VW == 2) {
            const float2 x = make_float2(v[0], v[1]);
            if constexpr (STREAM) __stcs(reinterpret_cast<float2*>(p), x); else *reinterpret_cast<float2*>(p) = x;
        } else {
            if constexpr (STREAM) __stcs(p, v[0]); else p[0] = v[0];
        }
    }
};


template <typename OffT, int VW, int MODE>
__global__ void __launch_bounds__(256) k_spmm32(Csr<OffT> g, const float* __restrict__ rsh, const float* __restrict__ X,
                                                const float* __restrict__ G, float* __restrict__ out) {
    constexpr int L = 32 * VW;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < g.n; i += warps) {
        float acc[VW];
        const float wi = MODE == SP_ADJ ? 0.f : __ldg(rsh + i);
        if constexpr (MODE == SP_ADJ) {
#pragma unroll
            for (int v = 0; v < VW; ++v) acc[v] = 0.f;
        } else {
            RowPiece<VW>::load(X + i * L + lane * VW, acc);
#pragma unroll
            for (int v = 0; v < VW; ++v) acc[v] = wi * acc[v];
        }
        const int64_t b = g.begin(i), e = g.end(i);
        int64_t p = b;
        for (; p + 8 <= e; p += 8) {
            int j[8];
            float w[8], x[8][VW];
#pragma unroll
            for (int u = 0; u < 8; ++u) j[u] = __ldg(g.col + p + u);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                w[u] = MODE == SP_ADJ ? 1.f : __ldg(rsh + j[u]);
                RowPiece<VW>::load(X + (int64_t)j[u] * L + lane * VW, x[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < VW; ++v) acc[v] = fmaf(w[u], x[u][v], acc[v]);
        }
        for (; p < e; ++p) {
            const int j = __ldg(g.col + p);
            const float w = MODE == SP_ADJ ? 1.f : __ldg(rsh + j);
            float x[VW];
            RowPiece<VW>::load(X + (int64_t)j * L + lane * VW, x);
#pragma unroll
            for (int v = 0; v < VW; ++v) acc[v] = fmaf(w, x[v], acc[v]);
        }
        float* o = out + i * L + lane * VW;
        if constexpr (MODE == SP_ADJ) {
            RowPiece<VW>::template store<true>(o, acc);
            continue;
        } else {
#pragma unroll
            for (int v = 0; v < VW; ++v) acc[v] *= wi;
        }
        if constexpr (MODE == SP_LINEAR) {
            RowPiece<VW>::template store<true>(o, acc);
            continue;
        }
        float T[VW], ss = 0.f;
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            T[v] = tanhf(acc[v]);
            ss = fmaf(T[v], T[v], ss);
        }
        ss = warp_sum(ss);
        const float r = sqrtf(ss);
        if (MODE == SP_GCN_FWD) {
            const float inv = r > 0.f ? 1.0f / r : 0.f;
            float h[VW];
#pragma unroll
            for (int v = 0; v < VW; ++v) h[v] = T[v] * inv;
            RowPiece<VW>::template store<true>(o, h);
        } else {
            float H[VW], gv[VW], dot = 0.f;
            const float inv = r > 0.f ? 1.0f / r : 0.f;
            RowPiece<VW>::load_once(G + i * L + lane * VW, gv);
#pragma unroll
            for (int v = 0; v < VW; ++v) {
                H[v] = T[v] * inv;
                dot = fmaf(H[v], gv[v], dot);
            }
            dot = warp_sum(dot);
            float d[VW];
#pragma unroll
            for (int v = 0; v < VW; ++v) d[v] = (gv[v] - H[v] * dot) * inv * (1.0f - T[v] * T[v]);
            RowPiece<VW>::template store<false>(o, d);   // dA: the next pass gathers it
        }
    }
}

// ------------------------------------------------------------------------------------
// dW = H^T dP over all rows: each block sums a contiguous row range into a LIN x LOUT FP32
// partial (thread owns an 8 x 8 (or smaller) tile), then one kernel adds the partials in
// block order in FP64.
// ------------------------------------------------------------------------------------
// Thread (ta, tb) owns rows {V ta + 16 V g + q} of dW (V = min(LIN / 16, 4) consecutive rows
// per group, LIN / 16 / V groups) and the same pattern of columns over LOUT: every shared read
// is a 16-byte (8-byte for width 32) piece, and a warp's pieces fall in distinct banks.
template <int W>
struct WgMap {
    static constexpr int T = W / 16;             // values per thread: 8, 4, 2
    static constexpr int V = T >= 4 ? 4 : T;     // consecutive values per group
    static constexpr int G = T / V;              // groups
    __device__ __forceinline__ static int idx(int t, int x) { return V * t + 16 * V * (x / V) + x % V; }
    __device__ __forceinline__ static void load(const float* row, int t, float* out) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float* p = row + V * t + 16 * V * g;
            if constexpr (V == 4) {
                const float4 v = *reinterpret_cast<const float4*>(p);
                out[4 * g] = v.x; out[4 * g + 1] = v.y; out[4 * g + 2] = v.z; out[4 * g + 3] = v.w;
            } else {
                const float2 v = *reinterpret_cast<const float2*>(p);
                out[2 * g] = v.x; out[2 * g + 1] = v.y;
            }
        }
    }
};

template <int LIN, int LOUT>
__global__ void __launch_bounds__(256) k_wgrad(int64_t n, int64_t rows_per_block, const float* __restrict__ H,
                                               const float* __restrict__ dP, float* __restrict__ partial) {
    using MA = WgMap<LIN>;
    using MB = WgMap<LOUT>;
    constexpr int TA = MA::T, TB = MB::T;
    __shared__ __align__(16) float sH[32][LIN];
    __shared__ __align__(16) float sP[32][LOUT];
    const int ta = threadIdx.x / 16, tb = threadIdx.x % 16;
    float acc[TA][TB];
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int c = 0; c < TB; ++c) acc[a][c] = 0.f;
    const int64_t lo = (int64_t)blockIdx.x * rows_per_block;
    const int64_t hi = lo + rows_per_block < n ? lo + rows_per_block : n;
    for (int64_t r0 = lo; r0 < hi; r0 += 32) {
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * LIN / 4; t += 256) {
            const int r = t / (LIN / 4), k = 4 * (t % (LIN / 4));
            *reinterpret_cast<float4*>(&sH[r][k]) =
                r0 + r < hi ? __ldg(reinterpret_cast<const float4*>(H + (r0 + r) * LIN + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int t = threadIdx.x; t < 32 * LOUT / 4; t += 256) {
            const int r = t / (LOUT / 4), k = 4 * (t % (LOUT / 4));
            *reinterpret_cast<float4*>(&sP[r][k]) =
                r0 + r < hi ? __ldg(reinterpret_cast<const float4*>(dP + (r0 + r) * LOUT + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 2
        for (int r = 0; r < 32; ++r) {
            float a[TA], b[TB];
            MA::load(sH[r], ta, a);
            MB::load(sP[r], tb, b);
#pragma unroll
            for (int x = 0; x < TA; ++x)
#pragma unroll
                for (int y = 0; y < TB; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
    }
    float* out = partial + (int64_t)blockIdx.x * LIN * LOUT;
#pragma unroll
    for (int x = 0; x < TA; ++x)
#pragma unroll
        for (int y = 0; y < TB; ++y) out[MA::idx(ta, x) * LOUT + MB::idx(tb, y)] = acc[x][y];
}

// dW from the block partials: 32 entries per CTA, each entry's blocks cut into SP_SEG
// contiguous ranges, a warp per range (lane = entry, so every read is 128 contiguous bytes);
// a range is summed in four FP64 chains (block b of the range into chain b mod 4, joined as
// (s0 + s1) + (s2 + s3)), then the ranges are added in order: a fixed order for a given block
// count.
constexpr int SP_SEG = 8;
__global__ void __launch_bounds__(256) k_sum_partials(const float* __restrict__ partial, int blocks, int count,
                                                      float* __restrict__ out) {
    __shared__ double part[SP_SEG][32];
    const int e = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + e;
    const int per = (blocks + SP_SEG - 1) / SP_SEG;
    const int b0 = seg * per, b1 = min(blocks, b0 + per);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (t < count) {
        int b = b0;
        for (; b + 4 <= b1; b += 4) {
            s0 += (double)partial[(int64_t)b * count + t];
            s1 += (double)partial[(int64_t)(b + 1) * count + t];
            s2 += (double)partial[(int64_t)(b + 2) * count + t];
            s3 += (double)partial[(int64_t)(b + 3) * count + t];
        }
        for (; b < b1; ++b) s0 += (double)partial[(int64_t)b * count + t];
    }
    part[seg][e] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (seg == 0 && t < count) {
        double s = 0.0;
        for (int k = 0; k < SP_SEG; ++k) s += part[k][e];
        out[t] = (float)s;
    }
}

// ------------------------------------------------------------------------------------
// Soft assignment: warp per point, lane owns centroids lane + 32u (u < 4); distances in
// ascending coordinates; S written as n x 128 (zeros past K).
// ------------------------------------------------------------------------------------
constexpr int SK = 128;   // padded soft-assignment width

// Squared distances from z (registers) to the lane's centroids lane + 32 u, u < NU, each over
// ascending coordinates; the coordinate loop is unrolled in full so z stays in registers
// (lanes past K read row K - 1 and their sums are discarded).
template <int D, int NU>
__device__ __forceinline__ void sa_dist(const float* z, const float* smu, int lane, int K, float* s) {
    constexpr int DP = D + 1;
    int row[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        row[u] = min(lane + 32 * u, K - 1) * DP;
        s[u] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const float t = z[k] - smu[row[u] + k];
            s[u] = fmaf(t, t, s[u]);
        }
}

template <int D>
__global__ void __launch_bounds__(256) k_soft_assign(int64_t n, const float* __restrict__ Z, const float* __restrict__ mu,
                                                     int K, float tau, float* __restrict__ S) {
    // K rows of D + 1 floats: lane c reads row c, so the padded stride puts the 32 lanes'
    // words in 32 different banks
    constexpr int DP = D + 1;
    extern __shared__ float smu[];   // K x DP
    for (int t = threadIdx.x; t < K * D; t += blockDim.x) smu[(t / D) * DP + t % D] = mu[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nu = (K + 31) / 32;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        float z[D];
#pragma unroll
        for (int k = 0; k < D; k += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(Z + i * D + k));
            z[k] = v.x; z[k + 1] = v.y; z[k + 2] = v.z; z[k + 3] = v.w;
        }
        float sq[4] = {0.f, 0.f, 0.f, 0.f};
        switch (nu) {
            case 1: sa_dist<D, 1>(z, smu, lane, K, sq); break;
            case 2: sa_dist<D, 2>(z, smu, lane, K, sq); break;
            case 3: sa_dist<D, 3>(z, smu, lane, K, sq); break;
            default: sa_dist<D, 4>(z, smu, lane, K, sq); break;
        }
        float lg[4], mx = -INFINITY;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            lg[u] = -INFINITY;
            if (lane + 32 * u < K) {
                lg[u] = -sq[u] / tau;
                mx = fmaxf(mx, lg[u]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float e[4], sum = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            e[u] = lane + 32 * u < K ? expf(lg[u] - mx) : 0.f;
            sum += e[u];
        }
        sum = warp_sum(sum);
        const float inv = 1.0f / sum;
#pragma unroll
        for (int u = 0; u < 4; ++u) S[i * SK + lane + 32 * u] = e[u] * inv;
    }
}

// Per-block FP64 partials of d^T S (SK columns) and of sum_i S_i . (AS)_i (column SK).  Each
// lane adds its products in FP32 over eight of its warp's rows, then moves that short sum into
// its FP64 totals: FP64 runs at a small fraction of the FP32 rate here, and one FP64 update per
// product made this kernel arithmetic-bound.
__global__ void __launch_bounds__(256) k_softmod_partials(int64_t n, const int32_t* __restrict__ deg,
                                                          const float* __restrict__ S, const float* __restrict__ AS,
                                                          int64_t rows_per_block, double* __restrict__ partial) {
    __shared__ double sdts[8][SK];
    __shared__ double sq[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double dts[4] = {0, 0, 0, 0}, q = 0.0;
    float fd[4] = {0.f, 0.f, 0.f, 0.f}, fq = 0.f;
    int rows = 0;
    const int64_t lo = (int64_t)blockIdx.x * rows_per_block;
    const int64_t hi = lo + rows_per_block < n ? lo + rows_per_block : n;
    for (int64_t i = lo + w; i < hi; i += 8) {
        const float di = (float)__ldg(deg + i);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float s = __ldg(S + i * SK + lane + 32 * u);
            fd[u] = fmaf(di, s, fd[u]);
            fq = fmaf(s, __ldg(AS + i * SK + lane + 32 * u), fq);
        }
        if (++rows == 8) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                dts[u] += (double)fd[u];
                fd[u] = 0.f;
            }
            q += (double)fq;
            fq = 0.f;
            rows = 0;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) dts[u] += (double)fd[u];
    q += (double)fq;
#pragma unroll
    for (int u = 0; u < 4; ++u) sdts[w][lane + 32 * u] = dts[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) sq[w] = q;
    __syncthreads();
    // column-major partials: column c of block b at partial[c * gridDim.x + b]
    for (int c = threadIdx.x; c < SK; c += blockDim.x) {
        double s = 0.0;
        for (int ww = 0; ww < 8; ++ww) s += sdts[ww][c];
        partial[(int64_t)c * gridDim.x + blockIdx.x] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int ww = 0; ww < 8; ++ww) s += sq[ww];
        partial[(int64_t)SK * gridDim.x + blockIdx.x] = s;
    }
}

// Adds the block partials, one warp per column: lane l takes blocks l, l + 32, ... in order,
// then the lanes' sums meet in a butterfly (every lane ends with the same total), a fixed
// order at any launch.  red[0..SK) = d^T S, red[SK] = sum S . AS; then red[SK + 1] = the loss
// -(sum S . AS - ||d^T S||^2 / 2e) / 2e, the squares added over ascending blocks c < K with
// every product and sum rounded on its own.
__global__ void __launch_bounds__(1024) k_softmod_finish(const double* __restrict__ partial, int blocks, int K,
                                                         double two_e, double* __restrict__ red) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = threadIdx.x >> 5; c <= SK; c += nw) {
        double s = 0.0;
        for (int b = lane; b < blocks; b += 32) s += partial[(int64_t)c * blocks + b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double dd = 0.0;
        for (int c = 0; c < K; ++c) dd = __dadd_rn(dd, __dmul_rn(red[c], red[c]));
        red[SK + 1] = -__ddiv_rn(__dsub_rn(red[SK], __ddiv_rn(dd, two_e)), two_e);
    }
}

// dL/dZ for tiles of SG_TP nodes.  Phase 1, a warp per node: G_i = -S_i (g_i - S_i . g_i) / tau
// with g_i = -(AS_i - d_i d^T S / 2e) / e, into shared memory with the node's sum of G.
// Phase 2: M = G mu for the tile from register tiles (thread: SG_TP / PG nodes x 8 coordinates
// 4 cg + 4 CG h + q, so a warp's 16-byte reads of mu fall in distinct banks; the G rows have an
// odd stride), each entry fmaf over ascending c from zero; then dZ = 2 (sum G z - M).
constexpr int SG_TP = 64;

template <int D>
__global__ void __launch_bounds__(256) k_softmod_grad(int64_t n, const float* __restrict__ Z, const float* __restrict__ mu,
                                                      int K, float tau, const int32_t* __restrict__ deg,
                                                      const float* __restrict__ S, const float* __restrict__ AS,
                                                      const double* __restrict__ red, double two_e,
                                                      float* __restrict__ dZ) {
    constexpr int CG = D / 8, PG = 256 / CG, PPT = SG_TP / PG;
    const int KP = K + ((K & 1) ? 2 : 1);   // odd row stride of the G tile
    extern __shared__ __align__(16) float smu[];   // K x D, SK values of d^T S / 2e, G tile, sums
    float* sdts = smu + K * D;
    float* sG = sdts + SK;
    float* sgs = sG + SG_TP * KP;
    for (int t = threadIdx.x; t < K * D; t += blockDim.x) smu[t] = mu[t];
    for (int c = threadIdx.x; c < SK; c += blockDim.x) sdts[c] = (float)(red[c] / two_e);
    const float inv_e = (float)(2.0 / two_e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cg = threadIdx.x % CG, pg = threadIdx.x / CG;
    const int64_t tiles = (n + SG_TP - 1) / SG_TP;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t t0 = tile * SG_TP;
        __syncthreads();   // the previous tile's G is consumed (and mu is in place)
        for (int pp = warp; pp < SG_TP; pp += 8) {
            const int64_t i = t0 + pp;
            if (i >= n) break;
            const float di = (float)__ldg(deg + i);
            float s[4], gs[4], sdot = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = lane + 32 * u;
                s[u] = __ldg(S + i * SK + c);
                gs[u] = c < K ? -(__ldg(AS + i * SK + c) - di * sdts[c]) * inv_e : 0.f;
                sdot = fmaf(s[u], gs[u], sdot);
            }
            sdot = warp_sum(sdot);
            float G[4], gsum = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                G[u] = -s[u] * (gs[u] - sdot) / tau;
                gsum += G[u];
            }
            gsum = warp_sum(gsum);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (lane + 32 * u < K) sG[pp * KP + lane + 32 * u] = G[u];
            if (lane == 0) sgs[pp] = gsum;
        }
        __syncthreads();
        float m[PPT][8];
#pragma unroll
        for (int a = 0; a < PPT; ++a)
#pragma unroll
            for (int j = 0; j < 8; ++j) m[a][j] = 0.f;
        for (int c = 0; c < K; ++c) {
            const float4 b0 = *reinterpret_cast<const float4*>(smu + c * D + 4 * cg);
            const float4 b1 = *reinterpret_cast<const float4*>(smu + c * D + 4 * CG + 4 * cg);
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < PPT; ++a) {
                const float g = sG[(pg + PG * a) * KP + c];
#pragma unroll
                for (int j = 0; j < 8; ++j) m[a][j] = fmaf(g, bv[j], m[a][j]);
            }
        }
#pragma unroll
        for (int a = 0; a < PPT; ++a) {
            const int pp = pg + PG * a;
            const int64_t i = t0 + pp;
            if (i < n) {
                const float gsum = sgs[pp];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k0 = 4 * cg + 4 * CG * h;
                    const float4 z = __ldg(reinterpret_cast<const float4*>(Z + i * D + k0));
                    float4 o;
                    o.x = 2.0f * (gsum * z.x - m[a][4 * h]);
                    o.y = 2.0f * (gsum * z.y - m[a][4 * h + 1]);
                    o.z = 2.0f * (gsum * z.z - m[a][4 * h + 2]);
                    o.w = 2.0f * (gsum * z.w - m[a][4 * h + 3]);
                    *reinterpret_cast<float4*>(dZ + i * D + k0) = o;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Adam (Kingma and Ba, 2015), FP32 state.
// ------------------------------------------------------------------------------------
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t count, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.0f - b1) * gt;
        const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    }
}

// ------------------------------------------------------------------------------------
// Centroids of a labelling: exact 2^-40 fixed-point sums (int64 atomics, order-free), FP64
// means; an empty cluster gets a zero row.
// ------------------------------------------------------------------------------------
__global__ void k_centroid_sums(int64_t n, int d, const float* __restrict__ Z, const int32_t* __restrict__ labels,
                                int K, long long* __restrict__ sums, int* __restrict__ counts, uint32_t* err) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * d; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / d;
        const int k = (int)(t % d);
        const int l = labels[i];
        if (l < 0 || l >= K) {
            if (k == 0) flag_error(err, DERR_LABEL_RANGE);
            continue;
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(sums + (int64_t)l * d + k),
                  (unsigned long long)__float2ll_rn(Z[t] * FIXED_SCALE_F));
        if (k == 0) atomicAdd(counts + l, 1);
    }
}

__global__ void k_centroid_means(int K, int d, const long long* __restrict__ sums, const int* __restrict__ counts,
                                 float* __restrict__ mu) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < K * d; t += gridDim.x * blockDim.x) {
        const int c = t / d;
        mu[t] = counts[c] > 0 ? (float)((double)sums[t] / ((double)counts[c] * FIXED_SCALE)) : 0.f;
    }
}

// ------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------
static int grid_for(int64_t warps_needed) {
    const int64_t cap = (int64_t)num_sms() * 16;
    int64_t b = (warps_needed * 32 + 255) / 256;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int LIN, int LOUT, bool TRANS>
static cudaError_t rowmm_t(int64_t n, const float* X, const float* W, float* Y, cudaStream_t s) {
    ProfScope ps(s, PF_DIFF_DENSE, 1);
    using C = RmCfg<LIN, LOUT>;
    const size_t smem = C::SMEM;
    auto kern = k_rowmm<LIN, LOUT, TRANS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + C::TR - 1) / C::TR;
    const int64_t cap = (int64_t)num_sms() * 2;
    if (blocks > cap) blocks = cap;
    kern<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, smem, s>>>(n, X, W, Y);
    return cudaGetLastError();
}

#define RAFTGP_WIDTHS(M)                                                                            \
    M(32, 32) M(32, 64) M(32, 128) M(64, 32) M(64, 64) M(64, 128) M(128, 32) M(128, 64) M(128, 128)

cudaError_t launch_rowmm(int64_t n, const float* X, int lin, const float* W, int lout, bool trans, float* Y,
                         cudaStream_t s) {
#define RAFTGP_RM(A, B)                                                                             \
    if (lin == A && lout == B) return trans ? rowmm_t<A, B, true>(n, X, W, Y, s) : rowmm_t<A, B, false>(n, X, W, Y, s);
    RAFTGP_WIDTHS(RAFTGP_RM)
#undef RAFTGP_RM
    return cudaErrorInvalidValue;
}

// CTAs of two warps, a warp per row: row lengths follow a power law, and small CTAs let the
// block scheduler balance them (a CTA's warp slots stay held until its slowest row is done).
template <typename OffT, int VW, int MODE>
static cudaError_t spmm32_launch(const Csr<OffT>& g, const float* rsh, const float* X, const float* G, float* out,
                                 cudaStream_t s) {
    int64_t blocks = (g.n + 1) / 2;
    if (blocks > (int64_t)INT32_MAX) blocks = INT32_MAX;
    if (blocks < 1) blocks = 1;
    k_spmm32<OffT, VW, MODE><<<(unsigned)blocks, 64, 0, s>>>(g, rsh, X, G, out);
    return cudaGetLastError();
}

template <typename OffT, int VW>
static cudaError_t spmm32_t(const Csr<OffT>& g, const float* rsh, const float* X, const float* G, float* out, int mode,
                            cudaStream_t s) {
    switch (mode) {
        case SP_GCN_FWD: return spmm32_launch<OffT, VW, SP_GCN_FWD>(g, rsh, X, G, out, s);
        case SP_GCN_BWD: return spmm32_launch<OffT, VW, SP_GCN_BWD>(g, rsh, X, G, out, s);
        case SP_LINEAR: return spmm32_launch<OffT, VW, SP_LINEAR>(g, rsh, X, G, out, s);
        default: return spmm32_launch<OffT, VW, SP_ADJ>(g, rsh, X, G, out, s);
    }
}

template <typename OffT>
static cudaError_t spmm32_w(const Csr<OffT>& g, int L, const float* rsh, const float* X, const float* G, float* out,
                            int mode, cudaStream_t s) {
    switch (L) {
        case 32: return spmm32_t<OffT, 1>(g, rsh, X, G, out, mode, s);
        case 64: return spmm32_t<OffT, 2>(g, rsh, X, G, out, mode, s);
        case 128: return spmm32_t<OffT, 4>(g, rsh, X, G, out, mode, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_spmm32(const raftgp_csr* g, int L, const float* rsh, const float* X, const float* G, float* out,
                          int mode, cudaStream_t s) {
    ProfScope ps(s, mode == 3 ? PF_DIFF_LOSS : PF_DIFF_SPMM, 1);
    if (g->row_ptr_bits == 64) {
        Csr<int64_t> c{g->n, g->nnz, (const int64_t*)g->row_ptr, g->col};
        return spmm32_w(c, L, rsh, X, G, out, mode, s);
    }
    Csr<int32_t> c{g->n, g->nnz, (const int32_t*)g->row_ptr, g->col};
    return spmm32_w(c, L, rsh, X, G, out, mode, s);
}

// Two CTAs on every SM (the widest form holds 101 registers a thread), rows split evenly.
int wgrad_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 2;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_wgrad(int64_t n, const float* H, int lin, const float* dP, int lout, float* partial, float* dW,
                         cudaStream_t s) {
    ProfScope ps(s, PF_DIFF_DENSE, 2);
    const int blocks = wgrad_blocks(n);
    const int64_t rpb = (n + blocks - 1) / blocks;
    bool done = false;
#define RAFTGP_WG(A, B)                                                                             \
    if (lin == A && lout == B) {                                                                    \
        k_wgrad<A, B><<<blocks, 256, 0, s>>>(n, rpb, H, dP, partial);                              \
        done = true;                                                                                \
    }
    RAFTGP_WIDTHS(RAFTGP_WG)
#undef RAFTGP_WG
    if (!done) return cudaErrorInvalidValue;
    const int count = lin * lout;
    k_sum_partials<<<(count + 31) / 32, 256, 0, s>>>(partial, blocks, count, dW);
    return cudaGetLastError();
}

int softmod_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 4;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_soft_assign(int64_t n, int d, const float* Z, const float* mu, int K, float tau, float* S,
                               cudaStream_t s) {
    ProfScope ps(s, PF_DIFF_LOSS, 1);
    const size_t smem = (size_t)K * (d + 1) * sizeof(float);   // rows padded to d + 1 floats
    const int blocks = grid_for(n);
    switch (d) {
        case 32: k_soft_assign<32><<<blocks, 256, smem, s>>>(n, Z, mu, K, tau, S); break;
        case 64: k_soft_assign<64><<<blocks, 256, smem, s>>>(n, Z, mu, K, tau, S); break;
        case 128:
            cudaFuncSetAttribute(k_soft_assign<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_soft_assign<128><<<blocks, 256, smem, s>>>(n, Z, mu, K, tau, S);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_softmod_reduce(int64_t n, const int32_t* deg, const float* S, const float* AS, int K,
                                  double two_e, double* partial, double* red, cudaStream_t s) {
    ProfScope ps(s, PF_DIFF_LOSS, 2);
    const int blocks = softmod_blocks(n);
    const int64_t rpb = (n + blocks - 1) / blocks;
    k_softmod_partials<<<blocks, 256, 0, s>>>(n, deg, S, AS, rpb, partial);
    k_softmod_finish<<<1, 1024, 0, s>>>(partial, blocks, K, two_e, red);
    return cudaGetLastError();
}

cudaError_t launch_softmod_grad(int64_t n, int d, const float* Z, const float* mu, int K, float tau, const int32_t* deg,
                                const float* S, const float* AS, const double* red, double two_e, float* dZ,
                                cudaStream_t s) {
    ProfScope ps(s, PF_DIFF_LOSS, 1);
    const int KP = K + ((K & 1) ? 2 : 1);
    const size_t smem = (size_t)(K * d + SK + SG_TP * KP + SG_TP) * sizeof(float);
    int64_t blocks = (n + SG_TP - 1) / SG_TP;
    const int64_t cap = (int64_t)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
#define RAFTGP_SG(DD)                                                                                   if (d == DD) {                                                                                          cudaError_t e = cudaFuncSetAttribute(k_softmod_grad<DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         if (e != cudaSuccess) return e;                                                                     k_softmod_grad<DD><<<(unsigned)blocks, 256, smem, s>>>(n, Z, mu, K, tau, deg, S, AS, red, two_e, dZ);         return cudaGetLastError();                                                                      }
    RAFTGP_SG(32)
    RAFTGP_SG(64)
    RAFTGP_SG(128)
#undef RAFTGP_SG
    return cudaErrorInvalidValue;
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s) {
    ProfScope ps(s, PF_DIFF, 1);
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    int64_t blocks = (count + 255) / 256;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    k_adam<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_centroids(int64_t n, int d, const float* Z, const int32_t* labels, int K, long long* sums,
                             int* counts, float* mu, uint32_t* err, cudaStream_t s) {
    ProfScope ps(s, PF_DIFF, 2);
    cudaMemsetAsync(sums, 0, (size_t)K * d * sizeof(long long), s);
    cudaMemsetAsync(counts, 0, (size_t)K * sizeof(int), s);
    int64_t blocks = (n * d + 255) / 256;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    k_centroid_sums<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(n, d, Z, labels, K, sums, counts, err);
    k_centroid_means<<<(K * d + 255) / 256, 256, 0, s>>>(K, d, sums, counts, mu);
    return cudaGetLastError();
}

}  // namespace raftgp
