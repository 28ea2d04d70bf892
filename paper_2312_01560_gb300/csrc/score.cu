// score.cu -- partition scoring (Eq. 1 NCut, Eq. 3 modularity via Eq. 7 with U = V) and the
// choice of K (Section III-C).
//
// Counting is exact integer work: for every row i and candidate c, the number of neighbours
// j with label_c(j) == label_c(i) is added to m[c][label_c(i)] (directed count, twice the
// undirected m_r), and d_i to vol[c][label_c(i)], with int64 atomics (order-free).
// Finalisation per candidate:
//   Mod  = (2 * (2e) * sum_r m_r - sum_r vol_r^2) / (2e)^2  -- exact int64 numerator and
//          denominator, one IEEE FP64 division
//   NCut = 1/2 * sum_{r ascending, vol_r > 0} (vol_r - 2 m_r) / vol_r  -- FP64
// so both are bit-identical to any other program that evaluates the same expressions.
// Range: the host rejects nnz >= 2^31, so |numerator| and the denominator stay below
// nnz^2 < 2^62 and the int64 terms are exact.  Their conversions to FP64 are exact while they
// are below 2^53 (2e up to about 9.49e7); above that each conversion rounds the exact integer
// once, to nearest, which any program converting the same integers reproduces bit for bit.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

// Batched count over the labels of a candidate batch (labels: N x cs int16).  SMEM: the block
// adds into 32-bit shared counters (every per-block sum is below 2^31 when nnz is) and flushes
// the non-zero ones with one global atomic each, instead of contending on a few hot words.
template <bool SMEM>
__global__ void __launch_bounds__(512) k_score_count(CandBatch b, int64_t n, const int32_t* rp32, const int64_t* rp64,
                                                     const int32_t* col, const int32_t* deg,
                                                     const int16_t* __restrict__ labels, ScoreOut so) {
    extern __shared__ uint32_t s_cnt[];   // SMEM: total_k m counters, then total_k vol counters
    uint32_t* s_m = s_cnt;
    uint32_t* s_vol = s_cnt + b.total_k;
    if (SMEM) {
        for (int t = threadIdx.x; t < 2 * b.total_k; t += blockDim.x) s_cnt[t] = 0;
        __syncthreads();
    }
    auto add_vol = [&](int slot, int v) {
        if (SMEM) atomicAdd(s_vol + slot, (uint32_t)v);
        else atomicAdd(reinterpret_cast<unsigned long long*>(so.vol + slot), (unsigned long long)v);
    };
    auto add_m = [&](int slot, int v) {
        if (SMEM) atomicAdd(s_m + slot, (uint32_t)v);
        else atomicAdd(reinterpret_cast<unsigned long long*>(so.m + slot), (unsigned long long)v);
    };
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const int64_t beg = rp64 ? rp64[i] : rp32[i];
        const int64_t end = rp64 ? rp64[i + 1] : rp32[i + 1];
        const int16_t* li = labels + i * b.cs;
        if (lane < b.n) add_vol(b.off[lane] + li[lane], deg[i]);
        if (lane + 32 < b.n) add_vol(b.off[lane + 32] + li[lane + 32], deg[i]);
        for (int g0 = 0; g0 < b.n; g0 += 8) {
            const uint4 rv = *reinterpret_cast<const uint4*>(li + g0);
            const uint32_t rw[4] = {rv.x, rv.y, rv.z, rv.w};
            int cnt[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) cnt[q] = 0;
            for (int64_t p = beg + lane; p < end; p += 32) {
                const int64_t j = __ldg(col + p);
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(labels + j * b.cs + g0));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t x = w[q] ^ rw[q];
                    cnt[2 * q] += (x & 0xffffu) == 0;
                    cnt[2 * q + 1] += (x >> 16) == 0;
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) cnt[q] = __reduce_add_sync(0xffffffffu, cnt[q]);
            if (lane < 8 && g0 + lane < b.n) {
                int v = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) v = (lane == q) ? cnt[q] : v;
                const int c = g0 + lane;
                if (v) add_m(b.off[c] + li[c], v);
            }
        }
    }
    if (SMEM) {
        __syncthreads();
        for (int t = threadIdx.x; t < b.total_k; t += blockDim.x) {
            if (s_m[t]) atomicAdd(reinterpret_cast<unsigned long long*>(so.m + t), (unsigned long long)s_m[t]);
            if (s_vol[t]) atomicAdd(reinterpret_cast<unsigned long long*>(so.vol + t), (unsigned long long)s_vol[t]);
        }
    }
}

// Block per candidate: the NCut terms (one FP64 division each) in parallel, summed by one
// thread in ascending block order; the integer sums are exact in any order.
constexpr int FIN_THREADS = 256;
constexpr int FIN_CHUNK = 1024;
__global__ void __launch_bounds__(FIN_THREADS) k_score_finalize(CandBatch b, int64_t two_e, ScoreOut so) {
    const int c = blockIdx.x;
    if (c >= b.n) return;
    __shared__ double terms[FIN_CHUNK];
    __shared__ long long s_m[FIN_THREADS / 32], s_v[FIN_THREADS / 32];
    const int K = b.k[c], off = b.off[c];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long msum = 0, vsq = 0;
    double s = 0.0;   // thread 0's running sum, in ascending block order
    for (int r0 = 0; r0 < K; r0 += FIN_CHUNK) {
        const int nr = K - r0 < FIN_CHUNK ? K - r0 : FIN_CHUNK;
        for (int j = threadIdx.x; j < nr; j += FIN_THREADS) {
            const long long m = so.m[off + r0 + j] / 2;
            const long long v = so.vol[off + r0 + j];
            msum += m;
            vsq += v * v;
            terms[j] = v > 0 ? (double)(v - 2 * m) / (double)v : 0.0;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int j = 0; j < nr; ++j) s += terms[j];
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        msum += __shfl_xor_sync(0xffffffffu, msum, o);
        vsq += __shfl_xor_sync(0xffffffffu, vsq, o);
    }
    if (lane == 0) {
        s_m[warp] = msum;
        s_v[warp] = vsq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        msum = 0;
        vsq = 0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) {
            msum += s_m[w];
            vsq += s_v[w];
        }
        const long long num = 2 * two_e * msum - vsq;
        const long long den = two_e * two_e;
        so.mod[c] = den > 0 ? (double)num / (double)den : 0.0;
        so.ncut[c] = 0.5 * s;
    }
}

__device__ __forceinline__ bool better(int criterion, double mod_a, double ncut_a, int k_a, double mod_b, double ncut_b,
                                       int k_b) {
    if (criterion == RAFTGP_CRIT_NCUT) {
        if (ncut_a != ncut_b) return ncut_a < ncut_b;
    } else {
        if (mod_a != mod_b) return mod_a > mod_b;
    }
    return k_a < k_b;
}

// Candidates compared in evaluation order against the best so far; exact ties to smaller K.
__global__ void k_select_best(CandBatch b, ScoreOut so, int criterion, BestState* best) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    BestState s = *best;
    s.copy_from = -1;
    for (int c = 0; c < b.n; ++c) {
        if (!s.has || better(criterion, so.mod[c], so.ncut[c], b.k[c], s.mod, s.ncut, s.k)) {
            s.has = 1;
            s.mod = so.mod[c];
            s.ncut = so.ncut[c];
            s.k = b.k[c];
            s.copy_from = c;
        }
    }
    *best = s;
}

__global__ void k_copy_best(const BestState* best, const int16_t* labels, int cs, int64_t n, int32_t* out) {
    const int c = best->copy_from;
    if (c < 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = labels[i * cs + c];
}

void launch_score_batch(const CandBatch& b, const raftgp_csr* g, const int32_t* deg, const int16_t* labels,
                        ScoreOut so, uint32_t* err, cudaStream_t s) {
    (void)err;
    ProfScope ps(s, PF_SCORE, 2);
    cudaMemsetAsync(so.m, 0, sizeof(long long) * (size_t)b.total_k, s);
    cudaMemsetAsync(so.vol, 0, sizeof(long long) * (size_t)b.total_k, s);
    const int32_t* rp32 = g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr;
    const int64_t* rp64 = g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr;
    const size_t smem = (size_t)b.total_k * 2 * sizeof(uint32_t);
    if (g->nnz < ((int64_t)1 << 31) && smem <= 160 * 1024) {
        int64_t blocks = (g->n * 32 + 511) / 512;
        const int64_t cap = (int64_t)num_sms() * 2;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        auto k = k_score_count<true>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)blocks, 512, smem, s>>>(b, g->n, rp32, rp64, g->col, deg, labels, so);
    } else {
        int64_t blocks = (g->n * 32 + 511) / 512;
        const int64_t cap = (int64_t)num_sms() * 4;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        k_score_count<false><<<(unsigned)blocks, 512, 0, s>>>(b, g->n, rp32, rp64, g->col, deg, labels, so);
    }
    k_score_finalize<<<b.n, FIN_THREADS, 0, s>>>(b, g->nnz, so);
}

void launch_select_best(const CandBatch& b, ScoreOut so, int criterion, BestState* best, const int16_t* labels,
                        int64_t n, int32_t* out_labels, cudaStream_t s) {
    ProfScope ps(s, PF_SELECT_BEST, 2);
    k_select_best<<<1, 32, 0, s>>>(b, so, criterion, best);
    int blocks = (int)((n + 255) / 256);
    if (blocks > num_sms() * 8) blocks = num_sms() * 8;
    if (blocks < 1) blocks = 1;
    k_copy_best<<<blocks, 256, 0, s>>>(best, labels, b.cs, n, out_labels);
}

// ------------------------------------------------------------------------------------
// Scoring of one given int32 labelling (the raftgp_score entry point).
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_score_one(int64_t n, const int32_t* rp32, const int64_t* rp64,
                                                   const int32_t* col, const int32_t* deg, const int32_t* labels, int K,
                                                   long long* m, long long* vol, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const int li = labels[i];
        if (li < 0 || li >= K) {
            if (lane == 0) flag_error(err, DERR_LABEL_RANGE);
            continue;
        }
        const int64_t beg = rp64 ? rp64[i] : rp32[i];
        const int64_t end = rp64 ? rp64[i + 1] : rp32[i + 1];
        int cnt = 0;
        for (int64_t p = beg + lane; p < end; p += 32) cnt += (__ldg(labels + __ldg(col + p)) == li);
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            if (cnt) atomicAdd(reinterpret_cast<unsigned long long*>(m + li), (unsigned long long)cnt);
            atomicAdd(reinterpret_cast<unsigned long long*>(vol + li), (unsigned long long)deg[i]);
        }
    }
}

// Halves the directed counts in place (m_r = undirected intra edges).
__global__ void k_halve(long long* m, int K) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < K; r += gridDim.x * blockDim.x) m[r] /= 2;
}

__global__ void k_score_one_finalize(const long long* m, const long long* vol, int K, int64_t two_e, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long msum = 0, vsq = 0;
    double s = 0.0;
    for (int r = 0; r < K; ++r) {
        msum += m[r];
        vsq += vol[r] * vol[r];
        if (vol[r] > 0) s += (double)(vol[r] - 2 * m[r]) / (double)vol[r];
    }
    const long long num = 2 * two_e * msum - vsq;
    const long long den = two_e * two_e;
    out[0] = den > 0 ? (double)num / (double)den : 0.0;
    out[1] = 0.5 * s;
}

cudaError_t launch_score_labels(const raftgp_csr* g, const int32_t* deg, const int32_t* labels, int K, long long* m,
                                long long* vol, double* out2, uint32_t* err, cudaStream_t s) {
    ProfScope ps(s, PF_SCORE, 3);
    cudaMemsetAsync(m, 0, sizeof(long long) * (size_t)K, s);
    cudaMemsetAsync(vol, 0, sizeof(long long) * (size_t)K, s);
    int64_t blocks = (g->n * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_score_one<<<(unsigned)blocks, 256, 0, s>>>(g->n, g->row_ptr_bits == 32 ? (const int32_t*)g->row_ptr : nullptr,
                                                 g->row_ptr_bits == 64 ? (const int64_t*)g->row_ptr : nullptr, g->col,
                                                 deg, labels, K, m, vol, err);
    k_halve<<<(K + 255) / 256 < 1024 ? (K + 255) / 256 : 1024, 256, 0, s>>>(m, K);
    k_score_one_finalize<<<1, 32, 0, s>>>(m, vol, K, g->nnz, out2);
    return cudaGetLastError();
}

}  // namespace raftgp
