// batch_score.cuh -- the exact score of one (graph, candidate) partition of the batched form,
// shared by its FP32 and tensor-core Lloyd kernels.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace raftgp {

// ------------------------------------------------------------------------------------
// Score of one (graph, candidate) partition: intra-block edge ends and volumes (exact
// integers, in the 2 BATCH_KMAX shared counters `m2`), then Mod (Eq. 3 via Eq. 7, one FP64
// division of exact integers) and NCut (Eq. 1, ascending blocks).  Every thread of the CTA
// calls it.
// ------------------------------------------------------------------------------------
__device__ inline void batch_score_item(const BatchDev& b, int g, int slot, int K, int64_t o, int64_t n, const int16_t* lab,
                                 int passes, unsigned long long* m2, const int64_t* __restrict__ rp64,
                                 const int32_t* __restrict__ rp32, const int32_t* __restrict__ col) {
    unsigned long long* vol = m2 + BATCH_KMAX;
    for (int t = threadIdx.x; t < 2 * BATCH_KMAX; t += blockDim.x) m2[t] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int li = lab[i];
        const int64_t a = rp64 ? rp64[o + i] : (int64_t)rp32[o + i];
        const int64_t e = rp64 ? rp64[o + i + 1] : (int64_t)rp32[o + i + 1];
        unsigned long long same = 0;
        for (int64_t q = a; q < e; ++q) same += lab[(int64_t)col[q] - o] == li ? 1ull : 0ull;
        atomicAdd(vol + li, (unsigned long long)(e - a));
        if (same) atomicAdd(m2 + li, same);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t ea = rp64 ? rp64[o] : (int64_t)rp32[o];
        const int64_t eb = rp64 ? rp64[o + n] : (int64_t)rp32[o + n];
        const long long two_e = eb - ea;
        long long sm = 0, sv = 0;
        double ncut = 0.0;
        for (int r = 0; r < K; ++r) {
            const long long mr = (long long)(m2[r] / 2), vr = (long long)vol[r];
            sm += mr;
            sv += vr * vr;
            if (vr > 0) ncut += (double)(vr - 2 * mr) / (double)vr;
        }
        const double mod = two_e > 0 ? (double)(2 * two_e * sm - sv) / ((double)two_e * (double)two_e) : 0.0;
        b.cand_mod[g * BATCH_SLOTS + slot] = mod;
        b.cand_ncut[g * BATCH_SLOTS + slot] = 0.5 * ncut;
        b.cand_passes[g * BATCH_SLOTS + slot] = passes;
    }
}

}  // namespace raftgp
