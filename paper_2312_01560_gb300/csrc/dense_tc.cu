// dense_tc.cu -- the weight product of a GCN layer (Eq. 6: Z^(k-1) W^(k)) on tcgen05 for BF16
// features:
//     P[i] = s_i * (X[i] . W),   X: N x LIN (BF16), W: LIN x LOUT, s_i = the next gather weight
// W is split into two BF16 halves (W = hi + lo) that multiply into the same FP32 accumulator,
// so the product carries about 16 bits of W.  W^T (hi, lo) is loaded into shared memory once
// per CTA; 128-row tiles of X stream in through TMA (double-buffered) and the accumulator is
// double-buffered in tensor memory.  Warp 0 issues the loads, warp 1 the MMAs, warps 2-5 read
// the accumulator (thread = row), scale, round to BF16 and store.  All waits are bounded.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace raftgp {

template <int LIN, int LOUT>
struct DnCfg {
    static constexpr int ATOM = LIN < 64 ? LIN : 64;       // K elements per swizzle-atom row
    static constexpr int ATOM_BYTES = ATOM * 2;
    static constexpr int NATOM = LIN / ATOM;
    static constexpr int A_ATOM_BYTES = 128 * ATOM_BYTES;
    static constexpr int A_BYTES = NATOM * A_ATOM_BYTES;   // one 128-row tile
    static constexpr int B_ATOM_BYTES = LOUT * ATOM_BYTES;
    static constexpr int B_BYTES = NATOM * B_ATOM_BYTES;   // one half (hi or lo) of W^T
    static constexpr int LAYOUT = ATOM_BYTES == 128 ? 2 : 4;
    static constexpr int SBO = 8 * ATOM_BYTES;
    static constexpr int TMEM_COLS = 2 * LOUT < 32 ? 32 : 2 * LOUT;
    static constexpr int SMEM = 1024 + 2 * A_BYTES + 2 * B_BYTES;
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

struct DnCtl {
    uint64_t a_full[2], a_empty[2], b_full, acc_full[2], acc_empty[2], drain;
    uint32_t tmem_base;
    int abort;
};

template <int LIN, int LOUT>
__global__ void __launch_bounds__(192, 1)
    k_dense_tc(int64_t n, const float* __restrict__ scale, __nv_bfloat16* __restrict__ out, uint32_t* err,
               const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmWhi,
               const __grid_constant__ CUtensorMap tmWlo) {
    using C = DnCfg<LIN, LOUT>;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ DnCtl ctl;
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;                      // two tiles
    uint8_t* sB = base + 2 * C::A_BYTES;     // hi then lo
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        ctl.abort = 0;
        for (int q = 0; q < 2; ++q) {
            mbar_init(&ctl.a_full[q], 1);
            mbar_init(&ctl.a_empty[q], 1);
            mbar_init(&ctl.acc_full[q], 1);
            mbar_init(&ctl.acc_empty[q], 128);
        }
        mbar_init(&ctl.b_full, 1);
        mbar_init(&ctl.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&ctl.tmem_base)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem_base;
    const int64_t ntiles = (n + 127) / 128;

    if (warp == 0) {
        if (lane == 0) {
            bool ok = true;
            mbar_expect_tx(&ctl.b_full, 2 * C::B_BYTES);
            for (int t = 0; t < C::NATOM; ++t) {
                tma_load_2d(sB + t * C::B_ATOM_BYTES, &tmWhi, &ctl.b_full, t * C::ATOM, 0);
                tma_load_2d(sB + C::B_BYTES + t * C::B_ATOM_BYTES, &tmWlo, &ctl.b_full, t * C::ATOM, 0);
            }
            int tl = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tl) {
                const int ab = tl & 1;
                if (!(ok = mbar_wait(&ctl.a_empty[ab], ((tl >> 1) & 1) ^ 1, &ctl, err))) break;
                mbar_expect_tx(&ctl.a_full[ab], C::A_BYTES);
                for (int t = 0; t < C::NATOM; ++t)
                    tma_load_2d(sA + ab * C::A_BYTES + t * C::A_ATOM_BYTES, &tmX, &ctl.a_full[ab], t * C::ATOM,
                                (int)(tile * 128));
            }
            if (!ok) {
                // let every copy issued land before the CTA can exit
                mbar_drain(&ctl.b_full, 0);
                for (int k = (tl > 2 ? tl - 2 : 0); k < tl; ++k) mbar_drain(&ctl.a_full[k & 1], (k >> 1) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(LOUT);
            const uint64_t dA = smem_desc(smem_addr(sA), C::LAYOUT, C::SBO);
            const uint64_t dB = smem_desc(smem_addr(sB), C::LAYOUT, C::SBO);
            bool ok = mbar_wait(&ctl.b_full, 0, &ctl, err);
            int tl = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tl) {
                const int ab = tl & 1;
                if (!(ok = mbar_wait(&ctl.a_full[ab], (tl >> 1) & 1, &ctl, err))) break;
                if (!(ok = mbar_wait(&ctl.acc_empty[ab], ((tl >> 1) & 1) ^ 1, &ctl, err))) break;
                tc_fence_after();
                const uint32_t dcol = tmem + (uint32_t)(ab * LOUT);
#pragma unroll
                for (int half = 0; half < 2; ++half)
#pragma unroll
                    for (int t = 0; t < C::NATOM; ++t)
#pragma unroll
                        for (int k = 0; k < C::ATOM / 16; ++k) {
                            const uint64_t ad = dA + (uint64_t)((ab * C::A_BYTES + t * C::A_ATOM_BYTES + k * 32) >> 4);
                            const uint64_t bd = dB + (uint64_t)((half * C::B_BYTES + t * C::B_ATOM_BYTES + k * 32) >> 4);
                            mma_bf16(dcol, ad, bd, idesc, (half | t | k) ? 1 : 0);
                        }
                mma_commit(&ctl.a_empty[ab]);
                mma_commit(&ctl.acc_full[ab]);
            }
            mma_commit(&ctl.drain);
            mbar_drain(&ctl.drain, 0);
        }
    } else {
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        bool ok = true;
        int tl = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tl) {
            const int ab = tl & 1;
            if (!(ok = mbar_wait(&ctl.acc_full[ab], (tl >> 1) & 1, &ctl, err))) break;
            tc_fence_after();
            const int64_t i = tile * 128 + row;
            const float sc = i < n ? __ldg(scale + i) : 0.f;
#pragma unroll
            for (int c0 = 0; c0 < LOUT; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(lane_base + (uint32_t)(ab * LOUT + c0), r);
                if (c0 + 32 >= LOUT) {
                    tc_fence_before();
                    mbar_arrive(&ctl.acc_empty[ab]);
                }
                if (i < n) {
                    uint4* dst = reinterpret_cast<uint4*>(out + i * LOUT + c0);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        uint32_t w[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(sc * __uint_as_float(r[8 * v + 2 * u]),
                                                                           sc * __uint_as_float(r[8 * v + 2 * u + 1]));
                            w[u] = *reinterpret_cast<const uint32_t*>(&h);
                        }
                        dst[v] = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
}

// W (LIN x LOUT, FP32, row-major) -> W^T hi and lo halves (LOUT x LIN, BF16).
__global__ void k_w_split(const float* W, int lin, int lout, __nv_bfloat16* whi, __nv_bfloat16* wlo) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= lin * lout) return;
    const int a = t / lout, c = t % lout;
    const float v = W[t];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    whi[(int64_t)c * lin + a] = h;
    wlo[(int64_t)c * lin + a] = __float2bfloat16_rn(v - __bfloat162float(h));
}

template <int LIN, int LOUT>
static cudaError_t launch_dense_t(int64_t n, const void* X, const __nv_bfloat16* whi, const __nv_bfloat16* wlo,
                                  const float* scale, void* out, uint32_t* err, cudaStream_t s) {
    using C = DnCfg<LIN, LOUT>;
    const CUtensorMapSwizzle swz = C::ATOM_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap tx, th, tl;
    cudaError_t e;
    if ((e = make_map_bf16(&tx, X, LIN, n, C::ATOM, 128, swz)) != cudaSuccess) return e;
    if ((e = make_map_bf16(&th, whi, LIN, LOUT, C::ATOM, LOUT, swz)) != cudaSuccess) return e;
    if ((e = make_map_bf16(&tl, wlo, LIN, LOUT, C::ATOM, LOUT, swz)) != cudaSuccess) return e;
    auto kern = k_dense_tc<LIN, LOUT>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM)) != cudaSuccess) return e;
    const int64_t ntiles = (n + 127) / 128;
    const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
    ProfScope ps(s, PF_DENSE_TC, 1);
    kern<<<grid, 192, C::SMEM, s>>>(n, scale, (__nv_bfloat16*)out, err, tx, th, tl);
    return cudaGetLastError();
}

template <int LIN>
static cudaError_t launch_dense_lout(int lout, int64_t n, const void* X, const __nv_bfloat16* whi,
                                     const __nv_bfloat16* wlo, const float* scale, void* out, uint32_t* err,
                                     cudaStream_t s) {
    switch (lout) {
        case 32: return launch_dense_t<LIN, 32>(n, X, whi, wlo, scale, out, err, s);
        case 64: return launch_dense_t<LIN, 64>(n, X, whi, wlo, scale, out, err, s);
        case 128: return launch_dense_t<LIN, 128>(n, X, whi, wlo, scale, out, err, s);
    }
    return cudaErrorInvalidValue;
}

void launch_w_split(const float* W, int lin, int lout, __nv_bfloat16* whi, __nv_bfloat16* wlo, cudaStream_t s) {
    ProfScope ps(s, PF_OTHER, 1);
    k_w_split<<<(lin * lout + 255) / 256, 256, 0, s>>>(W, lin, lout, whi, wlo);
}

cudaError_t launch_dense_tc(int lin, int lout, int64_t n, const void* X, const __nv_bfloat16* whi,
                            const __nv_bfloat16* wlo, const float* scale, void* out, uint32_t* err, cudaStream_t s) {
    switch (lin) {
        case 32: return launch_dense_lout<32>(lout, n, X, whi, wlo, scale, out, err, s);
        case 64: return launch_dense_lout<64>(lout, n, X, whi, wlo, scale, out, err, s);
        case 128: return launch_dense_lout<128>(lout, n, X, whi, wlo, scale, out, err, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace raftgp
