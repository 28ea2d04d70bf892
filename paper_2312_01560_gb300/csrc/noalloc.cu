// noalloc.cu -- k-means++ seeding without a caller-provided workspace.
//
// raftgp_kmeanspp needs scratch memory (the D^2 array, the chosen-point flags and the block
// sums of the sampling scan) and takes it from a workspace the caller allocates.  Some
// callers cannot allocate device memory at all: for example a plugin running inside another
// program's CUDA context, whose device memory is owned and budgeted by that program's own
// allocator, or a host process that has reserved all the device memory it may use before it
// starts partitioning.  raftgp_kmeanspp_noalloc serves them: its scratch is the file-scope
// array below, which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace raftgp {

// The scratch of raftgp_kmeanspp_noalloc: RAFTGP_NOALLOC_SCRATCH_BYTES bytes of device memory.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RAFTGP_NOALLOC_SCRATCH_BYTES];

// Layout inside the scratch for n points: D^2 (n floats), chosen flags (n bytes), block sums
// (one uint64 per 256 points), each part 256-byte aligned.
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// RAFTGP_NOALLOC_MAX_N points need 4 + 1 + 8/256 bytes each plus alignment: 30.2 MB < 32 MiB.
static_assert((size_t)RAFTGP_NOALLOC_MAX_N * 4 + RAFTGP_NOALLOC_MAX_N + (RAFTGP_NOALLOC_MAX_N / 256 + 1) * 8 + 768 <=
                  (size_t)RAFTGP_NOALLOC_SCRATCH_BYTES,
              "static scratch too small for RAFTGP_NOALLOC_MAX_N");

// Device address of the scratch, looked up once per device (the host-side name of a
// __device__ variable is not a device address).
constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {};

static cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace raftgp

using namespace raftgp;

extern "C" raftgp_status raftgp_kmeanspp_noalloc(const void* Z, int64_t n, int32_t d, int32_t z_dtype, int32_t K,
                                                 uint64_t seed, int32_t* seeds, raftgp_stream_t stream) {
    if (!Z || !seeds || n < 1) return set_error(RAFTGP_EINVAL, "NULL argument or n < 1");
    if (d != 32 && d != 64 && d != 128) return set_error(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (K < 1 || K > n) return set_error(RAFTGP_EINVAL, "need 1 <= K <= n");
    if (z_dtype != RAFTGP_F32 && z_dtype != RAFTGP_BF16) return set_error(RAFTGP_EINVAL, "unknown z_dtype");
    if (n > RAFTGP_NOALLOC_MAX_N)
        return set_error(RAFTGP_EUNSUPPORTED,
                         "n = %lld exceeds RAFTGP_NOALLOC_MAX_N = %d, the most points the static scratch holds; "
                         "use raftgp_kmeanspp with a workspace",
                         (long long)n, RAFTGP_NOALLOC_MAX_N);
    void* base = nullptr;
    const cudaError_t ae = scratch_address(&base);
    if (ae != cudaSuccess)
        return set_error(RAFTGP_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(ae));
    char* p = (char*)base;
    float* D2 = (float*)p;
    uint8_t* chosen = (uint8_t*)(p + align256((size_t)n * sizeof(float)));
    unsigned long long* bs = (unsigned long long*)(p + align256((size_t)n * sizeof(float)) + align256((size_t)n));
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the chosen flags must start at zero
    // (D^2 and the block sums are written before they are read)
    cudaError_t e = cudaMemsetAsync(chosen, 0, (size_t)n, s);
    if (e != cudaSuccess) return set_error(RAFTGP_ECUDA, "clearing the static scratch: %s", cudaGetErrorString(e));
    launch_seed_first(n, seed, seeds, chosen, s);
    for (int t = 1; t < K; ++t) launch_seed_round(Z, z_dtype, n, d, t, seed, seeds, chosen, D2, bs, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(RAFTGP_ECUDA, "raftgp_kmeanspp_noalloc: %s", cudaGetErrorString(e));
    return RAFTGP_OK;
}
