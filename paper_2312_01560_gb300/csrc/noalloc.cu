// noalloc.cu -- k-means++ seeding without a caller-provided workspace.
//
// raftgp_kmeanspp needs scratch memory (the D^2 array, the nearest-seed indices, the
// chosen-point flags and the block sums of the sampling scan) and takes it from a workspace the
// caller allocates.  Some
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

// Layout inside the scratch: the seeding state of carve_seed (D^2 floats, nearest-seed int16,
// chosen flags, block sums, seed-to-seed distances, grid barrier words), about 7 bytes per
// point plus 4 per seed.
static_assert((size_t)RAFTGP_NOALLOC_MAX_N * 7 + (RAFTGP_NOALLOC_MAX_N / 1024 + 2048) * 8 + 32767 * 4 + 6 * 256 <=
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
    if ((uintptr_t)Z & 15) return set_error(RAFTGP_EINVAL, "Z must be 16-byte aligned");
    if (d != 32 && d != 64 && d != 128) return set_error(RAFTGP_EUNSUPPORTED, "d must be 32, 64 or 128");
    if (K < 1 || K > n) return set_error(RAFTGP_EINVAL, "need 1 <= K <= n");
    if (K > 32767) return set_error(RAFTGP_EUNSUPPORTED, "K above 32767 is not supported");
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
    if (seed_scratch_bytes(n, K) > (size_t)RAFTGP_NOALLOC_SCRATCH_BYTES)
        return set_error(RAFTGP_EUNSUPPORTED, "n = %lld, K = %d do not fit the static scratch", (long long)n, K);
    // every part of the state is written before it is read except the chosen flags, which
    // carry the previous call's contents and are cleared by the seeding launch itself
    cudaError_t e = launch_seeding(Z, z_dtype, n, d, K, seed, carve_seed(base, n, K, seeds), (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(RAFTGP_ECUDA, "raftgp_kmeanspp_noalloc: %s", cudaGetErrorString(e));
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(RAFTGP_ECUDA, "raftgp_kmeanspp_noalloc: %s", cudaGetErrorString(e));
    return RAFTGP_OK;
}
