// noalloc.cu -- k-means++ seeding without a caller-provided workspace.
//
// raftgp_kmeanspp needs scratch memory (the D^2 array, the nearest-seed indices, the
// chosen-point flags and the block sums of the sampling scan) and takes it from a workspace the
// caller allocates.  Some
// callers cannot allocate device memory at all: for example a plugin running inside another
// program's CUDA context, whose device memory is owned and budgeted by that program's own
// allocator, or a host process that has reserved all the device memory it may use before it
// starts partitioning.  raftgp_kmeanspp_noalloc serves them: its scratch is the file-scope
// array below.  Each CUDA context that runs the call holds the array until the context ends
// (with lazy module loading, the default, its memory is committed by the first call in that
// context, not when the library is loaded).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

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

// Device address of the scratch.  The address of a __device__ variable belongs to the CUDA
// context that loaded the module (its host-side name is not a device address at all), so it
// is looked up once per context, with that context current, and cached under the context's
// unique id (cuCtxGetId: never reused within a process, so a destroyed and re-created context,
// or a second context on the same device, gets its own lookup).  With lazy module loading
// (the default), the first lookup in a context is also what commits the array's device memory.
// The cache is shared by every host thread, under a mutex.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

constexpr int kCacheSlots = 64;
struct ScratchSlot {
    unsigned long long ctx_id;
    void* ptr;
};
static std::mutex g_scratch_mu;
static ScratchSlot g_scratch_cache[kCacheSlots] = {};
static int g_scratch_next = 0;
static PfnCtxGetCurrent g_ctx_get_current = nullptr;
static PfnCtxGetId g_ctx_get_id = nullptr;

static cudaError_t driver_fn(const char* name, void** fn) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !*fn) return cudaErrorNotSupported;
    return cudaSuccess;
}

// The unique id of the context current on this thread (0 if none is current yet).
static cudaError_t current_ctx_id(unsigned long long* id) {
    *id = 0;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) return cudaSuccess;
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS || *id == 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

static cudaError_t scratch_address(void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    cudaError_t e;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        if ((e = driver_fn("cuCtxGetCurrent", &f1)) != cudaSuccess) return e;
        if ((e = driver_fn("cuCtxGetId", &f2)) != cudaSuccess) return e;
        g_ctx_get_current = (PfnCtxGetCurrent)f1;
        g_ctx_get_id = (PfnCtxGetId)f2;
    }
    unsigned long long id = 0;
    if ((e = current_ctx_id(&id)) != cudaSuccess) return e;
    if (id != 0)
        for (int s = 0; s < kCacheSlots; ++s)
            if (g_scratch_cache[s].ctx_id == id) {
                *out = g_scratch_cache[s].ptr;
                return cudaSuccess;
            }
    // a miss: look the address up in the current context (with no context current yet, the
    // runtime first makes the device's primary context current, and that is the one used)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (id == 0 && ((e = current_ctx_id(&id)) != cudaSuccess || id == 0))
        return e != cudaSuccess ? e : cudaErrorDeviceUninitialized;
    g_scratch_cache[g_scratch_next] = ScratchSlot{id, p};   // the oldest entry is replaced when full
    g_scratch_next = (g_scratch_next + 1) % kCacheSlots;
    *out = p;
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
