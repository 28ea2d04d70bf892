// prof.cu -- optional per-kernel-family device timing.  When enabled, every launcher brackets
// its kernels with a pair of CUDA events recorded on the launching stream; reading the
// profile synchronises the device and sums the elapsed times per family.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace raftgp {

static const char* kFamilyNames[PF_COUNT] = {
    "degrees", "theta", "spmm_project", "spmm_gcn", "dense_tc", "seed_update", "seed_pick", "batch_init", "assign_ffma",
    "assign_tc", "assign_tc_first", "assign_tc_final", "assign_recheck", "apply_changes", "apply_first", "lloyd_update",
    "score_count", "select_best", "diff_spmm", "diff_dense", "diff_loss", "diff_other", "other", "assign_ffma_final"};

struct Profiler {
    std::mutex mu;
    bool on = false;
    uint64_t mask = ~0ull;              // families that record events
    std::vector<cudaEvent_t> pool;      // 2 events per record
    size_t used = 0;                    // pairs used
    struct Rec { int fam; int kernels; };
    std::vector<Rec> recs;
    long long launches[PF_COUNT] = {};
    long long untimed[PF_COUNT] = {};
};

static Profiler& prof() {
    static Profiler p;
    return p;
}

static constexpr size_t kPairs = 1 << 15;

ProfScope::ProfScope(cudaStream_t s, int fam, int kernels) : s_(s), fam_(fam), kernels_(kernels), pair_(-1) {
    Profiler& p = prof();
    if (!p.on || !((p.mask >> fam) & 1ull)) return;
    // no events inside a stream capture (a captured graph is replayed without the profiler)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> g(p.mu);
    p.launches[fam] += kernels;
    if (p.used >= kPairs) {
        p.untimed[fam] += kernels;
        return;
    }
    pair_ = (long long)p.used++;
    p.recs.push_back({fam, kernels});
    cudaEventRecord(p.pool[2 * pair_], s_);
}

ProfScope::~ProfScope() {
    if (pair_ < 0) return;
    cudaEventRecord(prof().pool[2 * pair_ + 1], s_);
}

}  // namespace raftgp

using namespace raftgp;

extern "C" {

static raftgp_status profile_start(int32_t on, uint64_t mask) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.mask = mask;
    if (on && p.pool.empty()) {
        p.pool.resize(2 * kPairs);
        for (auto& e : p.pool)
            if (cudaEventCreate(&e) != cudaSuccess) return RAFTGP_ECUDA;
    }
    p.on = on != 0;
    p.used = 0;
    p.recs.clear();
    for (int f = 0; f < PF_COUNT; ++f) p.launches[f] = p.untimed[f] = 0;
    return RAFTGP_OK;
}

raftgp_status raftgp_profile_enable(int32_t on) { return profile_start(on, ~0ull); }

raftgp_status raftgp_profile_enable_family(const char* family) {
    if (!family) return profile_start(1, ~0ull);
    for (int f = 0; f < PF_COUNT; ++f)
        if (std::strcmp(family, kFamilyNames[f]) == 0) return profile_start(1, 1ull << f);
    return RAFTGP_EINVAL;
}

int32_t raftgp_profile_read(raftgp_prof_entry* out, int32_t cap) {
    Profiler& p = prof();
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> g(p.mu);
    double ms[PF_COUNT] = {};
    long long timed[PF_COUNT] = {};
    for (size_t r = 0; r < p.recs.size(); ++r) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.pool[2 * r], p.pool[2 * r + 1]) == cudaSuccess) {
            ms[p.recs[r].fam] += t;
            timed[p.recs[r].fam] += p.recs[r].kernels;
        }
    }
    int32_t k = 0;
    for (int f = 0; f < PF_COUNT && k < cap; ++f) {
        if (p.launches[f] == 0) continue;
        out[k].name = kFamilyNames[f];
        out[k].launches = p.launches[f];
        out[k].timed = timed[f];
        out[k].ms = ms[f];
        ++k;
    }
    return k;
}

}  // extern "C"
