// ising_run_noalloc: the persistent fused sweep + PT run of ising_run for
// callers that must not allocate device memory at run time (code running
// inside another framework's allocation-free execution phase, such as a
// real-time loop or a region where device allocations are forbidden).  The
// handle is created and initialised beforehand (that part allocates); this
// call then only launches kernels.  Its scratch -- the grid-barrier arrival
// counter, the block-completion counter and the double-buffered energies
// published for the PT pass -- lives in one file-scope __device__ array that
// every GPU loading the library holds until the process exits.
#include <cstring>
#include <mutex>

#include "handle.h"
#include "ising_gb300.h"
#include "ising_internal.cuh"

int32_t isg_fused_launch(ising_t g, isg::FusedLaunch* out);
int32_t isg_fail(int32_t code, const char* msg);
void isg_count_launches(ising_t g, long long all, long long sweeps);

namespace {

constexpr int kNoAllocMaxReplicas = 16384;
constexpr int kScratchHeader = 64;  // [0] grid barrier, [1] completed blocks, rest unused
constexpr int kScratchWords = kScratchHeader + 2 * kNoAllocMaxReplicas;

static __device__ __align__(256) unsigned int g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned int* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, resolved once
// per device (with that device current).  The library is built from separate
// device modules, and under lazy module loading the module holding the array
// is loaded -- its 128 KB placed on the device -- by the first
// cudaGetSymbolAddress; isg_noalloc_prepare makes that happen while a handle
// is initialised, so that ising_run_noalloc itself finds the address cached.
int32_t scratch_for_current_device(unsigned int** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return isg_fail(ISING_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return isg_fail(ISING_ERR_UNSUPPORTED, "device ordinal out of range for the scratch table");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return isg_fail(ISING_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned int*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ISING_OK;
}

}  // namespace

// Called by ising_replicas_init with the handle's device current.
int32_t isg_noalloc_prepare()
{
    unsigned int* p = nullptr;
    return scratch_for_current_device(&p);
}

extern "C" int32_t ising_run_noalloc(ising_t h, int64_t n, int32_t swap_every)
{
    if (n < 0)
        return isg_fail(ISING_ERR_INVALID_ARG, "n must be >= 0");
    // a launch runs whole groups of swap_every sweeps and at most 2^30 sweeps
    if (swap_every > (1 << 30) && n >= swap_every)
        return isg_fail(ISING_ERR_INVALID_ARG,
                        "ising_run_noalloc: swap_every > 2^30 with n >= swap_every (a PT group longer than "
                        "one launch)");
    ising_info_t info;
    int32_t rc = ising_get_info(h, &info);
    if (rc)
        return rc;
    if (info.replicas == 0)
        return isg_fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    if (info.rng_mode != ISING_RNG_PHILOX)
        return isg_fail(ISING_ERR_UNSUPPORTED,
                        "ising_run_noalloc needs ISING_RNG_PHILOX: MT19937 words are staged in a "
                        "buffer proportional to replicas x spins");
    if (info.replicas > kNoAllocMaxReplicas)
        return isg_fail(ISING_ERR_INVALID_ARG,
                        "ising_run_noalloc supports at most 16384 replicas (static scratch size)");
    if (swap_every > 0 && swap_every <= n && !isg_pt_ok(h))
        return isg_fail(ISING_ERR_UNSUPPORTED, "PT swap tables exceed 2^28 entries for this ladder: sweeps only");
    isg::FusedLaunch fl;
    if ((rc = isg_fused_launch(h, &fl)))
        return rc;
    if (n == 0)
        return ISING_OK;
    unsigned int* scratch = nullptr;
    if ((rc = scratch_for_current_device(&scratch)))
        return rc;

    isg::SweepArgs a = fl.args;
    a.gridbar = scratch + 0;
    a.done_blocks = scratch + 1;
    a.E_pub = reinterpret_cast<int*>(scratch + kScratchHeader);
    a.wbuf = nullptr;
    a.swbuf = nullptr;
    a.gen = 0;  // no word buffer: the slots compute their Philox words themselves
    cudaStream_t st = fl.stream;
    const long long every = swap_every > 0 ? swap_every : 0;
    long long done = 0;
    while (done < n) {
        // whole groups of `every` sweeps with the PT pass fused; the rest, or
        // everything when every == 0, without PT
        long long m;
        bool fused;
        if (every > 0 && n - done >= every) {
            m = ((n - done) / every) * every;
            fused = true;
        } else {
            m = n - done;
            fused = false;
        }
        if (m > (1LL << 30))
            m = (fused ? ((1LL << 30) / every) * every : (1LL << 30));
        // both counters start from zero for every launch
        cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned int), st);
        if (e == cudaSuccess) {
            a.nsweeps = int(m);
            a.swap_every = fused ? int(every) : 0;
            e = isg::launch_fast(a, fl.field_bits, fl.cmax, fl.threads, fl.blocks,
                                 fused ? fl.smem_fused : fl.smem_plain, fused, st, fl.variant);
        }
        if (e != cudaSuccess)
            return isg_fail(e == cudaErrorCooperativeLaunchTooLarge ? ISING_ERR_UNSUPPORTED : ISING_ERR_CUDA,
                            cudaGetErrorString(e));
        isg_count_launches(h, 1, 1);
        done += m;
    }
    return ISING_OK;
}
