// NSGA-III selection for callers that cannot allocate device memory.
//
// Some host programs cannot call cudaMalloc (or any allocator) around the
// selection: a plug-in whose host application owns every device allocation,
// a real-time loop that must not enter the driver's allocator, or a process
// whose memory budget is fixed up front. emo_nsga3_select_noalloc serves them
// by running the selection in a scratch area that is part of the library
// image itself: a file-scope device array of kScratchBytes (9 MiB). Every
// GPU on which the library is loaded holds that array until the process
// exits. Only inputs and outputs come from the caller.
//
// The host code never passes the array's name to a kernel (in host code it is
// a stand-in, not a device address). The first call on each device, with
// that device current, looks up the array's device address with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture. All calls share the one array: the selection initialises every
// counter and flag it reads, so stale contents of an earlier call are
// harmless, but two calls whose work overlaps on the GPU (different streams
// without ordering) race on the array and must not be issued.
#include <mutex>

#include "emo_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(9) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
emo_status scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EMO_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return EMO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return EMO_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return EMO_OK;
}

}  // namespace

extern "C" emo_status emo_nsga3_select_noalloc(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                               int64_t n_keep, uint64_t seed, uint64_t generation,
                                               int32_t* survivors, emo_select_info* info, emo_stream_t stream)
{
    const size_t need = emo_workspace_size(EMO_OP_NSGA3_SELECT, n2, m, n_r);
    if (need == 0) return EMO_ERR_INVALID_ARG;
    if (need > kScratchBytes) return EMO_ERR_WORKSPACE;  // population too large for the built-in scratch
    void* ws = nullptr;
    const emo_status st = scratch_address(&ws);
    if (st != EMO_OK) return st;
    return emo_nsga3_select(F, n2, m, R, n_r, n_keep, seed, generation, survivors, info, ws, kScratchBytes,
                            stream);
}
