// spgemm_merge_noalloc: the sort-free hash merge with no allocation at all.
//
// Some callers may not allocate device memory: code that runs under another
// framework's fixed device-memory pool, or inside a loop where cudaMalloc's
// implicit device synchronisation and failure modes are not acceptable. This
// entry point serves them: every work buffer of the merge (per-column counts,
// offsets, tier lists, scan partials, the part table) is carved from one
// file-scope __device__ array of kNoAllocScratchBytes, and small device-to-host
// reads land in a static host array, one per device. Each GPU that loads this
// library keeps the array until the process exits.
//
// The array's address is looked up once per device (cudaGetSymbolAddress, with
// that device current) on that device's first call. Every call synchronises its
// stream once, to read the merged size. All calls on one device share that device's array and
// host staging, and the array keeps the last call's contents; the merge clears
// what it reads before writing. Calls on one device that overlap (other
// streams, other host threads) race on both and must be serialised by the
// caller; calls on different devices use different arrays.
#include <mutex>
#include <string>

#include "../../include/spgemm.h"
#include "plan.h"

using namespace spg;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
int g_nsm[kMaxDevices] = {};
std::mutex g_setup_mu;
int32_t g_host_stage[kMaxDevices][1024];   // host staging of small device-to-host reads

}  // namespace

extern "C" spgemm_status spgemm_merge_noalloc(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                                              cudaStream_t stream) {
    spgemm_status s = check_merge_args(parts, nparts, out);
    if (s != SPGEMM_OK) return s;
    if (nparts > 64) { set_error("spgemm_merge_noalloc takes at most 64 parts"); return SPGEMM_ERR_INVALID; }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal out of range"); return SPGEMM_ERR_INVALID; }
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            // the host-side name of the array is not a device address: ask the
            // runtime for this device's copy
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
            int nsm = 0;
            e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
            g_nsm[dev] = nsm;
            g_scratch_addr[dev] = p;
        }
    }
    return merge_noalloc_dispatch(parts, nparts, out, stream,
                                  static_cast<unsigned char *>(g_scratch_addr[dev]),
                                  kNoAllocScratchBytes, g_host_stage[dev], g_nsm[dev]);
}
