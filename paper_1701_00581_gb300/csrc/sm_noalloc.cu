// Whole-path reconstruction for callers that must not allocate device memory.
//
// Some programs cannot call cudaMalloc once they are running: a camera or
// telescope control loop that fixes all of its device memory at start-up
// (an allocation can synchronise the device and stall frame acquisition),
// or a plug-in whose host framework owns every device allocation.  This
// entry point serves them: its scratch workspace is a fixed array in the
// library's own device image, so the call itself allocates nothing.
#include <mutex>

#include "sm_plan.h"

using namespace smi;

// Fixed scratch workspace.  Every GPU that loads this library holds these
// bytes until the process exits.  In host code the name is only a handle for
// cudaGetSymbolAddress, never a device pointer.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" int sm_reconstruct_noalloc(const sm_plan* plan, const void* frames, int frame_type, int F,
                                      const double* stf, float* out, uint8_t* valid, void* stream) {
    if (!plan || !frames || !out) { set_error("NULL plan, frames or out"); return SM_EINVAL; }
    if (F < 1 || F > plan->ch.max_frames) { set_error("F out of range 1..max_frames"); return SM_EINVAL; }
    if (plan->device < 0 || plan->device >= kMaxDevices) { set_error("device index too large"); return SM_EINVAL; }
    // the largest chunk of subfields whose workspace fits the fixed scratch
    const int n = plan->dev.n_sub;
    sm_workspace_layout lay;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        int rc = sm_workspace_query(plan, F, mid, &lay);
        if (rc) return rc;
        if (lay.bytes <= SM_NOALLOC_SCRATCH_BYTES) lo = mid; else hi = mid - 1;
    }
    if (lo == 0) {
        sm_workspace_query(plan, F, 1, &lay);
        set_error("this channel needs " + std::to_string(lay.bytes) + " bytes of workspace even one " +
                  "subfield at a time; the fixed no-alloc scratch holds " +
                  std::to_string((size_t)SM_NOALLOC_SCRATCH_BYTES) + " bytes");
        return SM_ENOMEM;
    }
    sm_workspace_query(plan, F, lo, &lay);
    int old = 0;
    cudaGetDevice(&old);
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    void* ws = nullptr;
    {
        // first call on a device: look up the device address of the array
        // (host code cannot use the symbol itself as a device pointer)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[plan->device]) {
            e = cudaGetSymbolAddress(&g_addr[plan->device], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[plan->device] = nullptr;
                cudaSetDevice(old);
                return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
            }
        }
        ws = g_addr[plan->device];
    }
    const int rc = sm_reconstruct(plan, frames, frame_type, F, stf, lo, ws, &lay, out, valid, stream);
    if (old != plan->device) cudaSetDevice(old);
    return rc;
}
