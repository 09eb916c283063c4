// gcb_noalloc.cu -- gcb_push_sr_noalloc: the push with its scratch memory in a
// fixed array that the library owns, for callers that cannot allocate device
// memory themselves.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host callback or another library's plugin hook that forbids allocation, a
// process whose device memory is fully reserved by a pool it does not
// control, or a real-time loop that must not allocate after start-up.  Such
// a caller still owns the particle arrays and the field records; only the
// scratch (the step counters, and for small problems the sort buffers) comes
// from here.
//
// The array below lives in every device context that loads this library and
// stays there until the process exits (GCB_NOALLOC_SCRATCH_BYTES per GPU).
// Its name is a host-side stand-in, not a device address, so each call looks
// the address up with cudaGetSymbolAddress while the call's device is
// current.  Looking it up again on every call keeps a device reset
// (cudaDeviceReset unloads the module, which may put the array elsewhere
// when it is reloaded) from leaving a stale address behind.  While the
// call's stream is capturing, no lookup is made (it may load the module);
// the address the last call outside a capture found on that device is used,
// so the first call on each device must come before any stream capture.
// Every call shares the one array: gcb_push_sr clears what must start at
// zero at the start of each call, and two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "gcb.h"
#include "gcb_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[GCB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" gcb_status gcb_push_sr_noalloc(const gcb_particles *p, const gcb_grid *g,
                                          const gcb_params *prm, int n_steps, void *cuda_stream,
                                          gcb_stats *out)
{
    const size_t need = gcb_workspace_bytes(p, g, prm);
    if (need > (size_t)GCB_NOALLOC_SCRATCH_BYTES) {
        gcb::set_error("gcb_push_sr_noalloc: this problem needs %zu bytes of scratch, more than "
                       "the fixed %zu-byte array; use gcb_push_sr with a workspace (or no sorting)",
                       need, (size_t)GCB_NOALLOC_SCRATCH_BYTES);
        return GCB_ENOMEM;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        gcb::set_error("gcb_push_sr_noalloc: no usable current device");
        return GCB_ECUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap) != cudaSuccess) {
        gcb::set_error("gcb_push_sr_noalloc: cudaStreamIsCapturing failed: %s",
                       cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void *a = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&a, g_scratch);
            if (e != cudaSuccess || !a) {
                gcb::set_error("gcb_push_sr_noalloc: cudaGetSymbolAddress failed: %s",
                               cudaGetErrorString(e));
                return GCB_ECUDA;
            }
            g_ptr[dev] = a;
        } else if (!g_ptr[dev]) {
            gcb::set_error("gcb_push_sr_noalloc: the first call on a device must not be made "
                           "while its stream is capturing a graph");
            return GCB_EINVAL;
        }
        ptr = g_ptr[dev];
    }
    return gcb_push_sr(p, g, prm, n_steps, cuda_stream, ptr, (size_t)GCB_NOALLOC_SCRATCH_BYTES, out);
}
