// Allocation-free forward entry point.
//
// Some callers cannot call cudaMalloc: code running under an allocator that
// owns all device memory (a framework's memory pool, a serving runtime with a
// fixed budget), a real-time loop where an allocation would stall or fail, or
// a plugin host that hands out no device memory.  fd_forward_noalloc runs the
// same forward path as fd_forward but takes its scratch from a fixed array
// compiled into this library instead of a caller-provided workspace.  The
// caller still provides the model, wavelet, traces and optional states.
//
// The array is a file-scope static __device__ object of kNoallocScratchBytes:
// every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address, so the address is
// resolved once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on it.
#include <mutex>

#include "internal.h"
#include "runtime.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fdw::set_error(FD_ERR_CUDA, "fd_forward_noalloc: cudaGetDevice failed: %s",
                              cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fdw::set_error(FD_ERR_UNSUPPORTED, "fd_forward_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fdw::set_error(FD_ERR_CUDA, "fd_forward_noalloc: cudaGetSymbolAddress failed: %s",
                                  cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FD_OK;
}

}  // namespace

extern "C" int fd_forward_noalloc(fd_plan *plan, int model_kind, const float *model_d, int nsrc,
                                  const int64_t *src_idx, const float *wavelet_d, int nrec,
                                  const int64_t *rec_idx, float *traces_d, const float *state_in_d,
                                  float *state_out_d, void *stream)
{
    fdw::clear_error();
    size_t need = 0;
    int st = fd_forward_workspace_size(plan, nsrc, nrec, &need);
    if (st) return st;
    if (need > kNoallocScratchBytes)
        return fdw::set_error(FD_ERR_NOMEM,
                              "fd_forward_noalloc: this problem needs %zu bytes of scratch but the "
                              "static scratch holds %zu bytes; use fd_forward with a workspace",
                              need, kNoallocScratchBytes);
    void *ws = nullptr;
    if ((st = scratch_address(&ws))) return st;
    // The forward path clears the status word and both wavefield buffers on every
    // call, so nothing left in the array by an earlier call leaks into this one.
    // Steps are launched one by one: no graph is captured or instantiated and no
    // cached graph is evicted (which would synchronise the device).
    return fdw::forward_impl(plan, model_kind, model_d, nsrc, src_idx, wavelet_d, nrec, rec_idx,
                             traces_d, state_in_d, state_out_d, ws, kNoallocScratchBytes, stream,
                             false);
}

// The status word of the last fd_forward_noalloc call on the current device
// sits at the start of the static array; this reads and clears it like
// fd_status_read does for a caller's workspace.
extern "C" int fd_status_read_noalloc(const fd_plan *plan, void *stream)
{
    fdw::clear_error();
    void *ws = nullptr;
    int st = scratch_address(&ws);
    if (st) return st;
    return fd_status_read(plan, ws, stream);
}
