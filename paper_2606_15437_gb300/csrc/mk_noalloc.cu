// mk_noalloc.cu -- the census for callers that cannot allocate device memory.
//
// mk_census takes its scratch space (the S4/S5 frame lists and the
// prefix-sum counters used to build them) from a workspace the caller
// allocates.  Some callers cannot do that: a plain C program or a foreign-
// function binding that can hand over pointers it already owns but has no
// device allocator of its own, or code that must not call cudaMalloc /
// cudaFree at all because those calls synchronise the whole device and
// would stall other work in flight.  mk_census_noalloc serves them: the
// scratch is a fixed array in this library's own device memory, so the
// caller passes only inputs and outputs.
//
// The array is a file-scope __device__ variable, so every GPU that loads
// the library holds MK_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Host code cannot use the variable's name as a device address; a call
// asks the runtime for the address on the current device with
// cudaGetSymbolAddress (a lookup: it allocates nothing).  Calls outside
// stream capture look it up every time, so an address made stale by a
// device reset is never used; calls on a capturing stream use the address
// the last uncaptured call on that device found.  Nothing here calls
// cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "mk.h"

namespace {

static __device__ __align__(256) uint8_t g_census_scratch[MK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices];

// Device address of g_census_scratch on the current device: looked up
// afresh unless `stream` is being captured (then the address remembered for
// the device, looked up only if there is none).
int scratch_address(cudaStream_t stream, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MK_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return MK_E_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    bool capturing = true;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess) capturing = cs != cudaStreamCaptureStatusNone;
    else (void)cudaGetLastError();   // e.g. the legacy stream queried during another thread's capture
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!capturing || !g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_census_scratch) != cudaSuccess || !p) return MK_E_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MK_OK;
}

}  // namespace

// mk_census.cu: the frame lists' share of the workspace (the least that
// mk_census accepts; with it alone every layer runs unsplit).
size_t mk_census_min_workspace(const mk_census_cfg *cfg, int32_t nprog);

extern "C" int mk_census_noalloc(const mk_program *d_progs, int32_t nprog, const mk_census_cfg *cfg,
                                 mk_result *d_out, int32_t *d_status, void *stream) {
    const size_t need = mk_census_min_workspace(cfg, nprog);
    if (need == 0) return MK_E_ARG;
    if (need > MK_NOALLOC_SCRATCH_BYTES) return MK_E_WORKSPACE;
    void *scratch = nullptr;
    const int rc = scratch_address((cudaStream_t)stream, &scratch);
    if (rc != MK_OK) return rc;
    return mk_census(d_progs, nprog, cfg, d_out, d_status, scratch, MK_NOALLOC_SCRATCH_BYTES, stream);
}
