// Measurement entry point that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they measure.
// Examples are code running under a memory manager that owns every allocation of the
// process (a framework's caching allocator, a fixed arena sized at start-up), code
// that must not trigger the implicit device synchronisation a cudaMalloc/cudaFree can
// cause in the middle of a pipeline, and plugins that are handed device buffers but
// no allocation rights.  Such a caller keeps its lattice in memory it already owns
// and passes it in; this entry point writes the derived observables to the caller's
// output buffer, and keeps the integer records it needs on the way in a fixed array
// that lives in the library's own device image.
//
// The scratch array is a file-scope __device__ array, so every GPU that loads the
// library holds it (1 MiB) until the process exits.  Host code must not hand the
// array's name to a kernel: on the host that name is only a stand-in.  The device
// address is looked up with cudaGetSymbolAddress once per device, the first time the
// entry point runs on that device (with that device current); that first call should
// therefore happen before any stream capture.
#include <mutex>

#include "../../include/ising.h"
#include "common.cuh"
#include "kernels.h"

namespace {

__device__ __align__(256) int64_t g_noalloc_records[ISING_NOALLOC_MAX_RECORD_WORDS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
int64_t *g_records_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once.
cudaError_t scratch_for_current_device(int64_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_records_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_records);
        if (e != cudaSuccess) return e;
        g_records_ptr[dev] = static_cast<int64_t *>(p);
    }
    *out = g_records_ptr[dev];
    return cudaSuccess;
}

bool packed_size_ok(int L) { return (L >= 64 && L % 64 == 0) || L == 4 || L == 8 || L == 16 || L == 32; }

}  // namespace

extern "C" int ising_measure_derived_noalloc(const uint32_t *lattice, int L, int replicas, double c,
                                             unsigned flags, double *derived, void *stream)
{
    if (!lattice || !derived || replicas < 1 || !packed_size_ok(L) || L > 4096) return ISING_EINVAL;
    // ISING_MEAS_DEVICE is accepted and ignored: the output is always device memory here
    if (flags & ~(ISING_MEAS_DEVICE | ISING_MEAS_CONNECTED | ISING_MEAS_NO_CORR)) return ISING_EINVAL;
    const int64_t RL = 3 + 3 * (int64_t)(L / 2 + 1);
    if ((int64_t)replicas * RL > ISING_NOALLOC_MAX_RECORD_WORDS) return ISING_EINVAL;
    int64_t *records = nullptr;
    if (scratch_for_current_device(&records) != cudaSuccess) return ISING_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // launch_measure first rewrites every record word it uses (t, zeroed M, B and D),
    // so nothing left over from an earlier call reaches the result.
    if (ising::launch_measure(lattice, L, replicas, 0, !(flags & ISING_MEAS_NO_CORR), records, s, nullptr) !=
        cudaSuccess)
        return ISING_ECUDA;
    if (ising::launch_derived(records, L, replicas, c, flags & ISING_MEAS_CONNECTED, derived, s, nullptr) !=
        cudaSuccess)
        return ISING_ECUDA;
    return ISING_OK;
}
