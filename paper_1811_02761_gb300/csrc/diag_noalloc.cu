// diag_noalloc.cu -- nbody_diagnostics_noalloc: the FP64 energy / momentum
// diagnostics without any device allocation.
//
// Some callers cannot call cudaMalloc: their device memory is reserved up
// front by another allocator (a framework's caching allocator or a fixed
// arena), or they run in a loop where an allocation's implicit device-wide
// synchronisation is not acceptable.  For them this entry point takes its
// scratch (the per-block FP64 partial sums, and an 8-double result slot) from
// a file-scope device array instead of from a context.
//
// The array is fixed-size and shared by every call in the process:
//   * every GPU that loads the library holds it (kNoallocScratchDoubles
//     doubles, 65.6 KB) until the process exits;
//   * nothing in it has to start at zero -- a call overwrites every partial
//     slot it later reads, and the result slot;
//   * two calls whose kernels overlap on the GPU (different streams, or
//     different host threads) race on the array and may return mixed results.
// On the first call on a device (with that device current) the library looks
// up the array's device address with cudaGetSymbolAddress and caches it; make
// that first call before any stream capture.  The cached address belongs to
// the device's current CUDA context: after a cudaDeviceReset the array may
// sit elsewhere, so the library must not be used across a reset (nor must any
// nbody_ctx, whose device memory a reset frees).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace nb {

// True for memory the current device dev can read in place: its own device
// memory, or managed memory.  Device memory of another GPU is refused (the
// kernel runs on dev and would read it across the peer link, or fault when
// peer access is off).
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace nb

namespace {

// Partial sums of up to kNoallocBlocks blocks (8 doubles each) + the result.
constexpr int kNoallocBlocks = 1024;
constexpr int kNoallocScratchDoubles = kNoallocBlocks * 8 + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
nbody_status fail(nbody_status st, const std::string &msg) {
    nb::set_stateless_error(msg);  // read back by nbody_last_error(NULL, ...)
    return st;
}

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" nbody_status nbody_diagnostics_noalloc(int64_t n, const double *x, const double *y,
                                                  const double *z, const float *vx,
                                                  const float *vy, const float *vz,
                                                  const float *m, const float *phi, double *out,
                                                  void *cuda_stream) {
    if (n < 1 || n >= ((int64_t)1 << 31))
        return fail(NBODY_EINVAL, "nbody_diagnostics_noalloc: n must be in 1..2^31-1");
    if (!x || !y || !z || !vx || !vy || !vz || !m || !out)
        return fail(NBODY_EINVAL, "nbody_diagnostics_noalloc: NULL array");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(NBODY_ECUDA, "nbody_diagnostics_noalloc: no current CUDA device");
    }
    const void *in[8] = {x, y, z, vx, vy, vz, m, phi};
    for (int k = 0; k < 8; k++)
        if (in[k] && !nb::on_device(in[k], dev))
            return fail(NBODY_EINVAL,
                        "nbody_diagnostics_noalloc: input arrays must be device pointers of the "
                        "current device (staging host arrays would need an allocation)");
    cudaPointerAttributes oat;
    if (cudaPointerGetAttributes(&oat, out) != cudaSuccess) cudaGetLastError();
    else if (oat.type == cudaMemoryTypeDevice && oat.device != dev)
        return fail(NBODY_EINVAL,
                    "nbody_diagnostics_noalloc: out is device memory of another GPU");
    // the diagnostics kernel grid-strides over at most kNoallocBlocks blocks,
    // so the partial sums of every n fit the array
    if (nb::diag_temp_bytes() > (size_t)kNoallocBlocks * 8 * sizeof(double))
        return fail(NBODY_EINVAL, "nbody_diagnostics_noalloc: scratch array too small");
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess)
        return fail(NBODY_ECUDA, std::string("nbody_diagnostics_noalloc: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool out_dev = nb::on_device(out, dev);
    double *result = out_dev ? out : scratch + kNoallocBlocks * 8;
    nb::launch_diagnostics(s, n, x, y, z, vx, vy, vz, m, phi, scratch, result);
    e = cudaGetLastError();
    if (e == cudaSuccess && !out_dev)
        e = cudaMemcpyAsync(out, result, 8 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return fail(NBODY_ECUDA, std::string("nbody_diagnostics_noalloc: ") + cudaGetErrorString(e));
    return NBODY_OK;
}
