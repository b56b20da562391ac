// kpm_spectrum_static: the spectrum reconstruction without any allocation.
//
// kpm_spectrum allocates device buffers for every call.  Some callers cannot
// call cudaMalloc: processes whose device memory is entirely reserved by
// another allocator (a framework's caching pool, a fixed memory plan), where
// cudaMalloc fails, and latency-critical loops that cannot pay for
// cudaMalloc/cudaFree, which synchronise the device.  This entry point takes the
// moments and both outputs as caller-owned device buffers and keeps its only
// scratch -- the damped moments g_n Omega_n -- in a file-scope __device__ array
// of fixed size that every GPU loading the library holds until the process
// exits.
#include <mutex>

#include "common.cuh"

// Scratch for the damped moments: 2 MiB per device, file scope, internal linkage.
static __device__ __align__(256) double g_spectrum_scratch[KPM_SPECTRUM_STATIC_MAX_MOMENTS];

namespace kpm {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current and cached.  A cudaDeviceReset destroys
// the context that held the array; the cached address is then stale, so a
// process that resets a device must not call kpm_spectrum_static on it again.
double* scratch_address() {
    int dev = 0;
    KPM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        KPM_THROW(KPM_EUNSUPPORTED, "device index %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            KPM_THROW(KPM_ECUDA, "cudaGetSymbolAddress(spectrum scratch) failed: %s",
                      cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    return g_scratch_addr[dev];
}

}  // namespace
}  // namespace kpm

using namespace kpm;

extern "C" kpm_status kpm_spectrum_static(const double* moments_dev, int nmoments, double a,
                                          double b, int npoints, int kernel, double* omega_dev,
                                          double* intensity_dev, void* cuda_stream) {
    try {
        if (!moments_dev || !omega_dev || !intensity_dev)
            KPM_THROW(KPM_EINVAL, "NULL argument");
        if (nmoments < 1 || npoints < 1 || kernel < 0 || kernel > 2)
            KPM_THROW(KPM_EINVAL, "bad spectrum arguments");
        if (nmoments > KPM_SPECTRUM_STATIC_MAX_MOMENTS)
            KPM_THROW(KPM_EINVAL,
                      "nmoments = %d exceeds the static scratch of %d moments; use kpm_spectrum",
                      nmoments, KPM_SPECTRUM_STATIC_MAX_MOMENTS);
        if (!(a > 0.0)) KPM_THROW(KPM_EINVAL, "a must be > 0");
        double* scratch = scratch_address();
        // Every element of the scratch that is read is written first (k_damp
        // writes g_n Omega_n for n < nmoments before the reconstruction reads
        // them, in stream order), so nothing needs clearing between calls.
        spectrum_dev(moments_dev, nmoments, a, b, npoints, kernel, scratch, omega_dev,
                     intensity_dev, (cudaStream_t)cuda_stream);
        return KPM_OK;
    } catch (const Error& e) {
        set_thread_error(e.msg);
        return e.status;
    } catch (...) {
        set_thread_error("unknown error");
        return KPM_ECUDA;
    }
}
