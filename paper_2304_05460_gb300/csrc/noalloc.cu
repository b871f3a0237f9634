// noalloc.cu -- the FP64 kernel matvec for callers that must not allocate.
//
// Some callers cannot call cudaMalloc at all: services whose device memory is
// planned up front and handed out by their own pool (an allocation behind
// the pool's back breaks its budget, or fails once the pool holds the rest of
// the device), and plug-ins loaded into a host process that must not grow
// that process's device footprint.  afn_kernel_matvec allocates its split-K
// partial sums on every call; this entry point runs the same kernels with
// those partials in a fixed array that is part of the library image instead.
//
// The array is a file-scope __device__ buffer of NOALLOC_SCRATCH_BYTES
// (16 MiB).  Every GPU that loads this library holds it until the process
// exits.  Host code cannot use the array's name as a device address, so on
// the first call on each device (with that device current) the address is
// looked up once with cudaGetSymbolAddress and cached; make that first call
// on each device before any stream capture begins.  The call synchronises its
// stream before it returns.  All calls share the one array and it
// keeps whatever the last call left in it: every partial is written before it
// is read, so nothing needs clearing, but two calls whose kernels overlap on
// the GPU (different streams, no ordering between them) race on it.
#include <mutex>

#include "afn_internal.cuh"

namespace afn {

static constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB
static constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / sizeof(double)];

static void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
static std::mutex g_noalloc_mu;

// device memory of another GPU is refused: the kernels run on the current one
static bool on_current_device(const void *ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || a.device == dev;
}

// device address of the scratch array on the current device (looked up once)
static afn_status noalloc_scratch(void **out)
{
    int dev = 0;
    AFN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("afn_kernel_matvec_noalloc: device %d above the supported %d", dev,
                  NOALLOC_MAX_DEVICES);
        return AFN_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return AFN_OK;
}

}  // namespace afn

using namespace afn;

extern "C" afn_status afn_kernel_matvec_noalloc(const double *points, int64_t n, int32_t d,
                                                int32_t kernel, double l, double mu,
                                                const double *p, int32_t nrhs, double *q,
                                                void *stream)
{
    if (!points || !p || !q || n < 1 || d < 1 || d > 16 || nrhs < 1 || !(l > 0) || !(mu >= 0) ||
        (kernel != 0 && kernel != 1)) {
        set_error("afn_kernel_matvec_noalloc: invalid argument");
        return AFN_ERR_ARG;
    }
    if (!is_device_ptr(points) || !is_device_ptr(p) || !is_device_ptr(q)) {
        set_error("afn_kernel_matvec_noalloc: points, p and q must be device memory");
        return AFN_ERR_ARG;
    }
    if (!on_current_device(points) || !on_current_device(p) || !on_current_device(q)) {
        set_error("afn_kernel_matvec_noalloc: points, p and q must be on the current device");
        return AFN_ERR_ARG;
    }
    // columns per pass: the widest group whose partials fit the fixed scratch
    int g = 8;
    while (g > 1 && matvec64_scratch(n, g) > NOALLOC_SCRATCH_BYTES) g /= 2;
    if (matvec64_scratch(n, g) > NOALLOC_SCRATCH_BYTES) {
        set_error("afn_kernel_matvec_noalloc: n=%lld needs %zu bytes of scratch, the fixed "
                  "array holds %zu", (long long)n, matvec64_scratch(n, 1), NOALLOC_SCRATCH_BYTES);
        return AFN_ERR_ARG;
    }
    void *scratch = nullptr;
    AFN_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    KParams kp{kernel, l, mu};
    for (int c0 = 0; c0 < nrhs; c0 += g) {
        int cols = nrhs - c0 < g ? nrhs - c0 : g;
        AFN_TRY(matvec64(points, n, d, kp, p + (int64_t)c0 * n, cols, q + (int64_t)c0 * n, scratch,
                         NOALLOC_SCRATCH_BYTES, s));
    }
    AFN_CUDA(cudaStreamSynchronize(s));
    return AFN_OK;
}
