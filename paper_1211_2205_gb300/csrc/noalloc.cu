// Allocation-free variant of the FP64 diagnostics reduction.
//
// Some callers cannot allocate device memory at the point where they need
// the reduction: a host application whose GPU memory is budgeted and handed
// out once at start-up, a plug-in that runs inside another framework's
// callback, or a real-time loop in which an allocation (and the implicit
// device synchronisation that cudaMalloc/cudaFree may bring) is not allowed.
// starmap_diagnostics_noalloc serves them: it runs the same two reduction
// kernels as starmap_diagnostics, but its per-block partial sums live in the
// file-scope array below instead of memory from cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "../../include/starmap.h"

namespace starmap {

namespace {

// Per-block partial sums (mass, sum of squares, non-finite count) of the
// first reduction kernel.  Every GPU that loads the library holds this array
// until the process exits.
constexpr int NOALLOC_BLOCKS = STARMAP_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_noalloc_partials[3 * NOALLOC_BLOCKS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[MAX_DEVICES] = {nullptr};
void* g_partials_ctx[MAX_DEVICES] = {nullptr};   // context the address was looked up in

// The current context's handle through the driver's cuCtxGetCurrent (found
// once by the runtime's entry-point query; the library does not link the
// driver library itself).  Null if it cannot be had.
void* current_context() {
    using GetCurrent = int (*)(void**);
    static GetCurrent fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (GetCurrent) nullptr;
        return reinterpret_cast<GetCurrent>(p);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of the scratch array on the current device, looked up
// with that device current (the array's name is only a host-side stand-in)
// the first time a device is used and again whenever the device's current
// context has changed since (after cudaDeviceReset, for instance).
int scratch_address(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return STARMAP_E_CUDA;
    void* ctx = current_context();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev] || ctx != g_partials_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) return STARMAP_E_CUDA;
        g_partials_addr[dev] = static_cast<double*>(p);
        g_partials_ctx[dev] = current_context();     // the lookup may have made the primary context current
    }
    *out = g_partials_addr[dev];
    return STARMAP_OK;
}

template <class T>
int run(const void* data, int ncomp, int nx, int ny, long pitch, long comp_stride, long origin, double cell,
        double* out_device, void* stream) {
    double* partials = nullptr;
    int rc = scratch_address(&partials);
    if (rc) return rc;
    ReduceArgs<T> a;
    a.g[0].base = const_cast<T*>(static_cast<const T*>(data)) + origin;   // point (0, 0): inside the caller's buffer
    a.row0 = 0;                                                          // row y sits at base + y * pitch
    a.g[0].cstride = comp_stride;
    a.g[0].nx = nx;
    a.g[0].ny = ny;
    a.g[0].K = ncomp;
    a.g[0].coef = nullptr;
    for (int g = 1; g < 4; ++g) a.g[g] = GridDev<T>();
    a.pitch = pitch;
    a.cell = cell;
    const long rows = (long)ncomp * ny;
    const int nblocks = (int)(rows < NOALLOC_BLOCKS ? rows : NOALLOC_BLOCKS);
    if (launch_reduce<T>(a, partials, nblocks, out_device, stream)) return STARMAP_E_CUDA;
    return STARMAP_OK;
}

}  // namespace

}  // namespace starmap

extern "C" int starmap_diagnostics_noalloc(const void* data, int precision, int ncomp, int nx, int ny, long pitch,
                                           long comp_stride, long origin, double cell, double* out_device,
                                           void* stream) {
    using namespace starmap;
    if (!data || !out_device) return STARMAP_E_ARG;
    if (precision != STARMAP_FP64 && precision != STARMAP_FP32) return STARMAP_E_ARG;
    if (ncomp < 1 || nx < 1 || ny < 1 || origin < 0) return STARMAP_E_ARG;
    if ((long)ncomp * ny > STARMAP_NOALLOC_MAX_ROWS || nx > STARMAP_NOALLOC_MAX_ROW_LENGTH) return STARMAP_E_ARG;
    // bounded before they are multiplied: ny <= 2^26 and pitch <= 2^31 keep pitch * ny far from overflow
    if (pitch < nx || pitch > STARMAP_NOALLOC_MAX_PITCH || comp_stride < pitch * (long)ny) return STARMAP_E_ARG;
    return precision == STARMAP_FP64
               ? run<double>(data, ncomp, nx, ny, pitch, comp_stride, origin, cell, out_device, stream)
               : run<float>(data, ncomp, nx, ny, pitch, comp_stride, origin, cell, out_device, stream);
}
