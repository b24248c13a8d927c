// ds_tucker_static: the FP64 Tucker operator without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// Tucker operator: code running inside a custom allocator or memory-pool
// callback (where a nested cudaMalloc would re-enter the allocator),
// real-time or embedded hosts that forbid allocation after start-up, and
// plugins of frameworks that own the whole device heap.  For them the two
// intermediate tensors of the mode-product chain live in one fixed
// file-scope device array instead of temporaries.  That array is part of the
// loaded module: every GPU on which the library is loaded holds it until the
// process exits.
#include <mutex>
#include <string>

#include "ds_internal.h"

namespace {

// Largest grid (number of points N = n_1 ... n_d) the static scratch serves.
constexpr int64_t kStaticMaxPoints = (int64_t)1 << 20;

// Two FP64 intermediates of kStaticMaxPoints entries each (16 MiB).  Shared
// by every call on a device; it keeps whatever the last call left in it.
__device__ __align__(256) double g_static_scratch[2 * kStaticMaxPoints];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current, and cached for the life of the
// process.  The address belongs to the device's context: a cudaDeviceReset
// ends that context, and the cached address with it.
ds_status scratch_address(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ds::fail(DS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return ds::fail(DS_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return ds::fail(DS_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                             cudaGetErrorString(e));
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return DS_OK;
}

}  // namespace

extern "C" ds_status ds_tucker_static(const ds_grid *grid, const double *X, double *Y,
                                      const double *const *L, int transpose, void *stream)
{
    if (!grid || !X || !Y || !L) return ds::fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (grid->d < 2 || grid->d > ds::kMaxD) return ds::fail(DS_ERR_INVALID_ARG, "d must be 2, 3 or 4");
    int64_t N = 1;
    for (int q = 0; q < grid->d; ++q) {
        if (grid->n[q] < 2 || grid->n[q] > kStaticMaxPoints)
            return ds::fail(DS_ERR_INVALID_ARG, "n_mu must be in [2, 2^20]");
        if (!L[q]) return ds::fail(DS_ERR_INVALID_ARG, "L[mu] is NULL");
        N *= grid->n[q];
        if (N > kStaticMaxPoints)
            return ds::fail(DS_ERR_INVALID_ARG,
                            "grid has more than 1048576 points, the size of the static scratch of "
                            "ds_tucker_static; use ds_tucker");
    }
    ds_status r = ds::check_device();
    if (r != DS_OK) return r;
    double *scratch = nullptr;
    r = scratch_address(&scratch);
    if (r != DS_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    // every mode product writes all of its output (beta = 0), so nothing in
    // the scratch needs clearing between calls
    const double *in = X;
    for (int mu = 0; mu < grid->d; ++mu) {
        double *out = (mu == grid->d - 1) ? Y : scratch + (mu % 2) * kStaticMaxPoints;
        ds::launch_mode_product_f64(grid->d, grid->n, in, mu, L[mu], transpose, out, 1.0, 0.0, st);
        in = out;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ds::fail(DS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return DS_OK;
}
