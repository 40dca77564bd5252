// Allocation-free variant of the FP64 mass sums (include/lbe.h,
// lbe_mass_noalloc).  The per-block partial sums live in a fixed array in
// the library's device memory instead of memory obtained from cudaMalloc.
#include <mutex>

#include "lbe_internal.cuh"

namespace {

constexpr int SCRATCH_BLOCKS = 1024;  // partial sums per component

// Scratch of the mass sums: 2 x 1024 doubles (16 KiB) on every GPU that
// loads the library, held until the process exits.  Every call shares it.
static __device__ __align__(256) double g_mass_scratch[2 * SCRATCH_BLOCKS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on `dev` (which must be current).
// The host-side name of the array is only a stand-in, so the address is
// looked up once per device and cached for the life of the process.  A
// device reset (cudaDeviceReset) reloads the module, after which the cached
// address is stale: callers that reset a device must not call
// lbe_mass_noalloc on it afterwards.
cudaError_t scratch_on(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" LBE_API lbe_status lbe_mass_noalloc(const void *f, int32_t storage, const uint8_t *node_type,
                                               int64_t nodes, int64_t slot_stride, const double rho_ref[2],
                                               int32_t device, void *cuda_stream, double *out)
{
    using namespace lbe;
    if (!f || !node_type || !out) return LBE_EINVAL;
    if (nodes < 1 || nodes > LBE_NOALLOC_MAX_NODES || slot_stride < nodes) return LBE_EINVAL;
    if (storage < LBE_STORE_F32 || storage > LBE_STORE_F16_OFS) return LBE_EINVAL;
    if (storage != LBE_STORE_F32 && !rho_ref) return LBE_EINVAL;
    if (device < -1) return LBE_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return LBE_ECUDA;
    const int dev = device >= 0 ? device : prev;
    if (dev >= MAX_DEVICES) return LBE_EINVAL;
    if (dev != prev && cudaSetDevice(dev) != cudaSuccess) return LBE_EINVAL;
    lbe_status st = LBE_OK;
    double *scratch = nullptr;
    if (scratch_on(dev, &scratch) != cudaSuccess) {
        st = LBE_ECUDA;
    } else {
        Lat L{};
        L.nx = (int)nodes;
        L.ny = 1;
        L.nz = 1;
        L.N = (int)nodes;
        L.S = slot_stride;
        for (int c = 0; c < 2; c++)
            for (int i = 0; i < Q; i++)
                L.base[c][i] = storage == LBE_STORE_F32 ? 0.f : (float)(wgtd(i) * rho_ref[c]);
        // every block writes its own partial sums, so nothing needs clearing
        launch_mass(storage, L, f, node_type, scratch, SCRATCH_BLOCKS, out, (cudaStream_t)cuda_stream);
        if (cudaGetLastError() != cudaSuccess) st = LBE_ECUDA;
    }
    // the caller's current device is left as it was
    if (dev != prev) cudaSetDevice(prev);
    return st;
}
