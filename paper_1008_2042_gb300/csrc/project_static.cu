// cbct_project_static: the forward projection of cbct_project for callers that must not
// allocate device memory once they are running, e.g. services that fix their device
// memory footprint at start-up and treat any later allocation as a failure, or
// latency-critical loops that cannot afford the device-wide synchronisation an allocation
// may cause. cbct_project keeps its scratch (the volume rearranged into the projector's
// z-contiguous layout) in memory it allocates on first use; this entry point keeps the
// same scratch in a fixed array compiled into the library instead, so a call allocates
// nothing.
#include <mutex>

#include "cbct_internal.cuh"

namespace cbct {

// Fixed scratch: the z-contiguous copy of the input volume, plus the slack the projector
// may read past a volume's end. Every GPU that loads the library holds this array (16 MiB)
// until the process exits.
static __device__ __align__(256) float g_static_volume[CBCT_PROJECT_STATIC_MAX_VOXELS + PROJECT_VOLUME_SLACK / 4];

// In host code `g_static_volume` names a host-side stand-in, not device memory, so the
// device address is looked up once per device (with that device current) and cached for
// the life of the process (a device reset after the first call is not supported).
constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static float *g_static_ptr[kMaxDevices];

static cbct_status static_volume_address(int device, float **out)
{
    if (device < 0 || device >= kMaxDevices)
        return set_error(CBCT_ERR_UNSUPPORTED, "project_static: device ordinal %d not supported", device);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_volume);
        if (e != cudaSuccess) return check_cuda(e, "project_static: scratch address");
        g_static_ptr[device] = static_cast<float *>(p);
    }
    *out = g_static_ptr[device];
    return CBCT_OK;
}

} // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_project_static(const cbct_geometry *g, const float *f, float *g_out,
                                           cbct_stream_t stream)
{
    if (!g) return set_error(CBCT_ERR_INVALID_ARG, "project_static: null geometry");
    if (!f || !g_out) return set_error(CBCT_ERR_INVALID_ARG, "project_static: null pointer");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "project_static: current device");
    if (dev != g->device)
        return set_error(CBCT_ERR_INVALID_ARG, "project_static: geometry belongs to device %d, current is %d",
                         g->device, dev);
    const GeomDev G = level_geom(g, 0);
    const long long n = (long long)G.nx * G.ny * G.nz;
    if (n > (long long)CBCT_PROJECT_STATIC_MAX_VOXELS)
        return set_error(CBCT_ERR_INVALID_ARG,
                         "project_static: volume of %lld voxels exceeds the fixed scratch of %d voxels", n,
                         (int)CBCT_PROJECT_STATIC_MAX_VOXELS);
    float *scratch = nullptr;
    cbct_status st = static_volume_address(dev, &scratch);
    if (st != CBCT_OK) return st;
    // the whole scratch region used is overwritten by the layout change before it is read
    cudaStream_t s = (cudaStream_t)stream;
    st = transpose(f, scratch, G.nx, G.ny, G.nz, true, s);
    if (st != CBCT_OK) return st;
    return launch_project(G, scratch, G.nz, (long long)G.nx * G.nz, 1, nullptr, g_out, PM_PLAIN, nullptr, 0.0f, s);
}
