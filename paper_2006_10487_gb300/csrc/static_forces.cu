// Drag and lift coefficients from caller-owned device buffers, computed with
// no device allocation at all: the per-block partial sums of the two-pass
// reduction live in a fixed file-scope device array instead of memory taken
// from cudaMalloc or an allocator callback.
//
// Who needs this: callers that cannot call cudaMalloc, for instance code whose
// device memory is owned entirely by another framework's pool, or monitoring
// loops that must not pay for (or synchronise on) an allocation every time
// they evaluate the forces of a state they already hold.
//
// Limits and sharing rules:
//   - at most kStaticMaxEdges wall edges per call (larger inputs are rejected
//     with HLBM_EINVAL);
//   - every call on a device uses the same array, which keeps the partial sums
//     of the last call; nothing in it has to start at zero (each call writes
//     every slot it later reads), but calls that overlap on the GPU race, so
//     they must be ordered (one stream, or synchronised streams);
//   - the array exists on every device that loads the library, until exit;
//   - its device address is looked up on the first call per device and kept
//     for the life of the process, so it does not survive cudaDeviceReset (or
//     any other destruction of the device's primary context): a process that
//     resets a device must not call this entry point on it afterwards;
//   - edge end points outside [0, n_nodes) are not read: such edges are
//     skipped and the call writes NaN to both outputs.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "hlbm_internal.h"

namespace hlbm {
namespace {

constexpr int kStaticThreads = 128;
constexpr int kStaticMaxBlocks = 1024;
constexpr int kStaticMaxEdges = kStaticThreads * kStaticMaxBlocks;  // 131 072
constexpr int kMaxDevices = 64;

// Per block of the first pass: the (F_x, F_y) partial sum and a flag (1.0
// when one of the block's edges had an end point outside [0, n_nodes)).
static __device__ __align__(256) double g_force_scratch[3 * kStaticMaxBlocks];

// Device address of g_force_scratch per device (host code only sees a
// host-side stand-in for the symbol, so the address is looked up once per
// device with that device current).
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__device__ __forceinline__ int vx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__device__ __forceinline__ int vy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }

// Traction -(p - p0) n - Pi^neq . n of one wall edge a -> b (fluid on the
// left, n L = (-dy, dx)) with p = rho/3 and Pi^neq = sum c c (f - f^eq), edge
// values the mean of the two end nodes (Eq. 10-11).
__device__ void static_edge_force(const double *f, const double *xy, int a, int b, double &fx, double &fy)
{
    double p = 0.0, pxx = 0.0, pxy = 0.0, pyy = 0.0;
    for (int s = 0; s < 2; s++) {
        const double *fn = f + 9 * size_t(s ? b : a);
        double rho = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; i++) {
            rho += fn[i];
            jx += vx(i) * fn[i];
            jy += vy(i) * fn[i];
        }
        double ux = jx / rho, uy = jy / rho, uu = ux * ux + uy * uy;
        p += 0.5 * rho / 3.0;
        for (int i = 0; i < 9; i++) {
            double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
            double cu = vx(i) * ux + vy(i) * uy;
            double neq = fn[i] - w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            pxx += 0.5 * vx(i) * vx(i) * neq;
            pxy += 0.5 * vx(i) * vy(i) * neq;
            pyy += 0.5 * vy(i) * vy(i) * neq;
        }
    }
    double nx = -(xy[2 * b + 1] - xy[2 * a + 1]), ny = xy[2 * b] - xy[2 * a];
    double pm = p - 1.0 / 3.0;
    fx = -pm * nx - (pxx * nx + pxy * ny);
    fy = -pm * ny - (pxy * nx + pyy * ny);
}

__device__ __forceinline__ void static_block_sum(double &fx, double &fy)
{
    __shared__ double sx[32], sy[32];
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o);
        fy += __shfl_down_sync(0xffffffffu, fy, o);
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sx[warp] = fx; sy[warp] = fy; }
    __syncthreads();
    if (warp == 0) {
        int nw = (blockDim.x + 31) >> 5;
        fx = lane < nw ? sx[lane] : 0.0;
        fy = lane < nw ? sy[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_down_sync(0xffffffffu, fx, o);
            fy += __shfl_down_sync(0xffffffffu, fy, o);
        }
    }
}

__global__ void __launch_bounds__(kStaticThreads)
k_static_force_partial(const double *f, const double *xy, const int32_t *ea, const int32_t *eb, int n_edges,
                       int n_nodes, double *scratch)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    double fx = 0.0, fy = 0.0;
    int bad = 0;
    if (e < n_edges) {
        int a = ea[e], b = eb[e];
        if (a >= 0 && a < n_nodes && b >= 0 && b < n_nodes) static_edge_force(f, xy, a, b, fx, fy);
        else bad = 1;  // never read past f or xy
    }
    bad = __syncthreads_or(bad);
    static_block_sum(fx, fy);
    if (threadIdx.x == 0) {
        scratch[3 * blockIdx.x] = fx;
        scratch[3 * blockIdx.x + 1] = fy;
        scratch[3 * blockIdx.x + 2] = bad ? 1.0 : 0.0;
    }
}

// Second pass: the partials in block order (fixed order: deterministic).
__global__ void __launch_bounds__(kStaticThreads)
k_static_force_final(const double *scratch, int n_part, double qdyn, double *out)
{
    double fx = 0.0, fy = 0.0;
    int bad = 0;
    for (int b = threadIdx.x; b < n_part; b += blockDim.x) {
        fx += scratch[3 * b];
        fy += scratch[3 * b + 1];
        bad |= scratch[3 * b + 2] != 0.0;
    }
    bad = __syncthreads_or(bad);
    static_block_sum(fx, fy);
    if (threadIdx.x == 0) {
        out[0] = bad ? CUDART_NAN : fx / qdyn;
        out[1] = bad ? CUDART_NAN : fy / qdyn;
    }
}

// Device address of the scratch array on the current device; the lookup
// runs on the first call per device.
cudaError_t scratch_on_current_device(double **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_force_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *ptr = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace hlbm

extern "C" int hlbm_wall_forces_static(const double *f, int n_nodes, const double *xy, const int32_t *edge_a,
                                       const int32_t *edge_b, int n_edges, double qdyn, double *out, void *stream)
{
    using namespace hlbm;
    if (!f || !xy || !edge_a || !edge_b || !out || n_nodes < 1 || n_edges < 1 || !(qdyn > 0.0)) {
        set_thread_error("hlbm_wall_forces_static: missing buffer, empty input or non-positive qdyn");
        return HLBM_EINVAL;
    }
    if (n_edges > kStaticMaxEdges) {
        set_thread_error("hlbm_wall_forces_static: " + std::to_string(n_edges) + " wall edges exceed the limit of " +
                         std::to_string(kStaticMaxEdges) + " of the fixed scratch array");
        return HLBM_EINVAL;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) {
        set_thread_error(std::string("hlbm_wall_forces_static: scratch address lookup failed: ") +
                         cudaGetErrorString(e));
        return HLBM_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nb = (n_edges + kStaticThreads - 1) / kStaticThreads;
    k_static_force_partial<<<nb, kStaticThreads, 0, s>>>(f, xy, edge_a, edge_b, n_edges, n_nodes, scratch);
    k_static_force_final<<<1, kStaticThreads, 0, s>>>(scratch, nb, qdyn, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(std::string("hlbm_wall_forces_static: launch failed: ") + cudaGetErrorString(e));
        return HLBM_ECUDA;
    }
    return HLBM_OK;
}
