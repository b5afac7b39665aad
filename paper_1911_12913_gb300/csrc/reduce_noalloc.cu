// Allocation-free reduction entry point (declared in include/fdlbm.h as
// fdlbm_reduce_noalloc).
//
// Some callers cannot allocate device memory at the point where they want a
// conservation check: code running inside a framework that owns every device
// allocation (a memory pool or arena handed out by someone else), a
// fixed-footprint service loop that must not grow its memory after start-up,
// or a host thread that is not allowed to call cudaMalloc while other work is
// in flight.  This entry point takes only the caller's input and output
// buffers; its scratch (three partial sums per grid row: mass, |u|^2 and
// |u - u_prev|^2) lives in a file-scope device array that every GPU which
// loads the library holds until the process exits.
//
// Set-up: the first call on a device looks up the device address of that
// array (cudaGetSymbolAddress, with that device current) and caches it for
// the device's current CUDA context, so that first call should be made before
// any stream capture.  If that context is destroyed and another one is made
// current (cudaDeviceReset, or a library releasing the primary context), the
// module is loaded again, possibly at another address, and the next call looks
// the address up again; it should then also come before any capture.  All calls on a
// device share the array, and it keeps the previous call's partials; the row
// partials are rewritten in full by every call and the final pass writes the
// outputs directly, so nothing has to be cleared.  Two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fdlbm.h"

namespace {

constexpr int kMaxRows = 8192;    // largest ny accepted (scratch = 3 doubles per row)
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_row_partials[kMaxRows * 3];

std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};
void *g_ctx[kMaxDevices] = {};  // the context each cached address belongs to

// cuCtxGetCurrent from the driver, through the runtime's entry-point query (so
// that the library need not link the driver library itself).
using CtxGetCurrentFn = int (*)(void **);
CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    return fn;
}

// D2Q9 velocity components of the populations (Sec. 3 order).
__device__ __constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

__device__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;  // valid in thread 0
}

// One block per row: sums of rho/(m_x m_y), |u|^2 and |u - u_prev|^2, with
// rho = sum f and u = sum xi f / rho (no body-force correction).
__global__ void __launch_bounds__(kThreads)
    k_rows(const double *f, int nx, int ny, const double *mx, const double *my,
           const double *uprev, double *rows)
{
    __shared__ double red[kThreads / 32];
    const int y = blockIdx.x;
    const size_t N = (size_t)nx * ny;
    double m = 0.0, uu = 0.0, du = 0.0;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const size_t n = (size_t)y * nx + x;
        double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double v = f[i * N + n];
            r += v;
            jx += kCx[i] * v;
            jy += kCy[i] * v;
        }
        const double ux = jx / r, uy = jy / r;
        m += r / (mx[x] * my[y]);
        uu += ux * ux + uy * uy;
        if (uprev) {
            const double ex = ux - uprev[n], ey = uy - uprev[N + n];
            du += ex * ex + ey * ey;
        }
    }
    const double sm = block_sum(m, red);
    const double su = block_sum(uu, red);
    const double sd = block_sum(du, red);
    if (threadIdx.x == 0) {
        rows[3 * y + 0] = sm;
        rows[3 * y + 1] = su;
        rows[3 * y + 2] = sd;
    }
}

// Rows in a fixed order; out = (mass, residual or -1, sum |u|^2).
__global__ void __launch_bounds__(kThreads)
    k_final(const double *rows, int ny, int have_prev, double *out)
{
    __shared__ double red[kThreads / 32];
    double m = 0.0, uu = 0.0, du = 0.0;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        m += rows[3 * y + 0];
        uu += rows[3 * y + 1];
        du += rows[3 * y + 2];
    }
    const double sm = block_sum(m, red);
    const double su = block_sum(uu, red);
    const double sd = block_sum(du, red);
    if (threadIdx.x == 0) {
        out[0] = sm;
        // relative residual; a fluid exactly at rest (sum |u|^2 = 0) gets the
        // absolute one, which is 0 if it was at rest before as well
        out[1] = have_prev ? (su > 0.0 ? sqrt(sd / su) : sqrt(sd)) : -1.0;
        out[2] = su;
    }
}

// Device address of the scratch array on the current device, looked up once
// per device and context (again when the device's context has changed).
cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch[dev]) {
        void *ctx = nullptr;
        CtxGetCurrentFn get = ctx_get_current();
        // without the query every call looks the address up (no stale cache)
        if (get && get(&ctx) == 0 && ctx && ctx == g_ctx[dev]) {
            *out = g_scratch[dev];
            return cudaSuccess;
        }
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_row_partials);  // makes the context current if needed
    if (e != cudaSuccess) return e;
    void *ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (!get || get(&ctx) != 0) ctx = nullptr;
    g_scratch[dev] = static_cast<double *>(p);
    g_ctx[dev] = ctx;
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

int fdlbm_reduce_noalloc_max_rows(void) { return kMaxRows; }

fdlbm_status fdlbm_reduce_noalloc(const double *f, int nx, int ny, const double *dzeta_dx,
                                  const double *dmu_dy, const double *uprev, double *out,
                                  void *stream)
{
    if (!f || !dzeta_dx || !dmu_dy || !out || nx < 1 || ny < 1) return FDLBM_EINVAL;
    if (ny > kMaxRows) return FDLBM_ETOOBIG;
    // An error left pending by earlier, unrelated work on this thread is not
    // ours to clear or report as our own: refuse to launch and leave it.
    if (cudaPeekAtLastError() != cudaSuccess) return FDLBM_ECUDA;
    double *rows = nullptr;
    cudaError_t e = scratch_for_current_device(&rows);
    if (e != cudaSuccess) return FDLBM_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_rows<<<ny, kThreads, 0, s>>>(f, nx, ny, dzeta_dx, dmu_dy, uprev, rows);
    if (cudaGetLastError() != cudaSuccess) return FDLBM_ECUDA;
    k_final<<<1, kThreads, 0, s>>>(rows, ny, uprev != nullptr, out);
    return cudaGetLastError() == cudaSuccess ? FDLBM_OK : FDLBM_ECUDA;
}

}  // extern "C"
