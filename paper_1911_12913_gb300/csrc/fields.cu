// Kernels that move data between the caller's FP64 fields and the stored
// deviations g_i = f~_i - w_i rho0 (in FP64 or FP32), plus the moments of
// Eq. 3.3 and the FP64 mass / residual reductions.
//
// Every kernel here handles the rows [row0, row0 + nrows) of the grid; the
// caller-side arrays hold exactly those rows, x fastest, and multi-field
// arrays place field k at offset k * fstride elements.
#include "internal.h"

namespace fdlbm {
namespace {

constexpr int kRedThreads = 256;

// Initial f~ from (rho, u) and optionally the velocity gradient.  The physical
// distribution is f = f^eq (Eq. 3.2), plus the non-equilibrium part of Eq. 3.5
// with the coefficient rho0 w_i (2 tau + dt) / (2 cs^2) when grad is given; the
// stored variable is f~ = f - (dt/2) Omega-bar(f) (Eq. 2.19), which with a body
// force carries -(dt/2) F_i(rho, u) (Eq. 3.12), so that Eq. 3.3 reads back the
// given velocity.  The force is the handle's field at the time of the call.
// Fields of type T (FP64, or FP32 with DEV: the density given as rho - rho0,
// so that FP32 keeps its small variations); the arithmetic is in the storage
// precision R, whose rounding the stored deviations take anyway.
template <class R, class T, bool DEV>
__global__ void k_init(StepArgs<R> a, const R *force, const T *rho, const T *ux, const T *uy,
                       const T *grad, size_t fstride, int row0, int nrows, double tau, double dt,
                       double rho0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || j >= nrows) return;
    const size_t l = (size_t)j * a.nx + x;
    const R drho = DEV ? R(rho[l]) : R(double(rho[l]) - rho0);
    const R r0 = R(rho0), u = R(ux[l]), v = R(uy[l]);
    const R r = r0 + drho;
    R geq[9], F[9];
    equilibrium_dev<R>(drho, a.c.incomp ? r0 : r, u, v, geq);
    const size_t o = (size_t)(row0 + j) * a.pitch + x;
    if (force) {
        force_terms<R>(r0, geq, u, v, force[o], force[a.plane + o], F, a.c.incomp ? drho : R(0));
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) F[i] = R(0);
    }
    // Eq. 3.5 with the coefficient rho0 w_i (2 tau + dt) / (2 cs^2)
    const R k = R(rho0 * (2.0 * tau + dt) * 1.5);
    const R hdt = R(0.5 * dt);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R val = geq[i] - hdt * F[i];
        if (grad) {
            const R gxx = R(grad[l]), gxy = R(grad[fstride + l]), gyx = R(grad[2 * fstride + l]),
                    gyy = R(grad[3 * fstride + l]);
            const R d = R(cx(i) * cx(i)) * gxx + R(cx(i) * cy(i)) * (gxy + gyx) + R(cy(i) * cy(i)) * gyy;
            val -= k * wq<R>(i) * d;
        }
        a.gout[i * a.plane + o] = val;
    }
}

template <class R>
__global__ void k_convert_in(StepArgs<R> a, const double *f, size_t fstride, int row0, int nrows,
                             double rho0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || j >= nrows) return;
    const size_t l = (size_t)j * a.nx + x, o = (size_t)(row0 + j) * a.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) a.gout[i * a.plane + o] = R(f[i * fstride + l] - wq<double>(i) * rho0);
}

template <class R>
__global__ void k_convert_out(StepArgs<R> a, double *f, size_t fstride, int row0, int nrows,
                              double rho0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || j >= nrows) return;
    const size_t l = (size_t)j * a.nx + x, o = (size_t)(row0 + j) * a.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * fstride + l] = double(a.gin[i * a.plane + o]) + wq<double>(i) * rho0;
}

template <class R>
__global__ void k_set_force(StepArgs<R> a, R *force, const double *src, size_t fstride, int row0,
                            int nrows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || j >= nrows) return;
    const size_t l = (size_t)j * a.nx + x, o = (size_t)(row0 + j) * a.pitch + x;
    force[o] = R(src[l]);
    force[a.plane + o] = R(src[fstride + l]);
}

// Eq. 3.3 in the storage precision R: rho - rho0 and u.
template <class R>
__device__ void node_moments_r(const StepArgs<R> &a, const R *force, size_t o, R rho0, R half_dt,
                               R &drho, R &ux, R &uy)
{
    R g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = a.gin[i * a.plane + o];
    R jx, jy;
    moments_dev<R>(g, drho, jx, jy);
    const R rm = a.c.incomp ? rho0 : rho0 + drho;
    if (force) {
        jx += half_dt * rm * force[o];
        jy += half_dt * rm * force[a.plane + o];
    }
    const R inv = node_reciprocal<R>(rm);
    ux = jx * inv;
    uy = jy * inv;
}

// Density (or with DEV its deviation rho - rho0) and velocity into fields of
// type T, computed in the storage precision.
template <class R, class T, bool DEV>
__global__ void k_moments(StepArgs<R> a, const R *force, T *rho, T *ux, T *uy, int row0, int nrows,
                          double rho0, double half_dt)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || j >= nrows) return;
    const size_t l = (size_t)j * a.nx + x, o = (size_t)(row0 + j) * a.pitch + x;
    R dr, u, v;
    node_moments_r<R>(a, force, o, R(rho0), R(half_dt), dr, u, v);
    rho[l] = DEV ? T(dr) : T(rho0 + double(dr));
    ux[l] = T(u);
    uy[l] = T(v);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// Per-block partial sums of  J rho,  |u|^2,  |u - u_prev|^2  (J = 1/(m_x m_y)),
// then u_prev <- u.  Rows are dealt to the blocks in a fixed stride and each
// block's threads sweep a row's columns (coalesced, no index division); the
// block count is fixed, so the order of the sums is too.
template <class R>
__global__ void __launch_bounds__(kRedThreads)
    k_reduce_partial(StepArgs<R> a, const R *force, const double *mxd, const double *myd,
                     double *uprev, int use_prev, double rho0, double half_dt, double *partials)
{
    __shared__ double red[3][kRedThreads / 32];
    const size_t N = (size_t)a.nx * a.ny;
    double m = 0.0, uu = 0.0, du = 0.0;
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
        const double my = myd[y];
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            const size_t n = (size_t)y * a.nx + x;
            const size_t o = (size_t)y * a.pitch + x;
            // moments in the storage precision (FP32 states carry no more), sums
            // in FP64
            R dr, ur, vr;
            node_moments_r<R>(a, force, o, R(rho0), R(half_dt), dr, ur, vr);
            const double r = rho0 + double(dr), u = double(ur), v = double(vr);
            m += r / (mxd[x] * my);
            uu += u * u + v * v;
            if (use_prev) {
                const double eu = u - uprev[n], ev = v - uprev[N + n];
                du += eu * eu + ev * ev;
            }
            uprev[n] = u;
            uprev[N + n] = v;
        }
    }
    m = warp_sum(m);
    uu = warp_sum(uu);
    du = warp_sum(du);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = m;
        red[1][wid] = uu;
        red[2][wid] = du;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) s += red[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kRedThreads)
    k_reduce_final(const double *partials, int nblocks, double *out)
{
    __shared__ double red[3][kRedThreads / 32];
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 3; ++k) s[k] += partials[(size_t)b * 3 + k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) {
        s[k] = warp_sum(s[k]);
        if (lane == 0) red[k][wid] = s[k];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += red[threadIdx.x][w];
        out[threadIdx.x] = t;
    }
}

template <class R>
StepArgs<R> view(fdlbm_ctx *h)
{
    StepArgs<R> a{};
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.gin = reinterpret_cast<const R *>(h->ws + h->lay.state[h->cur]);
    a.gout = reinterpret_cast<R *>(h->ws + h->lay.state[h->cur]);
    a.c.incomp = h->incomp;
    return a;
}

inline dim3 grid2(int nx, int nrows, dim3 blk)
{
    return dim3((nx + blk.x - 1) / blk.x, (nrows + blk.y - 1) / blk.y);
}

}  // namespace

#define DISPATCH(h, R, ...)                           \
    do {                                              \
        if ((h)->precision == FDLBM_FP32_DEV) {       \
            using R = float;                          \
            __VA_ARGS__;                              \
        } else {                                      \
            using R = double;                         \
            __VA_ARGS__;                              \
        }                                             \
    } while (0)

template <class T>
cudaError_t launch_init_fields(fdlbm_ctx *h, const T *rho, const T *ux, const T *uy, const T *grad,
                               int row0, int nrows, size_t fstride)
{
    const dim3 blk(32, 8);
    constexpr bool dev = sizeof(T) == 4;  // FP32 fields give the density as rho - rho0
    DISPATCH(h, R,
             const R *force = h->has_force ? reinterpret_cast<const R *>(h->ws + h->lay.force)
                                           : nullptr;
             k_init<R, T, dev><<<grid2(h->nx, nrows, blk), blk, 0, h->stream>>>(
                 view<R>(h), force, rho, ux, uy, grad, fstride, row0, nrows, h->tau, h->dt,
                 h->rho0));
    return cudaGetLastError();
}
template cudaError_t launch_init_fields<double>(fdlbm_ctx *, const double *, const double *,
                                                const double *, const double *, int, int, size_t);
template cudaError_t launch_init_fields<float>(fdlbm_ctx *, const float *, const float *,
                                               const float *, const float *, int, int, size_t);

cudaError_t launch_convert_in(fdlbm_ctx *h, const double *f, int row0, int nrows, size_t fstride)
{
    const dim3 blk(32, 8);
    DISPATCH(h, R, k_convert_in<R><<<grid2(h->nx, nrows, blk), blk, 0, h->stream>>>(
                       view<R>(h), f, fstride, row0, nrows, h->rho0));
    return cudaGetLastError();
}

cudaError_t launch_convert_out(fdlbm_ctx *h, double *f, int row0, int nrows, size_t fstride)
{
    const dim3 blk(32, 8);
    DISPATCH(h, R, k_convert_out<R><<<grid2(h->nx, nrows, blk), blk, 0, h->stream>>>(
                       view<R>(h), f, fstride, row0, nrows, h->rho0));
    return cudaGetLastError();
}

cudaError_t launch_set_force(fdlbm_ctx *h, const double *force, int row0, int nrows,
                             size_t fstride)
{
    const dim3 blk(32, 8);
    DISPATCH(h, R, k_set_force<R><<<grid2(h->nx, nrows, blk), blk, 0, h->stream>>>(
                       view<R>(h), reinterpret_cast<R *>(h->ws + h->lay.force), force, fstride,
                       row0, nrows));
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_moments(fdlbm_ctx *h, T *rho, T *ux, T *uy, int row0, int nrows,
                           size_t /*fstride*/)
{
    const dim3 blk(32, 8);
    constexpr bool dev = sizeof(T) == 4;  // FP32 fields get the density as rho - rho0
    DISPATCH(h, R,
             const R *force = h->has_force ? reinterpret_cast<const R *>(h->ws + h->lay.force)
                                           : nullptr;
             k_moments<R, T, dev><<<grid2(h->nx, nrows, blk), blk, 0, h->stream>>>(
                 view<R>(h), force, rho, ux, uy, row0, nrows, h->rho0, 0.5 * h->dt));
    return cudaGetLastError();
}
template cudaError_t launch_moments<double>(fdlbm_ctx *, double *, double *, double *, int, int,
                                            size_t);
template cudaError_t launch_moments<float>(fdlbm_ctx *, float *, float *, float *, int, int, size_t);

cudaError_t launch_reduce(fdlbm_ctx *h, int use_prev)
{
    double *partials = reinterpret_cast<double *>(h->ws + h->lay.partials);
    double *out = reinterpret_cast<double *>(h->ws + h->lay.red);
    const double *mxd = reinterpret_cast<const double *>(h->ws + h->lay.mxd);
    const double *myd = reinterpret_cast<const double *>(h->ws + h->lay.myd);
    double *uprev = reinterpret_cast<double *>(h->ws + h->lay.uprev);
    DISPATCH(h, R,
             const R *force = h->has_force ? reinterpret_cast<const R *>(h->ws + h->lay.force)
                                           : nullptr;
             k_reduce_partial<R><<<h->lay.nblocks_red, kRedThreads, 0, h->stream>>>(
                 view<R>(h), force, mxd, myd, uprev, use_prev, h->rho0, 0.5 * h->dt, partials));
    k_reduce_final<<<1, kRedThreads, 0, h->stream>>>(partials, h->lay.nblocks_red, out);
    return cudaGetLastError();
}

}  // namespace fdlbm
