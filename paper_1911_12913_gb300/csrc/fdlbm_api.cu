// C ABI of the T2S2-FDLBM library (declared in include/fdlbm.h): argument
// checks, workspace layout, host<->device staging and kernel dispatch.  No
// arithmetic of the method runs here; every step runs in the kernels of
// step_fused.cu, step_staged.cu and fields.cu.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace fdlbm;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStagingBytes = size_t(64) << 20;  // host<->device staging chunk
constexpr int kRedBlocks = 152 * 4;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

fdlbm_status fail(fdlbm_ctx *h, fdlbm_status s, const char *what)
{
    if (h) h->err = what;
    return s;
}

fdlbm_status cuda_fail(fdlbm_ctx *h, cudaError_t e, const char *where)
{
    if (h) {
        h->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return FDLBM_ECUDA;
}

bool valid_axis(const double *c, int n)
{
    if (!c || n < 3) return false;
    for (int i = 1; i < n; ++i)
        if (!(c[i] > c[i - 1]) || !std::isfinite(c[i])) return false;
    return std::isfinite(c[0]);
}

double period(const double *c, int n, double l)
{
    return l > 0 ? l : n * (c[1] - c[0]);
}

double min_spacing(const double *c, int n, bool periodic, double l)
{
    double m = INFINITY;
    for (int i = 1; i < n; ++i) m = std::min(m, c[i] - c[i - 1]);
    if (periodic) m = std::min(m, c[0] + period(c, n, l) - c[n - 1]);
    return m;
}

bool grid_ok(const fdlbm_grid *g)
{
    if (!g) return false;
    if (g->bc_x != FDLBM_PERIODIC && g->bc_x != FDLBM_WALL) return false;
    if (g->bc_y != FDLBM_PERIODIC && g->bc_y != FDLBM_WALL) return false;
    if (!valid_axis(g->x, g->nx) || !valid_axis(g->y, g->ny)) return false;
    if (g->bc_x == FDLBM_PERIODIC && !(g->x[0] + period(g->x, g->nx, g->lx) > g->x[g->nx - 1]))
        return false;
    if (g->bc_y == FDLBM_PERIODIC && !(g->y[0] + period(g->y, g->ny, g->ly) > g->y[g->ny - 1]))
        return false;
    return true;
}

int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

bool fused_ok(const fdlbm_grid *g) { return g->nx >= 4 && g->ny >= 4; }

bool walled(const fdlbm_grid *g) { return g->bc_x == FDLBM_WALL || g->bc_y == FDLBM_WALL; }

// The automatic choice takes the fused sweep for T2S2-FDLBM1, except on walled
// grids in FP64: there the work is bound by the FP64 units, and the halo rows
// the sweep recomputes on small walled grids cost more than the staged
// kernels' extra traffic (257^2 cavity: 198 against 81 us per step on GB300).
// Both schemes have fused sweeps, for periodic and walled grids.
int choose_path(const fdlbm_grid *g, const fdlbm_opts *o)
{
    const bool can_fuse = fused_ok(g);
    if (o->path == FDLBM_PATH_STAGED) return FDLBM_PATH_STAGED;
    if (o->path == FDLBM_PATH_FUSED) return can_fuse ? FDLBM_PATH_FUSED : -1;
    if (walled(g) && o->precision == FDLBM_FP64) return FDLBM_PATH_STAGED;
    return can_fuse ? FDLBM_PATH_FUSED : FDLBM_PATH_STAGED;
}

// Rows per CTA of the fused kernel.  Each CTA recomputes 8 halo rows, so tall
// tiles waste less; the grid should also fill whole waves of resident CTAs.
// Pick the height that minimises (waves) x (rows + 8), the modelled sweep time
// (on small grids that is a short segment: more CTAs, each walking fewer rows).
int choose_rows(int nx, int ny, int precision, int variant, bool walls, int scheme)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f32 = precision == FDLBM_FP32_DEV;
    int per_sm;
    if (variant == FDLBM_VARIANT_WARP)
        per_sm = fused_warp_blocks_per_sm();
    else if (scheme == FDLBM_SCHEME_T2S2_2)
        per_sm = f32 ? fused_s2_blocks_per_sm<float>() : fused_s2_blocks_per_sm<double>();
    else if (walls)
        per_sm = f32 ? fused_walls_blocks_per_sm<float>() : fused_walls_blocks_per_sm<double>();
    else
        per_sm = f32 ? fused_blocks_per_sm<float>() : fused_blocks_per_sm<double>();
    if (per_sm <= 0) per_sm = 1;
    const long long slots = (long long)per_sm * sms;
    const int W = variant == FDLBM_VARIANT_WARP ? fused_warp_tile_width() : fused_tile_width();
    const long long strips = (nx + W - 1) / W;
    int best = std::min(ny, 64);
    double best_cost = 1e300;
    for (int rows = 1; rows <= std::min(ny, 512); ++rows) {
        const long long ctas = strips * ((ny + rows - 1) / rows);
        const long long waves = (ctas + slots - 1) / slots;
        const double cost = (double)waves * (rows + 8);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = rows;
        }
    }
    return std::max(1, std::min(best, ny));
}

template <class R>
StepArgs<R> step_args(fdlbm_ctx *h)
{
    StepArgs<R> a{};
    a.gin = reinterpret_cast<const R *>(h->ws + h->lay.state[h->cur]);
    a.gout = reinterpret_cast<R *>(h->ws + h->lay.state[1 - h->cur]);
    a.mx = reinterpret_cast<const R *>(h->ws + h->lay.mx);
    a.my = reinterpret_cast<const R *>(h->ws + h->lay.my);
    a.force = h->has_force ? reinterpret_cast<const R *>(h->ws + h->lay.force) : nullptr;
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.bc_x = h->bc_x;
    a.bc_y = h->bc_y;
    for (int s = 0; s < 4; ++s)
        for (int k = 0; k < 2; ++k) a.wall_u[s][k] = R(h->wall_u[s][k]);
    // T2S2-FDLBM2 marches its characteristic estimate over h = dt
    a.c = make_coeffs<R>(h->tau, h->dt, h->scheme == FDLBM_SCHEME_T2S2_2 ? 1.0 : h->A, h->rho0);
    a.c.incomp = h->incomp;
    a.scheme = h->scheme;
    a.st = make_stencil<R>(h->beta);
    a.stc = make_stencil<R>(0.0);
    a.rows = h->rows;
    a.err = reinterpret_cast<int *>(h->ws + h->lay.err);
    if (h->path == FDLBM_PATH_STAGED || h->adjoint) {
        a.P = reinterpret_cast<R *>(h->ws + h->lay.P);
        a.Q = reinterpret_cast<R *>(h->ws + h->lay.Q);
        a.S = reinterpret_cast<R *>(h->ws + h->lay.S);
    }
    return a;
}

// One step of whichever kernel the handle uses, reading state[cur], on stream s.
cudaError_t launch_step(fdlbm_ctx *h, cudaStream_t s)
{
    const bool walls = h->bc_x == FDLBM_WALL || h->bc_y == FDLBM_WALL;
    if (h->precision == FDLBM_FP32_DEV) {
        auto a = step_args<float>(h);
        if (h->path == FDLBM_PATH_STAGED) return launch_staged(a, s);
        if (h->variant == FDLBM_VARIANT_WARP) return launch_fused_warp(a, h->wmaps, h->cur, s);
        if (h->scheme == FDLBM_SCHEME_T2S2_2) return launch_fused_s2(a, s);
        if (walls) return launch_fused_walls(a, s);
        return launch_fused(a, s);
    }
    auto a = step_args<double>(h);
    if (h->path == FDLBM_PATH_STAGED) return launch_staged(a, s);
    if (h->scheme == FDLBM_SCHEME_T2S2_2) return launch_fused_s2(a, s);
    if (walls) return launch_fused_walls(a, s);
    return launch_fused(a, s);
}

fdlbm_status step_direct(fdlbm_ctx *h, int n)
{
    for (int k = 0; k < n; ++k) {
        cudaError_t e = launch_step(h, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step");
        h->cur = 1 - h->cur;
        ++h->steps;
    }
    return FDLBM_OK;
}

void drop_step_graph(fdlbm_ctx *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
}

// Record graph_steps steps starting from state[0] on a private stream (capture
// is not allowed on the legacy default stream); the graph is then replayed on
// the handle's stream.  Every kernel argument is fixed for the handle's life
// (buffers live in the workspace), so one capture serves every replay.
fdlbm_status capture_step_graph(fdlbm_ctx *h)
{
    drop_step_graph(h);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "step graph stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    cudaError_t el = cudaSuccess;
    const int cur0 = h->cur;
    if (e == cudaSuccess) {
        for (int k = 0; k < h->graph_steps && el == cudaSuccess; ++k) {
            h->cur = k & 1;
            el = launch_step(h, cs);
        }
        h->cur = cur0;
        e = cudaStreamEndCapture(cs, &h->graph);
    }
    if (e == cudaSuccess && el == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, h->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || el != cudaSuccess) {
        drop_step_graph(h);
        return cuda_fail(h, e != cudaSuccess ? e : el, "step graph capture");
    }
    return FDLBM_OK;
}

// The address under which the device reads and writes a host array directly:
// pinned host memory is mapped into the device's address space (unified
// addressing), so kernels can use it in place of a staged copy.  nullptr for
// pageable memory (or on any query error, which is cleared).
template <class T>
T *device_view(const T *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return static_cast<T *>(at.devicePointer);
}

// Device views of all non-null host arrays, or false if any has none.
template <class T>
bool device_views(const T *const *p, int n, T **out)
{
    for (int k = 0; k < n; ++k) {
        out[k] = nullptr;
        if (p[k] && !(out[k] = device_view(p[k]))) return false;
    }
    return true;
}

// Hand `nfields` host or device fields ([ny][nx] of T each) to
// `kernel(ptr, row0, nrows, fstride)`: device fields and pinned host fields in
// place (one pass; the call still waits for it, so host arrays are free on
// return), pageable host fields through the staging area in row chunks.
template <class T, class K>
fdlbm_status staged_in(fdlbm_ctx *h, const T *const *fields, int nfields, int where, K kernel,
                       const char *what)
{
    const size_t row_bytes = (size_t)h->nx * sizeof(T);
    if (where == FDLBM_MEM_DEVICE) {
        // device fields: consecutive pointers are expected for multi-field args
        cudaError_t e = kernel(fields, h->ny, (size_t)h->nx * h->ny, 0);
        return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, what);
    }
    {
        std::vector<T *> views(nfields);
        if (device_views(fields, nfields, views.data())) {
            std::vector<const T *> cv(views.begin(), views.end());
            cudaError_t e = kernel(cv.data(), h->ny, (size_t)h->nx * h->ny, 0);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, what);
        }
    }
    T *stage = reinterpret_cast<T *>(h->ws + h->lay.staging);
    const size_t stage_elems = h->lay.staging_elems * (sizeof(double) / sizeof(T));
    const int rows = (int)std::max<size_t>(1, stage_elems / ((size_t)nfields * h->nx));
    for (int r0 = 0; r0 < h->ny; r0 += rows) {
        const int nr = std::min(rows, h->ny - r0);
        const size_t fstride = (size_t)nr * h->nx;
        std::vector<const T *> ptrs(nfields);
        for (int k = 0; k < nfields; ++k) {
            if (!fields[k]) {
                ptrs[k] = nullptr;
                continue;
            }
            cudaError_t e = cudaMemcpyAsync(stage + k * fstride, fields[k] + (size_t)r0 * h->nx,
                                            nr * row_bytes, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, what);
            ptrs[k] = stage + k * fstride;
        }
        cudaError_t e = kernel(ptrs.data(), nr, fstride, r0);
        if (e != cudaSuccess) return cuda_fail(h, e, what);
        // the staging area is reused by the next chunk
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, what);
    }
    return FDLBM_OK;
}

// Initialisation from fields of type T (see fdlbm_init_fields / _f32).
template <class T>
fdlbm_status init_fields_t(fdlbm_t h, const T *rho, const T *ux, const T *uy, const T *grad,
                           int where)
{
    if (!h) return FDLBM_EINVAL;
    if (!rho || !ux || !uy || (where != FDLBM_MEM_HOST && where != FDLBM_MEM_DEVICE))
        return fail(h, FDLBM_EINVAL, "init_fields: NULL field or bad `where`");
    const size_t N = (size_t)h->nx * h->ny;
    const T *f[7] = {rho, ux, uy, grad, grad ? grad + N : nullptr, grad ? grad + 2 * N : nullptr,
                     grad ? grad + 3 * N : nullptr};
    h->have_uprev = false;
    return staged_in<T>(
        h, f, grad ? 7 : 3, where,
        [&](const T *const *p, int nr, size_t fstride, int r0) {
            return launch_init_fields<T>(h, p[0], p[1], p[2], grad ? p[3] : nullptr, r0, nr, fstride);
        },
        "init_fields");
}

// Moments into fields of type T (see fdlbm_moments / _f32).
template <class T>
fdlbm_status moments_t(fdlbm_t h, T *rho, T *ux, T *uy, int where)
{
    if (!h) return FDLBM_EINVAL;
    if (!rho || !ux || !uy || (where != FDLBM_MEM_HOST && where != FDLBM_MEM_DEVICE))
        return fail(h, FDLBM_EINVAL, "moments: NULL or bad `where`");
    const size_t N = (size_t)h->nx * h->ny;
    cudaError_t e;
    if (where == FDLBM_MEM_DEVICE) {
        e = launch_moments<T>(h, rho, ux, uy, 0, h->ny, N);
        return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "moments");
    }
    {
        const T *outs[3] = {rho, ux, uy};
        T *v[3];
        if (device_views(outs, 3, v)) {  // pinned host memory: written in place
            e = launch_moments<T>(h, v[0], v[1], v[2], 0, h->ny, N);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "moments");
        }
    }
    T *stage = reinterpret_cast<T *>(h->ws + h->lay.staging);
    const size_t stage_elems = h->lay.staging_elems * (sizeof(double) / sizeof(T));
    const int rows = (int)std::max<size_t>(1, stage_elems / (3 * (size_t)h->nx));
    for (int r0 = 0; r0 < h->ny; r0 += rows) {
        const int nr = std::min(rows, h->ny - r0);
        const size_t fs = (size_t)nr * h->nx;
        e = launch_moments<T>(h, stage, stage + fs, stage + 2 * fs, r0, nr, fs);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments");
        T *dst[3] = {rho, ux, uy};
        for (int k = 0; k < 3; ++k) {
            e = cudaMemcpyAsync(dst[k] + (size_t)r0 * h->nx, stage + k * fs, fs * sizeof(T),
                                cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "moments");
        }
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments");
    }
    return FDLBM_OK;
}

// Kernel-side failure flag (a bounded wait that gave up).  Synchronises.
fdlbm_status check_flag(fdlbm_ctx *h)
{
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, h->ws + h->lay.err, sizeof(int), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "error flag");
    if (flag) return fail(h, FDLBM_ECUDA, "a step kernel timed out waiting for its row copies");
    return FDLBM_OK;
}

}  // namespace

namespace fdlbm {

size_t real_size(int precision) { return precision == FDLBM_FP32_DEV ? 4 : 8; }

Layout make_layout(int nx, int ny, int pitch, int precision, int has_force, bool staged)
{
    Layout L{};
    const size_t rs = real_size(precision);
    const size_t plane = (size_t)pitch * ny;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    L.state[0] = take(9 * plane * rs);
    L.state[1] = take(9 * plane * rs);
    L.mx = take(nx * rs);
    L.my = take(ny * rs);
    L.mxd = take(nx * sizeof(double));
    L.myd = take(ny * sizeof(double));
    L.force = has_force ? take(2 * plane * rs) : 0;
    if (staged) {
        L.P = take(9 * plane * rs);
        L.Q = take(9 * plane * rs);
        L.S = take(9 * plane * rs);
    }
    L.uprev = take(2 * (size_t)nx * ny * sizeof(double));
    L.nblocks_red = kRedBlocks;
    L.partials = take((size_t)kRedBlocks * 3 * sizeof(double));
    L.red = take(4 * sizeof(double));
    L.err = take(sizeof(int) * 4);
    const size_t need_rows = (size_t)9 * nx * sizeof(double);  // one row of 9 fields
    const size_t sbytes = std::max(std::min(kStagingBytes, 9 * (size_t)nx * ny * sizeof(double)),
                                   need_rows);
    L.staging = take(sbytes);
    L.staging_elems = sbytes / sizeof(double);
    L.total = off;
    return L;
}

// Validate the arguments and fill a new handle (no device work).  With
// force_staged the staged kernels are used whatever the grid (batched cases).
fdlbm_status handle_prepare(const fdlbm_grid *g, const fdlbm_metrics *metrics, double nu,
                            double cfl, double blend, const fdlbm_opts &o, bool force_staged,
                            fdlbm_ctx **out, std::vector<double> &mx, std::vector<double> &my)
{
    if (!grid_ok(g) || !(nu > 0) || !(cfl > 0) || !(blend >= 0 && blend <= 1) ||
        !(o.A >= 0 && o.A <= 1) || !(o.rho0 > 0) ||
        (o.precision != FDLBM_FP64 && o.precision != FDLBM_FP32_DEV) || o.rows_per_cta < 0 || o.graph_steps < 0 ||
        (o.variant != FDLBM_VARIANT_AUTO && o.variant != FDLBM_VARIANT_SCALAR &&
         o.variant != FDLBM_VARIANT_WARP) ||
        (o.scheme != FDLBM_SCHEME_T2S2_1 && o.scheme != FDLBM_SCHEME_T2S2_2) ||
        (o.equilibrium != FDLBM_EQ_STANDARD && o.equilibrium != FDLBM_EQ_INCOMPRESSIBLE))
        return FDLBM_EINVAL;
    // the adjoint is written for the standard equilibrium only
    if (o.equilibrium == FDLBM_EQ_INCOMPRESSIBLE && o.adjoint) return FDLBM_EUNSUPPORTED;
    const int path = force_staged ? FDLBM_PATH_STAGED : choose_path(g, &o);
    if (path < 0) return FDLBM_EUNSUPPORTED;
    const bool fused = path == FDLBM_PATH_FUSED;
    const bool f32 = o.precision == FDLBM_FP32_DEV;
    // the warp-tile kernel runs both schemes, on periodic and walled grids (a
    // single grid: batches keep their T2S2-FDLBM2 cases on the scalar sweep)
    const bool s1 = o.scheme == FDLBM_SCHEME_T2S2_1;
    const bool s2_warp = o.scheme == FDLBM_SCHEME_T2S2_2 && !force_staged;
    // (a batch case, force_staged: the batch's mode picks the kernels; the
    // variant is the one its FUSED mode runs the case on)
    const bool warp_ok = (s1 || s2_warp) && (fused || force_staged) && f32 &&
                         fused_warp_ok(g->nx, g->ny, g->bc_x == FDLBM_WALL);
    if (o.variant == FDLBM_VARIANT_WARP && !warp_ok) return FDLBM_EUNSUPPORTED;
    int variant = o.variant;
    // a walled grid on the warp-tile kernel pays a fixed 25-35 us for its frame
    // launch (rows of the walls sweep are a chain of dependent work): below
    // about 1.5 M nodes the walls sweep alone is faster (measured on GB300:
    // 1025^2 channel 40 us against 43, 2049^2 cavity 164 us against 107)
    const bool small_walled = walled(g) && (long long)g->nx * g->ny < (3ll << 19);
    if (variant == FDLBM_VARIANT_AUTO)
        variant = warp_ok && !small_walled ? FDLBM_VARIANT_WARP : FDLBM_VARIANT_SCALAR;
    mx.assign(g->nx, 0.0);
    my.assign(g->ny, 0.0);
    for (int i = 0; i < g->nx; ++i)
        mx[i] = (metrics && metrics->dzeta_dx) ? metrics->dzeta_dx[i] : 1.0 / (g->x[1] - g->x[0]);
    for (int j = 0; j < g->ny; ++j)
        my[j] = (metrics && metrics->dmu_dy) ? metrics->dmu_dy[j] : 1.0 / (g->y[1] - g->y[0]);
    for (double v : mx)
        if (!(v > 0) || !std::isfinite(v)) return FDLBM_EINVAL;
    for (double v : my)
        if (!(v > 0) || !std::isfinite(v)) return FDLBM_EINVAL;

    fdlbm_ctx *h = new (std::nothrow) fdlbm_ctx();
    if (!h) return FDLBM_ENOMEM;
    h->nx = g->nx;
    h->ny = g->ny;
    h->pitch = pitch_of(g->nx);
    h->plane = (size_t)h->pitch * h->ny;
    h->bc_x = g->bc_x;
    h->bc_y = g->bc_y;
    std::memcpy(h->wall_u, g->wall_u, sizeof(h->wall_u));
    h->precision = o.precision;
    h->scheme = o.scheme;
    h->incomp = o.equilibrium == FDLBM_EQ_INCOMPRESSIBLE ? 1 : 0;
    h->nu = nu;
    h->tau = nu * 3.0;  // tau = nu / cs^2
    h->cfl = cfl;
    h->dt = fdlbm_time_step(g, cfl);
    h->beta = blend;
    h->A = o.A;
    h->rho0 = o.rho0;
    h->has_force = o.has_force ? 1 : 0;
    h->path = path;
    h->rows = 1;
    h->variant = variant;
    if (path == FDLBM_PATH_FUSED)
        h->rows = o.rows_per_cta > 0 ? std::min(o.rows_per_cta, g->ny)
                                     : choose_rows(g->nx, g->ny, o.precision, variant, walled(g),
                                                   o.scheme);
    h->stream = static_cast<cudaStream_t>(o.stream);
    h->adjoint = o.adjoint != 0;
    h->graph_steps = o.graph_steps > 0 ? o.graph_steps + (o.graph_steps & 1) : 0;
    h->lay = make_layout(h->nx, h->ny, h->pitch, h->precision, h->has_force,
                         path == FDLBM_PATH_STAGED || h->adjoint);
    cudaGetDevice(&h->device);
    *out = h;
    return FDLBM_OK;
}

// Zero the state (fluid at rest) and the force, clear the error flag, upload
// the metrics in both precisions.  h->ws must be attached.  Synchronises.
fdlbm_status handle_upload(fdlbm_ctx *h, const std::vector<double> &mx, const std::vector<double> &my)
{
    cudaError_t e = cudaMemsetAsync(h->ws + h->lay.state[0], 0,
                                    h->lay.state[1] - h->lay.state[0], h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->ws + h->lay.state[1], 0, h->lay.state[1] - h->lay.state[0], h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->lay.err, 0, sizeof(int) * 4, h->stream);
    if (e == cudaSuccess && h->has_force)
        e = cudaMemsetAsync(h->ws + h->lay.force, 0, 2 * h->plane * real_size(h->precision),
                            h->stream);
    if (e == cudaSuccess) {
        if (h->precision == FDLBM_FP32_DEV) {
            std::vector<float> fx(mx.begin(), mx.end()), fy(my.begin(), my.end());
            e = cudaMemcpy(h->ws + h->lay.mx, fx.data(), fx.size() * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(h->ws + h->lay.my, fy.data(), fy.size() * 4, cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(h->ws + h->lay.mx, mx.data(), mx.size() * 8, cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(h->ws + h->lay.my, my.data(), my.size() * 8, cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(h->ws + h->lay.mxd, mx.data(), mx.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->ws + h->lay.myd, my.data(), my.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? FDLBM_OK : FDLBM_ECUDA;
}

template <class R>
StepArgs<R> handle_step_args(fdlbm_ctx *h)
{
    return step_args<R>(h);
}
template StepArgs<float> handle_step_args<float>(fdlbm_ctx *);
template StepArgs<double> handle_step_args<double>(fdlbm_ctx *);

}  // namespace fdlbm

extern "C" {

void fdlbm_default_opts(fdlbm_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->A = 0.5;
    o->rho0 = 1.0;
    o->precision = FDLBM_FP64;
    o->path = FDLBM_PATH_AUTO;
}

double fdlbm_time_step(const fdlbm_grid *g, double cfl)
{
    if (!grid_ok(g) || !(cfl > 0)) return -1.0;
    const double dx = std::min(min_spacing(g->x, g->nx, g->bc_x == FDLBM_PERIODIC, g->lx),
                               min_spacing(g->y, g->ny, g->bc_y == FDLBM_PERIODIC, g->ly));
    return cfl * dx / 1.0;  // xi = 1
}

size_t fdlbm_workspace_bytes(const fdlbm_grid *g, const fdlbm_opts *opts)
{
    fdlbm_opts o;
    fdlbm_default_opts(&o);
    if (opts) o = *opts;
    if (!grid_ok(g)) return 0;
    const int path = choose_path(g, &o);
    if (path < 0) return 0;
    return make_layout(g->nx, g->ny, pitch_of(g->nx), o.precision, o.has_force,
                       path == FDLBM_PATH_STAGED || o.adjoint)
        .total;
}

fdlbm_status fdlbm_create(const fdlbm_grid *g, const fdlbm_metrics *metrics, double nu,
                          double cfl, double blend, const fdlbm_opts *opts, fdlbm_t *out)
{
    if (!out) return FDLBM_EINVAL;
    *out = nullptr;
    fdlbm_opts o;
    fdlbm_default_opts(&o);
    if (opts) o = *opts;
    fdlbm_ctx *h = nullptr;
    std::vector<double> mx, my;
    fdlbm_status st = handle_prepare(g, metrics, nu, cfl, blend, o, false, &h, mx, my);
    if (st != FDLBM_OK) return st;
    if (o.workspace) {
        if (o.workspace_bytes < h->lay.total ||
            (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0) {
            delete h;
            return FDLBM_ENOMEM;
        }
        h->ws = static_cast<char *>(o.workspace);
        h->ws_bytes = o.workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc(&h->ws, h->lay.total);
        if (e != cudaSuccess) {
            delete h;
            return FDLBM_ENOMEM;
        }
        h->owns_ws = true;
        h->ws_bytes = h->lay.total;
    }
    st = handle_upload(h, mx, my);
    if (st == FDLBM_OK && h->variant == FDLBM_VARIANT_WARP) {
        // tensor maps of both ping-pong buffers (and of the force field) for the
        // warp-tile kernel
        if (fused_warp_encode(&h->wmaps, reinterpret_cast<const float *>(h->ws + h->lay.state[0]),
                              reinterpret_cast<const float *>(h->ws + h->lay.state[1]),
                              h->has_force ? reinterpret_cast<const float *>(h->ws + h->lay.force)
                                           : nullptr,
                              h->nx, h->ny, h->pitch, h->plane) != cudaSuccess)
            st = FDLBM_EUNSUPPORTED;
    }
    if (st != FDLBM_OK) {
        fdlbm_destroy(h);
        return st;
    }
    *out = h;
    return FDLBM_OK;
}

void fdlbm_destroy(fdlbm_t h)
{
    if (!h || h->in_batch) return;  // batch cases are released by fdlbm_batch_destroy
    if (h->owns_ws && h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
    }
    drop_step_graph(h);
    delete h;
}

fdlbm_status fdlbm_init_fields(fdlbm_t h, const double *rho, const double *ux, const double *uy,
                               const double *grad, int where)
{
    return init_fields_t<double>(h, rho, ux, uy, grad, where);
}

fdlbm_status fdlbm_init_fields_f32(fdlbm_t h, const float *drho, const float *ux, const float *uy,
                                   const float *grad, int where)
{
    return init_fields_t<float>(h, drho, ux, uy, grad, where);
}

fdlbm_status fdlbm_set_state(fdlbm_t h, const double *f, int where)
{
    if (!h) return FDLBM_EINVAL;
    if (!f || (where != FDLBM_MEM_HOST && where != FDLBM_MEM_DEVICE))
        return fail(h, FDLBM_EINVAL, "set_state: NULL or bad `where`");
    const size_t N = (size_t)h->nx * h->ny;
    const double *p[9];
    for (int i = 0; i < 9; ++i) p[i] = f + i * N;
    h->have_uprev = false;
    return staged_in(
        h, p, 9, where,
        [&](const double *const *q, int nr, size_t fstride, int r0) {
            return launch_convert_in(h, q[0], r0, nr, fstride);
        },
        "set_state");
}

fdlbm_status fdlbm_set_force(fdlbm_t h, const double *force, int where)
{
    if (!h) return FDLBM_EINVAL;
    if (!h->has_force) return fail(h, FDLBM_EUNSUPPORTED, "set_force: created without has_force");
    if (!force || (where != FDLBM_MEM_HOST && where != FDLBM_MEM_DEVICE))
        return fail(h, FDLBM_EINVAL, "set_force: NULL or bad `where`");
    const size_t N = (size_t)h->nx * h->ny;
    const double *p[2] = {force, force + N};
    return staged_in(
        h, p, 2, where,
        [&](const double *const *q, int nr, size_t fstride, int r0) {
            return launch_set_force(h, q[0], r0, nr, fstride);
        },
        "set_force");
}

fdlbm_status fdlbm_get_state(fdlbm_t h, double *f, int where)
{
    if (!h) return FDLBM_EINVAL;
    if (!f || (where != FDLBM_MEM_HOST && where != FDLBM_MEM_DEVICE))
        return fail(h, FDLBM_EINVAL, "get_state: NULL or bad `where`");
    const size_t N = (size_t)h->nx * h->ny;
    cudaError_t e;
    if (where == FDLBM_MEM_DEVICE) {
        e = launch_convert_out(h, f, 0, h->ny, N);
        return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "get_state");
    }
    if (double *v = device_view(f)) {  // pinned host memory: written in place
        e = launch_convert_out(h, v, 0, h->ny, N);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "get_state");
    }
    double *stage = reinterpret_cast<double *>(h->ws + h->lay.staging);
    const int rows = (int)std::max<size_t>(1, h->lay.staging_elems / (9 * (size_t)h->nx));
    for (int r0 = 0; r0 < h->ny; r0 += rows) {
        const int nr = std::min(rows, h->ny - r0);
        const size_t fstride = (size_t)nr * h->nx;
        e = launch_convert_out(h, stage, r0, nr, fstride);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
        for (int i = 0; i < 9; ++i) {
            e = cudaMemcpyAsync(f + i * N + (size_t)r0 * h->nx, stage + i * fstride,
                                fstride * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
        }
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
    }
    return FDLBM_OK;
}

fdlbm_status fdlbm_step(fdlbm_t h, int n)
{
    if (!h) return FDLBM_EINVAL;
    if (n < 0) return fail(h, FDLBM_EINVAL, "step: n < 0");
    if (h->in_batch)
        return fail(h, FDLBM_EUNSUPPORTED, "step: a batch case advances with fdlbm_batch_step");
    const int G = h->graph_steps;
    if (G > 0 && n >= G + h->cur) {
        if (h->cur) {  // the graph starts from state[0]
            fdlbm_status st = step_direct(h, 1);
            if (st != FDLBM_OK) return st;
            --n;
        }
        if (!h->gexec) {
            fdlbm_status st = capture_step_graph(h);
            if (st != FDLBM_OK) return st;
        }
        for (; n >= G; n -= G) {
            cudaError_t e = cudaGraphLaunch(h->gexec, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "step (graph launch)");
            h->steps += G;
        }
    }
    return step_direct(h, n);
}

fdlbm_status fdlbm_moments(fdlbm_t h, double *rho, double *ux, double *uy, int where)
{
    return moments_t<double>(h, rho, ux, uy, where);
}

fdlbm_status fdlbm_moments_f32(fdlbm_t h, float *drho, float *ux, float *uy, int where)
{
    return moments_t<float>(h, drho, ux, uy, where);
}

fdlbm_status fdlbm_reduce(fdlbm_t h, double *mass, double *resid)
{
    if (!h) return FDLBM_EINVAL;
    cudaError_t e = launch_reduce(h, h->have_uprev ? 1 : 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce");
    double r[4];
    e = cudaMemcpyAsync(r, h->ws + h->lay.red, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce");
    fdlbm_status fs = check_flag(h);
    if (fs != FDLBM_OK) return fs;
    // relative residual; a fluid exactly at rest gets the absolute one
    const double res =
        h->have_uprev ? (r[1] > 0.0 ? std::sqrt(r[2] / r[1]) : std::sqrt(r[2])) : -1.0;
    h->have_uprev = true;
    if (mass) *mass = r[0];
    if (resid) *resid = res;
    if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || !std::isfinite(r[2]))
        return fail(h, FDLBM_ENONFINITE, "reduce: non-finite mass or velocity (diverged)");
    return FDLBM_OK;
}

fdlbm_status fdlbm_set_stream(fdlbm_t h, void *stream)
{
    if (!h) return FDLBM_EINVAL;
    if (h->in_batch) return fail(h, FDLBM_EUNSUPPORTED, "set_stream: batch cases use the batch stream");
    h->stream = static_cast<cudaStream_t>(stream);
    return FDLBM_OK;
}

fdlbm_status fdlbm_sync(fdlbm_t h)
{
    if (!h) return FDLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    return check_flag(h);
}

double fdlbm_dt(fdlbm_t h) { return h ? h->dt : -1.0; }
double fdlbm_tau(fdlbm_t h) { return h ? h->tau : -1.0; }
long long fdlbm_steps_done(fdlbm_t h) { return h ? h->steps : -1; }
int fdlbm_path(fdlbm_t h) { return h ? h->path : -1; }
fdlbm_status fdlbm_tile_plan(const fdlbm_grid *g, int rows, int scheme, int *tiles, int cap, int *count)
{
    if (!grid_ok(g) || rows <= 0 || cap < 0 || !count || (cap > 0 && !tiles) ||
        (scheme != FDLBM_SCHEME_T2S2_1 && scheme != FDLBM_SCHEME_T2S2_2))
        return FDLBM_EINVAL;
    if (!fused_warp_ok(g->nx, g->ny, g->bc_x == FDLBM_WALL)) return FDLBM_EUNSUPPORTED;
    *count = warp_tile_plan(g->nx, g->ny, g->bc_x == FDLBM_WALL, g->bc_y == FDLBM_WALL, rows,
                            scheme == FDLBM_SCHEME_T2S2_2, tiles, cap);
    return FDLBM_OK;
}

int fdlbm_kernels_per_step(fdlbm_t h)
{
    if (!h) return -1;
    const bool walls = h->bc_x == FDLBM_WALL || h->bc_y == FDLBM_WALL;
    if (h->path == FDLBM_PATH_FUSED) {
        // a walled grid on the warp-tile kernel: the frame's launch and the interior's
        if (h->precision == FDLBM_FP32_DEV && h->variant == FDLBM_VARIANT_WARP && walls) {
            int interior = 0, frame = 0;
            fused_warp_tiles(step_args<float>(h), &interior, &frame);
            return (interior > 0) + (frame > 0);
        }
        return 1;
    }
    if (h->scheme == FDLBM_SCHEME_T2S2_2) return walls ? 6 : 3;
    return walls ? 5 : 3;
}

size_t fdlbm_state_bytes(fdlbm_t h)
{
    return h ? 9 * h->plane * real_size(h->precision) : 0;
}

fdlbm_status fdlbm_state_layout(fdlbm_t h, int *pitch, int *elem_bytes)
{
    if (!h || !pitch || !elem_bytes) return FDLBM_EINVAL;
    *pitch = h->pitch;
    *elem_bytes = (int)real_size(h->precision);
    return FDLBM_OK;
}

fdlbm_status fdlbm_copy_state(fdlbm_t h, void *buf, int to_handle)
{
    if (!h || !buf) return FDLBM_EINVAL;
    char *st = h->ws + h->lay.state[h->cur];
    const size_t n = fdlbm_state_bytes(h);
    cudaError_t e = to_handle ? cudaMemcpyAsync(st, buf, n, cudaMemcpyDeviceToDevice, h->stream)
                              : cudaMemcpyAsync(buf, st, n, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy_state");
    if (to_handle) h->have_uprev = false;
    return FDLBM_OK;
}

fdlbm_status fdlbm_adjoint_step(fdlbm_t h, const void *state_n, const void *lam_next,
                                void *lam_prev, double *dforce)
{
    if (!h) return FDLBM_EINVAL;
    if (!state_n || !lam_next || !lam_prev || lam_next == lam_prev)
        return fail(h, FDLBM_EINVAL, "adjoint_step: NULL or aliased buffers");
    if (!h->adjoint || h->bc_x != FDLBM_PERIODIC || h->bc_y != FDLBM_PERIODIC ||
        h->scheme != FDLBM_SCHEME_T2S2_1)
        return fail(h, FDLBM_EUNSUPPORTED,
                    "adjoint_step: needs opts.adjoint, a periodic grid and scheme T2S2_1");
    cudaError_t e;
    double *fB = reinterpret_cast<double *>(h->ws + h->lay.S);
    if (h->precision == FDLBM_FP32_DEV) {
        StepArgs<float> a = step_args<float>(h);
        a.gin = static_cast<const float *>(state_n);
        e = launch_adjoint<float>(a, static_cast<const float *>(lam_next), static_cast<float *>(lam_prev),
                                  a.P, a.Q, fB, dforce, h->stream);
    } else {
        StepArgs<double> a = step_args<double>(h);
        a.gin = static_cast<const double *>(state_n);
        e = launch_adjoint<double>(a, static_cast<const double *>(lam_next),
                                   static_cast<double *>(lam_prev), a.P, a.Q, fB, dforce, h->stream);
    }
    return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "adjoint_step");
}

fdlbm_status fdlbm_moments_vjp(fdlbm_t h, const void *state, const double *du, void *lam,
                               double *dforce)
{
    if (!h) return FDLBM_EINVAL;
    if (!state || !du || !lam) return fail(h, FDLBM_EINVAL, "moments_vjp: NULL buffer");
    cudaError_t e;
    if (h->precision == FDLBM_FP32_DEV) {
        StepArgs<float> a = step_args<float>(h);
        a.gin = static_cast<const float *>(state);
        e = launch_moments_vjp<float>(a, du, static_cast<float *>(lam), dforce, h->stream);
    } else {
        StepArgs<double> a = step_args<double>(h);
        a.gin = static_cast<const double *>(state);
        e = launch_moments_vjp<double>(a, du, static_cast<double *>(lam), dforce, h->stream);
    }
    return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "moments_vjp");
}

fdlbm_status fdlbm_init_vjp(fdlbm_t h, const double *rho, const double *ux, const double *uy,
                            const void *lam, double *drho, double *dux, double *duy,
                            double *dforce)
{
    if (!h) return FDLBM_EINVAL;
    if (!rho || !ux || !uy || !lam || !dux || !duy)
        return fail(h, FDLBM_EINVAL, "init_vjp: NULL buffer");
    cudaError_t e;
    if (h->precision == FDLBM_FP32_DEV)
        e = launch_init_vjp<float>(step_args<float>(h), rho, ux, uy, static_cast<const float *>(lam),
                                   h->dt, drho, dux, duy, dforce, h->stream);
    else
        e = launch_init_vjp<double>(step_args<double>(h), rho, ux, uy,
                                    static_cast<const double *>(lam), h->dt, drho, dux, duy,
                                    dforce, h->stream);
    return e == cudaSuccess ? FDLBM_OK : cuda_fail(h, e, "init_vjp");
}

const char *fdlbm_last_error(fdlbm_t h) { return h ? h->err.c_str() : "NULL handle"; }

const char *fdlbm_describe(fdlbm_t h)
{
    if (!h) return "NULL handle";
    const char *prec = h->precision == FDLBM_FP32_DEV ? "fp32dev" : "fp64";
    if (h->scheme == FDLBM_SCHEME_T2S2_2) {
        h->desc = std::string(h->path == FDLBM_PATH_STAGED         ? "staged-scheme2 "
                              : h->variant == FDLBM_VARIANT_WARP ? "fused-warp-scheme2 "
                                                                 : "fused-scheme2 ") +
                  prec;
        if (h->path == FDLBM_PATH_FUSED) h->desc += " rows=" + std::to_string(h->rows);
        if (h->path == FDLBM_PATH_FUSED && h->variant == FDLBM_VARIANT_WARP &&
            (h->bc_x == FDLBM_WALL || h->bc_y == FDLBM_WALL))
            h->desc += " walls";
        if (h->graph_steps) h->desc += " graph_steps=" + std::to_string(h->graph_steps);
        if (h->incomp) h->desc += " incompressible";
        return h->desc.c_str();
    }
    const bool walls = h->bc_x == FDLBM_WALL || h->bc_y == FDLBM_WALL;
    const char *kern = h->path == FDLBM_PATH_STAGED        ? "staged"
                       : h->variant == FDLBM_VARIANT_WARP   ? "fused-warp"
                       : walls                              ? "fused-walls"
                                                            : "fused";
    h->desc = std::string(kern) + " " + prec + " rows=" + std::to_string(h->rows);
    if (walls && h->path == FDLBM_PATH_FUSED && h->variant == FDLBM_VARIANT_WARP) h->desc += " walls";
    if (h->graph_steps) h->desc += " graph_steps=" + std::to_string(h->graph_steps);
    if (h->incomp) h->desc += " incompressible";
    return h->desc.c_str();
}

const char *fdlbm_status_string(fdlbm_status s)
{
    switch (s) {
    case FDLBM_OK: return "ok";
    case FDLBM_EINVAL: return "invalid argument";
    case FDLBM_ENOMEM: return "out of memory / workspace too small";
    case FDLBM_ECUDA: return "CUDA error";
    case FDLBM_ENONFINITE: return "non-finite result";
    case FDLBM_EUNSUPPORTED: return "unsupported option";
    case FDLBM_ETOOBIG: return "size beyond the fixed capacity";
    }
    return "unknown status";
}

}  // extern "C"
