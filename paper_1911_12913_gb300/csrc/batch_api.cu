// Batched mode of the C ABI (fdlbm_batch_*, declared in include/fdlbm.h):
// many independent cases in one workspace, advanced together by the batched
// staged kernels (one launch per stage for all cases, step_batched.cu) or, in
// the persistent mode, by one cooperative launch for any number of steps
// (step_persist.cu); a fixed number of steps is captured once into a CUDA
// graph and replayed, and a small autotuner picks the block shape.
//
// Each case is an ordinary handle (fdlbm_t) whose memory lies inside the batch
// workspace, so the per-case calls (init_fields, set_force, get_state,
// moments, reduce) work unchanged on fdlbm_batch_case(b, c); only stepping is
// reserved to the batch, which keeps every case on the same ping-pong parity.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"
#include "staged_nodes.cuh"

using namespace fdlbm;

struct fdlbm_batch_ctx {
    std::vector<fdlbm_ctx *> cases;
    std::vector<size_t> off;
    int precision = FDLBM_FP64;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool owns_ws = false;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    void *d_args = nullptr;    // 2 x ncases argument blocks
    int *d_ints = nullptr;     // blk_start | tiles_x | wall_start | frame_start | grid barrier | blk_case
    size_t d_ints_cap = 0;
    BatchTables tab{};
    void *bar = nullptr;       // grid barrier of the persistent kernel (in d_ints)
    unsigned spin_limit = 1u << 24;  // polls before a persistent block gives up
    int mode = FDLBM_BATCH_STAGED;  // FDLBM_BATCH_FUSED / _STAGED / _PERSISTENT
    int fused_rows = 0;             // tile height of the fused sweep (0: staged tables)
    dim3 blk{32, 8, 1};
    int graph_steps = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long steps = 0;
    bool tuned = false;
    double tuned_ms = -1.0;
    // FUSED mode: the interiors of T2S2-FDLBM1 cases on the warp-tile kernel,
    // in groups of one kernel instance each (tiles [off, off + count) of the
    // tables), the frames of the walled ones (walls sweep in blocks of one
    // warp, a group without and one with a force field), then the walls sweep
    // for the other T2S2-FDLBM1 cases (tiles [walls_off, blocks_s1)), then the
    // T2S2-FDLBM2 cases
    void *d_wargs = nullptr;  // 2 x ncases warp-tile argument blocks (tensor maps, scalars)
    struct WGroup {
        WarpKind kind;
        int off, count;
    };
    std::vector<WGroup> wgroups;
    struct FGroup {
        bool force;
        int off, count;
    };
    std::vector<FGroup> fgroups;
    const int *frame_start = nullptr;  // [ncases] first frame tile of each case (in d_ints)
    int walls_off = 0;
    std::string err, desc;
};

namespace {

constexpr size_t kAlignB = 256;
size_t align_b(size_t v) { return (v + kAlignB - 1) / kAlignB * kAlignB; }

size_t args_size(int precision)
{
    return precision == FDLBM_FP32_DEV ? sizeof(StepArgs<float>) : sizeof(StepArgs<double>);
}

fdlbm_status bfail(fdlbm_batch_ctx *b, fdlbm_status s, const std::string &what)
{
    b->err = what;
    return s;
}

// Host-side tables, uploaded to the device: for the staged kernels, node tiles
// of block shape `blk`; for the fused sweep (fused_rows > 0), tiles of one
// strip of the sweep's width by min(fused_rows, ny) rows (each case's tile
// height goes into its argument block).
fdlbm_status build_tables(fdlbm_batch_ctx *b, dim3 blk, int fused_rows = 0)
{
    const int n = (int)b->cases.size();
    std::vector<int> blk_start(n), tiles_x(n), wall_start(n), frame_start(n, 0), frame_tiles(n, 0), blk_case;
    int total_wall = 0, total_blocks = 0, blocks_s1 = 0;
    bool any2 = false;
    // the tiles of T2S2-FDLBM1 cases first (in FUSED mode those on the
    // warp-tile kernel, grouped by kernel instance, then those on the walls
    // sweep), then those of T2S2-FDLBM2 cases; the fused batch runs each group
    // with its own launch
    const bool warp = fused_rows > 0 && b->mode == FDLBM_BATCH_FUSED;
    auto on_warp = [&](const fdlbm_ctx *h) {
        return warp && h->scheme == FDLBM_SCHEME_T2S2_1 && h->variant == FDLBM_VARIANT_WARP;
    };
    std::vector<WarpKind> kinds(n);
    for (int c = 0; c < n; ++c)
        if (on_warp(b->cases[c])) {
            fdlbm_ctx *h = b->cases[c];
            h->rows = std::min(fused_rows, h->ny);
            kinds[c] = warp_kind(handle_step_args<float>(h));
        }
    std::vector<int> order;
    b->wgroups.clear();
    b->fgroups.clear();
    for (int c = 0; c < n; ++c) {
        if (!on_warp(b->cases[c])) continue;
        if (std::find(order.begin(), order.end(), c) != order.end()) continue;
        for (int d = c; d < n; ++d)
            if (on_warp(b->cases[d]) && kinds[d] == kinds[c]) order.push_back(d);
    }
    const int nwarp_cases = (int)order.size();
    for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < n; ++c)
            if (!on_warp(b->cases[c]) && (b->cases[c]->scheme == FDLBM_SCHEME_T2S2_2) == (pass == 1))
                order.push_back(c);
    int walls_off = -1;
    // after the warp-tile interiors: the frames of the walled ones
    auto emit_frames = [&]() {
        for (int force = 0; force < 2; ++force)
            for (int k = 0; k < nwarp_cases; ++k) {
                const int c = order[k];
                if (frame_tiles[c] == 0 || b->cases[c]->has_force != (force == 1)) continue;
                if (b->fgroups.empty() || b->fgroups.back().force != (force == 1))
                    b->fgroups.push_back({force == 1, total_blocks, 0});
                frame_start[c] = total_blocks;
                b->fgroups.back().count += frame_tiles[c];
                total_blocks += frame_tiles[c];
                blk_case.insert(blk_case.end(), (size_t)frame_tiles[c], c);
            }
        blocks_s1 = total_blocks;
        walls_off = total_blocks;
    };
    for (int k = 0; k < (int)order.size(); ++k) {
        const int c = order[k];
        fdlbm_ctx *h = b->cases[c];
        if (k == nwarp_cases) emit_frames();
        int tx, ty;
        if (k < nwarp_cases) {
            tx = 1;
            fused_warp_tiles(handle_step_args<float>(h), &ty, &frame_tiles[c]);
            if (b->wgroups.empty() || !(b->wgroups.back().kind == kinds[c]))
                b->wgroups.push_back({kinds[c], total_blocks, 0});
            b->wgroups.back().count += tx * ty;
        } else if (fused_rows > 0) {
            h->rows = std::min(fused_rows, h->ny);
            tx = (h->nx + fused_tile_width_walls() - 1) / fused_tile_width_walls();
            ty = (h->ny + h->rows - 1) / h->rows;
        } else {
            h->rows = 1;
            tx = (h->nx + (int)blk.x - 1) / (int)blk.x;
            ty = (h->ny + (int)blk.y - 1) / (int)blk.y;
        }
        blk_start[c] = total_blocks;
        tiles_x[c] = tx;
        total_blocks += tx * ty;
        if (h->scheme != FDLBM_SCHEME_T2S2_2) blocks_s1 = total_blocks;
        blk_case.insert(blk_case.end(), (size_t)tx * ty, c);
        any2 = any2 || h->scheme == FDLBM_SCHEME_T2S2_2;
    }
    if (nwarp_cases > 0 && nwarp_cases == (int)order.size()) emit_frames();
    // wall nodes in case order (the wall kernels find a node's case by a binary
    // search over these prefix sums, whatever the order of the tiles)
    for (int c = 0; c < n; ++c) {
        const fdlbm_ctx *h = b->cases[c];
        wall_start[c] = total_wall;
        const bool wy = h->bc_y == FDLBM_WALL, wx = h->bc_x == FDLBM_WALL;
        total_wall += (wy ? 2 * h->nx : 0) + (wx ? 2 * (wy ? h->ny - 2 : h->ny) : 0);
    }
    const size_t nbar = (persistent_barrier_bytes() + sizeof(int) - 1) / sizeof(int);
    const size_t nints = 4 * (size_t)n + nbar + blk_case.size();
    if (nints > b->d_ints_cap) {
        if (b->d_ints) cudaFree(b->d_ints);
        b->d_ints = nullptr;
        if (cudaMalloc(&b->d_ints, nints * sizeof(int)) != cudaSuccess)
            return bfail(b, FDLBM_ENOMEM, "batch: table allocation failed");
        b->d_ints_cap = nints;
    }
    std::vector<int> all;
    all.reserve(nints);
    all.insert(all.end(), blk_start.begin(), blk_start.end());
    all.insert(all.end(), tiles_x.begin(), tiles_x.end());
    all.insert(all.end(), wall_start.begin(), wall_start.end());
    all.insert(all.end(), frame_start.begin(), frame_start.end());
    all.resize(4 * (size_t)n + nbar, 0);
    all.insert(all.end(), blk_case.begin(), blk_case.end());
    if (cudaMemcpy(b->d_ints, all.data(), nints * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, FDLBM_ECUDA, "batch: table upload failed");
    // argument blocks for both parities (every case at cur = 0 for even steps)
    const size_t as = args_size(b->precision);
    std::vector<unsigned char> host(2 * n * as);
    for (int p = 0; p < 2; ++p)
        for (int c = 0; c < n; ++c) {
            fdlbm_ctx *h = b->cases[c];
            const int saved = h->cur;
            h->cur = p;
            if (b->precision == FDLBM_FP32_DEV) {
                StepArgs<float> a = handle_step_args<float>(h);
                std::memcpy(&host[(p * n + c) * as], &a, as);
            } else {
                StepArgs<double> a = handle_step_args<double>(h);
                std::memcpy(&host[(p * n + c) * as], &a, as);
            }
            h->cur = saved;
        }
    if (cudaMemcpy(b->d_args, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, FDLBM_ECUDA, "batch: argument upload failed");
    // the warp-tile argument blocks (tensor maps of each parity's input state)
    if (nwarp_cases > 0) {
        const size_t ws = fused_warp_args_bytes();
        std::vector<unsigned char> wh(2 * n * ws, 0);
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < nwarp_cases; ++k) {
                const int c = order[k];
                fdlbm_ctx *h = b->cases[c];
                const int saved = h->cur;
                h->cur = p;
                const cudaError_t e = fused_warp_args(&wh[(p * n + c) * ws], handle_step_args<float>(h),
                                                      h->wmaps, p);
                h->cur = saved;
                if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, "batch: warp-tile arguments");
            }
        if (cudaMemcpy(b->d_wargs, wh.data(), wh.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, FDLBM_ECUDA, "batch: argument upload failed");
    }
    b->tab.args[0] = b->d_args;
    b->tab.args[1] = static_cast<char *>(b->d_args) + n * as;
    b->tab.blk_start = b->d_ints;
    b->tab.tiles_x = b->d_ints + n;
    b->tab.wall_start = b->d_ints + 2 * n;
    b->frame_start = b->d_ints + 3 * n;
    b->bar = b->d_ints + 4 * n;
    b->tab.blk_case = b->d_ints + 4 * n + nbar;
    b->tab.ncases = n;
    b->tab.total_blocks = total_blocks;
    b->tab.total_wall = total_wall;
    b->tab.any_scheme2 = any2;
    b->tab.blocks_s1 = blocks_s1;
    b->walls_off = walls_off >= 0 ? std::min(walls_off, blocks_s1) : blocks_s1;
    b->blk = blk;
    b->fused_rows = fused_rows;
    return FDLBM_OK;
}

// FP32: the fused sweeps apply, one kernel for the T2S2-FDLBM1 cases and one
// for the T2S2-FDLBM2 cases (FP64 walled cases are bound by the FP64 units,
// where the staged kernels do better).
bool fused_eligible(const fdlbm_batch_ctx *b) { return b->precision == FDLBM_FP32_DEV; }

// The persistent fused sweep runs T2S2-FDLBM1 cases only.
bool all_scheme1(const fdlbm_batch_ctx *b)
{
    for (const fdlbm_ctx *h : b->cases)
        if (h->scheme != FDLBM_SCHEME_T2S2_1) return false;
    return true;
}

// The fused sweep's tiles for FUSED, and for PERSISTENT where the fused sweep
// applies (one grid barrier per step); node tiles of the staged kernels
// otherwise.
bool uses_fused_sweep(const fdlbm_batch_ctx *b)
{
    return b->mode == FDLBM_BATCH_FUSED ||
           (b->mode == FDLBM_BATCH_PERSISTENT && fused_eligible(b) && all_scheme1(b));
}

// Tile height of the fused batch: minimise (waves) x (rows + 8) over the tiles
// of all cases, as for a single grid, with the waves of the warp-tile launches
// and of the walls sweep counted separately (they run one after the other).
int fused_rows_model(const fdlbm_batch_ctx *b)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)std::max(1, fused_walls_blocks_per_sm<float>()) * sms;
    const long long wslots = (long long)std::max(1, fused_warp_blocks_per_sm()) * sms;
    const int W = fused_tile_width_walls(), WW = fused_warp_tile_width();
    const bool warp = b->mode == FDLBM_BATCH_FUSED;
    int best = 64;
    double best_cost = 1e300;
    for (int rows = 1; rows <= 512; ++rows) {
        long long ctas = 0, wtiles = 0;
        for (const fdlbm_ctx *h : b->cases) {
            const int r = std::min(rows, h->ny), ty = (h->ny + r - 1) / r;
            if (warp && h->scheme == FDLBM_SCHEME_T2S2_1 && h->variant == FDLBM_VARIANT_WARP)
                wtiles += (long long)((h->nx + WW - 1) / WW) * ty;
            else
                ctas += (long long)((h->nx + W - 1) / W) * ty;
        }
        const double cost = (double)((ctas + slots - 1) / slots + (wtiles + wslots - 1) / wslots) * (rows + 8);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = rows;
        }
    }
    return best;
}

// n steps starting at ping-pong parity `parity`: one persistent launch, or one
// launch per stage and step.
cudaError_t launch_steps(fdlbm_batch_ctx *b, int parity, int n)
{
    const bool f32 = b->precision == FDLBM_FP32_DEV;
    if (b->mode == FDLBM_BATCH_FUSED) {
        const int n1 = b->tab.blocks_s1, n2 = b->tab.total_blocks - n1;
        const int nw = n1 - b->walls_off;
        const size_t wsz = fused_warp_args_bytes() * b->cases.size();
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < n && e == cudaSuccess; ++k) {
            const int p = (parity + k) & 1;
            for (const auto &g : b->fgroups) {
                if (e != cudaSuccess) break;
                e = launch_batched_frame(static_cast<const char *>(b->d_wargs) + p * wsz, b->tab.args[p],
                                         b->tab.blk_case, b->frame_start, g.off, g.count, g.force,
                                         b->stream);
            }
            for (const auto &g : b->wgroups) {
                if (e != cudaSuccess) break;
                e = launch_batched_warp(static_cast<const char *>(b->d_wargs) + p * wsz, b->tab.blk_case,
                                        b->tab.blk_start, g.off, g.count, g.kind, b->stream);
            }
            if (e == cudaSuccess && nw > 0)
                e = f32 ? launch_batched_fused<float>(b->tab, p, b->walls_off, nw, b->stream)
                        : launch_batched_fused<double>(b->tab, p, b->walls_off, nw, b->stream);
            if (e == cudaSuccess && n2 > 0)
                e = f32 ? launch_batched_fused_s2<float>(b->tab, p, n1, n2, b->stream)
                        : launch_batched_fused_s2<double>(b->tab, p, n1, n2, b->stream);
        }
        return e;
    }
    if (b->mode == FDLBM_BATCH_PERSISTENT && b->fused_rows > 0)  // the fused sweep, persistent
        return f32 ? launch_persistent_fused<float>(b->tab, b->bar, parity, n, b->stream,
                                                    b->spin_limit)
                   : launch_persistent_fused<double>(b->tab, b->bar, parity, n, b->stream,
                                                     b->spin_limit);
    if (b->mode == FDLBM_BATCH_PERSISTENT)
        return f32 ? launch_persistent<float>(b->tab, b->bar, parity, n, b->blk, b->stream,
                                              b->spin_limit)
                   : launch_persistent<double>(b->tab, b->bar, parity, n, b->blk, b->stream,
                                               b->spin_limit);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; ++k)
        e = f32 ? launch_batched<float>(b->tab, (parity + k) & 1, b->blk, b->stream)
                : launch_batched<double>(b->tab, (parity + k) & 1, b->blk, b->stream);
    return e;
}

void advance_bookkeeping(fdlbm_batch_ctx *b, long long n)
{
    b->steps += n;
    for (fdlbm_ctx *h : b->cases) {
        if (n & 1) h->cur = 1 - h->cur;
        h->steps += n;
    }
}

fdlbm_status step_direct(fdlbm_batch_ctx *b, int n)
{
    if (n <= 0) return FDLBM_OK;
    cudaError_t e = launch_steps(b, (int)(b->steps & 1), n);
    if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, std::string("batch step: ") + cudaGetErrorString(e));
    advance_bookkeeping(b, n);
    return FDLBM_OK;
}

void drop_graph(fdlbm_batch_ctx *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Capture graph_steps batch steps starting from an even step.
fdlbm_status capture(fdlbm_batch_ctx *b)
{
    drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    const cudaError_t el = launch_steps(b, 0, b->graph_steps);
    e = cudaStreamEndCapture(b->stream, &b->graph);
    if (el != cudaSuccess || e != cudaSuccess) {
        drop_graph(b);
        return bfail(b, FDLBM_ECUDA, "capture failed");
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        drop_graph(b);
        return bfail(b, FDLBM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return FDLBM_OK;
}

std::string signature(const fdlbm_batch_ctx *b)
{
    std::ostringstream os;
    os << b->precision << '/' << b->mode;
    for (const fdlbm_ctx *h : b->cases)
        os << ';' << h->nx << 'x' << h->ny << ':' << h->bc_x << h->bc_y << h->has_force << h->scheme;
    return os.str();
}

std::mutex g_tune_mu;
struct TuneChoice {
    dim3 blk;  // staged: node tile shape
    int rows;  // fused: tile height (0 for staged)
};
std::map<std::string, std::pair<TuneChoice, double>> g_tune_cache;

// Reset every case to fluid at rest (after tuning runs on the state).
fdlbm_status reset_states(fdlbm_batch_ctx *b)
{
    for (fdlbm_ctx *h : b->cases) {
        const size_t sz = h->lay.state[1] - h->lay.state[0];
        cudaError_t e = cudaMemsetAsync(h->ws + h->lay.state[0], 0, 2 * sz, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->lay.err, 0, 4 * sizeof(int), b->stream);
        if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, "reset");
        h->cur = 0;
        h->steps = 0;
        h->have_uprev = false;
    }
    b->steps = 0;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? FDLBM_OK
                                                           : bfail(b, FDLBM_ECUDA, "reset sync");
}

// Time each candidate block shape on the batch as created and keep the fastest.
fdlbm_status autotune(fdlbm_batch_ctx *b)
{
    const std::string key = signature(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->tuned = true;
            b->tuned_ms = it->second.second;
            return build_tables(b, it->second.first.blk, it->second.first.rows);
        }
    }
    std::vector<TuneChoice> cand;
    if (uses_fused_sweep(b)) {
        const int r0 = fused_rows_model(b);
        for (int r : {r0, std::max(1, r0 / 2), std::max(1, 3 * r0 / 4), std::min(512, 2 * r0)})
            if (std::none_of(cand.begin(), cand.end(), [&](const TuneChoice &c) { return c.rows == r; }))
                cand.push_back({dim3(128, 1), r});
    } else {
        for (const dim3 &d : {dim3(32, 8), dim3(64, 4), dim3(128, 2), dim3(32, 4), dim3(16, 16), dim3(256, 1)})
            cand.push_back({d, 0});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    TuneChoice best = cand[0];
    float best_ms = 1e30f;
    for (const TuneChoice &c : cand) {
        fdlbm_status st = build_tables(b, c.blk, c.rows);
        if (st == FDLBM_OK) st = step_direct(b, 2);
        if (st != FDLBM_OK) break;
        cudaEventRecord(e0, b->stream);
        st = step_direct(b, 6);
        cudaEventRecord(e1, b->stream);
        if (st != FDLBM_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned = true;
    b->tuned_ms = best_ms / 6.0;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = {best, b->tuned_ms};
    }
    fdlbm_status st = build_tables(b, best.blk, best.rows);
    if (st != FDLBM_OK) return st;
    return reset_states(b);
}

// Tables of the current mode with its default parameters.
fdlbm_status default_tables(fdlbm_batch_ctx *b)
{
    return uses_fused_sweep(b) ? build_tables(b, dim3(128, 1), fused_rows_model(b))
                               : build_tables(b, dim3(32, 8));
}

void release(fdlbm_batch_ctx *b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (fdlbm_ctx *h : b->cases) delete h;
    if (b->d_args) cudaFree(b->d_args);
    if (b->d_wargs) cudaFree(b->d_wargs);
    if (b->d_ints) cudaFree(b->d_ints);
    if (b->owns_ws && b->ws) cudaFree(b->ws);
    if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

size_t fdlbm_batch_workspace_bytes(int ncases, const fdlbm_grid *grids, const fdlbm_opts *opts)
{
    if (ncases <= 0 || !grids) return 0;
    size_t total = 0;
    for (int c = 0; c < ncases; ++c) {
        fdlbm_opts o;
        fdlbm_default_opts(&o);
        if (opts) o = opts[c];
        o.path = FDLBM_PATH_STAGED;
        const size_t s = fdlbm_workspace_bytes(&grids[c], &o);
        if (s == 0) return 0;
        total += align_b(s);
    }
    return total;
}

fdlbm_status fdlbm_batch_create(int ncases, const fdlbm_grid *grids, const fdlbm_metrics *metrics,
                                const double *nu, const double *cfl, const double *blend,
                                const fdlbm_opts *opts, int graph_steps, int autotune_blocks,
                                void *workspace, size_t workspace_bytes, fdlbm_batch_t *out)
{
    if (!out || ncases <= 0 || !grids || !nu || !cfl || !blend || graph_steps < 0)
        return FDLBM_EINVAL;
    *out = nullptr;
    fdlbm_batch_ctx *b = new (std::nothrow) fdlbm_batch_ctx();
    if (!b) return FDLBM_ENOMEM;
    std::vector<std::vector<double>> mxs(ncases), mys(ncases);
    size_t total = 0;
    for (int c = 0; c < ncases; ++c) {
        fdlbm_opts o;
        fdlbm_default_opts(&o);
        if (opts) o = opts[c];
        o.workspace = nullptr;
        if (c > 0 && o.precision != b->precision) {
            release(b);
            return FDLBM_EINVAL;  // one precision per batch
        }
        b->precision = o.precision;
        fdlbm_ctx *h = nullptr;
        fdlbm_status st = handle_prepare(&grids[c], metrics ? &metrics[c] : nullptr, nu[c], cfl[c],
                                         blend[c], o, true, &h, mxs[c], mys[c]);
        if (st != FDLBM_OK) {
            release(b);
            return st;
        }
        h->in_batch = true;
        b->cases.push_back(h);
        b->off.push_back(total);
        total += align_b(h->lay.total);
    }
    // stream: the caller's, or a private one (graph capture needs a non-legacy stream)
    fdlbm_opts o0;
    fdlbm_default_opts(&o0);
    if (opts) o0 = opts[0];
    b->stream = static_cast<cudaStream_t>(o0.stream);
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            release(b);
            return FDLBM_ECUDA;
        }
        b->owns_stream = true;
    }
    if (workspace) {
        if (workspace_bytes < total || reinterpret_cast<uintptr_t>(workspace) % kAlignB) {
            release(b);
            return FDLBM_ENOMEM;
        }
        b->ws = static_cast<char *>(workspace);
        b->ws_bytes = workspace_bytes;
    } else {
        if (cudaMalloc(&b->ws, total) != cudaSuccess) {
            release(b);
            return FDLBM_ENOMEM;
        }
        b->owns_ws = true;
        b->ws_bytes = total;
    }
    for (int c = 0; c < ncases; ++c) {
        fdlbm_ctx *h = b->cases[c];
        h->ws = b->ws + b->off[c];
        h->ws_bytes = h->lay.total;
        h->stream = b->stream;
        if (handle_upload(h, mxs[c], mys[c]) != FDLBM_OK) {
            release(b);
            return FDLBM_ECUDA;
        }
    }
    if (cudaMalloc(&b->d_args, 2 * ncases * args_size(b->precision)) != cudaSuccess) {
        release(b);
        return FDLBM_ENOMEM;
    }
    // FP32 T2S2-FDLBM1 cases that the warp-tile kernel takes (FUSED mode): the
    // tensor maps of their state buffers and force field
    if (b->precision == FDLBM_FP32_DEV) {
        for (fdlbm_ctx *h : b->cases) {
            // the case's own choice (its options, or the automatic one of a
            // single grid, which leaves small walled grids to the walls sweep)
            const bool want = h->variant == FDLBM_VARIANT_WARP;
            h->variant = FDLBM_VARIANT_SCALAR;
            if (!want || h->scheme != FDLBM_SCHEME_T2S2_1 ||
                !fused_warp_ok(h->nx, h->ny, h->bc_x == FDLBM_WALL))
                continue;
            if (fused_warp_encode(&h->wmaps, reinterpret_cast<const float *>(h->ws + h->lay.state[0]),
                                  reinterpret_cast<const float *>(h->ws + h->lay.state[1]),
                                  h->has_force ? reinterpret_cast<const float *>(h->ws + h->lay.force)
                                               : nullptr,
                                  h->nx, h->ny, h->pitch, h->plane) == cudaSuccess)
                h->variant = FDLBM_VARIANT_WARP;
        }
        if (cudaMalloc(&b->d_wargs, 2 * ncases * fused_warp_args_bytes()) != cudaSuccess) {
            release(b);
            return FDLBM_ENOMEM;
        }
    }
    b->graph_steps = graph_steps + (graph_steps & 1);  // even: starts and ends on the same parity
    b->mode = fused_eligible(b) ? FDLBM_BATCH_FUSED : FDLBM_BATCH_STAGED;
    fdlbm_status st = autotune_blocks ? autotune(b) : default_tables(b);
    if (st != FDLBM_OK) {
        release(b);
        return st;
    }
    *out = b;
    return FDLBM_OK;
}

fdlbm_t fdlbm_batch_case(fdlbm_batch_t b, int c)
{
    if (!b || c < 0 || c >= (int)b->cases.size()) return nullptr;
    return b->cases[c];
}

int fdlbm_batch_size(fdlbm_batch_t b) { return b ? (int)b->cases.size() : -1; }

long long fdlbm_batch_cells(fdlbm_batch_t b)
{
    if (!b) return -1;
    long long n = 0;
    for (const fdlbm_ctx *h : b->cases) n += (long long)h->nx * h->ny;
    return n;
}

fdlbm_status fdlbm_batch_step(fdlbm_batch_t b, int n)
{
    if (!b) return FDLBM_EINVAL;
    if (n < 0) return bfail(b, FDLBM_EINVAL, "batch step: n < 0");
    if ((b->steps & 1) && n > 0) {  // realign on an even step for the graph
        fdlbm_status st = step_direct(b, 1);
        if (st != FDLBM_OK) return st;
        --n;
    }
    if (b->graph_steps > 0 && n >= b->graph_steps) {
        if (!b->exec) {
            fdlbm_status st = capture(b);
            if (st != FDLBM_OK) return st;
        }
        while (n >= b->graph_steps) {
            cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
            if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            advance_bookkeeping(b, b->graph_steps);
            n -= b->graph_steps;
        }
    }
    return step_direct(b, n);
}

fdlbm_status fdlbm_batch_set_mode(fdlbm_batch_t b, int mode)
{
    if (!b) return FDLBM_EINVAL;
    if (mode != FDLBM_BATCH_FUSED && mode != FDLBM_BATCH_STAGED && mode != FDLBM_BATCH_PERSISTENT)
        return bfail(b, FDLBM_EINVAL, "batch set_mode: unknown mode");
    if (mode == FDLBM_BATCH_FUSED && !fused_eligible(b))
        return bfail(b, FDLBM_EUNSUPPORTED, "batch set_mode: the fused sweeps need FP32");
    fdlbm_status st = fdlbm_batch_sync(b);
    if (st != FDLBM_OK) return st;
    drop_graph(b);
    b->mode = mode;
    b->tuned = false;
    return default_tables(b);
}

int fdlbm_batch_mode(fdlbm_batch_t b) { return b ? b->mode : -1; }

fdlbm_status fdlbm_batch_sync(fdlbm_batch_t b)
{
    if (!b) return FDLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, cudaGetErrorString(e));
    // the kernel-side failure flags of the cases (bounded waits that gave up):
    // reported here once, then cleared
    const int n = (int)b->cases.size();
    std::vector<int> flags(n, 0);
    for (int c = 0; c < n && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(&flags[c], b->cases[c]->ws + b->cases[c]->lay.err, sizeof(int),
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, cudaGetErrorString(e));
    int bad = 0;
    for (int c = 0; c < n; ++c) bad += flags[c] != 0;
    if (!bad) return FDLBM_OK;
    for (int c = 0; c < n && e == cudaSuccess; ++c)
        if (flags[c])
            e = cudaMemsetAsync(b->cases[c]->ws + b->cases[c]->lay.err, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FDLBM_ECUDA, cudaGetErrorString(e));
    return bfail(b, FDLBM_ECUDA,
                 "batch: a kernel gave up waiting (grid barrier or row copy) in " +
                     std::to_string(bad) + " of " + std::to_string(n) +
                     " cases; their states are not valid");
}

fdlbm_status fdlbm_batch_set_spin_limit(fdlbm_batch_t b, unsigned polls)
{
    if (!b) return FDLBM_EINVAL;
    fdlbm_status st = fdlbm_batch_sync(b);
    if (st != FDLBM_OK) return st;
    drop_graph(b);  // a captured graph holds the old limit
    b->spin_limit = polls;
    return FDLBM_OK;
}

void *fdlbm_batch_stream(fdlbm_batch_t b) { return b ? (void *)b->stream : nullptr; }

const char *fdlbm_batch_describe(fdlbm_batch_t b)
{
    if (!b) return "NULL batch";
    std::ostringstream os;
    const char *prec = b->precision == FDLBM_FP32_DEV ? "fp32dev" : "fp64";
    if (b->mode == FDLBM_BATCH_FUSED) {
        const int n1 = b->tab.blocks_s1, n2 = b->tab.total_blocks - n1, nw = n1 - b->walls_off;
        os << "batched-fused " << prec << " cases=" << b->cases.size() << " rows=" << b->fused_rows
           << " graph_steps=" << b->graph_steps << " warp_tiles=" << b->walls_off
           << " launches_per_step=" << (int)(b->wgroups.size() + b->fgroups.size()) + (nw > 0) + (n2 > 0);
    } else if (b->mode == FDLBM_BATCH_PERSISTENT && b->fused_rows > 0) {
        os << "batched-persistent-fused " << prec << " cases=" << b->cases.size()
           << " rows=" << b->fused_rows << " graph_steps=" << b->graph_steps
           << " grid_barriers_per_step=1";
    } else {
        const int per_step =
            3 + (b->tab.total_wall > 0 ? 2 : 0) + (b->tab.total_wall > 0 && b->tab.any_scheme2 ? 1 : 0);
        const bool pers = b->mode == FDLBM_BATCH_PERSISTENT;
        os << (pers ? "batched-persistent " : "batched-staged ") << prec << " cases=" << b->cases.size()
           << " block=" << b->blk.x << "x" << b->blk.y << " graph_steps=" << b->graph_steps
           << (pers ? " grid_barriers_per_step=" : " launches_per_step=") << per_step;
    }
    if (b->tuned) os << " tuned_ms_per_step=" << b->tuned_ms;
    b->desc = os.str();
    return b->desc.c_str();
}

const char *fdlbm_batch_last_error(fdlbm_batch_t b) { return b ? b->err.c_str() : "NULL batch"; }

void fdlbm_batch_destroy(fdlbm_batch_t b)
{
    if (b) release(b);
}

}  // extern "C"
