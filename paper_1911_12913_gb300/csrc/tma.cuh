// 1-D bulk copies (TMA engine, cp.async.bulk) from global to shared memory,
// completed on an mbarrier, with bounded waits.
//
// Every wait here gives up after a bounded number of polls (well over a
// second with the sleeps) and reports failure to the caller; kernels record
// the failure in an error flag and keep their control flow uniform, so no
// __syncthreads() is ever left waiting for a thread that bailed out.
#pragma once

#include <cstdint>

namespace fdlbm {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make initialised barriers visible to the async proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a preceding __syncthreads) before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive on `bar` and announce `bytes` of incoming transactions for this phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity; false after ~2^20 polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t k = 0; k < (1u << 20); ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if (k > 16) __nanosleep(k < 1024 ? 32 : 1024);
    }
    return false;
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global to
// the shared address `dst`; completion counts against the mbarrier at `bar`.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Tiled 3-D tensor copy (cp.async.bulk.tensor) of the box at coordinates
// (c0, c1, c2) of the tensor map `tmap` (a __grid_constant__ kernel parameter)
// into shared memory at `dst` (128-byte aligned); completion counts against
// the mbarrier at `bar`.  c0 times the element size must be a multiple of 16
// bytes; parts of the box outside the tensor are filled with zeros.
__device__ __forceinline__ void tensor_copy_3d(uint32_t dst, const void *tmap, int c0, int c1,
                                               int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Pieces of a periodic row segment: columns xs .. xs+n-1 (may start below 0 or
// run past nx, n <= nx) split where they wrap.  Piece k (0 or 1) goes to
// segment column c, comes from global column g and has `len` columns; returns
// false when piece k does not exist.
__device__ __forceinline__ bool wrap_piece(int xs, int n, int nx, int k, int &c, int &g, int &len)
{
    int g0 = xs % nx;
    if (g0 < 0) g0 += nx;
    const int len0 = min(n, nx - g0);
    if (k == 0) {
        c = 0;
        g = g0;
        len = len0;
        return true;
    }
    c = len0;
    g = 0;
    len = n - len0;
    return len > 0;
}

}  // namespace fdlbm
