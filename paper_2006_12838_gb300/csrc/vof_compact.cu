// vof_compact.cu -- interface-cell compaction (Sec. 4.1, Eq. 33): the ordered
// list of interior cells with 0 < phi < 1, and plic_workspace_bytes().
//
// Three launches, no atomics and no inter-block waiting, so the list is in
// ascending cell order and identical run to run:
//   1. k_compact_count : each block counts the interface cells of its tile of
//                        TILE consecutive cells (coalesced row reads).
//   2. k_compact_scan  : one block turns the per-tile counts into exclusive
//                        offsets (in place) and writes the total to *d_count.
//   3. k_compact_write : each block re-reads its tile (it is L2-resident right
//                        after pass 1 for fields up to the 129 MB L2) and writes
//                        the indices at its offset, in order, via warp ballots
//                        and a block scan.
// HBM roofline: 4 B per field cell read once (pass 3 mostly hits L2), plus
// 4 B per interface cell written.
#include <mutex>
#include <stdio.h>

#include "host_common.h"

namespace plic {

constexpr int CT_THREADS = 256;
constexpr int CT_ROUNDS = 16;
constexpr int CT_TILE = CT_THREADS * CT_ROUNDS;   // 4096 cells per tile

__device__ __forceinline__ bool is_curv_cell(const float* __restrict__ phi, int64_t c, int nx,
                                             int ny, int nz, int64_t ncell) {
    if (c >= ncell) return false;
    const float v = __ldg(phi + c);
    if (!(v > 0.0f && v < 1.0f)) return false;
    const int64_t nxy = (int64_t)nx * ny;
    const int z = (int)(c / nxy);
    const int64_t r = c - (int64_t)z * nxy;
    const int y = (int)(r / nx);
    const int x = (int)(r - (int64_t)y * nx);
    return x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2;
}

__global__ void __launch_bounds__(CT_THREADS)
k_compact_count(const float* __restrict__ phi, int nx, int ny, int nz, int64_t ncell,
                int* __restrict__ tile_count) {
    const int64_t base = (int64_t)blockIdx.x * CT_TILE;
    int cnt = 0;
#pragma unroll 4
    for (int r = 0; r < CT_ROUNDS; ++r)
        cnt += is_curv_cell(phi, base + r * CT_THREADS + threadIdx.x, nx, ny, nz, ncell);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    __shared__ int ws[CT_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < CT_THREADS / 32; ++w) t += ws[w];
        tile_count[blockIdx.x] = t;
    }
}

// Exclusive scan of ntiles ints by one block of 1024 threads; total -> *d_count.
__global__ void __launch_bounds__(1024)
k_compact_scan(int* __restrict__ tile_count, int64_t ntiles, int64_t* __restrict__ d_count) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < ntiles; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        long long v = i < ntiles ? tile_count[i] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const long long excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
        if (i < ntiles) tile_count[i] = (int)excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_count = carry;
}

__global__ void __launch_bounds__(CT_THREADS)
k_compact_write(const float* __restrict__ phi, int nx, int ny, int nz, int64_t ncell,
                const int* __restrict__ tile_offset, int32_t* __restrict__ idx, int64_t cap) {
    __shared__ int wcnt[CT_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * CT_TILE;
    int64_t pos = tile_offset[blockIdx.x];
    for (int r = 0; r < CT_ROUNDS; ++r) {
        const int64_t c = base + r * CT_THREADS + threadIdx.x;
        const bool f = is_curv_cell(phi, c, nx, ny, nz, ncell);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < CT_THREADS / 32; ++w) {
            const int cw = wcnt[w];
            before += w < warp ? cw : 0;
            total += cw;
        }
        if (f) {
            const int64_t p = pos + before + __popc(bal & ((1u << lane) - 1u));
            if (p < cap) idx[p] = (int32_t)c;
        }
        pos += total;
        __syncthreads();
    }
}

static int64_t compact_tiles(int64_t ncell) { return (ncell + CT_TILE - 1) / CT_TILE; }

}  // namespace plic

extern "C" size_t plic_workspace_bytes(int op, int64_t arg) {
    if (arg < 0) return 0;
    switch (op) {
        case PLIC_WS_COMPACT: {
            const size_t b = (size_t)plic::compact_tiles(arg) * sizeof(int);
            return (b + 255) / 256 * 256;
        }
        case PLIC_WS_BATCHED: {
            // descriptor table + per-field cell prefix + the ticket counter
            const size_t b = (size_t)arg * (sizeof(vof_field) + sizeof(int64_t)) + 2 * sizeof(int64_t);
            return (b + 255) / 256 * 256 + 256;
        }
        default: return 0;
    }
}

extern "C" plic_status vof_interface_compact(const float* phi, int nx, int ny, int nz,
                                             int32_t* idx, int64_t idx_capacity, int64_t* d_count,
                                             void* workspace, size_t ws_bytes, void* stream) {
    using namespace plic;
    if (nx < 0 || ny < 0 || nz < 0 || idx_capacity < 0) return PLIC_ERR_ARG;
    const int64_t ncell = (int64_t)nx * ny * nz;
    if (ncell > 2147483647LL) return PLIC_ERR_ARG;
    if (!d_count) return PLIC_ERR_ARG;
    if (!aligned(d_count, 8)) return PLIC_ERR_ALIGN;
    cudaStream_t s = as_stream(stream);
    if (ncell == 0) {
        cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) { set_last_error("vof_interface_compact", e); return PLIC_ERR_CUDA; }
        return PLIC_OK;
    }
    if (!phi || (!idx && idx_capacity > 0) || !workspace) return PLIC_ERR_ARG;
    if (ws_bytes < plic_workspace_bytes(PLIC_WS_COMPACT, ncell)) return PLIC_ERR_ARG;
    if (!aligned(phi, 4) || (idx && !aligned(idx, 4)) || !aligned(workspace, 256)) return PLIC_ERR_ALIGN;
    const int64_t nt = compact_tiles(ncell);
    if (nt > 2147483647LL) return PLIC_ERR_ARG;
    int* tiles = reinterpret_cast<int*>(workspace);
    k_compact_count<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, ncell, tiles);
    k_compact_scan<<<1, 1024, 0, s>>>(tiles, nt, d_count);
    k_compact_write<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, ncell, tiles, idx, idx_capacity);
    return check_launch("vof_interface_compact");
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  The per-tile scratch of the three passes lives in
// a file-scope device array instead of a caller-provided workspace.  Every
// GPU that loads the library holds these 256 KiB until the process exits.
// ---------------------------------------------------------------------------
namespace plic {

constexpr int64_t kNoAllocMaxTiles = PLIC_NOALLOC_MAX_CELLS / CT_TILE;
static_assert(kNoAllocMaxTiles * CT_TILE == PLIC_NOALLOC_MAX_CELLS, "limit is whole tiles");

static __device__ __align__(256) int g_noalloc_tiles[kNoAllocMaxTiles];

// Device address of g_noalloc_tiles, looked up once per device (with that
// device current) and cached; host code must not pass the symbol itself.
static int* noalloc_scratch(plic_status* st) {
    static std::mutex mu;
    static int* addr[256] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        set_last_error("vof_interface_compact_noalloc: cudaGetDevice", e);
        *st = PLIC_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
        if (e != cudaSuccess || !p) {
            set_last_error("vof_interface_compact_noalloc: cudaGetSymbolAddress", e);
            *st = PLIC_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = reinterpret_cast<int*>(p);
    }
    return addr[dev];
}

}  // namespace plic

extern "C" plic_status vof_interface_compact_noalloc(const float* phi, int nx, int ny, int nz,
                                                     int32_t* idx, int64_t idx_capacity,
                                                     int64_t* d_count, void* stream) {
    using namespace plic;
    if (nx < 0 || ny < 0 || nz < 0 || idx_capacity < 0 || !d_count) return PLIC_ERR_ARG;
    const int64_t ncell = (int64_t)nx * ny * nz;
    if (ncell > (int64_t)PLIC_NOALLOC_MAX_CELLS) {
        set_limit_error(ncell);
        return PLIC_ERR_ARG;
    }
    if (ncell > 0 && (!phi || (!idx && idx_capacity > 0))) return PLIC_ERR_ARG;
    if (!aligned(d_count, 8) || (phi && !aligned(phi, 4)) || (idx && !aligned(idx, 4)))
        return PLIC_ERR_ALIGN;
    plic_status st = PLIC_OK;
    int* tiles = noalloc_scratch(&st);
    if (!tiles) return st;
    cudaStream_t s = as_stream(stream);
    if (ncell == 0) {
        cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) { set_last_error("vof_interface_compact_noalloc", e); return PLIC_ERR_CUDA; }
        return PLIC_OK;
    }
    // every tile entry that a pass reads is written earlier in the same call,
    // so the contents left by a previous call need no clearing
    const int64_t nt = compact_tiles(ncell);
    k_compact_count<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, ncell, tiles);
    k_compact_scan<<<1, 1024, 0, s>>>(tiles, nt, d_count);
    k_compact_write<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, ncell, tiles, idx, idx_capacity);
    return check_launch("vof_interface_compact_noalloc");
}
