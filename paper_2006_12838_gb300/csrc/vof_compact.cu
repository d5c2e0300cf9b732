// vof_compact.cu -- interface-cell compaction (Sec. 4.1, Eq. 33): the ordered
// list of interior cells with 0 < phi < 1, and plic_workspace_bytes().
//
// Three launches, no atomics and no inter-block waiting, so the list is in
// ascending cell order and identical run to run.  A tile is a run of whole
// x-rows (about 4096 cells):
//   1. k_compact_count : each block counts the interface cells of its tile.
//   2. k_compact_scan  : one block turns the per-tile counts into exclusive
//                        offsets (in place) and writes the total to *d_count.
//   3. k_compact_write : each block re-reads its tile (L2-resident right after
//                        pass 1 for fields up to the 129 MB L2), keeps the row
//                        ballots in shared memory, scans the row counts and
//                        writes the indices at its offset, in order.
// HBM roofline: 4 B per field cell read once (pass 3 mostly hits L2), plus
// 4 B per interface cell written.
#include <mutex>
#include <stdio.h>

#include "host_common.h"

namespace plic {

constexpr int CT_THREADS = 256;
constexpr int CT_WARPS = CT_THREADS / 32;
constexpr int CT_TILE = 4096;            // cells per tile (whole x-rows)
constexpr int CT_MAX_ROWS = 1024;        // rows per tile at most (nx >= 4)
constexpr int CT_MAX_WORDS = 2048;       // ballot words per tile at most

// Rows (x-lines) per tile: as many whole rows as fit in CT_TILE cells.
__host__ __device__ inline int tile_rows(int nx) {
    const int r = nx > 0 ? CT_TILE / nx : 1;
    return r < 1 ? 1 : (r > CT_MAX_ROWS ? CT_MAX_ROWS : r);
}

// Work is split by rows: warp w of a block takes rows w, w + 8, ... of the
// block's tile.  A row's (y, z) is computed once per warp (one division), rows
// on the field boundary are skipped without reading them, and a row is read
// as coalesced 128-byte segments.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_count(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                int* __restrict__ tile_count) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rbeg = (int64_t)blockIdx.x * R;
    const int64_t rend = rbeg + R < rows ? rbeg + R : rows;
    int cnt = 0;
    for (int64_t r = rbeg + warp; r < rend; r += CT_WARPS) {
        const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
        if (y < 1 || y > ny - 2 || z < 1 || z > nz - 2) continue;
        const float* row = phi + r * nx;
        for (int x = lane; x < nx; x += 32) {
            const float v = __ldg(row + x);
            cnt += (x >= 1 && x <= nx - 2 && v > 0.0f && v < 1.0f);
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    __shared__ int ws[CT_WARPS];
    if (lane == 0) ws[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < CT_WARPS; ++w) t += ws[w];
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

// Pass 3: the warps ballot their rows into shared memory (one 32-bit word per
// 32 cells of a row), the block scans the per-row counts, and each warp writes
// its rows' indices at the row offsets -- in ascending cell order.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_write(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                const int* __restrict__ tile_offset, int32_t* __restrict__ idx, int64_t cap) {
    __shared__ unsigned bal[CT_MAX_WORDS];
    __shared__ int rowoff[CT_MAX_ROWS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rbeg = (int64_t)blockIdx.x * R;
    const int64_t rend = rbeg + R < rows ? rbeg + R : rows;
    const int nr = (int)(rend - rbeg);
    const int wpr = (nx + 31) >> 5;                 // ballot words per row
    const bool in_smem = (int64_t)nr * wpr <= CT_MAX_WORDS;
    for (int k = warp; k < nr; k += CT_WARPS) {
        const int64_t r = rbeg + k;
        const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
        const bool row_ok = y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2;
        int cnt = 0;
        if (row_ok) {
            const float* row = phi + r * nx;
            for (int x0 = 0; x0 < nx; x0 += 32) {
                const int x = x0 + lane;
                const float v = x < nx ? __ldg(row + x) : 0.0f;
                const unsigned b = __ballot_sync(0xffffffffu, x >= 1 && x <= nx - 2 && v > 0.0f && v < 1.0f);
                if (in_smem && lane == 0) bal[k * wpr + (x0 >> 5)] = b;
                cnt += __popc(b);
            }
        } else if (in_smem) {
            for (int w = lane; w < wpr; w += 32) bal[k * wpr + w] = 0u;
        }
        if (lane == 0) rowoff[k] = cnt;
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of nr <= 1024 row counts: each lane sums a run of rows
        const int per = (nr + 31) >> 5;
        const int k0 = lane * per, k1 = min(k0 + per, nr);
        int s = 0;
        for (int k = k0; k < k1; ++k) s += rowoff[k];
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - s;
        for (int k = k0; k < k1; ++k) {
            const int c = rowoff[k];
            rowoff[k] = run;
            run += c;
        }
    }
    __syncthreads();
    const int64_t base = tile_offset[blockIdx.x];
    for (int k = warp; k < nr; k += CT_WARPS) {
        const int64_t r = rbeg + k;
        const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
        if (!(y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2)) continue;
        int64_t pos = base + rowoff[k];
        const float* row = phi + r * nx;
        for (int x0 = 0; x0 < nx; x0 += 32) {
            const int x = x0 + lane;
            unsigned b;
            if (in_smem) {
                b = bal[k * wpr + (x0 >> 5)];
            } else {
                const float v = x < nx ? __ldg(row + x) : 0.0f;
                b = __ballot_sync(0xffffffffu, x >= 1 && x <= nx - 2 && v > 0.0f && v < 1.0f);
            }
            if ((b >> lane) & 1u) {
                const int64_t p = pos + __popc(b & ((1u << lane) - 1u));
                if (p < cap) idx[p] = (int32_t)(r * nx + x);
            }
            pos += __popc(b);
        }
    }
}

// Tiles of a field: whole x-rows, tile_rows(nx) per tile.
static int64_t compact_tiles(int nx, int64_t rows) {
    const int R = tile_rows(nx);
    return (rows + R - 1) / R;
}

}  // namespace plic

extern "C" size_t plic_workspace_bytes(int op, int64_t arg) {
    if (arg < 0) return 0;
    switch (op) {
        case PLIC_WS_COMPACT: {
            // at least one tile per 4096 cells or per row (for rows longer
            // than 4096 cells), rounded up; an upper bound for any shape with
            // arg cells and at most CT_MAX_ROWS rows per tile
            const int64_t t = (arg + plic::CT_TILE - 1) / plic::CT_TILE * 2 + 1;
            const size_t b = (size_t)t * sizeof(int);
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
    if (nx < 3 || ny < 3 || nz < 3) {        // no cell has all 26 neighbours inside
        cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) { set_last_error("vof_interface_compact", e); return PLIC_ERR_CUDA; }
        return PLIC_OK;
    }
    if (!phi || (!idx && idx_capacity > 0) || !workspace) return PLIC_ERR_ARG;
    if (ws_bytes < plic_workspace_bytes(PLIC_WS_COMPACT, ncell)) return PLIC_ERR_ARG;
    if (!aligned(phi, 4) || (idx && !aligned(idx, 4)) || !aligned(workspace, 256)) return PLIC_ERR_ALIGN;
    const int64_t rows = (int64_t)ny * nz;
    const int R = tile_rows(nx);
    const int64_t nt = compact_tiles(nx, rows);
    if ((size_t)nt * sizeof(int) > ws_bytes) return PLIC_ERR_ARG;
    int* tiles = reinterpret_cast<int*>(workspace);
    k_compact_count<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles);
    k_compact_scan<<<1, 1024, 0, s>>>(tiles, nt, d_count);
    k_compact_write<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles, idx, idx_capacity);
    return check_launch("vof_interface_compact");
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  The per-tile scratch of the three passes lives in
// a file-scope device array instead of a caller-provided workspace.  Every
// GPU that loads the library holds these 256 KiB until the process exits.
// ---------------------------------------------------------------------------
namespace plic {

// one int per tile; a field of at most PLIC_NOALLOC_MAX_CELLS cells has at most
// 2 * cells / CT_TILE + 1 tiles (see plic_workspace_bytes)
constexpr int64_t kNoAllocMaxTiles = 2 * (PLIC_NOALLOC_MAX_CELLS / CT_TILE) + 1;

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
    if (nx < 3 || ny < 3 || nz < 3) {        // no cell has all 26 neighbours inside
        cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) { set_last_error("vof_interface_compact_noalloc", e); return PLIC_ERR_CUDA; }
        return PLIC_OK;
    }
    // every tile entry that a pass reads is written earlier in the same call,
    // so the contents left by a previous call need no clearing
    const int64_t rows = (int64_t)ny * nz;
    const int R = tile_rows(nx);
    const int64_t nt = compact_tiles(nx, rows);
    if (nt > kNoAllocMaxTiles) {
        set_limit_error(ncell);
        return PLIC_ERR_ARG;
    }
    k_compact_count<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles);
    k_compact_scan<<<1, 1024, 0, s>>>(tiles, nt, d_count);
    k_compact_write<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles, idx, idx_capacity);
    return check_launch("vof_interface_compact_noalloc");
}
