// vof_compact.cu -- interface-cell compaction (Sec. 4.1, Eq. 33): the ordered
// list of interior cells with 0 < phi < 1, and plic_workspace_bytes().
//
// Two or three launches, no atomics and no inter-block waiting, so the list
// is in ascending cell order and identical run to run.  A tile is a run of
// whole x-rows (about 8192 cells):
//   1. k_compact_count : each block counts the interface cells of its tile and,
//                        with room in the workspace, stores the tile's
//                        interface bits (one word per 32 cells of a row);
//                        k_compact_count_p2 does the same for 16-byte aligned
//                        rows of 128 * 2^k cells with slot arithmetic in
//                        shifts and masks.
//   2. k_compact_scan  : one block turns the per-tile counts into exclusive
//                        offsets (in place) and writes the total to *d_count;
//                        only for fields of more than 4096 tiles (about 33 M
//                        cells): below, pass 3 sums the counts of the tiles
//                        before each block, and the warp of the last tile
//                        writes the total.
//   3. k_compact_emit  : one warp per tile writes the indices of the tile's
//                        cells from the stored bits.  Without room for the bits
//                        (rows shorter than 32 cells) or without a workspace
//                        (the allocation-free entry), k_compact_write recounts
//                        each row from the field and scans the row counts
//                        itself.
// HBM roofline: 4 B per field cell read once + 1/8 B per cell of bits written
// and read back for the tiles holding interface cells, plus 4 B per interface
// cell written.
#include <mutex>
#include <stdio.h>

#include "host_common.h"

namespace plic {

constexpr int CT_THREADS = 256;
constexpr int CT_WARPS = CT_THREADS / 32;
constexpr int CT_TILE = 8192;            // cells per tile (whole x-rows)
constexpr int CT_MAX_ROWS = 4096;        // rows per tile at most (CT_TILE / 3 for nx >= 3)
constexpr int CT_MAX_WORDS = 2048;       // ballot words per tile kept in shared memory
constexpr int64_t CT_FUSED_SCAN_TILES = 4096;   // tiles up to which pass 3 does its own prefix sum

// Rows (x-lines) per tile: as many whole rows as fit in CT_TILE cells.
__host__ __device__ inline int tile_rows(int nx) {
    const int r = nx > 0 ? CT_TILE / nx : 1;
    return r < 1 ? 1 : (r > CT_MAX_ROWS ? CT_MAX_ROWS : r);
}

__device__ __forceinline__ bool iface(float v) { return v > 0.0f && v < 1.0f; }

// Interface bits of one row, 32 cells per word (bit x % 32 of word x / 32),
// with the boundary columns x = 0 and x = nx - 1 cleared; the caller has
// checked the row's y and z.  `fn(word_index, bits)` is called by one lane per
// word; returns the row's count in every lane.  With 16-byte aligned rows
// (nx % 4 == 0) each lane loads 4 cells at once.
template <typename F>
__device__ __forceinline__ int row_bits(const float* __restrict__ row, int nx, bool vec, F fn) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    if (vec) {
        for (int x0 = 0; x0 < nx; x0 += 128) {
            const int x = x0 + 4 * lane;
            unsigned m = 0u;
            if (x < nx) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(row + x));
                m = (unsigned)iface(v.x) | ((unsigned)iface(v.y) << 1) |
                    ((unsigned)iface(v.z) << 2) | ((unsigned)iface(v.w) << 3);
                if (x == 0) m &= ~1u;
                if (x + 3 == nx - 1) m &= ~8u;
            }
            // gather the nibbles of 8 lanes into one 32-bit word
            unsigned w = m << (4 * (lane & 7));
            w |= __shfl_xor_sync(0xffffffffu, w, 1);
            w |= __shfl_xor_sync(0xffffffffu, w, 2);
            w |= __shfl_xor_sync(0xffffffffu, w, 4);
            cnt += __popc(m);
            if ((lane & 7) == 0 && x < nx) fn((x0 >> 5) + (lane >> 3), w);
        }
    } else {
        for (int x0 = 0; x0 < nx; x0 += 32) {
            const int x = x0 + lane;
            const float v = x < nx ? __ldg(row + x) : 0.0f;
            const unsigned b = __ballot_sync(0xffffffffu, x >= 1 && x <= nx - 2 && iface(v));
            cnt += (b >> lane) & 1u;
            if (lane == 0) fn(x0 >> 5, b);
        }
    }
    return __reduce_add_sync(0xffffffffu, cnt);
}

// The interface test 0 < phi < 1 on the float's bits: the positive floats
// below 1.0f are exactly the bit patterns 1 .. 0x3F7FFFFF (zero, negative
// values, 1.0f and above, infinities and NaNs all fall outside), so one
// unsigned compare of u - 1 decides it.
__device__ __forceinline__ bool iface_bits(unsigned u) { return u - 1u < 0x3F7FFFFFu; }

// Vector path helpers: the 4-bit interface mask of the float4 at column x of
// a row (boundary columns cleared), and the gather of the nibbles of 8 lanes
// into the row's 32-bit word (x0 / 32 + lane / 8), stored by `fn`.
__device__ __forceinline__ unsigned nib4(float4 v, int x, int nx) {
    unsigned m = (unsigned)iface_bits(__float_as_uint(v.x)) |
                 ((unsigned)iface_bits(__float_as_uint(v.y)) << 1) |
                 ((unsigned)iface_bits(__float_as_uint(v.z)) << 2) |
                 ((unsigned)iface_bits(__float_as_uint(v.w)) << 3);
    if (x == 0) m &= ~1u;
    if (x + 3 == nx - 1) m &= ~8u;
    return x < nx ? m : 0u;
}

template <typename F>
__device__ __forceinline__ void emit_nibbles(unsigned m, int x0, int nx, F fn) {
    const int lane = threadIdx.x & 31;
    unsigned w = m << (4 * (lane & 7));
    w |= __shfl_xor_sync(0xffffffffu, w, 1);
    w |= __shfl_xor_sync(0xffffffffu, w, 2);
    w |= __shfl_xor_sync(0xffffffffu, w, 4);
    if ((lane & 7) == 0 && x0 + 4 * lane < nx) fn((x0 >> 5) + (lane >> 3), w);
}

__device__ __forceinline__ float4 ld_row4(const float* __restrict__ row, bool ok, int x, int nx) {
    return (ok && x < nx) ? __ldg(reinterpret_cast<const float4*>(row + x))
                          : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Pass 1.  Work is split by rows: warp w of a block takes rows w, w + 8, ...
// of the block's tile.  A row's (y, z) is computed once per warp, rows on the
// field boundary are skipped without reading them.  The per-tile count goes
// to tile_count; with `bits` given, the row's interface bits are stored too
// (wpr words per row), so that pass 3 need not read the field again.  In the
// vector path a warp takes two rows at a time and issues the four 16-byte
// loads per lane of 256 columns of both rows before using any of them, so
// every lane keeps 64 bytes in flight (the pass is bound by load latency, not
// by the compare work); rows of more than 512 cells are cut into 512-cell
// segments, four loads per lane each (1024-cell rows: 0.26 -> 0.19 ms on a
// 1 GiB field, the same as for 512-cell rows).  Eight blocks per SM (32
// registers, a few bytes spilled) keep more loads in flight than the six that
// 40 registers allow.
__global__ void __launch_bounds__(CT_THREADS, 8)
k_compact_count(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                int* __restrict__ tile_count, unsigned* __restrict__ bits, int vec) {
    pdl_wait();                                     // the kernel that wrote the field complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpr = (nx + 31) >> 5;
    const int64_t rbeg = (int64_t)blockIdx.x * R;
    const int64_t rend = rbeg + R < rows ? rbeg + R : rows;
    // rows < 2^31 (fields of at most 2^31 - 1 cells): 32-bit division
    auto interior = [&](int64_t r) {
        const unsigned z = (unsigned)r / (unsigned)ny, y = (unsigned)r - z * (unsigned)ny;
        return y >= 1u && y + 2u <= (unsigned)ny && z >= 1u && z + 2u <= (unsigned)nz;
    };
    int cnt = 0;
    if (vec && nx > 512) {
        // long rows (fewer than 16 per tile): the tile's rows are cut into
        // 512-cell segments (the last of a row partial), warp w takes segments
        // w, w + 8, ..., and each lane issues its four 16-byte loads of a
        // segment together, as in the two-row form below
        const int spr = (nx + 511) >> 9;
        const int nseg = (int)(rend - rbeg) * spr;
        for (int sg = warp; sg < nseg; sg += CT_WARPS) {
            const int rr = sg / spr;
            const int x0 = (sg - rr * spr) << 9;
            const int64_t r = rbeg + rr;
            const bool ok = interior(r);
            const float* row = phi + r * nx;
            unsigned* br = bits ? bits + r * wpr : nullptr;
            const int xa = x0 + 4 * lane;
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld_row4(row, ok, xa + 128 * u, nx);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned m = ok ? nib4(v[u], xa + 128 * u, nx) : 0u;
                cnt += __popc(m);
                emit_nibbles(m, x0 + 128 * u, nx, [&](int w, unsigned b) { if (br) br[w] = b; });
            }
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
    } else if (vec) {
        for (int64_t ra = rbeg + warp; ra < rend; ra += 2 * CT_WARPS) {
            const int64_t rb = ra + CT_WARPS;
            const bool oka = interior(ra), hasb = rb < rend, okb = hasb && interior(rb);
            const float* rowa = phi + ra * nx;
            const float* rowb = phi + (hasb ? rb : ra) * nx;
            unsigned* ba = bits ? bits + ra * wpr : nullptr;
            unsigned* bb = (bits && hasb) ? bits + rb * wpr : nullptr;
            int ca = 0, cb = 0;
            for (int x0 = 0; x0 < nx; x0 += 256) {
                const int xa = x0 + 4 * lane, xb = xa + 128;
                const float4 a0 = ld_row4(rowa, oka, xa, nx), a1 = ld_row4(rowa, oka, xb, nx);
                const float4 b0 = ld_row4(rowb, okb, xa, nx), b1 = ld_row4(rowb, okb, xb, nx);
                const unsigned ma0 = oka ? nib4(a0, xa, nx) : 0u, ma1 = oka ? nib4(a1, xb, nx) : 0u;
                const unsigned mb0 = okb ? nib4(b0, xa, nx) : 0u, mb1 = okb ? nib4(b1, xb, nx) : 0u;
                ca += __popc(ma0) + __popc(ma1);
                cb += __popc(mb0) + __popc(mb1);
                emit_nibbles(ma0, x0, nx, [&](int w, unsigned b) { if (ba) ba[w] = b; });
                emit_nibbles(ma1, x0 + 128, nx, [&](int w, unsigned b) { if (ba) ba[w] = b; });
                emit_nibbles(mb0, x0, nx, [&](int w, unsigned b) { if (bb) bb[w] = b; });
                emit_nibbles(mb1, x0 + 128, nx, [&](int w, unsigned b) { if (bb) bb[w] = b; });
            }
            cnt += ca + cb;                       // the lane's share
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
    } else {
        for (int64_t r = rbeg + warp; r < rend; r += CT_WARPS) {
            unsigned* rb = bits ? bits + r * wpr : nullptr;
            if (!interior(r)) {
                if (rb)
                    for (int w = lane; w < wpr; w += 32) rb[w] = 0u;
                continue;
            }
            const int c = row_bits(phi + r * nx, nx, false, [&](int w, unsigned b) {
                if (rb) rb[w] = b;
            });
            cnt += c;
        }
    }
    __shared__ int ws[CT_WARPS];
    if (lane == 0) ws[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < CT_WARPS; ++w) t += ws[w];
        tile_count[blockIdx.x] = t;
    }
    pdl_trigger();                                  // the next pass may be scheduled
}

// Pass 1 for 16-byte aligned rows of 128 * 2^k cells (the power-of-two edges
// of the workloads), streamlined: the tile is a run of 128-cell slots (spr =
// nx / 128 per row, 2^lspr), slot s of the tile is row s >> lspr at column
// (s & (spr - 1)) * 128, so no column test is needed and a slot's bit words
// are contiguous; warp w takes slots 4 w + u + 32 k and issues the four
// 16-byte loads per lane of a trip together.  A row's (y, z) is stepped from
// the tile's first row (a division only where the tile wraps to the next z).
// The bits are the nibble layout of the general pass (word x / 32 of a row,
// bit x % 32), so pass 3 is the same.
__global__ void __launch_bounds__(CT_THREADS, 8)
k_compact_count_p2(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                   int lspr, int* __restrict__ tile_count, unsigned* __restrict__ bits) {
    pdl_wait();                                     // the kernel that wrote the field complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rbeg = (int64_t)blockIdx.x * R;
    const int nr = (int)(rbeg + R < rows ? R : rows - rbeg);
    const int nslot = nr << lspr;
    const unsigned smask = (1u << lspr) - 1u;
    const unsigned z0 = (unsigned)rbeg / (unsigned)ny, y0 = (unsigned)rbeg - z0 * (unsigned)ny;
    const float4* base = reinterpret_cast<const float4*>(phi + rbeg * nx) + lane;
    unsigned* tb = bits + (rbeg * nx >> 5) + (lane >> 3);
    const unsigned shl = 4u * (unsigned)(lane & 7);
    const bool writer = (lane & 7) == 0;
    // the columns x = 0 and x = nx - 1 are lane 0's first and lane 31's last
    // component of a row's first and last slot
    const unsigned first_clear = lane == 0 ? 1u : 0u, last_clear = lane == 31 ? 8u : 0u;
    int cnt = 0;
    for (int s0 = warp * 4; s0 < nslot; s0 += 4 * CT_WARPS) {
        float4 v[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int sl = s0 + u;
            const unsigned row = (unsigned)sl >> lspr;
            unsigned y = y0 + row, z = z0;
            if (y >= (unsigned)ny) {                // the tile wraps to the next z plane
                const unsigned k = y / (unsigned)ny;
                z += k;
                y -= k * (unsigned)ny;
            }
            ok[u] = sl < nslot && y - 1u < (unsigned)ny - 2u && z - 1u < (unsigned)nz - 2u;
            v[u] = ok[u] ? __ldg(base + 32 * sl) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int sl = s0 + u;
            const unsigned col = (unsigned)sl & smask;
            unsigned m = (unsigned)iface_bits(__float_as_uint(v[u].x)) |
                         ((unsigned)iface_bits(__float_as_uint(v[u].y)) << 1) |
                         ((unsigned)iface_bits(__float_as_uint(v[u].z)) << 2) |
                         ((unsigned)iface_bits(__float_as_uint(v[u].w)) << 3);
            m &= ~((col == 0u ? first_clear : 0u) | (col == smask ? last_clear : 0u));
            m = ok[u] ? m : 0u;
            cnt += __popc(m);
            unsigned w = m << shl;
            w |= __shfl_xor_sync(0xffffffffu, w, 1);
            w |= __shfl_xor_sync(0xffffffffu, w, 2);
            w |= __shfl_xor_sync(0xffffffffu, w, 4);
            if (writer && sl < nslot) tb[4 * sl] = w;
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
    pdl_trigger();                                  // the next pass may be scheduled
}

// Pass 2: exclusive scan of ntiles ints by one block of 1024 threads, 32
// consecutive entries per thread and round (eight 16-byte loads issued
// together: one round up to 32 768 tiles, about 268 M cells); the total goes
// to *d_count.  tile_count is 16-byte aligned (the workspace start).
__global__ void __launch_bounds__(1024)
k_compact_scan(int* __restrict__ tile_count, int64_t ntiles, int64_t* __restrict__ d_count) {
    __shared__ long long wsum[32];
    pdl_wait();                                     // pass 1 complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += 32 * 1024) {
        const int64_t i0 = b0 + 32 * (int64_t)threadIdx.x;
        const bool full = i0 + 32 <= ntiles;
        int v[32];
        if (full) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int4 x = reinterpret_cast<const int4*>(tile_count + i0)[j];
                v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = i0 + j < ntiles ? tile_count[i0 + j] : 0;
        }
        int own = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) own += v[j];
        long long x = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        long long run = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - own;
        if (full) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int4 o4;
                o4.x = (int)run; run += v[4 * j];
                o4.y = (int)run; run += v[4 * j + 1];
                o4.z = (int)run; run += v[4 * j + 2];
                o4.w = (int)run; run += v[4 * j + 3];
                reinterpret_cast<int4*>(tile_count + i0)[j] = o4;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (i0 + j < ntiles) tile_count[i0 + j] = (int)run;
                run += v[j];
            }
        }
        carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_count = carry;
    pdl_trigger();
}

// Pass 3 without stored bits: each warp recomputes its rows' interface bits
// from the field, the block scans the row counts, and every warp writes its
// rows' indices at the row offsets, in ascending cell order.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_write(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                const int* __restrict__ tile_offset, int32_t* __restrict__ idx, int64_t cap, int vec,
                int64_t* __restrict__ d_count) {
    __shared__ unsigned bal[CT_MAX_WORDS];
    __shared__ int rowoff[CT_MAX_ROWS + 1];
    __shared__ int rowcnt[CT_MAX_ROWS];
    __shared__ long long s_base[CT_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_wait();                                     // the passes before complete
    // with d_count given, tile_offset holds the per-tile counts of pass 1 and
    // the block sums those of the tiles before its own (few tiles: no scan
    // launch); the last block writes the total
    if (d_count) {
        long long part = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += CT_THREADS) part += __ldg(tile_offset + i);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_base[warp] = part;
    }
    const int64_t rbeg = (int64_t)blockIdx.x * R;
    const int64_t rend = rbeg + R < rows ? rbeg + R : rows;
    const int nr = (int)(rend - rbeg);
    const int wpr = (nx + 31) >> 5;                 // words per row
    // the tile's bits are kept in shared memory when they fit, else each
    // word is recomputed when it is written
    const bool in_smem = (int64_t)nr * wpr <= CT_MAX_WORDS;
    for (int k = warp; k < nr; k += CT_WARPS) {
        const int64_t r = rbeg + k;
        int cnt = 0;
        const unsigned z = (unsigned)r / (unsigned)ny, y = (unsigned)r - z * (unsigned)ny;
        if (y >= 1u && y + 2u <= (unsigned)ny && z >= 1u && z + 2u <= (unsigned)nz) {
            cnt = row_bits(phi + r * nx, nx, vec != 0, [&](int w, unsigned b) {
                if (in_smem) bal[k * wpr + w] = b;
            });
        } else if (in_smem) {
            for (int w = lane; w < wpr; w += 32) bal[k * wpr + w] = 0u;
        }
        if (lane == 0) rowoff[k] = rowcnt[k] = cnt;
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
    int64_t base;
    if (d_count) {
        long long b = 0;
#pragma unroll
        for (int w = 0; w < CT_WARPS; ++w) b += s_base[w];
        base = b;
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_count = b + tile_offset[blockIdx.x];
    } else {
        base = tile_offset[blockIdx.x];
    }
    for (int k = warp; k < nr; k += CT_WARPS) {
        if (rowcnt[k] == 0) continue;               // most rows of a field hold no interface cell
        const int64_t r = rbeg + k;
        int64_t pos = base + rowoff[k];
        // one lane per 32-cell word: warp prefix of the word counts, then each
        // lane writes its word's cells in order
        for (int w0 = 0; w0 < wpr; w0 += 32) {
            const int w = w0 + lane;
            unsigned b = 0u;
            if (w < wpr) {
                if (in_smem) {
                    b = bal[k * wpr + w];
                } else {
                    // recompute this word (rare: tiles of very long rows)
                    const float* row = phi + r * nx;
                    const unsigned z = (unsigned)r / (unsigned)ny, y = (unsigned)r - z * (unsigned)ny;
                    if (y >= 1u && y + 2u <= (unsigned)ny && z >= 1u && z + 2u <= (unsigned)nz)
                        for (int j = 0; j < 32; ++j) {
                            const int x = 32 * w + j;
                            if (x >= 1 && x <= nx - 2 && iface(__ldg(row + x))) b |= 1u << j;
                        }
                }
            }
            const int c = __popc(b);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int64_t p = pos + incl - c;
            const int64_t cell0 = r * nx + 32 * (int64_t)w;
            while (b) {
                const int j = __ffs(b) - 1;
                b &= b - 1u;
                if (p < cap) idx[p] = (int32_t)(cell0 + j);
                ++p;
            }
            pos += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    pdl_trigger();
}

// Pass 3 with pass 1's interface bits: one warp per tile, a block of CT_WARPS
// consecutive tiles.  The tile's base is the sum of the counts of the tiles
// before it (fused: few tiles; the block sums the counts before its first
// tile, each warp adds those of the block's tiles before its own, and the
// warp of the last tile writes the total) or the exclusive offset written by
// the scan launch (then the tile's count is the next offset, or the total,
// minus its own).  A tile's words are contiguous (its rows, wpr words each):
// each lane takes 8 consecutive words (two int4 loads when aligned), one warp
// scan of the lane counts gives each lane its first slot, and the lane writes
// its words' cells in ascending order.  One dependent load per tile (the
// words, issued with the tile counts) and one barrier, in the fused prefix.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_emit(int nx, int R, int64_t rows, int64_t ntiles, const int* __restrict__ tiles,
               const unsigned* __restrict__ bits, int32_t* __restrict__ idx, int64_t cap,
               int fused, int64_t* __restrict__ d_count) {
    __shared__ long long s_part[CT_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * CT_WARPS;
    pdl_wait();                                     // the passes before complete
    const int64_t t = t0 + warp;
    const bool live = t < ntiles;
    const int64_t rbeg = t * R;
    const int nr = live ? (int)(rbeg + R < rows ? R : rows - rbeg) : 0;
    const unsigned wpr = ((unsigned)nx + 31u) >> 5;
    const int nw = nr * (int)wpr;
    const unsigned* tb = bits + rbeg * (int64_t)wpr;
    const bool al = ((rbeg * (int64_t)wpr) & 3) == 0;
    // the lane's 8 words from word wl of the tile (none past the tile's end)
    auto words = [&](unsigned (&b)[8], int wl) {
        if (al && wl + 8 <= nw) {
            const int4 x = __ldg(reinterpret_cast<const int4*>(tb + wl));
            const int4 y = __ldg(reinterpret_cast<const int4*>(tb + wl + 4));
            b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w;
            b[4] = y.x; b[5] = y.y; b[6] = y.z; b[7] = y.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) b[k] = wl + k < nw ? __ldg(tb + wl + k) : 0u;
        }
    };
    // the first 256 words of the tile are loaded before the tile counts are
    // summed (the whole tile for rows of up to 256 cells): one round trip
    unsigned b[8];
    words(b, 8 * lane);
    long long base = 0;
    int tcount = 0;
    if (fused) {
        long long part = 0;
        const int4* t4 = reinterpret_cast<const int4*>(tiles);
        const int n4 = (int)(t0 >> 2);
        int4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = threadIdx.x + u * CT_THREADS;
            v[u] = q < n4 ? __ldg(t4 + q) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) part += (long long)v[u].x + v[u].y + v[u].z + v[u].w;
        if (threadIdx.x < (int)(t0 & 3)) part += __ldg(tiles + 4 * n4 + threadIdx.x);
        const int cj = (lane < CT_WARPS && t0 + lane < ntiles) ? __ldg(tiles + t0 + lane) : 0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_part[warp] = part;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < CT_WARPS; ++w) base += s_part[w];
        base += __reduce_add_sync(0xffffffffu, lane < warp ? cj : 0);
        tcount = __shfl_sync(0xffffffffu, cj, warp);
        if (t == ntiles - 1 && lane == 0) *d_count = base + tcount;
    } else {
        if (!live) return;
        base = __ldg(tiles + t);
        const long long next = t + 1 < ntiles ? (long long)__ldg(tiles + t + 1) : *d_count;
        tcount = (int)(next - base);
    }
    if (!live || tcount == 0) return;
    const unsigned invw = wpr > 1u ? 0xFFFFFFFFu / wpr + 1u : 0u;
    long long pos = base;
    for (int w0 = 0; w0 < nw; w0 += 256) {
        const int wl = w0 + 8 * lane;
        if (w0 > 0) words(b, wl);
        int c = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) c += __popc(b[k]);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        long long p = pos + incl - c;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            unsigned bb = b[k];
            if (!bb) continue;
            const unsigned w = (unsigned)(wl + k);
            const unsigned r = wpr > 1u ? __umulhi(w, invw) : w, wr = w - r * wpr;
            const int64_t cell0 = (rbeg + r) * (int64_t)nx + 32 * (int64_t)wr;
            while (bb) {
                const int q = __ffs(bb) - 1;
                bb &= bb - 1u;
                if (p < cap) idx[p] = (int32_t)(cell0 + q);
                ++p;
            }
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    pdl_trigger();
}

// The passes as programmatic dependent launches (launch_after): each waits
// for the kernel before it on the stream, the first for the one that wrote
// the field.
static cudaError_t launch_count(const float* phi, int nx, int ny, int nz, int R, int64_t rows,
                                int64_t nt, int* tiles, unsigned* bits, int vec, cudaStream_t s) {
    void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&nz, (void*)&R, (void*)&rows,
                    (void*)&tiles, (void*)&bits, (void*)&vec};
    return launch_after(reinterpret_cast<const void*>(&k_compact_count), dim3((unsigned)nt),
                        dim3(CT_THREADS), args, s);
}
static cudaError_t launch_scan(int* tiles, int64_t nt, int64_t* d_count, cudaStream_t s) {
    void* args[] = {(void*)&tiles, (void*)&nt, (void*)&d_count};
    return launch_after(reinterpret_cast<const void*>(&k_compact_scan), dim3(1), dim3(1024), args, s);
}
static cudaError_t launch_write(const float* phi, int nx, int ny, int nz, int R, int64_t rows, int64_t nt,
                                const int* tiles, int32_t* idx, int64_t cap, int vec, int64_t* d_count,
                                cudaStream_t s) {
    void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&nz, (void*)&R, (void*)&rows,
                    (void*)&tiles, (void*)&idx, (void*)&cap, (void*)&vec, (void*)&d_count};
    return launch_after(reinterpret_cast<const void*>(&k_compact_write), dim3((unsigned)nt),
                        dim3(CT_THREADS), args, s);
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
            // tile counts: tiles hold >= CT_TILE/2 cells (or one whole row), so a
            // field of arg cells has at most 2 arg / CT_TILE + 1 tiles; interface
            // bits: one word per 32 cells of each row, at most arg / 16 words
            // for rows of >= 32 cells (shorter rows keep no bits)
            const int64_t t = (arg + plic::CT_TILE - 1) / plic::CT_TILE * 2 + 1;
            const size_t a = ((size_t)t * sizeof(int) + 255) / 256 * 256;
            const size_t b = ((size_t)(arg / 16 + 1) * sizeof(unsigned) + 255) / 256 * 256;
            return a + b;
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
    const size_t tile_bytes = ((size_t)nt * sizeof(int) + 255) / 256 * 256;
    if (tile_bytes > ws_bytes) return PLIC_ERR_ARG;
    int* tiles = reinterpret_cast<int*>(workspace);
    const int64_t words = rows * ((nx + 31) / 32);
    const size_t bits_bytes = ((size_t)words * sizeof(unsigned) + 255) / 256 * 256;
    unsigned* bits = nullptr;
    if (nx >= 32 && tile_bytes + bits_bytes <= ws_bytes)
        bits = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(workspace) + tile_bytes);
    const int vec = (nx % 4 == 0) && aligned(phi, 16);
    // rows of 128 * 2^k cells: the streamlined count pass
    int lspr = -1;
    if (vec && bits && nx >= 128 && nx % 128 == 0 && ((nx / 128) & (nx / 128 - 1)) == 0)
        for (lspr = 0; (128 << lspr) < nx; ++lspr) {}
    cudaError_t e;
    if (lspr >= 0) {
        void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&nz, (void*)&R, (void*)&rows,
                        (void*)&lspr, (void*)&tiles, (void*)&bits};
        e = launch_after(reinterpret_cast<const void*>(&k_compact_count_p2), dim3((unsigned)nt),
                         dim3(CT_THREADS), args, s);
    } else {
        e = launch_count(phi, nx, ny, nz, R, rows, nt, tiles, bits, vec, s);
    }
    // up to CT_FUSED_SCAN_TILES tiles pass 3 sums the counts of the tiles
    // before each block (at most that many L2 reads per block); beyond, one
    // block scans them first
    const bool fused = nt <= CT_FUSED_SCAN_TILES;
    if (e == cudaSuccess && !fused) e = launch_scan(tiles, nt, d_count, s);
    if (e == cudaSuccess) {
        int fz = fused ? 1 : 0;
        if (bits) {
            const int64_t nb = (nt + CT_WARPS - 1) / CT_WARPS;
            void* args[] = {(void*)&nx, (void*)&R, (void*)&rows, (void*)&nt, (void*)&tiles, (void*)&bits,
                            (void*)&idx, (void*)&idx_capacity, (void*)&fz, (void*)&d_count};
            e = launch_after(reinterpret_cast<const void*>(&k_compact_emit), dim3((unsigned)nb),
                             dim3(CT_THREADS), args, s);
        } else {
            e = launch_write(phi, nx, ny, nz, R, rows, nt, tiles, idx, idx_capacity, vec,
                             fused ? d_count : nullptr, s);
        }
    }
    if (e != cudaSuccess) { set_last_error("vof_interface_compact", e); return PLIC_ERR_CUDA; }
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
    // the built-in scratch holds the tile counts only; pass 3 re-reads the field
    const int vec = (nx % 4 == 0) && aligned(phi, 16);
    cudaError_t e = launch_count(phi, nx, ny, nz, R, rows, nt, tiles, nullptr, vec, s);
    const bool fused = nt <= CT_FUSED_SCAN_TILES;
    if (e == cudaSuccess && !fused) e = launch_scan(tiles, nt, d_count, s);
    if (e == cudaSuccess)
        e = launch_write(phi, nx, ny, nz, R, rows, nt, tiles, idx, idx_capacity, vec,
                         fused ? d_count : nullptr, s);
    if (e != cudaSuccess) { set_last_error("vof_interface_compact_noalloc", e); return PLIC_ERR_CUDA; }
    return check_launch("vof_interface_compact_noalloc");
}
