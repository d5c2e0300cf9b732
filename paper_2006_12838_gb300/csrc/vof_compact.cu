// vof_compact.cu -- interface-cell compaction (Sec. 4.1, Eq. 33): the ordered
// list of interior cells with 0 < phi < 1, and plic_workspace_bytes().
//
// Two or three launches, no atomics and no inter-block waiting, so the list
// is in ascending cell order and identical run to run.  A tile is a run of
// whole x-rows (about 8192 cells):
//   1. k_compact_count : each block counts the interface cells of its tile
//                        (one warp vote per 32 cells of a row), stores the
//                        interface bits of every row and each row's offset
//                        within the tile in the workspace, and the tile count.
//   2. k_compact_scan  : one block turns the per-tile counts into exclusive
//                        offsets (in place) and writes the total to *d_count;
//                        only for fields of more than 4096 tiles (about 33 M
//                        cells): below, each block of pass 3 sums the counts
//                        of the tiles before its own, and the last writes the
//                        total.
//   3. k_compact_emit  : each warp writes the indices of its tile's non-empty
//                        rows from the stored bits at the stored row offsets.
//                        Without room for the bits (rows shorter than 32
//                        cells) or without a workspace (the allocation-free
//                        entry), k_compact_write recounts each row from the
//                        field and scans the row counts itself.
// HBM roofline: 4 B per field cell read once + 1/8 B per cell of bits written
// and read back for the non-empty rows, plus 4 B per interface cell written.
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

constexpr int CT_U = 8;                  // 32-cell words of a row loaded per warp and step

// Pass 1.  Warp w of a block takes rows w, w + 8, ... of the block's tile, two
// rows at a time.  Each lane loads one float of every 32-cell word of the
// row (coalesced 128-byte rows of loads, 8 words per step issued before any
// is used), and one warp vote per word gives the word's interface bits in
// cell order; the boundary columns x = 0 and x = nx - 1 are masked out of the
// first and last word.  Rows with y or z on the field boundary are not read.
// The row counts (warp-uniform popcounts) go to shared memory; warp 0 then
// writes the tile's count and, with `row_off` given, each row's offset
// within the tile (exclusive scan); with `bits` given each word is stored
// (wpr = ceil(nx/32) words per row) so that pass 3 need not read the field
// again.  Rows of a tile: R <= CT_MAX_ROWS.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_count(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                int* __restrict__ tile_count, unsigned* __restrict__ bits,
                int* __restrict__ row_off) {
    __shared__ int rc[CT_MAX_ROWS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpr = (nx + 31) >> 5;
    const int64_t rbeg = (int64_t)blockIdx.x * R;
    const int nr = (int)(rbeg + R < rows ? R : rows - rbeg);
    const unsigned* __restrict__ u32 = reinterpret_cast<const unsigned*>(phi);
    const int lastw = wpr - 1;
    const unsigned lastmask = (1u << ((nx - 1) & 31)) - 1u;   // drops x = nx - 1 and beyond
    auto interior = [&](int64_t r) {
        const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
        return y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2;
    };
    for (int k = warp; k < nr; k += 2 * CT_WARPS) {
        const int kb = k + CT_WARPS;
        const bool hasb = kb < nr;
        const int64_t ra = rbeg + k, rb = rbeg + (hasb ? kb : k);
        const bool oka = interior(ra), okb = hasb && interior(rb);
        const unsigned* rowa = u32 + ra * nx;
        const unsigned* rowb = u32 + rb * nx;
        int ca = 0, cb = 0;
        for (int w0 = 0; w0 < wpr; w0 += CT_U) {
            unsigned va[CT_U], vb[CT_U];
#pragma unroll
            for (int u = 0; u < CT_U; ++u) {
                const int x = (w0 + u) * 32 + lane;
                va[u] = (oka && x < nx) ? __ldg(rowa + x) : 0u;
                vb[u] = (okb && x < nx) ? __ldg(rowb + x) : 0u;
            }
            unsigned mya = 0u, myb = 0u;
#pragma unroll
            for (int u = 0; u < CT_U; ++u) {
                const int w = w0 + u;
                unsigned ma = __ballot_sync(0xffffffffu, iface_bits(va[u]));
                unsigned mb = __ballot_sync(0xffffffffu, iface_bits(vb[u]));
                const unsigned cm = (w == 0 ? ~1u : ~0u) & (w == lastw ? lastmask : ~0u);
                ma &= cm;
                mb &= cm;
                ca += __popc(ma);
                cb += __popc(mb);
                mya = lane == u ? ma : mya;
                myb = lane == u ? mb : myb;
            }
            if (bits && lane < CT_U && w0 + lane < wpr) {
                if (oka) bits[ra * wpr + w0 + lane] = mya;
                if (okb) bits[rb * wpr + w0 + lane] = myb;
            }
        }
        if (lane == 0) {
            rc[k] = ca;
            if (hasb) rc[kb] = cb;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the nr row counts: each lane sums a run of rows
        const int per = (nr + 31) >> 5;
        const int k0 = lane * per, k1 = min(k0 + per, nr);
        int sum = 0;
        for (int k = k0; k < k1; ++k) sum += rc[k];
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (row_off) {
            int run = incl - sum;
            for (int k = k0; k < k1; ++k) {
                row_off[rbeg + k] = run;
                run += rc[k];
            }
        }
        if (lane == 31) tile_count[blockIdx.x] = incl;
    }
}

// ---------------------------------------------------------------------------
// Pass 1, streaming form (rows of nx % 4 == 0 cells, at most CT_TILE cells,
// 16-byte aligned field): a persistent grid of blocks, each taking tiles
// t = blockIdx.x, + gridDim.x, ...  One thread streams every tile (whole rows,
// contiguous in memory) into shared memory with a cp.async.bulk copy that
// completes on the stage's mbarrier, CT_STAGES tiles ahead; all warps count
// from shared memory (one float per lane and word, one vote per word), warp
// 0 scans the row counts into row offsets.  Waits on the mbarriers are
// bounded: after CT_WAIT_LIMIT polls a block marks the count of each tile it
// has not finished with CT_FAILED (which the scan and the write pass turn
// into *d_count = -1 and no list), waits (bounded) for its copies in flight
// and leaves.
// ---------------------------------------------------------------------------
constexpr int CT_STAGES = 3;
constexpr int CT_WAIT_LIMIT = 1 << 16;   // hardware-suspended polls (each up to a few us)
constexpr int CT_FAILED = -2147483647 - 1;  // tile count of a tile whose copy never arrived

constexpr int CT_STREAM_ROWS = CT_TILE / 4;   // rows of a tile when nx >= 4

struct CountSmem {
    float buf[CT_STAGES][CT_TILE];           // 3 x 32 KB
    int rc[2][CT_STREAM_ROWS];               // row counts of two consecutive tiles
    unsigned long long bar[CT_STAGES];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One potentially blocking test of the phase `parity` of an mbarrier: the
// thread is suspended in hardware until the phase completes or a
// system-defined time limit passes (then false).
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0u;
}

// Bounded wait for the phase `parity` of an mbarrier to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < CT_WAIT_LIMIT; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Thread 0: stream tile t (rows rbeg .. rbeg + nr - 1) into stage s.
__device__ __forceinline__ void issue_tile(CountSmem& sm, int s, const float* phi, int nx,
                                           int64_t rbeg, int nr) {
    const uint32_t bytes = (uint32_t)nr * (uint32_t)nx * 4u;
    const uint32_t bar = smem_addr(&sm.bar[s]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(sm.buf[s])), "l"(phi + rbeg * nx), "r"(bytes), "r"(bar)
                 : "memory");
}

__global__ void __launch_bounds__(CT_THREADS)
k_compact_count_stream(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                       int64_t ntiles, int* __restrict__ tile_count, unsigned* __restrict__ bits,
                       int* __restrict__ row_off) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CountSmem& sm = *reinterpret_cast<CountSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpr = (nx + 31) >> 5;
    const int lastw = wpr - 1;
    const unsigned lastmask = (1u << ((nx - 1) & 31)) - 1u;   // drops x = nx - 1
    auto tile_rows_of = [&](int64_t t) {
        const int64_t rb = t * R;
        return (int)(rb + R < rows ? R : rows - rb);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < CT_STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&sm.bar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // tiles of this block: t_k = blockIdx.x + k gridDim.x
    const int64_t first = blockIdx.x, step = gridDim.x;
    const int64_t nmine = first < ntiles ? (ntiles - first + step - 1) / step : 0;
    if (threadIdx.x == 0)
        for (int64_t k = 0; k < CT_STAGES && k < nmine; ++k) {
            const int64_t t = first + k * step;
            issue_tile(sm, (int)k, phi, nx, t * R, tile_rows_of(t));
        }
    int64_t k = 0;
    bool ok = true;
    for (; k < nmine; ++k) {
        const int s = (int)(k % CT_STAGES);
        const uint32_t parity = (uint32_t)((k / CT_STAGES) & 1);
        const int64_t t = first + k * step;
        const int64_t rbeg = t * R;
        const int nr = tile_rows_of(t);
        int* rc = sm.rc[k & 1];
        // one thread waits for the copy, the barrier releases the others
        if (threadIdx.x == 0) ok = mbar_wait(smem_addr(&sm.bar[s]), parity);
        if (__syncthreads_or(!ok)) { ok = false; break; }
        const float* tb = sm.buf[s];
        for (int kk = warp; kk < nr; kk += CT_WARPS) {
            const int64_t r = rbeg + kk;
            const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
            int cnt = 0;
            if (y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2) {
                const unsigned* row = reinterpret_cast<const unsigned*>(tb + kk * nx);
                for (int w0 = 0; w0 < wpr; w0 += 32) {
                    unsigned mine = 0u;
#pragma unroll 4
                    for (int u = 0; u < 32 && w0 + u < wpr; ++u) {
                        const int w = w0 + u;
                        const int x = 32 * w + lane;
                        const unsigned v = x < nx ? row[x] : 0u;
                        unsigned b = __ballot_sync(0xffffffffu, iface_bits(v));
                        b &= (w == 0 ? ~1u : ~0u) & (w == lastw ? lastmask : ~0u);
                        cnt += __popc(b);
                        mine = lane == u ? b : mine;
                    }
                    if (bits && w0 + lane < wpr) bits[r * wpr + w0 + lane] = mine;
                }
            }
            if (lane == 0) rc[kk] = cnt;
        }
        __syncthreads();                              // stage s and rc[] complete
        if (threadIdx.x == 0 && k + CT_STAGES < nmine) {
            const int64_t tn = first + (k + CT_STAGES) * step;
            issue_tile(sm, s, phi, nx, tn * R, tile_rows_of(tn));
        }
        if (warp == 0) {
            // exclusive scan of the nr row counts: each lane sums a run of rows
            const int per = (nr + 31) >> 5;
            const int k0 = lane * per, k1 = min(k0 + per, nr);
            int sum = 0;
            for (int q = k0; q < k1; ++q) sum += rc[q];
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (row_off) {
                int run = incl - sum;
                for (int q = k0; q < k1; ++q) {
                    row_off[rbeg + q] = run;
                    run += rc[q];
                }
            }
            if (lane == 31) tile_count[t] = incl;
        }
    }
    if (!ok && threadIdx.x == 0) {
        // tiles k .. of this block were not counted; their copies (at most
        // CT_STAGES, tiles k .. k + CT_STAGES - 1) may still be in flight
        for (int64_t j = k; j < nmine; ++j) tile_count[first + j * step] = CT_FAILED;
        for (int64_t j = k; j < nmine && j < k + CT_STAGES; ++j)
            mbar_wait(smem_addr(&sm.bar[j % CT_STAGES]), (uint32_t)((j / CT_STAGES) & 1));
    }
}

// Pass 2: exclusive scan of ntiles ints by one block of 1024 threads (four
// consecutive entries per thread and round); total -> *d_count.
__global__ void __launch_bounds__(1024)
k_compact_scan(int* __restrict__ tile_count, int64_t ntiles, int64_t* __restrict__ d_count) {
    __shared__ long long wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // a tile that pass 1 could not count (CT_FAILED) voids the list: every
    // offset becomes -1 and so does the count
    int neg = 0;
    for (int64_t i = threadIdx.x; i < ntiles; i += 1024) neg |= tile_count[i] < 0;
    if (__syncthreads_or(neg)) {
        for (int64_t i = threadIdx.x; i < ntiles; i += 1024) tile_count[i] = -1;
        if (threadIdx.x == 0) *d_count = -1;
        return;
    }
    long long carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += 4096) {
        const int64_t i0 = b0 + 4 * (int64_t)threadIdx.x;
        int v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = i0 + j < ntiles ? tile_count[i0 + j] : 0;
        const long long own = (long long)v[0] + v[1] + v[2] + v[3];
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
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i0 + j < ntiles) tile_count[i0 + j] = (int)run;
            run += v[j];
        }
        carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_count = carry;
}

// Pass 3: each warp takes its rows' interface bits (from pass 1's bit array,
// or recomputed from the field when none was kept), the block scans the row
// counts, and every warp writes its rows' indices at the row offsets, in
// ascending cell order.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_write(const float* __restrict__ phi, int nx, int ny, int nz, int R, int64_t rows,
                const int* __restrict__ tile_offset, const unsigned* __restrict__ bits,
                const int* __restrict__ row_count, int32_t* __restrict__ idx, int64_t cap, int vec,
                int64_t* __restrict__ d_count) {
    __shared__ unsigned bal[CT_MAX_WORDS];
    __shared__ int rowoff[CT_MAX_ROWS + 1];
    __shared__ int rowcnt[CT_MAX_ROWS];
    __shared__ long long s_base[CT_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    // with pass 1's row counts the rows need not be recounted here, and their
    // bits are read from global memory only for the non-empty rows
    const bool in_smem = !row_count && (int64_t)nr * wpr <= CT_MAX_WORDS;
    if (row_count) {
        for (int k = threadIdx.x; k < nr; k += CT_THREADS) rowoff[k] = rowcnt[k] = __ldg(row_count + rbeg + k);
    }
    for (int k = warp; k < (row_count ? 0 : nr); k += CT_WARPS) {
        const int64_t r = rbeg + k;
        int cnt = 0;
        if (bits) {
            const unsigned* rb = bits + r * wpr;
            for (int w = lane; w < wpr; w += 32) {
                const unsigned b = __ldg(rb + w);
                cnt += __popc(b);
                if (in_smem) bal[k * wpr + w] = b;
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
        } else {
            const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
            if (y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2) {
                cnt = row_bits(phi + r * nx, nx, vec != 0, [&](int w, unsigned b) {
                    if (in_smem) bal[k * wpr + w] = b;
                });
            } else if (in_smem) {
                for (int w = lane; w < wpr; w += 32) bal[k * wpr + w] = 0u;
            }
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
                } else if (bits) {
                    b = __ldg(bits + r * wpr + w);
                } else {
                    // recompute this word (rare: tiles of very long rows)
                    const float* row = phi + r * nx;
                    const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
                    if (y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2)
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
}

// Pass 3 with pass 1's interface bits and row offsets: no field reads, no
// row scan.  The block's base is the sum of the counts of the tiles before
// its own (fused: few tiles, every block sums them, the last block writes the
// total) or the exclusive offset written by the scan launch (then the tile's
// count is the next offset, or the total, minus its own).  Each warp takes
// rows w, w + 8, ...; a non-empty row is written one 32-cell word per lane:
// a warp prefix of the word popcounts gives each lane its first slot, and
// the lane writes its word's cells in ascending order.
__global__ void __launch_bounds__(CT_THREADS)
k_compact_emit(int nx, int R, int64_t rows, const int* __restrict__ tiles,
               const unsigned* __restrict__ bits, const int* __restrict__ row_off,
               int32_t* __restrict__ idx, int64_t cap, int fused, int64_t* __restrict__ d_count) {
    __shared__ long long s_part[CT_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = blockIdx.x;
    long long base;
    int tcount;
    if (fused) {
        // the counts of the tiles before this one (t <= 4096): four int4
        // loads per thread at most, all issued before any is summed
        long long part = 0;
        int neg = 0;
        const int4* t4 = reinterpret_cast<const int4*>(tiles);
        const int n4 = t >> 2;
        int4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = threadIdx.x + u * CT_THREADS;
            v[u] = q < n4 ? __ldg(t4 + q) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            part += (long long)v[u].x + v[u].y + v[u].z + v[u].w;
            neg |= (v[u].x | v[u].y | v[u].z | v[u].w) < 0;
        }
        if (threadIdx.x < (t & 3)) {
            const int c = __ldg(tiles + 4 * n4 + threadIdx.x);
            part += c;
            neg |= c < 0;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_part[warp] = part;
        tcount = __ldg(tiles + t);
        neg = __syncthreads_or(neg | (tcount < 0));
        base = 0;
#pragma unroll
        for (int w = 0; w < CT_WARPS; ++w) base += s_part[w];
        if (t == (int)gridDim.x - 1 && threadIdx.x == 0) *d_count = neg ? -1 : base + tcount;
        if (neg) return;                            // a tile before (or this one) was not counted
    } else {
        base = __ldg(tiles + t);
        if (base < 0) return;                       // the scan found an uncounted tile
        const long long next = t + 1 < (int)gridDim.x ? (long long)__ldg(tiles + t + 1) : *d_count;
        tcount = (int)(next - base);
    }
    const int64_t rbeg = (int64_t)t * R;
    const int nr = (int)(rbeg + R < rows ? R : rows - rbeg);
    const int wpr = (nx + 31) >> 5;
    for (int k = warp; k < nr; k += CT_WARPS) {
        const int off = __ldg(row_off + rbeg + k);
        const int end = k + 1 < nr ? __ldg(row_off + rbeg + k + 1) : tcount;
        if (end == off) continue;                   // most rows hold no interface cell
        const int64_t r = rbeg + k;
        int64_t pos = base + off;
        for (int w0 = 0; w0 < wpr; w0 += 32) {
            const int w = w0 + lane;
            unsigned b = w < wpr ? __ldg(bits + r * wpr + w) : 0u;
            const int c = __popc(b);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
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
}

// Grid of the streaming count pass: resident blocks (shared memory allows
// two per SM) times the SMs, at most one block per tile; 0 when the kernel
// cannot be given its shared memory.  The attribute is set once per device.
static int count_stream_grid(int64_t nt) {
    static std::mutex mu;
    static int per_sm[256] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (per_sm[dev] == 0) {
            const void* k = reinterpret_cast<const void*>(&k_compact_count_stream);
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(CountSmem)) != cudaSuccess) {
                cudaGetLastError();
                per_sm[dev] = -1;
            } else {
                int b = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, CT_THREADS, sizeof(CountSmem)) !=
                        cudaSuccess || b < 1) {
                    cudaGetLastError();
                    b = -1;
                }
                per_sm[dev] = b;
            }
        }
        if (per_sm[dev] < 0) return 0;
    }
    const int64_t g = (int64_t)sm_count() * per_sm[dev];
    return (int)(g < nt ? g : nt);
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
            // row counts: one int per row of >= 32 cells, at most arg / 32 + 1
            const int64_t t = (arg + plic::CT_TILE - 1) / plic::CT_TILE * 2 + 1;
            const size_t a = ((size_t)t * sizeof(int) + 255) / 256 * 256;
            const size_t b = ((size_t)(arg / 16 + 1) * sizeof(unsigned) + 255) / 256 * 256;
            const size_t c = ((size_t)(arg / 32 + 1) * sizeof(int) + 255) / 256 * 256;
            return a + b + c;
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
    int* rowc = nullptr;
    if (nx >= 32 && tile_bytes + bits_bytes + (size_t)rows * sizeof(int) <= ws_bytes) {
        bits = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(workspace) + tile_bytes);
        rowc = reinterpret_cast<int*>(reinterpret_cast<char*>(workspace) + tile_bytes + bits_bytes);
    }
    const int vec = (nx % 4 == 0) && aligned(phi, 16);
    // the streaming count pass needs whole rows of 16-byte multiples that fit
    // one shared-memory stage, and the bits and row offsets in the workspace
    const int stream_blocks = (vec && nx <= CT_TILE && bits) ? count_stream_grid(nt) : 0;
    if (stream_blocks > 0) {
        k_compact_count_stream<<<(unsigned)stream_blocks, CT_THREADS, sizeof(CountSmem), s>>>(
            phi, nx, ny, nz, R, rows, nt, tiles, bits, rowc);
    } else {
        k_compact_count<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles, bits,
                                                            rowc);
    }
    // up to CT_FUSED_SCAN_TILES tiles each block of pass 3 sums the counts of
    // the tiles before it (at most that many L2 reads per block); beyond, one
    // block scans them first
    const bool fused = nt <= CT_FUSED_SCAN_TILES;
    if (!fused) k_compact_scan<<<1, 1024, 0, s>>>(tiles, nt, d_count);
    if (bits) {
        k_compact_emit<<<(unsigned)nt, CT_THREADS, 0, s>>>(nx, R, rows, tiles, bits, rowc, idx,
                                                           idx_capacity, fused ? 1 : 0, d_count);
    } else {
        k_compact_write<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles, nullptr,
                                                            nullptr, idx, idx_capacity, vec,
                                                            fused ? d_count : nullptr);
    }
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
    k_compact_count<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles, nullptr,
                                                        nullptr);
    const bool fused = nt <= CT_FUSED_SCAN_TILES;
    if (!fused) k_compact_scan<<<1, 1024, 0, s>>>(tiles, nt, d_count);
    k_compact_write<<<(unsigned)nt, CT_THREADS, 0, s>>>(phi, nx, ny, nz, R, rows, tiles, nullptr,
                                                        nullptr, idx, idx_capacity, vec,
                                                        fused ? d_count : nullptr);
    return check_launch("vof_interface_compact_noalloc");
}
