// vof_curvature_coop.cuh -- the curvature step (Sec. 4.2, Appendix B) with
// eight lanes per interface cell.
//
// A warp handles a batch of up to 32 list entries in eight rounds of four
// cells (one 8-lane group per cell), then solves the 32 normal-equation
// systems one per lane:
//   group phase, per cell:
//     - each lane loads 3-4 of the 27 stencil values; the Parker-Youngs sums
//       (Eq. 38) and the 27-bit interface mask are reduced over the group;
//     - every lane forms the normal and the frame (Sec. 4.2);
//     - the centre and the m interface neighbours (Eq. 36) are dealt out to
//       the 8 lanes in ascending order (lane g takes the g-th, (g+8)-th, ...
//       entry of the list), so the PLIC solves are dense: ceil((m+1)/8) per
//       lane instead of 26 mostly idle loop trips per cell;
//     - each lane accumulates its points into partial normal equations
//       (20 sums), reduce-scattered over the group with 18 shuffles, and the
//       totals go to shared memory;
//   lane phase: lane t takes cell t of the batch, factorises its 5x5 system
//   (the fit precision of the flags) and writes kappa (Eq. 42).
#pragma once
#include "vof_curvature.cuh"

namespace plic {

constexpr int CO_BATCH = 32;          // cells per warp batch
constexpr int TPC_THREADS = 128;      // block of the one-thread-per-cell kernels
constexpr int CO_VALS = 24;           // per-cell smem record: M (15), b (5), m, pad

// Source of one list entry: its field, cell index and output slot.
struct CoCell {
    const float* phi;
    int nx;
    int64_t nxy;
    int64_t c;
    float* out;
    bool valid;
};

// Stencil offset of D3Q27 entry i.
__device__ __forceinline__ int64_t st_off(int i, int nx, int64_t nxy) {
    int ex, ey, ez;
    e_of(i, ex, ey, ez);
    return ex + (int64_t)ey * nx + (int64_t)ez * nxy;
}

// Position of the (p+1)-th set bit of `list` (p < popc(list)), by binary
// search on prefix popcounts.
__device__ __forceinline__ int nth_set_bit(unsigned list, int p) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int hi = lo + step;
        const unsigned low = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
        if (__popc(list & low) <= p) lo = hi;
    }
    return lo;
}

// Group reduce-scatter of 20 partial sums over the 8 lanes of a group: after
// the call, lane g (0..7) holds the totals of the values listed by
// co_value_of(g, j) for j < co_count(g).
__device__ __forceinline__ void group_reduce_scatter(float v[20], int g, float out[3]) {
    // step 1 (xor 4): keep values [0,10) if bit 2 of g is clear, else [10,20)
    float a[10];
    const bool hi4 = (g & 4) != 0;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const float keep = hi4 ? v[10 + j] : v[j];
        const float send = hi4 ? v[j] : v[10 + j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    // step 2 (xor 2): keep [0,5) or [5,10) of the 10
    float b[5];
    const bool hi2 = (g & 2) != 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const float keep = hi2 ? a[5 + j] : a[j];
        const float send = hi2 ? a[j] : a[5 + j];
        b[j] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    // step 3 (xor 1): keep 3 ([0,3)) or 2 ([3,5)) of the 5
    const bool hi1 = (g & 1) != 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float keep = hi1 ? (j < 2 ? b[3 + j] : 0.0f) : b[j];
        const float send = hi1 ? b[j] : (j < 2 ? b[3 + j] : 0.0f);
        out[j] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
}

// Index (0..19) of the j-th total held by lane g after group_reduce_scatter.
__device__ __forceinline__ int co_value_of(int g, int j) {
    return ((g & 4) ? 10 : 0) + ((g & 2) ? 5 : 0) + ((g & 1) ? 3 : 0) + j;
}
__device__ __forceinline__ int co_count(int g) { return (g & 1) ? 2 : 3; }

// Group phase for one cell (all 32 lanes call it; `cell` is this group's).
// Writes the cell's normal equations to rec[0..20] (M packed upper, b, m) or
// m = -1 when the normal is undefined.
template <int METHOD>
__device__ __forceinline__ void co_group_cell(const CoCell& cell, int g, uint32_t flags,
                                              float* rec) {
    const bool on = cell.valid;
    const bool cm = (flags & PLIC_FLAG_NORMAL_CM) != 0;
    // 1. stencil entries i = g, g+8, g+16, g+24 (i < 27) and the PY (or CM)
    //    partial sums
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    unsigned mask = 0u;
    float phi0 = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = g + 8 * j;
        if (i < 27 && on) {
            int ex, ey, ez;
            e_of(i, ex, ey, ez);
            const float v = __ldg(cell.phi + cell.c + ex + (int64_t)ey * cell.nx + (int64_t)ez * cell.nxy);
            const int e2 = ex * ex + ey * ey + ez * ez;
            const float w = cm ? 1.0f : (e2 == 1 ? 4.0f : (e2 == 2 ? 2.0f : 1.0f));
            gx = fmaf(w * ex, v, gx);
            gy = fmaf(w * ey, v, gy);
            gz = fmaf(w * ez, v, gz);
            if (i == 0) phi0 = v;
            else if (v > 0.0f && v < 1.0f) mask |= 1u << i;
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    }
    phi0 = __shfl_sync(0xffffffffu, phi0, (threadIdx.x & 31) & ~7);
    // 2. normal and frame
    const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
    const bool ok = on && gl > 0.0f;
    const float inv = ok ? -1.0f / gl : 0.0f;
    const float nx_ = gx * inv, ny_ = gy * inv, nz_ = gz * inv;
    float rx = 0.56270900f, ry = 0.32704452f, rz = 0.75921047f;
    float byx = ny_ * rz - nz_ * ry, byy = nz_ * rx - nx_ * rz, byz = nx_ * ry - ny_ * rx;
    float bl = byx * byx + byy * byy + byz * byz;
    if (!(bl > 1e-12f)) {
        rx = 0.32704452f; ry = 0.75921047f; rz = 0.56270900f;
        byx = ny_ * rz - nz_ * ry; byy = nz_ * rx - nx_ * rz; byz = nx_ * ry - ny_ * rx;
        bl = byx * byx + byy * byy + byz * byz;
    }
    const float ib = ok ? rsqrtf(bl) : 0.0f;
    byx *= ib; byy *= ib; byz *= ib;
    const float bxx = byy * nz_ - byz * ny_, bxy = byz * nx_ - byx * nz_, bxz = byx * ny_ - byy * nx_;
    // 3. PLIC offsets of the list [centre, interface neighbours...], dealt out
    const unsigned list = mask | 1u;
    const int cnt = __popc(list);
    CellPlic<METHOD> pl;
    pl.prepare(ok ? nx_ : 1.0f, ok ? ny_ : 0.0f, ok ? nz_ : 0.0f);
    const bool centroid = (flags & PLIC_FLAG_POINT_CENTROID) != 0;
    int ent[4];
    float d0s[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = g + 8 * j;
        ent[j] = -1;
        d0s[j] = 0.0f;
        if (ok && p < cnt) {
            const int i = nth_set_bit(list, p);
            ent[j] = i;
            const float v = i == 0 ? phi0 : __ldg(cell.phi + cell.c + st_off(i, cell.nx, cell.nxy));
            d0s[j] = pl.offset(v);
        }
    }
    // the centre is entry 0 of the list, held by lane g = 0 of the group
    const int leader = (threadIdx.x & 31) & ~7;
    const float d00 = __shfl_sync(0xffffffffu, d0s[0], leader);
    float c0x = 0.0f, c0y = 0.0f, c0z = 0.0f;
    if (centroid) {
        float A;
        if (g == 0 && ok) area_centroid<float>(nx_, ny_, nz_, d00, A, c0x, c0y, c0z);
        c0x = __shfl_sync(0xffffffffu, c0x, leader);
        c0y = __shfl_sync(0xffffffffu, c0y, leader);
        c0z = __shfl_sync(0xffffffffu, c0z, leader);
    }
    // 4. points and partial normal equations
    float acc[20];
#pragma unroll
    for (int q = 0; q < 20; ++q) acc[q] = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = ent[j];
        if (i > 0) {
            int ex, ey, ez;
            e_of(i, ex, ey, ez);
            float qx = (float)ex, qy = (float)ey, qz = (float)ez, z;
            if (centroid) {
                float A, cx, cy, cz;
                area_centroid<float>(nx_, ny_, nz_, d0s[j], A, cx, cy, cz);
                qx += cx - c0x; qy += cy - c0y; qz += cz - c0z;
                z = qx * nx_ + qy * ny_ + qz * nz_;
            } else {
                z = qx * nx_ + qy * ny_ + qz * nz_ + (d0s[j] - d00);
            }
            const float x = qx * bxx + qy * bxy + qz * bxz;
            const float y = qx * byx + qy * byy + qz * byz;
            const float Q[5] = {x * x, y * y, x * y, x, y};
#pragma unroll
            for (int a = 0; a < 5; ++a) {
#pragma unroll
                for (int b = a; b < 5; ++b) acc[uidx(a, b)] = fmaf(Q[a], Q[b], acc[uidx(a, b)]);
                acc[15 + a] = fmaf(z, Q[a], acc[15 + a]);
            }
        }
    }
    float tot[3];
    group_reduce_scatter(acc, g, tot);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (j < co_count(g)) rec[co_value_of(g, j)] = tot[j];
    if (g == 0) rec[20] = ok ? (float)(cnt - 1) : -1.0f;
}

// Lane phase: solve one cell's record and return kappa (Eq. 42 sign per flags).
// FIT_AUTO factorises in FP32 and repeats the factorisation in FP64 only for
// cells whose normal matrix looks ill-conditioned (smallest pivot below 1e-2
// of the largest, or a fit dimension reduced by the FP32 pivots): FP64 where
// the conditioning asks for it, the FP32 pipes everywhere else.
template <int FIT>
__device__ __forceinline__ float co_solve(const float* rec, uint32_t flags) {
    const int m = (int)rec[20];
    if (m <= 0) return 0.0f;
    float xs[5];
    int dim;
    if constexpr (FIT == FIT_AUTO) {
        Ldlt<FIT_FP32> f;
        f.factor(rec, m);
        const int want = m < 5 ? m : 5;
        float dmin = 3.4e38f, dmax = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if (j < f.dim) { dmin = fminf(dmin, f.D[j]); dmax = fmaxf(dmax, f.D[j]); }
        if (f.dim == want && dmin > 1e-2f * dmax) {
            f.solve(rec + 15, xs);
            dim = f.dim;
        } else {
            dim = fit_solve<FIT_FP64>(rec, rec + 15, m, xs);
        }
    } else {
        dim = fit_solve<FIT>(rec, rec + 15, m, xs);
    }
    if (dim == 0) return 0.0f;
    const float k = paraboloid_kappa(xs);
    return (flags & PLIC_FLAG_KAPPA_PAPER_SIGN) ? k : -k;
}

// One warp batch of `batch` cells (a multiple of 4, at most CO_BATCH):
// `fetch(slot)` gives the CoCell of batch slot 0..batch-1 (with valid == false
// past the end of the list).  `smem` holds CO_BATCH * CO_VALS floats for this
// warp.  The stored value is scale * kappa (scale = 1 for the curvature
// itself, 2 sigma for the Young-Laplace pressure).
template <int METHOD, int FIT, typename Fetch>
__device__ __forceinline__ void co_warp_batch(Fetch fetch, int batch, uint32_t flags, float scale,
                                              float* smem) {
    const int lane = threadIdx.x & 31;
    const int g = lane & 7, grp = lane >> 3;
#pragma unroll 1
    for (int round = 0; round < batch / 4; ++round) {
        const int slot = round * 4 + grp;
        const CoCell cell = fetch(slot);
        co_group_cell<METHOD>(cell, g, flags, smem + slot * CO_VALS);
    }
    __syncwarp();
    const CoCell mine = fetch(lane);          // every lane: fetch may shuffle
    if (lane < batch && mine.valid) *mine.out = scale * co_solve<FIT>(smem + lane * CO_VALS, flags);
    __syncwarp();
}

// The one-thread-per-cell kernels (vof_curvature_tpc.cu): k_vof_curvature_tpc
// (single field; arguments as k_vof_curvature without `batch`) or
// k_vof_curvature_batched_tpc (arguments as k_vof_curvature_batched) for a
// method and fit mode; nullptr for an invalid pair.
const void* select_tpc(bool batched, plic_method m, int fit);

}  // namespace plic
