// vof_curvature_tpc.cu -- the curvature step (Sec. 4.2, Appendix B) with one
// thread per interface cell, for long interface lists.
//
// The eight-lane layout of vof_curvature_coop.cuh shortens the dependent
// chain of a cell (it wins when the list is too short to fill the GPU), but
// every lane of a group repeats the normal, the frame and the per-normal
// solver constants, and the group reductions add shuffles.  With enough
// cells to fill every warp slot many times over (the batched workload), the
// instruction count decides instead, and one thread per cell does each step
// once:
//   - the 27 stencil values with compile-time offsets, the Parker-Youngs (or
//     centre-of-mass) sums and the interface mask in registers;
//   - normal, frame, centre offset d0(phi_0, n) and the per-normal constants
//     of the solver once;
//   - a loop over the set bits of the mask only (the interface neighbours of
//     Eq. 36), two neighbours per trip: their values are re-read (L1 hits: the
//     stencil was just loaded), their offsets solved together (paired FP32
//     instructions for the optimised SZ solution), their points accumulated
//     into the normal equations in registers;
//   - the 5x5 solve of the fit precision and Eq. 42, as in the lane phase of
//     the eight-lane layout (co_solve).
// The results equal those of the eight-lane layout up to the summation order
// of the stencil sums and of the normal equations.
#include "host_common.h"
#include "plic_pair.cuh"
#include "vof_curvature_coop.cuh"

namespace plic {

// Offsets d0(V0, n) of two neighbours of a cell (both with the centre normal
// of `pl`): for the optimised SZ solution, CellPlic<M_SZ_OPT>::offset on the
// paired FP32 instructions (two neighbours per instruction; the arcsine and
// the case-(1) cube root of the paired path); other methods solve one after
// the other.
template <int METHOD>
__device__ __forceinline__ p2::f2 offset_two(const CellPlic<METHOD>& pl, p2::f2 V0) {
    return make_float2(pl.offset(V0.x), pl.offset(V0.y));
}
template <>
__device__ __forceinline__ p2::f2 offset_two<M_SZ_OPT>(const CellPlic<M_SZ_OPT>& P, p2::f2 V0) {
    using namespace p2;
    const f2 V = make_float2(fminf(V0.x, 1.0f - V0.x), fminf(V0.y, 1.0f - V0.y));
    const b2 c5 = {V.x >= P.V5, V.y >= P.V5};
    const b2 c1 = lt(V, mk(P.V1)), c2 = lt(V, mk(P.V2)), c3 = lt(V, mk(P.V3));
    const f2 d5 = fma(mk(P.m3), V, mk(0.5f * P.n12));
    const f2 d2 = mul(mk(0.5f), add(mk(P.m1), sqrtp(fmax0(fma(mk(P.k2a), V, mk(-P.k2b))))));
    const f2 d1 = mul(mk(P.cb1), cbrt_(V));
    const f2 x = sel(c3, fma(mk(-2.0f * P.m3), V, mk(P.n12)), fma(mk(-2.0f), V, mk(1.0f)));
    f2 arg = mul(x, sel(c3, mk(P.s3), mk(P.s4)));
    arg = make_float2(fminf(fmaxf(arg.x, 0.0f), 1.0f), fminf(fmaxf(arg.y, 0.0f), 1.0f));
    const f2 t = sel(c3, mk(P.t3), mk(P.t4)), c = sel(c3, mk(P.n12), mk(0.5f));
    const f2 th = mul(mk(0.33333333333333333f), asin01(arg));
    f2 d = fma(mul(mk(-2.0f), t), make_float2(__sinf(th.x), __sinf(th.y)), c);
    // Newton polish of the trigonometric root (cases 3/4)
    const f2 e2 = sub(d, mk(P.m2)), e3 = fmax0(sub(d, mk(P.m3)));
    const f2 e22 = mul(e2, e2), e33 = mul(e3, e3);
    const f2 cub = fma(e22, e2, mul(e33, e3));
    f2 g = fma(mul(mk(3.0f), d), sub(d, mk(P.m1)), mk(P.m1 * P.m1));
    g = fma(make_float2(-cub.x, -cub.y), mk(P.inv1), g);
    g = fma(mk(-P.k6), V, g);
    f2 gp = fma(mk(6.0f), d, mk(-3.0f * P.m1));
    gp = fma(mul(mk(-3.0f), add(e22, e33)), mk(P.inv1), gp);
    d = sub(d, mul(g, rcp(gp)));
    d = sel(c2, d2, d);
    d = sel(c1, d1, d);
    d = sel(c5, d5, d);
    const f2 h = mul(mk(P.L), sub(mk(0.5f), d));
    return make_float2(copysignf(h.x, V0.x - 0.5f), copysignf(h.y, V0.y - 0.5f));
}

// kappa (sign per flags) of interface cell c of a field, one thread.
template <int METHOD, int FIT>
__device__ __forceinline__ float tpc_kappa(const float* __restrict__ phi, int nx, int64_t nxy,
                                           int64_t c, uint32_t flags, const E27Shared& tab) {
    const bool cm = (flags & PLIC_FLAG_NORMAL_CM) != 0;
    const float* p0 = phi + c;
    // offsets within the field in 32 bits (list entries are int32 cell indices)
    const int nxy32 = (int)nxy;
    // 1. stencil: normal sums (Eq. 38 weights or all 1) and interface mask
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    unsigned mask = 0u;
    const float phi0 = __ldg(p0);
    for_e27<1>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int p = E27Table::v[i];
        constexpr int ex = p % 3 - 1, ey = (p / 3) % 3 - 1, ez = p / 9 - 1;
        constexpr int e2 = ex * ex + ey * ey + ez * ez;
        constexpr float wpy = e2 == 1 ? 4.0f : (e2 == 2 ? 2.0f : 1.0f);
        const float v = __ldg(p0 + (ex + ey * nx + ez * nxy32));
        const float w = cm ? 1.0f : wpy;
        if (ex != 0) gx = fmaf(w * (float)ex, v, gx);
        if (ey != 0) gy = fmaf(w * (float)ey, v, gy);
        if (ez != 0) gz = fmaf(w * (float)ez, v, gz);
        // 0 < v < 1 as one unsigned compare of the bits: the positive floats
        // below 1.0f are the patterns 1 .. 0x3F7FFFFF
        if (__float_as_uint(v) - 1u < 0x3F7FFFFFu) mask |= 1u << i;
    });
    // 2. normal and frame (Sec. 4.2)
    const float gl2 = gx * gx + gy * gy + gz * gz;
    if (!(gl2 > 0.0f)) return 0.0f;                    // undefined normal: kappa = 0
    const float inv = -rsqrtf(gl2);
    const float nx_ = gx * inv, ny_ = gy * inv, nz_ = gz * inv;
    float rx = 0.56270900f, ry = 0.32704452f, rz = 0.75921047f;
    float byx = ny_ * rz - nz_ * ry, byy = nz_ * rx - nx_ * rz, byz = nx_ * ry - ny_ * rx;
    float bl = byx * byx + byy * byy + byz * byz;
    if (!(bl > 1e-12f)) {
        rx = 0.32704452f; ry = 0.75921047f; rz = 0.56270900f;
        byx = ny_ * rz - nz_ * ry; byy = nz_ * rx - nx_ * rz; byz = nx_ * ry - ny_ * rx;
        bl = byx * byx + byy * byy + byz * byz;
    }
    const float ib = rsqrtf(bl);
    byx *= ib; byy *= ib; byz *= ib;
    const float bxx = byy * nz_ - byz * ny_, bxy = byz * nx_ - byx * nz_, bxz = byx * ny_ - byy * nx_;
    // 3. centre offset and, for centroid points, the centre centroid
    CellPlic<METHOD> pl;
    pl.prepare(nx_, ny_, nz_);
    const float d00 = pl.offset(phi0);
    const bool centroid = (flags & PLIC_FLAG_POINT_CENTROID) != 0;
    float c0x = 0.0f, c0y = 0.0f, c0z = 0.0f;
    if (centroid) {
        float A;
        area_centroid<float>(nx_, ny_, nz_, d00, A, c0x, c0y, c0z);
    }
    // 4. interface neighbours (Eq. 36): points and normal equations
    float rec[21];
#pragma unroll
    for (int q = 0; q < 20; ++q) rec[q] = 0.0f;
    rec[20] = (float)__popc(mask);
    // two neighbours per trip (in ascending order; an odd last one pairs with
    // a zero point that adds nothing)
    unsigned list = mask;
#pragma unroll 1
    while (list) {
        const int i1 = __ffs(list) - 1;
        list &= list - 1u;
        const bool two = list != 0u;
        const int i2 = two ? __ffs(list) - 1 : i1;
        list &= list - 1u;                          // no-op on an empty list
        const int4 e1 = tab.ei[i1], e2 = tab.ei[i2];
        const float4 f1 = tab.ef[i1], f2 = tab.ef[i2];
        const float v1 = __ldg(p0 + (e1.x + e1.y * nx + e1.z * nxy32));
        const float v2 = __ldg(p0 + (e2.x + e2.y * nx + e2.z * nxy32));
        const p2::f2 d0i = offset_two<METHOD>(pl, make_float2(v1, v2));
        float qx[2] = {f1.x, f2.x}, qy[2] = {f1.y, f2.y};
        float qz[2] = {f1.z, f2.z}, z[2];
        const float dd[2] = {d0i.x, d0i.y};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (centroid) {
                float A, cx, cy, cz;
                area_centroid<float>(nx_, ny_, nz_, dd[j], A, cx, cy, cz);
                qx[j] += cx - c0x; qy[j] += cy - c0y; qz[j] += cz - c0z;
                z[j] = qx[j] * nx_ + qy[j] * ny_ + qz[j] * nz_;
            } else {
                z[j] = qx[j] * nx_ + qy[j] * ny_ + qz[j] * nz_ + (dd[j] - d00);
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float w = (j == 0 || two) ? 1.0f : 0.0f;
            const float x = w * (qx[j] * bxx + qy[j] * bxy + qz[j] * bxz);
            const float y = w * (qx[j] * byx + qy[j] * byy + qz[j] * byz);
            const float zz = w * z[j];
            const float Q[5] = {x * x, y * y, x * y, x, y};
            // the 12 distinct moments of the normal matrix: the entries
            // (xy, xy), (xy, x), (xy, y) equal (x^2, y^2), (x^2, y), (y^2, x)
            // and are copied after the loop
#pragma unroll
            for (int a = 0; a < 5; ++a) {
#pragma unroll
                for (int b = a; b < 5; ++b)
                    if (a != 2) rec[uidx(a, b)] = fmaf(Q[a], Q[b], rec[uidx(a, b)]);
                rec[15 + a] = fmaf(zz, Q[a], rec[15 + a]);
            }
        }
    }
    rec[uidx(2, 2)] = rec[uidx(0, 1)];
    rec[uidx(2, 3)] = rec[uidx(0, 4)];
    rec[uidx(2, 4)] = rec[uidx(1, 3)];
    // 5. fit and Eq. 42
    return co_solve<FIT>(rec, flags);
}

// Single field: thread per list entry, grid-stride.
template <int METHOD, int FIT>
__global__ void __launch_bounds__(TPC_THREADS)
k_vof_curvature_tpc(const float* __restrict__ phi, int nx, int ny, const int32_t* __restrict__ idx,
                    int64_t n, const int64_t* __restrict__ d_n, float* __restrict__ kappa,
                    uint32_t flags, float scale) {
    pdl_wait();                  // a kernel before it (the compaction) has completed
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    __shared__ E27Shared tab;
    tab.fill();
    const int64_t nxy = (int64_t)nx * ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lim;
         k += (int64_t)gridDim.x * blockDim.x)
        kappa[k] = scale * tpc_kappa<METHOD, FIT>(phi, nx, nxy, (int64_t)__ldg(idx + k), flags, tab);
    pdl_trigger();
}

// Persistent batched kernel: each warp claims tickets of `chunk` cells (a
// multiple of 32) of the concatenated lists and gives one cell to each lane.
template <int METHOD, int FIT>
__global__ void __launch_bounds__(TPC_THREADS)
k_vof_curvature_batched_tpc(const vof_field* __restrict__ fields, const int64_t* __restrict__ prefix,
                            int n_fields, int64_t total, int chunk,
                            unsigned long long* __restrict__ ticket, uint32_t flags) {
    const int lane = threadIdx.x & 31;
    __shared__ E27Shared tab;
    tab.fill();
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ticket, (unsigned long long)chunk);
        const int64_t start = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        if (start >= total) break;
        const int64_t end = start + chunk < total ? start + chunk : total;
        // the field of the ticket's first cell, found once per ticket (lane 0,
        // binary search over the list prefix); each lane then steps forward
        // from it to its own cell's field (the lists are long: rarely a step)
        int f0 = 0;
        if (lane == 0) {
            int lo = 0, hi = n_fields - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(prefix + mid) <= start) lo = mid; else hi = mid - 1;
            }
            f0 = lo;
        }
        f0 = __shfl_sync(0xffffffffu, f0, 0);
        for (int64_t gi = start + lane; gi < end; gi += 32) {
            int lo = f0;
            while (lo + 1 < n_fields && __ldg(prefix + lo + 1) <= gi) ++lo;
            const int64_t kk = gi - __ldg(prefix + lo);
            const vof_field& F = fields[lo];
            const float k = tpc_kappa<METHOD, FIT>(F.phi, F.nx, (int64_t)F.nx * F.ny,
                                                   (int64_t)__ldg(F.idx + kk), flags, tab);
            F.kappa[kk] = k;
        }
    }
}

template <int METHOD>
static const void* pick_tpc(bool batched, int fit) {
#define PLIC_TPC(K) \
    {reinterpret_cast<const void*>(&K<METHOD, FIT_FP64>), reinterpret_cast<const void*>(&K<METHOD, FIT_FP32>), \
     reinterpret_cast<const void*>(&K<METHOD, FIT_DF32>), reinterpret_cast<const void*>(&K<METHOD, FIT_AUTO>)}
    static const void* single[4] = PLIC_TPC(k_vof_curvature_tpc);
    static const void* many[4] = PLIC_TPC(k_vof_curvature_batched_tpc);
#undef PLIC_TPC
    return batched ? many[fit] : single[fit];
}

const void* select_tpc(bool batched, plic_method m, int fit) {
    if (fit < 0 || fit > 3) return nullptr;
    switch (m) {
        case PLIC_ANALYTIC: return pick_tpc<M_ANALYTIC>(batched, fit);
        case PLIC_SZ_ORIG: return pick_tpc<M_SZ_ORIG>(batched, fit);
        case PLIC_SZ_OPT: return pick_tpc<M_SZ_OPT>(batched, fit);
        case PLIC_NEWTON: return pick_tpc<M_NEWTON>(batched, fit);
        case PLIC_NESTED: return pick_tpc<M_NESTED>(batched, fit);
    }
    return nullptr;
}

}  // namespace plic
