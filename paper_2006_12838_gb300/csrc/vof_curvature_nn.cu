// vof_curvature_nn.cu -- interface normals of listed cells (vof_normal) and
// the neighbour-normal curvature variant that Sec. 4.2 discusses and
// compares in its curvature-error figure.
//
// Variant: in Eq. 36 every interface neighbour is placed with the centre
// normal n.  Here neighbour i gets its own normal n_i from its own 3^3
// stencil (so the curvature reads a 5^3 neighbourhood), its own PLIC offset
// d0(phi_i, n_i), and the point is the foot of its plane,
//     q_i = e_i + d0(phi_i, n_i) n_i - d0(phi_0, n) n,
// projected on the centre frame (x = q.b_x, y = q.b_y, z = q.n); with
// PLIC_FLAG_POINT_CENTROID the cut-polygon centroids c(n_i) - c(n) replace the
// foot points.  For n_i = n this is Eq. 36.  A neighbour whose own stencil
// leaves the field, or whose normal is undefined, keeps the centre normal.
// Every neighbour solve now needs its own normal-dependent constants, so the
// per-cell hoisting of the default kernel does not apply; one thread per
// list entry, grid-stride, the interface neighbours two at a time (the
// optimised SZ and analytic solutions solve both on the paired FP32 path).
#include "host_common.h"
#include "plic_pair.cuh"
#include "vof_curvature.cuh"

namespace plic {

constexpr int NN_THREADS = 128;

template <int METHOD>
__global__ void __launch_bounds__(NN_THREADS)
k_vof_curvature_nn(const float* __restrict__ phi, int nx, int ny, int nz,
                   const int32_t* __restrict__ idx, int64_t n, const int64_t* __restrict__ d_n,
                   float* __restrict__ out, uint32_t flags, int fit, float scale) {
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    const int64_t nxy = (int64_t)nx * ny;
    const bool cm = (flags & PLIC_FLAG_NORMAL_CM) != 0;
    const bool centroid = (flags & PLIC_FLAG_POINT_CENTROID) != 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lim;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = __ldg(idx + k);
        // 32-bit arithmetic: list entries are int32 cell indices
        const unsigned cu = (unsigned)c, zu = cu / (unsigned)nxy, ru = cu - zu * (unsigned)nxy;
        const int z = (int)zu, y = (int)(ru / (unsigned)nx), x = (int)(ru - (unsigned)y * (unsigned)nx);
        float nx_, ny_, nz_;
        if (!stencil_normal(phi, c, nx, nxy, cm, nx_, ny_, nz_)) { out[k] = 0.0f; continue; }
        // frame (Sec. 4.2)
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
        // centre plane
        CellPlic<METHOD> pl;
        pl.prepare(nx_, ny_, nz_);
        const float d00 = pl.offset(__ldg(phi + c));
        float c0x = 0.0f, c0y = 0.0f, c0z = 0.0f;
        if (centroid) {
            float A;
            area_centroid<float>(nx_, ny_, nz_, d00, A, c0x, c0y, c0z);
        }
        float M[15], bv[5];
#pragma unroll
        for (int q = 0; q < 15; ++q) M[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < 5; ++q) bv[q] = 0.0f;
        // the interface neighbours first (compile-time offsets), then a loop
        // over them only, so a warp runs as many trips as its busiest lane
        // has interface neighbours instead of 26
        unsigned mask = 0u;
        for_e27<1>([&](auto I) {
            constexpr int i = decltype(I)::value;
            int ex, ey, ez;
            e_of_c<i>(ex, ey, ez);
            const float v = __ldg(phi + c + ex + (int64_t)ey * nx + (int64_t)ez * nxy);
            if (v > 0.0f && v < 1.0f) mask |= 1u << i;
        });
        const int m = __popc(mask);
        unsigned list = mask;
#pragma unroll 1
        while (list) {
            // two neighbours per trip (an odd last one pairs with itself at
            // weight 0); each with its own normal, so no per-normal constants
            // are shared: the optimised SZ and analytic solutions solve the
            // two on the paired FP32 path, the other methods one by one
            int ii[2];
            ii[0] = __ffs(list) - 1;
            list &= list - 1u;
            const bool two = list != 0u;
            ii[1] = two ? __ffs(list) - 1 : ii[0];
            list &= list - 1u;                      // no-op on an empty list
            int ex[2], ey[2], ez[2];
            float v[2], mx[2], my[2], mz[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                e_of_lanes(ii[j], ex[j], ey[j], ez[j]);
                const int64_t ci = c + ex[j] + (int64_t)ey[j] * nx + (int64_t)ez[j] * nxy;
                v[j] = __ldg(phi + ci);
                mx[j] = nx_; my[j] = ny_; mz[j] = nz_;
                const int xi = x + ex[j], yi = y + ey[j], zi = z + ez[j];
                if (xi >= 1 && yi >= 1 && zi >= 1 && xi <= nx - 2 && yi <= ny - 2 && zi <= nz - 2) {
                    float ax, ay, az;
                    if (stencil_normal(phi, ci, nx, nxy, cm, ax, ay, az)) { mx[j] = ax; my[j] = ay; mz[j] = az; }
                }
            }
            float d0i[2];
            if (METHOD == M_SZ_OPT || METHOD == M_ANALYTIC) {
                int bad = 0;
                const p2::f2 r = p2::offset_pair<METHOD, true, false>(
                    make_float2(mx[0], mx[1]), make_float2(my[0], my[1]), make_float2(mz[0], mz[1]),
                    make_float2(v[0], v[1]), bad);
                d0i[0] = r.x;
                d0i[1] = r.y;
            } else {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    CellPlic<METHOD> pi;
                    pi.prepare(mx[j], my[j], mz[j]);
                    d0i[j] = pi.offset(v[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                float qx = (float)ex[j], qy = (float)ey[j], qz = (float)ez[j];
                if (centroid) {
                    float A, cx, cy, cz;
                    area_centroid<float>(mx[j], my[j], mz[j], d0i[j], A, cx, cy, cz);
                    qx += cx - c0x; qy += cy - c0y; qz += cz - c0z;
                } else {
                    qx += d0i[j] * mx[j] - d00 * nx_;
                    qy += d0i[j] * my[j] - d00 * ny_;
                    qz += d0i[j] * mz[j] - d00 * nz_;
                }
                const float w = (j == 0 || two) ? 1.0f : 0.0f;
                const float px = w * (qx * bxx + qy * bxy + qz * bxz);
                const float py = w * (qx * byx + qy * byy + qz * byz);
                const float pz = w * (qx * nx_ + qy * ny_ + qz * nz_);
                const float Q[5] = {px * px, py * py, px * py, px, py};
#pragma unroll
                for (int a = 0; a < 5; ++a) {
#pragma unroll
                    for (int b = a; b < 5; ++b) M[uidx(a, b)] = fmaf(Q[a], Q[b], M[uidx(a, b)]);
                    bv[a] = fmaf(pz, Q[a], bv[a]);
                }
            }
        }
        float xs[5];
        int dim;
        if (fit == FIT_FP32) {
            dim = fit_solve<FIT_FP32>(M, bv, m, xs);
        } else if (fit == FIT_DF32) {
            dim = fit_solve<FIT_DF32>(M, bv, m, xs);
        } else if (fit == FIT_FP64) {
            dim = fit_solve<FIT_FP64>(M, bv, m, xs);
        } else {
            // adaptive: FP32 unless the pivots show an ill-conditioned matrix
            Ldlt<FIT_FP32> f;
            f.factor(M, m);
            const int want = m < 5 ? m : 5;
            float dmin = 3.4e38f, dmax = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (j < f.dim) { dmin = fminf(dmin, f.D[j]); dmax = fmaxf(dmax, f.D[j]); }
            if (f.dim == want && dmin > 1e-2f * dmax) {
                f.solve(bv, xs);
                dim = f.dim;
            } else {
                dim = fit_solve<FIT_FP64>(M, bv, m, xs);
            }
        }
        float kap = 0.0f;
        if (dim > 0) {
            const float kk = paraboloid_kappa(xs);
            kap = (flags & PLIC_FLAG_KAPPA_PAPER_SIGN) ? kk : -kk;
        }
        out[k] = scale * kap;
    }
}

__global__ void __launch_bounds__(256)
k_vof_normal(const float* __restrict__ phi, int nx, int ny, const int32_t* __restrict__ idx,
             int64_t n, const int64_t* __restrict__ d_n, float* __restrict__ ox,
             float* __restrict__ oy, float* __restrict__ oz, int cm) {
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    const int64_t nxy = (int64_t)nx * ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lim;
         k += (int64_t)gridDim.x * blockDim.x) {
        float a, b, c;
        stencil_normal(phi, __ldg(idx + k), nx, nxy, cm != 0, a, b, c);
        ox[k] = a;
        oy[k] = b;
        oz[k] = c;
    }
}

plic_status launch_curvature_nn(const float* phi, int nx, int ny, int nz, const int32_t* idx,
                                int64_t n_iface, const int64_t* d_n_iface, float* out,
                                plic_method m, uint32_t flags, int fit, float scale,
                                void* stream, const char* who) {
    const void* k = nullptr;
    switch (m) {
        case PLIC_ANALYTIC: k = reinterpret_cast<const void*>(&k_vof_curvature_nn<M_ANALYTIC>); break;
        case PLIC_SZ_ORIG: k = reinterpret_cast<const void*>(&k_vof_curvature_nn<M_SZ_ORIG>); break;
        case PLIC_SZ_OPT: k = reinterpret_cast<const void*>(&k_vof_curvature_nn<M_SZ_OPT>); break;
        case PLIC_NEWTON: k = reinterpret_cast<const void*>(&k_vof_curvature_nn<M_NEWTON>); break;
        case PLIC_NESTED: k = reinterpret_cast<const void*>(&k_vof_curvature_nn<M_NESTED>); break;
    }
    if (!k) return PLIC_ERR_ARG;
    const int grid = stride_grid(k, NN_THREADS, n_iface);
    void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&nz, (void*)&idx, (void*)&n_iface,
                    (void*)&d_n_iface, (void*)&out, (void*)&flags, (void*)&fit, (void*)&scale};
    cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(NN_THREADS), args, 0, as_stream(stream));
    if (e != cudaSuccess) { set_last_error(who, e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}

}  // namespace plic

extern "C" plic_status vof_normal(const float* phi, int nx, int ny, int nz, const int32_t* idx,
                                  int64_t n_iface, const int64_t* d_n_iface, float* n_x,
                                  float* n_y, float* n_z, uint32_t flags, void* stream) {
    using namespace plic;
    if (nx < 3 || ny < 3 || nz < 3 || n_iface < 0 || (flags & ~(uint32_t)PLIC_FLAG_NORMAL_CM))
        return PLIC_ERR_ARG;
    if (n_iface == 0) return PLIC_OK;
    if (!phi || !idx || !n_x || !n_y || !n_z) return PLIC_ERR_ARG;
    if (!aligned(phi, 4) || !aligned(idx, 4) || !aligned(n_x, 4) || !aligned(n_y, 4) ||
        !aligned(n_z, 4) || (d_n_iface && !aligned(d_n_iface, 8)))
        return PLIC_ERR_ALIGN;
    const int cm = (flags & PLIC_FLAG_NORMAL_CM) ? 1 : 0;
    const int grid = stride_grid(reinterpret_cast<const void*>(&k_vof_normal), 256, n_iface);
    k_vof_normal<<<grid, 256, 0, as_stream(stream)>>>(phi, nx, ny, idx, n_iface, d_n_iface, n_x,
                                                     n_y, n_z, cm);
    return check_launch("vof_normal");
}
