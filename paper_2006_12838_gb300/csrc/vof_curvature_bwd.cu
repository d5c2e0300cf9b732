// vof_curvature_bwd.cu -- vector-Jacobian product of the curvature step
// (Sec. 4.2, Appendix B) with respect to the fill field:
//   g_phi = d(sum_k g_kappa[k] kappa[k]) / d phi,
// with the interface set (the list and the 0 < phi < 1 flags of the stencil)
// held fixed.
//
// Per interface cell (eight lanes, see k_vof_curvature_vjp), the forward step is
// recomputed and reversed:
//   kappa = s N / (1 + H^2 + I^2)^(3/2), N = A (I^2+1) + B (H^2+1) - C H I (Eq. 42)
//     -> pbar = dkappa/d(A,B,C,H,I) * g_kappa
//   M p = b (leading block, Appendix B)  ->  bbar = M^-1 pbar (same LDL^T factors),
//     Mbar = -bbar p^T
//   M = sum Q Q^T, b = sum z Q  ->  Qbar_i = bbar (z_i - p.Q_i) - p (bbar.Q_i),
//     zbar_i = bbar.Q_i; Q = (x^2, y^2, xy, x, y) -> xbar_i, ybar_i
//   x_i = e_i.b_x, y_i = e_i.b_y, z_i = e_i.n + d0_i - d0_0 (Eq. 36)
//   d0_i = d0(phi_i, n): dd0/dphi = 1/A_i, dd0/dn = c_i (cut-polygon area and
//     centroid, implicit function theorem on Eq. 1)
//   b_x = b_y x n, b_y = u/|u|, u = n x r (Sec. 4.2)
//   n = -g/|g|, g = sum w_i e_i phi_i (Eq. 38)
// The 27 partial derivatives of each cell go to the workspace; a second kernel
// sums, for every field cell j, the entries of the (at most 27) interface cells
// whose stencil contains j, in a fixed order -- deterministic, no atomics.
// Only the foot-point variant (Eq. 36) is differentiated.
#include <type_traits>

#include "host_common.h"
#include "vof_curvature_coop.cuh"

namespace plic {

constexpr int CB_THREADS = 128;       // 4 warps per block
constexpr int CB_WARPS = CB_THREADS / 32;
constexpr int CB_REC = 21 + 27;       // per cell: M (15), b (5), m, then 27 point terms

__device__ __forceinline__ void cross3(float ax, float ay, float az, float bx, float by, float bz,
                                       float& cx, float& cy, float& cz) {
    cx = ay * bz - az * by;
    cy = az * bx - ax * bz;
    cz = ax * by - ay * bx;
}

// Sum over the 8 lanes of a group (every lane gets the total).
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Eight lanes per interface cell, four cells per warp at a time (as the
// forward kernel): lane g of a group loads stencil entries g, g+8, g+16, g+24,
// and takes the g-th, (g+8)-th, ... entry of the cell's list [centre,
// interface neighbours] for the PLIC solves (forward) and for the point terms
// of the reverse pass.  The normal equations go through shared memory; every
// lane of the group then factorises and solves them (no divergence), and the
// reverse pass of the frame and normal is likewise computed by all 8 lanes.
template <int METHOD, int FIT>
__global__ void __launch_bounds__(CB_THREADS)
k_vof_curvature_vjp(const float* __restrict__ phi, int nx, int ny,
                    const int32_t* __restrict__ idx, int64_t n, const int64_t* __restrict__ d_n,
                    const float* __restrict__ g_kappa, float* __restrict__ contrib, uint32_t flags) {
    __shared__ float smem[CB_WARPS][4][CB_REC];
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane & 7, grp = lane >> 3, leader = lane & ~7;
    const bool cm = (flags & PLIC_FLAG_NORMAL_CM) != 0;
    const float sgn = (flags & PLIC_FLAG_KAPPA_PAPER_SIGN) ? 1.0f : -1.0f;
    const int64_t nxy = (int64_t)nx * ny;
    float* rec = smem[warp][grp];
    const int64_t gw = (int64_t)blockIdx.x * CB_WARPS + warp;
    const int64_t nw = (int64_t)gridDim.x * CB_WARPS;
    for (int64_t k0 = gw * 4; k0 < lim; k0 += nw * 4) {
        const int64_t k = k0 + grp;
        const bool on = k < lim;
        const int64_t c = on ? (int64_t)__ldg(idx + k) : 0;
        const float gk = on ? __ldg(g_kappa + k) : 0.0f;
        // ---- forward: stencil, Parker-Youngs (or CM) sums, interface mask ----
        float gx = 0.0f, gy = 0.0f, gz = 0.0f, phi0 = 0.0f;
        unsigned mask = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = g + 8 * j;
            if (i < 27 && on) {
                int ex, ey, ez;
                e_of(i, ex, ey, ez);
                const float v = __ldg(phi + c + ex + (int64_t)ey * nx + (int64_t)ez * nxy);
                const int e2 = ex * ex + ey * ey + ez * ez;
                const float w = cm ? 1.0f : (e2 == 1 ? 4.0f : (e2 == 2 ? 2.0f : 1.0f));
                gx = fmaf(w * ex, v, gx);
                gy = fmaf(w * ey, v, gy);
                gz = fmaf(w * ez, v, gz);
                if (i == 0) phi0 = v;
                else if (v > 0.0f && v < 1.0f) mask |= 1u << i;
            }
        }
        gx = group_sum(gx); gy = group_sum(gy); gz = group_sum(gz);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
        phi0 = __shfl_sync(0xffffffffu, phi0, leader);
        const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
        bool live = on && gl > 0.0f && gk != 0.0f;
        const float inv = live ? -1.0f / gl : 0.0f;
        const float nx_ = live ? gx * inv : 1.0f, ny_ = gy * inv, nz_ = gz * inv;
        // ---- frame: u = n x r, b_y = u/|u|, b_x = b_y x n (Sec. 4.2) ----
        float rx = 0.56270900f, ry = 0.32704452f, rz = 0.75921047f, ux, uy, uz;
        cross3(nx_, ny_, nz_, rx, ry, rz, ux, uy, uz);
        float u2 = ux * ux + uy * uy + uz * uz;
        if (!(u2 > 1e-12f)) {
            rx = 0.32704452f; ry = 0.75921047f; rz = 0.56270900f;
            cross3(nx_, ny_, nz_, rx, ry, rz, ux, uy, uz);
            u2 = ux * ux + uy * uy + uz * uz;
        }
        const float ul = sqrtf(u2), iu = 1.0f / ul;
        const float byx = ux * iu, byy = uy * iu, byz = uz * iu;
        float bxx, bxy, bxz;
        cross3(byx, byy, byz, nx_, ny_, nz_, bxx, bxy, bxz);
        // ---- PLIC offsets of the list entries dealt to this lane ----
        CellPlic<METHOD> pl;
        pl.prepare(nx_, ny_, nz_);
        const unsigned list = mask | 1u;
        const int cnt = __popc(list);
        int ent[4];
        float d0s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = g + 8 * j;
            ent[j] = -1;
            d0s[j] = 0.0f;
            if (live && p < cnt) {
                const int i = nth_set_bit(list, p);
                ent[j] = i;
                int ex, ey, ez;
                e_of(i, ex, ey, ez);
                const float v = i == 0 ? phi0 : __ldg(phi + c + ex + (int64_t)ey * nx + (int64_t)ez * nxy);
                d0s[j] = pl.offset(v);
            }
        }
        const float d00 = __shfl_sync(0xffffffffu, d0s[0], leader);
        // ---- points (Eq. 36) and partial normal equations ----
        float acc[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) acc[q] = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = ent[j];
            if (i > 0) {
                int ex, ey, ez;
                e_of(i, ex, ey, ez);
                const float x = ex * bxx + ey * bxy + ez * bxz;
                const float y = ex * byx + ey * byy + ez * byz;
                const float z = ex * nx_ + ey * ny_ + ez * nz_ + (d0s[j] - d00);
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
        if (g == 0) rec[20] = live ? (float)(cnt - 1) : -1.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (g + 8 * j < 27) rec[21 + g + 8 * j] = 0.0f;
        __syncwarp();
        // ---- solve (all lanes of the group) and Eq. 42 backward ----
        const int m = (int)rec[20];
        live = live && m > 0;
        typename std::conditional<FIT == FIT_AUTO, LdltAuto, Ldlt<FIT>>::type fac;
        float p[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, bb[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (live) {
            fac.factor(rec, m);
            fac.solve(rec + 15, p);
            live = fac.dim > 0;
        }
        float sx[10];                  // b_x bar (3), b_y bar (3), n bar (3), d00 bar
#pragma unroll
        for (int q = 0; q < 10; ++q) sx[q] = 0.0f;
        if (live) {
            const float A = p[0], B = p[1], C = p[2], H = p[3], I = p[4];
            const float w = 1.0f + H * H + I * I;
            const float rw = rsqrtf(w);
            const float iD = rw * rw * rw;                        // (1+H^2+I^2)^(-3/2)
            const float N = A * (I * I + 1.0f) + B * (H * H + 1.0f) - C * H * I;
            const float sg = sgn * gk * iD;
            float pbar[5];
            pbar[0] = sg * (I * I + 1.0f);
            pbar[1] = sg * (H * H + 1.0f);
            pbar[2] = -sg * H * I;
            pbar[3] = sg * (2.0f * B * H - C * I - 3.0f * H * N / w);
            pbar[4] = sg * (2.0f * A * I - C * H - 3.0f * I * N / w);
            fac.solve(pbar, bb);                                  // b bar = M^-1 p bar
            // ---- reverse pass over this lane's points ----
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = ent[j];
                if (i > 0) {
                    int ex, ey, ez;
                    e_of(i, ex, ey, ez);
                    const float x = ex * bxx + ey * bxy + ez * bxz;
                    const float y = ex * byx + ey * byy + ez * byz;
                    const float z = ex * nx_ + ey * ny_ + ez * nz_ + (d0s[j] - d00);
                    const float Q[5] = {x * x, y * y, x * y, x, y};
                    float pQ = 0.0f, bQ = 0.0f;
#pragma unroll
                    for (int a = 0; a < 5; ++a) {
                        pQ = fmaf(p[a], Q[a], pQ);
                        bQ = fmaf(bb[a], Q[a], bQ);
                    }
                    const float res = z - pQ;
                    float Qb[5];
#pragma unroll
                    for (int a = 0; a < 5; ++a) Qb[a] = bb[a] * res - p[a] * bQ;
                    const float xb = 2.0f * x * Qb[0] + y * Qb[2] + Qb[3];
                    const float yb = 2.0f * y * Qb[1] + x * Qb[2] + Qb[4];
                    const float zb = bQ;
                    sx[0] += xb * ex; sx[1] += xb * ey; sx[2] += xb * ez;
                    sx[3] += yb * ex; sx[4] += yb * ey; sx[5] += yb * ez;
                    sx[6] += zb * ex; sx[7] += zb * ey; sx[8] += zb * ez;
                    sx[9] -= zb;
                    // d0_i = d0(phi_i, n): dd0/dphi = 1/A_i, dd0/dn = c_i
                    float Ai, cx, cy, cz;
                    if (area_centroid<float>(nx_, ny_, nz_, d0s[j], Ai, cx, cy, cz)) {
                        rec[21 + i] = zb / Ai;
                        sx[6] += zb * cx; sx[7] += zb * cy; sx[8] += zb * cz;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) sx[q] = group_sum(sx[q]);
        float gbx = 0.0f, gby = 0.0f, gbz = 0.0f;
        if (live) {
            float nbx = sx[6], nby = sx[7], nbz = sx[8];
            float bybx = sx[3], byby = sx[4], bybz = sx[5];
            const float bxbx = sx[0], bxby = sx[1], bxbz = sx[2], d00b = sx[9];
            {   // the centre's d0 = d0(phi_0, n)
                float A0, cx, cy, cz;
                if (area_centroid<float>(nx_, ny_, nz_, d00, A0, cx, cy, cz)) {
                    if (g == 0) rec[21] = d00b / A0;
                    nbx += d00b * cx; nby += d00b * cy; nbz += d00b * cz;
                }
            }
            // ---- frame backward: b_x = b_y x n ----
            float tx, ty, tz;
            cross3(bxbx, bxby, bxbz, byx, byy, byz, tx, ty, tz);     // nbar += bxbar x b_y
            nbx += tx; nby += ty; nbz += tz;
            cross3(nx_, ny_, nz_, bxbx, bxby, bxbz, tx, ty, tz);     // bybar += n x bxbar
            bybx += tx; byby += ty; bybz += tz;
            // b_y = u/|u|, u = n x r
            const float dp = byx * bybx + byy * byby + byz * bybz;
            const float ubx = (bybx - byx * dp) * iu, uby = (byby - byy * dp) * iu, ubz = (bybz - byz * dp) * iu;
            cross3(rx, ry, rz, ubx, uby, ubz, tx, ty, tz);           // nbar += r x ubar
            nbx += tx; nby += ty; nbz += tz;
            // ---- normal backward: n = -g/|g| ----
            const float nn = nx_ * nbx + ny_ * nby + nz_ * nbz;
            const float ig = -1.0f / gl;
            gbx = (nbx - nx_ * nn) * ig; gby = (nby - ny_ * nn) * ig; gbz = (nbz - nz_ * nn) * ig;
        }
        __syncwarp();
        // ---- Parker-Youngs backward and the cell's 27 partial derivatives ----
        if (on) {
            float* out = contrib + k * 27;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = g + 8 * j;
                if (i < 27) {
                    int ex, ey, ez;
                    e_of(i, ex, ey, ez);
                    const int e2 = ex * ex + ey * ey + ez * ez;
                    const float wi = cm ? 1.0f : (e2 == 1 ? 4.0f : (e2 == 2 ? 2.0f : 1.0f));
                    out[i] = rec[21 + i] + wi * (ex * gbx + ey * gby + ez * gbz);
                }
            }
        }
        __syncwarp();
    }
}

__global__ void k_curv_slot_scatter(const int32_t* __restrict__ idx, int64_t n,
                                    const int64_t* __restrict__ d_n, int32_t* __restrict__ slot) {
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lim;
         k += (int64_t)gridDim.x * blockDim.x)
        slot[idx[k]] = (int32_t)k;
}

// g_phi[j] = sum over the 27 offsets o of contrib[slot[j - e_o]][o] (when cell
// j - e_o is in the field and in the list), in the fixed order o = 0..26.
// Only cells in the 3^3 neighbourhood of an interface cell can be non-zero,
// so the work runs over the (list entry k, offset o) pairs: pair (k, o) looks
// at j = idx[k] + e_o, and computes and stores g_phi[j] only if k is the
// first list entry (smallest index, i.e. smallest cell) whose stencil holds j,
// so every such j is written exactly once, with the same summation order as a
// dense pass.  The rest of g_phi was zeroed before.  O(27 * 27 * K) loads of
// the slot map instead of 27 per field cell.
__global__ void __launch_bounds__(256)
k_curv_gather(const int32_t* __restrict__ idx, int64_t n, const int64_t* __restrict__ d_n,
              const int32_t* __restrict__ slot, const float* __restrict__ contrib, int nx, int ny,
              int nz, float* __restrict__ g_phi) {
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    // fields hold < 2^31 cells (checked by the entry point): 32-bit index math;
    // the pair index t = 27 k + o fits 32 bits unless the list is longer than
    // 2^32 / 27 (then the 64-bit division)
    const int nxy = nx * ny;
    const bool small = lim * 27 <= (int64_t)0xffffffffu;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < lim * 27;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = small ? (int)((uint32_t)t / 27u) : (int)(t / 27);
        const int o = (int)(t - (int64_t)k * 27);
        int ex, ey, ez;
        e_of_lanes(o, ex, ey, ez);                  // o differs across the warp
        const int c = __ldg(idx + k);
        const int cz = c / nxy, cr = c - cz * nxy, cy = cr / nx, cx = cr - cy * nx;
        const int x = cx + ex, y = cy + ey, z = cz + ez;
        const int j = c + ex + ey * nx + ez * nxy;
        float acc = 0.0f;
        int32_t first = 0x7fffffff;
        for_e27<0>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            int fx, fy, fz;
            e_of_c<q>(fx, fy, fz);
            const int sx = x - fx, sy = y - fy, sz = z - fz;
            if (sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz) return;
            const int32_t sl = __ldg(slot + (j - fx - fy * nx - fz * nxy));
            if (sl >= 0) {
                acc += __ldg(contrib + (int64_t)sl * 27 + q);
                first = sl < first ? sl : first;
            }
        });
        if (first == k) g_phi[j] = acc;
    }
}

template <int METHOD>
static const void* pick_vjp(int fit) {
    switch (fit) {
        case FIT_FP32: return reinterpret_cast<const void*>(&k_vof_curvature_vjp<METHOD, FIT_FP32>);
        case FIT_DF32: return reinterpret_cast<const void*>(&k_vof_curvature_vjp<METHOD, FIT_DF32>);
        case FIT_FP64: return reinterpret_cast<const void*>(&k_vof_curvature_vjp<METHOD, FIT_FP64>);
        default: return reinterpret_cast<const void*>(&k_vof_curvature_vjp<METHOD, FIT_AUTO>);
    }
}

}  // namespace plic

extern "C" size_t plic_curv_bwd_workspace_bytes(int64_t cells, int64_t n_iface) {
    if (cells < 0 || n_iface < 0) return 0;
    const size_t a = ((size_t)cells * sizeof(int32_t) + 255) / 256 * 256;
    const size_t b = ((size_t)n_iface * 27 * sizeof(float) + 255) / 256 * 256;
    return a + b;
}

extern "C" plic_status vof_curvature_backward(const float* phi, int nx, int ny, int nz,
                                              const int32_t* idx, int64_t n_iface,
                                              const int64_t* d_n_iface, const float* g_kappa,
                                              float* g_phi, plic_method m, uint32_t flags,
                                              void* workspace, size_t ws_bytes, void* stream) {
    using namespace plic;
    if (nx < 3 || ny < 3 || nz < 3 || n_iface < 0) return PLIC_ERR_ARG;
    if ((int)m < 0 || (int)m > 4) return PLIC_ERR_ARG;
    const uint32_t known = PLIC_FLAG_POINT_CENTROID | PLIC_FLAG_KAPPA_PAPER_SIGN |
                           PLIC_FLAG_FIT_FP32 | PLIC_FLAG_FIT_DF32 | PLIC_FLAG_FIT_FP64 |
                           PLIC_FLAG_NORMAL_CM | PLIC_FLAG_NEIGHBOR_NORMAL;
    const uint32_t fitf = flags & (PLIC_FLAG_FIT_FP32 | PLIC_FLAG_FIT_DF32 | PLIC_FLAG_FIT_FP64);
    if ((flags & ~known) || (fitf & (fitf - 1u))) return PLIC_ERR_ARG;
    if (flags & (PLIC_FLAG_POINT_CENTROID | PLIC_FLAG_NEIGHBOR_NORMAL)) return PLIC_ERR_UNSUPPORTED;
    const int64_t cells = (int64_t)nx * ny * nz;
    if (cells > 2147483647LL) return PLIC_ERR_ARG;
    if (!phi || !g_phi || (n_iface > 0 && (!idx || !g_kappa)) || !workspace) return PLIC_ERR_ARG;
    if (ws_bytes < plic_curv_bwd_workspace_bytes(cells, n_iface)) return PLIC_ERR_ARG;
    if (!aligned(phi, 4) || !aligned(g_phi, 4) || (idx && !aligned(idx, 4)) ||
        (g_kappa && !aligned(g_kappa, 4)) || !aligned(workspace, 256) ||
        (d_n_iface && !aligned(d_n_iface, 8)))
        return PLIC_ERR_ALIGN;
    cudaStream_t s = as_stream(stream);
    char* ws = reinterpret_cast<char*>(workspace);
    int32_t* slot = reinterpret_cast<int32_t*>(ws);
    float* contrib = reinterpret_cast<float*>(ws + ((size_t)cells * sizeof(int32_t) + 255) / 256 * 256);
    cudaError_t e = cudaMemsetAsync(slot, 0xff, (size_t)cells * sizeof(int32_t), s);
    if (e != cudaSuccess) { set_last_error("vof_curvature_backward", e); return PLIC_ERR_CUDA; }
    if (n_iface > 0) {
        // the same fit policy as the forward call: adaptive unless a FIT flag is given
        const int fit = (flags & PLIC_FLAG_FIT_DF32) ? FIT_DF32 : (flags & PLIC_FLAG_FIT_FP32) ? FIT_FP32
                      : (flags & PLIC_FLAG_FIT_FP64) ? FIT_FP64 : FIT_AUTO;
        const void* k = nullptr;
        switch (m) {
            case PLIC_ANALYTIC: k = pick_vjp<M_ANALYTIC>(fit); break;
            case PLIC_SZ_ORIG: k = pick_vjp<M_SZ_ORIG>(fit); break;
            case PLIC_SZ_OPT: k = pick_vjp<M_SZ_OPT>(fit); break;
            case PLIC_NEWTON: k = pick_vjp<M_NEWTON>(fit); break;
            case PLIC_NESTED: k = pick_vjp<M_NESTED>(fit); break;
        }
        const int grid = stride_grid(k, CB_THREADS, (n_iface + 3) / 4 * 32);   // 8 lanes per cell
        void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&idx, (void*)&n_iface,
                        (void*)&d_n_iface, (void*)&g_kappa, (void*)&contrib, (void*)&flags};
        e = cudaLaunchKernel(k, dim3(grid), dim3(CB_THREADS), args, 0, s);
        if (e != cudaSuccess) { set_last_error("vof_curvature_backward", e); return PLIC_ERR_CUDA; }
        const int sg = stride_grid(reinterpret_cast<const void*>(&k_curv_slot_scatter), 256, n_iface);
        k_curv_slot_scatter<<<sg, 256, 0, s>>>(idx, n_iface, d_n_iface, slot);
    }
    e = cudaMemsetAsync(g_phi, 0, (size_t)cells * sizeof(float), s);
    if (e != cudaSuccess) { set_last_error("vof_curvature_backward", e); return PLIC_ERR_CUDA; }
    if (n_iface > 0) {
        const int gg = stride_grid(reinterpret_cast<const void*>(&k_curv_gather), 256, n_iface * 27);
        k_curv_gather<<<gg, 256, 0, s>>>(idx, n_iface, d_n_iface, slot, contrib, nx, ny, nz, g_phi);
    }
    return check_launch("vof_curvature_backward");
}
