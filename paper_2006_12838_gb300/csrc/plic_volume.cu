// plic_volume.cu -- forward volume V0(n, d0) (Sec. 2.2, Eq. 10) and the
// adjoints of the forward and inverse problems, with their C entry points.
//
// Adjoints (implicit function theorem on Eq. 1, unit n): with A the area and
// c the centroid of the cut polygon of the plane n . x = d0,
//   dV0/dd0 = A,   dV0/dn = -A c,   dd0/dV0 = 1/A,   dd0/dn = c.
// All three kernels stream structure-of-arrays data through 16-byte vectors in
// a grid-stride loop on up to 16 waves of blocks (stream_grid), as plic_offset
// does.
#include "host_common.h"
#include "plic_polygon.cuh"

namespace plic {

template <typename T> struct V16;
template <> struct V16<float> { typedef float4 type; static constexpr int W = 4; };
template <> struct V16<double> { typedef double2 type; static constexpr int W = 2; };
__device__ __forceinline__ void unpack(float4 v, float* a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ void unpack(double2 v, double* a) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ float4 pack(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 pack(const double* a) { return make_double2(a[0], a[1]); }

template <typename T>
__global__ void __launch_bounds__(256)
k_plic_volume(const T* __restrict__ nx, const T* __restrict__ ny, const T* __restrict__ nz,
              const T* __restrict__ d0, T* __restrict__ V0, int64_t n, int vec_ok) {
    typedef typename V16<T>::type VT;
    constexpr int W = V16<T>::W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nvec = vec_ok ? n / W : 0;
    for (int64_t i = tid; i < nvec; i += stride) {
        T a[W], b[W], c[W], d[W], r[W];
        unpack(__ldcs(reinterpret_cast<const VT*>(nx) + i), a);
        unpack(__ldcs(reinterpret_cast<const VT*>(ny) + i), b);
        unpack(__ldcs(reinterpret_cast<const VT*>(nz) + i), c);
        unpack(__ldcs(reinterpret_cast<const VT*>(d0) + i), d);
#pragma unroll
        for (int j = 0; j < W; ++j) r[j] = volume_cell<T>(a[j], b[j], c[j], d[j]);
        __stcs(reinterpret_cast<VT*>(V0) + i, pack(r));
    }
    for (int64_t i = nvec * W + tid; i < n; i += stride) V0[i] = volume_cell<T>(nx[i], ny[i], nz[i], d0[i]);
}

// MODE 0: offset backward  (gV0 = g/A, gn = g c)
// MODE 1: volume backward  (gd0 = g A, gn = -g A c)
template <typename T, int MODE>
__device__ __forceinline__ void adjoint_cell(T nx, T ny, T nz, T d0, T g, T& gs, T& gx, T& gy,
                                             T& gz) {
    T A, cx, cy, cz;
    const bool ok = area_centroid<T>(nx, ny, nz, d0, A, cx, cy, cz);
    if (MODE == 0) {
        gs = ok ? Fm<T>::div_(g, A) : (g == T(0) ? T(0) : copysign(T(INFINITY), g));
        gx = g * cx; gy = g * cy; gz = g * cz;
        if (!ok && !(fabs(nx) + fabs(ny) + fabs(nz) > T(0))) gs = gx = gy = gz = T(NAN);
    } else {
        gs = g * A;
        const T s = -g * A;
        gx = s * cx; gy = s * cy; gz = s * cz;
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
k_plic_adjoint(const T* __restrict__ nx, const T* __restrict__ ny, const T* __restrict__ nz,
               const T* __restrict__ d0, const T* __restrict__ g, T* __restrict__ gs,
               T* __restrict__ gx, T* __restrict__ gy, T* __restrict__ gz, int64_t n, int vec_ok) {
    typedef typename V16<T>::type VT;
    constexpr int W = V16<T>::W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nvec = vec_ok ? n / W : 0;
    for (int64_t i = tid; i < nvec; i += stride) {
        T a[W], b[W], c[W], d[W], e[W], o0[W], o1[W], o2[W], o3[W];
        unpack(__ldcs(reinterpret_cast<const VT*>(nx) + i), a);
        unpack(__ldcs(reinterpret_cast<const VT*>(ny) + i), b);
        unpack(__ldcs(reinterpret_cast<const VT*>(nz) + i), c);
        unpack(__ldcs(reinterpret_cast<const VT*>(d0) + i), d);
        unpack(__ldcs(reinterpret_cast<const VT*>(g) + i), e);
#pragma unroll
        for (int j = 0; j < W; ++j) adjoint_cell<T, MODE>(a[j], b[j], c[j], d[j], e[j], o0[j], o1[j], o2[j], o3[j]);
        if (gs) __stcs(reinterpret_cast<VT*>(gs) + i, pack(o0));
        if (gx) __stcs(reinterpret_cast<VT*>(gx) + i, pack(o1));
        if (gy) __stcs(reinterpret_cast<VT*>(gy) + i, pack(o2));
        if (gz) __stcs(reinterpret_cast<VT*>(gz) + i, pack(o3));
    }
    for (int64_t i = nvec * W + tid; i < n; i += stride) {
        T o0, o1, o2, o3;
        adjoint_cell<T, MODE>(nx[i], ny[i], nz[i], d0[i], g[i], o0, o1, o2, o3);
        if (gs) gs[i] = o0;
        if (gx) gx[i] = o1;
        if (gy) gy[i] = o2;
        if (gz) gz[i] = o3;
    }
}

static bool all_aligned(size_t a, std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (p && !aligned(p, a)) return false;
    return true;
}

template <typename T>
static plic_status launch_volume(const void* nx, const void* ny, const void* nz, const void* d0,
                                 void* V0, int64_t n, void* stream) {
    const int vec_ok = all_aligned(16, {nx, ny, nz, d0, V0});
    const void* k = reinterpret_cast<const void*>(&k_plic_volume<T>);
    const int W = V16<T>::W;
    const int grid = stream_grid(k, 256, vec_ok ? (n + W - 1) / W : n);
    k_plic_volume<T><<<grid, 256, 0, as_stream(stream)>>>(
        (const T*)nx, (const T*)ny, (const T*)nz, (const T*)d0, (T*)V0, n, vec_ok);
    return check_launch("plic_volume");
}

template <typename T, int MODE>
static plic_status launch_adjoint(const void* nx, const void* ny, const void* nz, const void* d0,
                                  const void* g, void* gs, void* gx, void* gy, void* gz,
                                  int64_t n, void* stream) {
    const int vec_ok = all_aligned(16, {nx, ny, nz, d0, g, gs, gx, gy, gz});
    const void* k = reinterpret_cast<const void*>(&k_plic_adjoint<T, MODE>);
    const int W = V16<T>::W;
    const int grid = stream_grid(k, 256, vec_ok ? (n + W - 1) / W : n);
    k_plic_adjoint<T, MODE><<<grid, 256, 0, as_stream(stream)>>>(
        (const T*)nx, (const T*)ny, (const T*)nz, (const T*)d0, (const T*)g, (T*)gs, (T*)gx,
        (T*)gy, (T*)gz, n, vec_ok);
    return check_launch(MODE == 0 ? "plic_offset_backward" : "plic_volume_backward");
}

static plic_status check_common(std::initializer_list<const void*> req,
                                std::initializer_list<const void*> opt, int64_t n,
                                plic_precision p) {
    if (n < 0 || (int)p < 0 || (int)p > 2) return PLIC_ERR_ARG;
    if (n == 0) return PLIC_OK;
    for (const void* q : req)
        if (!q) return PLIC_ERR_ARG;
    const size_t es = p == PLIC_FP64 ? 8 : 4;
    if (!all_aligned(es, req) || !all_aligned(es, opt)) return PLIC_ERR_ALIGN;
    return PLIC_OK;
}

}  // namespace plic

extern "C" plic_status plic_volume(const void* nx, const void* ny, const void* nz,
                                   const void* d0, void* V0, int64_t n, plic_precision p,
                                   void* stream) {
    using namespace plic;
    plic_status s = check_common({nx, ny, nz, d0, V0}, {}, n, p);
    if (s != PLIC_OK || n == 0) return s;
    return p == PLIC_FP64 ? launch_volume<double>(nx, ny, nz, d0, V0, n, stream)
                          : launch_volume<float>(nx, ny, nz, d0, V0, n, stream);
}

extern "C" plic_status plic_offset_backward(const void* nx, const void* ny, const void* nz,
                                            const void* d0, const void* g_d0, void* g_V0,
                                            void* g_nx, void* g_ny, void* g_nz, int64_t n,
                                            plic_precision p, void* stream) {
    using namespace plic;
    plic_status s = check_common({nx, ny, nz, d0, g_d0}, {g_V0, g_nx, g_ny, g_nz}, n, p);
    if (s != PLIC_OK || n == 0) return s;
    return p == PLIC_FP64
               ? launch_adjoint<double, 0>(nx, ny, nz, d0, g_d0, g_V0, g_nx, g_ny, g_nz, n, stream)
               : launch_adjoint<float, 0>(nx, ny, nz, d0, g_d0, g_V0, g_nx, g_ny, g_nz, n, stream);
}

extern "C" plic_status plic_volume_backward(const void* nx, const void* ny, const void* nz,
                                            const void* d0, const void* g_V0, void* g_d0,
                                            void* g_nx, void* g_ny, void* g_nz, int64_t n,
                                            plic_precision p, void* stream) {
    using namespace plic;
    plic_status s = check_common({nx, ny, nz, d0, g_V0}, {g_d0, g_nx, g_ny, g_nz}, n, p);
    if (s != PLIC_OK || n == 0) return s;
    return p == PLIC_FP64
               ? launch_adjoint<double, 1>(nx, ny, nz, d0, g_V0, g_d0, g_nx, g_ny, g_nz, n, stream)
               : launch_adjoint<float, 1>(nx, ny, nz, d0, g_V0, g_d0, g_nx, g_ny, g_nz, n, stream);
}
