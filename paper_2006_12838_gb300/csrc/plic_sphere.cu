// plic_sphere.cu -- the plane-sphere problem of Sec. 3 and its C entry points.
//
// The cell is a ball of unit volume, radius r = (3/(4 pi))^(1/3); a plane at
// signed distance d0 from the centre cuts off the spherical cap
// V0 = pi/3 (r + d0)^2 (2r - d0) on its lower side (0 below -r, 1 above r).
// With the symmetry V0(-d0) = 1 - V0(d0) and the cap height in units of r,
// u = (r + d0)/r for d0 <= 0, the forward problem is
//     W = u^2 (3 - u) / 4,   u in [0, 1],  W = min(V0, 1 - V0) in [0, 1/2],
// because pi r^3 = 3/4.  The inverse is solved per cell without
// trigonometric functions: a polynomial start in s = sqrt(W) (see cap_u_f32)
// and one Newton step on u^2 (3 - u) = 4W in FP32 with the MUFU reciprocal
// (|d0 - d0*| < 1e-7).  FP64 continues from the FP32 root with two Newton
// steps whose residual is evaluated in FP64 and whose
// derivative is the FP32 reciprocal: each step multiplies the error by about
// 1e-7, so the result is within a few ulp.  The paper's closed form (an arc
// tangent and a sine) is the reference the oracle is pinned to; this kernel
// spends a handful of FMAs and one MUFU reciprocal per step instead.
//
// Data: one array in, one out (SoA streams of float or double), 16-byte
// vectors in a grid-stride loop on up to 16 waves of blocks (stream_grid);
// 8 (FP32) or 16 (FP64) bytes per cell.
#include "host_common.h"
#include "plic_math.cuh"

namespace plic {
namespace sphere {

constexpr double R = 0.620350490899400016668;      // (3/(4 pi))^(1/3)
constexpr double INV_R = 1.0 / R;

// u^2 (3 - u) = 4W, W in [0, 1/2] -> u in [0, 1] (FP32).  Start:
// u0 = s (2/sqrt3 + s p(s)), s = sqrt(W), with the exact leading term of the
// small-W expansion u = sqrt(4W/3) + ... and a degree-4 least-squares p
// (|u0 - u| < 1.5e-5 on [0, 1/2]); one Newton step then leaves the FP32
// rounding of the result (|d0 - d0*| < 1e-7).
__device__ __forceinline__ float cap_u_f32(float W) {
    const float s = W > 0.0f ? W * rsqrtf(W) : 0.0f;
    float p = fmaf(s, 0.4812777f, -0.55447954f);
    p = fmaf(s, p, 0.3771915f);
    p = fmaf(s, p, 0.03742398f);
    p = fmaf(s, p, 0.22763859f);
    float u = s * fmaf(s, p, 1.1547005f);
    const float f = fmaf(u * u, 3.0f - u, -4.0f * W);
    const float fp = 3.0f * u * (2.0f - u);
    return fp > 0.0f ? u - f * Fm<float>::rcp_(fp) : u;
}

template <typename T> __device__ __forceinline__ T offset_cell(T V0);

template <> __device__ __forceinline__ float offset_cell<float>(float V0) {
    const float W = fminf(V0, 1.0f - V0);
    const float u = cap_u_f32(W);
    const float d = fmaf((float)R, u, -(float)R);     // r (u - 1) <= 0
    const float out = V0 <= 0.5f ? d : -d;
    return (V0 >= 0.0f && V0 <= 1.0f) ? out : __int_as_float(0x7fc00000);
}

template <> __device__ __forceinline__ double offset_cell<double>(double V0) {
    const double W = fmin(V0, 1.0 - V0);
    double u = (double)cap_u_f32((float)W);
    const double W4 = 4.0 * W;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double f = fma(u * u, 3.0 - u, -W4);
        const float fp = (float)(3.0 * u * (2.0 - u));
        u = fp > 0.0f ? u - f * (double)Fm<float>::rcp_(fp) : u;
    }
    const double d = fma(R, u, -R);
    const double out = V0 <= 0.5 ? d : -d;
    return (V0 >= 0.0 && V0 <= 1.0) ? out : __longlong_as_double(0x7ff8000000000000LL);
}

template <typename T> __device__ __forceinline__ T volume_cell(T d0) {
    const T a = fabs(d0) * T(INV_R);
    const T u = a < T(1) ? T(1) - a : T(0);           // cap height / r on the smaller side
    const T w = T(0.25) * u * u * (T(3) - u);
    const T out = d0 <= T(0) ? w : T(1) - w;
    return d0 == d0 ? out : d0;                       // NaN passes through
}

template <typename T> struct V16;
template <> struct V16<float> { typedef float4 type; static constexpr int W = 4; };
template <> struct V16<double> { typedef double2 type; static constexpr int W = 2; };
__device__ __forceinline__ void unpack(float4 v, float* a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ void unpack(double2 v, double* a) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ float4 pack(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 pack(const double* a) { return make_double2(a[0], a[1]); }

// INVERSE = 1: V0 -> d0; 0: d0 -> V0
template <typename T, int INVERSE>
__global__ void __launch_bounds__(256)
k_plic_sphere(const T* __restrict__ in, T* __restrict__ out, int64_t n, int vec_ok) {
    typedef typename V16<T>::type VT;
    constexpr int W = V16<T>::W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nvec = vec_ok ? n / W : 0;
    for (int64_t i = tid; i < nvec; i += stride) {
        T a[W], r[W];
        unpack(__ldcs(reinterpret_cast<const VT*>(in) + i), a);
#pragma unroll
        for (int j = 0; j < W; ++j) r[j] = INVERSE ? offset_cell<T>(a[j]) : volume_cell<T>(a[j]);
        __stcs(reinterpret_cast<VT*>(out) + i, pack(r));
    }
    for (int64_t i = nvec * W + tid; i < n; i += stride)
        out[i] = INVERSE ? offset_cell<T>(in[i]) : volume_cell<T>(in[i]);
}

template <typename T, int INVERSE>
static plic_status launch(const void* in, void* out, int64_t n, void* stream, const char* who) {
    const int vec_ok = aligned(in, 16) && aligned(out, 16);
    const void* k = reinterpret_cast<const void*>(&k_plic_sphere<T, INVERSE>);
    const int W = V16<T>::W;
    const int grid = stream_grid(k, 256, vec_ok ? (n + W - 1) / W : n);
    k_plic_sphere<T, INVERSE><<<grid, 256, 0, as_stream(stream)>>>((const T*)in, (T*)out, n, vec_ok);
    return check_launch(who);
}

static plic_status entry(const void* in, void* out, int64_t n, plic_precision p, void* stream,
                         int inverse, const char* who) {
    if (n < 0 || (int)p < 0 || (int)p > 3) return PLIC_ERR_ARG;
    if (n == 0) return PLIC_OK;
    if (!in || !out) return PLIC_ERR_ARG;
    const bool f64 = p == PLIC_FP64 || p == PLIC_FP64_REFINED;
    const size_t es = f64 ? 8 : 4;
    if (!aligned(in, es) || !aligned(out, es)) return PLIC_ERR_ALIGN;
    if (f64)
        return inverse ? launch<double, 1>(in, out, n, stream, who) : launch<double, 0>(in, out, n, stream, who);
    return inverse ? launch<float, 1>(in, out, n, stream, who) : launch<float, 0>(in, out, n, stream, who);
}

}  // namespace sphere
}  // namespace plic

extern "C" plic_status plic_sphere_volume(const void* d0, void* V0, int64_t n, plic_precision p,
                                          void* stream) {
    return plic::sphere::entry(d0, V0, n, p, stream, 0, "plic_sphere_volume");
}

extern "C" plic_status plic_sphere_offset(const void* V0, void* d0, int64_t n, plic_precision p,
                                          void* stream) {
    return plic::sphere::entry(V0, d0, n, p, stream, 1, "plic_sphere_offset");
}
