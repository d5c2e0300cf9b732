// plic_offset.cu -- batched PLIC inversion d0(V0, n) (Sec. 2, Eq. 1) with the
// five solvers of Sec. 2.3-2.5, and the C entry point plic_offset().
//
// Layout: structure of arrays nx, ny, nz, V0 -> d0.  One thread handles one
// 16-byte vector of each array per step of a grid-stride loop (4 cells in FP32,
// 2 in FP64), so every warp issues fully coalesced 512-byte loads; the grid is
// up to 16 waves of resident blocks (stream_grid: measured faster than one
// persistent wave).  Loads and the store are streaming (evict-first): every
// byte is touched once.
//
// Roofline: 20 B/cell in FP32 (16 in, 4 out), 40 B/cell in FP64.  The FP32
// solvers sit near the HBM/ALU balance point; FP64 is bound by the FP64 pipe.
#include "host_common.h"
#include "plic_pair.cuh"
#include "plic_solvers.cuh"

namespace plic {

template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; static constexpr int W = 4; };
template <> struct Vec16<double> { typedef double2 type; static constexpr int W = 2; };

template <typename V> __device__ __forceinline__ V ld_stream(const V* p) { return __ldcs(p); }
template <typename V> __device__ __forceinline__ void st_stream(V* p, V v) { __stcs(p, v); }

__device__ __forceinline__ void to_arr(float4 v, float* a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ void to_arr(double2 v, double* a) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ float4 from_arr(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 from_arr(const double* a) { return make_double2(a[0], a[1]); }

__device__ __forceinline__ void count_invalid(int bad, unsigned long long* counter) {
    if (counter == nullptr) return;
    const unsigned mask = __activemask();
    const int tot = __reduce_add_sync(mask, bad);
    const int leader = __ffs(mask) - 1;
    if ((int)(threadIdx.x & 31) == leader && tot > 0) atomicAdd(counter, (unsigned long long)tot);
}

template <int METHOD, typename T, bool POLISH, bool FAITHFUL>
__global__ void __launch_bounds__(256)
k_plic_offset(const T* __restrict__ nx, const T* __restrict__ ny, const T* __restrict__ nz,
              const T* __restrict__ V0, T* __restrict__ d0, int64_t n, int vec_ok,
              unsigned long long* invalid, void* /* round trip: not fused here */) {
    typedef typename Vec16<T>::type VT;
    constexpr int W = Vec16<T>::W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    const int64_t nvec = vec_ok ? n / W : 0;
    for (int64_t i = tid; i < nvec; i += stride) {
        T a[W], b[W], c[W], v[W], r[W];
        to_arr(ld_stream(reinterpret_cast<const VT*>(nx) + i), a);
        to_arr(ld_stream(reinterpret_cast<const VT*>(ny) + i), b);
        to_arr(ld_stream(reinterpret_cast<const VT*>(nz) + i), c);
        to_arr(ld_stream(reinterpret_cast<const VT*>(V0) + i), v);
#pragma unroll
        for (int j = 0; j < W; ++j) r[j] = offset_cell<METHOD, T, POLISH, FAITHFUL>(a[j], b[j], c[j], v[j], bad);
        st_stream(reinterpret_cast<VT*>(d0) + i, from_arr(r));
    }
    for (int64_t i = nvec * W + tid; i < n; i += stride)
        d0[i] = offset_cell<METHOD, T, POLISH, FAITHFUL>(nx[i], ny[i], nz[i], V0[i], bad);
    count_invalid(bad, invalid);
}

// Work-compacted form of k_plic_offset for the default (non-literal) solvers:
// the warp runs the symmetry front end and the closed-form cases (Eqs. 24-25)
// on its 32 x W cells, then gathers the cells that need the heavy part (the
// trigonometric root of cases (3)/(4), or the Newton / nested-interval
// iterations) into a dense per-warp task list -- one warp vote per cell slot
// and a popcount prefix give each task its place -- and runs the heavy part
// on those tasks only, 32 at a time; the owners then take their results
// back.  Without this every lane of the warp would pass through the heavy
// part whenever any lane needed it (about every time: 40-60 % of random cells
// are in cases (3)/(4)), and lanes with closed-form cells would idle through
// it.  The task list lives in shared memory (4 values per task).
// The symmetry front end of Sec. 2.1 for one double cell on the bit patterns:
// the FP64 kernels are bound by the FP64 pipe, so the sort of |n| (the order
// of non-negative doubles is that of their bits; a NaN sorts last and makes L
// NaN), the validity tests and the choice V = V0 or 1 - V0 (exact) run as
// integer instructions; L keeps the FP64 sum |nx| + |ny| + |nz| in that order.
__device__ __forceinline__ bool front_bits(double nx, double ny, double nz, double V0, double& n1,
                                           double& n2, double& n3, double& L, double& V) {
    const unsigned long long S = 0x8000000000000000ull;
    const unsigned long long ux = (unsigned long long)__double_as_longlong(nx) & ~S;
    const unsigned long long uy = (unsigned long long)__double_as_longlong(ny) & ~S;
    const unsigned long long uz = (unsigned long long)__double_as_longlong(nz) & ~S;
    const unsigned long long lo = ux < uy ? ux : uy, hi = ux < uy ? uy : ux;
    const unsigned long long b1 = lo < uz ? lo : uz, b3 = hi > uz ? hi : uz;
    n1 = __longlong_as_double((long long)b1);
    n3 = __longlong_as_double((long long)b3);
    n2 = __longlong_as_double((long long)(ux ^ uy ^ uz ^ b1 ^ b3));
    L = (__longlong_as_double((long long)ux) + __longlong_as_double((long long)uy)) +
        __longlong_as_double((long long)uz);
    const unsigned long long bv = (unsigned long long)__double_as_longlong(V0), va = bv & ~S;
    const unsigned long long bl = (unsigned long long)__double_as_longlong(L);
    // 0 <= V0 <= 1 (-0 accepted, NaN refused) and 0 < L <= 3
    const bool ok = ((bv >> 63) == 0ull || va == 0ull) && va <= 0x3FF0000000000000ull && bl != 0ull &&
                    bl <= 0x4008000000000000ull;
    V = va <= 0x3FE0000000000000ull ? __longlong_as_double((long long)va) : 1.0 - V0;
    return ok;
}

// |h| with the sign of V0 - 1/2 (+ for V0 >= 1/2), on the bits.
__device__ __forceinline__ double sign_of_side(double h, double V0) {
    const unsigned long long S = 0x8000000000000000ull;
    const unsigned long long va = (unsigned long long)__double_as_longlong(V0) & ~S;
    const unsigned long long m = (unsigned long long)__double_as_longlong(h) & ~S;
    return __longlong_as_double((long long)(va >= 0x3FE0000000000000ull ? m : (m | S)));
}

template <int METHOD, typename T, bool POLISH>
__global__ void __launch_bounds__(256)
k_plic_offset_compact(const T* __restrict__ nx, const T* __restrict__ ny, const T* __restrict__ nz,
                      const T* __restrict__ V0, T* __restrict__ d0, int64_t n, int vec_ok,
                      unsigned long long* invalid, void* /* round trip: not fused here */) {
    typedef typename Vec16<T>::type VT;
    constexpr int W = Vec16<T>::W;
    constexpr bool SZ = METHOD == M_SZ_ORIG || METHOD == M_SZ_OPT;
    typedef Solver<METHOD, T, false> S;
    // FP64: one task list for the block's 8 warps (heavy parts long enough
    // to repay the barriers; only the block's last round is partly empty);
    // FP32: one list per warp, no barriers
    constexpr bool POOL = sizeof(T) == 8;
    // FP64: the front end on the bit patterns (front_bits), except for nested
    // intervals (4-5 % faster for the other four solvers, 3 % slower there)
    constexpr bool BITS = sizeof(T) == 8 && METHOD != M_NESTED;
    __shared__ T task[8][32 * W][4];
    __shared__ int wtot[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    const int64_t nvec = vec_ok ? n / W : 0;
    // the loop bound is the same for the 32 lanes of a warp (votes below),
    // and with POOL for the whole block (barriers)
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (POOL ? 0 : warp * 32); i0 < nvec;
         i0 += wstride) {
        const int64_t i = i0 + (POOL ? threadIdx.x : lane);
        const bool have = i < nvec;
        T a[W], b[W], c[W], v[W];
        if (have) {
            to_arr(ld_stream(reinterpret_cast<const VT*>(nx) + i), a);
            to_arr(ld_stream(reinterpret_cast<const VT*>(ny) + i), b);
            to_arr(ld_stream(reinterpret_cast<const VT*>(nz) + i), c);
            to_arr(ld_stream(reinterpret_cast<const VT*>(V0) + i), v);
        }
        // front end (Sec. 2.1) and the closed-form cases
        T red[W][4], scale[W], res[W];
        unsigned need = 0u;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            res[j] = T(0);
            scale[j] = T(0);
            if (!have) continue;
            T n1, n2, n3, L, V;
            bool ok;
            if constexpr (BITS) {
                ok = front_bits(a[j], b[j], c[j], v[j], n1, n2, n3, L, V);
            } else {
                reduce_normal<T, false>(a[j], b[j], c[j], n1, n2, n3);
                L = fabs(a[j]) + fabs(b[j]) + fabs(c[j]);
                ok = (v[j] >= T(0)) && (v[j] <= T(1)) && (L > T(0)) && (L <= T(3));
            }
            if (!ok) {
                bad += 1;
                res[j] = T(NAN);
                continue;
            }
            if constexpr (!BITS) V = reduce_volume<T, false>(v[j]);
            if (SZ) {
                const T il = Fm<T>::rcp_(L);
                n1 *= il;
                n3 *= il;
                n2 = Fm<T>::fdim_(T(1), n1 + n3);
                scale[j] = L;
            } else {
                scale[j] = BITS ? L : T(1);             // with BITS, L/2 is the offset's origin
            }
            red[j][0] = V; red[j][1] = n1; red[j][2] = n2; red[j][3] = n3;
            T d;
            if (S::easy(V, n1, n2, n3, d)) res[j] = d;
            else need |= 1u << j;
        }
        // the heavy part on the packed task list of the warp (of the block)
        unsigned m[W];
        int pre[W + 1];
        pre[0] = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            m[j] = __ballot_sync(0xffffffffu, (need >> j) & 1u);
            pre[j + 1] = pre[j] + __popc(m[j]);
        }
        if constexpr (POOL) {
            T (*flat)[4] = &task[0][0];
            if (lane == 0) wtot[warp] = pre[W];
            __syncthreads();
            int base = 0, total = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const int x = wtot[w];
                base += w < warp ? x : 0;
                total += x;
            }
#pragma unroll
            for (int j = 0; j < W; ++j)
                if ((need >> j) & 1u) {
                    T* q = flat[base + pre[j] + __popc(m[j] & lt)];
                    q[0] = red[j][0]; q[1] = red[j][1]; q[2] = red[j][2]; q[3] = red[j][3];
                }
            __syncthreads();
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                T* q = flat[t];
                q[0] = S::hard(q[0], q[1], q[2], q[3]);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < W; ++j)
                if ((need >> j) & 1u) res[j] = flat[base + pre[j] + __popc(m[j] & lt)][0];
            __syncthreads();
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j)
                if ((need >> j) & 1u) {
                    T* q = task[warp][pre[j] + __popc(m[j] & lt)];
                    q[0] = red[j][0]; q[1] = red[j][1]; q[2] = red[j][2]; q[3] = red[j][3];
                }
            __syncwarp();
            for (int t = lane; t < pre[W]; t += 32) {
                T* q = task[warp][t];
                q[0] = S::hard(q[0], q[1], q[2], q[3]);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < W; ++j)
                if ((need >> j) & 1u) res[j] = task[warp][pre[j] + __popc(m[j] & lt)][0];
            __syncwarp();
        }
        // polish and the symmetry back to d0 (Eqs. 5-8)
        T r[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (!(scale[j] > T(0))) {
                r[j] = res[j];                       // invalid cell: NaN
                continue;
            }
            T x = res[j];
            if (POLISH) x = polish<T>(x, red[j][0], red[j][1], red[j][2], red[j][3]);
            if constexpr (BITS) {
                // the sign of V0 - 1/2 on the bits (no FP64 subtraction)
                r[j] = sign_of_side(SZ ? scale[j] * (T(0.5) - x) : T(0.5) * scale[j] - x, v[j]);
            } else {
                if (SZ) r[j] = scale[j] * copysign(T(0.5) - x, v[j] - T(0.5));
                else r[j] = copysign(T(0.5) * (red[j][1] + red[j][2] + red[j][3]) - x, v[j] - T(0.5));
            }
        }
        if (have) st_stream(reinterpret_cast<VT*>(d0) + i, from_arr(r));
    }
    for (int64_t i = nvec * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += wstride)
        d0[i] = offset_cell<METHOD, T, POLISH, false>(nx[i], ny[i], nz[i], V0[i], bad);
    count_invalid(bad, invalid);
}

// The optimised SZ solution in FP32 (the paper's recommended solver, Sec.
// 2.5) on paired FP32 instructions: each thread takes 4 cells per step as two
// pairs.  Tail and unaligned cells go through the same pair code with the
// cell duplicated in both lanes, so every cell sees identical arithmetic.
// With ROUNDTRIP the forward volume of each stored d0 is written to vrt in
// the same pass (plic_offset_roundtrip); COUNT (an invalid-cell counter was
// given) keeps the per-cell count of invalid inputs, which otherwise costs
// instructions for nothing.
template <int METHOD, bool POLISH, bool ROUNDTRIP, bool COUNT>
__global__ void __launch_bounds__(256)
k_plic_offset_pair(const float* __restrict__ nx, const float* __restrict__ ny,
                   const float* __restrict__ nz, const float* __restrict__ V0,
                   float* __restrict__ d0, int64_t n, int vec_ok,
                   unsigned long long* invalid, float* __restrict__ vrt) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    const int64_t nvec = vec_ok ? n / 4 : 0;
    for (int64_t i = tid; i < nvec; i += stride) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(nx) + i);
        const float4 b = __ldcs(reinterpret_cast<const float4*>(ny) + i);
        const float4 c = __ldcs(reinterpret_cast<const float4*>(nz) + i);
        const float4 v = __ldcs(reinterpret_cast<const float4*>(V0) + i);
        float2 w0, w1;
        const float2 r0 = p2::offset_pair<METHOD, POLISH, ROUNDTRIP, COUNT>(
            make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y), make_float2(v.x, v.y),
            bad, &w0);
        const float2 r1 = p2::offset_pair<METHOD, POLISH, ROUNDTRIP, COUNT>(
            make_float2(a.z, a.w), make_float2(b.z, b.w), make_float2(c.z, c.w), make_float2(v.z, v.w),
            bad, &w1);
        __stcs(reinterpret_cast<float4*>(d0) + i, make_float4(r0.x, r0.y, r1.x, r1.y));
        if (ROUNDTRIP) __stcs(reinterpret_cast<float4*>(vrt) + i, make_float4(w0.x, w0.y, w1.x, w1.y));
    }
    for (int64_t i = nvec * 4 + tid; i < n; i += stride) {
        int bad2 = 0;
        float2 w;
        const float2 r = p2::offset_pair<METHOD, POLISH, ROUNDTRIP, COUNT>(
            make_float2(nx[i], nx[i]), make_float2(ny[i], ny[i]), make_float2(nz[i], nz[i]),
            make_float2(V0[i], V0[i]), bad2, &w);
        bad += bad2 >> 1;
        d0[i] = r.x;
        if (ROUNDTRIP) vrt[i] = w.x;
    }
    if (COUNT) count_invalid(bad, invalid);
}

// PLIC_FP64_REFINED: double in/out, FP32 solve + two FP64 Newton steps.
template <int METHOD>
__global__ void __launch_bounds__(256)
k_plic_offset_refined(const double* __restrict__ nx, const double* __restrict__ ny,
                      const double* __restrict__ nz, const double* __restrict__ V0,
                      double* __restrict__ d0, int64_t n, int vec_ok,
                      unsigned long long* invalid, void* /* round trip: not fused here */) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    const int64_t nvec = vec_ok ? n / 2 : 0;
    for (int64_t i = tid; i < nvec; i += stride) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(nx) + i);
        const double2 b = __ldcs(reinterpret_cast<const double2*>(ny) + i);
        const double2 c = __ldcs(reinterpret_cast<const double2*>(nz) + i);
        const double2 v = __ldcs(reinterpret_cast<const double2*>(V0) + i);
        const double r0 = offset_cell_refined<METHOD>(a.x, b.x, c.x, v.x, bad);
        const double r1 = offset_cell_refined<METHOD>(a.y, b.y, c.y, v.y, bad);
        __stcs(reinterpret_cast<double2*>(d0) + i, make_double2(r0, r1));
    }
    for (int64_t i = nvec * 2 + tid; i < n; i += stride)
        d0[i] = offset_cell_refined<METHOD>(nx[i], ny[i], nz[i], V0[i], bad);
    count_invalid(bad, invalid);
}

template <int METHOD, typename T, bool POLISH, bool FAITHFUL>
static const void* kptr() {
    return reinterpret_cast<const void*>(&k_plic_offset<METHOD, T, POLISH, FAITHFUL>);
}

template <int METHOD, typename T, bool POLISH>
static const void* cptr() {
    return reinterpret_cast<const void*>(&k_plic_offset_compact<METHOD, T, POLISH>);
}

// The default solvers run work-compacted (k_plic_offset_compact); the
// paper-literal ones keep one cell after the other per lane.
// In FP32 the optimised SZ, Kawano's SZ and the analytic solution take the
// paired kernel (k_plic_offset_pair, chosen in offset_entry); Kawano's SZ in
// FP32 is packed in no form here: its heavy part (one arccosine and one
// cosine on the FP32 pipes) is too short to repay the packing (measured 102
// against 130 G solves/s one cell after the other, on 2^26 cells), and only
// its faithful form reaches this function in FP32.  In FP64, and for the
// iterative solvers, packing wins (e.g. nested intervals FP32 27 -> 40, FP64
// SZ-opt 3.3 -> 4.5 G solves/s).
template <int METHOD>
static const void* pick(plic_precision p, bool faithful) {
    if (p == PLIC_FP64_REFINED) return reinterpret_cast<const void*>(&k_plic_offset_refined<METHOD>);
    if (p == PLIC_FP64)
        return faithful ? kptr<METHOD, double, false, true>() : cptr<METHOD, double, false>();
    const bool packed = !faithful && METHOD != M_SZ_ORIG;
    if (p == PLIC_FP32_POLISHED)
        return packed ? cptr<METHOD, float, true>()
                      : (faithful ? kptr<METHOD, float, true, true>() : kptr<METHOD, float, true, false>());
    return packed ? cptr<METHOD, float, false>()
                  : (faithful ? kptr<METHOD, float, false, true>() : kptr<METHOD, float, false, false>());
}

// The paired FP32 kernels (optimised SZ, analytic); *fused is set when the
// round-trip volume comes out of the same kernel.
template <int METHOD, bool COUNT>
static const void* pick_pair_c(bool polish, bool roundtrip) {
    if (polish)
        return roundtrip ? reinterpret_cast<const void*>(&k_plic_offset_pair<METHOD, true, true, COUNT>)
                         : reinterpret_cast<const void*>(&k_plic_offset_pair<METHOD, true, false, COUNT>);
    return roundtrip ? reinterpret_cast<const void*>(&k_plic_offset_pair<METHOD, false, true, COUNT>)
                     : reinterpret_cast<const void*>(&k_plic_offset_pair<METHOD, false, false, COUNT>);
}

template <int METHOD>
static const void* pick_pair(bool polish, bool roundtrip, bool count, bool* fused) {
    *fused = roundtrip;
    return count ? pick_pair_c<METHOD, true>(polish, roundtrip) : pick_pair_c<METHOD, false>(polish, roundtrip);
}

static plic_status offset_entry(const void* nx, const void* ny, const void* nz, const void* V0,
                                void* d0, void* vrt, int64_t n, plic_method m, plic_precision p,
                                uint32_t flags, int64_t* d_invalid_count, void* stream,
                                bool* fused, const char* who) {
    *fused = false;
    if (n < 0) return PLIC_ERR_ARG;
    if ((int)m < 0 || (int)m > 4 || (int)p < 0 || (int)p > 3) return PLIC_ERR_ARG;
    if (flags & ~(uint32_t)PLIC_FLAG_FAITHFUL) return PLIC_ERR_ARG;
    if (p == PLIC_FP64_REFINED && (flags & PLIC_FLAG_FAITHFUL)) return PLIC_ERR_UNSUPPORTED;
    if (n == 0) return PLIC_OK;
    if (!nx || !ny || !nz || !V0 || !d0) return PLIC_ERR_ARG;
    const bool dbl = p == PLIC_FP64 || p == PLIC_FP64_REFINED;
    const size_t es = dbl ? 8 : 4;
    if (!aligned(nx, es) || !aligned(ny, es) || !aligned(nz, es) || !aligned(V0, es) ||
        !aligned(d0, es) || (vrt && !aligned(vrt, es)) ||
        (d_invalid_count && !aligned(d_invalid_count, 8)))
        return PLIC_ERR_ALIGN;
    const int vec_ok = aligned(nx, 16) && aligned(ny, 16) && aligned(nz, 16) && aligned(V0, 16) &&
                       aligned(d0, 16) && (!vrt || aligned(vrt, 16));
    const bool faithful = (flags & PLIC_FLAG_FAITHFUL) != 0;
    const void* k = nullptr;
    switch (m) {
        case PLIC_ANALYTIC:
            k = (!dbl && !faithful) ? pick_pair<M_ANALYTIC>(p == PLIC_FP32_POLISHED, vrt != nullptr,
                                                            d_invalid_count != nullptr, fused)
                                    : pick<M_ANALYTIC>(p, faithful);
            break;
        case PLIC_SZ_ORIG:
            k = (!dbl && !faithful) ? pick_pair<M_SZ_ORIG>(p == PLIC_FP32_POLISHED, vrt != nullptr,
                                                           d_invalid_count != nullptr, fused)
                                    : pick<M_SZ_ORIG>(p, faithful);
            break;
        case PLIC_SZ_OPT:
            k = (!dbl && !faithful) ? pick_pair<M_SZ_OPT>(p == PLIC_FP32_POLISHED, vrt != nullptr,
                                                          d_invalid_count != nullptr, fused)
                                    : pick<M_SZ_OPT>(p, faithful);
            break;
        case PLIC_NEWTON: k = pick<M_NEWTON>(p, faithful); break;
        case PLIC_NESTED: k = pick<M_NESTED>(p, faithful); break;
    }
    const int threads = 256;
    const int W = dbl ? 2 : 4;
    const int64_t work = vec_ok ? (n + W - 1) / W : n;
    const int grid = stream_grid(k, threads, work);
    unsigned long long* inv = reinterpret_cast<unsigned long long*>(d_invalid_count);
    void* args[] = {(void*)&nx, (void*)&ny, (void*)&nz, (void*)&V0, (void*)&d0,
                    (void*)&n, (void*)&vec_ok, (void*)&inv, (void*)&vrt};
    cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(threads), args, 0, as_stream(stream));
    if (e != cudaSuccess) {
        set_last_error(who, e);
        return PLIC_ERR_CUDA;
    }
    return PLIC_OK;
}

}  // namespace plic

extern "C" plic_status plic_offset(const void* nx, const void* ny, const void* nz,
                                   const void* V0, void* d0, int64_t n, plic_method m,
                                   plic_precision p, uint32_t flags, int64_t* d_invalid_count,
                                   void* stream) {
    bool fused;
    return plic::offset_entry(nx, ny, nz, V0, d0, nullptr, n, m, p, flags, d_invalid_count, stream,
                              &fused, "plic_offset");
}

extern "C" plic_status plic_offset_roundtrip(const void* nx, const void* ny, const void* nz,
                                             const void* V0, void* d0, void* V0_rt, int64_t n,
                                             plic_method m, plic_precision p, uint32_t flags,
                                             int64_t* d_invalid_count, void* stream) {
    if (n > 0 && !V0_rt) return PLIC_ERR_ARG;
    bool fused;
    plic_status s = plic::offset_entry(nx, ny, nz, V0, d0, V0_rt, n, m, p, flags, d_invalid_count,
                                       stream, &fused, "plic_offset_roundtrip");
    if (s != PLIC_OK || fused || n == 0) return s;
    const plic_precision vp = (p == PLIC_FP64 || p == PLIC_FP64_REFINED) ? PLIC_FP64 : PLIC_FP32;
    return plic_volume(nx, ny, nz, d0, V0_rt, n, vp, stream);
}
