// pipe_probe.cu -- throughput probes of the execution pipes the PLIC kernels
// use, for the compute side of their rooflines: FP32 FMA (scalar and paired),
// FP64 FMA, the MUFU functions (ex2/lg2, rsqrt, sin) and the FP64 library
// functions the FP64 solvers call (sqrt, division, cbrt, sin, cos, asin,
// acos, atan2).  Each thread runs PROBE_CHAINS independent dependency chains
// of one operation for `iters` rounds; the caller times the launch with CUDA
// events and divides the operation count (returned by the entry point) by it.
// The chains are kept inside their functions' ordinary domains (bounded
// values, no denormals, no NaN) so that no special-case path is timed, and
// their results are stored only when an impossible condition holds, so that
// the compiler keeps every operation.
//
// plic_read_probe is the memory-side counterpart: a plain streaming read of a
// float buffer, the fastest a pass that reads the buffer once can go from the
// cache state it finds (HBM after a flush, L2 for a buffer already there).
#include "host_common.h"

namespace plic {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

enum ProbeKind {
    PROBE_FFMA = 0,      // fmaf                          (1 FP32 operation)
    PROBE_FFMA2 = 1,     // __ffma2_rn                    (2 FP32 operations)
    PROBE_DFMA = 2,      // fma (double)                  (1 FP64 operation)
    PROBE_MUFU_EX2 = 3,  // ex2.approx then lg2.approx    (2 MUFU operations)
    PROBE_MUFU_RSQ = 4,  // rsqrtf                        (1 MUFU operation)
    PROBE_MUFU_SIN = 5,  // __sinf                        (1 MUFU operation)
    PROBE_D_SQRT = 6,    // sqrt(x + 1): one call and one add
    PROBE_D_DIV = 7,     // 1 / (x + 1): one division and one add
    PROBE_D_CBRT = 8,    // cbrt(x + 1): one call and one add
    PROBE_D_SIN = 9,
    PROBE_D_COS = 10,
    PROBE_D_ASIN = 11,   // asin(0.5 x): one call and one multiply
    PROBE_D_ACOS = 12,   // acos(0.5 x): one call and one multiply
    PROBE_D_ATAN2 = 13,
    PROBE_KINDS = 14
};

__device__ __forceinline__ float ex2a(float x) {
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2a(float x) {
    float r;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_pipe_probe(int iters, float seed, float* sink) {
    const float s = seed + 1e-3f * (float)(threadIdx.x & 7);
    if (KIND == PROBE_FFMA || KIND == PROBE_MUFU_EX2 || KIND == PROBE_MUFU_RSQ ||
        KIND == PROBE_MUFU_SIN) {
        float a[PROBE_CHAINS];
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = s + 0.125f * (float)j;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < PROBE_CHAINS; ++j) {
                if (KIND == PROBE_FFMA) a[j] = fmaf(a[j], 0.99999994f, 1e-7f);   // fixed point ~1.7
                if (KIND == PROBE_MUFU_EX2) a[j] = lg2a(ex2a(a[j]));            // stays near s
                if (KIND == PROBE_MUFU_RSQ) a[j] = rsqrtf(a[j]);                // tends to 1
                if (KIND == PROBE_MUFU_SIN) a[j] = __sinf(a[j]);                // stays in [-1, 1]
            }
        }
        float t = 0.0f;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j];
        if (t == -12345.678f) sink[0] = t;
    } else if (KIND == PROBE_FFMA2) {
        float2 a[PROBE_CHAINS];
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = make_float2(s + 0.125f * j, s - 0.125f * j);
        const float2 b = make_float2(0.99999994f, 0.99999994f), c = make_float2(1e-7f, 1e-7f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = __ffma2_rn(a[j], b, c);
        }
        float t = 0.0f;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j].x + a[j].y;
        if (t == -12345.678f) sink[0] = t;
    } else {
        double a[PROBE_CHAINS];
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (double)s + 0.0625 * j;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < PROBE_CHAINS; ++j) {
                const double x = a[j];
                if (KIND == PROBE_DFMA) a[j] = fma(x, 0.99999999999999989, 1e-16);
                if (KIND == PROBE_D_SQRT) a[j] = sqrt(x + 1.0);                  // tends to 1.62
                if (KIND == PROBE_D_DIV) a[j] = 1.0 / (x + 1.0);                 // tends to 0.62
                if (KIND == PROBE_D_CBRT) a[j] = cbrt(x + 1.0);                  // tends to 1.32
                if (KIND == PROBE_D_SIN) a[j] = sin(x);                          // in [-1, 1]
                if (KIND == PROBE_D_COS) a[j] = cos(x);                          // tends to 0.74
                if (KIND == PROBE_D_ASIN) a[j] = asin(0.5 * x);                  // tends to 0
                if (KIND == PROBE_D_ACOS) a[j] = acos(0.5 * x);                  // tends to 1.03
                if (KIND == PROBE_D_ATAN2) a[j] = atan2(x, 1.5);                 // tends to 0
            }
        }
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j];
        if (t == -12345.678) sink[0] = (float)t;
    }
}

template <int K>
static const void* probe_ptr() {
    return reinterpret_cast<const void*>(&k_pipe_probe<K>);
}

static const void* probe_kernel(int kind) {
    static const void* tab[PROBE_KINDS] = {
        probe_ptr<0>(), probe_ptr<1>(), probe_ptr<2>(),  probe_ptr<3>(),  probe_ptr<4>(),
        probe_ptr<5>(), probe_ptr<6>(), probe_ptr<7>(),  probe_ptr<8>(),  probe_ptr<9>(),
        probe_ptr<10>(), probe_ptr<11>(), probe_ptr<12>(), probe_ptr<13>()};
    return (kind >= 0 && kind < PROBE_KINDS) ? tab[kind] : nullptr;
}

}  // namespace plic

extern "C" plic_status plic_pipe_probe(int kind, int iters, float* d_sink, int64_t* ops,
                                       void* stream) {
    using namespace plic;
    const void* k = probe_kernel(kind);
    if (!k || iters < 1 || !d_sink || !ops) return PLIC_ERR_ARG;
    if (!aligned(d_sink, 4)) return PLIC_ERR_ALIGN;
    // enough resident warps per scheduler to cover the FMA and MUFU latencies
    const int per_sm = blocks_per_sm(k, PROBE_THREADS, 0);
    const int grid = sm_count() * (per_sm > 0 ? per_sm : 1);
    const int64_t per_round = (kind == PROBE_FFMA2 || kind == PROBE_MUFU_EX2) ? 2 : 1;
    *ops = (int64_t)grid * PROBE_THREADS * PROBE_CHAINS * (int64_t)iters * per_round;
    float seed = 0.3f;
    void* args[] = {(void*)&iters, (void*)&seed, (void*)&d_sink};
    cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(PROBE_THREADS), args, 0, as_stream(stream));
    if (e != cudaSuccess) {
        set_last_error("plic_pipe_probe", e);
        return PLIC_ERR_CUDA;
    }
    return PLIC_OK;
}

namespace plic {

constexpr int READ_THREADS = 256;
constexpr int READ_UNROLL = 4;          // 16-byte loads per thread and trip, issued together

// Sum of a float buffer that is written out only in an impossible case: every
// thread issues READ_UNROLL independent 16-byte loads per trip of a
// grid-stride loop over one wave of resident blocks (measured on GB300 as the
// fastest plain read both from HBM and from L2: 143 us for 1 GiB, 5.1 us for
// a 64 MiB buffer in L2; more blocks per launch are slower).
__global__ void __launch_bounds__(READ_THREADS)
k_read_probe(const float4* __restrict__ p, int64_t n4, const float* __restrict__ tail, int ntail,
             float* __restrict__ sink) {
    float s = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * READ_THREADS * READ_UNROLL;
    for (int64_t i = (int64_t)blockIdx.x * READ_THREADS * READ_UNROLL + threadIdx.x; i < n4; i += stride) {
        float4 v[READ_UNROLL];
#pragma unroll
        for (int u = 0; u < READ_UNROLL; ++u) {
            const int64_t j = i + (int64_t)u * READ_THREADS;
            v[u] = j < n4 ? __ldg(p + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < READ_UNROLL; ++u) s += (v[u].x + v[u].y) + (v[u].z + v[u].w);
    }
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) s += __ldg(tail + threadIdx.x);
    if (s == -1.2345e38f) sink[0] = s;
}

}  // namespace plic

extern "C" plic_status plic_read_probe(const float* buf, int64_t n, float* d_sink, void* stream) {
    using namespace plic;
    if (n < 0 || !d_sink || (n > 0 && !buf)) return PLIC_ERR_ARG;
    if ((buf && !aligned(buf, 16)) || !aligned(d_sink, 4)) return PLIC_ERR_ALIGN;
    if (n == 0) return PLIC_OK;
    const void* k = reinterpret_cast<const void*>(&k_read_probe);
    const int64_t n4 = n / 4;
    const int ntail = (int)(n - 4 * n4);
    const float4* p4 = reinterpret_cast<const float4*>(buf);
    const float* tail = buf + 4 * n4;
    const int per_sm = blocks_per_sm(k, READ_THREADS, 0);
    const int64_t need = (n4 + READ_THREADS * READ_UNROLL - 1) / (READ_THREADS * READ_UNROLL);
    int64_t grid = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    void* args[] = {(void*)&p4, (void*)&n4, (void*)&tail, (void*)&ntail, (void*)&d_sink};
    cudaError_t e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(READ_THREADS), args, 0, as_stream(stream));
    if (e != cudaSuccess) {
        set_last_error("plic_read_probe", e);
        return PLIC_ERR_CUDA;
    }
    return PLIC_OK;
}
