// paper_bench.cu -- the paper's accuracy/throughput harness (Sec. 2.5) as a
// kernel: each thread takes one normal and solves PLIC for L equally spaced
// fill levels V0_j = j/(L-1) in series, accumulating the round-trip error
// E = |V0(n, d0(V0_j, n)) - V0_j| (Eqs. 27-28, with the forward volume of
// Eq. 10).  The "blank run" replaces the solve by d0 = V0_j - 1/2 and keeps the
// loads, the forward volume and the stores of the error sum (Sec. 2.5); its
// time is what the paper subtracts.
//
// The normal is loop-invariant, so everything that depends on it alone is
// computed once per thread: for the optimised SZ solution in FP32 with the
// polish this is the per-normal constant set of CellPlic<M_SZ_OPT>.
//
// Normals are taken in a grid-stride loop on up to 16 waves of resident blocks
// (stream_grid; 13 % faster than one persistent wave for 2^24 normals x 256
// levels), and each block adds its error sum with one atomic.
#include "host_common.h"
#include "vof_curvature.cuh"

namespace plic {

template <int METHOD, typename T, bool POLISH, bool HOIST>
__global__ void __launch_bounds__(256)
k_paper_bench(const T* __restrict__ nx, const T* __restrict__ ny, const T* __restrict__ nz,
              int64_t n, int L, int blank, double* __restrict__ err_sum) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const T step = T(1) / T(L - 1);
    double acc = 0.0;
    for (int64_t i = tid; i < n; i += stride) {
        const T a = nx[i], b = ny[i], c = nz[i];
        T e = T(0);
        if (HOIST) {
            CellPlic<M_SZ_OPT> pl;
            pl.prepare((float)a, (float)b, (float)c);
#pragma unroll 4
            for (int j = 0; j < L; ++j) {
                const T V0 = T(j) * step;
                const T d0 = blank ? V0 - T(0.5) : (T)pl.offset((float)V0);
                e += fabs(volume_cell<T>(a, b, c, d0) - V0);
            }
        } else {
            int bad = 0;
#pragma unroll 4
            for (int j = 0; j < L; ++j) {
                const T V0 = T(j) * step;
                const T d0 = blank ? V0 - T(0.5) : offset_cell<METHOD, T, POLISH, false>(a, b, c, V0, bad);
                e += fabs(volume_cell<T>(a, b, c, d0) - V0);
            }
        }
        acc += (double)e;
    }
    // block sum, one atomic per block
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        atomicAdd(err_sum, s);
    }
}

template <int METHOD>
static const void* pick_bench(plic_precision p) {
    if (p == PLIC_FP64) return reinterpret_cast<const void*>(&k_paper_bench<METHOD, double, false, false>);
    if (p == PLIC_FP32_POLISHED) {
        if (METHOD == M_SZ_OPT) return reinterpret_cast<const void*>(&k_paper_bench<M_SZ_OPT, float, true, true>);
        return reinterpret_cast<const void*>(&k_paper_bench<METHOD, float, true, false>);
    }
    return reinterpret_cast<const void*>(&k_paper_bench<METHOD, float, false, false>);
}

}  // namespace plic

extern "C" plic_status plic_paper_benchmark(const void* nx, const void* ny, const void* nz,
                                            int64_t n_normals, int L, plic_method m,
                                            plic_precision p, int blank, double* d_err_sum,
                                            void* stream) {
    using namespace plic;
    if (n_normals < 0 || L < 2 || (int)m < 0 || (int)m > 4 || (int)p < 0 || (int)p > 2)
        return PLIC_ERR_ARG;
    if (!d_err_sum) return PLIC_ERR_ARG;
    if (n_normals == 0) return PLIC_OK;
    if (!nx || !ny || !nz) return PLIC_ERR_ARG;
    const size_t es = p == PLIC_FP64 ? 8 : 4;
    if (!aligned(nx, es) || !aligned(ny, es) || !aligned(nz, es) || !aligned(d_err_sum, 8))
        return PLIC_ERR_ALIGN;
    const void* k = nullptr;
    switch (m) {
        case PLIC_ANALYTIC: k = pick_bench<M_ANALYTIC>(p); break;
        case PLIC_SZ_ORIG: k = pick_bench<M_SZ_ORIG>(p); break;
        case PLIC_SZ_OPT: k = pick_bench<M_SZ_OPT>(p); break;
        case PLIC_NEWTON: k = pick_bench<M_NEWTON>(p); break;
        case PLIC_NESTED: k = pick_bench<M_NESTED>(p); break;
    }
    const int grid = stream_grid(k, 256, n_normals);
    void* args[] = {(void*)&nx, (void*)&ny, (void*)&nz, (void*)&n_normals, (void*)&L,
                    (void*)&blank, (void*)&d_err_sum};
    cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(256), args, 0, as_stream(stream));
    if (e != cudaSuccess) { set_last_error("plic_paper_benchmark", e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}
