// plic_offset_bulk.cu -- the optimised-SZ FP32 solve (plic_offset and
// plic_offset_roundtrip with PLIC_SZ_OPT, FP32 / FP32_POLISHED, 16-byte
// aligned arrays) with its inputs staged through shared memory by bulk
// asynchronous copies.
//
// Each block owns every gridDim.x-th tile of BK_TILE cells.  One thread issues,
// per tile, four cp.async.bulk copies (nx, ny, nz, V0: 4 KB each) into one of
// BK_STAGES shared-memory stages, completing on that stage's mbarrier (expected
// transaction bytes); all threads wait on the barrier, solve their four cells
// from shared memory with the paired arithmetic of plic_pair.cuh, store d0 (and
// the round-trip volume) with streaming stores, and release the stage, which is
// then refilled with the tile BK_STAGES ahead.  The loads of the next tiles are
// thus in flight while the current one is solved, without holding them in
// registers.
//
// Every mbarrier wait is bounded (BK_SPIN polls).  A wait that gives up is
// counted in a device word (read and cleared by plic_device_check); the block
// then waits, again bounded, for its copies still in flight and returns.
#include <mutex>

#include "host_common.h"
#include "plic_pair.cuh"

namespace plic {

constexpr int BK_THREADS = 256;
constexpr int BK_TILE = 1024;                     // cells per stage: 4 per thread
constexpr int BK_STAGES = 3;
constexpr unsigned BK_SPIN = 1u << 22;            // polls before a wait gives up
constexpr size_t BK_SMEM = (size_t)BK_STAGES * 4 * BK_TILE * sizeof(float);

__device__ unsigned g_bulk_timeouts;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy; bytes a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    for (unsigned it = 0; it < BK_SPIN; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <bool POLISH, bool ROUNDTRIP>
__global__ void __launch_bounds__(BK_THREADS)
k_plic_offset_sz_opt_bulk(const float* __restrict__ nx, const float* __restrict__ ny,
                          const float* __restrict__ nz, const float* __restrict__ V0,
                          float* __restrict__ d0, int64_t n, unsigned long long* invalid,
                          float* __restrict__ vrt) {
    extern __shared__ __align__(128) float buf[];  // [stage][array][BK_TILE]
    __shared__ uint64_t bar[BK_STAGES];
    const int64_t n4 = n & ~(int64_t)3;            // cells in whole float4s
    const int64_t ntiles = (n4 + BK_TILE - 1) / BK_TILE;
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const float* src[4] = {nx, ny, nz, V0};
    if (threadIdx.x == 0) {
        for (int s = 0; s < BK_STAGES; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // thread 0: load local tile k into stage k % BK_STAGES
    auto issue = [&](int64_t k) {
        const int s = (int)(k % BK_STAGES);
        const int64_t c0 = ((int64_t)blockIdx.x + k * gridDim.x) * BK_TILE;
        const int64_t cnt = n4 - c0 < BK_TILE ? n4 - c0 : BK_TILE;
        const unsigned bytes = (unsigned)(cnt * sizeof(float));
        mbar_arrive_expect_tx(&bar[s], 4 * bytes);
#pragma unroll
        for (int a = 0; a < 4; ++a) bulk_load(buf + (s * 4 + a) * BK_TILE, src[a] + c0, bytes, &bar[s]);
    };
    if (threadIdx.x == 0)
        for (int64_t k = 0; k < mine && k < BK_STAGES; ++k) issue(k);
    int bad = 0;
    for (int64_t k = 0; k < mine; ++k) {
        const int s = (int)(k % BK_STAGES);
        const bool ok = mbar_wait(&bar[s], (unsigned)((k / BK_STAGES) & 1));
        if (__syncthreads_or(!ok)) {
            // give up: record it, let the copies in flight land, return
            if (threadIdx.x == 0) {
                atomicAdd(&g_bulk_timeouts, 1u);
                for (int64_t q = k; q < mine && q < k + BK_STAGES; ++q)
                    mbar_wait(&bar[q % BK_STAGES], (unsigned)((q / BK_STAGES) & 1));
            }
            __syncthreads();
            return;
        }
        const int64_t c0 = ((int64_t)blockIdx.x + k * gridDim.x) * BK_TILE;
        const int64_t cnt = n4 - c0 < BK_TILE ? n4 - c0 : BK_TILE;
        const int q = 4 * threadIdx.x;
        if (q < cnt) {
            const float* st = buf + s * 4 * BK_TILE;
            const float4 a = *reinterpret_cast<const float4*>(st + q);
            const float4 b = *reinterpret_cast<const float4*>(st + BK_TILE + q);
            const float4 c = *reinterpret_cast<const float4*>(st + 2 * BK_TILE + q);
            const float4 v = *reinterpret_cast<const float4*>(st + 3 * BK_TILE + q);
            float2 w0, w1;
            const float2 r0 = p2::offset_sz_opt<POLISH, ROUNDTRIP>(
                make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y),
                make_float2(v.x, v.y), bad, &w0);
            const float2 r1 = p2::offset_sz_opt<POLISH, ROUNDTRIP>(
                make_float2(a.z, a.w), make_float2(b.z, b.w), make_float2(c.z, c.w),
                make_float2(v.z, v.w), bad, &w1);
            __stcs(reinterpret_cast<float4*>(d0 + c0 + q), make_float4(r0.x, r0.y, r1.x, r1.y));
            if (ROUNDTRIP)
                __stcs(reinterpret_cast<float4*>(vrt + c0 + q), make_float4(w0.x, w0.y, w1.x, w1.y));
        }
        __syncthreads();                            // stage s is free again
        if (threadIdx.x == 0 && k + BK_STAGES < mine) issue(k + BK_STAGES);
    }
    // the last n % 4 cells: block 0, one lane pair each
    if (blockIdx.x == 0 && n4 + threadIdx.x < n) {
        const int64_t i = n4 + threadIdx.x;
        int bad2 = 0;
        float2 w;
        const float2 r = p2::offset_sz_opt<POLISH, ROUNDTRIP>(
            make_float2(nx[i], nx[i]), make_float2(ny[i], ny[i]), make_float2(nz[i], nz[i]),
            make_float2(V0[i], V0[i]), bad2, &w);
        bad += bad2 >> 1;
        d0[i] = r.x;
        if (ROUNDTRIP) vrt[i] = w.x;
    }
    if (invalid) {
        const unsigned mask = __activemask();
        const int tot = __reduce_add_sync(mask, bad);
        if ((int)(threadIdx.x & 31) == __ffs(mask) - 1 && tot > 0) atomicAdd(invalid, (unsigned long long)tot);
    }
}

// Launch of the staged kernel (the caller has checked that all arrays are
// 16-byte aligned).  One wave: as many blocks as fit on the GPU with the
// staging buffers, at most one per tile.
plic_status launch_sz_opt_bulk(const float* nx, const float* ny, const float* nz, const float* V0,
                               float* d0, float* vrt, int64_t n, bool polish,
                               unsigned long long* invalid, void* stream, const char* who) {
    const void* k = polish ? (vrt ? reinterpret_cast<const void*>(&k_plic_offset_sz_opt_bulk<true, true>)
                                  : reinterpret_cast<const void*>(&k_plic_offset_sz_opt_bulk<true, false>))
                           : (vrt ? reinterpret_cast<const void*>(&k_plic_offset_sz_opt_bulk<false, true>)
                                  : reinterpret_cast<const void*>(&k_plic_offset_sz_opt_bulk<false, false>));
    // the 48 KB of staging buffers plus the barriers need the dynamic
    // shared-memory opt-in, once per kernel and device
    static std::mutex mu;
    static bool attr_set[64][4] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int ki = (polish ? 2 : 0) + (vrt ? 1 : 0);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 0 || dev >= 64 || !attr_set[dev][ki]) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BK_SMEM);
            if (e != cudaSuccess) { set_last_error(who, e); return PLIC_ERR_CUDA; }
            if (dev >= 0 && dev < 64) attr_set[dev][ki] = true;
        }
    }
    const int64_t tiles = ((n & ~(int64_t)3) + BK_TILE - 1) / BK_TILE;
    int64_t grid = (int64_t)sm_count() * blocks_per_sm(k, BK_THREADS, BK_SMEM);
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    void* args[] = {(void*)&nx, (void*)&ny, (void*)&nz, (void*)&V0, (void*)&d0,
                    (void*)&n, (void*)&invalid, (void*)&vrt};
    cudaError_t e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(BK_THREADS), args, BK_SMEM,
                                     as_stream(stream));
    if (e != cudaSuccess) { set_last_error(who, e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}

}  // namespace plic

extern "C" plic_status plic_device_check(void) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { plic::set_last_error("plic_device_check", e); return PLIC_ERR_CUDA; }
    unsigned t = 0, zero = 0;
    e = cudaMemcpyFromSymbol(&t, plic::g_bulk_timeouts, sizeof t);
    if (e == cudaSuccess && t) e = cudaMemcpyToSymbol(plic::g_bulk_timeouts, &zero, sizeof zero);
    if (e != cudaSuccess) { plic::set_last_error("plic_device_check", e); return PLIC_ERR_CUDA; }
    return t ? PLIC_ERR_TIMEOUT : PLIC_OK;
}
