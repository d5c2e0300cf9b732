// vof_curvature.cu -- curvature over interface-cell lists (Sec. 4.2), for one
// field (vof_curvature) and for many fields in one persistent launch
// (vof_curvature_batched).
//
// One thread per interface cell.  Consecutive list entries are mostly x-
// neighbours (the list is in ascending cell order), so a warp's 27-point
// stencils overlap in 3 x 3 rows of ~34 consecutive floats: the gathers hit L1.
// The work per cell is dominated by up to 27 PLIC solves (the paper's
// observation that PLIC is the main cost) and the 5x5 solve.
#include "host_common.h"
#include "vof_curvature.cuh"

namespace plic {

template <int METHOD, int FIT>
__global__ void __launch_bounds__(128)
k_vof_curvature(const float* __restrict__ phi, int nx, int ny, const int32_t* __restrict__ idx,
                int64_t n, const int64_t* __restrict__ d_n, float* __restrict__ kappa,
                uint32_t flags) {
    int64_t lim = n;
    if (d_n) {
        const int64_t dn = *d_n;
        lim = dn < n ? dn : n;
    }
    const int64_t nxy = (int64_t)nx * ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lim;
         k += (int64_t)gridDim.x * blockDim.x) {
        const CurvOut o = curvature_cell<METHOD, FIT>(phi, (int64_t)__ldg(idx + k), nx, nxy, flags);
        kappa[k] = o.kappa;
    }
}

// Persistent batched kernel: blocks claim chunks of the concatenated interface
// lists from a ticket counter and stop when the tickets pass the total.
template <int METHOD, int FIT>
__global__ void __launch_bounds__(128)
k_vof_curvature_batched(const vof_field* __restrict__ fields, const int64_t* __restrict__ prefix,
                        int n_fields, int64_t total, int chunk,
                        unsigned long long* __restrict__ ticket, uint32_t flags) {
    __shared__ long long s_start;
    for (;;) {
        if (threadIdx.x == 0) s_start = (long long)atomicAdd(ticket, (unsigned long long)chunk);
        __syncthreads();
        const int64_t start = s_start;
        __syncthreads();
        if (start >= total) break;
        const int64_t end = start + chunk < total ? start + chunk : total;
        for (int64_t g = start + threadIdx.x; g < end; g += blockDim.x) {
            // field f with prefix[f] <= g < prefix[f+1]
            int lo = 0, hi = n_fields - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(prefix + mid) <= g) lo = mid; else hi = mid - 1;
            }
            const vof_field& F = fields[lo];
            const int64_t k = g - __ldg(prefix + lo);
            const int64_t nxy = (int64_t)F.nx * F.ny;
            const CurvOut o = curvature_cell<METHOD, FIT>(F.phi, (int64_t)__ldg(F.idx + k), F.nx, nxy, flags);
            F.kappa[k] = o.kappa;
        }
    }
}

template <int METHOD>
static const void* pick_single(int fit) {
    switch (fit) {
        case FIT_FP32: return reinterpret_cast<const void*>(&k_vof_curvature<METHOD, FIT_FP32>);
        case FIT_DF32: return reinterpret_cast<const void*>(&k_vof_curvature<METHOD, FIT_DF32>);
        default: return reinterpret_cast<const void*>(&k_vof_curvature<METHOD, FIT_FP64>);
    }
}

template <int METHOD>
static const void* pick_batched(int fit) {
    switch (fit) {
        case FIT_FP32: return reinterpret_cast<const void*>(&k_vof_curvature_batched<METHOD, FIT_FP32>);
        case FIT_DF32: return reinterpret_cast<const void*>(&k_vof_curvature_batched<METHOD, FIT_DF32>);
        default: return reinterpret_cast<const void*>(&k_vof_curvature_batched<METHOD, FIT_FP64>);
    }
}

static int fit_mode(uint32_t flags) {
    return (flags & PLIC_FLAG_FIT_DF32) ? FIT_DF32 : (flags & PLIC_FLAG_FIT_FP32) ? FIT_FP32 : FIT_FP64;
}

static const void* select(bool batched, plic_method m, int fit) {
    switch (m) {
        case PLIC_ANALYTIC: return batched ? pick_batched<M_ANALYTIC>(fit) : pick_single<M_ANALYTIC>(fit);
        case PLIC_SZ_ORIG: return batched ? pick_batched<M_SZ_ORIG>(fit) : pick_single<M_SZ_ORIG>(fit);
        case PLIC_SZ_OPT: return batched ? pick_batched<M_SZ_OPT>(fit) : pick_single<M_SZ_OPT>(fit);
        case PLIC_NEWTON: return batched ? pick_batched<M_NEWTON>(fit) : pick_single<M_NEWTON>(fit);
        case PLIC_NESTED: return batched ? pick_batched<M_NESTED>(fit) : pick_single<M_NESTED>(fit);
    }
    return nullptr;
}

static const uint32_t kCurvFlags = PLIC_FLAG_POINT_CENTROID | PLIC_FLAG_KAPPA_PAPER_SIGN |
                                   PLIC_FLAG_FIT_FP32 | PLIC_FLAG_FIT_DF32;

}  // namespace plic

extern "C" plic_status vof_curvature(const float* phi, int nx, int ny, int nz, const int32_t* idx,
                                     int64_t n_iface, const int64_t* d_n_iface, float* kappa,
                                     plic_method m, uint32_t flags, void* stream) {
    using namespace plic;
    if (nx < 3 || ny < 3 || nz < 3 || n_iface < 0) return PLIC_ERR_ARG;
    if ((int)m < 0 || (int)m > 4 || (flags & ~kCurvFlags)) return PLIC_ERR_ARG;
    if ((flags & PLIC_FLAG_FIT_FP32) && (flags & PLIC_FLAG_FIT_DF32)) return PLIC_ERR_ARG;
    if (n_iface == 0) return PLIC_OK;
    if (!phi || !idx || !kappa) return PLIC_ERR_ARG;
    if (!aligned(phi, 4) || !aligned(idx, 4) || !aligned(kappa, 4) || (d_n_iface && !aligned(d_n_iface, 8)))
        return PLIC_ERR_ALIGN;
    const void* k = select(false, m, fit_mode(flags));
    const int threads = 128;
    const int grid = stride_grid(k, threads, n_iface);
    void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&idx, (void*)&n_iface,
                    (void*)&d_n_iface, (void*)&kappa, (void*)&flags};
    cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(threads), args, 0, as_stream(stream));
    if (e != cudaSuccess) { set_last_error("vof_curvature", e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}

extern "C" plic_status vof_curvature_batched(const vof_field* fields, int n_fields,
                                             const vof_tuning* tuning, plic_method m,
                                             uint32_t flags, void* workspace, size_t ws_bytes,
                                             void* stream) {
    using namespace plic;
    if (n_fields < 0 || (int)m < 0 || (int)m > 4 || (flags & ~kCurvFlags)) return PLIC_ERR_ARG;
    if ((flags & PLIC_FLAG_FIT_FP32) && (flags & PLIC_FLAG_FIT_DF32)) return PLIC_ERR_ARG;
    if (n_fields == 0) return PLIC_OK;
    if (!fields || !workspace) return PLIC_ERR_ARG;
    if (ws_bytes < plic_workspace_bytes(PLIC_WS_BATCHED, n_fields)) return PLIC_ERR_ARG;
    if (!aligned(workspace, 256)) return PLIC_ERR_ALIGN;
    int threads = 128, chunk = 512, bps = 0;
    if (tuning) {
        threads = tuning->block_threads;
        chunk = tuning->cells_per_chunk;
        bps = tuning->blocks_per_sm;
        if (threads < 32 || threads > 1024 || (threads & 31) || chunk < 1 || bps < 0)
            return PLIC_ERR_ARG;
        if (threads > 128) return PLIC_ERR_UNSUPPORTED;     // kernels are built for <= 128
    }
    // host-side prefix of the list lengths and argument checks
    const size_t nf = (size_t)n_fields;
    int64_t* pre = (int64_t*)malloc((nf + 1) * sizeof(int64_t));
    if (!pre) return PLIC_ERR_ARG;
    pre[0] = 0;
    for (size_t i = 0; i < nf; ++i) {
        const vof_field& F = fields[i];
        if (F.nx < 3 || F.ny < 3 || F.nz < 3 || F.n_iface < 0 ||
            (F.n_iface > 0 && (!F.phi || !F.idx || !F.kappa))) { free(pre); return PLIC_ERR_ARG; }
        if (!aligned(F.phi, 4) || !aligned(F.idx, 4) || !aligned(F.kappa, 4)) { free(pre); return PLIC_ERR_ALIGN; }
        pre[i + 1] = pre[i] + F.n_iface;
    }
    const int64_t total = pre[nf];
    char* ws = reinterpret_cast<char*>(workspace);
    vof_field* d_fields = reinterpret_cast<vof_field*>(ws);
    const size_t off_pre = (nf * sizeof(vof_field) + 255) / 256 * 256;
    int64_t* d_pre = reinterpret_cast<int64_t*>(ws + off_pre);
    const size_t off_tk = off_pre + ((nf + 1) * sizeof(int64_t) + 255) / 256 * 256;
    unsigned long long* d_ticket = reinterpret_cast<unsigned long long*>(ws + off_tk);
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(d_fields, fields, nf * sizeof(vof_field), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pre, pre, (nf + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), s);
    // the pageable source buffers are staged by the time the copies return
    free(pre);
    if (e != cudaSuccess) { set_last_error("vof_curvature_batched", e); return PLIC_ERR_CUDA; }
    if (total == 0) return PLIC_OK;
    const void* k = select(true, m, fit_mode(flags));
    const int occ = blocks_per_sm(k, threads, 0);
    const int per_sm = bps > 0 ? (bps < occ ? bps : occ) : occ;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t need = (total + chunk - 1) / chunk;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    int n_f = n_fields;
    void* args[] = {(void*)&d_fields, (void*)&d_pre, (void*)&n_f, (void*)&total, (void*)&chunk,
                    (void*)&d_ticket, (void*)&flags};
    e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(threads), args, 0, s);
    if (e != cudaSuccess) { set_last_error("vof_curvature_batched", e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}
