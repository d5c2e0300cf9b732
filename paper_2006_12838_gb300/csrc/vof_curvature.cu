// vof_curvature.cu -- curvature over interface-cell lists (Sec. 4.2), for one
// field (vof_curvature, vof_laplace_pressure) and for many fields in one
// persistent launch (vof_curvature_batched).
//
// Two layouts of the per-cell work: one thread per interface cell
// (vof_curvature_tpc.cu; every single-field call and the batched default)
// and eight lanes per cell (vof_curvature_coop.cuh; a batched tuning
// option).  Measured on GB300: the 56 478-cell list of the 256^3 curvature
// field in 12.5 us with one thread per cell against 33.3 us with eight lanes;
// 2.69 M cells of 64 fields in 0.33 ms against 1.11 ms; a 5 538-cell list in
// 8.6 us against 8.9 us.  The single-field entry keeps one layout for every
// list length, so that a cell's kappa does not depend on the list (or the
// buffer) it comes in.
#include "host_common.h"
#include "vof_curvature_coop.cuh"

namespace plic {

constexpr int CO_THREADS = 128;       // 4 warps per block
constexpr int CO_WARPS = CO_THREADS / 32;
static_assert(TPC_THREADS == CO_THREADS, "one block shape for both layouts");
// Layout of the batched kernel when the tuning leaves it open (lanes per cell).
constexpr int BATCHED_DEFAULT_LANES = 1;

// Persistent batched kernel: each warp claims tickets of `chunk` cells (a
// multiple of 32) of the concatenated interface lists from a device counter
// and stops when the tickets pass the total; no warp waits for another.
template <int METHOD, int FIT>
__global__ void __launch_bounds__(CO_THREADS)
k_vof_curvature_batched(const vof_field* __restrict__ fields, const int64_t* __restrict__ prefix,
                        int n_fields, int64_t total, int chunk,
                        unsigned long long* __restrict__ ticket, uint32_t flags) {
    __shared__ float smem[CO_WARPS][CO_BATCH * CO_VALS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ticket, (unsigned long long)chunk);
        const int64_t start = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        if (start >= total) break;
        const int64_t end = start + chunk < total ? start + chunk : total;
        for (int64_t b0 = start; b0 < end; b0 += CO_BATCH) {
            // lane l locates entry b0 + l: field (binary search on the prefix)
            // and position in that field's list
            const int64_t gi = b0 + lane;
            int f = 0;
            int64_t kk = 0;
            if (gi < end) {
                int lo = 0, hi = n_fields - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(prefix + mid) <= gi) lo = mid; else hi = mid - 1;
                }
                f = lo;
                kk = gi - __ldg(prefix + lo);
            }
            auto fetch = [&](int slot) {
                const int fs = __shfl_sync(0xffffffffu, f, slot);
                const long long ks = __shfl_sync(0xffffffffu, (long long)kk, slot);
                const vof_field& F = fields[fs];
                CoCell c;
                c.phi = F.phi; c.nx = F.nx; c.nxy = (int64_t)F.nx * F.ny;
                c.valid = b0 + slot < end;
                c.c = c.valid ? (int64_t)__ldg(F.idx + ks) : 0;
                c.out = F.kappa + ks;
                return c;
            };
            co_warp_batch<METHOD, FIT>(fetch, CO_BATCH, flags, 1.0f, smem[warp]);
        }
    }
}

#define PLIC_FIT_TABLE(K, M) \
    static const void* K##_tab[4] = { \
        reinterpret_cast<const void*>(&K<M, FIT_FP64>), reinterpret_cast<const void*>(&K<M, FIT_FP32>), \
        reinterpret_cast<const void*>(&K<M, FIT_DF32>), reinterpret_cast<const void*>(&K<M, FIT_AUTO>)};

template <int METHOD>
static const void* pick_batched(int fit) {
    PLIC_FIT_TABLE(k_vof_curvature_batched, METHOD)
    return k_vof_curvature_batched_tab[fit];
}

// Fit precision from the flags: one of FIT_FP32 / FIT_DF32 / FIT_FP64, or the
// adaptive default; -1 when more than one is set.
static int fit_mode(uint32_t flags) {
    const uint32_t f = flags & (PLIC_FLAG_FIT_FP32 | PLIC_FLAG_FIT_DF32 | PLIC_FLAG_FIT_FP64);
    if (f == 0) return FIT_AUTO;
    if (f == PLIC_FLAG_FIT_FP32) return FIT_FP32;
    if (f == PLIC_FLAG_FIT_DF32) return FIT_DF32;
    if (f == PLIC_FLAG_FIT_FP64) return FIT_FP64;
    return -1;
}

// The eight-lane batched kernel for a method and fit mode.
static const void* select_coop(plic_method m, int fit) {
    switch (m) {
        case PLIC_ANALYTIC: return pick_batched<M_ANALYTIC>(fit);
        case PLIC_SZ_ORIG: return pick_batched<M_SZ_ORIG>(fit);
        case PLIC_SZ_OPT: return pick_batched<M_SZ_OPT>(fit);
        case PLIC_NEWTON: return pick_batched<M_NEWTON>(fit);
        case PLIC_NESTED: return pick_batched<M_NESTED>(fit);
    }
    return nullptr;
}

static const uint32_t kCurvFlags = PLIC_FLAG_POINT_CENTROID | PLIC_FLAG_KAPPA_PAPER_SIGN |
                                   PLIC_FLAG_FIT_FP32 | PLIC_FLAG_FIT_DF32 | PLIC_FLAG_FIT_FP64 |
                                   PLIC_FLAG_NORMAL_CM | PLIC_FLAG_NEIGHBOR_NORMAL;

// vof_curvature and vof_laplace_pressure: out[k] = scale * kappa[k]
static plic_status curvature_entry(const float* phi, int nx, int ny, int nz, const int32_t* idx,
                                   int64_t n_iface, const int64_t* d_n_iface, float* out,
                                   plic_method m, uint32_t flags, float scale, void* stream,
                                   const char* who) {
    // fields of at most 2^31 - 1 cells (int32 list entries; 32-bit stencil offsets)
    if (nx < 3 || ny < 3 || nz < 3 || n_iface < 0 || (int64_t)nx * ny * nz > 2147483647LL)
        return PLIC_ERR_ARG;
    if ((int)m < 0 || (int)m > 4 || (flags & ~kCurvFlags) || fit_mode(flags) < 0) return PLIC_ERR_ARG;
    if (n_iface == 0) return PLIC_OK;
    if (!phi || !idx || !out) return PLIC_ERR_ARG;
    if (!aligned(phi, 4) || !aligned(idx, 4) || !aligned(out, 4) || (d_n_iface && !aligned(d_n_iface, 8)))
        return PLIC_ERR_ALIGN;
    if (flags & PLIC_FLAG_NEIGHBOR_NORMAL)
        return launch_curvature_nn(phi, nx, ny, nz, idx, n_iface, d_n_iface, out, m, flags,
                                   fit_mode(flags), scale, stream, who);
    const void* k = select_tpc(false, m, fit_mode(flags));
    if (!k) return PLIC_ERR_ARG;
    const int grid = stride_grid(k, TPC_THREADS, n_iface);
    void* args[] = {(void*)&phi, (void*)&nx, (void*)&ny, (void*)&idx, (void*)&n_iface,
                    (void*)&d_n_iface, (void*)&out, (void*)&flags, (void*)&scale};
    // a programmatic dependent launch: the list usually comes from the
    // compaction launched just before on the same stream
    cudaError_t e = launch_after(k, dim3(grid), dim3(TPC_THREADS), args, as_stream(stream));
    if (e != cudaSuccess) { set_last_error(who, e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}

}  // namespace plic

extern "C" plic_status vof_curvature(const float* phi, int nx, int ny, int nz, const int32_t* idx,
                                     int64_t n_iface, const int64_t* d_n_iface, float* kappa,
                                     plic_method m, uint32_t flags, void* stream) {
    return plic::curvature_entry(phi, nx, ny, nz, idx, n_iface, d_n_iface, kappa, m, flags, 1.0f,
                                 stream, "vof_curvature");
}

extern "C" plic_status vof_laplace_pressure(const float* phi, int nx, int ny, int nz,
                                            const int32_t* idx, int64_t n_iface,
                                            const int64_t* d_n_iface, float sigma, float* dp,
                                            plic_method m, uint32_t flags, void* stream) {
    if (!(sigma == sigma)) return PLIC_ERR_ARG;
    return plic::curvature_entry(phi, nx, ny, nz, idx, n_iface, d_n_iface, dp, m, flags,
                                 2.0f * sigma, stream, "vof_laplace_pressure");
}

extern "C" plic_status vof_curvature_batched(const vof_field* fields, int n_fields,
                                             const vof_tuning* tuning, plic_method m,
                                             uint32_t flags, void* workspace, size_t ws_bytes,
                                             void* stream) {
    using namespace plic;
    if (n_fields < 0 || (int)m < 0 || (int)m > 4 || (flags & ~kCurvFlags) || fit_mode(flags) < 0)
        return PLIC_ERR_ARG;
    if (flags & PLIC_FLAG_NEIGHBOR_NORMAL) return PLIC_ERR_UNSUPPORTED;
    if (n_fields == 0) return PLIC_OK;
    if (!fields || !workspace) return PLIC_ERR_ARG;
    if (ws_bytes < plic_workspace_bytes(PLIC_WS_BATCHED, n_fields)) return PLIC_ERR_ARG;
    if (!aligned(workspace, 256)) return PLIC_ERR_ALIGN;
    int threads = CO_THREADS, chunk = 128, bps = 0, lanes = 0;
    if (tuning) {
        threads = tuning->block_threads;
        chunk = tuning->cells_per_chunk;
        bps = tuning->blocks_per_sm;
        lanes = tuning->lanes_per_cell;
        if (threads < 32 || threads > 1024 || (threads & 31) || chunk < 1 || bps < 0 ||
            (lanes != 0 && lanes != 1 && lanes != 8))
            return PLIC_ERR_ARG;
        if (threads != CO_THREADS) return PLIC_ERR_UNSUPPORTED;   // built for 4 warps per block
    }
    if (lanes == 0) lanes = BATCHED_DEFAULT_LANES;
    chunk = (chunk + CO_BATCH - 1) / CO_BATCH * CO_BATCH;     // whole warp batches
    // host-side prefix of the list lengths and argument checks
    const size_t nf = (size_t)n_fields;
    int64_t* pre = (int64_t*)malloc((nf + 1) * sizeof(int64_t));
    if (!pre) return PLIC_ERR_ARG;
    pre[0] = 0;
    for (size_t i = 0; i < nf; ++i) {
        const vof_field& F = fields[i];
        if (F.nx < 3 || F.ny < 3 || F.nz < 3 || F.n_iface < 0 ||
            (int64_t)F.nx * F.ny * F.nz > 2147483647LL ||
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
    const void* k = lanes == 1 ? select_tpc(true, m, fit_mode(flags)) : select_coop(m, fit_mode(flags));
    if (!k) return PLIC_ERR_ARG;
    const int occ = blocks_per_sm(k, threads, 0);
    const int per_sm = bps > 0 ? (bps < occ ? bps : occ) : occ;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t need = ((total + chunk - 1) / chunk + CO_WARPS - 1) / CO_WARPS;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    int n_f = n_fields;
    void* args[] = {(void*)&d_fields, (void*)&d_pre, (void*)&n_f, (void*)&total, (void*)&chunk,
                    (void*)&d_ticket, (void*)&flags};
    e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(threads), args, 0, s);
    if (e != cudaSuccess) { set_last_error("vof_curvature_batched", e); return PLIC_ERR_CUDA; }
    return PLIC_OK;
}
