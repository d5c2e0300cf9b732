/*
 * plic.h -- C ABI of the GB300 (sm_103a) PLIC library (libplic.so).
 *
 * Lehmann & Gekle, "Analytic Solution to the Piecewise Linear Interface
 * Construction Problem and its Application in Curvature Calculation for
 * Volume-of-Fluid Simulation Codes", arXiv 2006.12838.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every data pointer is caller-owned DEVICE memory (cudaMalloc'd or a torch
 *   tensor's storage) or page-locked host memory mapped into the device's
 *   address space, passed as the address plic_host_device_pointer() returns
 *   for it (the kernels then read and write it over the host link; on a
 *   Grace-Blackwell node that is NVLink-C2C); contiguous, structure-of-arrays.
 *   The library never
 *   keeps a pointer after the call returns and allocates nothing; scratch
 *   memory is passed in as `workspace` (size from plic_workspace_bytes()).
 * - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *   asynchronous on that stream: they return once the kernels are queued.
 * - Arguments are validated on the host before anything is launched; an
 *   invalid argument returns PLIC_ERR_ARG (or PLIC_ERR_ALIGN) and launches
 *   nothing.  A launch failure returns PLIC_ERR_CUDA; the CUDA error text is
 *   available from plic_last_error() on the calling thread.
 * - FP32 precisions take float arrays, PLIC_FP64 and PLIC_FP64_REFINED take
 *   double arrays.
 * - Fill fields are float, laid out x-fastest: phi[x + nx*(y + ny*z)].
 *   Interface-cell lists hold int32 linear indices into that layout.
 * - No entry point throws, blocks on the device, or keeps global state other
 *   than the thread-local error text; all are safe to call from several host
 *   threads at once.
 * - Vectorised loads are used when every array is 16-byte aligned; any other
 *   alignment takes a scalar-load path of the same kernel (never a CPU path).
 */
#ifndef PLIC_H
#define PLIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLIC_OK = 0,
    PLIC_ERR_ARG = 1,          /* bad size, NULL pointer, unknown enum value   */
    PLIC_ERR_ALIGN = 2,        /* a pointer is not aligned to its element size  */
    PLIC_ERR_CUDA = 3,         /* a CUDA call failed; see plic_last_error()     */
    PLIC_ERR_UNSUPPORTED = 4,  /* valid but unsupported combination             */
    PLIC_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up            */
} plic_status;

/* The five PLIC inversions compared in Sec. 2.3-2.5 of the paper. */
typedef enum {
    PLIC_ANALYTIC = 0,  /* the paper's analytic inversion (Sec. 2.3, Eqs. 11-25)   */
    PLIC_SZ_ORIG = 1,   /* Scardovelli-Zaleski as implemented by Kawano (Sec. 2.4)  */
    PLIC_SZ_OPT = 2,    /* the paper's micro-optimised SZ with edge cases (Sec. 2.4) */
    PLIC_NEWTON = 3,    /* Newton-Raphson for cases (1), (3), (4) (Sec. 2.5)        */
    PLIC_NESTED = 4     /* nested intervals for cases (3), (4) (Sec. 2.5)           */
} plic_method;

typedef enum {
    PLIC_FP32 = 0,           /* float in/out, fast-math solver                      */
    PLIC_FP32_POLISHED = 1,  /* float in/out, solver + one Newton step on Eq. 10    */
    PLIC_FP64 = 2,           /* double in/out, the solver in double                 */
    PLIC_FP64_REFINED = 3    /* double in/out, the FP32 solver (polished) on the
                                reduced problem, then two Newton steps on Eq. 10
                                in double-float arithmetic (48-bit significands on
                                the FP32 pipes; doubles converted by integer bit
                                operations, one FP64 add per cell): |d0 error| below
                                1e-14 for |n| = 1, V0 >= 2^-126 (plic_offset only;
                                the plane-sphere entries refine in FP64)        */
} plic_precision;

enum {
    /* Paper-literal variants: the listing front end V = 1/2 - |V0 - 1/2| and
     * n2 = |nx|+|ny|+|nz|-n1-n3, the printed iteration counts of the Newton
     * and nested-interval solvers, no clamp of the SZ asin argument. */
    PLIC_FLAG_FAITHFUL = 1u,
    /* Curvature: use the centroid of each neighbour's cut polygon instead of
     * the foot point of Eq. 36. */
    PLIC_FLAG_POINT_CENTROID = 2u,
    /* Curvature: return Eq. 42 as printed (negative for a convex fluid region
     * with the Parker-Youngs normal); default is -(Eq. 42). */
    PLIC_FLAG_KAPPA_PAPER_SIGN = 4u,
    /* Curvature fit precision (at most one of the three; default: adaptive,
     * an FP32 LDL^T that is redone in FP64 for the cells whose normal matrix
     * is ill-conditioned -- smallest pivot below 1e-2 of the largest).
     * FIT_FP32: the 5x5 normal equations in FP32 only. */
    PLIC_FLAG_FIT_FP32 = 8u,
    /* FIT_DF32: in double-float (pairs of FP32 numbers, about 48 significant
     * bits) on the FP32 pipes. */
    PLIC_FLAG_FIT_DF32 = 16u,
    /* FIT_FP64: in FP64 for every cell. */
    PLIC_FLAG_FIT_FP64 = 32u,
    /* Normals (vof_normal, vof_curvature, vof_curvature_backward): the
     * centre-of-mass normal of Appendix B (all 26 weights 1) instead of the
     * Parker-Youngs normal of Eq. 38. */
    PLIC_FLAG_NORMAL_CM = 64u,
    /* vof_curvature only: the neighbour-normal variant of Sec. 4.2.  Each
     * interface neighbour i is placed with its own normal n_i (from its own
     * 3^3 stencil): point e_i + d0(phi_i, n_i) n_i relative to the centre's
     * d0(phi_0, n) n (with POINT_CENTROID: e_i + c(n_i) - c(n)); this is Eq. 36
     * when n_i = n.  A neighbour whose stencil leaves the field, or whose normal
     * is undefined, uses the centre normal.  Not available in the batched and
     * backward calls (PLIC_ERR_UNSUPPORTED). */
    PLIC_FLAG_NEIGHBOR_NORMAL = 128u
};

/* plic_volume -- forward problem ("inverse PLIC", Sec. 2.2, Eq. 10 with Eqs.
 * 2-8): V0[i] = volume of {x in [-1/2,1/2]^3 : n_i . x <= d0[i]} for a unit
 * normal n_i = (nx[i], ny[i], nz[i]).  d0 outside [-L/2, L/2] (L = |n|_1)
 * gives 0 or 1.  NaN inputs or n = 0 give NaN.
 * Arrays: nx, ny, nz, d0 (in), V0 (out), n elements each. */
plic_status plic_volume(const void *nx, const void *ny, const void *nz, const void *d0,
                        void *V0, int64_t n, plic_precision p, void *stream);

/* plic_offset -- the PLIC problem (Sec. 2, Eq. 1): for each cell, the plane
 * offset d0[i] in [-L/2, L/2] such that the plane n_i . x = d0[i] cuts the
 * volume V0[i] in [0, 1] from the unit cube, by solver `m`.  The normal must be
 * unit length (the analytic, Newton and nested-interval solvers assume it, as
 * the paper does; SZ normalises by L1 itself).  V0 = 0 / 1 give -L/2 / +L/2.
 * Invalid cells (NaN input, V0 outside [0,1], n = 0) give NaN and, when
 * d_invalid_count (device int64, nullable) is given, are added to it.
 * PLIC_SZ_ORIG reproduces Kawano's -NaN for axis-aligned n with V0 in {0,1}
 * (Sec. 2.4); those cells are not counted as invalid.
 * Arrays: nx, ny, nz, V0 (in), d0 (out), n elements each. */
plic_status plic_offset(const void *nx, const void *ny, const void *nz, const void *V0,
                        void *d0, int64_t n, plic_method m, plic_precision p, uint32_t flags,
                        int64_t *d_invalid_count, void *stream);

/* plic_offset_roundtrip -- plic_offset together with the forward volume of
 * its own result, the round trip of the paper's accuracy measure (Sec. 2.5,
 * Eqs. 27-28): d0[i] exactly as plic_offset returns it, and
 * V0_rt[i] = V0(n_i, d0[i]) (Eq. 10) evaluated on the stored d0[i] in the
 * precision of the call, so |V0_rt - V0| is the cell's round-trip error.  For
 * the optimised SZ solver in FP32 / FP32_POLISHED the two are one kernel (n
 * and V0 read once: 16 bytes in, 8 out per cell); the other methods and
 * precisions run plic_offset and then plic_volume.  Arguments, flags and
 * errors as plic_offset; V0_rt (out) has the type and length of d0. */
plic_status plic_offset_roundtrip(const void *nx, const void *ny, const void *nz, const void *V0,
                                  void *d0, void *V0_rt, int64_t n, plic_method m,
                                  plic_precision p, uint32_t flags, int64_t *d_invalid_count,
                                  void *stream);

/* plic_offset_backward -- vector-Jacobian product of plic_offset at its
 * solution d0 (implicit function theorem on Eq. 1 for unit n):
 *   g_V0 = g_d0 / A,    g_n = g_d0 * c,
 * with A the area and c the centroid (cube-centred) of the cut polygon of the
 * plane n . x = d0.  Cells with A = 0 (V0 in {0,1}) get g_V0 = +inf*g (sign of
 * g), g_n = g * c.  Arrays: nx, ny, nz, d0, g_d0 (in); g_V0, g_nx, g_ny, g_nz
 * (out); any output may be NULL to skip it.  FP32 precisions only use float;
 * PLIC_FP64 uses double. */
plic_status plic_offset_backward(const void *nx, const void *ny, const void *nz,
                                 const void *d0, const void *g_d0, void *g_V0, void *g_nx,
                                 void *g_ny, void *g_nz, int64_t n, plic_precision p,
                                 void *stream);

/* plic_volume_backward -- vector-Jacobian product of plic_volume (unit n):
 *   g_d0 = g_V0 * A,    g_n = -g_V0 * A * c.
 * The volume of Eq. 10 (Sec. 2.2) grows with d0 at the rate of the cut
 * polygon's area A; a change dn of the normal moves the plane at each point x
 * of the polygon by -dn . x, so dV0 = -A dn . c (c the centroid).
 * Arrays: nx, ny, nz, d0, g_V0 (in); g_d0, g_nx, g_ny, g_nz (out, nullable). */
plic_status plic_volume_backward(const void *nx, const void *ny, const void *nz,
                                 const void *d0, const void *g_V0, void *g_d0, void *g_nx,
                                 void *g_ny, void *g_nz, int64_t n, plic_precision p,
                                 void *stream);

/* vof_interface_compact -- the interface set of the VOF model (Sec. 4.1,
 * Eq. 33): the linear indices of all cells with 0 < phi < 1 whose 26
 * neighbours lie inside the field, in ascending order, written to idx
 * (capacity idx_capacity entries); the count goes to *d_count (device int64).
 * If the count exceeds idx_capacity, only the first idx_capacity indices are
 * written and *d_count still holds the full count.
 * workspace: >= plic_workspace_bytes(PLIC_WS_COMPACT, nx*ny*nz) bytes of device
 * memory, 256-byte aligned; its contents on entry do not matter.  Fields up to
 * 2^31 - 1 cells. */
plic_status vof_interface_compact(const float *phi, int nx, int ny, int nz, int32_t *idx,
                                  int64_t idx_capacity, int64_t *d_count, void *workspace,
                                  size_t ws_bytes, void *stream);

/* vof_interface_compact_noalloc -- the same interface-cell list and count as
 * vof_interface_compact (identical output), for callers that cannot allocate
 * device memory: a solver that owns every byte of the GPU through its own
 * pool, code that runs where cudaMalloc is not allowed or too slow to call (a
 * real-time step loop, a callback that must not synchronise the device), or a
 * foreign-language host without a device allocator.  The paper has no
 * counterpart; this is a deployment variant.
 * Its scratch (one int per tile of at least 8192 cells) is a fixed array inside the
 * library, held by every GPU that loads the library until the process exits,
 * so fields are limited to PLIC_NOALLOC_MAX_CELLS cells; larger fields return
 * PLIC_ERR_ARG with an explanation in plic_last_error() and launch nothing.
 * The call allocates nothing.  Its first call on a device looks up the
 * scratch address (cudaGetSymbolAddress) with that device current and keeps
 * it for the life of the process; make that first call before capturing a
 * stream into a graph, and do not keep calling it across a reset of the
 * device (cudaDeviceReset): the kept address belongs to the old context.
 * All calls on a device share the one scratch array: calls that may run at
 * the same time on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  The scratch needs no clearing between calls
 * (every entry a call reads is written earlier in the same call).  Other
 * arguments and the output are as for vof_interface_compact. */
#define PLIC_NOALLOC_MAX_CELLS 268435456LL  /* 2^28 cells: at most 65537 tiles, 256 KiB */
plic_status vof_interface_compact_noalloc(const float *phi, int nx, int ny, int nz,
                                          int32_t *idx, int64_t idx_capacity,
                                          int64_t *d_count, void *stream);

/* vof_curvature -- curvature step of Sec. 4.2 with Appendix B, per interface
 * cell idx[k]: 3^3 stencil -> Parker-Youngs normal (Eq. 38) -> local frame ->
 * PLIC offsets d0(phi_i, n) of the centre and of every interface neighbour
 * with the centre normal (Eq. 36), by solver m in FP32 with one Newton polish
 * -> least-squares paraboloid (Appendix B; fit precision per the FIT flags,
 * default adaptive FP32/FP64) -> mean curvature (Eq. 42) into kappa[k].
 * n_iface: number of list entries (host).  d_n_iface (device int64, nullable):
 * if given, only the first min(n_iface, *d_n_iface) entries are processed, so
 * the call can follow vof_interface_compact without a host round trip.
 * Sign: kappa = -(Eq. 42), positive for a convex fluid region (1/R for a
 * sphere of radius R); PLIC_FLAG_KAPPA_PAPER_SIGN returns Eq. 42 as printed.
 * A degenerate normal (zero weighted gradient) or no interface neighbour gives
 * kappa = 0.  Every listed cell must have its 26 neighbours inside the field
 * (as vof_interface_compact guarantees); this is not re-checked.  Fields of
 * at most 2^31 - 1 cells (PLIC_ERR_ARG otherwise), as for the compaction. */
plic_status vof_curvature(const float *phi, int nx, int ny, int nz, const int32_t *idx,
                          int64_t n_iface, const int64_t *d_n_iface, float *kappa,
                          plic_method m, uint32_t flags, void *stream);

/* vof_normal -- interface normals of the listed cells (Appendix B): the
 * Parker-Youngs normal n = -sum w_i e_i phi_i / |.| (Eq. 38), or with
 * PLIC_FLAG_NORMAL_CM the centre-of-mass normal (unit weights), written as
 * three float arrays n_x[k], n_y[k], n_z[k] (structure of arrays, caller-owned
 * device memory, n_iface entries each).  A zero weighted sum gives (0, 0, 0).
 * n_iface / d_n_iface as for vof_curvature; every listed cell must have its
 * 26 neighbours inside the field.  Errors: PLIC_ERR_ARG (sizes, null
 * pointers, flags other than NORMAL_CM), PLIC_ERR_ALIGN, PLIC_ERR_CUDA. */
plic_status vof_normal(const float *phi, int nx, int ny, int nz, const int32_t *idx,
                       int64_t n_iface, const int64_t *d_n_iface, float *n_x, float *n_y,
                       float *n_z, uint32_t flags, void *stream);

/* vof_laplace_pressure -- the Young-Laplace pressure jump of Sec. 4.1,
 * dp[k] = 2 sigma kappa[k], with kappa computed exactly as vof_curvature does
 * (same arguments, flags and solver) and the factor applied in the kernel's
 * epilogue (no second pass over the list). */
plic_status vof_laplace_pressure(const float *phi, int nx, int ny, int nz, const int32_t *idx,
                                 int64_t n_iface, const int64_t *d_n_iface, float sigma,
                                 float *dp, plic_method m, uint32_t flags, void *stream);

/* vof_curvature_backward -- vector-Jacobian product of vof_curvature (the
 * curvature step of Sec. 4.2 and Appendix B: Eqs. 36, 38 and 42) with
 * respect to the fill field: g_phi = d(sum_k g_kappa[k] kappa[k]) / d phi,
 * with the interface set (idx and the neighbour flags 0 < phi < 1) held fixed.
 * g_phi is dense (nx*ny*nz floats) and overwritten.  Per interface cell the 27
 * partial derivatives are written to the workspace and gathered per field
 * cell, so the result is deterministic (no atomics).
 * workspace: >= plic_curv_bwd_workspace_bytes(nx*ny*nz, n_iface) bytes,
 * 256-byte aligned; its contents on entry do not matter. */
plic_status vof_curvature_backward(const float *phi, int nx, int ny, int nz,
                                   const int32_t *idx, int64_t n_iface,
                                   const int64_t *d_n_iface, const float *g_kappa,
                                   float *g_phi, plic_method m, uint32_t flags,
                                   void *workspace, size_t ws_bytes, void *stream);

/* One field of a batched curvature call (all pointers device memory). */
typedef struct {
    const float *phi;        /* fill field, nx*ny*nz floats                     */
    int nx, ny, nz;
    const int32_t *idx;      /* interface-cell list of this field               */
    int64_t n_iface;         /* entries in idx                                  */
    float *kappa;            /* output, n_iface floats                          */
} vof_field;

/* Launch shape of the batched curvature kernel (chosen by an autotuner). */
typedef struct {
    int block_threads;       /* threads per block (multiple of 32, <= 1024)     */
    int cells_per_chunk;     /* interface cells claimed per work-queue ticket   */
    int blocks_per_sm;       /* resident blocks per SM of the persistent grid   */
    int lanes_per_cell;      /* 8: eight lanes per interface cell (cooperative);
                                1: one thread per cell; 0: the library's default */
} vof_tuning;

/* vof_curvature_batched -- vof_curvature (Sec. 4.2, Appendix B) over many
 * fields of uneven size in ONE persistent launch: the interface lists are
 * concatenated logically, and
 * a grid of (#SMs x blocks_per_sm) blocks claims chunks of cells from a
 * device-side ticket counter until the work is exhausted (no waiting on other
 * blocks).  `fields` is a HOST array of n_fields descriptors; it is copied to
 * the workspace before the launch and may be reused once the call returns.
 * tuning: nullable (defaults are used).  workspace: >=
 * plic_workspace_bytes(PLIC_WS_BATCHED, n_fields) bytes, 256-byte aligned. */
plic_status vof_curvature_batched(const vof_field *fields, int n_fields,
                                  const vof_tuning *tuning, plic_method m, uint32_t flags,
                                  void *workspace, size_t ws_bytes, void *stream);

/* plic_paper_benchmark -- the accuracy/throughput harness of Sec. 2.5: each
 * of the n_normals unit normals (nx, ny, nz: device arrays) is solved for the
 * L equally spaced fill levels V0_j = j/(L-1), j = 0..L-1, in series, and the
 * round-trip errors E = |V0(n, d0(V0_j, n)) - V0_j| (Eqs. 27-28) are summed into
 * *d_err_sum (device double, accumulated: zero it first); E_avg is the sum
 * over n_normals * L.  blank != 0 runs the paper's "blank run": d0 = V0_j - 1/2
 * instead of the solve, same loads, forward volume and sums.  Precisions
 * PLIC_FP32, PLIC_FP32_POLISHED (float normals) and PLIC_FP64 (double).  Kawano's
 * SZ returns NaN for axis-aligned normals at V0 in {0, 1}, so its sum is NaN
 * when such a normal is present, as the paper reports. */
plic_status plic_paper_benchmark(const void *nx, const void *ny, const void *nz,
                                 int64_t n_normals, int L, plic_method m, plic_precision p,
                                 int blank, double *d_err_sum, void *stream);

/* plic_sphere_volume / plic_sphere_offset -- the plane-sphere problem of
 * Sec. 3.  The cell is the ball of unit volume, radius r = (3/(4 pi))^(1/3);
 * d0 is the signed distance of the plane from the centre (the normal's
 * direction does not matter) and V0 the volume on the side n.x <= d0, the
 * spherical cap V0 = pi/3 (r + d0)^2 (2r - d0).
 *   plic_sphere_volume: d0[n] -> V0[n]; d0 outside [-r, r] gives 0 or 1,
 *                       NaN gives NaN.
 *   plic_sphere_offset: V0[n] -> d0[n] in [-r, r]; V0 outside [0, 1] or NaN
 *                       gives NaN.
 * Arrays: caller-owned device memory, float (PLIC_FP32, PLIC_FP32_POLISHED)
 * or double (PLIC_FP64, PLIC_FP64_REFINED); the FP32 inverse always ends with
 * Newton steps, so the two FP32 precisions (and the two FP64 ones) are the
 * same computation.  16-byte aligned arrays take the vector path.  Errors:
 * PLIC_ERR_ARG (n < 0, null pointer, bad precision), PLIC_ERR_ALIGN (element
 * misalignment), PLIC_ERR_CUDA (launch failure).  Asynchronous on stream. */
plic_status plic_sphere_volume(const void *d0, void *V0, int64_t n, plic_precision p,
                               void *stream);
plic_status plic_sphere_offset(const void *V0, void *d0, int64_t n, plic_precision p,
                               void *stream);

/* The functions below are library plumbing (workspace sizes, status text,
 * version, host-memory addressing); the paper has no counterpart. */

/* Workspace kinds for plic_workspace_bytes(). */
enum {
    PLIC_WS_COMPACT = 0,     /* arg: number of field cells nx*ny*nz             */
    PLIC_WS_BATCHED = 2      /* arg: number of fields                           */
};

/* Workspace bytes for an operation (0 if it needs none). */
size_t plic_workspace_bytes(int op, int64_t arg);

/* Workspace bytes of vof_curvature_backward for a field of `cells` cells and
 * an interface list of n_iface entries: a dense int32 slot map of the field
 * plus 27 floats per interface cell, each part 256-byte aligned. */
size_t plic_curv_bwd_workspace_bytes(int64_t cells, int64_t n_iface);

/* Human-readable name of a status code (static storage). */
const char *plic_status_string(plic_status s);

/* Text of the last CUDA error seen on this host thread (static storage of the
 * thread; empty when none). */
const char *plic_last_error(void);

/* Library version, for the binding's load check. */
int plic_abi_version(void);

/* plic_host_device_pointer -- the address under which the current device
 * reaches page-locked host memory (cudaHostAlloc / cudaMallocHost memory, or
 * cudaHostRegister'ed memory registered as mapped; on a unified-address system
 * every page-locked allocation is mapped and the address equals host_ptr).
 * The result may be passed to any entry point in place of a device array:
 * the kernels then move the data over the host link themselves (no staging
 * copy).  Any other memory (pageable host memory, device memory, an unknown
 * address) returns PLIC_ERR_ARG and leaves *dev_ptr untouched, so that nothing
 * is ever launched on an address the device cannot reach.  Host-side query
 * only (cudaPointerGetAttributes); no launch, no synchronisation. */
plic_status plic_host_device_pointer(const void *host_ptr, void **dev_ptr);

/* plic_pipe_probe -- a throughput probe of one execution pipe, for the
 * compute side of the kernels' rooflines (the paper has no counterpart).
 * kind: 0 FP32 FMA, 1 paired FP32 FMA (FFMA2, two operations), 2 FP64 FMA,
 * 3 MUFU ex2 + lg2 (two operations), 4 MUFU rsqrt, 5 MUFU sin; FP64 library
 * calls: 6 sqrt(x+1), 7 1/(x+1), 8 cbrt(x+1) (each with one FP64 add),
 * 9 sin, 10 cos, 11 asin(x/2), 12 acos(x/2) (each with one FP64 multiply),
 * 13 atan2.  Launches one wave of resident blocks on `stream`, every thread
 * running 8 independent chains of `iters` operations; *ops (host) receives
 * the number of operations (or calls) the launch performs, so that the
 * caller's CUDA-event time of the launch gives the rate.  d_sink: a device
 * float that is written only in the impossible event that keeps the chains
 * alive.  Errors: PLIC_ERR_ARG (unknown kind, iters < 1, null pointers),
 * PLIC_ERR_ALIGN, PLIC_ERR_CUDA. */
plic_status plic_pipe_probe(int kind, int iters, float *d_sink, int64_t *ops, void *stream);

/* plic_read_probe -- the plain streaming read of n floats at buf (device,
 * 16-byte aligned), for the memory side of the kernels' rooflines (the paper
 * has no counterpart): one launch on `stream` of one wave of resident blocks,
 * each thread issuing four independent 16-byte loads per trip of a
 * grid-stride loop.  Timed with CUDA events from a given cache state (the
 * buffer in L2, or L2 flushed), it is the fastest that a pass reading the
 * buffer once can go from that state.  d_sink: a device float written only in
 * the impossible event that keeps the loads alive.  Errors: PLIC_ERR_ARG
 * (n < 0, null pointers), PLIC_ERR_ALIGN (buf not 16-byte aligned),
 * PLIC_ERR_CUDA. */
plic_status plic_read_probe(const float *buf, int64_t n, float *d_sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PLIC_H */
