// host_common.h -- host-side helpers shared by the entry points of libplic.so:
// status/error bookkeeping, argument checks, and launch geometry.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/plic.h"

namespace plic {

// Thread-local text of the last CUDA error (plic_last_error()).
void set_last_error(const char* where, cudaError_t e);

// Records "field of n cells exceeds the allocation-free limit" as the error text.
void set_limit_error(int64_t ncell);

// Returns PLIC_ERR_CUDA (and records the text) if the last launch failed.
plic_status check_launch(const char* where);

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Number of SMs of the current device (cached per device).
int sm_count();

// Blocks of `kernel` that fit on one SM with `threads` threads and `smem` bytes
// of dynamic shared memory (cached per kernel pointer).
int blocks_per_sm(const void* kernel, int threads, size_t smem);

// A grid for a grid-stride loop over `work` items of `threads` threads each:
// min(ceil(work/threads), SMs x resident blocks per SM), at least 1.
int stride_grid(const void* kernel, int threads, int64_t work, size_t smem = 0);
// The streaming kernels' grid: up to STREAM_WAVES waves of resident blocks
// (each thread still loops when the work is larger).  Measured on the fused
// PLIC step: one persistent wave 1.502 ms, 2 waves 1.446, 4 1.409, 8 1.391,
// 32 1.386, one block per 256 vectors (no loop) 1.447.
constexpr int STREAM_WAVES = 16;
int stream_grid(const void* kernel, int threads, int64_t work);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Programmatic dependent launch: a kernel launched with launch_after() may be
// scheduled while the kernel before it on the stream is still finishing (once
// that kernel's blocks have all executed pdl_trigger() or exited), and waits
// in pdl_wait() until that kernel has completed and its writes are visible.
// Every kernel launched this way calls pdl_wait() before it reads what the
// kernel before it wrote; the overlap hides the launch of short dependent
// kernels (the compaction's write pass, the curvature step after it).  After
// an operation that is not a kernel, or with no kernel before it, the launch
// is an ordinary one and pdl_wait() returns at once.
cudaError_t launch_after(const void* kernel, dim3 grid, dim3 block, void** args, cudaStream_t s);

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

}  // namespace plic
