// Internal helpers shared by the libshm translation units (host side).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>

#include "../../include/shm.h"

namespace shm {

// Records msg as this thread's last error and returns st.
shm_status fail(shm_status st, const std::string& msg);
shm_status fail_cuda(cudaError_t e, const char* what);
void clear_error();

// Checks that [p, p + bytes) is device-accessible memory inside one
// allocation of the current device (cuMemGetAddressRange), so that a wrong
// pointer or size is rejected on the host instead of faulting the GPU.
// `what` names the argument in the error message.
shm_status check_device_range(const void* p, size_t bytes, const char* what);

// True when the byte ranges [a, a + na) and [b, b + nb) intersect.
bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb);

int current_device();
int sm_count(int dev);

// The library's own device and pinned allocations (serve pool and batch
// descriptors, tuner probe buffers) go through these, so that a test can make
// any of them fail without exhausting memory: the environment variable
// SHM_FAIL_ALLOC lists the failing sites ("serve_pool", "serve_pinned",
// "serve_batch", "autotune", comma-separated, or "all").  A failing site
// returns cudaErrorMemoryAllocation without calling CUDA; fail_alloc turns
// either kind of failure into SHM_ENOMEM with a message that says which.
bool alloc_fail_injected(const char* site);
cudaError_t dev_malloc(void** p, size_t bytes, const char* site);
cudaError_t pinned_malloc(void** p, size_t bytes, const char* site);
shm_status fail_alloc(cudaError_t e, const char* site, const std::string& what);

// NVTX range around an entry point (header-only NVTX 3: inert unless a
// profiler injects its library).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Tensor map of a row-major FP64 matrix [n][cols] at `base` for TMA tensor
// stores of [box_rows][box_cols] boxes (no swizzle).  False (nothing
// launched, the caller takes its non-TMA path) when the driver entry point
// is unavailable or the layout breaks a TMA rule: base and row pitch 16-byte
// aligned, box width a multiple of 16 bytes, box sides <= 256, n < 2^31.
bool encode_rows_map(CUtensorMap* map, void* base, int64_t n, int cols, int box_cols, int box_rows);

}  // namespace shm
