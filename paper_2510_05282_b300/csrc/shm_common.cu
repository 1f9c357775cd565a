// Error reporting, pointer checks and device queries shared by libshm.
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>

#include "shm_internal.h"

namespace shm {

namespace {
thread_local std::string g_last_error;

// cuMemGetAddressRange through the runtime's driver entry-point query, so the
// library does not link libcuda directly and loads on machines without a GPU
// driver (the CPU-side tests check its exports there).
typedef CUresult (*AddrRangeFn)(CUdeviceptr*, size_t*, CUdeviceptr);
AddrRangeFn addr_range_fn() {
  static AddrRangeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (AddrRangeFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}
// cuTensorMapEncodeTiled, fetched the same way.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}
}  // namespace

bool encode_rows_map(CUtensorMap* map, void* base, int64_t n, int cols, int box_cols, int box_rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (enc == nullptr || n <= 0 || n > INT32_MAX || box_cols <= 0 || box_cols > 256 || box_rows <= 0 ||
      box_rows > 256 || (box_cols * 8) % 16 != 0 || ((int64_t)cols * 8) % 16 != 0 || !aligned(base, 16))
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

shm_status fail(shm_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

shm_status fail_cuda(cudaError_t e, const char* what) {
  return fail(SHM_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

void clear_error() { g_last_error.clear(); }

shm_status check_device_range(const void* p, size_t bytes, const char* what) {
  if (p == nullptr) return fail(SHM_EINVAL, std::string(what) + " is null");
  if (bytes == 0) return SHM_OK;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SHM_EINVAL, std::string(what) + " is not a pointer CUDA knows");
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(SHM_EINVAL, std::string(what) + " is not device memory");
  if (attr.type == cudaMemoryTypeDevice && attr.device != current_device())
    return fail(SHM_EINVAL, std::string(what) + " belongs to another device");
  CUdeviceptr base = 0;
  size_t size = 0;
  AddrRangeFn range = addr_range_fn();
  if (range == nullptr) return fail(SHM_ECUDA, "cuMemGetAddressRange is unavailable");
  CUresult r = range(&base, &size, (CUdeviceptr)(uintptr_t)p);
  if (r != CUDA_SUCCESS) {
    if (attr.type == cudaMemoryTypeManaged) return SHM_OK;  // no range query for managed memory
    return fail(SHM_EINVAL, std::string(what) + ": allocation range unknown");
  }
  const uintptr_t lo = (uintptr_t)p, hi = lo + bytes;
  if (hi < lo || lo < (uintptr_t)base || hi > (uintptr_t)base + size)
    return fail(SHM_EINVAL, std::string(what) + ": " + std::to_string(bytes) +
                                " bytes from this pointer run past the end of its allocation");
  return SHM_OK;
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return na > 0 && nb > 0 && a0 < b0 + nb && b0 < a0 + na;
}

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return d;
}

// Allocation-failure injection: SHM_FAIL_ALLOC names the allocation sites
// that fail ("serve_pool", "serve_pinned", "serve_batch", "autotune",
// comma-separated, or "all"), read at every allocation.
bool alloc_fail_injected(const char* site) {
  const char* v = getenv("SHM_FAIL_ALLOC");
  if (!v || !*v) return false;
  const std::string list = std::string(",") + v + ",";
  return list.find(",all,") != std::string::npos || list.find(std::string(",") + site + ",") != std::string::npos;
}

cudaError_t dev_malloc(void** p, size_t bytes, const char* site) {
  *p = nullptr;
  if (alloc_fail_injected(site)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t pinned_malloc(void** p, size_t bytes, const char* site) {
  *p = nullptr;
  if (alloc_fail_injected(site)) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

shm_status fail_alloc(cudaError_t e, const char* site, const std::string& what) {
  if (alloc_fail_injected(site)) return fail(SHM_ENOMEM, what + " (failure injected by SHM_FAIL_ALLOC)");
  cudaGetLastError();
  return fail(SHM_ENOMEM, what + ": " + cudaGetErrorString(e));
}

int sm_count(int dev) {
  static int cache[64] = {0};
  if (dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 148;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

}  // namespace shm

extern "C" {

const char* shm_last_error(void) { return shm::g_last_error.c_str(); }

const char* shm_status_string(shm_status s) {
  switch (s) {
    case SHM_OK: return "SHM_OK";
    case SHM_EINVAL: return "SHM_EINVAL";
    case SHM_ENOMEM: return "SHM_ENOMEM";
    case SHM_ECUDA: return "SHM_ECUDA";
    case SHM_EBUSY: return "SHM_EBUSY";
    case SHM_ETIMEOUT: return "SHM_ETIMEOUT";
    case SHM_EUNSUPPORTED: return "SHM_EUNSUPPORTED";
    case SHM_ENOTFOUND: return "SHM_ENOTFOUND";
  }
  return "SHM_UNKNOWN";
}

int shm_num_harmonics(int lmax) { return (lmax >= 0 && lmax <= SHM_LMAX_EXT) ? (lmax + 1) * (lmax + 1) : 0; }

}  // extern "C"
