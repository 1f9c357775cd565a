// shm_probe_fp64_rate: the FP64 pipe's rate on this device, measured.  The
// all-binary64 rows are bound by FP64 instructions, so their roofline needs
// the rate at which this GPU retires them: a kernel of independent DFMA
// chains (eight per thread, 2,048 threads per SM) times itself with CUDA
// events.  One DFMA is one FP64 pipe instruction (two flops).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <limits>

#include "shm_internal.h"

namespace shm {

// written only when the chains hit a value the host never passes, so the
// compiler keeps every DFMA
__device__ double g_fp64_probe_sink;

constexpr int kProbeTPB = 256;

template <int CHAINS>
__global__ void __launch_bounds__(kProbeTPB) k_fp64_rate(int64_t iters, double a, double b, double sentinel) {
  double x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = 1e-3 * (double)threadIdx.x + (double)c;
#pragma unroll 4
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == sentinel) g_fp64_probe_sink = s;
}

}  // namespace shm

namespace {

// One timed launch of k_fp64_rate<CHAINS> with `per_sm` CTAs per SM after a
// short warm-up launch; DFMA per second, or a negative value on error.
template <int CHAINS>
double probe_once(int64_t iters, int per_sm, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  using namespace shm;
  const int grid = sm_count(current_device()) * per_sm;
  const double nan = std::numeric_limits<double>::quiet_NaN();  // the sentinel never compares equal
  k_fp64_rate<CHAINS><<<grid, kProbeTPB, 0, s>>>(iters / 8 + 1, 0.999999999, 1e-9, nan);
  cudaEventRecord(e0, s);
  k_fp64_rate<CHAINS><<<grid, kProbeTPB, 0, s>>>(iters, 0.999999999, 1e-9, nan);
  cudaEventRecord(e1, s);
  float t = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || t <= 0.f)
    return -1.0;
  *ms = t;
  return (double)grid * kProbeTPB * CHAINS * (double)iters / (t * 1e-3);
}

}  // namespace

extern "C" shm_status shm_probe_fp64_rate(int64_t iters, double* dfma_per_s, double* ms) {
  using namespace shm;
  clear_error();
  if (iters <= 0 || iters > ((int64_t)1 << 24) || !dfma_per_s)
    return fail(SHM_EINVAL, "iters in 1..2^24, non-null result");
  if (current_device() < 0) return fail(SHM_ECUDA, "no current device");
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return fail_cuda(e, "cudaStreamCreate");
  shm_status st = SHM_OK;
  double best = -1.0;
  float best_ms = 0.f;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = fail_cuda(e, "cudaEventCreate");
  } else {
    // launch shapes: 4, 8 or 16 independent chains per thread, 2 to 8
    // resident 256-thread CTAs per SM; the fastest is the pipe's rate
    const int shapes[][2] = {{8, 8}, {4, 8}, {16, 4}, {8, 4}, {16, 2}, {8, 2}};
    for (const auto& sh : shapes) {
      float t = 0.f;
      const int64_t it = iters * 8 / sh[0];  // the same DFMAs per thread for every shape
      const double r = sh[0] == 4 ? probe_once<4>(it, sh[1], s, e0, e1, &t)
                       : sh[0] == 8 ? probe_once<8>(it, sh[1], s, e0, e1, &t)
                                    : probe_once<16>(it, sh[1], s, e0, e1, &t);
      if (r < 0) {
        st = fail_cuda(cudaGetLastError(), "k_fp64_rate");
        break;
      }
      if (r > best) {
        best = r;
        best_ms = t;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st != SHM_OK) return st;
  *dfma_per_s = best;
  if (ms) *ms = best_ms;
  return SHM_OK;
}
