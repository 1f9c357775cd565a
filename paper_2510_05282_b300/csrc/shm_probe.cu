// shm_probe_fp64_rate: the FP64 pipe's rate on this device, measured.  The
// all-binary64 rows are bound by FP64 instructions, so their roofline needs
// the rate at which this GPU retires them: a kernel of independent DFMA
// chains (eight per thread, 2,048 threads per SM) times itself with CUDA
// events.  One DFMA is one FP64 pipe instruction (two flops).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <limits>

#include "sh_core.cuh"
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

// ---------------------------------------------------------------------------
// shm_probe_dmul: dmul_int (the binary64 product on the integer pipes) against
// the DMUL instruction on n operand pairs drawn from SplitMix64 words: random
// significands with exponents over most of the normal range; operands whose
// products are exact ties (a significand 1 + k 2^-52, k odd, times 1.5 2^j);
// all-ones significands (products that round up to the next binade);
// products at the edges of the normal range, zeros and subnormals (which
// dmul_int must decline).  Counts the pairs where dmul_int returned a value
// that is not bitwise DMUL's, and the pairs it declined.

namespace shm {

__device__ unsigned long long g_dmul_probe[2];  // mismatches, declined

__device__ __forceinline__ unsigned long long probe_word(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double with_exp(unsigned long long w, unsigned e) {  // sign and significand of w, biased exponent e
  return __longlong_as_double((long long)((w & 0x800fffffffffffffull) | ((unsigned long long)e << 52)));
}

__global__ void k_probe_dmul(int64_t n, unsigned long long seed) {
  unsigned long long bad_bits = 0, declined = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long w0 = probe_word(seed, 3ull * i), w1 = probe_word(seed, 3ull * i + 1),
                             w2 = probe_word(seed, 3ull * i + 2);
    double a, b;
    switch (w2 & 7u) {
      case 0:  // exact ties: (1 + k 2^-52) x 1.5, k odd, scaled
        a = with_exp((w0 & 0x800fffffffffffffull) | 1ull, 1023u + (unsigned)((w2 >> 8) % 200u) - 100u);
        b = __longlong_as_double((long long)(0x3ff8000000000000ull | (w1 & 0x8000000000000000ull))) *
            (double)(1u << ((w2 >> 16) & 15u));
        break;
      case 1:  // all-ones significands
        a = with_exp(w0 | 0x000fffffffffffffull, 1023u + (unsigned)((w2 >> 8) % 100u) - 50u);
        b = with_exp(w1, 1023u + (unsigned)((w2 >> 16) % 100u) - 50u);
        break;
      case 2:  // products near the bottom and the top of the normal range
        a = with_exp(w0, 1u + (unsigned)((w2 >> 8) % 1100u));
        b = with_exp(w1, 1u + (unsigned)((w2 >> 24) % 40u) + ((w2 >> 40) & 1u ? 0u : 1000u));
        break;
      case 3:  // zeros and subnormals among the operands
        a = (w2 >> 8) & 1u ? __longlong_as_double((long long)(w0 & 0x800fffffffffffffull)) : with_exp(w0, 1000u);
        b = (w2 >> 9) & 1u ? 0.0 : with_exp(w1, 1100u);
        break;
      default:  // random significands, exponents over most of the normal range
        a = with_exp(w0, 1023u + (unsigned)((w2 >> 8) % 1000u) - 500u);
        b = with_exp(w1, 1023u + (unsigned)((w2 >> 24) % 1000u) - 500u);
        break;
    }
    unsigned flag = 0u;
    const double r = dmul_int(a, b, flag);
    if (flag) {
      ++declined;
    } else if (__double_as_longlong(r) != __double_as_longlong(__dmul_rn(a, b))) {
      ++bad_bits;
    }
  }
  if (bad_bits) atomicAdd(&g_dmul_probe[0], bad_bits);
  if (declined) atomicAdd(&g_dmul_probe[1], declined);
}

}  // namespace shm

extern "C" shm_status shm_probe_dmul(int64_t n, uint64_t seed, int64_t* mismatches, int64_t* declined) {
  using namespace shm;
  clear_error();
  if (n < 0 || n > ((int64_t)1 << 40) || !mismatches || !declined) return fail(SHM_EINVAL, "bad arguments");
  const unsigned long long zero[2] = {0ull, 0ull};
  cudaError_t e = cudaMemcpyToSymbol(g_dmul_probe, zero, sizeof zero);
  if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpyToSymbol");
  if (n > 0) {
    k_probe_dmul<<<sm_count(current_device()) * 8, 256>>>(n, (unsigned long long)seed);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "k_probe_dmul launch");
  }
  unsigned long long got[2];
  if ((e = cudaMemcpyFromSymbol(got, g_dmul_probe, sizeof got)) != cudaSuccess) return fail_cuda(e, "cudaMemcpyFromSymbol");
  *mismatches = (int64_t)got[0];
  *declined = (int64_t)got[1];
  return SHM_OK;
}
