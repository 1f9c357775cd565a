// shm_eval_complex: the complex harmonics Y_l^m (Sec. II Eq. 5, with Eq. 10
// for negative m) fused into the evaluator.  With the real harmonics of the
// same rows, Y_l^0 = R_l^0 and, for m > 0,
//   Y_l^{+m} = (-1)^m (R_l^m + i R_l^{-m}) / sqrt2,
//   Y_l^{-m} =        (R_l^m - i R_l^{-m}) / sqrt2
// (the paper's Sec. III relation without its missing 1/sqrt2).  The rows are
// computed by the real-harmonic row code with the scale constants divided by
// sqrt2 for m > 0 (coefficient set CX), so each real value v lands, with a
// sign, in the real or imaginary part of Y_l^{+m} and Y_l^{-m} at no extra
// arithmetic.  Output: [n][(lmax+1)^2][2] (re, im) of the dtype.
//
// FP64 rows use the hybrid arithmetic in l-major order (binary64 for 1/r and
// m = 0, 1, float-float for m >= 2), staged as real values one group of
// l-shells at a time; the copy-out pairs them into (re, im) with a per-CTA map
// and writes 16-byte complex values.  With SHM_STRICT_FP64 the FP64 rows are
// the all-binary64 m-major rows (sh_row), staged whole and paired the same way.  (Scattering the values into complex
// slots as they are produced raised the row code's register use from 96 to
// 162 and cut the resident warps.)  FP32 rows use the FP32 row code, staged a
// full row at a time in complex layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sh_core.cuh"
#include "sh_phased.cuh"
#include "sh_tile.cuh"
#include "sh_tma.cuh"
#include "shm_internal.h"

namespace shm {

// Writes the real value v = R_l^m (already divided by sqrt2 for m != 0) of
// k = l*l + l + m into the complex row c[2k + part], relative to base k0.
template <typename T>
__device__ __forceinline__ void cx_store(T* c, int k, int k0, T v) {
  const int l = l_of_k(k);
  const int m = k - l * l - l;
  const int kc = l * l + l;
  if (m == 0) {
    c[2 * (k - k0)] = v;
    c[2 * (k - k0) + 1] = (T)0;
  } else if (m > 0) {  // Re Y_l^{+m} = (-1)^m v, Re Y_l^{-m} = v
    c[2 * (k - k0)] = (m & 1) ? -v : v;
    c[2 * (kc - m - k0)] = v;
  } else {  // v = R_l^{-mu}: Im Y_l^{+mu} = (-1)^mu v, Im Y_l^{-mu} = -v
    const int mu = -m;
    c[2 * (kc + mu - k0) + 1] = (mu & 1) ? -v : v;
    c[2 * (k - k0) + 1] = -v;
  }
}

constexpr int kCxTPB64 = 128;
constexpr int kCxPhase = 37;  // real values staged per row and phase
constexpr int kCxTPB32 = 64;

// Copy-out map of complex slot k = l*l + l + m: the real values it is made of
// (ka = index of R_l^{|m|}, kb = index of R_l^{-|m|}) and their signs.
__device__ __forceinline__ uint32_t cx_map_entry(int k) {
  int l = 0;
  while ((l + 1) * (l + 1) <= k) ++l;
  const int kc = l * l + l, m = k - kc, mu = m < 0 ? -m : m;
  uint32_t e = (uint32_t)(kc + mu) | ((uint32_t)(kc - mu) << 10);
  if (m == 0) e |= 1u << 29;                            // Y_l^0 = R_l^0
  else if (m > 0 && (m & 1)) e |= (1u << 30) | (1u << 31);  // (-1)^m (a + i b)
  else if (m < 0) e |= 1u << 31;                        // a - i b
  return e;
}

__device__ __forceinline__ double flip_if(double v, uint32_t bit) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)bit << 63));
}

template <int LMAX>
__global__ void __launch_bounds__(kCxTPB64, 5) k_eval_cx64(const double* __restrict__ pts, int64_t n,
                                                        double* __restrict__ out, int64_t ntiles, int normalized,
                                                        int vec) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int RS = LPhases<LMAX, kCxPhase>::max_width() | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t cxmap[L2];
  double* tile = reinterpret_cast<double*>(smem_raw);
  for (int k = threadIdx.x; k < L2; k += kCxTPB64) cxmap[k] = cx_map_entry(k);
  __syncthreads();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kCxTPB64;
    const int rows = (int)min((int64_t)kCxTPB64, n - p0);
    const bool valid = (int)threadIdx.x < rows;
    double x = 0.0, y = 0.0, z = 1.0;
    if (valid) {
      const int64_t p = p0 + threadIdx.x;
      x = pts[3 * p];
      y = pts[3 * p + 1];
      z = pts[3 * p + 2];
    }
    const bool origin = valid && is_origin(x, y, z);
    double xb = 0.0, yb = 0.0, zb = 1.0;
    if (valid && !origin) {
      if (normalized) {
        xb = x;
        yb = y;
        zb = z;
      } else {
        unit_dir(x, y, z, xb, yb, zb);
      }
    }
    double* row = tile + threadIdx.x * RS;
    const bool bad = nonfinite3(xb, yb, zb);  // NaN row (the hybrid row code needs a finite direction)
    auto store = [&](int k, int k0, double v) { row[k - k0] = v; };
    auto flush = [&](int k0, int w) {
      if (origin || bad) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
        const double fill = origin ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
        for (int c = 0; c < w; ++c) row[c] = (k0 + c == 0) ? kInvSqrt4Pi : fill;
      }
      __syncthreads();
      // thread (rs, c) = divmod(threadIdx, w) writes complex slot c of rows rs,
      // rs + RP, ... (RP = TPB / w): its map entry and source offsets are
      // read once per phase, the addresses advance by constant steps
      const int RP = kCxTPB64 / w;
      const int rs = (int)threadIdx.x / w;
      const int c = (int)threadIdx.x - rs * w;
      if (rs < RP) {
        const uint32_t e = cxmap[k0 + c];
        const int ka = (int)(e & 1023u) - k0, kb = (int)((e >> 10) & 1023u) - k0;
        const uint32_t fa = (e >> 30) & 1u, fb = e >> 31;
        const bool zero_im = (e & (1u << 29)) != 0u;
        const double* src = tile + rs * RS;
        double* o = out + 2 * ((p0 + rs) * L2 + k0 + c);
        for (int r = rs; r < rows; r += RP) {
          const double re = flip_if(src[ka], fa);
          const double im = zero_im ? 0.0 : flip_if(src[kb], fb);
          if (vec) {
            __stcs(reinterpret_cast<double2*>(o), make_double2(re, im));
          } else {
            __stcs(o, re);
            __stcs(o + 1, im);
          }
          src += RP * RS;
          o += 2 * RP * L2;
        }
      }
      __syncthreads();
    };
    sh_row_hybrid_lmajor<LMAX, true, kCxPhase>(xb, yb, zb, store, flush);
  }
}

// All-binary64 complex rows (SHM_STRICT_FP64): the m-major real row of
// sh_row<LMAX, CX> (scale constants divided by sqrt2 for m != 0), staged
// whole with an odd row stride, then paired into (re, im) slots by the map.
// 128 rows per tile, so that every complex slot of l <= 9 has its own thread
// in the copy-out (3.26 ms on the 192^3 grid; 3.43 ms with 64 rows, 3.65 ms
// with the copy-out over flat (row, slot) indices).
constexpr int kCxTPBs = 128;

template <int LMAX>
__global__ void __launch_bounds__(kCxTPBs) k_eval_cx64s(const double* __restrict__ pts, int64_t n,
                                                       double* __restrict__ out, int64_t ntiles, int normalized,
                                                       int vec) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int RS = L2 | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t cxmap[L2];
  double* tile = reinterpret_cast<double*>(smem_raw);
  for (int k = threadIdx.x; k < L2; k += kCxTPBs) cxmap[k] = cx_map_entry(k);
  __syncthreads();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kCxTPBs;
    const int rows = (int)min((int64_t)kCxTPBs, n - p0);
    if ((int)threadIdx.x < rows) {
      const int64_t p = p0 + threadIdx.x;
      double* row = tile + threadIdx.x * RS;
      // the output products on the integer pipes (dmul_int): the same bits
      sh_point<LMAX, false, true, kEmuOut>(pts[3 * p], pts[3 * p + 1], pts[3 * p + 2], normalized != 0,
                                           [&](int k, double v) { row[k] = v; });
    }
    __syncthreads();
    // thread t writes complex slots c = t, t + TPB, ... of every row of the
    // tile: its map entries are decoded once per tile and the addresses
    // advance by constant steps, while a warp's stores still cover adjacent
    // slots of one row
    for (int c = threadIdx.x; c < L2; c += kCxTPBs) {
      const uint32_t e = cxmap[c];
      const int ka = (int)(e & 1023u), kb = (int)((e >> 10) & 1023u);
      const uint32_t fa = (e >> 30) & 1u, fb = e >> 31;
      const bool zero_im = (e & (1u << 29)) != 0u;
      const double* src = tile;
      double* o = out + 2 * (p0 * L2 + c);
      for (int r = 0; r < rows; ++r) {
        const double re = flip_if(src[ka], fa);
        const double im = zero_im ? 0.0 : flip_if(src[kb], fb);
        if (vec) {
          __stcs(reinterpret_cast<double2*>(o), make_double2(re, im));
        } else {
          __stcs(o, re);
          __stcs(o + 1, im);
        }
        src += RS;
        o += 2 * L2;
      }
    }
    __syncthreads();
  }
}

template <int LMAX>
__global__ void __launch_bounds__(kCxTPB32) k_eval_cx32(const float* __restrict__ pts, int64_t n,
                                                        float* __restrict__ out, int64_t ntiles, int normalized,
                                                        int vec) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int RS = (2 * L2) | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tile = reinterpret_cast<float*>(smem_raw);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kCxTPB32;
    const int rows = (int)min((int64_t)kCxTPB32, n - p0);
    if ((int)threadIdx.x < rows) {
      const int64_t p = p0 + threadIdx.x;
      const float x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
      float* row = tile + threadIdx.x * RS;
      if (is_origin(x, y, z)) {
        for (int c = 0; c < 2 * L2; ++c) row[c] = c == 0 ? (float)kInvSqrt4Pi : 0.0f;
      } else {
        float xb = x, yb = y, zb = z;
        if (!normalized) unit_dir(x, y, z, xb, yb, zb);
        if (nonfinite3(xb, yb, zb)) {  // NaN in every value but Y_0^0 (and the zero imaginary parts of m = 0)
          cx_store(row, 0, 0, (float)kInvSqrt4Pi);
#pragma unroll
          for (int k = 1; k < L2; ++k) cx_store(row, k, 0, __int_as_float(0x7fc00000));
        } else {
          sh_row<LMAX, true>(xb, yb, zb, [&](int k, float v) { cx_store(row, k, 0, v); });
        }
      }
    }
    __syncthreads();
    copy_out_tile<float, 2 * L2, RS, kCxTPB32>(tile, rows, out + p0 * 2 * L2, vec != 0);
    __syncthreads();
  }
}

template <int LMAX>
shm_status cx_launch(const void* pts, int64_t n, bool f64, void* out, bool normalized, bool vec, cudaStream_t s,
                     bool strict) {
  constexpr int MAXDEV = 64;
  static int bps[3][MAXDEV] = {};
  const int dev = current_device();
  if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
  strict = strict && f64;
  const int tpb = strict ? kCxTPBs : (f64 ? kCxTPB64 : kCxTPB32);
  const size_t smem = strict ? (size_t)kCxTPBs * (NH<LMAX>::value | 1) * 8
                      : f64  ? (size_t)kCxTPB64 * (LPhases<LMAX, kCxPhase>::max_width() | 1) * 8
                             : (size_t)kCxTPB32 * ((2 * NH<LMAX>::value) | 1) * 4;
  const void* kern = strict ? (const void*)k_eval_cx64s<LMAX>
                     : f64  ? (const void*)k_eval_cx64<LMAX>
                            : (const void*)k_eval_cx32<LMAX>;
  int& b = bps[strict ? 2 : (f64 ? 1 : 0)][dev];
  if (b == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_eval_cx)");
    int bb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, kern, tpb, smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_eval_cx)");
    b = std::max(bb, 1);
  }
  const int64_t ntiles = (n + tpb - 1) / tpb;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * b);
  if (strict)
    k_eval_cx64s<LMAX><<<(unsigned)grid, tpb, smem, s>>>((const double*)pts, n, (double*)out, ntiles, normalized,
                                                          vec);
  else if (f64)
    k_eval_cx64<LMAX><<<(unsigned)grid, tpb, smem, s>>>((const double*)pts, n, (double*)out, ntiles, normalized, vec);
  else
    k_eval_cx32<LMAX><<<(unsigned)grid, tpb, smem, s>>>((const float*)pts, n, (float*)out, ntiles, normalized, vec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "k_eval_cx launch");
  return SHM_OK;
}

}  // namespace shm

extern "C" shm_status shm_eval_complex(const void* points, int64_t n, int lmax, shm_dtype dtype, unsigned flags,
                                       void* out, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_eval_complex");
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (lmax < 0 || lmax > SHM_LMAX_CAP) return fail(SHM_EINVAL, "lmax must be in 0..9");
  if (n < 0) return fail(SHM_EINVAL, "n must be >= 0");
  if (flags & ~(SHM_NORMALIZED_INPUT | SHM_STRICT_FP64)) return fail(SHM_EINVAL, "unknown flag bits");
  if (n == 0) return SHM_OK;
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  const int64_t L2 = (int64_t)(lmax + 1) * (lmax + 1);
  if (n > (INT64_MAX / 16) / (L2 * 16)) return fail(SHM_EINVAL, "n too large");
  if (!points || !out) return fail(SHM_EINVAL, "points and out must be non-null");
  if (!aligned(points, es) || !aligned(out, es))
    return fail(SHM_EINVAL, "points and out must be aligned to the element size");
  const size_t in_bytes = (size_t)n * 3 * es, out_bytes = (size_t)n * L2 * 2 * es;
  if (ranges_overlap(points, in_bytes, out, out_bytes)) return fail(SHM_EINVAL, "points and out overlap");
  shm_status st = check_device_range(points, in_bytes, "points");
  if (st != SHM_OK) return st;
  if ((st = check_device_range(out, out_bytes, "out")) != SHM_OK) return st;
  const bool f64 = dtype == SHM_F64, norm = (flags & SHM_NORMALIZED_INPUT) != 0, vec = aligned(out, 16);
  const bool strict = (flags & SHM_STRICT_FP64) != 0;
  cudaStream_t s = (cudaStream_t)stream;
  switch (lmax) {
    case 0: return cx_launch<0>(points, n, f64, out, norm, vec, s, strict);
    case 1: return cx_launch<1>(points, n, f64, out, norm, vec, s, strict);
    case 2: return cx_launch<2>(points, n, f64, out, norm, vec, s, strict);
    case 3: return cx_launch<3>(points, n, f64, out, norm, vec, s, strict);
    case 4: return cx_launch<4>(points, n, f64, out, norm, vec, s, strict);
    case 5: return cx_launch<5>(points, n, f64, out, norm, vec, s, strict);
    case 6: return cx_launch<6>(points, n, f64, out, norm, vec, s, strict);
    case 7: return cx_launch<7>(points, n, f64, out, norm, vec, s, strict);
    case 8: return cx_launch<8>(points, n, f64, out, norm, vec, s, strict);
    default: return cx_launch<9>(points, n, f64, out, norm, vec, s, strict);
  }
}

// ---------------------------------------------------------------------------
// Angular interface: (theta, phi) per point (Sec. II Eq. 3-4 read backwards:
// x/r = sin(theta) cos(phi), y/r = sin(theta) sin(phi), z/r = cos(theta)),
// then the rows of shm_eval.  FP64: CUDA's binary64 sincos of theta and the
// float-float sine and cosine of phi (angles_to_unit), then the hybrid rows;
// with SHM_STRICT_FP64 binary64 sincos of both angles and the all-binary64
// rows (rows-tma-64, or the staged kernel below).  FP32: sincosf.

namespace shm {

constexpr int kAngTPB = 64;     // FP32 staged kernel
constexpr int kAngTPB64 = 128;  // FP64 phased hybrid kernel

// FP32, and FP64 with SHM_STRICT_FP64 where TMA does not apply.
template <typename T, int LMAX>
__global__ void __launch_bounds__(kAngTPB) k_eval_angles(const T* __restrict__ ang, int64_t n, T* __restrict__ out,
                                                          int64_t ntiles, int vec) {
  constexpr int L2 = TileShape<LMAX>::L2;
  constexpr int RS = TileShape<LMAX>::RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kAngTPB;
    const int rows = (int)min((int64_t)kAngTPB, n - p0);
    if ((int)threadIdx.x < rows) {
      const int64_t p = p0 + threadIdx.x;
      T xb, yb, zb;
      if constexpr (sizeof(T) == 8) {
        angles_to_unit<true>(ang[2 * p], ang[2 * p + 1], xb, yb, zb);
      } else {
        T st, ct, sp, cp;
        sincosf(ang[2 * p], &st, &ct);
        sincosf(ang[2 * p + 1], &sp, &cp);
        xb = st * cp;
        yb = st * sp;
        zb = ct;
      }
      T* row = tile + threadIdx.x * RS;
      if (nonfinite3(xb, yb, zb)) {  // a non-finite angle: NaN in every value but l = 0
        for (int k = 0; k < L2; ++k) row[k] = k == 0 ? (T)kInvSqrt4Pi : (T)__longlong_as_double(0x7ff8000000000000ll);
      } else {
        sh_row<LMAX>(xb, yb, zb, [&](int k, T v) { row[k] = v; });
      }
    }
    __syncthreads();
    copy_out_tile<T, L2, RS, kAngTPB>(tile, rows, out + p0 * L2, vec != 0);
    __syncthreads();
  }
}

// FP64 angles run the phased hybrid evaluator with angle input -- with TMA
// stores (sh_tma.cuh) where they apply, else sh_phased.cuh; FP32 angles the
// staged kernel above.
template <typename T, int LMAX>
shm_status ang_launch(const T* ang, int64_t n, T* out, bool vec, cudaStream_t s, bool strict) {
  strict = strict && sizeof(T) == 8;
  if constexpr (sizeof(T) == 8) {
    if (vec) {
      bool launched = false;
      // strict: the default all-binary64 form of shm_eval (rows-tma-emu-o-32:
      // the output products on the integer pipes, the same bits)
      shm_status st = strict ? launch_rows_tma<LMAX, 32, kInAngles, kEmuOut>(ang, n, out, false, s, &launched)
                             : launch_phased_tma<LMAX, kAngTPB64, kInAngles>(ang, n, out, false, s, &launched);
      if (st != SHM_OK || launched) return st;
    }
  }
  constexpr int MAXDEV = 64;
  static int bps[2][MAXDEV] = {};
  const int dev = current_device();
  if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
  const bool phased = sizeof(T) == 8 && !strict;  // the FP64 hybrid rows
  const int TPB = phased ? kAngTPB64 : kAngTPB;
  const size_t smem = phased ? (size_t)TPB * (LPhases<LMAX>::max_width() | 1) * 8
                             : (size_t)TPB * TileShape<LMAX>::RS * sizeof(T);
  const void* kern = phased ? (const void*)k_eval_phased<LMAX, kAngTPB64, true, kInAngles>
                            : (const void*)k_eval_angles<T, LMAX>;
  int& bb = bps[phased ? 1 : 0][dev];
  if (bb == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(angles)");
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TPB, smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(angles)");
    bb = std::max(b, 1);
  }
  const int64_t ntiles = (n + TPB - 1) / TPB;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * bb);
  if (phased)
    k_eval_phased<LMAX, kAngTPB64, true, kInAngles><<<(unsigned)grid, TPB, smem, s>>>(
        reinterpret_cast<const double*>(ang), n, reinterpret_cast<double*>(out), ntiles, 0, vec ? 1 : 0);
  else
    k_eval_angles<T, LMAX><<<(unsigned)grid, TPB, smem, s>>>(ang, n, out, ntiles, vec ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "angles launch");
  return SHM_OK;
}

template <typename T>
shm_status ang_dispatch(const T* ang, int64_t n, int lmax, T* out, bool vec, cudaStream_t s, bool strict) {
  switch (lmax) {
    case 0: return ang_launch<T, 0>(ang, n, out, vec, s, strict);
    case 1: return ang_launch<T, 1>(ang, n, out, vec, s, strict);
    case 2: return ang_launch<T, 2>(ang, n, out, vec, s, strict);
    case 3: return ang_launch<T, 3>(ang, n, out, vec, s, strict);
    case 4: return ang_launch<T, 4>(ang, n, out, vec, s, strict);
    case 5: return ang_launch<T, 5>(ang, n, out, vec, s, strict);
    case 6: return ang_launch<T, 6>(ang, n, out, vec, s, strict);
    case 7: return ang_launch<T, 7>(ang, n, out, vec, s, strict);
    case 8: return ang_launch<T, 8>(ang, n, out, vec, s, strict);
    default: return ang_launch<T, 9>(ang, n, out, vec, s, strict);
  }
}

}  // namespace shm

extern "C" shm_status shm_eval_angles_ex(const void* angles, int64_t n, int lmax, shm_dtype dtype, unsigned flags,
                                         void* out, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_eval_angles_ex");
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (lmax < 0 || lmax > SHM_LMAX_CAP) return fail(SHM_EINVAL, "lmax must be in 0..9");
  if (n < 0) return fail(SHM_EINVAL, "n must be >= 0");
  if (flags & ~SHM_STRICT_FP64) return fail(SHM_EINVAL, "unknown flag bits");
  if (n == 0) return SHM_OK;
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  const int64_t L2 = (int64_t)(lmax + 1) * (lmax + 1);
  if (n > (INT64_MAX / 8) / (L2 * 8)) return fail(SHM_EINVAL, "n too large");
  if (!angles || !out) return fail(SHM_EINVAL, "angles and out must be non-null");
  if (!aligned(angles, es) || !aligned(out, es))
    return fail(SHM_EINVAL, "angles and out must be aligned to the element size");
  const size_t in_bytes = (size_t)n * 2 * es, out_bytes = (size_t)n * L2 * es;
  if (ranges_overlap(angles, in_bytes, out, out_bytes)) return fail(SHM_EINVAL, "angles and out overlap");
  shm_status st = check_device_range(angles, in_bytes, "angles");
  if (st != SHM_OK) return st;
  if ((st = check_device_range(out, out_bytes, "out")) != SHM_OK) return st;
  const bool vec = aligned(out, 16);
  const bool strict = (flags & SHM_STRICT_FP64) != 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == SHM_F64) return ang_dispatch<double>((const double*)angles, n, lmax, (double*)out, vec, s, strict);
  return ang_dispatch<float>((const float*)angles, n, lmax, (float*)out, vec, s, false);
}

extern "C" shm_status shm_eval_angles(const void* angles, int64_t n, int lmax, shm_dtype dtype, void* out,
                                      void* stream) {
  return shm_eval_angles_ex(angles, n, lmax, dtype, 0u, out, stream);
}
