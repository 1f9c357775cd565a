// shm_eval_spinor: the spin-1/2 spinor harmonics of Sec. II Eq. 7 fused into
// the evaluator.  For orbital l, j = l + s/2 (s = +-1) and m_j:
//   upper = s sqrt((l + s m_j + 1/2) / (2l+1)) Y_l^{m_j - 1/2}
//   lower =   sqrt((l - s m_j + 1/2) / (2l+1)) Y_l^{m_j + 1/2}
// and, from the real harmonics of the same point, Y_l^0 = R_l^0,
// Y_l^{+m} = (-1)^m (R_l^m + i R_l^{-m}) / sqrt2, Y_l^{-m} = (R_l^m - i R_l^{-m}) / sqrt2.
// So every output value is a constant times one real harmonic: the kernels
// stage the real rows in shared memory (as shm_eval does) and the copy-out
// reads, per complex output component, a per-CTA map entry (the two real
// values and the two constants) and writes coefficient x value.  In FP64 the
// products are split between the FP64 pipe (real parts) and float-float
// arithmetic on the FP32 pipe (imaginary parts): 800 binary64 products per
// point at l = 9 would make the kernel FP64-bound well above its HBM time.
// With SHM_STRICT_FP64 (k_eval_spinor64s) the rows are the all-binary64
// m-major rows, staged whole, and both parts are binary64 products: the
// arithmetic of the definition, FP64-pipe bound.
// Output [n][2 (lmax+1)^2 spinors][upper, lower][re, im].
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "sh_core.cuh"
#include "sh_tile.cuh"
#include "shm_internal.h"

namespace shm {

constexpr int kSpTPB64 = 128;
constexpr int kSpPhase = 25;  // real values staged per row and phase (FP64; fastest of 19, 25, 37 measured)
constexpr int kSpTPB32 = 64;
constexpr double kRsqrt2 = 0.70710678118654752440;

// Map entry of output component q = 2 * spinor + c (c = 0 upper, 1 lower):
// the real part is cre * R[ka], the imaginary part cim * R[kb] (0 when
// im_zero: m = 0), ka = l*l + l + |m|, kb = l*l + l - |m|.  Components with
// |m| > l get coefficient 0.
struct SpinorTerm {
  int ka, kb;
  double cre, cim;
  bool im_zero;
};

__device__ SpinorTerm spinor_term(int q) {
  const int sp = q >> 1, c = q & 1;
  int l = 0;
  while (2 * (l + 1) * (l + 1) <= sp) ++l;
  int t = sp - 2 * l * l;  // position in the l block: j = l - 1/2 first (2l values), then j = l + 1/2
  int s = 1, tj = 2 * l + 1;
  if (t < 2 * l) {
    s = -1;
    tj = 2 * l - 1;
  } else {
    t -= 2 * l;
  }
  const int tmj = 2 * t - tj;                      // 2 m_j
  const int m = (c == 0 ? tmj - 1 : tmj + 1) / 2;  // m of the Y this component carries
  const int num = c == 0 ? 2 * l + s * tmj + 1 : 2 * l - s * tmj + 1;  // 2 (l +- s m_j + 1/2)
  double a = sqrt((double)num / (double)(2 * (2 * l + 1)));
  if (c == 0 && s < 0) a = -a;
  int mu = m < 0 ? -m : m;
  if (mu > l) {
    a = 0.0;
    mu = 0;
  }
  SpinorTerm r;
  r.im_zero = mu == 0;
  if (mu == 0) {
    r.cre = a;
    r.cim = 0.0;
  } else if (m > 0) {
    r.cre = r.cim = ((m & 1) ? -a : a) * kRsqrt2;
  } else {
    r.cre = a * kRsqrt2;
    r.cim = -r.cre;
  }
  const int kc = l * l + l;
  r.ka = kc + mu;
  r.kb = kc - mu;
  return r;
}

__device__ __forceinline__ uint32_t spinor_idx(const SpinorTerm& t) {
  return (uint32_t)t.ka | ((uint32_t)t.kb << 16) | (t.im_zero ? 0x80000000u : 0u);
}

// FP64 map entry: binary64 coefficient for the real part (R_l^{|m|} is staged
// as binary64), float-float coefficient for the imaginary part (R_l^{-|m|} is
// staged as float-float).  Padded to 24 bytes: read as two 8-byte loads, the
// kernel took 7.96 ms on the 192^3 grid against 8.20 ms with 16-byte entries
// read by one 16-byte load, and 8.10 ms with the two parts in separate arrays
// (the cause was not isolated; register allocation differs between the three).
struct __align__(8) SpinorCoef64 {
  double re;
  float im_hi, im_lo;
  float pad[2];
};

__device__ __forceinline__ void st_pair(double* p, double a, double b) { __stcs(reinterpret_cast<double2*>(p), make_double2(a, b)); }
__device__ __forceinline__ void st_pair(float* p, float a, float b) { __stcs(reinterpret_cast<float2*>(p), make_float2(a, b)); }

__device__ __forceinline__ void st_out(double* o, double re, double im, bool vec) {
  if (vec) {
    st_pair(o, re, im);
  } else {
    __stcs(o, re);
    __stcs(o + 1, im);
  }
}
__device__ __forceinline__ void st_out(float* o, float re, float im, bool vec) {
  if (vec) {
    st_pair(o, re, im);
  } else {
    __stcs(o, re);
    __stcs(o + 1, im);
  }
}

// Copy-out of the staged real values [k0, k0 + w) (whole l-shells) of `rows`
// points: component q = 4 k0 + c, c < 4w, of point r goes to
// dst[(r * NC + q) * 2 + {0, 1}].
//
// FP64: the tile slot of R_l^m holds binary64 for m >= 0 and float-float
// (hi, lo) for m < 0.  The real part is one binary64 multiply; the imaginary
// part is a float-float multiply by the split coefficient and an exact
// integer-assembled conversion, so the FP64 pipe carries half the products.
template <int TPB, int RS, int NC>
__device__ __forceinline__ void spinor_copy_out64(const double* __restrict__ tile, int rows, int k0, int w,
                                                  const uint32_t* __restrict__ midx,
                                                  const SpinorCoef64* __restrict__ mcoef, double* __restrict__ dst,
                                                  bool vec) {
  // thread (rs, c) = divmod(threadIdx, w) writes the components
  // 4 k0 + c + u w, u = 0..3, of rows rs, rs + RP, ... (RP = TPB / w): the
  // map entries are read once per phase, the addresses advance by constant
  // steps, and each store instruction of a warp covers adjacent components
  const int RP = TPB / w;
  const int rs = (int)threadIdx.x / w;
  const int c = (int)threadIdx.x - rs * w;
  if (rs >= RP) return;
  const int q0 = 4 * k0 + c;
  uint32_t e[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) e[u] = midx[q0 + u * w];
  const double* src = tile + rs * RS - k0;
  double* o = dst + 2 * ((int64_t)rs * NC + q0);
  for (int r = rs; r < rows; r += RP) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const SpinorCoef64 cf = mcoef[q0 + u * w];
      const double re = cf.re * src[e[u] & 0x7fffu];
      const float2 b = reinterpret_cast<const float2*>(src)[(e[u] >> 16) & 0x7fffu];
      const double im = (e[u] >> 31) ? 0.0 : ff_to_double(ff_mul_c(ff{b.x, b.y}, cf.im_hi, cf.im_lo));
      st_out(o + 2 * u * w, re, im, vec);
    }
    src += RP * RS;
    o += 2 * (int64_t)RP * NC;
  }
}

// FP32: coefficient x value for both parts.
template <int TPB, int RS, int NC>
__device__ __forceinline__ void spinor_copy_out32(const float* __restrict__ tile, int rows,
                                                  const uint32_t* __restrict__ midx, const float2* __restrict__ mcoef,
                                                  float* __restrict__ dst, bool vec) {
  const int nv = rows * NC;
  for (int j = threadIdx.x; j < nv; j += TPB) {
    const int r = j / NC;
    const int q = j - r * NC;
    const uint32_t e = midx[q];
    const float2 cf = mcoef[q];
    const float* src = tile + r * RS;
    st_out(dst + 2 * (int64_t)j, cf.x * src[e & 0x7fffu], cf.y * src[(e >> 16) & 0x7fffu], vec);
  }
}

// FP64 rows: hybrid real rows in l-major order, staged one group of l-shells
// at a time (as shm_eval's phased-hybrid variant).
template <int LMAX, int TPB = kSpTPB64, int PH = kSpPhase>
__global__ void __launch_bounds__(TPB, 640 / TPB) k_eval_spinor64(const double* __restrict__ pts, int64_t n,
                                                       double* __restrict__ out, int64_t ntiles, int normalized,
                                                       int vec) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int NC = 4 * L2;
  constexpr int RS = LPhases<LMAX, PH>::max_width() | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t midx[NC];
  __shared__ SpinorCoef64 mcoef[NC];
  double* tile = reinterpret_cast<double*>(smem_raw);
  for (int q = threadIdx.x; q < NC; q += TPB) {
    const SpinorTerm t = spinor_term(q);
    const float hi = (float)t.cim;
    midx[q] = spinor_idx(t);
    mcoef[q] = SpinorCoef64{t.cre, hi, (float)(t.cim - (double)hi), {0.0f, 0.0f}};
  }
  __syncthreads();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * TPB;
    const int rows = (int)min((int64_t)TPB, n - p0);
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
    float2* rowf = reinterpret_cast<float2*>(row);
    const bool bad = nonfinite3(xb, yb, zb);  // the hybrid row code needs a finite direction
    double* dst = out + p0 * 2 * NC;
    auto store = [&](int k, int k0, auto v) {
      if constexpr (std::is_same<decltype(v), double>::value)
        row[k - k0] = v;  // m >= 0: binary64
      else
        rowf[k - k0] = make_float2(v.hi, v.lo);  // m < 0: float-float
    };
    auto flush = [&](int k0, int w) {
      if (origin || bad) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0 (zero is 0 in both formats)
        // a non-finite direction: a pattern that is NaN both as binary64 and
        // as a float pair, for the binary64 and the float-float slots alike
        const double fill = origin ? 0.0 : __longlong_as_double(0x7ff800007fc00000ll);
        for (int c = 0; c < w; ++c) row[c] = (k0 + c == 0) ? kInvSqrt4Pi : fill;
      }
      __syncthreads();
      spinor_copy_out64<TPB, RS, NC>(tile, rows, k0, w, midx, mcoef, dst, vec != 0);
      __syncthreads();
    };
    sh_row_hybrid_lmajor<LMAX, false, PH, true>(xb, yb, zb, store, flush);
  }
}

// All-binary64 spinors (SHM_STRICT_FP64): real rows of sh_row<LMAX>, staged
// whole with an odd row stride; every component part is one binary64
// product coefficient x real value.
constexpr int kSpTPBs = 64;

template <int LMAX>
__global__ void __launch_bounds__(kSpTPBs) k_eval_spinor64s(const double* __restrict__ pts, int64_t n,
                                                           double* __restrict__ out, int64_t ntiles, int normalized,
                                                           int vec) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int NC = 4 * L2;
  constexpr int RS = L2 | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // per component: the index word (spinor_idx, with the signs of the real
  // and imaginary coefficients in bits 29 and 30) and one coefficient
  // magnitude (|cre| = |cim| whenever the imaginary part is not zero): 4.8 KB
  // instead of 8 KB for two signed coefficients, so that four CTAs fit an SM
  __shared__ uint32_t midx[NC];
  __shared__ double mmag[NC];
  double* tile = reinterpret_cast<double*>(smem_raw);
  for (int q = threadIdx.x; q < NC; q += kSpTPBs) {
    const SpinorTerm t = spinor_term(q);
    const uint32_t sre = __double_as_longlong(t.cre) < 0 ? (1u << 29) : 0u;
    const uint32_t sim = __double_as_longlong(t.cim) < 0 ? (1u << 30) : 0u;
    midx[q] = spinor_idx(t) | sre | sim;
    mmag[q] = fabs(t.cre);
  }
  __syncthreads();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kSpTPBs;
    const int rows = (int)min((int64_t)kSpTPBs, n - p0);
    if ((int)threadIdx.x < rows) {
      const int64_t p = p0 + threadIdx.x;
      double* row = tile + threadIdx.x * RS;
      // the output products on the integer pipes (dmul_int): the same bits
      sh_point<LMAX, false, false, kEmuOut>(pts[3 * p], pts[3 * p + 1], pts[3 * p + 2], normalized != 0,
                                            [&](int k, double v) { row[k] = v; });
    }
    __syncthreads();
    const int nv = rows * NC;
    double* dst = out + p0 * 2 * NC;
    for (int j = threadIdx.x; j < nv; j += kSpTPBs) {
      const int r = j / NC, q = j - r * NC;
      const uint32_t e = midx[q];
      const unsigned long long mg = (unsigned long long)__double_as_longlong(mmag[q]);
      const double cre = __longlong_as_double((long long)(mg | ((unsigned long long)((e >> 29) & 1u) << 63)));
      const double cim = __longlong_as_double((long long)(mg | ((unsigned long long)((e >> 30) & 1u) << 63)));
      const double* src = tile + r * RS;
      const double re = cre * src[e & 0x7fffu];
      const double im = (e >> 31) ? 0.0 : cim * src[(e >> 16) & 0x1fffu];  // bits 29, 30: the signs
      st_out(dst + 2 * (int64_t)j, re, im, vec != 0);
    }
    __syncthreads();
  }
}

// FP32 rows: the FP32 row code, staged a full row at a time.
template <int LMAX>
__global__ void __launch_bounds__(kSpTPB32) k_eval_spinor32(const float* __restrict__ pts, int64_t n,
                                                            float* __restrict__ out, int64_t ntiles, int normalized,
                                                            int vec) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int NC = 4 * L2;
  constexpr int RS = TileShape<LMAX>::RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t midx[NC];
  __shared__ float2 mcoef[NC];
  float* tile = reinterpret_cast<float*>(smem_raw);
  for (int q = threadIdx.x; q < NC; q += kSpTPB32) {
    const SpinorTerm t = spinor_term(q);
    midx[q] = spinor_idx(t);
    mcoef[q] = make_float2((float)t.cre, (float)t.cim);
  }
  __syncthreads();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kSpTPB32;
    const int rows = (int)min((int64_t)kSpTPB32, n - p0);
    if ((int)threadIdx.x < rows) {
      const int64_t p = p0 + threadIdx.x;
      const float x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
      float* row = tile + threadIdx.x * RS;
      if (is_origin(x, y, z)) {
        for (int c = 0; c < L2; ++c) row[c] = c == 0 ? (float)kInvSqrt4Pi : 0.0f;
      } else {
        float xb = x, yb = y, zb = z;
        if (!normalized) unit_dir(x, y, z, xb, yb, zb);
        if (nonfinite3(xb, yb, zb)) {  // NaN in every value but l = 0
          for (int c = 0; c < L2; ++c) row[c] = c == 0 ? (float)kInvSqrt4Pi : __int_as_float(0x7fc00000);
        } else {
          sh_row<LMAX>(xb, yb, zb, [&](int k, float v) { row[k] = v; });
        }
      }
    }
    __syncthreads();
    spinor_copy_out32<kSpTPB32, RS, NC>(tile, rows, midx, mcoef, out + p0 * 2 * NC, vec != 0);
    __syncthreads();
  }
}

template <int LMAX>
shm_status spinor_launch(const void* pts, int64_t n, bool f64, void* out, bool normalized, bool vec,
                         cudaStream_t s, bool strict) {
  constexpr int MAXDEV = 64;
  static int bps[3][MAXDEV] = {};
  const int dev = current_device();
  if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
  strict = strict && f64;
  const int tpb = strict ? kSpTPBs : (f64 ? kSpTPB64 : kSpTPB32);
  const size_t smem = strict ? (size_t)kSpTPBs * (NH<LMAX>::value | 1) * 8
                      : f64  ? (size_t)kSpTPB64 * (LPhases<LMAX, kSpPhase>::max_width() | 1) * 8
                             : (size_t)kSpTPB32 * TileShape<LMAX>::RS * 4;
  const void* kern = strict ? (const void*)k_eval_spinor64s<LMAX>
                     : f64  ? (const void*)k_eval_spinor64<LMAX>
                            : (const void*)k_eval_spinor32<LMAX>;
  int& b = bps[strict ? 2 : (f64 ? 1 : 0)][dev];
  if (b == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_eval_spinor)");
    int bb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, kern, tpb, smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_eval_spinor)");
    b = std::max(bb, 1);
  }
  const int64_t ntiles = (n + tpb - 1) / tpb;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * b);
  if (strict)
    k_eval_spinor64s<LMAX><<<(unsigned)grid, tpb, smem, s>>>((const double*)pts, n, (double*)out, ntiles,
                                                              normalized, vec);
  else if (f64)
    k_eval_spinor64<LMAX><<<(unsigned)grid, tpb, smem, s>>>((const double*)pts, n, (double*)out, ntiles,
                                                             normalized, vec);
  else
    k_eval_spinor32<LMAX><<<(unsigned)grid, tpb, smem, s>>>((const float*)pts, n, (float*)out, ntiles,
                                                             normalized, vec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "k_eval_spinor launch");
  return SHM_OK;
}

}  // namespace shm

extern "C" int shm_num_spinors(int lmax) {
  return (lmax < 0 || lmax > SHM_LMAX_CAP) ? -1 : 2 * (lmax + 1) * (lmax + 1);
}

extern "C" shm_status shm_eval_spinor(const void* points, int64_t n, int lmax, shm_dtype dtype, unsigned flags,
                                      void* out, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_eval_spinor");
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (lmax < 0 || lmax > SHM_LMAX_CAP) return fail(SHM_EINVAL, "lmax must be in 0..9");
  if (n < 0) return fail(SHM_EINVAL, "n must be >= 0");
  if (flags & ~(SHM_NORMALIZED_INPUT | SHM_STRICT_FP64)) return fail(SHM_EINVAL, "unknown flag bits");
  if (n == 0) return SHM_OK;
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  const int64_t L2 = (int64_t)(lmax + 1) * (lmax + 1);
  if (n > (INT64_MAX / 16) / (L2 * 64)) return fail(SHM_EINVAL, "n too large");
  if (!points || !out) return fail(SHM_EINVAL, "points and out must be non-null");
  if (!aligned(points, es) || !aligned(out, es))
    return fail(SHM_EINVAL, "points and out must be aligned to the element size");
  const size_t in_bytes = (size_t)n * 3 * es, out_bytes = (size_t)n * L2 * 8 * es;
  if (ranges_overlap(points, in_bytes, out, out_bytes)) return fail(SHM_EINVAL, "points and out overlap");
  shm_status st = check_device_range(points, in_bytes, "points");
  if (st != SHM_OK) return st;
  if ((st = check_device_range(out, out_bytes, "out")) != SHM_OK) return st;
  const bool f64 = dtype == SHM_F64, norm = (flags & SHM_NORMALIZED_INPUT) != 0, vec = aligned(out, 2 * es);
  const bool strict = (flags & SHM_STRICT_FP64) != 0;
  cudaStream_t s = (cudaStream_t)stream;
  switch (lmax) {
    case 0: return spinor_launch<0>(points, n, f64, out, norm, vec, s, strict);
    case 1: return spinor_launch<1>(points, n, f64, out, norm, vec, s, strict);
    case 2: return spinor_launch<2>(points, n, f64, out, norm, vec, s, strict);
    case 3: return spinor_launch<3>(points, n, f64, out, norm, vec, s, strict);
    case 4: return spinor_launch<4>(points, n, f64, out, norm, vec, s, strict);
    case 5: return spinor_launch<5>(points, n, f64, out, norm, vec, s, strict);
    case 6: return spinor_launch<6>(points, n, f64, out, norm, vec, s, strict);
    case 7: return spinor_launch<7>(points, n, f64, out, norm, vec, s, strict);
    case 8: return spinor_launch<8>(points, n, f64, out, norm, vec, s, strict);
    default: return spinor_launch<9>(points, n, f64, out, norm, vec, s, strict);
  }
}
