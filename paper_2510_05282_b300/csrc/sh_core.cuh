// Per-point evaluation of all real spherical harmonics R_l^m, l <= LMAX, in
// normalised Cartesian coordinates (arXiv 2510.05282, Sec. II Eq. 8: on the
// unit sphere the harmonics are polynomials in xb, yb, zb).
//
// Scheme (constants in sh_coeffs.h, derivation in gen_coeffs.py):
//   A_m + i B_m = (xb + i yb)^m                 (sin^m(theta) e^{i m phi})
//   Qh_m^m = 1, Qh_{m+1}^m = zb,
//   Qh_l^m = zb Qh_{l-1}^m - G_lm q Qh_{l-2}^m   (q = 1 on the sphere)
//   R_l^0 = S_l0 Qh_l^0,  R_l^{+m} = S_lm Qh_l^m A_m,  R_l^{-m} = S_lm Qh_l^m B_m.
// This is the paper's structure -- a polynomial in zb (Horner/roots in App. C)
// times a homogeneous polynomial in xb, yb that the App. B rotations relate
// between m and -m -- reorganised so that all (l, m) share the powers A_m, B_m
// and the zb-polynomials are produced by one recurrence per m instead of one
// formula per (l, m): about 2.3 floating-point operations per harmonic at l = 9
// instead of about 14 for independent formulas.
#pragma once

#include <cstdint>

#include "sh_coeffs.h"

namespace shm {

constexpr double kInvSqrt4Pi = 0.28209479177387814347;

template <int LMAX>
struct NH {
  static constexpr int value = (LMAX + 1) * (LMAX + 1);
};

// ---------------------------------------------------------------------------
// Cartesian -> normalised coordinates.

// True when all three coordinates are +-0 (the r = 0 convention of Sec. II).
__device__ __forceinline__ bool is_origin(double x, double y, double z) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x) |
                                  (unsigned long long)__double_as_longlong(y) |
                                  (unsigned long long)__double_as_longlong(z);
  return (bits << 1) == 0ull;
}
__device__ __forceinline__ bool is_origin(float x, float y, float z) {
  const unsigned bits = __float_as_uint(x) | __float_as_uint(y) | __float_as_uint(z);
  return (bits << 1) == 0u;
}

// Scale (x, y, z) by a power of two so that the largest |component| lies in
// [1, 2): exact, and keeps x^2 + y^2 + z^2 away from overflow and underflow.
static __device__ __noinline__ void rescale_pow2(double& x, double& y, double& z) {
  const double ax = fabs(x), ay = fabs(y), az = fabs(z);
  const double mx = fmax(ax, fmax(ay, az));
  int e;
  (void)frexp(mx, &e);             // mx = f * 2^e, f in [0.5, 1)
  x = ldexp(x, 1 - e);
  y = ldexp(y, 1 - e);
  z = ldexp(z, 1 - e);
}

// FP64 unit direction.  The common case costs one rsqrt and five multiplies or
// FMAs; points whose r^2 would leave [2^-1000, 2^1000] are first rescaled by
// an exact power of two.
__device__ __forceinline__ void unit_dir(double x, double y, double z, double& xb, double& yb, double& zb) {
  double r2 = fma(z, z, fma(y, y, x * x));
  const unsigned ex = ((unsigned)__double2hiint(r2) >> 20) & 0x7ffu;  // biased exponent
  if (ex < 23u || ex > 2023u) {  // rare: tiny, huge, zero or non-finite
    rescale_pow2(x, y, z);
    r2 = fma(z, z, fma(y, y, x * x));
  }
  const double ri = rsqrt(r2);
  xb = x * ri;
  yb = y * ri;
  zb = z * ri;
}

// FP32 unit direction.  1/r is taken in FP64 when r < 1e-2 (and for r^2
// outside the safe float range); otherwise rsqrtf refined by one Newton step
// whose residual is formed with an FMA.
__device__ __forceinline__ void unit_dir(float x, float y, float z, float& xb, float& yb, float& zb) {
  const float r2 = fmaf(z, z, fmaf(y, y, x * x));
  if (!(r2 >= 1e-4f && r2 <= 1e30f)) {  // r < 1e-2, huge, or non-finite: FP64
    double dx = x, dy = y, dz = z;
    double ux, uy, uz;
    unit_dir(dx, dy, dz, ux, uy, uz);
    xb = (float)ux;
    yb = (float)uy;
    zb = (float)uz;
    return;
  }
  float ri = rsqrtf(r2);
  const float h = r2 * ri;              // ~ r
  const float e = fmaf(-h, ri, 1.0f);   // 1 - r^2 ri^2 (to first order)
  ri = fmaf(0.5f * ri, e, ri);
  xb = x * ri;
  yb = y * ri;
  zb = z * ri;
}

// ---------------------------------------------------------------------------
// FP64 row: writes R_l^m (k = l*l + l + m) through store(k, value).
// q = 1 (the non-homogeneous form): in binary64 the extra rounding of the
// coordinates costs < 1e-14 normwise at l = 9.

template <int LMAX, typename Store>
__device__ __forceinline__ void sh_row(double xb, double yb, double zb, Store&& store) {
  // m = 0
  store(0, SHM_S[0][0]);
  if constexpr (LMAX >= 1) {
    store(2, SHM_S[1][0] * zb);
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -SHM_G[l][0] * q2);
      store(l * l + l, SHM_S[l][0] * q);
      q2 = q1;
      q1 = q;
    }
  }
  double A = xb, B = yb;
#pragma unroll
  for (int m = 1; m <= LMAX; ++m) {
    if (m > 1) {
      const double An = fma(A, xb, -B * yb);
      const double Bn = fma(A, yb, B * xb);
      A = An;
      B = Bn;
    }
    store(m * m + 2 * m, SHM_S[m][m] * A);
    store(m * m, SHM_S[m][m] * B);
    if (m + 1 <= LMAX) {
      const double s = SHM_S[m + 1][m] * zb;
      const int k0 = (m + 1) * (m + 1) + (m + 1);
      store(k0 + m, s * A);
      store(k0 - m, s * B);
    }
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -SHM_G[l][m] * q2);
      const double s = SHM_S[l][m] * q;
      store(l * l + l + m, s * A);
      store(l * l + l - m, s * B);
      q2 = q1;
      q1 = q;
    }
  }
}

// FP64 row in l-major order: same arithmetic as sh_row<LMAX>(double...) (the
// same operations on the same operands, so bit-identical results), but the
// values come out l by l: all (x+iy)^m first, then for each l the next step of
// every m-recurrence.  The l-shells are grouped into phases of at most
// PHMAX values; phase(k0, width) is called after each group so the caller can
// stage and flush it.  store(k - k0, v) writes within the current phase.
template <int LMAX>
struct LPhases {
  // phase p covers l in [first[p], first[p+1])
  static constexpr int PHMAX = 37;
  static constexpr int count() {
    int n = 0, w = 0;
    for (int l = 0; l <= LMAX; ++l) {
      const int wl = 2 * l + 1;
      if (w > 0 && w + wl > PHMAX) {
        ++n;
        w = 0;
      }
      w += wl;
    }
    return n + 1;
  }
  static constexpr bool ends_phase(int l) {  // true if l is the last shell of its phase
    if (l == LMAX) return true;
    int w = 0;
    for (int ll = 0; ll <= l; ++ll) {
      const int wl = 2 * ll + 1;
      if (w > 0 && w + wl > PHMAX) w = 0;
      w += wl;
    }
    return w + 2 * (l + 1) + 1 > PHMAX;
  }
  static constexpr int max_width() {
    int w = 0, mx = 0;
    for (int l = 0; l <= LMAX; ++l) {
      const int wl = 2 * l + 1;
      if (w > 0 && w + wl > PHMAX) w = 0;
      w += wl;
      mx = w > mx ? w : mx;
    }
    return mx;
  }
};

template <int LMAX, typename Store, typename Phase>
__device__ __forceinline__ void sh_row_lmajor(double xb, double yb, double zb, Store&& store, Phase&& phase) {
  double A[LMAX + 1], B[LMAX + 1], q1[LMAX + 1], q2[LMAX + 1];
  A[0] = 1.0;
  B[0] = 0.0;
  if constexpr (LMAX >= 1) {
    A[1] = xb;
    B[1] = yb;
  }
#pragma unroll
  for (int m = 2; m <= LMAX; ++m) {
    A[m] = fma(A[m - 1], xb, -B[m - 1] * yb);
    B[m] = fma(A[m - 1], yb, B[m - 1] * xb);
  }
  int k0 = 0;
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      double s;
      if (l == m) {
        s = SHM_S[l][m];
        q2[m] = 1.0;
        q1[m] = 1.0;  // Qh_m^m
      } else if (l == m + 1) {
        s = SHM_S[l][m] * zb;
        q2[m] = 1.0;
        q1[m] = zb;
      } else {
        const double q = fma(zb, q1[m], -SHM_G[l][m] * q2[m]);
        s = SHM_S[l][m] * q;
        q2[m] = q1[m];
        q1[m] = q;
      }
      const int k = l * l + l;
      if (m == 0) {
        store(k - k0, s);
      } else {
        store(k + m - k0, (l == m) ? SHM_S[l][m] * A[m] : s * A[m]);
        store(k - m - k0, (l == m) ? SHM_S[l][m] * B[m] : s * B[m]);
      }
    }
    if (LPhases<LMAX>::ends_phase(l)) {
      phase(k0, (l + 1) * (l + 1) - k0);
      k0 = (l + 1) * (l + 1);
    }
  }
}

// ---------------------------------------------------------------------------
// Float-float (unevaluated sum hi + lo) helpers for the FP32 path.  The
// error-free transformations use the _rn intrinsics so that the compiler
// cannot contract them into FMAs.

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// FP32 row.  FP32 arithmetic throughout; two measures keep the error within
// 2e-6 of the l-shell norm up to l = 9:
//  * the homogeneous form q = xb^2 + yb^2 + zb^2 (1 only up to rounding in
//    FP32) keeps R a homogeneous polynomial of degree l, so the rounding of
//    the coordinates off the sphere costs ~l ulps instead of ~l(l+1)/2 near
//    the poles; q is formed exactly as a float-float 1 + dq;
//  * for m = 0 and m = 1, whose recurrences amplify rounding most near the
//    poles, the zb-recurrence runs in float-float (FMA-based error-free
//    products and sums, constants split into hi + lo); the result is rounded
//    to float once per value.
template <int LMAX, int M, typename Store>
__device__ __forceinline__ void sh_column_ff(float zb, float dq, float A, float B, Store&& store) {
  ff q2 = {1.0f, 0.0f}, q1 = {zb, 0.0f};
  auto emit = [&](int l, ff Q) {
    const ff p = two_prod(SHM_S_HI[l][M], Q.hi);
    const float v = __fadd_rn(p.hi, fmaf(SHM_S_HI[l][M], Q.lo, fmaf(SHM_S_LO[l][M], Q.hi, p.lo)));
    if constexpr (M == 0) {
      store(l * l + l, v);
    } else {
      store(l * l + l + M, v * A);
      store(l * l + l - M, v * B);
    }
  };
  if constexpr (M == 0) {
    store(0, SHM_S_HI[0][0]);
  } else {
    store(M * M + 2 * M, SHM_S_HI[M][M] * A);
    store(M * M, SHM_S_HI[M][M] * B);
  }
  if constexpr (M + 1 <= LMAX) emit(M + 1, q1);
#pragma unroll
  for (int l = M + 2; l <= LMAX; ++l) {
    ff t1 = two_prod(zb, q1.hi);
    t1.lo = fmaf(zb, q1.lo, t1.lo);
    ff t2 = two_prod(SHM_G_HI[l][M], q2.hi);
    t2.lo = fmaf(SHM_G_HI[l][M], q2.lo, fmaf(SHM_G_LO[l][M], q2.hi, t2.lo));
    t2.lo = fmaf(t2.hi, dq, t2.lo);  // times q = 1 + dq
    const ff d = two_sum(t1.hi, -t2.hi);
    const ff q = fast_two_sum(d.hi, __fadd_rn(d.lo, __fsub_rn(t1.lo, t2.lo)));
    emit(l, q);
    q2 = q1;
    q1 = q;
  }
}

template <int LMAX, typename Store>
__device__ __forceinline__ void sh_row(float xb, float yb, float zb, Store&& store) {
  // q = xb^2 + yb^2 + zb^2 as a float-float, then dq = q - 1
  const ff px = two_prod(xb, xb), py = two_prod(yb, yb), pz = two_prod(zb, zb);
  const ff s1 = two_sum(px.hi, py.hi);
  const ff s2 = two_sum(s1.hi, pz.hi);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(s1.lo, s2.lo), px.lo), __fadd_rn(py.lo, pz.lo));
  const ff qf = fast_two_sum(s2.hi, lo);
  const float dq = __fadd_rn(__fsub_rn(qf.hi, 1.0f), qf.lo);
  const float qq = qf.hi;

  sh_column_ff<LMAX, 0>(zb, dq, 0.0f, 0.0f, store);
  if constexpr (LMAX >= 1) sh_column_ff<LMAX, 1>(zb, dq, xb, yb, store);
  float A = xb, B = yb;
#pragma unroll
  for (int m = 2; m <= LMAX; ++m) {
    const float An = fmaf(A, xb, -B * yb);
    const float Bn = fmaf(A, yb, B * xb);
    A = An;
    B = Bn;
    store(m * m + 2 * m, (float)SHM_S[m][m] * A);
    store(m * m, (float)SHM_S[m][m] * B);
    if (m + 1 <= LMAX) {
      const float s = (float)SHM_S[m + 1][m] * zb;
      const int k0 = (m + 1) * (m + 1) + (m + 1);
      store(k0 + m, s * A);
      store(k0 - m, s * B);
    }
    float q2 = 1.0f, q1 = zb;
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l) {
      const float q = fmaf(zb, q1, -(float)SHM_G[l][m] * (qq * q2));
      const float s = (float)SHM_S[l][m] * q;
      store(l * l + l + m, s * A);
      store(l * l + l - m, s * B);
      q2 = q1;
      q1 = q;
    }
  }
}

// Full point: Cartesian (or already normalised) input -> row of harmonics.
template <int LMAX, typename T, typename Store>
__device__ __forceinline__ void sh_point(T x, T y, T z, bool normalized, Store&& store) {
  if (is_origin(x, y, z)) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
    store(0, (T)kInvSqrt4Pi);
#pragma unroll
    for (int k = 1; k < NH<LMAX>::value; ++k) store(k, (T)0);
    return;
  }
  T xb = x, yb = y, zb = z;
  if (!normalized) unit_dir(x, y, z, xb, yb, zb);
  sh_row<LMAX>(xb, yb, zb, store);
}

}  // namespace shm
