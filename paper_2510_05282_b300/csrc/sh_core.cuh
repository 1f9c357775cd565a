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

// Scale constants: S for the real harmonics, S / sqrt2 (m > 0) for the
// complex ones (Y_l^{+-m} = (+-1)^m (R_l^m +- i R_l^{-m}) / sqrt2, m > 0).
template <bool CX>
__device__ __forceinline__ constexpr double Sd(int l, int m) { return CX ? SHM_SC[l][m] : SHM_S[l][m]; }
template <bool CX>
__device__ __forceinline__ constexpr float Shi(int l, int m) { return CX ? SHM_SC_HI[l][m] : SHM_S_HI[l][m]; }
template <bool CX>
__device__ __forceinline__ constexpr float Slo(int l, int m) { return CX ? SHM_SC_LO[l][m] : SHM_S_LO[l][m]; }

__device__ __forceinline__ constexpr int l_of_k(int k) { return SHM_L_OF_K[k]; }

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

template <int LMAX, bool CX = false, typename Store>
__device__ __forceinline__ void sh_row(double xb, double yb, double zb, Store&& store) {
  // m = 0
  store(0, Sd<CX>(0, 0));
  if constexpr (LMAX >= 1) {
    store(2, Sd<CX>(1, 0) * zb);
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -SHM_G[l][0] * q2);
      store(l * l + l, Sd<CX>(l, 0) * q);
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
    store(m * m + 2 * m, Sd<CX>(m, m) * A);
    store(m * m, Sd<CX>(m, m) * B);
    if (m + 1 <= LMAX) {
      const double s = Sd<CX>(m + 1, m) * zb;
      const int k0 = (m + 1) * (m + 1) + (m + 1);
      store(k0 + m, s * A);
      store(k0 - m, s * B);
    }
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -SHM_G[l][m] * q2);
      const double s = Sd<CX>(l, m) * q;
      store(l * l + l + m, s * A);
      store(l * l + l - m, s * B);
      q2 = q1;
      q1 = q;
    }
  }
}

// ---------------------------------------------------------------------------
// Binary64 multiplication on the integer pipes.
//
// The all-binary64 rows are bound by the FP64 pipe of a B300 (about 2
// instructions per SM-cycle) while its integer pipes idle.  dmul_int returns
// the IEEE-754 binary64 product a*b rounded to nearest-even -- the value the
// DMUL instruction returns, bit for bit -- computed with 32-bit integer
// multiply-adds, shifts and adds: the exact 106-bit product of the 53-bit
// significands, then the rounding of IEEE 754-2008 Sec. 4.3.1.  It covers
// normal operands with a normal product, and sets `bad` for anything else
// (a zero, subnormal, infinite or NaN operand, or a product that would
// overflow or be subnormal) without giving a meaningful value: the callers
// then compute the whole row again with the FP64 instructions.
//
// With ma, mb the significands (2^52 <= ma, mb < 2^53) split into 21 + 32
// bits, P = ma mb (2^104 <= P < 2^106) is accumulated in three 64-bit partial
// sums (four 32x32 -> 64-bit multiply-adds): P = t3 2^64 + lo(t2) 2^32 +
// lo(p0).  The significand of the result is P >> s, s = 52 + (P >= 2^105);
// the round bit is bit s-1 of P, the sticky bit the OR of the bits below it;
// round up when round && (sticky || the significand is odd).  The biased
// exponent is ea + eb - 1023 + (s - 52); adding the significand (with its
// implicit bit 52) and the round-up to (exponent - 1) << 52 carries into the
// exponent by itself when the rounding reaches 2^53.
__device__ __forceinline__ double dmul_int(double a, double b, unsigned& bad) {
  const unsigned ah = (unsigned)__double2hiint(a), al = (unsigned)__double2loint(a);
  const unsigned bh = (unsigned)__double2hiint(b), bl = (unsigned)__double2loint(b);
  const unsigned ea = (ah >> 20) & 0x7ffu, eb = (bh >> 20) & 0x7ffu;
  const unsigned mah = (ah & 0xfffffu) | 0x100000u, mbh = (bh & 0xfffffu) | 0x100000u;
  const unsigned long long p0 = (unsigned long long)al * bl;
  const unsigned long long t1 = (unsigned long long)mah * bl + (p0 >> 32);
  const unsigned long long t2 = (unsigned long long)al * mbh + (t1 & 0xffffffffull);
  const unsigned long long t3 = (unsigned long long)mah * mbh + (t1 >> 32) + (t2 >> 32);
  const unsigned mid = (unsigned)t2, low = (unsigned)p0;
  const unsigned top = (unsigned)(t3 >> 41);  // 1 when P >= 2^105
  const unsigned sh = 20u + top;               // s - 32: the shift of the middle word
  const unsigned long long M = (t3 << (32u - sh)) | (unsigned long long)(mid >> sh);
  const unsigned round = (mid >> (sh - 1u)) & 1u;
  const unsigned sticky = (mid & ((1u << (sh - 1u)) - 1u)) | low;
  const unsigned inc = round & (((sticky != 0u) ? 1u : 0u) | (unsigned)(M & 1ull));
  const int e = (int)ea + (int)eb - 1023 + (int)top;  // biased exponent of the result
  bad |= ((ea - 1u) >= 2046u) | ((eb - 1u) >= 2046u) | ((unsigned)(e - 1) >= 2045u);
  const unsigned long long r = ((unsigned long long)(unsigned)(e - 1) << 52) + M + inc;
  return __longlong_as_double((long long)(r | ((unsigned long long)((ah ^ bh) & 0x80000000u) << 32)));
}

// sh_row<LMAX>(double...) with some of its products computed by dmul_int:
// the same binary64 operations on the same operands, so the same bits when
// `bad` stays 0.  EMU selects the products by role (bit mask):
//   kEmuOut   -- the products that leave as harmonics: s A, s B and S A, S B;
//   kEmuScale -- the scales s = S_lm Qh (and S zb at l = m + 1), m >= 1;
//   kEmuRec   -- G_lm Qh_{l-2} inside the recurrences, m >= 1;
//   kEmuM0    -- the products of the m = 0 column (its scales and G Qh).
// Every product dmul_int cannot do exactly raises `bad`; the caller then
// recomputes the row with sh_row (a point with a zero or subnormal power of
// x + iy, for instance on an axis, takes that path).
enum : int { kEmuOut = 1, kEmuScale = 2, kEmuRec = 4, kEmuM0 = 8 };

template <int LMAX, int EMU, bool CX = false, typename Store>
__device__ __forceinline__ unsigned sh_row_emu(double xb, double yb, double zb, Store&& store) {
  unsigned bad = 0u;
  auto mul = [&](bool emu, double a, double b) { return emu ? dmul_int(a, b, bad) : a * b; };
  constexpr bool OUT = (EMU & kEmuOut) != 0, SCL = (EMU & kEmuScale) != 0, REC = (EMU & kEmuRec) != 0,
                 M0 = (EMU & kEmuM0) != 0;
  store(0, Sd<CX>(0, 0));
  if constexpr (LMAX >= 1) {
    store(2, mul(M0, Sd<CX>(1, 0), zb));
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -mul(M0, SHM_G[l][0], q2));
      store(l * l + l, mul(M0, Sd<CX>(l, 0), q));
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
    store(m * m + 2 * m, mul(OUT, Sd<CX>(m, m), A));
    store(m * m, mul(OUT, Sd<CX>(m, m), B));
    if (m + 1 <= LMAX) {
      const double s = mul(SCL, Sd<CX>(m + 1, m), zb);
      const int k0 = (m + 1) * (m + 1) + (m + 1);
      store(k0 + m, mul(OUT, s, A));
      store(k0 - m, mul(OUT, s, B));
    }
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -mul(REC, SHM_G[l][m], q2));
      const double s = mul(SCL, Sd<CX>(l, m), q);
      store(l * l + l + m, mul(OUT, s, A));
      store(l * l + l - m, mul(OUT, s, B));
      q2 = q1;
      q1 = q;
    }
  }
  return bad;
}

// FP64 row in l-major order: same arithmetic as sh_row<LMAX>(double...) (the
// same operations on the same operands, so bit-identical results), but the
// values come out l by l: all (x+iy)^m first, then for each l the next step of
// every m-recurrence.  The l-shells are grouped into phases of at most
// PHMAX values; phase(k0, width) is called after each group so the caller can
// stage and flush it.  store(k, k0, v) writes value k of the current phase,
// which starts at k0.
template <int LMAX, int PHMAX_ = 37>
struct LPhases {
  static constexpr int PHMAX = PHMAX_;  // values per phase at most (a single shell may exceed it)
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

template <int LMAX, bool CX = false, int PHMAX = 37, typename Store, typename Phase>
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
        s = Sd<CX>(l, m);
        q2[m] = 1.0;
        q1[m] = 1.0;  // Qh_m^m
      } else if (l == m + 1) {
        s = Sd<CX>(l, m) * zb;
        q2[m] = 1.0;
        q1[m] = zb;
      } else {
        const double q = fma(zb, q1[m], -SHM_G[l][m] * q2[m]);
        s = Sd<CX>(l, m) * q;
        q2[m] = q1[m];
        q1[m] = q;
      }
      const int k = l * l + l;
      if (m == 0) {
        store(k, k0, s);
      } else {
        store(k + m, k0, (l == m) ? Sd<CX>(l, m) * A[m] : s * A[m]);
        store(k - m, k0, (l == m) ? Sd<CX>(l, m) * B[m] : s * B[m]);
      }
    }
    if (LPhases<LMAX, PHMAX>::ends_phase(l)) {
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

// Float-float arithmetic (hi + lo, ~48-bit significand) and exact
// conversions between binary64 and float-float, done with integer and FP32
// instructions only (the FP64 pipe of a B300 is ~1/58 of its FP32 pipe).
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_c(ff a, float ch, float cl) {  // times the constant ch + cl
  ff p = two_prod(ch, a.hi);
  p.lo = fmaf(ch, a.lo, fmaf(cl, a.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
// Products left unnormalised (|lo| may reach ~ulp(hi)): for operands of a
// following ff_add or ff_mul, which renormalise.
__device__ __forceinline__ ff ff_mul_u(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return p;
}
__device__ __forceinline__ ff ff_mul_c_u(ff a, float ch, float cl) {
  ff p = two_prod(ch, a.hi);
  p.lo = fmaf(ch, a.lo, fmaf(cl, a.hi, p.lo));
  return p;
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// Conversions between binary64 and float-float use integer instructions
// only: on a B300 the int<->float and float<->double conversion instructions
// issue to the same narrow pipe as FP64 arithmetic.

// binary64 -> float-float, both parts rounded to nearest (ties away from
// zero): hi = d rounded to a 24-bit significand (an add of half a unit to the
// bit pattern, whose carry moves into the exponent by itself); the remainder
// d - hi is an integer count of d's ulp below 2^29 in magnitude, of the
// opposite sign when hi was rounded up, and lo is that count rounded to 24
// bits.  |hi + lo - d| <= 2^-49 |d| with no bias (a truncating conversion
// biases every coordinate towards zero, and the biases add up along the
// recurrences: 9e-14 instead of 4e-14 normwise at l = 9).  |d| below 2^-74
// maps to 0 (absolute error < 2^-73); NaN and |d| >= 2^128 map to a
// NaN/infinite hi.  Branch-free (selects only).
__device__ __forceinline__ ff ff_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;         // unbiased exponent of d
  const unsigned low = (unsigned)(b & 0x1fffffffull);      // the 29 bits below hi's significand
  const bool up = low >= 0x10000000u;
  const unsigned long long bh = (b & ~0x1fffffffull) + (up ? 0x20000000ull : 0ull);
  const int eh = (int)((bh >> 52) & 0x7ffu) - 1023;        // hi's exponent (one more after a carry)
  const bool tiny = e < -74, big = eh > 127;
  const unsigned ef = big ? 255u : (unsigned)(eh + 127);
  const unsigned mf = (unsigned)((bh >> 29) & 0x7fffffull) | ((big && (b << 12) != 0ull) ? 0x400000u : 0u);
  const unsigned hib = tiny ? 0u : (sign | (ef << 23) | mf);
  const unsigned mag = up ? 0x20000000u - low : low;       // |d - hi| in units of 2^(e-52)
  const unsigned lsign = up ? (sign ^ 0x80000000u) : sign;
  int p = 31 - __clz(mag | 1u);                            // top set bit, 0..29
  const int sh = p - 23;
  unsigned m = sh > 0 ? (mag + (1u << (sh - 1))) >> sh : mag << (-sh);  // 24-bit significand, rounded
  const bool carry = m >> 24;                              // rounding reached 2^24
  m = carry ? m >> 1 : m;
  p += carry ? 1 : 0;
  const unsigned lob = (tiny || big || mag == 0u) ? 0u : (lsign | ((unsigned)(p + e + 75) << 23) | (m & 0x7fffffu));
  return {__uint_as_float(hib), __uint_as_float(lob)};
}

// float-float (normalised: |lo| <= ulp(hi)/2, hi finite) -> binary64.  The
// double of hi is assembled from its bits (exponent rebiased by 1023 - 127 =
// 896, significand extended by 29 zero bits); lo is then added as a signed
// count k of units of the result's last place, directly on the bit pattern
// (a double's bit pattern is monotonic in its magnitude, and the carry or
// borrow moves into the exponent by itself).  k = trunc(lo * sign(hi) *
// 2^(52 - E)), E the exponent of hi + lo: one FP32 multiply by a power of two
// built from the exponent bits and one float -> int conversion (neither uses
// the FP64 pipe).  E comes from hi + lo added toward zero, which differs from
// hi's exponent exactly when hi is a power of two and lo has the opposite sign
// -- the case where the result lies in the binade below, whose units are half
// as large.  |k| < 2^30, so the count fits the conversion; the truncated part
// is below one unit (result within 1 ulp of hi + lo).  hi = +-0 gives +-0.
// For |hi| < 2^-75 the scale leaves the FP32 range and the result is off by
// less than 2^-96 in absolute terms.  A NaN or infinite hi gives a meaningless
// finite value: the row code, which only meets finite values for a finite
// direction, uses this form, and the callers write NaN rows for non-finite
// points.  Branch-free.
__device__ __forceinline__ double ff_to_double_finite(ff a) {
  const unsigned hb = __float_as_uint(a.hi);
  const unsigned sg = hb & 0x80000000u;
  unsigned hi32 = ((hb >> 3) & 0x0fffffffu) + (896u << 20) + sg;
  hi32 = (hb & 0x7f800000u) == 0u ? sg : hi32;
  const unsigned lo32 = hb << 29;
  const unsigned es = __float_as_uint(__fadd_rz(a.hi, a.lo)) & 0x7f800000u;  // binade of hi + lo
  const float scale = __uint_as_float((306u << 23) - es + sg);                  // sign(hi) 2^(52 - E)
  const int k = __float2int_rz(a.lo * scale);
  return __longlong_as_double((long long)(((unsigned long long)hi32 << 32) | lo32) + (long long)k);
}
// The same with a NaN or infinite hi mapped to NaN.
__device__ __forceinline__ double ff_to_double(ff a) {
  const double d = ff_to_double_finite(a);
  return (__float_as_uint(a.hi) & 0x7f800000u) == 0x7f800000u ? __longlong_as_double(0x7ff8000000000000ll) : d;
}

// binary64 -> float-float, the cheap way: hi = d with its significand
// truncated to 24 bits (integer instructions on the bit pattern), lo = the
// remaining 29 bits as an integer, converted (one rounding to 24 bits) and
// scaled by 2^(E-52).  hi + lo is within 2^-48 |d| of d, |lo| < ulp(hi).
// For |d| < 2^127 only; |d| < 2^-74 gives +-0 (absolute error < 2^-74).
__device__ __forceinline__ ff ff_from_double_fast(double d) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const unsigned sg = h & 0x80000000u;
  const unsigned mag = h & 0x7fffffffu;
  const bool tiny = mag < (949u << 20);
  const unsigned hb = tiny ? sg : (__funnelshift_l(l, mag - (896u << 20), 3) | sg);
  const float scale = __uint_as_float((((mag >> 20) - 948u) << 23) | sg);  // sign(d) 2^(E-52)
  const float lo = tiny ? 0.0f : __uint2float_rn(l & 0x1fffffffu) * scale;
  return {__uint_as_float(hb), lo};
}

// sin and cos of a (radians) as float-float, for |a| <= 800; error below
// ~2^-47.  Argument reduction: k = nearest integer to a 2/pi, r = a - k pi/2
// with pi/2 = P1 + P2 + P3 (P1 with 15 significant bits, so k P1 is exact for
// |k| < 512; the three parts carry pi/2 to 2^-88): a - k P1 in binary64 is
// exact (the operands are within a factor 2, or k = 0), and the rest runs in
// float-float on the small remainder; |r| <= pi/4 (plus rounding of k).  Then
// the Taylor series in z = r^2 -- sin r to r^15, cos r to r^18, truncation
// below 2^-53 at |r| = pi/4 -- by Horner's rule in float-float, and the
// quadrant of k.  Two FP64-pipe instructions (the subtraction and the
// float -> binary64 conversion of k P1), the rest on the FP32 pipe.
__device__ __forceinline__ ff ff_horner(ff p, ff z, float chi, float clo) { return ff_add(ff_mul_u(p, z), ff{chi, clo}); }
__device__ __forceinline__ void ff_sincos(double a, ff& s, ff& c) {
  const float kf = rintf(ff_from_double_fast(a).hi * 0x1.45f306p-1f);  // a 2/pi, rounded to an integer
  ff r = ff_from_double(a - (double)(kf * 0x1.921cp+0f));
  r = ff_add(r, ff_neg(two_prod(kf, 0x1.daa222p-15f)));
  r = ff_add(r, ff{-kf * -0x1.2e7b96p-40f, 0.0f});
  const ff z = ff_mul(r, r);
  // sin r = r + r z (-1/3! + z/5! - z^2/7! + ... - z^6/15!)
  ff ps = {-0x1.ae7f3ep-41f, -0x1.ccee08p-67f};              // -1/15!
  ps = ff_horner(ps, z, 0x1.6124620p-33f, -0x1.8af25ep-58f);  // +1/13!
  ps = ff_horner(ps, z, -0x1.ae64560p-26f, -0x1.fd5138p-52f); // -1/11!
  ps = ff_horner(ps, z, 0x1.71de3ap-19f, 0x1.55b1ccp-45f);    // +1/9!
  ps = ff_horner(ps, z, -0x1.a01a02p-13f, 0x1.7f97fap-39f);   // -1/7!
  ps = ff_horner(ps, z, 0x1.111112p-7f, -0x1.dddddep-32f);    // +1/5!
  ps = ff_horner(ps, z, -0x1.555556p-3f, 0x1.555556p-28f);    // -1/3!
  const ff sr = ff_add(r, ff_mul_u(ff_mul_u(r, z), ps));
  // cos r = 1 + z (-1/2! + z/4! - ... - z^8/18!)
  ff pc = {-0x1.682786p-53f, -0x1.dcbeccp-80f};              // -1/18!
  pc = ff_horner(pc, z, 0x1.ae7f3ep-45f, 0x1.ccee08p-71f);    // +1/16!
  pc = ff_horner(pc, z, -0x1.93974ap-37f, -0x1.180f94p-62f);  // -1/14!
  pc = ff_horner(pc, z, 0x1.1eed8ep-29f, 0x1.ff1b12p-54f);    // +1/12!
  pc = ff_horner(pc, z, -0x1.27e4fcp-22f, 0x1.10ec14p-47f);   // -1/10!
  pc = ff_horner(pc, z, 0x1.a01a02p-16f, -0x1.7f97fap-42f);   // +1/8!
  pc = ff_horner(pc, z, -0x1.6c16c2p-10f, 0x1.27d27ep-35f);   // -1/6!
  pc = ff_horner(pc, z, 0x1.555556p-5f, -0x1.555556p-30f);    // +1/4!
  pc = ff_horner(pc, z, -0.5f, 0.0f);                          // -1/2!
  const ff cr = ff_add(ff{1.0f, 0.0f}, ff_mul_u(z, pc));
  // quadrant k mod 4: (sin, cos) = (s, c), (c, -s), (-s, -c), (-c, s)
  const int q = (int)kf & 3;
  const ff s1 = (q & 1) ? cr : sr, c1 = (q & 1) ? sr : cr;
  s = (q & 2) ? ff_neg(s1) : s1;
  c = ((q + 1) & 2) ? ff_neg(c1) : c1;
}

// Unit vector of the angles (theta, phi), Eq. 3-4 read backwards.  cos theta
// drives the z-recurrences, whose coefficients amplify its error by up to
// ~l^2, so theta takes the binary64 sincos; sin theta, cos phi and sin phi
// enter only through the products x, y and the float-float powers of x + iy,
// where 48 bits suffice, so phi takes the float-float sine/cosine (FP32 pipe)
// when |phi| <= 800 and the binary64 one otherwise (also for non-finite phi,
// which then gives NaN components).  STRICT: binary64 sincos for phi too, and
// x, y as binary64 products (for the all-binary64 rows).
template <bool STRICT = false>
__device__ __forceinline__ void angles_to_unit(double theta, double phi, double& xb, double& yb, double& zb) {
  double st, ct;
  sincos(theta, &st, &ct);
  if (!STRICT && fabs(phi) <= 800.0) {
    ff sp, cp;
    ff_sincos(phi, sp, cp);
    const ff s = ff_from_double(st);
    xb = ff_to_double_finite(ff_mul(s, cp));
    yb = ff_to_double_finite(ff_mul(s, sp));
  } else {
    double sp, cp;
    sincos(phi, &sp, &cp);
    xb = st * cp;
    yb = st * sp;
  }
  zb = ct;
}

// True if any component is infinite or NaN.  Every evaluator gives such a
// point a row of NaN except the constant l = 0 value.
__device__ __forceinline__ bool nonfinite3(double x, double y, double z) {
  const int ex = 0x7ff00000;
  return ((__double2hiint(x) & ex) == ex) | ((__double2hiint(y) & ex) == ex) | ((__double2hiint(z) & ex) == ex);
}
__device__ __forceinline__ bool nonfinite3(float x, float y, float z) {
  const unsigned ex = 0x7f800000u;
  return ((__float_as_uint(x) & ex) == ex) | ((__float_as_uint(y) & ex) == ex) | ((__float_as_uint(z) & ex) == ex);
}

// FP64-output row with most of the arithmetic on the FP32 pipe.  1/r and the
// m = 0 and m = 1 columns -- whose recurrences amplify rounding most near the
// poles -- run in binary64 exactly as sh_row<LMAX>(double...) does (so those
// 28 values are bit-identical to the FP64 path); every m >= 2 column (72 of
// 100 values at lmax 9) runs in float-float: (x+iy)^m, the scaled
// z-recurrence, the scale and the two products, then one exact conversion to
// binary64 per value.  Normwise error against the FP64 oracle stays below
// 5e-14 at l = 9 (the FP64 path: 1.4e-14; tolerance 1e-13) while the FP64
// instructions per point drop from ~242 to ~75.  The direction must be
// finite: for a non-finite one the float-float columns are meaningless
// (callers test nonfinite3 and write a NaN row instead).
// SCALED: every value of shell l comes out multiplied by a per-l factor,
// given as binary64 (fd[l], for the binary64 columns) and as float-float
// (fff[l], folded into the float-float products before their conversion, so
// the m >= 2 values need no extra binary64 multiply).  Unscaled rows are
// bitwise unchanged.
template <int LMAX, bool CX = false, bool SCALED = false, typename Store>
__device__ __forceinline__ void sh_row_hybrid(double xb, double yb, double zb, Store&& store,
                                              const double* fd = nullptr, const ff* fff = nullptr) {
  auto sc = [&](int l, double v) {  // the binary64 columns' values
    if constexpr (SCALED)
      return v * fd[l];
    else
      return v;
  };
  store(0, sc(0, Sd<CX>(0, 0)));
  if constexpr (LMAX >= 1) {
    store(2, sc(1, Sd<CX>(1, 0) * zb));
    double q2 = 1.0, q1 = zb;
#pragma unroll
    for (int l = 2; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -SHM_G[l][0] * q2);
      store(l * l + l, sc(l, Sd<CX>(l, 0) * q));
      q2 = q1;
      q1 = q;
    }
    const double s1 = sc(1, Sd<CX>(1, 1));
    store(3, s1 * xb);
    store(1, s1 * yb);
    if constexpr (LMAX >= 2) {
      const double s = sc(2, Sd<CX>(2, 1) * zb);
      store(7, s * xb);
      store(5, s * yb);
    }
    q2 = 1.0;
    q1 = zb;
#pragma unroll
    for (int l = 3; l <= LMAX; ++l) {
      const double q = fma(zb, q1, -SHM_G[l][1] * q2);
      const double s = sc(l, Sd<CX>(l, 1) * q);
      store(l * l + l + 1, s * xb);
      store(l * l + l - 1, s * yb);
      q2 = q1;
      q1 = q;
    }
  }
  if constexpr (LMAX >= 2) {
    const ff X = ff_from_double(xb), Y = ff_from_double(yb), Z = ff_from_double(zb);
    ff A = X, B = Y;
#pragma unroll
    for (int m = 2; m <= LMAX; ++m) {
      const ff An = ff_add(ff_mul_u(A, X), ff_neg(ff_mul_u(B, Y)));
      const ff Bn = ff_add(ff_mul_u(A, Y), ff_mul_u(B, X));
      A = An;
      B = Bn;
      if constexpr (SCALED) {
        const ff sf = ff_mul_c_u(fff[m], Shi<CX>(m, m), Slo<CX>(m, m));
        store(m * m + 2 * m, ff_to_double_finite(ff_mul(sf, A)));
        store(m * m, ff_to_double_finite(ff_mul(sf, B)));
      } else {
        store(m * m + 2 * m, ff_to_double_finite(ff_mul_c(A, Shi<CX>(m, m), Slo<CX>(m, m))));
        store(m * m, ff_to_double_finite(ff_mul_c(B, Shi<CX>(m, m), Slo<CX>(m, m))));
      }
      ff q2 = {1.0f, 0.0f}, q1 = Z;
      if (m + 1 <= LMAX) {
        ff s = ff_mul_c_u(Z, Shi<CX>(m + 1, m), Slo<CX>(m + 1, m));
        if constexpr (SCALED) s = ff_mul_u(s, fff[m + 1]);
        const int k0 = (m + 1) * (m + 1) + (m + 1);
        store(k0 + m, ff_to_double_finite(ff_mul(s, A)));
        store(k0 - m, ff_to_double_finite(ff_mul(s, B)));
      }
#pragma unroll
      for (int l = m + 2; l <= LMAX; ++l) {
        const ff q = ff_add(ff_mul_u(Z, q1), ff_neg(ff_mul_c_u(q2, SHM_G_HI[l][m], SHM_G_LO[l][m])));
        ff s = ff_mul_c_u(q, Shi<CX>(l, m), Slo<CX>(l, m));
        if constexpr (SCALED) s = ff_mul_u(s, fff[l]);
        store(l * l + l + m, ff_to_double_finite(ff_mul(s, A)));
        store(l * l + l - m, ff_to_double_finite(ff_mul(s, B)));
        q2 = q1;
        q1 = q;
      }
    }
  }
}

// sh_row_hybrid in l-major order (see sh_row_lmajor for the phase protocol):
// the same operations on the same operands as sh_row_hybrid, so the rows are
// bitwise identical to it; all m-recurrences advance together, one l at a
// time, which exposes ~l independent chains to the scheduler.
// NEG_FF: the m < 0 values are handed to store as normalised float-float
// (type ff) instead of binary64 -- the m <= -2 ones before their conversion,
// the m = -1 ones converted exactly to 48 bits -- for callers that keep
// working on them with FP32 instructions.
// Ends: the phase plan (ends_phase(l): shell l closes a phase), by default
// groups of whole shells of at most PHMAX values.
// EMU (a mask of kEmuScale, kEmuOut): the binary64 products of the m = 0, 1
// columns -- their scales S q (kEmuScale) and the m = 1 outputs s x, s y
// (kEmuOut) -- on the integer pipes by dmul_int, the same bits; returns 1
// when dmul_int declined one of them (the caller then writes the row again
// with sh_row_hybrid), 0 otherwise and always for EMU = 0.
template <int LMAX, bool CX = false, int PHMAX = 37, bool NEG_FF = false, typename Ends = LPhases<LMAX, PHMAX>,
          int EMU = 0, typename Store, typename Phase>
__device__ __forceinline__ unsigned sh_row_hybrid_lmajor(double xb, double yb, double zb, Store&& store,
                                                         Phase&& phase) {
  unsigned bad = 0u;
  auto mul = [&](bool emu, double a, double b) { return emu ? dmul_int(a, b, bad) : a * b; };
  constexpr bool ESC = (EMU & kEmuScale) != 0, EOUT = (EMU & kEmuOut) != 0;
  auto store_neg_d = [&](int k, int kbase, double v) {
    if constexpr (NEG_FF)
      store(k, kbase, ff_from_double(v));
    else
      store(k, kbase, v);
  };
  auto store_neg_ff = [&](int k, int kbase, ff v) {
    if constexpr (NEG_FF)
      store(k, kbase, v);
    else
      store(k, kbase, ff_to_double_finite(v));
  };
  const ff X = ff_from_double(xb), Y = ff_from_double(yb), Z = ff_from_double(zb);
  ff A[LMAX + 1], B[LMAX + 1], q1[LMAX + 1], q2[LMAX + 1];
  double d1[2], d2[2];
  if constexpr (LMAX >= 2) {
    A[1] = X;
    B[1] = Y;
#pragma unroll
    for (int m = 2; m <= LMAX; ++m) {
      A[m] = ff_add(ff_mul_u(A[m - 1], X), ff_neg(ff_mul_u(B[m - 1], Y)));
      B[m] = ff_add(ff_mul_u(A[m - 1], Y), ff_mul_u(B[m - 1], X));
    }
  }
  int k0 = 0;
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    const int kc = l * l + l;
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      if (m <= 1) {  // binary64 columns, as sh_row_hybrid
        double s;
        if (l == m) {
          s = Sd<CX>(l, m);
          d2[m] = 1.0;
          d1[m] = 1.0;
        } else if (l == m + 1) {
          s = mul(ESC, Sd<CX>(l, m), zb);
          d2[m] = 1.0;
          d1[m] = zb;
        } else {
          const double q = fma(zb, d1[m], -SHM_G[l][m] * d2[m]);
          s = mul(ESC, Sd<CX>(l, m), q);
          d2[m] = d1[m];
          d1[m] = q;
        }
        if (m == 0) {
          store(kc, k0, s);
        } else {
          store(kc + 1, k0, mul(EOUT, (l == 1) ? Sd<CX>(1, 1) : s, xb));
          store_neg_d(kc - 1, k0, mul(EOUT, (l == 1) ? Sd<CX>(1, 1) : s, yb));
        }
      } else {  // float-float columns
        if (l == m) {
          store(kc + m, k0, ff_to_double_finite(ff_mul_c(A[m], Shi<CX>(m, m), Slo<CX>(m, m))));
          store_neg_ff(kc - m, k0, ff_mul_c(B[m], Shi<CX>(m, m), Slo<CX>(m, m)));
          q2[m] = {1.0f, 0.0f};
          q1[m] = Z;
        } else {
          ff sv;
          if (l == m + 1) {
            sv = ff_mul_c_u(Z, Shi<CX>(l, m), Slo<CX>(l, m));
          } else {
            const ff q = ff_add(ff_mul_u(Z, q1[m]), ff_neg(ff_mul_c_u(q2[m], SHM_G_HI[l][m], SHM_G_LO[l][m])));
            sv = ff_mul_c_u(q, Shi<CX>(l, m), Slo<CX>(l, m));
            q2[m] = q1[m];
            q1[m] = q;
          }
          store(kc + m, k0, ff_to_double_finite(ff_mul(sv, A[m])));
          store_neg_ff(kc - m, k0, ff_mul(sv, B[m]));
        }
      }
    }
    if (Ends::ends_phase(l)) {
      phase(k0, (l + 1) * (l + 1) - k0);
      k0 = (l + 1) * (l + 1);
    }
  }
  return bad;
}

// Short FP64 row (LMAX <= 4) entirely in float-float, every value of shell
// l multiplied by fff[l]: the columns m = 0, 1 too, which sh_row_hybrid keeps
// in binary64 because their long recurrences amplify float-float rounding
// near the poles.  Up to l = 4 the recurrences have at most three steps, so
// the float-float rounding (2^-48) stays near 1e-14 of the shell norm while
// the binary64 multiplies per value (scale, factor, x or y) leave the FP64
// pipe.  The direction must be finite.
template <int LMAX, typename Store>
__device__ __forceinline__ void sh_row_ff_scaled(double xb, double yb, double zb, Store&& store, const ff* fff) {
  static_assert(LMAX <= 4, "short rows only");
  const ff X = ff_from_double(xb), Y = ff_from_double(yb), Z = ff_from_double(zb);
  ff A = {1.0f, 0.0f}, B = {0.0f, 0.0f};
#pragma unroll
  for (int m = 0; m <= LMAX; ++m) {
    if (m == 1) {
      A = X;
      B = Y;
    } else if (m >= 2) {
      const ff An = ff_add(ff_mul_u(A, X), ff_neg(ff_mul_u(B, Y)));
      const ff Bn = ff_add(ff_mul_u(A, Y), ff_mul_u(B, X));
      A = An;
      B = Bn;
    }
    ff q2 = {1.0f, 0.0f}, q1 = Z;
#pragma unroll
    for (int l = m; l <= LMAX; ++l) {
      ff s;
      if (l == m) {
        s = ff_mul_c_u(fff[l], Shi<false>(l, m), Slo<false>(l, m));
      } else if (l == m + 1) {
        s = ff_mul_u(ff_mul_c_u(Z, Shi<false>(l, m), Slo<false>(l, m)), fff[l]);
      } else {
        const ff q = ff_add(ff_mul_u(Z, q1), ff_neg(ff_mul_c_u(q2, SHM_G_HI[l][m], SHM_G_LO[l][m])));
        s = ff_mul_u(ff_mul_c_u(q, Shi<false>(l, m), Slo<false>(l, m)), fff[l]);
        q2 = q1;
        q1 = q;
      }
      if (m == 0) {
        const ff sn = fast_two_sum(s.hi, s.lo);
        store(l * l + l, ff_to_double_finite(sn));
      } else {
        store(l * l + l + m, ff_to_double_finite(ff_mul(s, A)));
        store(l * l + l - m, ff_to_double_finite(ff_mul(s, B)));
      }
    }
  }
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
template <int LMAX, int M, bool CX, typename Store>
__device__ __forceinline__ void sh_column_ff(float zb, float dq, float A, float B, Store&& store) {
  ff q2 = {1.0f, 0.0f}, q1 = {zb, 0.0f};
  auto emit = [&](int l, ff Q) {
    const ff p = two_prod(Shi<CX>(l, M), Q.hi);
    const float v = __fadd_rn(p.hi, fmaf(Shi<CX>(l, M), Q.lo, fmaf(Slo<CX>(l, M), Q.hi, p.lo)));
    if constexpr (M == 0) {
      store(l * l + l, v);
    } else {
      store(l * l + l + M, v * A);
      store(l * l + l - M, v * B);
    }
  };
  if constexpr (M == 0) {
    store(0, Shi<CX>(0, 0));
  } else {
    store(M * M + 2 * M, Shi<CX>(M, M) * A);
    store(M * M, Shi<CX>(M, M) * B);
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

// The m = 0, 1 columns with the plain FP32 recurrence (for short rows: at
// l <= 4 their rounding stays far inside the FP32 tolerances).
template <int LMAX, int M, bool CX, typename Store>
__device__ __forceinline__ void sh_column_f32(float zb, float qq, float A, float B, Store&& store) {
  if constexpr (M == 0) {
    store(0, Shi<CX>(0, 0));
  } else {
    store(M * M + 2 * M, (float)Sd<CX>(M, M) * A);
    store(M * M, (float)Sd<CX>(M, M) * B);
  }
  auto emit = [&](int l, float q) {
    const float v = (float)Sd<CX>(l, M) * q;
    if constexpr (M == 0) {
      store(l * l + l, v);
    } else {
      store(l * l + l + M, v * A);
      store(l * l + l - M, v * B);
    }
  };
  if constexpr (M + 1 <= LMAX) emit(M + 1, zb);
  float q2 = 1.0f, q1 = zb;
#pragma unroll
  for (int l = M + 2; l <= LMAX; ++l) {
    const float q = fmaf(zb, q1, -(float)SHM_G[l][M] * (qq * q2));
    emit(l, q);
    q2 = q1;
    q1 = q;
  }
}

// FF01 = false: the m = 0, 1 columns use the plain FP32 recurrence
// (sh_column_f32), for short rows only.
template <int LMAX, bool CX = false, bool FF01 = true, typename Store>
__device__ __forceinline__ void sh_row(float xb, float yb, float zb, Store&& store) {
  float qq;
  if constexpr (FF01) {
    // q = xb^2 + yb^2 + zb^2 as a float-float, then dq = q - 1
    const ff px = two_prod(xb, xb), py = two_prod(yb, yb), pz = two_prod(zb, zb);
    const ff s1 = two_sum(px.hi, py.hi);
    const ff s2 = two_sum(s1.hi, pz.hi);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(s1.lo, s2.lo), px.lo), __fadd_rn(py.lo, pz.lo));
    const ff qf = fast_two_sum(s2.hi, lo);
    const float dq = __fadd_rn(__fsub_rn(qf.hi, 1.0f), qf.lo);
    qq = qf.hi;
    sh_column_ff<LMAX, 0, CX>(zb, dq, 0.0f, 0.0f, store);
    if constexpr (LMAX >= 1) sh_column_ff<LMAX, 1, CX>(zb, dq, xb, yb, store);
  } else {
    // the plain recurrences need q only to FP32 accuracy: two FMAs and a product
    qq = fmaf(xb, xb, fmaf(yb, yb, zb * zb));
    sh_column_f32<LMAX, 0, CX>(zb, qq, 0.0f, 0.0f, store);
    if constexpr (LMAX >= 1) sh_column_f32<LMAX, 1, CX>(zb, qq, xb, yb, store);
  }
  float A = xb, B = yb;
#pragma unroll
  for (int m = 2; m <= LMAX; ++m) {
    const float An = fmaf(A, xb, -B * yb);
    const float Bn = fmaf(A, yb, B * xb);
    A = An;
    B = Bn;
    store(m * m + 2 * m, (float)Sd<CX>(m, m) * A);
    store(m * m, (float)Sd<CX>(m, m) * B);
    if (m + 1 <= LMAX) {
      const float s = (float)Sd<CX>(m + 1, m) * zb;
      const int k0 = (m + 1) * (m + 1) + (m + 1);
      store(k0 + m, s * A);
      store(k0 - m, s * B);
    }
    float q2 = 1.0f, q1 = zb;
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l) {
      const float q = fmaf(zb, q1, -(float)SHM_G[l][m] * (qq * q2));
      const float s = (float)Sd<CX>(l, m) * q;
      store(l * l + l + m, s * A);
      store(l * l + l - m, s * B);
      q2 = q1;
      q1 = q;
    }
  }
}

// Full point: Cartesian (or already normalised) input -> row of harmonics.
// HYBRID selects sh_row_hybrid for binary64 rows.  EMU (all-binary64 rows):
// sh_row_emu<LMAX, EMU, CX>, the same bits, with sh_row for a point where
// dmul_int declines a product.
template <int LMAX, bool HYBRID = false, bool CX = false, int EMU = 0, typename T, typename Store>
__device__ __forceinline__ void sh_point(T x, T y, T z, bool normalized, Store&& store) {
  if (is_origin(x, y, z)) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
    store(0, (T)kInvSqrt4Pi);
#pragma unroll
    for (int k = 1; k < NH<LMAX>::value; ++k) store(k, (T)0);
    return;
  }
  T xb = x, yb = y, zb = z;
  if (!normalized) unit_dir(x, y, z, xb, yb, zb);
  if (nonfinite3(xb, yb, zb)) {  // NaN in every value but the constant l = 0
    store(0, (T)kInvSqrt4Pi);
#pragma unroll
    for (int k = 1; k < NH<LMAX>::value; ++k) store(k, (T)__longlong_as_double(0x7ff8000000000000ll));
    return;
  }
  if constexpr (HYBRID && sizeof(T) == 8) {
    sh_row_hybrid<LMAX, CX>(xb, yb, zb, store);
  } else if constexpr (EMU != 0 && sizeof(T) == 8) {
    if (sh_row_emu<LMAX, EMU, CX>(xb, yb, zb, store)) sh_row<LMAX, CX>(xb, yb, zb, store);
  } else {
    sh_row<LMAX, CX>(xb, yb, zb, store);
  }
}

}  // namespace shm
