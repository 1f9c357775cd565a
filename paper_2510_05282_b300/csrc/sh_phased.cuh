// The phased FP64 evaluator kernel, shared by shm_eval (Cartesian points)
// and shm_eval_angles (theta, phi pairs).
//
// l-major evaluation (sh_row_lmajor / sh_row_hybrid_lmajor) staged one phase
// of l-shells at a time (<= 37 values per row), so a tile needs ~1/3 of the
// shared memory of a full-row tile and ~2.5x more warps fit on an SM; every
// l-step advances up to 10 independent m-recurrences, which feeds the FP64
// pipe with independent work.  Rows are written phase by phase (one
// contiguous segment of each row per phase, in 16-byte pairs when the output
// allows).  Results are bit-identical to the full-row variants.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sh_core.cuh"

namespace shm {

enum { kInPoints = 0, kInAngles = 1 };

// Rows of one tile: every thread of the CTA calls this with the unit vector
// of its point (xb, yb, zb; `origin` for r = 0); rows [0, rows) of the tile
// are written to dst[r * L2 + k].  `tile` is the CTA's staging buffer of
// TPB x (LPhases<LMAX>::max_width() | 1) doubles.  vec: dst is 16-byte
// aligned (the copy-out then writes 16-byte pairs where L2 allows).
template <int LMAX, int TPB, bool HYB>
__device__ __forceinline__ void phased_rows(double xb, double yb, double zb, bool origin, int rows,
                                            double* __restrict__ dst, bool vec, double* __restrict__ tile) {
  constexpr int L2 = NH<LMAX>::value;
  constexpr int RS = LPhases<LMAX>::max_width() | 1;
  double* row = tile + threadIdx.x * RS;
  const bool bad = nonfinite3(xb, yb, zb);  // NaN row but l = 0 (the hybrid row code needs a finite direction)
  auto store = [&](int k, int k0, double v) { row[k - k0] = v; };
  auto flush = [&](int k0, int w) {
    if (origin || bad) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
      const double fill = origin ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
      for (int c = 0; c < w; ++c) row[c] = (k0 + c == 0) ? kInvSqrt4Pi : fill;
    }
    __syncthreads();
    if (vec && L2 % 2 == 0 && ((k0 | w) & 1) == 0) {
      // pairs: the segment of every row starts on a 16-byte boundary.  Thread
      // (rs, cp) = divmod(threadIdx, hw) copies column pair cp of rows rs,
      // rs + RP, rs + 2 RP, ... (RP = TPB / hw rows per pass): one division
      // per phase and incremental addresses, instead of a division per pair
      // (1.85 -> 1.82 ms on the 192^3 grid).
      const int hw = w >> 1;
      const int RP = TPB / hw;
      const int rs = (int)threadIdx.x / hw;
      const int cp = (int)threadIdx.x - rs * hw;
      if (rs < RP) {
        const double* t = tile + rs * RS + 2 * cp;
        double2* o = reinterpret_cast<double2*>(dst + (int64_t)rs * L2 + k0 + 2 * cp);
#pragma unroll 2  // two loads in flight per store (1.94 -> 1.84 ms before this mapping; 4: slower)
        for (int r = rs; r < rows; r += RP) {
          __stcs(o, make_double2(t[0], t[1]));
          t += RP * RS;
          o += RP * L2 / 2;
        }
      }
    } else {
      const int nv = rows * w;
      for (int j = threadIdx.x; j < nv; j += TPB) {
        const int r = j / w;
        const int c = j - r * w;
        __stcs(dst + (int64_t)r * L2 + k0 + c, tile[r * RS + c]);
      }
    }
    __syncthreads();
  };
  if constexpr (HYB)
    sh_row_hybrid_lmajor<LMAX>(xb, yb, zb, store, flush);
  else
    sh_row_lmajor<LMAX>(xb, yb, zb, store, flush);
}

// Registers are capped so that five 128-thread CTAs fit an SM (96 per
// thread, a few bytes of spill): measured 2.01 against 2.13 ms uncapped
// (109 registers, four CTAs) on the 192^3 grid.
template <int LMAX, int TPB, bool HYB, int IN = kInPoints>
__global__ void __launch_bounds__(TPB, 640 / TPB) k_eval_phased(const double* __restrict__ in, int64_t n,
                                                                double* __restrict__ out, int64_t ntiles,
                                                                int normalized, int vec) {
  constexpr int L2 = NH<LMAX>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tile = reinterpret_cast<double*>(smem_raw);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * TPB;
    const int rows = (int)min((int64_t)TPB, n - p0);
    const bool valid = (int)threadIdx.x < rows;
    bool origin = false;
    double xb = 0.0, yb = 0.0, zb = 1.0;
    if constexpr (IN == kInAngles) {
      if (valid) {  // Eq. 3-4 read backwards: the unit vector of (theta, phi)
        const int64_t p = p0 + threadIdx.x;
        angles_to_unit<!HYB>(in[2 * p], in[2 * p + 1], xb, yb, zb);
      }
    } else {
      double x = 0.0, y = 0.0, z = 1.0;
      if (valid) {
        const int64_t p = p0 + threadIdx.x;
        x = in[3 * p];
        y = in[3 * p + 1];
        z = in[3 * p + 2];
      }
      origin = valid && is_origin(x, y, z);
      if (valid && !origin) {
        if (normalized) {
          xb = x;
          yb = y;
          zb = z;
        } else {
          unit_dir(x, y, z, xb, yb, zb);
        }
      }
    }
    phased_rows<LMAX, TPB, HYB>(xb, yb, zb, origin, rows, out + p0 * L2, vec != 0, tile);
  }
}

}  // namespace shm
