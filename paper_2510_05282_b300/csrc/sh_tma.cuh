// The phased FP64 evaluator with TMA tensor stores.
//
// Rows are computed and staged phase by phase exactly as in sh_phased.cuh
// (same row code, same values), but a staged phase leaves the SM through the
// tensor memory accelerator: one thread issues cp.async.bulk.tensor stores of
// the phase's [TPB rows][w columns] block, which the TMA engine writes to
// global memory asynchronously while the SM goes on computing.  This removes
// the copy-out loop (shared loads, 16-byte global stores and their address
// arithmetic: ~200 instructions per point at l = 9) from the issue slots.
//
// Staging layout: a TMA box is dense in shared memory (row pitch = box
// width), and a box row must be a multiple of 16 bytes.  A phase of width w
// (even) is cut into two boxes of bw = w / 2 columns when bw is 2 mod 4 (18
// for w = 36, 14 for w = 28), else sent as one box: an even pitch leaves the
// 32 rows a warp writes at once at best 4-way bank-conflicted, which a pitch
// of 2 mod 4 doubles reaches (a multiple of 4 would give 8-way).
//
// A phase can go by TMA only if its width is even (an even number of
// l-shells) and the row pitch (lmax+1)^2 * 8 bytes is a multiple of 16:
// odd lmax <= 9 with 37-value phases.  Other lmax, outputs that are not
// 16-byte aligned, and n >= 2^31 take k_eval_phased.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sh_phased.cuh"
#include "shm_internal.h"

namespace shm {

template <int LMAX, int PHMAX = 37>
struct TmaPlan {
  static constexpr int L2 = NH<LMAX>::value;
  // width of the phase that starts at column k0 (branch-free so that it folds
  // to a constant in the unrolled row code)
  __host__ __device__ static constexpr int width_at(int k0) {
    int w = 0, start = 0, res = 0;
    for (int l = 0; l <= LMAX; ++l) {
      const int wl = 2 * l + 1;
      if (w > 0 && w + wl > PHMAX) {
        res = (start == k0) ? w : res;
        start += w;
        w = 0;
      }
      w += wl;
    }
    return (start == k0) ? w : res;
  }
  // box width of a phase of width w: w / 2 when that is 2 mod 4 and at
  // least 6 (36 -> 18, 28 -> 14), else w itself (a closed form, so that it
  // folds to a constant)
  __host__ __device__ static constexpr int box_width(int w) {
    return (w % 4 == 0 && (w / 2) % 4 == 2 && w / 2 >= 6) ? w / 2 : w;
  }
  // width_at in closed form for 37-value phases ([0, 36), [36, 64), [64,
  // 100) as far as LMAX reaches; one phase up to l = 5): the row code calls
  // the store callback once per value, and only a plain expression of k0
  // folds to a constant there (checked against width_at below)
  __host__ __device__ static constexpr int width_fast(int k0) {
    return PHMAX != 37 ? width_at(k0)
                       : (L2 <= 37 ? L2 : (k0 == 0 ? 36 : (k0 == 36 ? (L2 < 64 ? L2 - 36 : 28) : L2 - 64)));
  }
  static constexpr bool width_fast_ok() {
    int k0 = 0;
    while (k0 < L2) {
      if (width_fast(k0) != width_at(k0)) return false;
      k0 += width_at(k0);
    }
    return true;
  }
  __host__ __device__ static constexpr int box_at(int k0) { return box_width(width_fast(k0)); }
  // the distinct box widths, in order of first use (at most two are supported)
  static constexpr int box_a() { return box_at(0); }
  static constexpr int box_b() {
    int b = box_a(), k0 = 0;
    while (k0 < L2) {
      const int bw = box_at(k0);
      if (bw != box_a()) b = bw;
      k0 += width_at(k0);
    }
    return b;
  }
  static constexpr bool feasible() {
    if ((L2 * 8) % 16 != 0 || !width_fast_ok()) return false;
    int k0 = 0;
    while (k0 < L2) {
      const int w = width_at(k0), bw = box_at(k0);
      if (w % 2 != 0 || (bw * 8) % 16 != 0 || bw > 256 || (bw != box_a() && bw != box_b())) return false;
      k0 += w;
    }
    return true;
  }
  static constexpr int max_width() { return LPhases<LMAX, PHMAX>::max_width(); }
  static constexpr size_t smem_bytes(int tpb) { return (size_t)tpb * max_width() * 8 + 128; }
};

// Odd lmax <= 9 only (see the header comment); a run-time mirror for the
// host's variant choice.
inline bool tma_plan_feasible(int lmax) {
  switch (lmax) {
    case 1: return TmaPlan<1>::feasible();
    case 3: return TmaPlan<3>::feasible();
    case 5: return TmaPlan<5>::feasible();
    case 7: return TmaPlan<7>::feasible();
    case 9: return TmaPlan<9>::feasible();
  }
  return false;
}

// Rows of one tile with TMA stores: as phased_rows, for the tile's rows
// [p0, p0 + TPB) of the output described by map_a / map_b (boxes of
// TmaPlan::box_a() / box_b() columns by TPB rows; rows past n are clipped by
// the TMA unit).  `tile` is 128-byte aligned, TPB x max_width() doubles.
template <int LMAX, int TPB>
__device__ __forceinline__ void phased_rows_tma(double xb, double yb, double zb, bool origin, int64_t p0,
                                                double* __restrict__ tile, const CUtensorMap* map_a,
                                                const CUtensorMap* map_b) {
  using Plan = TmaPlan<LMAX>;
  const bool bad = nonfinite3(xb, yb, zb);  // NaN row but l = 0 (the hybrid row code needs a finite direction)
  const int t = (int)threadIdx.x;
  auto slot = [&](int k, int k0) -> double* {
    const int bw = Plan::box_at(k0);
    const int c = k - k0, b = c / bw;
    return tile + b * TPB * bw + t * bw + (c - b * bw);
  };
  auto store = [&](int k, int k0, double v) { *slot(k, k0) = v; };
  auto flush = [&](int k0, int w) {
    const int bw = Plan::box_at(k0);
    if (origin || bad) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
      const double fill = origin ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
      for (int b = 0; b < w / bw; ++b)
        for (int c = 0; c < bw; ++c) tile[b * TPB * bw + t * bw + c] = (k0 + b * bw + c == 0) ? kInvSqrt4Pi : fill;
    }
    // the staged values (generic proxy) must be visible to the TMA unit (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      const CUtensorMap* m = (bw == Plan::box_a()) ? map_a : map_b;
      for (int b = 0; b < w / bw; ++b) {
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(tile + b * TPB * bw);
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     :
                     : "l"(reinterpret_cast<uint64_t>(m)), "r"(k0 + b * bw), "r"((int)p0), "r"(sa)
                     : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      // the next phase overwrites the buffer: wait until the TMA unit has read it
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncthreads();
  };
  sh_row_hybrid_lmajor<LMAX>(xb, yb, zb, store, flush);
}

// Registers capped as k_eval_phased (five 128-thread CTAs per SM).
template <int LMAX, int TPB, int IN = kInPoints>
__global__ void __launch_bounds__(TPB, 640 / TPB) k_eval_phased_tma(const double* __restrict__ in, int64_t n,
                                                                    int64_t ntiles, int normalized,
                                                                    const __grid_constant__ CUtensorMap map_a,
                                                                    const __grid_constant__ CUtensorMap map_b) {
  static_assert(TmaPlan<LMAX>::feasible(), "no TMA phase plan for this lmax");
  extern __shared__ unsigned char smem_tma[];
  // TMA needs 128-byte aligned shared addresses: round the base up (the
  // launch adds 128 bytes)
  double* tile = reinterpret_cast<double*>(smem_tma + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_tma) & 127u)) & 127u));
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * TPB;
    const int rows = (int)min((int64_t)TPB, n - p0);
    const bool valid = (int)threadIdx.x < rows;
    bool origin = false;
    double xb = 0.0, yb = 0.0, zb = 1.0;
    if constexpr (IN == kInAngles) {
      if (valid) {  // Eq. 3-4 read backwards: the unit vector of (theta, phi)
        const int64_t p = p0 + threadIdx.x;
        double st, ct, sp, cp;
        sincos(in[2 * p], &st, &ct);
        sincos(in[2 * p + 1], &sp, &cp);
        xb = st * cp;
        yb = st * sp;
        zb = ct;
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
    phased_rows_tma<LMAX, TPB>(xb, yb, zb, origin, p0, tile, &map_a, &map_b);
  }
  // the last stores' global writes complete before the CTA retires
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Host side: encodes the two tensor maps of `out` and launches
// k_eval_phased_tma (grid = SMs x resident CTAs, CTAs loop over tiles).
// *launched = false with SHM_OK when TMA does not apply (no plan for LMAX,
// output not 16-byte aligned, n >= 2^31, or no driver entry point): the
// caller then runs k_eval_phased.
template <int LMAX, int TPB, int IN>
inline shm_status launch_phased_tma(const double* in, int64_t n, double* out, bool normalized, cudaStream_t stream,
                             bool* launched) {
  *launched = false;
  if constexpr (TmaPlan<LMAX>::feasible()) {
    using Plan = TmaPlan<LMAX>;
    CUtensorMap ma, mb;
    if (!encode_rows_map(&ma, out, n, Plan::L2, Plan::box_a(), TPB) ||
        !encode_rows_map(&mb, out, n, Plan::L2, Plan::box_b(), TPB))
      return SHM_OK;  // not launched: the caller takes the copy-out kernel
    constexpr int MAXDEV = 64;
    static int blocks_per_sm[MAXDEV] = {0};
    const int dev = current_device();
    if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
    auto kern = k_eval_phased_tma<LMAX, TPB, IN>;
    const size_t smem = Plan::smem_bytes(TPB);
    if (blocks_per_sm[dev] == 0) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_eval_phased_tma)");
      int b = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TPB, smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_eval_phased_tma)");
      blocks_per_sm[dev] = std::max(b, 1);
    }
    const int64_t ntiles = (n + TPB - 1) / TPB;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * blocks_per_sm[dev]);
    kern<<<(unsigned)grid, TPB, smem, stream>>>(in, n, ntiles, normalized ? 1 : 0, ma, mb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "k_eval_phased_tma launch");
    *launched = true;
  }
  return SHM_OK;
}
}  // namespace shm
