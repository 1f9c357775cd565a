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

#include <algorithm>
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
// EMU != 0 (phased-hybrid-tma-emu-128): the binary64 products of the m = 0, 1
// columns on the integer pipes (sh_row_hybrid_lmajor<..., EMU>, the same
// bits); a thread whose point made dmul_int decline one writes its row again
// with sh_row_hybrid, straight to `out`, after the tile's TMA writes have
// completed (a per-tile vote; no such row in most tiles).
template <int LMAX, int TPB, int EMU = 0>
__device__ __forceinline__ void phased_rows_tma(double xb, double yb, double zb, bool origin, int64_t p0,
                                                double* __restrict__ tile, const CUtensorMap* map_a,
                                                const CUtensorMap* map_b, double* __restrict__ out = nullptr,
                                                bool valid = true) {
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
  const unsigned declined =
      sh_row_hybrid_lmajor<LMAX, false, 37, false, LPhases<LMAX, 37>, EMU>(xb, yb, zb, store, flush);
  if constexpr (EMU != 0) {
    const bool redo = declined != 0u && valid && !origin && !bad;
    if (__syncthreads_or(redo)) {
      if (t == 0) {  // the tile's TMA writes are complete and visible before the overwrite
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
      }
      __syncthreads();
      if (redo) {
        double* row = out + (p0 + t) * Plan::L2;
        sh_row_hybrid<LMAX>(xb, yb, zb, [&](int k, double v) { row[k] = v; });
      }
    }
  }
}

// Registers capped as k_eval_phased (five 128-thread CTAs per SM).  With
// EMU the integer products spill at l = 9 (96 registers: 300 bytes of spill
// loads per thread; still 92 bytes at a 128-register cap), so the integer
// form pays at l = 5 only.
template <int LMAX, int TPB, int IN = kInPoints, int EMU = 0>
__global__ void __launch_bounds__(TPB, 640 / TPB) k_eval_phased_tma(const double* __restrict__ in, int64_t n,
                                                                    int64_t ntiles, int normalized,
                                                                    const __grid_constant__ CUtensorMap map_a,
                                                                    const __grid_constant__ CUtensorMap map_b,
                                                                    double* __restrict__ out) {
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
        angles_to_unit(in[2 * p], in[2 * p + 1], xb, yb, zb);
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
    phased_rows_tma<LMAX, TPB, EMU>(xb, yb, zb, origin, p0, tile, &map_a, &map_b, out, valid);
  }
  // the last stores' global writes complete before the CTA retires
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Double-buffered form (phased-hybrid-tma2-128).  In the kernel above every
// phase waits for the TMA unit to read its 37 KB buffer before the next phase
// may overwrite it; two such buffers per CTA do not fit five CTAs per SM.
// Here phases are at most 20 values wide and alternate between two 20-column
// buffers (41 KB per CTA), so a phase waits only for the read of the phase
// before it, issued a whole phase earlier.  Phases (odd lmax 3..9): shells
// 0-3 -> columns [0, 16), shells 4-5 -> [16, 36), then one shell each.  A box
// must start on an even column, so the last value of shell 6 (k = 48) and of
// shell 8 (k = 80) is kept in a register and sent with the next shell's box:
// boxes [36, 48), [48, 64), [64, 80), [80, 100).  Every box is 16 or 20
// columns (two boxes of 10 + 6 or 10 + 10 columns: pitches 2 mod 4) or 12
// (6 + 6).
template <int LMAX>
struct Tma2Plan {
  static constexpr int L2 = NH<LMAX>::value;
  static constexpr bool feasible() { return LMAX == 3 || LMAX == 5 || LMAX == 7 || LMAX == 9; }
  __host__ __device__ static constexpr bool ends_phase(int l) { return l == LMAX || l == 3 || l >= 5; }
  // per row-code phase (identified by its first column k0)
  __host__ __device__ static constexpr int index(int k0) {
    return k0 == 0 ? 0 : (k0 == 16 ? 1 : (k0 == 36 ? 2 : (k0 == 49 ? 3 : (k0 == 64 ? 4 : 5))));
  }
  __host__ __device__ static constexpr int next(int k0) {
    return k0 == 0 ? 16 : (k0 == 16 ? 36 : (k0 == 36 ? 49 : (k0 == 49 ? 64 : (k0 == 64 ? 81 : 100))));
  }
  __host__ __device__ static constexpr bool carried(int k) { return (k == 48 && LMAX >= 7) || (k == 80 && LMAX >= 9); }
  __host__ __device__ static constexpr int box_x(int k0) { return (k0 == 49 || k0 == 81) ? k0 - 1 : k0; }
  __host__ __device__ static constexpr int box_end(int k0) {
    return (next(k0) == 49 || next(k0) == 81) ? next(k0) - 1 : next(k0);
  }
  __host__ __device__ static constexpr int box_w(int k0) { return box_end(k0) - box_x(k0); }
  __host__ __device__ static constexpr int bw0(int k0) { return box_w(k0) == 12 ? 6 : 10; }
  static constexpr int kBufCols = 20;
  static constexpr size_t smem_bytes(int tpb) { return (size_t)2 * tpb * kBufCols * 8 + 128; }
};

// Rows of one tile, double-buffered TMA stores.  Rows of points at the
// origin or with a non-finite coordinate are sent as computed and then
// overwritten from registers, after the tile's stores have completed, by the
// threads that own them (a per-tile vote; no such row in most tiles).  A fill
// in every phase end, as the single-buffered kernel does, pushes the unrolled
// row past the compiler's unroll limit at lmax 9 (the l loop then stays a
// loop: 3x the instructions).
template <int LMAX, int TPB>
__device__ __forceinline__ void phased_rows_tma2(double xb, double yb, double zb, bool origin, int64_t p0, int rows,
                                                 double* __restrict__ tile, double* __restrict__ out,
                                                 const CUtensorMap* map10, const CUtensorMap* map6) {
  using P = Tma2Plan<LMAX>;
  const bool bad = nonfinite3(xb, yb, zb);  // NaN row but l = 0 (the hybrid row code needs a finite direction)
  const int t = (int)threadIdx.x;
  double carry = 0.0;
  // staging slot of column c of the box of the phase starting at k0
  auto at = [&](int k0, int c) -> double* {
    const int b0 = P::bw0(k0), bw = P::box_w(k0);
    double* buf = tile + (P::index(k0) & 1) * TPB * P::kBufCols;
    return c < b0 ? buf + t * b0 + c : buf + TPB * b0 + t * (bw - b0) + (c - b0);
  };
  auto store = [&](int k, int k0, double v) {
    if (P::carried(k))
      carry = v;
    else
      *at(k0, k - P::box_x(k0)) = v;
  };
  auto flush = [&](int k0, int w) {
    (void)w;
    const int x = P::box_x(k0), bw = P::box_w(k0), b0 = P::bw0(k0);
    if (x != k0) *at(k0, 0) = carry;  // the value carried from the previous shell
    // the staged values (generic proxy) must be visible to the TMA unit (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      double* buf = tile + (P::index(k0) & 1) * TPB * P::kBufCols;
      for (int j = 0; j < 2; ++j) {
        const int xj = x + (j ? b0 : 0), wj = j ? bw - b0 : b0;
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(buf + (j ? TPB * b0 : 0));
        const CUtensorMap* m = wj == 10 ? map10 : map6;
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     :
                     : "l"(reinterpret_cast<uint64_t>(m)), "r"(xj), "r"((int)p0), "r"(sa)
                     : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      // the next phase writes the other buffer: wait until the TMA unit has
      // read it (its stores were issued one phase ago)
      asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    }
    __syncthreads();
  };
  sh_row_hybrid_lmajor<LMAX, false, 37, false, P>(xb, yb, zb, store, flush);
  if (__syncthreads_or((origin || bad) && (int)threadIdx.x < rows)) {
    if (t == 0) {  // the tile's TMA writes are complete and visible before the overwrite
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    if ((origin || bad) && t < rows) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
      const double fill = origin ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
      double* row = out + (p0 + t) * P::L2;
      for (int k = 0; k < P::L2; ++k) row[k] = k == 0 ? kInvSqrt4Pi : fill;
    }
  }
}

template <int LMAX, int TPB, int IN = kInPoints>
__global__ void __launch_bounds__(TPB, 640 / TPB) k_eval_phased_tma2(const double* __restrict__ in, int64_t n,
                                                                     int64_t ntiles, int normalized,
                                                                     double* __restrict__ out,
                                                                     const __grid_constant__ CUtensorMap map10,
                                                                     const __grid_constant__ CUtensorMap map6) {
  static_assert(Tma2Plan<LMAX>::feasible(), "no double-buffered TMA plan for this lmax");
  extern __shared__ unsigned char smem_tma[];
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
        angles_to_unit(in[2 * p], in[2 * p + 1], xb, yb, zb);
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
    phased_rows_tma2<LMAX, TPB>(xb, yb, zb, origin, p0, rows, tile, out, &map10, &map6);
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Host side of the double-buffered form; as launch_phased_tma.
template <int LMAX, int TPB, int IN>
inline shm_status launch_phased_tma2(const double* in, int64_t n, double* out, bool normalized, cudaStream_t stream,
                                     bool* launched) {
  *launched = false;
  if constexpr (Tma2Plan<LMAX>::feasible()) {
    using Plan = Tma2Plan<LMAX>;
    CUtensorMap m10, m6;
    if (!encode_rows_map(&m10, out, n, Plan::L2, 10, TPB) || !encode_rows_map(&m6, out, n, Plan::L2, 6, TPB))
      return SHM_OK;
    constexpr int MAXDEV = 64;
    static int blocks_per_sm[MAXDEV] = {0};
    const int dev = current_device();
    if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
    auto kern = k_eval_phased_tma2<LMAX, TPB, IN>;
    const size_t smem = Plan::smem_bytes(TPB);
    if (blocks_per_sm[dev] == 0) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_eval_phased_tma2)");
      int b = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TPB, smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_eval_phased_tma2)");
      blocks_per_sm[dev] = std::max(b, 1);
    }
    const int64_t ntiles = (n + TPB - 1) / TPB;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * blocks_per_sm[dev]);
    kern<<<(unsigned)grid, TPB, smem, stream>>>(in, n, ntiles, normalized ? 1 : 0, out, m10, m6);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "k_eval_phased_tma2 launch");
    *launched = true;
  }
  return SHM_OK;
}

// Host side: encodes the two tensor maps of `out` and launches
// k_eval_phased_tma (grid = SMs x resident CTAs, CTAs loop over tiles).
// *launched = false with SHM_OK when TMA does not apply (no plan for LMAX,
// output not 16-byte aligned, n >= 2^31, or no driver entry point): the
// caller then runs k_eval_phased.
template <int LMAX, int TPB, int IN, int EMU = 0>
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
    auto kern = k_eval_phased_tma<LMAX, TPB, IN, EMU>;
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
    kern<<<(unsigned)grid, TPB, smem, stream>>>(in, n, ntiles, normalized ? 1 : 0, ma, mb, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "k_eval_phased_tma launch");
    *launched = true;
  }
  return SHM_OK;
}

// ---------------------------------------------------------------------------
// All-binary64 rows with TMA stores (rows-tma-TPB, the SHM_STRICT_FP64 path).
// sh_row<LMAX>(double...) produces a row in m-major order with few live
// registers (~40), so a whole row is staged: the tile [TPB rows][L2 columns]
// is held as column boxes of kBW = 10 columns (the last one narrower when L2
// is not a multiple of 10), each box dense [TPB][width] in shared memory.  A
// pitch of 10 doubles is 2 mod 4, so the 32 rows a warp writes at once are
// 4-way bank-conflicted, the least an even pitch allows.  Once the tile is
// complete one thread sends the boxes by cp.async.bulk.tensor; the next tile
// waits for the TMA unit to have read the buffer only after its points' unit
// vectors are formed, so the wait overlaps FP64 work.  These rows are bound
// by the FP64 pipe (~242 FP64 instructions per point at l = 9, against 824
// bytes of HBM traffic); the TMA store takes the copy-out loop and its
// second barrier off the SM, so the FP64 pipe idles only at the barrier.
// Odd lmax (the row pitch (lmax+1)^2 * 8 bytes must be a multiple of 16).
template <int LMAX>
struct RowsTmaPlan {
  static constexpr int L2 = NH<LMAX>::value;
  static constexpr int kBW = 10;
  static constexpr int nfull = L2 / kBW;
  static constexpr int rem = L2 - nfull * kBW;
  static constexpr int nbox = nfull + (rem ? 1 : 0);
  static constexpr bool feasible() { return L2 % 2 == 0; }
  // box widths of the two tensor maps (the second unused when rem == 0)
  static constexpr int width_a() { return nfull > 0 ? kBW : rem; }
  static constexpr int width_b() { return rem > 0 ? rem : kBW; }
  static constexpr size_t smem_bytes(int tpb) { return (size_t)tpb * L2 * 8 + 128; }
};

// Odd lmax up to SHM_LMAX_EXT (run-time mirror for the host's variant choice).
inline bool rows_tma_feasible(int lmax) { return lmax >= 1 && lmax <= SHM_LMAX_EXT && (lmax & 1) == 1; }

// EMU != 0 (rows-tma-emu-*): the rows of sh_row_emu<LMAX, EMU> -- part of
// the binary64 products on the integer pipes (dmul_int), bitwise the same
// values -- and, for a point where dmul_int declines a product, the rows of
// sh_row written over them.
template <int LMAX, int TPB, int IN = kInPoints, int EMU = 0>
__global__ void __launch_bounds__(TPB) k_eval_rows_tma(const double* __restrict__ in, int64_t n, int64_t ntiles,
                                                       int normalized, const __grid_constant__ CUtensorMap map_a,
                                                       const __grid_constant__ CUtensorMap map_b) {
  using Plan = RowsTmaPlan<LMAX>;
  static_assert(Plan::feasible(), "rows-tma needs an even row width (odd lmax)");
  constexpr int BW = Plan::kBW;
  extern __shared__ unsigned char smem_rt[];
  double* tile = reinterpret_cast<double*>(smem_rt + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_rt) & 127u)) & 127u));
  const int t = (int)threadIdx.x;
  bool pending = false;  // a previous tile's boxes may still be read from the buffer
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t p0 = tt * TPB;
    const bool valid = (int64_t)t < n - p0;
    double xb = 0.0, yb = 0.0, zb = 1.0;  // rows past n: a dummy direction (the TMA unit clips them)
    bool origin = false;
    if constexpr (IN == kInAngles) {
      if (valid) angles_to_unit<true>(in[2 * (p0 + t)], in[2 * (p0 + t) + 1], xb, yb, zb);
    } else {
      double x = 0.0, y = 0.0, z = 1.0;
      if (valid) {
        x = in[3 * (p0 + t)];
        y = in[3 * (p0 + t) + 1];
        z = in[3 * (p0 + t) + 2];
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
    if (pending) {  // the buffer is reused: wait until the TMA unit has read the last tile
      if (t == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncthreads();
    }
    auto store = [&](int k, double v) {
      const int b = k / BW;
      const int w = b < Plan::nfull ? BW : Plan::rem;
      tile[b * TPB * BW + t * w + (k - b * BW)] = v;
    };
    if (origin) {  // Sec. II: Y = 0 at r = 0 except the constant l = 0
      store(0, kInvSqrt4Pi);
#pragma unroll
      for (int k = 1; k < Plan::L2; ++k) store(k, 0.0);
    } else if (nonfinite3(xb, yb, zb)) {  // NaN in every value but the constant l = 0
      store(0, kInvSqrt4Pi);
#pragma unroll
      for (int k = 1; k < Plan::L2; ++k) store(k, __longlong_as_double(0x7ff8000000000000ll));
    } else if constexpr (EMU != 0) {
      if (sh_row_emu<LMAX, EMU>(xb, yb, zb, store)) sh_row<LMAX>(xb, yb, zb, store);
    } else {
      sh_row<LMAX>(xb, yb, zb, store);
    }
    // the staged values (generic proxy) must be visible to the TMA unit (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
#pragma unroll
      for (int b = 0; b < Plan::nbox; ++b) {
        const CUtensorMap* m = b < Plan::nfull ? &map_a : &map_b;
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(tile + b * TPB * BW);
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     :
                     : "l"(reinterpret_cast<uint64_t>(m)), "r"(b * BW), "r"((int)p0), "r"(sa)
                     : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    pending = true;
  }
  // the last stores' global writes complete before the CTA retires
  if (t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Host side: encodes the tensor maps of `out` and launches k_eval_rows_tma
// (grid = SMs x resident CTAs, CTAs loop over tiles).  *launched = false with
// SHM_OK when TMA does not apply (even lmax, output not 16-byte aligned,
// n >= 2^31, or no driver entry point): the caller then runs a copy-out
// kernel with the same rows.
template <int LMAX, int TPB, int IN, int EMU = 0>
inline shm_status launch_rows_tma(const double* in, int64_t n, double* out, bool normalized, cudaStream_t stream,
                                  bool* launched) {
  *launched = false;
  if constexpr (RowsTmaPlan<LMAX>::feasible()) {
    using Plan = RowsTmaPlan<LMAX>;
    CUtensorMap ma, mb;
    if (!encode_rows_map(&ma, out, n, Plan::L2, Plan::width_a(), TPB) ||
        !encode_rows_map(&mb, out, n, Plan::L2, Plan::width_b(), TPB))
      return SHM_OK;
    constexpr int MAXDEV = 64;
    static int blocks_per_sm[MAXDEV] = {0};
    const int dev = current_device();
    if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
    auto kern = k_eval_rows_tma<LMAX, TPB, IN, EMU>;
    const size_t smem = Plan::smem_bytes(TPB);
    if (blocks_per_sm[dev] == 0) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_eval_rows_tma)");
      int b = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TPB, smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_eval_rows_tma)");
      blocks_per_sm[dev] = std::max(b, 1);
    }
    const int64_t ntiles = (n + TPB - 1) / TPB;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * blocks_per_sm[dev]);
    kern<<<(unsigned)grid, TPB, smem, stream>>>(in, n, ntiles, normalized ? 1 : 0, ma, mb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "k_eval_rows_tma launch");
    *launched = true;
  }
  return SHM_OK;
}

}  // namespace shm
