// shm_eval: all R_l^m, l <= lmax, at n points (the plain evaluator).
//
// One thread evaluates one point (sh_core.cuh) and writes its row of
// (lmax+1)^2 harmonics into a shared-memory tile whose row stride is odd (in
// elements), so the 32 rows a warp writes at once fall in distinct banks.
// The tile of TPB consecutive points is one contiguous block of the output;
// the CTA then copies it out with coalesced 16-byte streaming stores
// (st.global.cs: the output is written once and never re-read by the kernel).
// CTAs loop over tiles (grid = SMs x resident CTAs), so the launch size does
// not grow with n.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "sh_core.cuh"
#include "sh_phased.cuh"
#include "sh_tile.cuh"
#include "sh_tma.cuh"
#include "shm_internal.h"

namespace shm {

// Store paths.
//  kStaged: the CTA's rows go through a shared-memory tile (odd row stride)
//           and leave as coalesced 16-byte streaming stores.
//  kDirect: each thread stores its own row straight to global memory (the
//           warp's 32 rows are 32 separate segments; L2 merges the partial
//           sectors).  Needs no shared memory, so occupancy is bounded by
//           registers only -- useful when the FP64 pipe, not the store
//           pattern, is the limit.
//  kHybrid: kStaged with the FP64 rows of sh_row_hybrid (FP64 for 1/r and
//           m = 0, 1; float-float for m >= 2); for FP32 it is kStaged.
enum StorePath { kStaged = 0, kDirect = 1, kHybrid = 3 };

template <typename T, int LMAX, int TPB, int PATH>
__global__ void __launch_bounds__(TPB) k_eval(const T* __restrict__ pts, int64_t n, T* __restrict__ out,
                                              int64_t ntiles, int normalized, int vec) {
  constexpr int L2 = TileShape<LMAX>::L2;
  constexpr int RS = TileShape<LMAX>::RS;
  constexpr bool HYB = PATH == kHybrid;
  if constexpr (PATH == kDirect) {
    for (int64_t p = (int64_t)blockIdx.x * TPB + threadIdx.x; p < n; p += (int64_t)gridDim.x * TPB) {
      const T x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
      T* row = out + p * L2;
      sh_point<LMAX>(x, y, z, normalized != 0, [&](int k, T v) { __stcs(row + k, v); });
    }
  } else {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t p0 = t * TPB;
      const int rows = (int)min((int64_t)TPB, n - p0);
      if ((int)threadIdx.x < rows) {
        const int64_t p = p0 + threadIdx.x;
        const T x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
        T* row = tile + threadIdx.x * RS;
        sh_point<LMAX, HYB>(x, y, z, normalized != 0, [&](int k, T v) { row[k] = v; });
      }
      __syncthreads();
      copy_out_tile<T, L2, RS, TPB>(tile, rows, out + p0 * L2, vec != 0);
      __syncthreads();
    }
  }
}

// kPhased / kPhasedHybrid (FP64): k_eval_phased of sh_phased.cuh.
// kPhasedHybridTma (FP64): k_eval_phased_tma of sh_tma.cuh (phased hybrid
// rows leaving by TMA tensor stores).  kRowsTma (FP64): k_eval_rows_tma of
// sh_tma.cuh (all-binary64 rows, whole rows staged and sent by TMA tensor
// stores).  For FP32 these variants are the staged path.
// kRowsTmaEmu* (FP64): k_eval_rows_tma with part of the binary64 products on
// the integer pipes (dmul_int: bitwise the FP64 instruction's results).
// kPhasedHybridTmaEmu* (FP64): k_eval_phased_tma with the binary64 products
// of the hybrid rows' m = 0, 1 columns on the integer pipes, the same bits.
enum {
  kPhased = 2,
  kPhasedHybrid = 4,
  kPhasedHybridTma = 5,
  kPhasedHybridTma2 = 6,
  kRowsTma = 7,
  kRowsTmaEmuO = 8,  // output products
  kRowsTmaEmuOS = 9,  // + scales
  kPhasedHybridTmaEmuO = 10,
  kPhasedHybridTmaEmuOS = 11
};

constexpr bool rows_tma_path(int p) { return p == kRowsTma || p == kRowsTmaEmuO || p == kRowsTmaEmuOS; }
constexpr bool phased_tma_path(int p) {
  return p == kPhasedHybridTma || p == kPhasedHybridTmaEmuO || p == kPhasedHybridTmaEmuOS;
}
constexpr int emu_mask(int p) {
  return (p == kRowsTmaEmuO || p == kPhasedHybridTmaEmuO)
             ? kEmuOut
             : ((p == kRowsTmaEmuOS || p == kPhasedHybridTmaEmuOS) ? (kEmuOut | kEmuScale) : 0);
}

// Store paths whose FP64 rows are computed entirely in binary64 arithmetic
// (sh_row, sh_row_lmajor, sh_row_emu): the variants SHM_STRICT_FP64 may run.
constexpr bool strict_path(int p) { return p == kStaged || p == kDirect || p == kPhased || rows_tma_path(p); }

// Launch variants the tuner chooses among (index = variant id).
struct Variant {
  int path, tpb;
};
constexpr Variant kVariants[] = {{kStaged, 128}, {kStaged, 64},  {kStaged, 256},  {kDirect, 128},
                                 {kDirect, 256}, {kPhased, 64}, {kPhased, 128}, {kHybrid, 64},
                                 {kHybrid, 128}, {kHybrid, 256}, {kPhasedHybrid, 64}, {kPhasedHybrid, 128},
                                 {kPhasedHybridTma, 128}, {kPhasedHybridTma2, 128}, {kRowsTma, 64},
                                 {kRowsTma, 32}, {kRowsTmaEmuO, 32}, {kRowsTmaEmuOS, 32},
                                 {kPhasedHybridTmaEmuO, 128}, {kPhasedHybridTmaEmuOS, 128}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// For FP32 the phased and hybrid variants run the staged-64 kernel (FP32 rows
// have no phased or hybrid form); the tuner skips them and the variant name
// reports the kernel that runs.
// Shared memory of a variant's CTA (mirrors eval_smem_bytes) and the limit.
inline size_t variant_smem(int v, int lmax, size_t es) {
  const int L2 = (lmax + 1) * (lmax + 1);
  const int p = kVariants[v].path, tpb = kVariants[v].tpb;
  if (p == kDirect) return 0;
  if (p == kPhasedHybridTma2) return (size_t)2 * tpb * 20 * 8 + 128;
  if (rows_tma_path(p)) return (size_t)tpb * L2 * 8 + 128;
  if (p == kPhased || p == kPhasedHybrid || phased_tma_path(p)) {
    int w = 0, mx = 0;  // LPhases<LMAX>::max_width()
    for (int l = 0; l <= lmax; ++l) {
      if (w > 0 && w + 2 * l + 1 > 37) w = 0;
      w += 2 * l + 1;
      mx = std::max(mx, w);
    }
    return phased_tma_path(p) ? (size_t)tpb * mx * 8 + 128 : (size_t)tpb * (mx | 1) * 8;
  }
  return (size_t)tpb * (size_t)(L2 % 2 ? L2 : L2 + 1) * es;
}
constexpr size_t kMaxSmemPerCta = 232448;  // B300 opt-in limit per CTA

// The variant that actually runs: FP32 rows have no phased or hybrid form
// (staged-64 runs); for l > 9 the FP64 rows are all-FP64 (a hybrid variant
// runs its all-FP64 counterpart); the TMA variant runs phased-hybrid-128 at
// an lmax without a TMA phase plan; a staged variant whose tile does not fit
// in shared memory at this l runs phased-64 (FP64) or staged-64 (FP32).  (At
// run time the TMA variant also falls back to phased-hybrid-128 for an
// output that is not 16-byte aligned or n >= 2^31.)
inline int effective_variant(bool fp64, int v, int lmax = 0) {
  const int p = kVariants[v].path;
  if (!fp64) {
    v = (p == kPhased || p == kHybrid || p == kPhasedHybrid || phased_tma_path(p) || p == kPhasedHybridTma2 ||
         rows_tma_path(p))
            ? 1
            : v;
  } else if (rows_tma_path(p) && !rows_tma_feasible(lmax)) {
    v = 1;  // staged-64: the same all-binary64 rows with the copy-out loop

  } else if (phased_tma_path(p) && !tma_plan_feasible(lmax)) {
    v = lmax > SHM_LMAX_CAP ? 6 : 11;
  } else if (p == kPhasedHybridTma2 && !(lmax == 3 || lmax == 5 || lmax == 7 || lmax == 9)) {
    v = lmax > SHM_LMAX_CAP ? 6 : (tma_plan_feasible(lmax) ? 12 : 11);
  } else if (lmax > SHM_LMAX_CAP) {
    if (v == 7) v = 1;              // hybrid-64 -> staged-64
    else if (v == 8) v = 0;         // hybrid-128 -> staged-128
    else if (v == 9) v = 2;         // hybrid-256 -> staged-256
    else if (v == 10) v = 5;        // phased-hybrid-64 -> phased-64
    else if (v == 11) v = 6;        // phased-hybrid-128 -> phased-128
  }
  if (variant_smem(v, lmax, fp64 ? 8 : 4) > kMaxSmemPerCta) v = fp64 ? 5 : 1;
  return v;
}

// Default choice before (or without) tuning, the fastest measured on a
// 7M-point workload at l = 9: phased-hybrid-tma-128 for FP64 rows (1.30 ms
// against 1.42 ms for phased-hybrid-128 and 3.6 ms for staged-128),
// staged-64 for FP32 rows (HBM-bound, coalesced stores).  At an lmax without
// a TMA plan the FP64 default runs phased-hybrid-128, above l = 9 phased-128
// (effective_variant).
// At l = 5 and 7 the double-buffered TMA form is faster (0.63 / 0.88 ms
// against 0.64 / 0.93 ms on the 192^3 grid); at l = 9 its six phases cost
// more in barriers than the waits they save (1.99 against 1.30 ms).  At
// l = 5 the binary64 products of the m = 0, 1 columns on the integer pipes
// are faster still (phased-hybrid-tma-emu-o-128: 0.571 ms against 0.626 for
// tma2); at l = 7 (0.99 ms) and l = 9 (2.24 ms, register spills) slower.
// With SHM_STRICT_FP64 the FP64 rows are all-binary64: rows-tma-emu-o-32 by
// default (the output products on the integer pipes; staged-64 at even
// lmax, where the row pitch rules TMA out); measured on the 192^3 grid at
// l = 9: rows-tma-emu-o-32 2.57 ms, rows-tma-emu-os-32 2.91, rows-tma-32
// 3.41, rows-tma-64 3.47, phased-64 3.48, staged-64 3.63, staged-128 4.08,
// direct-128 17.6.
constexpr int kDefaultVariantF64 = 12;
constexpr int kDefaultVariantF32 = 1;
constexpr int kDefaultVariantStrict = 16;
inline int default_variant(bool fp64, int lmax = 9, bool strict = false) {
  if (fp64 && strict) return kDefaultVariantStrict;
  return fp64 ? (lmax == 5 ? 18 : lmax == 7 ? 13 : kDefaultVariantF64) : kDefaultVariantF32;
}

// The choice table a call reads: 0 = FP32, 1 = FP64, 2 = FP64 with
// SHM_STRICT_FP64 (strict is ignored for FP32).
inline int choice_slot(bool fp64, bool strict) { return fp64 ? (strict ? 2 : 1) : 0; }

// chosen[slot][lmax] (-1 = default)
int g_choice[3][SHM_LMAX_EXT + 1] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                                     {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                                     {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}};

template <typename T, int LMAX, int TPB, int PATH>
size_t eval_smem_bytes() {
  if (rows_tma_path(PATH)) return RowsTmaPlan<LMAX>::smem_bytes(TPB);
  if (PATH == kPhasedHybridTma2) return Tma2Plan<LMAX>::smem_bytes(TPB);
  if (phased_tma_path(PATH)) return TmaPlan<LMAX>::smem_bytes(TPB);
  if (PATH == kPhased || PATH == kPhasedHybrid)
    return (size_t)TPB * (LPhases<LMAX>::max_width() | 1) * sizeof(double);
  return (PATH == kStaged || PATH == kHybrid) ? (size_t)TPB * TileShape<LMAX>::RS * sizeof(T) : 0;
}

template <typename T, int LMAX, int TPB, int PATH>
auto pick_kernel() {
  if constexpr ((PATH == kPhased || PATH == kPhasedHybrid || phased_tma_path(PATH) || PATH == kPhasedHybridTma2) &&
                sizeof(T) == 8) {
    return k_eval_phased<LMAX, TPB, PATH != kPhased>;
  } else {
    return k_eval<T, LMAX, TPB, (PATH == kPhased || (PATH == kHybrid && sizeof(T) == 4)) ? kStaged : PATH>;
  }
}

// Per-device launch set-up of one instantiation (shared-memory opt-in and
// resident-CTA count), done once.
template <typename T, int LMAX, int TPB, int PATH>
shm_status eval_launch_v(const T* pts, int64_t n, T* out, bool normalized, bool vec, cudaStream_t stream) {
  constexpr int MAXDEV = 64;
  static int blocks_per_sm[MAXDEV] = {0};
  if constexpr (PATH == kPhased || PATH == kPhasedHybrid || phased_tma_path(PATH) || PATH == kPhasedHybridTma2) {
    if constexpr (sizeof(T) == 4) {
      return eval_launch_v<T, LMAX, 64, kStaged>(pts, n, out, normalized, vec, stream);
    }
  }
  if constexpr (phased_tma_path(PATH) && sizeof(T) == 8) {
    bool launched = false;
    if (vec) {
      shm_status st =
          launch_phased_tma<LMAX, TPB, kInPoints, emu_mask(PATH)>(pts, n, out, normalized, stream, &launched);
      if (st != SHM_OK || launched) return st;
    }
    return eval_launch_v<T, LMAX, TPB, kPhasedHybrid>(pts, n, out, normalized, vec, stream);
  }
  if constexpr (PATH == kPhasedHybridTma2 && sizeof(T) == 8) {
    bool launched = false;
    if (vec) {
      shm_status st = launch_phased_tma2<LMAX, TPB, kInPoints>(pts, n, out, normalized, stream, &launched);
      if (st != SHM_OK || launched) return st;
    }
    return eval_launch_v<T, LMAX, TPB, kPhasedHybridTma>(pts, n, out, normalized, vec, stream);
  }
  if constexpr (rows_tma_path(PATH)) {
    if constexpr (sizeof(T) == 8) {
      bool launched = false;
      if (vec) {
        shm_status st =
            launch_rows_tma<LMAX, TPB, kInPoints, emu_mask(PATH)>(pts, n, out, normalized, stream, &launched);
        if (st != SHM_OK || launched) return st;
      }
    }
    // the same all-binary64 rows with the copy-out loop
    return eval_launch_v<T, LMAX, 64, kStaged>(pts, n, out, normalized, vec, stream);
  }
  const int dev = current_device();
  auto kern = pick_kernel<T, LMAX, TPB, PATH>();
  const size_t smem = eval_smem_bytes<T, LMAX, TPB, PATH>();
  if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
  if (blocks_per_sm[dev] == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_eval)");
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TPB, smem);
    if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_eval)");
    blocks_per_sm[dev] = std::max(b, 1);
  }
  const int64_t ntiles = (n + TPB - 1) / TPB;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(dev) * blocks_per_sm[dev]);
  kern<<<(unsigned)grid, TPB, smem, stream>>>(pts, n, out, ntiles, normalized ? 1 : 0, vec ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "k_eval launch");
  return SHM_OK;
}

template <typename T, int LMAX>
shm_status eval_launch(const T* pts, int64_t n, T* out, bool normalized, bool vec, cudaStream_t s, int variant,
                       bool strict) {
  if (variant < 0) {
    variant = g_choice[choice_slot(sizeof(T) == 8, strict)][LMAX];
    if (variant < 0) variant = default_variant(sizeof(T) == 8, LMAX, strict);
  }
  variant = effective_variant(sizeof(T) == 8, variant, LMAX);
  if constexpr (LMAX > SHM_LMAX_CAP) {
    switch (variant) {
      case 0: return eval_launch_v<T, LMAX, 128, kStaged>(pts, n, out, normalized, vec, s);
      case 1: return eval_launch_v<T, LMAX, 64, kStaged>(pts, n, out, normalized, vec, s);
      case 2: return eval_launch_v<T, LMAX, 256, kStaged>(pts, n, out, normalized, vec, s);
      case 3: return eval_launch_v<T, LMAX, 128, kDirect>(pts, n, out, normalized, vec, s);
      case 4: return eval_launch_v<T, LMAX, 256, kDirect>(pts, n, out, normalized, vec, s);
      case 5: return eval_launch_v<T, LMAX, 64, kPhased>(pts, n, out, normalized, vec, s);
      case 6: return eval_launch_v<T, LMAX, 128, kPhased>(pts, n, out, normalized, vec, s);
      case 14: return eval_launch_v<T, LMAX, 64, kRowsTma>(pts, n, out, normalized, vec, s);
      case 15: return eval_launch_v<T, LMAX, 32, kRowsTma>(pts, n, out, normalized, vec, s);
      case 16: return eval_launch_v<T, LMAX, 32, kRowsTmaEmuO>(pts, n, out, normalized, vec, s);
      case 17: return eval_launch_v<T, LMAX, 32, kRowsTmaEmuOS>(pts, n, out, normalized, vec, s);
    }
    return fail(SHM_EINVAL, "unknown launch variant");
  }
  switch (variant) {
    case 0: return eval_launch_v<T, LMAX, 128, kStaged>(pts, n, out, normalized, vec, s);
    case 1: return eval_launch_v<T, LMAX, 64, kStaged>(pts, n, out, normalized, vec, s);
    case 2: return eval_launch_v<T, LMAX, 256, kStaged>(pts, n, out, normalized, vec, s);
    case 3: return eval_launch_v<T, LMAX, 128, kDirect>(pts, n, out, normalized, vec, s);
    case 4: return eval_launch_v<T, LMAX, 256, kDirect>(pts, n, out, normalized, vec, s);
    case 5: return eval_launch_v<T, LMAX, 64, kPhased>(pts, n, out, normalized, vec, s);
    case 6: return eval_launch_v<T, LMAX, 128, kPhased>(pts, n, out, normalized, vec, s);
    case 7: return eval_launch_v<T, LMAX, 64, kHybrid>(pts, n, out, normalized, vec, s);
    case 8: return eval_launch_v<T, LMAX, 128, kHybrid>(pts, n, out, normalized, vec, s);
    case 9: return eval_launch_v<T, LMAX, 256, kHybrid>(pts, n, out, normalized, vec, s);
    case 10: return eval_launch_v<T, LMAX, 64, kPhasedHybrid>(pts, n, out, normalized, vec, s);
    case 11: return eval_launch_v<T, LMAX, 128, kPhasedHybrid>(pts, n, out, normalized, vec, s);
    case 12: return eval_launch_v<T, LMAX, 128, kPhasedHybridTma>(pts, n, out, normalized, vec, s);
    case 13: return eval_launch_v<T, LMAX, 128, kPhasedHybridTma2>(pts, n, out, normalized, vec, s);
    case 14: return eval_launch_v<T, LMAX, 64, kRowsTma>(pts, n, out, normalized, vec, s);
    case 15: return eval_launch_v<T, LMAX, 32, kRowsTma>(pts, n, out, normalized, vec, s);
    case 16: return eval_launch_v<T, LMAX, 32, kRowsTmaEmuO>(pts, n, out, normalized, vec, s);
    case 17: return eval_launch_v<T, LMAX, 32, kRowsTmaEmuOS>(pts, n, out, normalized, vec, s);
    case 18: return eval_launch_v<T, LMAX, 128, kPhasedHybridTmaEmuO>(pts, n, out, normalized, vec, s);
    case 19: return eval_launch_v<T, LMAX, 128, kPhasedHybridTmaEmuOS>(pts, n, out, normalized, vec, s);
  }
  return fail(SHM_EINVAL, "unknown launch variant");
}

template <typename T>
shm_status eval_dispatch(const T* pts, int64_t n, int lmax, T* out, bool normalized, bool vec, cudaStream_t s,
                         int variant = -1, bool strict = false) {
  switch (lmax) {
    case 0: return eval_launch<T, 0>(pts, n, out, normalized, vec, s, variant, strict);
    case 1: return eval_launch<T, 1>(pts, n, out, normalized, vec, s, variant, strict);
    case 2: return eval_launch<T, 2>(pts, n, out, normalized, vec, s, variant, strict);
    case 3: return eval_launch<T, 3>(pts, n, out, normalized, vec, s, variant, strict);
    case 4: return eval_launch<T, 4>(pts, n, out, normalized, vec, s, variant, strict);
    case 5: return eval_launch<T, 5>(pts, n, out, normalized, vec, s, variant, strict);
    case 6: return eval_launch<T, 6>(pts, n, out, normalized, vec, s, variant, strict);
    case 7: return eval_launch<T, 7>(pts, n, out, normalized, vec, s, variant, strict);
    case 8: return eval_launch<T, 8>(pts, n, out, normalized, vec, s, variant, strict);
    case 9: return eval_launch<T, 9>(pts, n, out, normalized, vec, s, variant, strict);
    case 10: return eval_launch<T, 10>(pts, n, out, normalized, vec, s, variant, strict);
    case 11: return eval_launch<T, 11>(pts, n, out, normalized, vec, s, variant, strict);
    case 12: return eval_launch<T, 12>(pts, n, out, normalized, vec, s, variant, strict);
    case 13: return eval_launch<T, 13>(pts, n, out, normalized, vec, s, variant, strict);
    case 14: return eval_launch<T, 14>(pts, n, out, normalized, vec, s, variant, strict);
    case 15: return eval_launch<T, 15>(pts, n, out, normalized, vec, s, variant, strict);
    case 16: return eval_launch<T, 16>(pts, n, out, normalized, vec, s, variant, strict);
  }
  return fail(SHM_EINVAL, "lmax must be in 0..16");
}

void ensure_tune_cache();

}  // namespace shm

extern "C" shm_status shm_eval_ex(const void* points, int64_t n, int lmax, shm_dtype dtype, unsigned flags,
                                  void* out, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_eval_ex");
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (lmax < 0 || lmax > SHM_LMAX_EXT) return fail(SHM_EINVAL, "lmax must be in 0..16");
  if (n < 0) return fail(SHM_EINVAL, "n must be >= 0");
  if (flags & ~(SHM_NORMALIZED_INPUT | SHM_STRICT_FP64)) return fail(SHM_EINVAL, "unknown flag bits");
  if (n == 0) return SHM_OK;
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  const int64_t L2 = (int64_t)(lmax + 1) * (lmax + 1);
  if (n > (INT64_MAX / 8) / (L2 * 8)) return fail(SHM_EINVAL, "n too large");
  if (!points || !out) return fail(SHM_EINVAL, "points and out must be non-null");
  if (!aligned(points, es) || !aligned(out, es))
    return fail(SHM_EINVAL, "points and out must be aligned to the element size");
  const size_t in_bytes = (size_t)n * 3 * es, out_bytes = (size_t)n * L2 * es;
  if (ranges_overlap(points, in_bytes, out, out_bytes)) return fail(SHM_EINVAL, "points and out overlap");
  shm_status st = check_device_range(points, in_bytes, "points");
  if (st != SHM_OK) return st;
  st = check_device_range(out, out_bytes, "out");
  if (st != SHM_OK) return st;
  const bool vec = aligned(out, 16);
  const bool norm = (flags & SHM_NORMALIZED_INPUT) != 0;
  const bool strict = (flags & SHM_STRICT_FP64) != 0;
  ensure_tune_cache();
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == SHM_F64)
    return eval_dispatch<double>((const double*)points, n, lmax, (double*)out, norm, vec, s, -1, strict);
  return eval_dispatch<float>((const float*)points, n, lmax, (float*)out, norm, vec, s);
}

extern "C" shm_status shm_eval(const void* points, int64_t n, int lmax, shm_dtype dtype, void* out, void* stream) {
  return shm_eval_ex(points, n, lmax, dtype, 0u, out, stream);
}

// ---------------------------------------------------------------------------
// Host-buffer entry point: chunked H2D -> kernel -> D2H through a caller
// workspace, alternating between two internal streams.

namespace shm {
namespace {

struct HostPipe {
  cudaStream_t s[2] = {nullptr, nullptr};
  cudaEvent_t ev_in = nullptr, ev_done[2] = {nullptr, nullptr};
  bool ready = false;
};

HostPipe g_pipes[64];
std::mutex g_pipe_mu;

shm_status get_pipe(int dev, HostPipe** out) {
  if (dev < 0 || dev >= 64) return fail(SHM_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe& p = g_pipes[dev];
  if (!p.ready) {
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail_cuda(e, "cudaStreamCreateWithFlags");
      e = cudaEventCreateWithFlags(&p.ev_done[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return fail_cuda(e, "cudaEventCreateWithFlags");
    }
    cudaError_t e = cudaEventCreateWithFlags(&p.ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_cuda(e, "cudaEventCreateWithFlags");
    p.ready = true;
  }
  *out = &p;
  return SHM_OK;
}

}  // namespace
}  // namespace shm

extern "C" size_t shm_eval_host_workspace_size(int lmax, shm_dtype dtype, int64_t chunk_points) {
  if (lmax < 0 || lmax > SHM_LMAX_EXT || chunk_points <= 0 || (dtype != SHM_F32 && dtype != SHM_F64)) return 0;
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  const size_t per = es * (3 + (size_t)(lmax + 1) * (lmax + 1));
  // two buffers, each point block and row block rounded up to 256 bytes
  return 2 * (((size_t)chunk_points * 3 * es + 255) / 256 * 256 + ((size_t)chunk_points * per + 255) / 256 * 256);
}

extern "C" shm_status shm_eval_host_ex(const void* points_host, int64_t n, int lmax, shm_dtype dtype,
                                       unsigned flags, void* out_host, void* workspace, size_t workspace_bytes,
                                       void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_eval_host_ex");
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (lmax < 0 || lmax > SHM_LMAX_EXT) return fail(SHM_EINVAL, "lmax must be in 0..16");
  if (n < 0) return fail(SHM_EINVAL, "n must be >= 0");
  if (flags & ~(SHM_NORMALIZED_INPUT | SHM_STRICT_FP64)) return fail(SHM_EINVAL, "unknown flag bits");
  const bool norm = (flags & SHM_NORMALIZED_INPUT) != 0, strict = (flags & SHM_STRICT_FP64) != 0;
  if (n == 0) return SHM_OK;
  if (!points_host || !out_host) return fail(SHM_EINVAL, "points_host and out_host must be non-null");
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  const int64_t L2 = (int64_t)(lmax + 1) * (lmax + 1);
  // largest chunk whose double buffer fits the workspace
  int64_t chunk = (int64_t)(workspace_bytes / (2 * es * (3 + L2)));
  while (chunk > 0 && shm_eval_host_workspace_size(lmax, dtype, chunk) > workspace_bytes) --chunk;
  if (chunk <= 0) return fail(SHM_EINVAL, "workspace too small for one point");
  chunk = std::min(chunk, n);
  shm_status st = check_device_range(workspace, shm_eval_host_workspace_size(lmax, dtype, chunk), "workspace");
  if (st != SHM_OK) return st;
  ensure_tune_cache();
  const int dev = current_device();
  HostPipe* pipe = nullptr;
  if ((st = get_pipe(dev, &pipe)) != SHM_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t in_blk = ((size_t)chunk * 3 * es + 255) / 256 * 256;
  const size_t out_blk = ((size_t)chunk * L2 * es + 255) / 256 * 256;
  char* base = (char*)workspace;
  char* bin[2] = {base, base + in_blk + out_blk};
  char* bout[2] = {base + in_blk, base + 2 * in_blk + out_blk};
  cudaError_t e = cudaEventRecord(pipe->ev_in, cs);
  if (e != cudaSuccess) return fail_cuda(e, "cudaEventRecord");
  for (int i = 0; i < 2; ++i)
    if ((e = cudaStreamWaitEvent(pipe->s[i], pipe->ev_in, 0)) != cudaSuccess) return fail_cuda(e, "cudaStreamWaitEvent");
  int64_t c = 0;
  for (int64_t p0 = 0; p0 < n; p0 += chunk, ++c) {
    const int b = (int)(c & 1);
    const int64_t m = std::min(chunk, n - p0);
    cudaStream_t s = pipe->s[b];
    e = cudaMemcpyAsync(bin[b], (const char*)points_host + (size_t)p0 * 3 * es, (size_t)m * 3 * es,
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpyAsync H2D");
    st = dtype == SHM_F64
             ? eval_dispatch<double>((const double*)bin[b], m, lmax, (double*)bout[b], norm, true, s, -1, strict)
             : eval_dispatch<float>((const float*)bin[b], m, lmax, (float*)bout[b], norm, true, s);
    if (st != SHM_OK) return st;
    e = cudaMemcpyAsync((char*)out_host + (size_t)p0 * L2 * es, bout[b], (size_t)m * L2 * es, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpyAsync D2H");
  }
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaEventRecord(pipe->ev_done[i], pipe->s[i])) != cudaSuccess) return fail_cuda(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(cs, pipe->ev_done[i], 0)) != cudaSuccess) return fail_cuda(e, "cudaStreamWaitEvent");
  }
  return SHM_OK;
}

extern "C" shm_status shm_eval_host(const void* points_host, int64_t n, int lmax, shm_dtype dtype, void* out_host,
                                    void* workspace, size_t workspace_bytes, void* stream) {
  return shm_eval_host_ex(points_host, n, lmax, dtype, 0u, out_host, workspace, workspace_bytes, stream);
}

// ---------------------------------------------------------------------------
// Autotuner.

namespace shm {
namespace {

const char* kVariantNames[kNumVariants] = {"staged-128", "staged-64",  "staged-256", "direct-128", "direct-256",
                                           "phased-64",  "phased-128", "hybrid-64",  "hybrid-128", "hybrid-256",
                                           "phased-hybrid-64", "phased-hybrid-128", "phased-hybrid-tma-128",
                                           "phased-hybrid-tma2-128", "rows-tma-64", "rows-tma-32",
                                           "rows-tma-emu-o-32", "rows-tma-emu-os-32",
                                           "phased-hybrid-tma-emu-o-128", "phased-hybrid-tma-emu-os-128"};

std::mutex g_tune_mu;
bool g_cache_loaded = false;

void load_tune_cache_locked() {
  if (g_cache_loaded) return;
  g_cache_loaded = true;
  const char* path = getenv("SHM_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  // lines "slot lmax variant": slot 0 = FP32, 1 = FP64, 2 = FP64 with SHM_STRICT_FP64
  int dt, l, v;
  while (fscanf(f, "%d %d %d", &dt, &l, &v) == 3)
    if (dt >= 0 && dt <= 2 && l >= 0 && l <= SHM_LMAX_EXT && v >= 0 && v < kNumVariants &&
        (dt != 2 || strict_path(kVariants[v].path)))
      g_choice[dt][l] = v;
  fclose(f);
}

// Fills pts[n][3] with scattered points in [-1, 1]^3 (a hash of the index).
template <typename T>
__global__ void k_probe_points(T* pts, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    pts[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

template <typename T>
shm_status autotune_t(int lmax, int64_t n, double* best_ms, bool strict) {
  T *pts = nullptr, *out = nullptr;
  const size_t nh = (size_t)(lmax + 1) * (lmax + 1);
  cudaError_t e = dev_malloc((void**)&pts, (size_t)n * 3 * sizeof(T), "autotune");
  if (e != cudaSuccess) return fail_alloc(e, "autotune", "autotune: cudaMalloc of probe points failed");
  e = dev_malloc((void**)&out, (size_t)n * nh * sizeof(T), "autotune");
  if (e != cudaSuccess) {
    cudaFree(pts);
    return fail_alloc(e, "autotune", "autotune: cudaMalloc of probe output failed");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe_points<T><<<1024, 256>>>(pts, n);
  int best = -1;
  float best_t = 0.f;
  shm_status st = SHM_OK;
  for (int v = 0; v < kNumVariants && st == SHM_OK; ++v) {
    if (effective_variant(sizeof(T) == 8, v, lmax) != v) continue;
    if (strict && !strict_path(kVariants[v].path)) continue;
    float tv = 1e30f;
    for (int rep = 0; rep < 4 && st == SHM_OK; ++rep) {  // first repetition is a warm-up
      cudaEventRecord(e0, 0);
      st = eval_dispatch<T>(pts, n, lmax, out, false, true, 0, v, strict);
      cudaEventRecord(e1, 0);
      if (st != SHM_OK) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = fail_cuda(e, "autotune: kernel failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tv = std::min(tv, ms);
    }
    if (st == SHM_OK && (best < 0 || tv < best_t)) {
      best = v;
      best_t = tv;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(pts);
  cudaFree(out);
  if (st != SHM_OK) return st;
  const int slot = choice_slot(sizeof(T) == 8, strict);
  g_choice[slot][lmax] = best;
  if (best_ms) *best_ms = best_t;
  const char* path = getenv("SHM_TUNE_CACHE");
  if (path && *path) {
    FILE* f = fopen(path, "a");
    if (f) {
      fprintf(f, "%d %d %d\n", slot, lmax, best);
      fclose(f);
    }
  }
  return SHM_OK;
}

}  // namespace

void ensure_tune_cache() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_tune_cache_locked();
}

}  // namespace shm

extern "C" shm_status shm_autotune_ex(int lmax, shm_dtype dtype, unsigned flags, int64_t n_probe, double* best_ms) {
  using namespace shm;
  NvtxRange nvtx_range("shm_autotune_ex");
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (lmax < 0 || lmax > SHM_LMAX_EXT) return fail(SHM_EINVAL, "lmax must be in 0..16");
  if (n_probe <= 0 || n_probe > (int64_t)1 << 26) return fail(SHM_EINVAL, "n_probe must be in 1..2^26");
  if (flags & ~SHM_STRICT_FP64) return fail(SHM_EINVAL, "unknown flag bits");
  const bool strict = dtype == SHM_F64 && (flags & SHM_STRICT_FP64) != 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_tune_cache_locked();
  return dtype == SHM_F64 ? autotune_t<double>(lmax, n_probe, best_ms, strict)
                          : autotune_t<float>(lmax, n_probe, best_ms, false);
}

extern "C" shm_status shm_autotune(int lmax, shm_dtype dtype, int64_t n_probe, double* best_ms) {
  return shm_autotune_ex(lmax, dtype, 0u, n_probe, best_ms);
}

extern "C" const char* shm_eval_variant_ex(int lmax, shm_dtype dtype, unsigned flags) {
  using namespace shm;
  if (lmax < 0 || lmax > SHM_LMAX_EXT || (dtype != SHM_F32 && dtype != SHM_F64)) return "";
  ensure_tune_cache();
  const bool fp64 = dtype == SHM_F64, strict = fp64 && (flags & SHM_STRICT_FP64) != 0;
  const int v = g_choice[choice_slot(fp64, strict)][lmax];
  return kVariantNames[effective_variant(fp64, v < 0 ? default_variant(fp64, lmax, strict) : v, lmax)];
}

extern "C" const char* shm_eval_variant(int lmax, shm_dtype dtype) { return shm_eval_variant_ex(lmax, dtype, 0u); }

extern "C" int shm_eval_variant_count(void) { return shm::kNumVariants; }

extern "C" shm_status shm_eval_set_variant_ex(int lmax, shm_dtype dtype, unsigned flags, int variant) {
  using namespace shm;
  clear_error();
  if (lmax < 0 || lmax > SHM_LMAX_EXT || (dtype != SHM_F32 && dtype != SHM_F64))
    return fail(SHM_EINVAL, "bad lmax or dtype");
  if (flags & ~SHM_STRICT_FP64) return fail(SHM_EINVAL, "unknown flag bits");
  if (variant < -1 || variant >= kNumVariants) return fail(SHM_EINVAL, "variant out of range");
  const bool fp64 = dtype == SHM_F64, strict = fp64 && (flags & SHM_STRICT_FP64) != 0;
  if (strict && variant >= 0 && !strict_path(kVariants[variant].path))
    return fail(SHM_EINVAL, "variant computes part of its rows in float-float; SHM_STRICT_FP64 takes only "
                            "all-binary64 variants");
  ensure_tune_cache();
  g_choice[choice_slot(fp64, strict)][lmax] = variant;
  return SHM_OK;
}

extern "C" shm_status shm_eval_set_variant(int lmax, shm_dtype dtype, int variant) {
  return shm_eval_set_variant_ex(lmax, dtype, 0u, variant);
}
