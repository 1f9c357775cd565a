// shm_projectors: fused non-local projectors f_{s,l}(|d|) R_l^m(d/|d|) on
// atom spheres of a periodic real-space grid (the use the paper's Sec. I
// motivates: projectors of pseudopotential / PAW methods on a 3-D grid).
//
// Launch structure (all on the caller's stream):
//  1. prepare, once per problem (shm_projectors_prepare): k_proj_setup (CTA
//     0) orders the atoms by the lmax of their species, largest first, then
//     by species (atom_order), validates every atom's offsets and species,
//     builds the tile table in that order (tiles = TILE consecutive sphere
//     points of one atom; tile_offsets[j] = number of tiles of the atoms
//     before atom_order[j], 0 tiles for an atom that failed validation) and
//     one descriptor per tile (first point, first output value, atom,
//     species, rows), and zeroes the error word; with the other CTAs it
//     writes the radial tables' interval cubics (FP32, float-float or
//     binary64) and, FP32, the exponent table of the log-grid index;
//     k_proj_disp writes the displacement tables (per atom, axis and grid
//     coordinate).  Tiles of one lmax then run together, so the SMs execute
//     one row code path at a time (instruction-cache locality); the output
//     layout, by atom, is unchanged.
//  2. run, every call (shm_projectors_run): k_proj (persistent: SMs x
//     resident CTAs, tiles dealt round robin) -- each CTA reads its next
//     tile's descriptor, evaluates its rows -- minimum-image displacement,
//     1/r, log-grid index, 4-point Lagrange interpolation of the l radial
//     functions, the real harmonics (sh_core.cuh), and their product -- into
//     a shared-memory tile, then copies the tile (one contiguous block of the
//     output) out with coalesced stores or one bulk copy.  The run writes
//     nothing but the output and the error word: one launch per call.
//  The launch variant (tile size, points per thread, register cap, store
//  path) is the tuner's choice (shm_projectors_autotune) or the default.
// Uneven sphere sizes (4k..65k points) become equal tiles, and the lmax
// order deals every CTA the same mix of row widths; a tile never spans two
// atoms, so every row of a tile has the same width.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "sh_core.cuh"
#include "sh_tile.cuh"
#include "shm_internal.h"

namespace shm {

constexpr int kExpLo = -160;  // FP32 log-grid exponent table covers frexpf exponents kExpLo..kExpHi
constexpr int kExpHi = 140;
constexpr int kExpN = kExpHi - kExpLo + 1;

// Tile descriptor (32 bytes), written by the set-up launch: the tile's first
// sphere point and first output value, its atom, species and row count.
struct __align__(16) ProjTile {
  long long p0, o0;
  int atom, species, rows, pad;
};
// Smallest tile of any launch variant: bounds the descriptor count of a
// problem, n_points / kProjMinTile + n_atoms.
constexpr int kProjMinTile = 128;

// Workspace layout (byte offsets; every block 256-byte aligned).
struct ProjWs {
  size_t words = 0;        // uint32 error word at +8
  size_t tiles = 256;      // int64 tile_offsets[n_atoms + 1]
  size_t order = 0;        // int32 atom_order[n_atoms]
  size_t desc = 0;         // ProjTile[n_points / kProjMinTile + n_atoms + 1]
  size_t etab = 0;         // FP32: int2 {I_e, bits(c_e)}[kExpN]
  size_t disp = 0;         // float (FP32) or double (FP64) disp[n_atoms][3][ng]: displacement tables
  size_t rad32 = 0;        // FP32: float4 {a0, a1, a2, a3}[n_species][n_rad][lstride] (cubic per interval)
  size_t coef = 0;         // FP64: {a0, a1, a2, a3}[n_species][n_rad][lstride] (cubic per interval), float-float
                           // (32 bytes a node) or, with SHM_STRICT_FP64, binary64 (32 bytes a node)
  size_t total = 0;
};

inline size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Host-side bounds that keep every size product below 2^63 (so no byte count
// of the layout or of a range check can wrap): tables of at most 2^26 nodes
// per function and 64 functions per species, so n_species x lstride x n_rad
// x 32 bytes < 2^43; at most 2^40 points and 2^44 values.
constexpr int32_t kProjMaxNRad = 1 << 26;
constexpr int32_t kProjMaxLstride = 64;
constexpr int64_t kProjMaxPoints = (int64_t)1 << 40;
constexpr int64_t kProjMaxValues = (int64_t)1 << 44;

// Validates the host-visible scalars and the host species table of a
// problem without touching the device (no CUDA call); *max_lmax receives the
// largest species lmax.  Every size the layout and the range checks multiply
// is bounded here first.
shm_status proj_validate(const shm_proj_problem* prob, shm_dtype dtype, int* max_lmax) {
  if (!prob) return fail(SHM_EINVAL, "prob is null");
  const shm_proj_problem& p = *prob;
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (p.n_atoms < 0 || p.n_points < 0 || p.n_values < 0) return fail(SHM_EINVAL, "negative size");
  if (p.n_atoms > INT32_MAX) return fail(SHM_EINVAL, "n_atoms must be below 2^31");
  if (p.n_points > kProjMaxPoints) return fail(SHM_EINVAL, "n_points must be at most 2^40");
  if (p.n_values > kProjMaxValues) return fail(SHM_EINVAL, "n_values must be at most 2^44");
  if (p.n_species < 1 || p.n_species > SHM_PROJ_MAX_SPECIES) return fail(SHM_EINVAL, "n_species must be 1..64");
  if (!p.species_lmax) return fail(SHM_EINVAL, "species_lmax (host) is null");
  if (p.n_rad < 4 || p.n_rad > kProjMaxNRad) return fail(SHM_EINVAL, "n_rad must be in 4..2^26");
  if (p.ng < 1 || p.ng > 1290) return fail(SHM_EINVAL, "ng must be in 1..1290");
  if (!(p.r_min > 0) || !(p.dlog > 0) || !(p.box > 0) || !(p.h > 0) || !std::isfinite(p.r_min) ||
      !std::isfinite(p.dlog) || !std::isfinite(p.box) || !std::isfinite(p.h))
    return fail(SHM_EINVAL, "r_min, dlog, box and h must be finite and > 0");
  if (std::fabs(p.ng * p.h - p.box) > 1e-9 * p.box) return fail(SHM_EINVAL, "box must equal ng * h");
  int ml = 0;
  for (int s = 0; s < p.n_species; ++s) {
    const int l = p.species_lmax[s];
    if (l < 0 || l > SHM_LMAX_CAP) return fail(SHM_EINVAL, "species_lmax must be in 0..9");
    ml = std::max(ml, l);
  }
  if (p.radial_lstride < ml + 1 || p.radial_lstride > kProjMaxLstride)
    return fail(SHM_EINVAL, "radial_lstride must be in (1 + max species lmax)..64");
  *max_lmax = ml;
  return SHM_OK;
}

// Workspace layout of a problem that passed proj_validate (its products
// cannot overflow).
ProjWs proj_layout(const shm_proj_problem& p, shm_dtype dt) {
  ProjWs w;
  w.tiles = 256;
  size_t end = w.tiles + round256((size_t)(p.n_atoms + 1) * 8);
  w.order = end;
  end += round256((size_t)std::max<int64_t>(p.n_atoms, 1) * 4);
  w.desc = end;
  end += round256((size_t)(p.n_points / kProjMinTile + p.n_atoms + 1) * sizeof(ProjTile));
  if (dt == SHM_F32) {
    w.etab = end;
    end += round256((size_t)kExpN * 8);
    w.rad32 = end;
    end += round256((size_t)p.n_species * p.radial_lstride * p.n_rad * 16);
  } else {
    w.coef = end;
    end += round256((size_t)p.n_species * p.radial_lstride * p.n_rad * 32);
  }
  w.disp = end;
  end += round256((size_t)p.n_atoms * 3 * p.ng * (dt == SHM_F64 ? 8 : 4));
  w.total = end;
  return w;
}

struct ProjParams {
  int64_t n_atoms, n_points, n_values;
  const double* atom_pos;
  const int32_t* atom_species;
  const double* radial;
  const int64_t* point_offsets;
  const int32_t* point_index;
  const int64_t* out_offsets;
  int32_t n_species, lstride, n_rad, ng;
  double r_min, dlog, box, h;
  signed char lmax[SHM_PROJ_MAX_SPECIES];
  unsigned ng_magic;  // division by ng without division instructions (see div_ng)
  int ng_shift;
  // workspace views
  unsigned* err;
  int64_t* tile_offsets;
  ProjTile* tiles;
  int64_t tiles_cap;  // descriptors the workspace holds (n_points / kProjMinTile + n_atoms + 1)
  int32_t* atom_order;
  int2* etab;
  float4* rad32;
  float* disp32;   // FP32: displacement tables [n_atoms][3][ng]
  float4* coef;  // two per node: {a0.hi, a0.lo, a1.hi, a1.lo}, {a2.hi, a2.lo, a3.hi, a3.lo}; strict: one double4
  int strict;    // FP64 with SHM_STRICT_FP64: binary64 tables, log-grid index and rows (1: products on
                 // the FP64 pipe; 2: the row's output products, 3: all its products on the integer pipes)
  double* disp64;  // FP64: displacement tables [n_atoms][3][ng]
  // derived on the host: 1/box, 1/r_min, 1/dlog, the log-grid constants
  // K0 = -ln(r_min)/dlog, K1 = ln2/(2 dlog), K2 = 1/(2 dlog), and FP32 h, 1/dlog
  double inv_box, inv_rmin, inv_dlog, lg_k0, lg_k1, lg_k2;
  float h32, inv_dlog32;
};

enum : unsigned { kErrOffsets = 1u, kErrSpecies = 2u, kErrGrid = 4u, kErrOut = 8u };

// ---------------------------------------------------------------------------
// Set-up: validation, tile table (block-wide scan), tile descriptors, error
// word, FP32 tables.

__global__ void __launch_bounds__(1024) k_proj_setup(ProjParams P, int tpb, int fp32) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  {  // the interval cubics of the radial tables, spread over every CTA of the grid
    const int64_t nt = (int64_t)P.n_species * P.lstride * P.n_rad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
      // 4-point Lagrange interpolation on the interval [it, it + 1] of the
      // table (stencil i0..i0+3, i0 = clamp(it - 1, 0, n_rad - 4)) as the
      // cubic a0 + a1 u + a2 u^2 + a3 u^3 in u = t - it: the stencil
      // polynomial b0 + b1 x + b2 x^2 + b3 x^3 in x = t - i0 from its forward
      // differences, shifted to x0 = it - i0, computed in binary64 and stored
      // as float-float (the FP64 row takes f_l in float-float), binary64
      // (strict rows) or FP32 (FP32 rows: one 16-byte load and three FMAs
      // per l, where the Lagrange weights of the stencil took four loads, four
      // FMAs and the weights' own arithmetic).
      const int64_t row = i / P.n_rad;  // s * lstride + l
      const int it = (int)(i - row * P.n_rad);
      const int i0 = min(max(it - 1, 0), P.n_rad - 4);
      // stored node-major: the cubics of all l of one interval are adjacent
      // (one or two cache lines per point), at ((s n_rad + it) lstride + l)
      const int64_t sp = row / P.lstride, l = row - sp * P.lstride;
      const int64_t o = (sp * P.n_rad + it) * P.lstride + l;
      const double* F = P.radial + row * P.n_rad + i0;
      const double d1 = F[1] - F[0], d2 = F[2] - 2.0 * F[1] + F[0], d3 = F[3] - 3.0 * F[2] + 3.0 * F[1] - F[0];
      const double b3 = d3 / 6.0, b2 = 0.5 * (d2 - d3), b1 = d1 - 0.5 * d2 + d3 / 3.0;
      const double x0 = (double)(it - i0);
      const double c0 = F[it - i0], c1 = b1 + x0 * (2.0 * b2 + 3.0 * b3 * x0), c2 = b2 + 3.0 * b3 * x0;
      if (fp32) {
        P.rad32[o] = make_float4((float)c0, (float)c1, (float)c2, (float)b3);
        continue;
      }
      if (P.strict) {  // the cubic kept in binary64 (the strict rows evaluate it by binary64 Horner)
        reinterpret_cast<double4*>(P.coef)[o] = make_double4(c0, c1, c2, b3);
        continue;
      }
      const ff f0 = ff_from_double(c0), f1 = ff_from_double(c1), f2 = ff_from_double(c2), f3 = ff_from_double(b3);
      P.coef[2 * o] = make_float4(f0.hi, f0.lo, f1.hi, f1.lo);
      P.coef[2 * o + 1] = make_float4(f2.hi, f2.lo, f3.hi, f3.lo);
    }
  }
  if (blockIdx.x != 0) return;  // the rest is one CTA's work
  if (tid == 0) {
    *P.err = 0u;
    carry = 0;
    P.tile_offsets[0] = 0;
  }
  // atom_order: a counting sort of the atoms by the lmax of their species,
  // largest lmax first, then by species (invalid species count as lmax 0
  // and come last): tiles of one species run together, so the SMs' L1
  // holds one species' radial cubics at a time
  constexpr int kKeys = (SHM_LMAX_CAP + 1) * SHM_PROJ_MAX_SPECIES;
  __shared__ int key_count[kKeys], key_next[kKeys];
  auto key_of = [&](int64_t a) {
    const int s = P.atom_species[a];
    return (s >= 0 && s < P.n_species) ? (SHM_LMAX_CAP - (int)P.lmax[s]) * SHM_PROJ_MAX_SPECIES + s : kKeys - 1;
  };
  for (int k = tid; k < kKeys; k += blockDim.x) key_count[k] = 0;
  __syncthreads();
  for (int64_t a = tid; a < P.n_atoms; a += blockDim.x) atomicAdd(&key_count[key_of(a)], 1);
  __syncthreads();
  if (tid == 0) {
    int start = 0;
    for (int k = 0; k < kKeys; ++k) {
      key_next[k] = start;
      start += key_count[k];
    }
  }
  __syncthreads();
  for (int64_t a = tid; a < P.n_atoms; a += blockDim.x) P.atom_order[atomicAdd(&key_next[key_of(a)], 1)] = (int)a;
  __syncthreads();
  unsigned err = 0;
  for (int64_t base = 0; base < P.n_atoms; base += blockDim.x) {
    const int64_t j = base + tid;
    int64_t ntiles = 0;
    if (j < P.n_atoms) {
      const int64_t a = P.atom_order[j];
      const int64_t p0 = P.point_offsets[a], p1 = P.point_offsets[a + 1];
      const int s = P.atom_species[a];
      bool ok = true;
      if (!(p0 >= 0 && p1 >= p0 && p1 <= P.n_points)) {
        err |= kErrOffsets;
        ok = false;
      }
      if (s < 0 || s >= P.n_species) {
        err |= kErrSpecies;
        ok = false;
      }
      if (ok) {
        const int64_t L2 = (int64_t)(P.lmax[s] + 1) * (P.lmax[s] + 1);
        const int64_t o0 = P.out_offsets[a], o1 = P.out_offsets[a + 1];
        if (!(o0 >= 0 && o1 <= P.n_values && o1 - o0 == (p1 - p0) * L2)) {
          err |= kErrOut;
          ok = false;
        }
      }
      if (ok) ntiles = (p1 - p0 + tpb - 1) / tpb;
    }
    // inclusive block scan of ntiles
    int64_t v = ntiles;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x >> 5;
      int64_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t incl = v + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
    if (j < P.n_atoms) P.tile_offsets[j + 1] = incl;
    __syncthreads();
    if (tid == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (err) atomicOr(P.err, err);
  // one descriptor per tile, each atom's tiles written by one warp (the
  // offsets of the scan above are visible to the whole CTA after its
  // barriers).  Atoms whose point ranges overlap can claim more tiles than
  // the problem has points for: nothing is written past the workspace's
  // descriptors (the run reads no further than that either), and the
  // offsets error bit is set.
  if (tid == 0 && P.tile_offsets[P.n_atoms] > P.tiles_cap) atomicOr(P.err, kErrOffsets);
  for (int64_t j = wid; j < P.n_atoms; j += blockDim.x >> 5) {
    const int64_t t0 = P.tile_offsets[j];
    const int64_t nt = min(P.tile_offsets[j + 1], P.tiles_cap) - t0;
    if (nt <= 0) continue;
    const int a = P.atom_order[j];
    const int s = P.atom_species[a];
    const int64_t pa0 = P.point_offsets[a], pa1 = P.point_offsets[a + 1], oa0 = P.out_offsets[a];
    const int64_t L2 = (int64_t)(P.lmax[s] + 1) * (P.lmax[s] + 1);
    for (int64_t c = lane; c < nt; c += 32) {
      const int64_t p0 = pa0 + c * tpb;
      ProjTile D;
      D.p0 = p0;
      D.o0 = oa0 + (p0 - pa0) * L2;
      D.atom = a;
      D.species = s;
      D.rows = (int)min((int64_t)tpb, pa1 - p0);
      D.pad = 0;
      P.tiles[t0 + c] = D;
    }
  }
  if (fp32) {
    // exponent table: r = m 2^e (m in [0.5, 1)), t = (e ln2 - ln r_min)/dlog + ln(m)/dlog
    //                 = I_e + c_e + ln(m)/dlog with I_e integer, c_e in [0, 1)
    for (int i = tid; i < kExpN; i += blockDim.x) {
      const int e = kExpLo + i;
      const double C = ((double)e * 0.69314718055994530942 - log(P.r_min)) / P.dlog;
      const double I = floor(C);
      const double I_cl = fmin(fmax(I, -2147483000.0), 2147483000.0);
      P.etab[i] = make_int2((int)I_cl, __float_as_int((float)(C - I)));
    }
  }
}

// ---------------------------------------------------------------------------
// Integer / float helpers without conversion instructions.  On a B300,
// integer division, int<->float conversion and float rounding-to-int issue to
// the same narrow pipe as FP64 arithmetic; these replacements use integer and
// FP32 instructions only.

// CTAs of the set-up launch: one, plus enough to convert the FP32 radial
// tables (float conversions issue to the narrow FP64-class pipe, so one SM
// alone would take tens of microseconds for 80k values).
inline unsigned setup_grid(const ProjParams& P, shm_dtype dtype) {
  (void)dtype;
  const int64_t nt = (int64_t)P.n_species * P.lstride * P.n_rad;
  const int64_t g = (nt + 1023) / 1024;
  const int dev = current_device();
  const int64_t cap = dev >= 0 ? sm_count(dev) : 1;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// floor(n / ng) for 0 <= n < 2^31 (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, unsigned case: m and
// l = ceil(log2 ng) precomputed on the host).
__device__ __forceinline__ unsigned div_ng(unsigned n, unsigned magic, int shift) {
  if (shift == 0) return n;  // ng = 1
  const unsigned t1 = __umulhi(magic, n);
  return (t1 + ((n - t1) >> 1)) >> (shift - 1);
}

// float <-> int for |v| < 2^22 through the 1.5 * 2^23 rounding constant.
__device__ __forceinline__ float small_int_to_float(int n) {
  return __int_as_float(0x4B400000 + n) - 12582912.0f;
}
__device__ __forceinline__ int floor_small(float v) {  // floor(v), |v| < 2^22
  const float r = v + 12582912.0f;                     // round to nearest integer, biased
  int n = __float_as_int(r) - 0x4B400000;
  return (r - 12582912.0f > v) ? n - 1 : n;
}

// ln(m) for m in [0.5, 1) to ~7e-8 absolute: range-reduce to m' in
// [1/sqrt2, sqrt2) (m' = 2m, e -= 1 below 1/sqrt2) and sum the atanh series
// ln(m') = 2 atanh(z), z = (m' - 1)/(m' + 1), |z| <= 0.172, to z^11.
__device__ __forceinline__ float log_unit(float m, int& e) {
  if (m < 0.70710678f) {
    m *= 2.0f;
    e -= 1;
  }
  const float z = __fdividef(m - 1.0f, m + 1.0f);
  const float z2 = z * z;
  float p = 1.0f / 11.0f;
  p = fmaf(p, z2, 1.0f / 9.0f);
  p = fmaf(p, z2, 1.0f / 7.0f);
  p = fmaf(p, z2, 1.0f / 5.0f);
  p = fmaf(p, z2, 1.0f / 3.0f);
  p = fmaf(p, z2, 1.0f);
  return 2.0f * z * p;
}

// ln m as a float-float (FP32 pipe) for m = 1 + f in [sqrt(1/2), sqrt(2)),
// with f exact in binary64: ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + ...),
// s = f / (2 + f), |s| <= 0.1716.  s by a quotient with two correction terms
// (each the remainder times the reciprocal of the divisor); the series to
// s^19, its terms from s^11 on (below 2^-28 of the sum) in FP32, the rest in
// float-float.  Emulated absolute error <= 3.3e-15 (2^-48).
__device__ __forceinline__ ff ff_log_mantissa(double f) {
  const ff F = ff_from_double(f);
  const ff D = ff_add(ff{2.0f, 0.0f}, F);
  const float rc = __frcp_rn(D.hi);
  const float q1 = F.hi * rc;
  ff p = two_prod(q1, D.hi);
  const ff R = ff_add(F, ff{-p.hi, -fmaf(q1, D.lo, p.lo)});
  const float q2 = R.hi * rc;
  p = two_prod(q2, D.hi);
  const float R2 = __fadd_rn(__fsub_rn(__fsub_rn(R.hi, p.hi), p.lo), __fsub_rn(R.lo, q2 * D.lo));
  const ff S = ff_add(fast_two_sum(q1, q2), ff{R2 * rc, 0.0f});
  const ff z = ff_mul(S, S);
  float h = 1.0f / 19.0f;
  h = fmaf(h, z.hi, 1.0f / 17.0f);
  h = fmaf(h, z.hi, 1.0f / 15.0f);
  h = fmaf(h, z.hi, 1.0f / 13.0f);
  h = fmaf(h, z.hi, 1.0f / 11.0f);
  ff P = {h, 0.0f};
#pragma unroll
  for (int k = 4; k >= 1; --k) {  // 1/(2k+1) split into hi + lo
    const float chi = (float)(1.0 / (2 * k + 1));
    P = ff_add(ff_mul_u(P, z), ff{chi, (float)(1.0 / (2 * k + 1) - (double)chi)});
  }
  P = ff_add(ff_mul_u(P, z), ff{1.0f, 0.0f});
  const ff L = ff_mul(S, P);
  return {2.0f * L.hi, 2.0f * L.lo};
}

// ---------------------------------------------------------------------------
// Displacement tables.  The minimum-image displacement of a grid point from
// an atom is separable: its component along axis c depends only on the
// point's grid coordinate i_c.  The set-up writes it for every atom, axis and
// i < ng (k_proj_disp), so a point reads three values instead of forming
// them: the same bits the formulas below give, with no per-point arithmetic.

// FP64: grid coordinate i h (the binary64 product) minus the atom coordinate,
// then the minimum image, d - box rint(d / box): the shift is decided on the
// bit pattern of |d| (0 up to box/2, +-box up to 1.5 box; ties at exactly
// box/2 go to 0 like rint's), the rounded product only beyond 1.5 box.  Each
// step is the correctly rounded binary64 operation the definition states.
__device__ __forceinline__ double disp_axis_f64(int i, double ac, const ProjParams& P) {
  double d = __dsub_rn(__dmul_rn((double)i, P.h), ac);
  const long long half_box = __double_as_longlong(0.5 * P.box), three_half_box = __double_as_longlong(1.5 * P.box);
  const long long b = __double_as_longlong(d);
  const long long mag = b & 0x7fffffffffffffffll;
  if (mag > half_box) {
    if (mag <= three_half_box)
      d = __dsub_rn(d, __longlong_as_double(__double_as_longlong(P.box) | (b & (long long)0x8000000000000000ull)));
    else
      d = __dsub_rn(d, __dmul_rn(P.box, rint(d * P.inv_box)));
  }
  return d;
}

// FP32: the atom coordinate in grid units, q = pos / h = U + frac + (whole
// boxes), U in [0, ng), frac in [0, 1) as the float-float fhi + flo; the
// displacement in grid units, (i - U) - frac, minimum image in [-ng/2,
// ng/2), formed exactly as a float-float (the integer part is exact), then
// rounded once, times h.
__device__ __forceinline__ float disp_axis_f32(int i, double pos, const ProjParams& P) {
  const int ng = P.ng;
  const double q = pos / P.h;
  const double Uf = floor(q);
  const double fr = q - Uf;
  // U modulo ng (whole boxes do not change the minimum image), so that
  // i - U lies in (-ng, ng) and one wrap reaches the image
  double Um = Uf - (double)ng * floor(Uf / (double)ng);
  Um = Um < 0.0 ? Um + (double)ng : (Um >= (double)ng ? Um - (double)ng : Um);
  const int U = (int)Um;
  const float fhi = (float)fr, flo = (float)(fr - (double)fhi);
  const float half_box = 0.5f * small_int_to_float(ng);
  int n = i - U;
  const float dn = small_int_to_float(n) - fhi;
  n = dn >= half_box ? n - ng : (dn < -half_box ? n + ng : n);
  const ff sdiff = two_sum(small_int_to_float(n), -fhi);
  const float lo = __fsub_rn(sdiff.lo, flo);
  const float v = __fadd_rn(sdiff.hi, lo);  // grid units, rounded once
  return v * P.h32;
}

// disp[a][c][i] for every atom, axis and grid coordinate (grid-stride).
__global__ void __launch_bounds__(256) k_proj_disp(ProjParams P, int fp32) {
  const int64_t ng = P.ng, n = P.n_atoms * 3 * ng;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ac = e / ng;  // a * 3 + c
    const int i = (int)(e - ac * ng);
    const double pos = P.atom_pos[ac];  // atom_pos[3 a + c]
    if (fp32)
      P.disp32[e] = disp_axis_f32(i, pos, P);
    else
      P.disp64[e] = disp_axis_f64(i, pos, P);
  }
}

// Continuous log-grid index t = ln(r / r_min) / dlog from r^2 (a positive
// normal binary64): r^2 = m 2^E with m in [sqrt(1/2), sqrt(2)), so
// t = E K1 + K0 + ln(m) K2 with K1 = ln 2 / (2 dlog), K2 = 1 / (2 dlog),
// K0 = -ln(r_min) / dlog.  E and m come from the bit pattern; ln m from
// ff_log_mantissa.  Four FP64-pipe instructions (m - 1, E as a double, two
// FMAs) instead of a binary64 logarithm.
struct LogGrid64 {
  double K0, K1, K2;
};
__device__ __forceinline__ double log_grid_index(double r2, const LogGrid64& G) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(r2);
  int E = (int)(b >> 52) - 1023;
  unsigned long long mb = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;  // m in [1, 2)
  const bool halve = mb >= 0x3ff6a09e667f3bcdull;                               // m >= sqrt(2)
  mb -= halve ? (1ull << 52) : 0ull;
  E += halve ? 1 : 0;
  const ff lm = ff_log_mantissa(__longlong_as_double((long long)mb) - 1.0);
  return fma(ff_to_double_finite(lm), G.K2, fma((double)E, G.K1, G.K0));
}

// ---------------------------------------------------------------------------
// Per-row pieces.

// FP32 row of lmax <= 4 times f_l: the plain FP32 recurrences of sh_row
// (at l <= 4 their rounding stays far inside the FP32 tolerance), with f_l
// folded into each pair's scale -- (S_lm f_l) q, then x A_m and x B_m --
// instead of a product by f_l per value.
template <int LMAX>
__device__ __forceinline__ void proj_row_f32_short(float xb, float yb, float zb, const float* f, float* row) {
  static_assert(LMAX <= 4, "short rows only");
  const float qq = fmaf(xb, xb, fmaf(yb, yb, zb * zb));  // |u|^2, ~1 within a few ulp
  row[0] = (float)Sd<false>(0, 0) * f[0];
  float A = xb, B = yb;
#pragma unroll
  for (int m = 0; m <= LMAX; ++m) {
    if (m >= 2) {
      const float An = fmaf(A, xb, -B * yb);
      const float Bn = fmaf(A, yb, B * xb);
      A = An;
      B = Bn;
    }
    auto put = [&](int l, float s) {  // s = S_lm f_l Qh_l^m
      if (m == 0) {
        row[l * l + l] = s;
      } else {
        row[l * l + l + m] = s * A;
        row[l * l + l - m] = s * B;
      }
    };
    if (m >= 1) put(m, (float)Sd<false>(m, m) * f[m]);
    if (m + 1 <= LMAX) put(m + 1, ((float)Sd<false>(m + 1, m) * f[m + 1]) * zb);
    float q2 = 1.0f, q1 = zb;
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l) {
      const float q = fmaf(zb, q1, -(float)SHM_G[l][m] * (qq * q2));
      put(l, ((float)Sd<false>(l, m) * f[l]) * q);
      q2 = q1;
      q1 = q;
    }
  }
}

// One row (lmax = LMAX): f_l(r) = radial(l) for l = 0..LMAX (float for the
// FP32 row, float-float for the FP64 row), then write f_l(r) R_l^m into
// row[0..(LMAX+1)^2).  (dx, dy, dz) is the displacement, or with `unit` its
// unit vector.
// STRICT (FP64): radial(l) returns binary64 f_l and the row is
// f_l(r) x R_l^m of the all-binary64 sh_row, one binary64 product per value;
// STRICT 1 runs every product on the FP64 pipe, STRICT 2 the products that
// leave the row (S A, S B, s A, s B and f_l R) on the integer pipes
// (dmul_int, the same bits), STRICT 3 every product of the row (also the
// scales, the G q products of the recurrences and the m = 0 column).
template <int LMAX, int STRICT = 0, typename T, typename Radial>
__device__ __forceinline__ void proj_row(T dx, T dy, T dz, bool origin, bool unit, Radial&& radial,
                                         T* __restrict__ row) {
  T xb = dx, yb = dy, zb = dz;
  if constexpr (STRICT) {
    static_assert(sizeof(T) == 8, "strict rows are FP64");
    double f[LMAX + 1];
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) f[l] = radial(l);
    if (origin) {
      row[0] = kInvSqrt4Pi * f[0];
#pragma unroll
      for (int k = 1; k < NH<LMAX>::value; ++k) row[k] = 0.0;
      return;
    }
    if (!unit) unit_dir(dx, dy, dz, xb, yb, zb);
    if constexpr (STRICT >= 2) {
      // the same binary64 operations with the products that leave the row
      // (S A, S B, s A, s B, then f_l R; STRICT 3: every product) by dmul_int
      // on the integer pipes: the same bits; a row where dmul_int declines a
      // product (a zero or subnormal factor, e.g. f_l = 0 or a point on an
      // axis) is written again with the FP64 instructions
      unsigned bad_f = 0u;
      const unsigned bad =
          sh_row_emu<LMAX, STRICT == 3 ? (kEmuOut | kEmuScale | kEmuRec | kEmuM0) : kEmuOut>(
              xb, yb, zb, [&](int k, double v) { row[k] = dmul_int(f[l_of_k(k)], v, bad_f); });
      if (bad | bad_f) sh_row<LMAX>(xb, yb, zb, [&](int k, double v) { row[k] = f[l_of_k(k)] * v; });
    } else {
      sh_row<LMAX>(xb, yb, zb, [&](int k, double v) { row[k] = f[l_of_k(k)] * v; });
    }
  } else if constexpr (sizeof(T) == 4) {
    float f[LMAX + 1];
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) f[l] = radial(l);
    if (origin) {
      row[0] = kInvSqrt4Pi * f[0];
#pragma unroll
      for (int k = 1; k < NH<LMAX>::value; ++k) row[k] = 0.0f;
      return;
    }
    if (!unit) unit_dir(dx, dy, dz, xb, yb, zb);
    if constexpr (LMAX <= 4)
      proj_row_f32_short<LMAX>(xb, yb, zb, f, row);
    else
      sh_row<LMAX, false, true>(xb, yb, zb, [&](int k, T v) { row[k] = v * f[l_of_k(k)]; });
  } else {
    ff fff[LMAX + 1];
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) fff[l] = radial(l);
    if (origin) {
      row[0] = kInvSqrt4Pi * ff_to_double_finite(fff[0]);
#pragma unroll
      for (int k = 1; k < NH<LMAX>::value; ++k) row[k] = 0.0;
      return;
    }
    if (!unit) unit_dir(dx, dy, dz, xb, yb, zb);
    if constexpr (LMAX >= 2 && LMAX <= 4) {  // short rows: every column in float-float, f_l folded in
      sh_row_ff_scaled<LMAX>(xb, yb, zb, [&](int k, T v) { row[k] = v; }, fff);
    } else {
      double f[LMAX + 1];
#pragma unroll
      for (int l = 0; l <= LMAX; ++l) f[l] = ff_to_double_finite(fff[l]);
      if constexpr (LMAX >= 5)  // the hybrid row (m >= 2 in float-float), f_l folded into its products
        sh_row_hybrid<LMAX, false, true>(xb, yb, zb, [&](int k, T v) { row[k] = v; }, f, fff);
      else
        sh_row<LMAX>(xb, yb, zb, [&](int k, T v) { row[k] = v * f[l_of_k(k)]; });
    }
  }
}

// Row of a runtime lmax.  LCAP: the largest lmax the instantiation holds
// code for (4 or 9; the launch picks 4 when no species goes above it, so
// that the register allocation and the code follow the short rows alone).
template <int LCAP, int STRICT = 0, typename T, typename Radial>
__device__ __forceinline__ void proj_row_dispatch(int lmax, T dx, T dy, T dz, bool origin, bool unit,
                                                  Radial&& L, T* row) {
  static_assert(LCAP == 4 || LCAP == 9, "LCAP is 4 or 9");
  switch (lmax) {
    case 0: proj_row<0, STRICT>(dx, dy, dz, origin, unit, L, row); break;
    case 1: proj_row<1, STRICT>(dx, dy, dz, origin, unit, L, row); break;
    case 2: proj_row<2, STRICT>(dx, dy, dz, origin, unit, L, row); break;
    case 3: proj_row<3, STRICT>(dx, dy, dz, origin, unit, L, row); break;
    case 4: proj_row<4, STRICT>(dx, dy, dz, origin, unit, L, row); break;
    default:
      if constexpr (LCAP == 9) {
        switch (lmax) {
          case 5: proj_row<5, STRICT>(dx, dy, dz, origin, unit, L, row); break;
          case 6: proj_row<6, STRICT>(dx, dy, dz, origin, unit, L, row); break;
          case 7: proj_row<7, STRICT>(dx, dy, dz, origin, unit, L, row); break;
          case 8: proj_row<8, STRICT>(dx, dy, dz, origin, unit, L, row); break;
          default: proj_row<9, STRICT>(dx, dy, dz, origin, unit, L, row); break;
        }
      }
      break;
  }
}

// FP64 row of grid point g for the atom whose displacement tables start at
// tb (the correctly rounded binary64 value of each step of the definition,
// disp_axis_f64).  STRICT (SHM_STRICT_FP64): the log-grid index from CUDA's
// binary64 log of r^2, the interval cubic by binary64 Horner from binary64
// coefficients, and the all-binary64 harmonic row times f_l.
template <int LCAP, int STRICT = 0>
__device__ __forceinline__ void proj_point_f64(const ProjParams& P, int g, const double* __restrict__ tb,
                                               int s, int lmax, double* row) {
  const double inv_rmin = P.inv_rmin, inv_dlog = P.inv_dlog;
  const LogGrid64 G = {P.lg_k0, P.lg_k1, P.lg_k2};
  const int ng = P.ng;
  const int q1 = (int)div_ng((unsigned)g, P.ng_magic, P.ng_shift);
  const int gi = (int)div_ng((unsigned)q1, P.ng_magic, P.ng_shift);
  const int gj = q1 - gi * ng, gk = g - q1 * ng;
  // the minimum-image displacement from the atom's tables (disp_axis_f64)
  double d[3] = {__ldg(tb + gi), __ldg(tb + ng + gj), __ldg(tb + 2 * ng + gk)};
  const bool origin = is_origin(d[0], d[1], d[2]);
  double t = 0.0;
  bool unit = false;
  if (!origin) {
    // r^2 by two FMAs (within an ulp of the unfused sum; it feeds 1/r and
    // the log-grid index, where an ulp moves t by ~1e-14)
    const double r2 = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
    if (__double_as_longlong(r2) > 0x05e0000000000000ll) {  // r^2 >= 2^-929 (and inf, NaN): the unit vector
      const double ri = rsqrt(r2);                            // by one reciprocal square root, t from r^2
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] *= ri;
      unit = true;
      if constexpr (STRICT)
        t = fma(log(r2), G.K2, G.K0);  // (ln(r^2) / 2 - ln r_min) / dlog
      else
        t = log_grid_index(r2, G);
    } else {
      t = log(sqrt(r2) * inv_rmin) * inv_dlog;
    }
  }
  // t clamped to [0, n_rad - 1] on its integer part (u = 0 at both ends)
  const double tf = floor(t);
  double u = t - tf;
  int it = (int)tf;  // saturates; NaN gives 0
  if (it >= P.n_rad - 1) {
    it = P.n_rad - 1;
    u = 0.0;
  } else if (it < 0 || !((unsigned long long)__double_as_longlong(u) < 0x7ff0000000000000ull)) {
    it = 0;  // below the grid, or t = -inf or NaN (u not finite)
    u = 0.0;
  }
  if constexpr (STRICT) {
    // f_l(r): the interval's cubic in u by binary64 Horner, one 32-byte node
    const double4* c = reinterpret_cast<const double4*>(P.coef) + ((int64_t)s * P.n_rad + it) * P.lstride;
    auto radial = [&](int l) {
      const double4 a = c[l];
      return fma(fma(fma(a.w, u, a.z), u, a.y), u, a.x);
    };
    proj_row_dispatch<LCAP, STRICT, double>(lmax, d[0], d[1], d[2], origin, unit, radial, row);
  } else {
    // f_l(r): the interval's cubic in u by Horner's rule in float-float (FP32
    // pipe), two 16-byte loads per l
    const float4* c = P.coef + 2 * ((int64_t)s * P.n_rad + it) * P.lstride;
    const ff U = ff_from_double(u);
    auto radial = [&](int l) {
      const float4 a01 = __ldg(c + 2 * l), a23 = __ldg(c + 2 * l + 1);
      ff p = ff_add(ff_mul_u(ff{a23.z, a23.w}, U), ff{a23.x, a23.y});
      p = ff_add(ff_mul_u(p, U), ff{a01.z, a01.w});
      return ff_add(ff_mul_u(p, U), ff{a01.x, a01.y});
    };
    proj_row_dispatch<LCAP, 0, double>(lmax, d[0], d[1], d[2], origin, unit, radial, row);
  }
}

// FP32 row of grid point g for the atom whose displacement tables start at
// tb (disp_axis_f32); the log-grid index uses the exponent table so that
// only ln(mantissa) is taken in FP32 and t keeps ~1e-5 absolute accuracy at
// t ~ 2000.  (The hardware log2 in place of log_unit saves ~12 instructions
// per point and 1 % of the time but raises the max scaled error from 8.0e-7
// to 1.0e-6; not used.)  LFIX >= 0: the row of lmax LFIX (lmax is then ignored), written
// with compile-time indices (row may be a register array).
template <int LCAP, int LFIX = -1>
__device__ __forceinline__ void proj_point_f32(const ProjParams& P, int g, const float* __restrict__ tb,
                                               const float4* __restrict__ rs, int lmax, float* row) {
  const float inv_dlog = P.inv_dlog32;
  const int ng = P.ng;
  const int q1 = (int)div_ng((unsigned)g, P.ng_magic, P.ng_shift);
  const int gi = (int)div_ng((unsigned)q1, P.ng_magic, P.ng_shift);
  // the minimum-image displacement from the atom's tables (disp_axis_f32)
  float d[3] = {__ldg(tb + gi), __ldg(tb + ng + (q1 - gi * ng)), __ldg(tb + 2 * ng + (g - q1 * ng))};
  const bool origin = is_origin(d[0], d[1], d[2]);
  int it = 0;
  float u = 0.0f;
  if (!origin) {
    const float r2 = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    float r;
    if (r2 < 1e-4f) {  // r < 1e-2: r and the unit vector in FP64
      const double rd = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
      r = (float)rd;
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] = (float)((double)d[c] / rd);
    } else {  // one reciprocal square root (and a Newton step) gives r and the unit vector
      float ri = rsqrtf(r2);
      const float hr = r2 * ri;
      ri = fmaf(0.5f * ri, fmaf(-hr, ri, 1.0f), ri);
      r = r2 * ri;
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] *= ri;
    }
    // r = m 2^e with m in [0.5, 1), read from the bits (r is a normal float here)
    const unsigned rb = __float_as_uint(r);
    int e = (int)((rb >> 23) & 0xffu) - 126;
    const float m = __uint_as_float((rb & 0x807fffffu) | (126u << 23));
    const float lm = log_unit(m, e);
    const int ei = min(max(e - kExpLo, 0), kExpN - 1);
    const int2 E = P.etab[ei];
    const float v = __int_as_float(E.y) + lm * inv_dlog;  // |v| < 64
    const int fl = floor_small(v);
    u = v - small_int_to_float(fl);
    it = E.x + fl;  // |E.x| <= 2147483000 (clamped by the set-up), |fl| < 64: no int32 overflow
    if (it < 0) {
      it = 0;
      u = 0.0f;
    } else if (it >= P.n_rad - 1) {
      it = P.n_rad - 1;
      u = 0.0f;
    }
  }
  // f_l(r): the interval's cubic in u, one 16-byte node per l (rs: the
  // species' table of n_rad x lstride nodes; 0 <= it < 2^26 and lstride <= 64,
  // so the unsigned product fits 32 bits)
  const float4* tab = rs + (unsigned)it * (unsigned)P.lstride;
  auto radial = [&](int l) {
    const float4 c = __ldg(tab + l);
    return fmaf(fmaf(fmaf(c.w, u, c.z), u, c.y), u, c.x);
  };
  if constexpr (LFIX >= 0)
    proj_row<LFIX, false, float>(d[0], d[1], d[2], origin, true, radial, row);
  else
    proj_row_dispatch<LCAP, 0, float>(lmax, d[0], d[1], d[2], origin, true, radial, row);
}

// Rows of 16 floats (lmax 3) staged contiguously with 16-byte stores.  The
// round's rows go to buf + p + 16 r (buf 16-byte aligned, p = the 16-byte
// phase of the output in floats), where a bulk copy sends them out; with
// p > 0 a row straddles 16-byte chunks, so the chunk that starts row r also
// holds the last p values of row r - 1, which come from the lane before by
// shuffles.  Lane 0 of a warp writes its first values one by one, and the
// last lane of a warp and the last row of the round write their last p
// values one by one (nobody after them in the warp holds them).  Every lane
// of the warp calls this (the shuffles); `active`: this lane has a row.
// Four 16-byte stores per row instead of sixteen 4-byte stores into a
// padded tile and the copy-out loop's loads, index arithmetic and stores.
__device__ __forceinline__ void stage_rows16(float* __restrict__ buf, int p, int r, bool active, bool last,
                                             const float (&v)[16]) {
  const int lane = (int)(threadIdx.x & 31u);
  float4* c4 = reinterpret_cast<float4*>(buf + 16 * r);  // the chunk that starts row r
  switch (p) {
    case 0:
      if (active) {
        c4[0] = make_float4(v[0], v[1], v[2], v[3]);
        c4[1] = make_float4(v[4], v[5], v[6], v[7]);
        c4[2] = make_float4(v[8], v[9], v[10], v[11]);
        c4[3] = make_float4(v[12], v[13], v[14], v[15]);
      }
      break;
    case 1: {
      const float x15 = __shfl_up_sync(0xffffffffu, v[15], 1);
      if (active) {
        if (lane == 0) {
          buf[16 * r + 1] = v[0];
          buf[16 * r + 2] = v[1];
          buf[16 * r + 3] = v[2];
        } else {
          c4[0] = make_float4(x15, v[0], v[1], v[2]);
        }
        c4[1] = make_float4(v[3], v[4], v[5], v[6]);
        c4[2] = make_float4(v[7], v[8], v[9], v[10]);
        c4[3] = make_float4(v[11], v[12], v[13], v[14]);
        if (last || lane == 31) buf[16 * r + 16] = v[15];
      }
      break;
    }
    case 2: {
      const float x14 = __shfl_up_sync(0xffffffffu, v[14], 1), x15 = __shfl_up_sync(0xffffffffu, v[15], 1);
      if (active) {
        if (lane == 0) {
          buf[16 * r + 2] = v[0];
          buf[16 * r + 3] = v[1];
        } else {
          c4[0] = make_float4(x14, x15, v[0], v[1]);
        }
        c4[1] = make_float4(v[2], v[3], v[4], v[5]);
        c4[2] = make_float4(v[6], v[7], v[8], v[9]);
        c4[3] = make_float4(v[10], v[11], v[12], v[13]);
        if (last || lane == 31) {
          buf[16 * r + 16] = v[14];
          buf[16 * r + 17] = v[15];
        }
      }
      break;
    }
    default: {
      const float x13 = __shfl_up_sync(0xffffffffu, v[13], 1), x14 = __shfl_up_sync(0xffffffffu, v[14], 1),
                  x15 = __shfl_up_sync(0xffffffffu, v[15], 1);
      if (active) {
        if (lane == 0)
          buf[16 * r + 3] = v[0];
        else
          c4[0] = make_float4(x13, x14, x15, v[0]);
        c4[1] = make_float4(v[1], v[2], v[3], v[4]);
        c4[2] = make_float4(v[5], v[6], v[7], v[8]);
        c4[3] = make_float4(v[9], v[10], v[11], v[12]);
        if (last || lane == 31) {
          buf[16 * r + 16] = v[13];
          buf[16 * r + 17] = v[14];
          buf[16 * r + 18] = v[15];
        }
      }
      break;
    }
  }
}

// ---------------------------------------------------------------------------
// Persistent main kernel.

// Copies nv contiguous staged values to dst: the part between dst's first
// and last 16-byte boundaries by one bulk copy (cp.async.bulk) issued by
// thread 0, which waits until the copy has read the staging buffer; the
// scalar head and tail by plain stores.  stage must have dst's address
// modulo 16, and the writers must have fenced their shared-memory stores for
// the async proxy before the barrier that precedes this call.
// tid: the calling thread's index among the copying threads (thread 0
// issues the copy); wait_read: thread 0 waits until the copy has read the
// staging buffer (else the caller waits before it next writes the buffer).
template <typename T>
__device__ __forceinline__ void bulk_rows_out(const T* stage, int nv, T* __restrict__ dst, int tid = threadIdx.x,
                                              bool wait_read = true) {
  const int head = min(nv, (int)(((16u - ((unsigned)(uintptr_t)dst & 15u)) & 15u) / sizeof(T)));
  const int nbody = (int)((((size_t)(nv - head) * sizeof(T)) & ~(size_t)15) / sizeof(T));
  const int tail = nv - head - nbody;
  if (tid == 0 && nbody > 0) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst + head),
                 "r"((unsigned)__cvta_generic_to_shared(stage + head)), "r"((unsigned)(nbody * sizeof(T)))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    if (wait_read) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
  if (tid < head) __stcs(dst + tid, stage[tid]);
  if (tid < tail) __stcs(dst + head + nbody + tid, stage[head + nbody + tid]);
}

// Copies rows [0, rows) of a staged tile (row stride RS) to dst[rows * L2],
// with 16-byte stores between a scalar head (up to the first 16-byte
// boundary of dst) and a scalar tail.  For odd L2 the tile rows are
// contiguous (RS = L2), so element j is tile[j]; otherwise its row is
// floor(j / L2) = umulhi(j, ceil(2^32 / L2)), exact for j < 2^32 / L2^2 (here
// j < 256 * 100): no division instructions, which on a B300 would issue
// conversions to the narrow FP64-class pipe.
template <typename T>
__device__ __forceinline__ void copy_rows_out(const T* __restrict__ tile, int rows, int L2, int RS,
                                              T* __restrict__ dst, int tid = threadIdx.x,
                                              int nthreads = blockDim.x) {
  constexpr int E = Vec16<T>::n;
  using V = typename Vec16<T>::type;
  const int nv = rows * L2;
  const unsigned inv = L2 > 1 ? (unsigned)((0x100000000ull + (unsigned)L2 - 1) / (unsigned)L2) : 0u;
  const bool flat = RS == L2;
  auto src = [&](int j) {
    if (flat) return j;
    const int r = (int)__umulhi((unsigned)j, inv);
    return r * RS + (j - r * L2);
  };
  const int head = min(nv, (int)(((16u - ((unsigned)(uintptr_t)dst & 15u)) & 15u) / sizeof(T)));
  for (int j = tid; j < head; j += nthreads) __stcs(dst + j, tile[src(j)]);
  const int nq = (nv - head) / E;
  V* d = reinterpret_cast<V*>(dst + head);
  for (int q = tid; q < nq; q += nthreads) {
    const int j = head + q * E;
    T v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = tile[src(j + i)];
    st_stream(d + q, v);
  }
  for (int j = head + nq * E + tid; j < nv; j += nthreads) __stcs(dst + j, tile[src(j)]);
}

// The persistent kernel.  NT threads per CTA; tiles of TILE = NT x ROUNDS
// sphere points of one atom, evaluated in ROUNDS rounds of NT rows (one per
// thread), each staged in shared memory and sent out before the next (the
// staging buffer holds NT rows); MINB resident CTAs per SM asked of the
// register allocator (0: no cap).  bulk: rows of odd width leave by one bulk
// copy per round, else by the copy-out loop.  The per-tile work (descriptor,
// checks, prefetches) is shared by the ROUNDS rounds.
//
// Static schedule: of G CTAs, CTA b takes tiles b, b + G, b + 2G, ...  The
// tiles are ordered by the lmax of their atom, largest first, then by
// species, so every CTA gets the same mix of row widths, and no counter,
// atomic or search sits between two tiles.  Thread 0 fetches descriptors
// two tiles ahead into shared memory by cp.async (a ring of three), and each
// thread reads the grid index of its next row (in this tile or the next) one
// round ahead into a register, so neither the index stream from DRAM nor
// the descriptor chain stalls the tile's arithmetic, and no shared memory
// holds indices (an index buffer of two tiles, filled by cp.async a tile
// ahead, cost 4 KB per CTA: seven CTAs per SM in FP64 instead of eight, and
// 0.893 against 0.875 ms FP64, 0.232 against 0.217 ms FP32 on the 512-atom
// problem); two barriers per round remain (before and after its stores).  Every
// descriptor is checked against the problem (atom, species, row count, point
// and value ranges) before it is used, and every grid index per point, so a
// workspace that does not hold this problem's tables sets error bits
// instead of reading or writing out of bounds; tile_limit caps the tile
// count read from the workspace.  Nothing in the workspace changes during a
// run: every launch is the same, and a CUDA graph replays it.
// LCAP: rows up to lmax 4 or 9 (proj_row_dispatch).  (Two staging buffers
// used in turn by consecutive rounds, which drop the barrier after each
// round's stores, cost more in occupancy than they save: 0.258 against
// 0.246 ms for FP32 on the 512-atom problem.)
template <typename T, int NT, int ROUNDS, int MINB, int STRICT = 0, int LCAP = 9>
__global__ void __launch_bounds__(NT, MINB) k_proj(ProjParams P, T* __restrict__ out, int tile_bytes,
                                                  int64_t tile_limit, int bulk) {
  constexpr int TILE = NT * ROUNDS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const tile = reinterpret_cast<T*>(smem_raw);
  (void)tile_bytes;
  __shared__ __align__(16) ProjTile s_desc[3];
  const int64_t total_tiles = min(max(P.tile_offsets[P.n_atoms], (int64_t)0), tile_limit);
  const int64_t G = gridDim.x;
  auto cp16 = [](void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
  };
  auto commit = [] { asm volatile("cp.async.commit_group;" ::: "memory"); };
  auto wait_all = [] { asm volatile("cp.async.wait_group 0;" ::: "memory"); };
  // thread 0: the descriptor of tile t into ring slot ds
  auto fetch_desc = [&](int64_t t, int ds) {
    if (t < total_tiles) {
      cp16(&s_desc[ds], P.tiles + t);
      cp16(reinterpret_cast<char*>(&s_desc[ds]) + 16, reinterpret_cast<const char*>(P.tiles + t) + 16);
    }
  };
  // the grid index of row r of tile t, whose descriptor is in ring slot ds
  // (-1 past the tile's rows, past the last tile, or for a descriptor whose
  // ranges do not fit the problem: the tile is skipped), read with the
  // streaming hint so that L1 keeps the radial cubics
  auto fetch_index = [&](int64_t t, int ds, int r) -> int {
    if (t >= total_tiles) return -1;
    const ProjTile D = s_desc[ds];
    if (!(D.rows >= 1 && D.rows <= TILE && D.p0 >= 0 && D.p0 <= P.n_points - D.rows && D.atom >= 0 &&
          D.atom < P.n_atoms) || r >= D.rows)
      return -1;
    return __ldcs(P.point_index + D.p0 + r);
  };
  if (threadIdx.x == 0) {
    fetch_desc(blockIdx.x, 0);
    fetch_desc(blockIdx.x + G, 1);
    commit();
    wait_all();
  }
  __syncthreads();
  // each thread's grid index for its row of the next round, read one round
  // ahead (a register, not a shared-memory buffer of the tile's indices)
  int g_next = fetch_index(blockIdx.x, 0, (int)threadIdx.x);
  int ds = 0;
  for (int64_t t = blockIdx.x; t < total_tiles; t += G) {
    const int ds1 = ds == 2 ? 0 : ds + 1, ds2 = ds1 == 2 ? 0 : ds1 + 1;
    if (threadIdx.x == 0) {
      fetch_desc(t + 2 * G, ds2);
      commit();
    }
    const ProjTile D = s_desc[ds];
    // the tile's atom, species and blocks, checked against the problem
    const int64_t a = D.atom;
    const int s = D.species;
    bool ok = a >= 0 && a < P.n_atoms && s >= 0 && s < P.n_species;
    const int lmax = ok ? P.lmax[s] : 0;
    const int L2 = (lmax + 1) * (lmax + 1);
    const int rows = D.rows;
    const int64_t p0 = D.p0, o0 = D.o0;
    ok = ok && rows >= 1 && rows <= TILE && p0 >= 0 && p0 <= P.n_points - rows && o0 >= 0 &&
         o0 <= P.n_values - (int64_t)rows * L2;
    const int RS = L2 | 1;
    // FP32: the species' interval cubics, once per tile
    const float4* const rad_s = (sizeof(T) == 4 && ok) ? P.rad32 + (int64_t)s * P.n_rad * P.lstride : nullptr;
    (void)rad_s;
    // odd row widths: each round's rows are staged contiguously (RS = L2),
    // shifted so that they have the 16-byte phase of their place in the
    // output (the same for every round: NT L2 values are a multiple of 16
    // bytes), and leave by one bulk copy
    // FP32 rows of 16 values (lmax 3) are staged contiguously too, by
    // stage_rows16, and leave by the same bulk copy (for FP64 the sixteen
    // values held in registers cost more occupancy than the copy-out loop:
    // 96 registers instead of 56, 1.08 against 1.02 ms on the 512-atom
    // problem)
    const bool rows16 = sizeof(T) == 4 && ok && bulk && L2 == 16;
    const bool flat = ok && bulk && ((L2 & 1) != 0 || rows16);
    T* dst = out + o0;
    const int phase = (int)(((uintptr_t)dst & 15u) / sizeof(T));
    if (!ok && threadIdx.x == 0) atomicOr(P.err, kErrOut);  // the same decision in every thread: the tile is skipped
    const int nrounds = ok ? (rows + NT - 1) / NT : 0;
    if (nrounds == 0) g_next = fetch_index(t + G, ds1, (int)threadIdx.x);
#pragma unroll 1
    for (int rd = 0; rd < nrounds; ++rd) {
      const int r0 = rd * NT, rr = min(NT, rows - r0);
      const int g = g_next;  // this thread's row r0 + threadIdx.x (if < rr)
      {
        const int rn = r0 + NT + (int)threadIdx.x;  // its row of the next round
        g_next = rd + 1 < nrounds ? (rn < rows ? __ldcs(P.point_index + p0 + rn) : -1)
                                  : fetch_index(t + G, ds1, (int)threadIdx.x);
      }
      T* const stage = tile + (flat ? phase : 0);
      if constexpr (sizeof(T) == 4) {
        if (rows16) {
          const bool active = (int)threadIdx.x < rr;
          float v[16];
          if (active) {
            if (g < 0 || g >= P.ng * P.ng * P.ng) {
              atomicOr(P.err, kErrGrid);
#pragma unroll
              for (int kk = 0; kk < 16; ++kk) v[kk] = 0.0f;
            } else {
              proj_point_f32<LCAP, 3>(P, g, P.disp32 + a * 3 * P.ng, rad_s, 3, v);
            }
          }
          stage_rows16(tile, phase, (int)threadIdx.x, active, (int)threadIdx.x == rr - 1, v);
        }
      }
      if (!rows16 && (int)threadIdx.x < rr) {
        T* row = stage + threadIdx.x * (flat ? L2 : RS);
        if (g < 0 || g >= P.ng * P.ng * P.ng) {
          atomicOr(P.err, kErrGrid);
          for (int kk = 0; kk < L2; ++kk) row[kk] = (T)0;
        } else if constexpr (sizeof(T) == 8) {
          proj_point_f64<LCAP, STRICT>(P, g, P.disp64 + a * 3 * P.ng, s, lmax, reinterpret_cast<double*>(row));
        } else {
          proj_point_f32<LCAP>(P, g, P.disp32 + a * 3 * P.ng, rad_s, lmax, reinterpret_cast<float*>(row));
        }
      }
      if (flat) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the rows, visible to the bulk copy
      __syncthreads();  // every thread has written its row
      if (flat)
        bulk_rows_out<T>(stage, rr * L2, dst);  // thread 0 waits until the copy has read the buffer
      else
        copy_rows_out<T>(tile, rr, L2, RS, dst);
      dst += (int64_t)rr * L2;
      if (rd + 1 < nrounds) __syncthreads();  // the buffer is free for the next round
    }
    if (threadIdx.x == 0) wait_all();  // the descriptor copies have landed
    __syncthreads();  // the tile buffer is free; the next tiles' descriptors are visible
    ds = ds1;
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Launch variants of the persistent kernel (index = variant id): tile size,
// threads per CTA (rows per round), resident-CTA request for the register
// allocator, and the store path of odd-width rows.  (Tiles of 64 points, one
// round of 256 rows, two points per thread in one round, and a form with
// one 32-point work unit per warp and no CTA barriers were measured slower
// on the 512-atom problem and are not kept.)
struct ProjVariant {
  int tile, nt, minb;
  bool bulk;
  const char* name;
};
constexpr ProjVariant kProjVariants[] = {
    {512, 128, 0, true, "tile512-4rounds"},           {512, 128, 0, false, "tile512-4rounds-copyout"},
    {512, 128, 8, true, "tile512-4rounds-regcap64"},  {512, 128, 10, true, "tile512-4rounds-regcap48"},
    {256, 128, 0, true, "tile256-2rounds"},           {128, 128, 0, true, "tile128"},
    {512, 64, 20, true, "tile512-8rounds-64t-regcap48"}, {512, 256, 5, true, "tile512-2rounds-256t-regcap48"},
    {512, 64, 0, true, "tile512-8rounds-64t"},        {256, 64, 0, true, "tile256-4rounds-64t"},
};
static_assert(kProjMinTile == 128, "every variant's tile is at least kProjMinTile points");
constexpr int kNumProjVariants = sizeof(kProjVariants) / sizeof(kProjVariants[0]);
// Default before (or without) tuning, the fastest on the 512-atom problem
// for both dtypes: tile512-8rounds-64t (FP32 0.215 ms, 0.216 with 128-thread
// rounds; FP64 0.873 ms, 0.876 with 128-thread rounds).  The all-binary64
// projectors run tile512-4rounds (kStrictProjVariant).
inline int default_proj_variant(shm_dtype) { return 8; }
constexpr int kStrictProjVariant = 0;  // SHM_STRICT_FP64 runs one launch shape: tile512-4rounds
constexpr size_t kProjMaxSmem = 232448;  // B300 opt-in shared memory per CTA

// Shared memory of a launch: the staging tile (with room for the 16-byte
// shift of a bulk-copied tile).
inline size_t proj_tile_bytes(int tile, int max_lmax, size_t es) {
  const int RS = ((max_lmax + 1) * (max_lmax + 1)) | 1;
  return ((size_t)tile * RS * es + 15) / 16 * 16 + 16;
}
inline size_t proj_smem(int variant, int max_lmax, size_t es, int64_t n_atoms) {
  (void)n_atoms;
  return proj_tile_bytes(kProjVariants[variant].nt, max_lmax, es);
}

std::mutex g_proj_mu;
int g_proj_choice[2] = {-1, -1};  // [dtype], -1 = default
// the variant a workspace was prepared with (its tile table depends on the
// tile size), with the problem sizes it was prepared for
struct ProjPrepared {
  int variant;
  shm_dtype dtype;
  int64_t n_atoms, n_points, n_values;
  int strict;  // ProjParams::strict of the prepare
};
std::unordered_map<const void*, ProjPrepared> g_prepared;
// Row form of later SHM_STRICT_FP64 prepares: 1 every binary64 product on
// the FP64 pipe, 2 the row's output products on the integer pipes, 3 (the
// default) every product of the row on the integer pipes; the same bits.
// On the 512-atom problem: 2.81, 2.08 and 1.97 ms.  (The unit vector's three
// products on the integer pipes as well: 2.00 ms.)
int g_strict_form = 3;

template <typename T, int NT, int ROUNDS, int MINB, int STRICT = 0>
shm_status launch_proj_v(const ProjParams& P, int max_lmax, T* out, int64_t tile_upper, bool bulk, cudaStream_t s) {
  auto kern = max_lmax <= 4 ? k_proj<T, NT, ROUNDS, MINB, STRICT, 4> : k_proj<T, NT, ROUNDS, MINB, STRICT, 9>;
  const int dev = current_device();
  const size_t tile_bytes = proj_tile_bytes(NT, max_lmax, sizeof(T));
  const size_t smem = tile_bytes;
  int b = 0;
  {
    // the shared-memory opt-in, once per kernel and device (kept at the
    // largest size any problem needs), and the resident-CTA count, once per
    // kernel, device and staging size (the occupancy query is not repeated
    // on every run)
    constexpr int MAXDEV = 64;
    static size_t optin[2][MAXDEV] = {};
    static std::unordered_map<unsigned long long, int> resident;
    std::lock_guard<std::mutex> lk(g_proj_mu);
    if (dev < 0 || dev >= MAXDEV) return fail(SHM_EUNSUPPORTED, "device index out of range");
    const int lc = max_lmax <= 4 ? 0 : 1;
    size_t& done = optin[lc][dev];
    if (done < smem) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(k_proj)");
      done = smem;
    }
    const unsigned long long key = ((unsigned long long)smem << 8) | ((unsigned long long)dev << 1) | (unsigned)lc;
    auto it = resident.find(key);
    if (it != resident.end()) {
      b = it->second;
    } else {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NT, smem);
      if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_proj)");
      resident.emplace(key, b);
    }
  }
  cudaError_t e;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tile_upper, (int64_t)sm_count(dev) * std::max(b, 1)));
  kern<<<(unsigned)grid, NT, smem, s>>>(P, out, (int)tile_bytes, tile_upper, bulk ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "k_proj launch");
  return SHM_OK;
}

template <typename T>
shm_status launch_proj(int variant, const ProjParams& P, int max_lmax, T* out, int64_t tile_upper, cudaStream_t s) {
  const bool bulk = kProjVariants[variant].bulk;
  if constexpr (sizeof(T) == 8) {
    // SHM_STRICT_FP64: one launch shape (kStrictProjVariant's)
    if (P.strict == 3) return launch_proj_v<T, 128, 4, 0, 3>(P, max_lmax, out, tile_upper, true, s);
    if (P.strict == 2) return launch_proj_v<T, 128, 4, 0, 2>(P, max_lmax, out, tile_upper, true, s);
    if (P.strict) return launch_proj_v<T, 128, 4, 0, 1>(P, max_lmax, out, tile_upper, true, s);
  }
  switch (variant) {
    case 0:
    case 1: return launch_proj_v<T, 128, 4, 0>(P, max_lmax, out, tile_upper, bulk, s);
    case 2: return launch_proj_v<T, 128, 4, 8>(P, max_lmax, out, tile_upper, bulk, s);
    case 3: return launch_proj_v<T, 128, 4, 10>(P, max_lmax, out, tile_upper, bulk, s);
    case 4: return launch_proj_v<T, 128, 2, 0>(P, max_lmax, out, tile_upper, bulk, s);
    case 5: return launch_proj_v<T, 128, 1, 0>(P, max_lmax, out, tile_upper, bulk, s);
    case 6: return launch_proj_v<T, 64, 8, 20>(P, max_lmax, out, tile_upper, bulk, s);
    case 7: return launch_proj_v<T, 256, 2, 5>(P, max_lmax, out, tile_upper, bulk, s);
    case 8: return launch_proj_v<T, 64, 8, 0>(P, max_lmax, out, tile_upper, bulk, s);
    case 9: return launch_proj_v<T, 64, 4, 0>(P, max_lmax, out, tile_upper, bulk, s);
  }
  return fail(SHM_EINVAL, "unknown projector launch variant");
}

// Validates the host-visible part of the problem and fills the kernel
// parameters; the device-side arrays are validated by k_proj_setup.
shm_status proj_params(const shm_proj_problem* prob, shm_dtype dtype, void* workspace, size_t ws_bytes,
                       int tile, ProjParams* P, int* max_lmax, int64_t* tile_upper) {
  int ml = 0;
  shm_status vst = proj_validate(prob, dtype, &ml);
  if (vst != SHM_OK) return vst;
  const shm_proj_problem& p = *prob;
  const ProjWs w = proj_layout(p, dtype);
  if (!workspace) return fail(SHM_EINVAL, "workspace is null");
  if (ws_bytes < w.total) return fail(SHM_EINVAL, "workspace too small (see shm_projectors_workspace_size)");
  if (!aligned(workspace, 256)) return fail(SHM_EINVAL, "workspace must be 256-byte aligned");
  shm_status st;
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  if ((st = check_device_range(workspace, w.total, "workspace")) != SHM_OK) return st;
  // the set-up and the run read every array with loads of its element
  // size, which need naturally aligned sources
  if (!aligned(p.point_index, 4) || !aligned(p.atom_pos, 8) || !aligned(p.atom_species, 4) ||
      !aligned(p.point_offsets, 8) || !aligned(p.out_offsets, 8) || !aligned(p.radial, 8))
    return fail(SHM_EINVAL, "problem arrays must be aligned to their element size");
  if (p.n_atoms > 0) {
    if ((st = check_device_range(p.atom_pos, (size_t)p.n_atoms * 24, "atom_pos")) != SHM_OK) return st;
    if ((st = check_device_range(p.atom_species, (size_t)p.n_atoms * 4, "atom_species")) != SHM_OK) return st;
    if ((st = check_device_range(p.point_offsets, (size_t)(p.n_atoms + 1) * 8, "point_offsets")) != SHM_OK) return st;
    if ((st = check_device_range(p.out_offsets, (size_t)(p.n_atoms + 1) * 8, "out_offsets")) != SHM_OK) return st;
  }
  if (p.n_points > 0 && (st = check_device_range(p.point_index, (size_t)p.n_points * 4, "point_index")) != SHM_OK)
    return st;
  if ((st = check_device_range(p.radial, (size_t)p.n_species * p.radial_lstride * p.n_rad * 8, "radial")) != SHM_OK)
    return st;
  memset(P, 0, sizeof(*P));
  P->n_atoms = p.n_atoms;
  P->n_points = p.n_points;
  P->n_values = p.n_values;
  P->atom_pos = p.atom_pos;
  P->atom_species = p.atom_species;
  P->radial = p.radial;
  P->point_offsets = p.point_offsets;
  P->point_index = p.point_index;
  P->out_offsets = p.out_offsets;
  P->n_species = p.n_species;
  P->lstride = p.radial_lstride;
  P->n_rad = p.n_rad;
  P->ng = p.ng;
  P->r_min = p.r_min;
  P->dlog = p.dlog;
  P->box = p.box;
  P->h = p.h;
  for (int s = 0; s < p.n_species; ++s) P->lmax[s] = (signed char)p.species_lmax[s];
  P->inv_box = 1.0 / p.box;
  P->inv_rmin = 1.0 / p.r_min;
  P->inv_dlog = 1.0 / p.dlog;
  P->lg_k0 = -std::log(p.r_min) * P->inv_dlog;
  P->lg_k1 = 0.69314718055994530942 * 0.5 * P->inv_dlog;
  P->lg_k2 = 0.5 * P->inv_dlog;
  P->h32 = (float)p.h;
  P->inv_dlog32 = (float)P->inv_dlog;
  {  // Granlund-Montgomery constants for division by ng (unsigned, dividends < 2^31)
    int l = 0;
    while ((1u << l) < (unsigned)p.ng) ++l;
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - (unsigned long long)p.ng)) / (unsigned long long)p.ng + 1ull;
    P->ng_magic = (unsigned)m;
    P->ng_shift = l;
  }
  char* ws = (char*)workspace;
  P->err = (unsigned*)(ws + w.words + 8);
  P->tile_offsets = (int64_t*)(ws + w.tiles);
  P->tiles = (ProjTile*)(ws + w.desc);
  P->tiles_cap = p.n_points / kProjMinTile + p.n_atoms + 1;
  P->atom_order = (int32_t*)(ws + w.order);
  P->etab = dtype == SHM_F32 ? (int2*)(ws + w.etab) : nullptr;
  P->disp32 = dtype == SHM_F32 ? (float*)(ws + w.disp) : nullptr;
  P->rad32 = dtype == SHM_F32 ? (float4*)(ws + w.rad32) : nullptr;
  P->coef = dtype == SHM_F64 ? (float4*)(ws + w.coef) : nullptr;
  P->disp64 = dtype == SHM_F64 ? (double*)(ws + w.disp) : nullptr;
  *max_lmax = ml;
  // an upper bound of the tile count: every point of every atom in its own partial tile
  *tile_upper = p.n_points / tile + p.n_atoms;
  (void)es;
  return SHM_OK;
}

}  // namespace shm

extern "C" size_t shm_projectors_workspace_size(const shm_proj_problem* prob, shm_dtype dtype) {
  using namespace shm;
  int ml = 0;
  if (proj_validate(prob, dtype, &ml) != SHM_OK) return 0;  // the reason is in shm_last_error()
  return proj_layout(*prob, dtype).total;
}

namespace shm {
namespace {

// Checks the output buffer of a call.
shm_status check_out(const shm_proj_problem* prob, shm_dtype dtype, void* out) {
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  if (prob->n_values > 0) {
    if (!out) return fail(SHM_EINVAL, "out is null");
    if (!aligned(out, es)) return fail(SHM_EINVAL, "out must be aligned to the element size");
    shm_status st = check_device_range(out, (size_t)prob->n_values * es, "out");
    if (st != SHM_OK) return st;
  }
  return SHM_OK;
}

// The variant a prepare uses: the tuned (or pinned) choice for the dtype if
// its shared memory fits this problem, else the default.
int prepare_variant(shm_dtype dtype, int max_lmax, int64_t n_atoms, bool strict = false) {
  if (strict) return kStrictProjVariant;
  int v;
  {
    std::lock_guard<std::mutex> lk(g_proj_mu);
    v = g_proj_choice[dtype == SHM_F64 ? 1 : 0];
  }
  if (v < 0) v = default_proj_variant(dtype);
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  if (proj_smem(v, max_lmax, es, n_atoms) > kProjMaxSmem) v = default_proj_variant(dtype);
  return v;
}

// Set-up launch into `workspace` for `variant`, recorded for later runs.
shm_status prepare_in(const shm_proj_problem* prob, shm_dtype dtype, void* workspace, size_t ws_bytes, int variant,
                      cudaStream_t s, bool strict = false) {
  ProjParams P;
  int max_lmax = 0;
  int64_t tile_upper = 0;
  shm_status st = proj_params(prob, dtype, workspace, ws_bytes, kProjVariants[variant].tile, &P, &max_lmax,
                              &tile_upper);
  if (st != SHM_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_proj_mu);
    P.strict = strict ? g_strict_form : 0;
  }
  if (proj_smem(variant, max_lmax, dtype == SHM_F64 ? 8 : 4, prob->n_atoms) > kProjMaxSmem)
    return fail(SHM_EINVAL, "projector tile does not fit in shared memory for this lmax");
  k_proj_setup<<<setup_grid(P, dtype), 1024, 0, s>>>(P, kProjVariants[variant].tile, dtype == SHM_F32 ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "k_proj_setup launch");
  if (P.n_atoms > 0) {
    const int dev = current_device();
    const int64_t nd = P.n_atoms * 3 * (int64_t)P.ng;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((nd + 255) / 256, (int64_t)(dev >= 0 ? sm_count(dev) : 1) * 8));
    k_proj_disp<<<(unsigned)grid, 256, 0, s>>>(P, dtype == SHM_F32 ? 1 : 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "k_proj_disp launch");
  }
  std::lock_guard<std::mutex> lk(g_proj_mu);
  g_prepared[workspace] = ProjPrepared{variant, dtype, prob->n_atoms, prob->n_points, prob->n_values, P.strict};
  return SHM_OK;
}

// The persistent launch on a prepared workspace.
shm_status run_in(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* workspace, size_t ws_bytes,
                  cudaStream_t s) {
  ProjPrepared rec;
  {
    std::lock_guard<std::mutex> lk(g_proj_mu);
    auto it = g_prepared.find(workspace);
    if (it == g_prepared.end())
      return fail(SHM_EINVAL, "workspace not prepared (call shm_projectors_prepare first)");
    rec = it->second;
  }
  if (rec.dtype != dtype || rec.n_atoms != prob->n_atoms || rec.n_points != prob->n_points ||
      rec.n_values != prob->n_values)
    return fail(SHM_EINVAL, "workspace was prepared for another problem or dtype");
  ProjParams P;
  int max_lmax = 0;
  int64_t tile_upper = 0;
  shm_status st = proj_params(prob, dtype, workspace, ws_bytes, kProjVariants[rec.variant].tile, &P, &max_lmax,
                              &tile_upper);
  if (st != SHM_OK) return st;
  P.strict = rec.strict;
  if ((st = check_out(prob, dtype, out)) != SHM_OK) return st;
  if (prob->n_atoms == 0 || prob->n_points == 0) return SHM_OK;
  return dtype == SHM_F64 ? launch_proj<double>(rec.variant, P, max_lmax, (double*)out, tile_upper, s)
                          : launch_proj<float>(rec.variant, P, max_lmax, (float*)out, tile_upper, s);
}

void load_proj_tune_cache();

}  // namespace
}  // namespace shm

extern "C" shm_status shm_projectors_prepare_ex(const shm_proj_problem* prob, shm_dtype dtype, unsigned flags,
                                                void* workspace, size_t workspace_bytes, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_projectors_prepare");
  clear_error();
  int ml = 0;
  shm_status st = proj_validate(prob, dtype, &ml);
  if (st != SHM_OK) return st;
  if (flags & ~SHM_STRICT_FP64) return fail(SHM_EINVAL, "unknown flag bits");
  const bool strict = dtype == SHM_F64 && (flags & SHM_STRICT_FP64) != 0;
  load_proj_tune_cache();
  return prepare_in(prob, dtype, workspace, workspace_bytes, prepare_variant(dtype, ml, prob->n_atoms, strict),
                    (cudaStream_t)stream, strict);
}

extern "C" shm_status shm_projectors_prepare(const shm_proj_problem* prob, shm_dtype dtype, void* workspace,
                                             size_t workspace_bytes, void* stream) {
  return shm_projectors_prepare_ex(prob, dtype, 0u, workspace, workspace_bytes, stream);
}

extern "C" shm_status shm_projectors_run(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* workspace,
                                         size_t workspace_bytes, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_projectors_run");
  clear_error();
  int ml = 0;
  shm_status st = proj_validate(prob, dtype, &ml);
  if (st != SHM_OK) return st;
  return run_in(prob, dtype, out, workspace, workspace_bytes, (cudaStream_t)stream);
}

extern "C" shm_status shm_projectors_ex(const shm_proj_problem* prob, shm_dtype dtype, unsigned flags, void* out,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_projectors");
  clear_error();
  int ml = 0;
  shm_status st = proj_validate(prob, dtype, &ml);
  if (st != SHM_OK) return st;
  if (flags & ~SHM_STRICT_FP64) return fail(SHM_EINVAL, "unknown flag bits");
  const bool strict = dtype == SHM_F64 && (flags & SHM_STRICT_FP64) != 0;
  if ((st = check_out(prob, dtype, out)) != SHM_OK) return st;
  load_proj_tune_cache();
  cudaStream_t s = (cudaStream_t)stream;
  st = prepare_in(prob, dtype, workspace, workspace_bytes, prepare_variant(dtype, ml, prob->n_atoms, strict), s,
                  strict);
  if (st != SHM_OK) return st;
  return run_in(prob, dtype, out, workspace, workspace_bytes, s);
}

extern "C" shm_status shm_projectors(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  return shm_projectors_ex(prob, dtype, 0u, out, workspace, workspace_bytes, stream);
}

namespace shm {
namespace {

// Projector choices in the tuner's cache file (SHM_TUNE_CACHE): lines
// "3 0 v" (FP32) and "4 0 v" (FP64), v a projector launch variant; the
// evaluator's lines (slots 0..2) share the file.
constexpr int kProjCacheSlotF32 = 3;

void load_proj_tune_cache() {
  static std::once_flag once;
  std::call_once(once, [] {
    const char* path = getenv("SHM_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    int slot, x, v;
    std::lock_guard<std::mutex> lk(g_proj_mu);
    while (fscanf(f, "%d %d %d", &slot, &x, &v) == 3)
      if ((slot == kProjCacheSlotF32 || slot == kProjCacheSlotF32 + 1) && v >= 0 && v < kNumProjVariants)
        g_proj_choice[slot - kProjCacheSlotF32] = v;
    fclose(f);
  });
}

}  // namespace
}  // namespace shm

extern "C" shm_status shm_projectors_autotune(const shm_proj_problem* prob, shm_dtype dtype, void* out,
                                              void* workspace, size_t workspace_bytes, double* best_ms) {
  using namespace shm;
  NvtxRange nvtx_range("shm_projectors_autotune");
  clear_error();
  int ml = 0;
  shm_status st = proj_validate(prob, dtype, &ml);
  if (st != SHM_OK) return st;
  if ((st = check_out(prob, dtype, out)) != SHM_OK) return st;
  load_proj_tune_cache();
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return fail_cuda(e, "cudaStreamCreate");
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = fail_cuda(e, "cudaEventCreate");
  }
  const size_t es = dtype == SHM_F64 ? 8 : 4;
  int best = -1;
  float best_t = 0.f;
  for (int v = 0; v < kNumProjVariants && st == SHM_OK; ++v) {
    if (proj_smem(v, ml, es, prob->n_atoms) > kProjMaxSmem) continue;
    if ((st = prepare_in(prob, dtype, workspace, workspace_bytes, v, s)) != SHM_OK) break;
    float tv = 1e30f;
    for (int rep = 0; rep < 4 && st == SHM_OK; ++rep) {  // the first run is a warm-up
      cudaEventRecord(e0, s);
      st = run_in(prob, dtype, out, workspace, workspace_bytes, s);
      cudaEventRecord(e1, s);
      if (st != SHM_OK) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = fail_cuda(e, "projector autotune: kernel failed");
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
  if (st == SHM_OK && best >= 0) {
    {
      std::lock_guard<std::mutex> lk(g_proj_mu);
      g_proj_choice[dtype == SHM_F64 ? 1 : 0] = best;
    }
    // leave the workspace prepared for the chosen variant
    st = prepare_in(prob, dtype, workspace, workspace_bytes, best, s);
    if (st == SHM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = fail_cuda(e, "cudaStreamSynchronize");
    const char* path = getenv("SHM_TUNE_CACHE");
    if (st == SHM_OK && path && *path) {
      FILE* f = fopen(path, "a");
      if (f) {
        fprintf(f, "%d 0 %d\n", kProjCacheSlotF32 + (dtype == SHM_F64 ? 1 : 0), best);
        fclose(f);
      }
    }
    if (best_ms) *best_ms = best_t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  return st;
}

extern "C" int shm_projectors_variant_count(void) { return shm::kNumProjVariants; }

extern "C" const char* shm_projectors_variant(shm_dtype dtype) {
  using namespace shm;
  if (dtype != SHM_F32 && dtype != SHM_F64) return "";
  load_proj_tune_cache();
  std::lock_guard<std::mutex> lk(g_proj_mu);
  const int v = g_proj_choice[dtype == SHM_F64 ? 1 : 0];
  return kProjVariants[v < 0 ? default_proj_variant(dtype) : v].name;
}

extern "C" shm_status shm_projectors_set_variant(shm_dtype dtype, int variant) {
  using namespace shm;
  clear_error();
  if (dtype != SHM_F32 && dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (variant < -1 || variant >= kNumProjVariants) return fail(SHM_EINVAL, "variant out of range");
  load_proj_tune_cache();
  std::lock_guard<std::mutex> lk(g_proj_mu);
  g_proj_choice[dtype == SHM_F64 ? 1 : 0] = variant;
  return SHM_OK;
}

extern "C" shm_status shm_projectors_set_strict_form(int form) {
  using namespace shm;
  clear_error();
  if (form < 1 || form > 3)
    return fail(SHM_EINVAL, "form must be 1 (every product on the FP64 pipe), 2 (the output products on the "
                            "integer pipes) or 3 (every product of the row on the integer pipes)");
  std::lock_guard<std::mutex> lk(g_proj_mu);
  g_strict_form = form;
  return SHM_OK;
}

extern "C" int shm_projectors_strict_form(void) {
  using namespace shm;
  std::lock_guard<std::mutex> lk(g_proj_mu);
  return g_strict_form;
}

extern "C" shm_status shm_projectors_check(const void* workspace, void* stream, uint32_t* error_bits) {
  using namespace shm;
  clear_error();
  if (!workspace || !error_bits) return fail(SHM_EINVAL, "null argument");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
  unsigned v = 0;
  e = cudaMemcpy(&v, (const char*)workspace + 8, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpy(error word)");
  *error_bits = v;
  return SHM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point: the same two launches with the scratch in a
// static device array of this library instead of a caller workspace.

static __device__ __align__(256) unsigned char g_proj_noalloc_scratch[SHM_PROJ_NOALLOC_SCRATCH_BYTES];

namespace shm {
namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of g_proj_noalloc_scratch on the current device, looked up
// once per device (host code only holds a stand-in for the array's name).
shm_status noalloc_scratch(void** ptr) {
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return fail(SHM_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_proj_noalloc_scratch);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(projector scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return SHM_OK;
}
}  // namespace
}  // namespace shm

extern "C" shm_status shm_projectors_noalloc(const shm_proj_problem* prob, shm_dtype dtype, void* out,
                                              void* stream) {
  using namespace shm;
  NvtxRange nvtx_range("shm_projectors_noalloc");
  clear_error();
  int ml = 0;
  shm_status vst = proj_validate(prob, dtype, &ml);  // the problem's fields first, then its scratch need
  if (vst != SHM_OK) return vst;
  const size_t need = proj_layout(*prob, dtype).total;
  if (need > SHM_PROJ_NOALLOC_SCRATCH_BYTES)
    return fail(SHM_EINVAL, "problem needs " + std::to_string(need) + " bytes of scratch; the allocation-free "
                            "entry point has " + std::to_string((size_t)SHM_PROJ_NOALLOC_SCRATCH_BYTES) +
                            " (use shm_projectors with a workspace)");
  void* scratch = nullptr;
  shm_status st = noalloc_scratch(&scratch);
  if (st != SHM_OK) return st;
  if ((st = check_out(prob, dtype, out)) != SHM_OK) return st;
  load_proj_tune_cache();
  // the set-up launch writes the tile descriptors and clears the error word
  // before the persistent launch reads them
  cudaStream_t s = (cudaStream_t)stream;
  st = prepare_in(prob, dtype, scratch, SHM_PROJ_NOALLOC_SCRATCH_BYTES, prepare_variant(dtype, ml, prob->n_atoms),
                  s);
  if (st != SHM_OK) return st;
  return run_in(prob, dtype, out, scratch, SHM_PROJ_NOALLOC_SCRATCH_BYTES, s);
}
