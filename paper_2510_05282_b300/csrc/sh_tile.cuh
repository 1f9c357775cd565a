// Shared-memory staging of a tile of harmonic rows and its coalesced copy-out
// (used by the evaluator and by the serving batch kernel).
#pragma once

#include "sh_core.cuh"

namespace shm {

template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};

__device__ __forceinline__ void st_stream(double2* p, const double (&v)[2]) { __stcs(p, make_double2(v[0], v[1])); }
__device__ __forceinline__ void st_stream(float4* p, const float (&v)[4]) {
  __stcs(p, make_float4(v[0], v[1], v[2], v[3]));
}

template <int LMAX>
struct TileShape {
  static constexpr int L2 = NH<LMAX>::value;
  static constexpr int RS = (L2 % 2 == 1) ? L2 : L2 + 1;  // odd row stride in elements
};

// Copies rows [0, rows) of a staged tile (row stride RS) to the contiguous
// destination dst[rows * L2].  vec: dst is 16-byte aligned.
template <typename T, int L2, int RS, int TPB>
__device__ __forceinline__ void copy_out_tile(const T* __restrict__ tile, int rows, T* __restrict__ dst, bool vec) {
  const int nv = rows * L2;
  int done = 0;
  if (vec) {
    constexpr int E = Vec16<T>::n;
    using V = typename Vec16<T>::type;
    const int nvec = nv / E;
    for (int v = threadIdx.x; v < nvec; v += TPB) {
      int j = v * E;
      int r = j / L2;
      int c = j - r * L2;
      T vals[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        vals[e] = tile[r * RS + c];
        if (++c == L2) {
          c = 0;
          ++r;
        }
      }
      st_stream(reinterpret_cast<V*>(dst) + v, vals);
    }
    done = nvec * E;
  }
  for (int j = done + threadIdx.x; j < nv; j += TPB) {
    const int r = j / L2;
    dst[j] = tile[r * RS + (j - r * L2)];
  }
}

}  // namespace shm
