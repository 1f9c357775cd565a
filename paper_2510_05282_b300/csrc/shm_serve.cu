// Serving: continuous batching of evaluation requests on one GPU.
//
// A scheduler thread owns the device side.  Each iteration it
//  1. retires finished batches (CUDA events, in stream order): requests whose
//     last chunk finished become complete, their latency is recorded and
//     waiters are woken; discarded outputs go back to the pool;
//  2. admits queued requests in arrival order while a request slot is free
//     and the device pool can hold the request's output (first fit);
//  3. if fewer than `inflight_batches` batches are on the GPU, forms the next
//     batch: a round robin over the admitted, unfinished requests taking at
//     most chunk_points points from each and batch_points in total, so large
//     requests progress in slices while newly admitted requests join at once;
//     the chunk descriptors (FP64 chunks first, then all-binary64 FP64
//     chunks, then FP32) go to the device with one copy from pinned memory,
//     and one launch per kind present (k_serve64, k_serve64s, k_serve32)
//     evaluates every tile of those chunks.
// Clients either wait for one ticket (shm_serve_wait) or collect requests in
// completion order (shm_serve_wait_any); the first successful return of
// either for a request records its client-side latency (submit -> the wait
// returning), reported beside the scheduler's submit -> done latency.
// The batch kernels evaluate each tile with the per-point code and tile
// structure of shm_eval's default variant for the dtype (sh_phased.cuh,
// sh_core.cuh, sh_tile.cuh), so a request's rows equal shm_eval's bit for
// bit and do not depend on which other requests shared its batches.  The
// kernels never wait on anything: there is no device-side polling to bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sh_core.cuh"
#include "sh_phased.cuh"
#include "sh_tile.cuh"
#include "shm_internal.h"

namespace shm {

constexpr int kMaxChunksPerBatch = 4096;

struct ServeChunk {
  const void* pts;          // device points, or null: generate from seed
  void* out;                // request output base
  unsigned long long seed;
  long long p0;             // first point of the chunk within its request
  long long tile0;          // first tile of the chunk within the batch
  int n;                    // points in the chunk
  int lmax;
  int dtype;                // SHM_F32 / SHM_F64
  int strict;               // 1: all-binary64 rows (SHM_REQ_STRICT_FP64)
};

// ---------------------------------------------------------------------------
// Counter-based point generator (SplitMix64 of Steele, Lea and Flood 2014 as
// a counter-based source: word(seed, c) = mix(seed + (c + 1) * golden gamma)).
// Point i takes the words c = 4i .. 4i+3:
//   s = v(w0) - 3, t = v(w1) - 3 in [-1, 1), v(w) = the double with bits
//       (w >> 12) | 0x4000000000000000 (in [2, 4), 52 random bits: exact);
//   direction (2s (1 - t^2), 2s 2t, (1 - s^2)(1 + t^2)), whose length is
//       (1 + s^2)(1 + t^2) (rational parametrisations of the circle in both
//       angles), x negated when bit 0 of w3 is 1, z when bit 1 is;
//   radius = the double with bits ((e + 1023) << 52) | (w2 >> 12),
//       e = -10 + ((w3 >> 32) mod 14), i.e. 2^e (1 + m 2^-52);
//   point = direction * radius.
// Only correctly rounded +, -, * (no division, square root or integer to
// float conversion, which on a B300 issue to the narrow FP64-class pipe), and
// _rn intrinsics so that no FMA contraction changes a bit: any binary64
// implementation reproduces the points exactly.

__host__ __device__ inline unsigned long long splitmix_word(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ inline unsigned long long gen_v_bits(unsigned long long w) {
  return (w >> 12) | 0x4000000000000000ull;
}
__host__ __device__ inline unsigned long long gen_radius_bits(unsigned long long w2, unsigned long long w3) {
  const unsigned long long e = (w3 >> 32) % 14ull;  // e + 10
  return ((e + 1013ull) << 52) | (w2 >> 12);
}

__device__ inline void gen_point_dev(unsigned long long seed, long long i, double& x, double& y, double& z) {
  const unsigned long long c = 4ull * (unsigned long long)i;
  const unsigned long long w0 = splitmix_word(seed, c), w1 = splitmix_word(seed, c + 1),
                           w2 = splitmix_word(seed, c + 2), w3 = splitmix_word(seed, c + 3);
  const double s = __dsub_rn(__longlong_as_double((long long)gen_v_bits(w0)), 3.0);
  const double t = __dsub_rn(__longlong_as_double((long long)gen_v_bits(w1)), 3.0);
  const double s2 = __dmul_rn(s, s), t2 = __dmul_rn(t, t);
  const double s_2 = __dadd_rn(s, s), t_2 = __dadd_rn(t, t);
  double dx = __dmul_rn(s_2, __dsub_rn(1.0, t2));
  const double dy = __dmul_rn(s_2, t_2);
  double dz = __dmul_rn(__dsub_rn(1.0, s2), __dadd_rn(1.0, t2));
  if (w3 & 1ull) dx = -dx;
  if (w3 & 2ull) dz = -dz;
  const double radius = __longlong_as_double((long long)gen_radius_bits(w2, w3));
  x = __dmul_rn(dx, radius);
  y = __dmul_rn(dy, radius);
  z = __dmul_rn(dz, radius);
}

// Host twin of gen_point_dev (host code is compiled without FMA contraction
// on x86-64, whose baseline ISA has no FMA; the volatiles keep every
// intermediate a rounded binary64).
static double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}
void gen_point_host(unsigned long long seed, long long i, double* xyz) {
  const unsigned long long c = 4ull * (unsigned long long)i;
  const unsigned long long w0 = splitmix_word(seed, c), w1 = splitmix_word(seed, c + 1),
                           w2 = splitmix_word(seed, c + 2), w3 = splitmix_word(seed, c + 3);
  volatile double s = bits_to_double(gen_v_bits(w0)) - 3.0;
  volatile double t = bits_to_double(gen_v_bits(w1)) - 3.0;
  volatile double s2 = s * s, t2 = t * t;
  volatile double s_2 = s + s, t_2 = t + t;
  volatile double omt = 1.0 - t2, oms = 1.0 - s2, opt = 1.0 + t2;
  volatile double dx = s_2 * omt;
  volatile double dy = s_2 * t_2;
  volatile double dz = oms * opt;
  const double ddx = (w3 & 1ull) ? -dx : dx;
  const double ddz = (w3 & 2ull) ? -dz : dz;
  const double radius = bits_to_double(gen_radius_bits(w2, w3));
  xyz[0] = ddx * radius;
  xyz[1] = dy * radius;
  xyz[2] = ddz * radius;
}

// ---------------------------------------------------------------------------
// Batch kernels: one launch per dtype of the chunks in a batch, each with the
// tile structure of shm_eval's default variant for that dtype, so a request's
// rows are bitwise those shm_eval gives for the same points: FP64 rows are
// the phased hybrid rows in 128-point tiles (96 registers, five CTAs per SM),
// FP32 rows the staged FP32 rows in 64-point tiles.

constexpr int kServeTPB64 = 128;
constexpr int kServeTPB32 = 64;
constexpr int kServeTPB64s = 64;  // all-binary64 rows: the staged-64 tile of shm_eval
constexpr int kServeRS64 = LPhases<SHM_LMAX_CAP>::max_width() | 1;  // staged doubles per row, any lmax
constexpr size_t kServeSmem64 = (size_t)kServeTPB64 * kServeRS64 * 8;
constexpr size_t kServeSmem64s = (size_t)kServeTPB64s * TileShape<SHM_LMAX_CAP>::RS * 8;
constexpr size_t kServeSmem32 = (size_t)kServeTPB32 * TileShape<SHM_LMAX_CAP>::RS * 4;

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// The chunk owning tile t (the last chunk with tile0 <= t), read by thread 0
// into shared memory.
__device__ __forceinline__ void serve_find_chunk(const ServeChunk* __restrict__ chunks, int nchunks, long long t,
                                                 ServeChunk& c) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = nchunks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunks[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    c = chunks[lo];
  }
  __syncthreads();
}

template <int LMAX>
__device__ __forceinline__ void serve_tile64(const ServeChunk& c, long long p, int rows, double* tile) {
  constexpr int L2 = NH<LMAX>::value;
  const bool valid = (int)threadIdx.x < rows;
  double x = 0.0, y = 0.0, z = 1.0;
  if (valid) {
    const long long pi = p + threadIdx.x;
    if (c.pts) {
      const double* P = reinterpret_cast<const double*>(c.pts);
      x = P[3 * pi];
      y = P[3 * pi + 1];
      z = P[3 * pi + 2];
    } else {
      gen_point_dev(c.seed, pi, x, y, z);
    }
  }
  const bool origin = valid && is_origin(x, y, z);
  double xb = 0.0, yb = 0.0, zb = 1.0;
  if (valid && !origin) unit_dir(x, y, z, xb, yb, zb);
  double* dst = reinterpret_cast<double*>(c.out) + p * L2;
  phased_rows<LMAX, kServeTPB64, true>(xb, yb, zb, origin, rows, dst, aligned16(dst), tile);
}

// All-binary64 rows (SHM_REQ_STRICT_FP64): shm_eval's staged-64 tile (the
// m-major rows staged whole, coalesced copy-out) with the output products
// on the integer pipes, bitwise the rows of shm_eval_ex with
// SHM_STRICT_FP64.
template <int LMAX>
__device__ __forceinline__ void serve_tile64s(const ServeChunk& c, long long p, int rows, double* tile) {
  constexpr int L2 = TileShape<LMAX>::L2;
  constexpr int RS = TileShape<LMAX>::RS;
  if ((int)threadIdx.x < rows) {
    const long long pi = p + threadIdx.x;
    double x, y, z;
    if (c.pts) {
      const double* P = reinterpret_cast<const double*>(c.pts);
      x = P[3 * pi];
      y = P[3 * pi + 1];
      z = P[3 * pi + 2];
    } else {
      gen_point_dev(c.seed, pi, x, y, z);
    }
    double* row = tile + threadIdx.x * RS;
    // the output products on the integer pipes (dmul_int), as the default
    // all-binary64 variant of shm_eval: the same bits
    sh_point<LMAX, false, false, kEmuOut>(x, y, z, false, [&](int k, double v) { row[k] = v; });
  }
  __syncthreads();
  double* dst = reinterpret_cast<double*>(c.out) + p * L2;
  copy_out_tile<double, L2, RS, kServeTPB64s>(tile, rows, dst, aligned16(dst));
}

template <int LMAX>
__device__ __forceinline__ void serve_tile32(const ServeChunk& c, long long p, int rows, float* tile) {
  constexpr int L2 = TileShape<LMAX>::L2;
  constexpr int RS = TileShape<LMAX>::RS;
  if ((int)threadIdx.x < rows) {
    const long long pi = p + threadIdx.x;
    float x, y, z;
    if (c.pts) {
      const float* P = reinterpret_cast<const float*>(c.pts);
      x = P[3 * pi];
      y = P[3 * pi + 1];
      z = P[3 * pi + 2];
    } else {
      double dx, dy, dz;
      gen_point_dev(c.seed, pi, dx, dy, dz);
      x = (float)dx;
      y = (float)dy;
      z = (float)dz;
    }
    float* row = tile + threadIdx.x * RS;
    sh_point<LMAX>(x, y, z, false, [&](int k, float v) { row[k] = v; });
  }
  __syncthreads();
  float* dst = reinterpret_cast<float*>(c.out) + p * L2;
  copy_out_tile<float, L2, RS, kServeTPB32>(tile, rows, dst, aligned16(dst));
}

__global__ void __launch_bounds__(kServeTPB64, 5) k_serve64(const ServeChunk* __restrict__ chunks, int nchunks,
                                                            long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tile = reinterpret_cast<double*>(smem_raw);
  __shared__ ServeChunk c;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    serve_find_chunk(chunks, nchunks, t, c);
    const long long p = c.p0 + (t - c.tile0) * kServeTPB64;
    const int rows = (int)min((long long)kServeTPB64, c.p0 + c.n - p);
    switch (c.lmax) {
      case 0: serve_tile64<0>(c, p, rows, tile); break;
      case 1: serve_tile64<1>(c, p, rows, tile); break;
      case 2: serve_tile64<2>(c, p, rows, tile); break;
      case 3: serve_tile64<3>(c, p, rows, tile); break;
      case 4: serve_tile64<4>(c, p, rows, tile); break;
      case 5: serve_tile64<5>(c, p, rows, tile); break;
      case 6: serve_tile64<6>(c, p, rows, tile); break;
      case 7: serve_tile64<7>(c, p, rows, tile); break;
      case 8: serve_tile64<8>(c, p, rows, tile); break;
      default: serve_tile64<9>(c, p, rows, tile); break;
    }
    __syncthreads();  // c and the tile are free
  }
}

__global__ void __launch_bounds__(kServeTPB64s) k_serve64s(const ServeChunk* __restrict__ chunks, int nchunks,
                                                           long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tile = reinterpret_cast<double*>(smem_raw);
  __shared__ ServeChunk c;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    serve_find_chunk(chunks, nchunks, t, c);
    const long long p = c.p0 + (t - c.tile0) * kServeTPB64s;
    const int rows = (int)min((long long)kServeTPB64s, c.p0 + c.n - p);
    switch (c.lmax) {
      case 0: serve_tile64s<0>(c, p, rows, tile); break;
      case 1: serve_tile64s<1>(c, p, rows, tile); break;
      case 2: serve_tile64s<2>(c, p, rows, tile); break;
      case 3: serve_tile64s<3>(c, p, rows, tile); break;
      case 4: serve_tile64s<4>(c, p, rows, tile); break;
      case 5: serve_tile64s<5>(c, p, rows, tile); break;
      case 6: serve_tile64s<6>(c, p, rows, tile); break;
      case 7: serve_tile64s<7>(c, p, rows, tile); break;
      case 8: serve_tile64s<8>(c, p, rows, tile); break;
      default: serve_tile64s<9>(c, p, rows, tile); break;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kServeTPB32) k_serve32(const ServeChunk* __restrict__ chunks, int nchunks,
                                                         long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tile = reinterpret_cast<float*>(smem_raw);
  __shared__ ServeChunk c;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    serve_find_chunk(chunks, nchunks, t, c);
    const long long p = c.p0 + (t - c.tile0) * kServeTPB32;
    const int rows = (int)min((long long)kServeTPB32, c.p0 + c.n - p);
    switch (c.lmax) {
      case 0: serve_tile32<0>(c, p, rows, tile); break;
      case 1: serve_tile32<1>(c, p, rows, tile); break;
      case 2: serve_tile32<2>(c, p, rows, tile); break;
      case 3: serve_tile32<3>(c, p, rows, tile); break;
      case 4: serve_tile32<4>(c, p, rows, tile); break;
      case 5: serve_tile32<5>(c, p, rows, tile); break;
      case 6: serve_tile32<6>(c, p, rows, tile); break;
      case 7: serve_tile32<7>(c, p, rows, tile); break;
      case 8: serve_tile32<8>(c, p, rows, tile); break;
      default: serve_tile32<9>(c, p, rows, tile); break;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side.

using Clock = std::chrono::steady_clock;

struct PoolAllocator {
  size_t size = 0, in_use = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t s) {
    size = s;
    free_.clear();
    free_[0] = s;
  }
  bool alloc(size_t len, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        *off = it->first;
        const size_t rest = it->second - len;
        const size_t noff = it->first + len;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        in_use += len;
        peak = std::max(peak, in_use);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t len) {
    in_use -= len;
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

enum ReqState { kQueued, kActive, kDone };

struct Request {
  shm_request r;
  ReqState state = kQueued;
  size_t L2 = 0, es = 0, out_bytes = 0, pool_off = 0;
  void* out = nullptr;
  int64_t next_point = 0, done_points = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool failed = false;     // a batch holding part of it failed to launch or run
  bool collected = false;  // a wait has returned it (client latency recorded)
};

struct Batch {
  cudaEvent_t start = nullptr, end = nullptr;
  ServeChunk* host = nullptr;  // pinned
  ServeChunk* dev = nullptr;
  std::vector<std::pair<uint64_t, int64_t>> parts;  // (ticket, points)
  bool inflight = false;
  bool failed = false;
  uint64_t seq = 0;
};

}  // namespace shm

struct shm_server {
  shm_serve_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  char* pool = nullptr;
  shm::PoolAllocator alloc;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;  // admitted and not yet fully scheduled, round-robin order
  size_t rr = 0;
  std::unordered_map<uint64_t, shm::Request> reqs;
  std::vector<shm::Batch> batches;
  uint64_t batch_seq = 0, next_retire = 0;
  uint64_t next_ticket = 1;
  int slots_used = 0;
  std::thread sched;
  bool stop = false;
  shm::Clock::time_point t0;
  // stats
  uint64_t submitted = 0, rejected = 0, admitted = 0, completed = 0, nbatches = 0;
  double harmonics = 0, busy_ms = 0;
  std::vector<double> lat;         // submit -> the scheduler seeing the request done
  std::vector<double> lat_client;  // submit -> a wait returning the request to the client
  std::deque<uint64_t> done_q;     // completed, not yet collected (shm_serve_wait_any)
  std::string thread_error;
  int grid64 = 0, grid64s = 0, grid32 = 0;  // resident CTAs of the batch kernels on the device

  double now_ms() const { return std::chrono::duration<double, std::milli>(shm::Clock::now() - t0).count(); }
  void run();
  bool retire_locked();
  bool admit_locked();
  bool launch_locked();
};

namespace shm {
namespace {
size_t round256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace
}  // namespace shm

bool shm_server::retire_locked() {
  bool any = false;
  for (;;) {
    // batches retire in launch order (one stream)
    shm::Batch* b = nullptr;
    for (auto& x : batches)
      if (x.inflight && x.seq == next_retire) b = &x;
    if (!b) break;
    const cudaError_t q = b->failed ? cudaSuccess : cudaEventQuery(b->end);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) {
      thread_error = std::string("batch failed: ") + cudaGetErrorString(q);
      cudaGetLastError();
      b->failed = true;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->start, b->end) == cudaSuccess) busy_ms += ms;
    else cudaGetLastError();
    const double t = now_ms();
    for (auto& pr : b->parts) {
      auto it = reqs.find(pr.first);
      if (it == reqs.end()) continue;
      shm::Request& R = it->second;
      R.done_points += pr.second;
      if (b->failed) R.failed = true;
      if (R.done_points == R.r.n) {
        R.state = shm::kDone;
        R.t_done = t;
        lat.push_back(R.t_done - R.t_submit);
        ++completed;
        harmonics += (double)R.r.n * (double)R.L2;
        --slots_used;
        if (R.r.flags & SHM_REQ_DISCARD) {
          alloc.release(R.pool_off, R.out_bytes);
          reqs.erase(it);
        } else {
          done_q.push_back(pr.first);
        }
      }
    }
    b->parts.clear();
    b->inflight = false;
    b->failed = false;
    ++next_retire;
    any = true;
  }
  if (any) cv_done.notify_all();
  return any;
}

bool shm_server::admit_locked() {
  bool any = false;
  while (!queue.empty() && slots_used < cfg.max_slots) {
    auto it = reqs.find(queue.front());
    if (it == reqs.end()) {
      queue.pop_front();
      continue;
    }
    shm::Request& R = it->second;
    size_t off = 0;
    if (!alloc.alloc(R.out_bytes, &off)) break;  // head of line waits for memory
    R.pool_off = off;
    R.out = pool + off;
    R.state = shm::kActive;
    R.t_admit = now_ms();
    ++admitted;
    ++slots_used;
    active.push_back(queue.front());
    queue.pop_front();
    any = true;
  }
  return any;
}

bool shm_server::launch_locked() {
  if (active.empty()) return false;
  shm::NvtxRange nvtx_range("shm_serve_batch");
  shm::Batch* b = nullptr;
  int inflight = 0;
  for (auto& x : batches) {
    if (x.inflight) ++inflight;
    else if (!b) b = &x;
  }
  if (!b) return false;
  int64_t budget = cfg.batch_points;
  int nch = 0;
  const size_t na = active.size();
  size_t visited = 0;
  if (rr >= na) rr = 0;
  size_t i = rr;
  std::vector<shm::ServeChunk> picked;
  while (budget > 0 && nch < shm::kMaxChunksPerBatch && visited < na) {
    shm::Request& R = reqs[active[i]];
    const int64_t left = R.r.n - R.next_point;
    if (left > 0) {
      const int64_t take = std::min<int64_t>({left, cfg.chunk_points, budget});
      shm::ServeChunk c;
      c.pts = R.r.points;
      c.out = R.out;
      c.seed = R.r.seed;
      c.p0 = R.next_point;
      c.tile0 = 0;
      c.n = (int)take;
      c.lmax = R.r.lmax;
      c.dtype = (int)R.r.dtype;
      c.strict = (R.r.dtype == SHM_F64 && (R.r.flags & SHM_REQ_STRICT_FP64)) ? 1 : 0;
      picked.push_back(c);
      ++nch;
      R.next_point += take;
      budget -= take;
      b->parts.emplace_back(active[i], take);
    }
    ++visited;
    i = (i + 1) % na;
  }
  rr = i;
  // drop fully scheduled requests from the round robin (they stay admitted until done)
  active.erase(std::remove_if(active.begin(), active.end(),
                              [&](uint64_t t) { return reqs[t].next_point >= reqs[t].r.n; }),
               active.end());
  if (nch == 0) return false;
  // FP64 chunks first, then all-binary64 FP64 chunks, then FP32; tiles
  // numbered per kind in its kernel's tile size
  int k = 0;
  long long tiles64 = 0, tiles64s = 0, tiles32 = 0;
  for (const auto& c : picked)
    if (c.dtype == SHM_F64 && !c.strict) {
      b->host[k] = c;
      b->host[k].tile0 = tiles64;
      tiles64 += (c.n + shm::kServeTPB64 - 1) / shm::kServeTPB64;
      ++k;
    }
  const int n64 = k;
  for (const auto& c : picked)
    if (c.dtype == SHM_F64 && c.strict) {
      b->host[k] = c;
      b->host[k].tile0 = tiles64s;
      tiles64s += (c.n + shm::kServeTPB64s - 1) / shm::kServeTPB64s;
      ++k;
    }
  const int n64s = k - n64;
  for (const auto& c : picked)
    if (c.dtype != SHM_F64) {
      b->host[k] = c;
      b->host[k].tile0 = tiles32;
      tiles32 += (c.n + shm::kServeTPB32 - 1) / shm::kServeTPB32;
      ++k;
    }
  const int n32 = k - n64 - n64s;
  cudaError_t e = cudaMemcpyAsync(b->dev, b->host, sizeof(shm::ServeChunk) * nch, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->start, stream);
  if (e == cudaSuccess && n64 > 0) {
    const long long g = std::max(1LL, std::min<long long>(tiles64, grid64));
    shm::k_serve64<<<(unsigned)g, shm::kServeTPB64, shm::kServeSmem64, stream>>>(b->dev, n64, tiles64);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n64s > 0) {
    const long long g = std::max(1LL, std::min<long long>(tiles64s, grid64s));
    shm::k_serve64s<<<(unsigned)g, shm::kServeTPB64s, shm::kServeSmem64s, stream>>>(b->dev + n64, n64s, tiles64s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n32 > 0) {
    const long long g = std::max(1LL, std::min<long long>(tiles32, grid32));
    shm::k_serve32<<<(unsigned)g, shm::kServeTPB32, shm::kServeSmem32, stream>>>(b->dev + n64 + n64s, n32,
                                                                                 tiles32);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->end, stream);
  if (e != cudaSuccess) {
    thread_error = std::string("batch launch failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    b->failed = true;
  }
  b->inflight = true;
  b->seq = batch_seq++;
  ++nbatches;
  return true;
}

void shm_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    bool progress = retire_locked();
    if (!stop) progress |= admit_locked();  // after destroy starts, only admitted work drains
    progress |= launch_locked();
    bool inflight = false;
    for (auto& b : batches) inflight |= b.inflight;
    if (stop && !inflight && active.empty()) break;  // queued, unadmitted requests are dropped
    if (!progress) {
      if (inflight)
        cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

extern "C" void shm_serve_generated_point(uint64_t seed, int64_t i, double xyz[3]) {
  shm::gen_point_host(seed, i, xyz);
}

extern "C" shm_status shm_serve_create(const shm_serve_config* cfg, shm_server** server) {
  using namespace shm;
  NvtxRange nvtx_range("shm_serve_create");
  clear_error();
  if (!cfg || !server) return fail(SHM_EINVAL, "null argument");
  if (cfg->pool_bytes < 256 || cfg->max_slots < 1 || cfg->queue_capacity < 1 || cfg->batch_points < 1 ||
      cfg->chunk_points < 1 || cfg->chunk_points > (1 << 30) || cfg->inflight_batches < 1 || cfg->inflight_batches > 8)
    return fail(SHM_EINVAL, "bad serve config");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceCount");
  if (cfg->device < 0 || cfg->device >= ndev) return fail(SHM_EINVAL, "device ordinal out of range");
  auto* S = new shm_server();
  S->cfg = *cfg;
  S->device = cfg->device;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  auto cleanup = [&](shm_status st) {
    for (auto& b : S->batches) {
      if (b.start) cudaEventDestroy(b.start);
      if (b.end) cudaEventDestroy(b.end);
      if (b.host) cudaFreeHost(b.host);
      if (b.dev) cudaFree(b.dev);
    }
    if (S->pool) cudaFree(S->pool);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    cudaSetDevice(prev);
    return st;
  };
  if ((e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaStreamCreateWithFlags"));
  if ((e = dev_malloc((void**)&S->pool, cfg->pool_bytes, "serve_pool")) != cudaSuccess)
    return cleanup(fail_alloc(e, "serve_pool",
                              "cannot allocate the serve pool of " + std::to_string(cfg->pool_bytes) + " bytes"));
  S->alloc.init(cfg->pool_bytes);
  S->batches.resize(cfg->inflight_batches);
  for (auto& b : S->batches) {
    if ((e = cudaEventCreate(&b.start)) != cudaSuccess || (e = cudaEventCreate(&b.end)) != cudaSuccess)
      return cleanup(fail_cuda(e, "cudaEventCreate"));
    if ((e = pinned_malloc((void**)&b.host, sizeof(ServeChunk) * kMaxChunksPerBatch, "serve_pinned")) != cudaSuccess)
      return cleanup(fail_alloc(e, "serve_pinned", "pinned batch descriptors"));
    if ((e = dev_malloc((void**)&b.dev, sizeof(ServeChunk) * kMaxChunksPerBatch, "serve_batch")) != cudaSuccess)
      return cleanup(fail_alloc(e, "serve_batch", "device batch descriptors"));
  }
  if ((e = cudaFuncSetAttribute(k_serve64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kServeSmem64)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(k_serve64s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kServeSmem64s)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(k_serve32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kServeSmem32)) !=
          cudaSuccess)
    return cleanup(fail_cuda(e, "cudaFuncSetAttribute(k_serve)"));
  int b64 = 0, b64s = 0, b32 = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_serve64, kServeTPB64, kServeSmem64)) !=
          cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64s, k_serve64s, kServeTPB64s, kServeSmem64s)) !=
          cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_serve32, kServeTPB32, kServeSmem32)) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_serve)"));
  S->grid64 = sm_count(S->device) * std::max(b64, 1);
  S->grid64s = sm_count(S->device) * std::max(b64s, 1);
  S->grid32 = sm_count(S->device) * std::max(b32, 1);
  S->t0 = Clock::now();
  cudaSetDevice(prev);
  S->sched = std::thread([S] { S->run(); });
  *server = S;
  return SHM_OK;
}

extern "C" shm_status shm_serve_submit(shm_server* S, const shm_request* req, uint64_t* ticket) {
  using namespace shm;
  NvtxRange nvtx_range("shm_serve_submit");
  clear_error();
  if (!S || !req || !ticket) return fail(SHM_EINVAL, "null argument");
  if (req->n < 1) return fail(SHM_EINVAL, "n must be >= 1");
  if (req->lmax < 0 || req->lmax > SHM_LMAX_CAP) return fail(SHM_EINVAL, "lmax must be in 0..9");
  if (req->dtype != SHM_F32 && req->dtype != SHM_F64) return fail(SHM_EINVAL, "dtype must be SHM_F32 or SHM_F64");
  if (req->flags & ~(SHM_REQ_DISCARD | SHM_REQ_STRICT_FP64)) return fail(SHM_EINVAL, "unknown request flags");
  Request R;
  R.r = *req;
  R.es = req->dtype == SHM_F64 ? 8 : 4;
  R.L2 = (size_t)(req->lmax + 1) * (req->lmax + 1);
  if (req->n > (int64_t)1 << 40) return fail(SHM_EINVAL, "n too large");
  R.out_bytes = round256((size_t)req->n * R.L2 * R.es);
  if (R.out_bytes > S->cfg.pool_bytes) return fail(SHM_EINVAL, "request output can never fit the serve pool");
  if (req->points) {
    if (!aligned(req->points, R.es)) return fail(SHM_EINVAL, "points must be aligned to the element size");
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != S->device) cudaSetDevice(S->device);
    const shm_status st = check_device_range(req->points, (size_t)req->n * 3 * R.es, "points");
    if (prev != S->device) cudaSetDevice(prev);
    if (st != SHM_OK) return st;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->submitted;
    if ((int)S->queue.size() >= S->cfg.queue_capacity) {
      ++S->rejected;
      return fail(SHM_EBUSY, "serve queue full");
    }
    R.t_submit = S->now_ms();
    const uint64_t t = S->next_ticket++;
    S->reqs.emplace(t, R);
    S->queue.push_back(t);
    *ticket = t;
  }
  S->cv_work.notify_one();
  return SHM_OK;
}

static void fill_result(const shm::Request& R, shm_result* res) {
  res->status = R.state != shm::kDone ? SHM_ETIMEOUT : (R.failed ? SHM_ECUDA : SHM_OK);
  res->out = (R.r.flags & SHM_REQ_DISCARD) ? nullptr : R.out;
  res->n = R.r.n;
  res->lmax = R.r.lmax;
  res->dtype = R.r.dtype;
  res->t_submit_ms = R.t_submit;
  res->t_admit_ms = R.t_admit;
  res->t_done_ms = R.t_done;
}

// Records the client-side latency of a completed request the first time a
// wait returns it (caller holds S->mu).
static void collect_locked(shm_server* S, shm::Request& R) {
  if (R.collected) return;
  R.collected = true;
  S->lat_client.push_back(S->now_ms() - R.t_submit);
}

extern "C" shm_status shm_serve_wait(shm_server* S, uint64_t ticket, int timeout_ms, shm_result* res) {
  using namespace shm;
  NvtxRange nvtx_range("shm_serve_wait");
  clear_error();
  if (!S || !res) return fail(SHM_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto done = [&] {
    auto it = S->reqs.find(ticket);
    return it == S->reqs.end() || it->second.state == kDone;
  };
  if (timeout_ms < 0)
    S->cv_done.wait(lk, done);
  else
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(SHM_ENOTFOUND, "unknown or released ticket");
  fill_result(it->second, res);
  if (it->second.state != kDone) return fail(SHM_ETIMEOUT, "request not complete");
  collect_locked(S, it->second);
  if (it->second.failed) return fail(SHM_ECUDA, "a batch holding this request failed: " + S->thread_error);
  return SHM_OK;
}

extern "C" shm_status shm_serve_wait_any(shm_server* S, int timeout_ms, uint64_t* ticket, shm_result* res) {
  using namespace shm;
  NvtxRange nvtx_range("shm_serve_wait_any");
  clear_error();
  if (!S || !ticket || !res) return fail(SHM_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  // the oldest completed request no wait has returned yet (released or
  // already collected tickets are skipped)
  auto next = [&]() -> shm::Request* {
    while (!S->done_q.empty()) {
      auto it = S->reqs.find(S->done_q.front());
      if (it != S->reqs.end() && !it->second.collected) return &it->second;
      S->done_q.pop_front();
    }
    return nullptr;
  };
  auto ready = [&] { return next() != nullptr; };
  if (timeout_ms < 0)
    S->cv_done.wait(lk, ready);
  else
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  shm::Request* R = next();
  if (!R) return fail(SHM_ETIMEOUT, "no request completed in time");
  *ticket = S->done_q.front();
  S->done_q.pop_front();
  fill_result(*R, res);
  collect_locked(S, *R);
  if (R->failed) return fail(SHM_ECUDA, "a batch holding this request failed: " + S->thread_error);
  return SHM_OK;
}

extern "C" shm_status shm_serve_release(shm_server* S, uint64_t ticket) {
  using namespace shm;
  NvtxRange nvtx_range("shm_serve_release");
  clear_error();
  if (!S) return fail(SHM_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(SHM_ENOTFOUND, "unknown or released ticket");
  if (it->second.state != kDone) return fail(SHM_EBUSY, "request not complete");
  S->alloc.release(it->second.pool_off, it->second.out_bytes);
  S->reqs.erase(it);
  S->cv_work.notify_one();
  return SHM_OK;
}

extern "C" shm_status shm_serve_stats_get(shm_server* S, shm_serve_stats* st) {
  using namespace shm;
  clear_error();
  if (!S || !st) return fail(SHM_EINVAL, "null argument");
  std::vector<double> lat, latc;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->rejected = S->rejected;
    st->admitted = S->admitted;
    st->completed = S->completed;
    st->batches = S->nbatches;
    st->queued_now = S->queue.size();
    st->active_now = (uint64_t)S->slots_used;
    st->harmonics_done = S->harmonics;
    st->busy_ms = S->busy_ms;
    st->pool_bytes = S->alloc.size;
    st->pool_in_use = S->alloc.in_use;
    st->pool_peak = S->alloc.peak;
    lat = S->lat;
    latc = S->lat_client;
    if (!S->thread_error.empty()) return fail(SHM_ECUDA, S->thread_error);
  }
  auto pct = [](std::vector<double>& v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  st->lat_p50_ms = pct(lat, 0.50);
  st->lat_p99_ms = pct(lat, 0.99);
  st->lat_max_ms = lat.empty() ? 0.0 : *std::max_element(lat.begin(), lat.end());
  st->collected = latc.size();
  st->client_lat_p50_ms = pct(latc, 0.50);
  st->client_lat_p99_ms = pct(latc, 0.99);
  st->client_lat_max_ms = latc.empty() ? 0.0 : *std::max_element(latc.begin(), latc.end());
  return SHM_OK;
}

extern "C" shm_status shm_serve_stats_reset(shm_server* S) {
  using namespace shm;
  clear_error();
  if (!S) return fail(SHM_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  S->submitted = S->rejected = S->admitted = S->completed = S->nbatches = 0;
  S->harmonics = S->busy_ms = 0;
  S->lat.clear();
  S->lat_client.clear();
  S->alloc.peak = S->alloc.in_use;
  return SHM_OK;
}

extern "C" shm_status shm_serve_destroy(shm_server* S) {
  using namespace shm;
  NvtxRange nvtx_range("shm_serve_destroy");
  clear_error();
  if (!S) return fail(SHM_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->sched.joinable()) S->sched.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  cudaStreamSynchronize(S->stream);
  for (auto& b : S->batches) {
    cudaEventDestroy(b.start);
    cudaEventDestroy(b.end);
    cudaFreeHost(b.host);
    cudaFree(b.dev);
  }
  cudaFree(S->pool);
  cudaStreamDestroy(S->stream);
  cudaGetLastError();
  cudaSetDevice(prev);
  delete S;
  return SHM_OK;
}
