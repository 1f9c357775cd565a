/*
 * shm.h -- C ABI of libshm: spherical harmonics (real, complex, spin-1/2 spinor) on a B300.
 *
 * The operation is the one defined in "SHarmonic: A fast and accurate
 * implementation of spherical harmonics for electronic-structure
 * calculations" (arXiv 2510.05282):
 *   - R_l^m, Sec. II Eq. 6 (from the complex Y_l^m of Eq. 5, Condon-Shortley
 *     sign included there), which comes out as
 *       R_l^0  = N_l^0 P_l^0(cos t),
 *       R_l^m  = sqrt2 N_l^m P_l^m(cos t) cos(m p),   m > 0,
 *       R_l^-m = sqrt2 N_l^m P_l^m(cos t) sin(m p),   m > 0,
 *     with P_l^m free of any further sign (this matches the App. C formulas
 *     and the App. D reference values);
 *   - evaluated in normalised Cartesian coordinates x/r, y/r, z/r
 *     (Sec. II Eq. 8: the harmonics are polynomials there);
 *   - at r = 0 every harmonic is 0 except R_0^0 = 1/sqrt(4 pi) (Sec. II);
 *   - l is limited to 9, as in the paper (Sec. III), except for the real rows
 *     of shm_eval, which extend the same recurrence to l = 16 (SHM_LMAX_EXT).
 *
 * Conventions shared by every entry point:
 *   - Pointers named "device" must point to device memory of the current CUDA
 *     device; pointers named "host" to host memory.  Nothing is copied between
 *     host and device unless stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued asynchronously on it; argument errors are
 *     detected synchronously, before anything is launched, and nothing is
 *     launched when an error is returned.
 *   - Output layout: row-major [n][(lmax+1)^2]; column k = l*l + l + m, m from
 *     -l to l (the App. C order).
 *   - A point with a NaN or infinite coordinate (or angle) gets NaN in every
 *     value except the constant l = 0 ones (R_0^0, Y_0^0, the l = 0
 *     spinors); imaginary parts that are zero by construction (complex
 *     m = 0) may stay 0.  The other points of the call are unaffected.
 *   - shm_eval, shm_eval_ex, shm_eval_complex, shm_eval_spinor and
 *     shm_eval_angles allocate nothing and only enqueue kernels on `stream`,
 *     so they can be captured into a CUDA graph once a call of the same
 *     (lmax, dtype) outside the capture has done the one-time per-device
 *     kernel set-up.
 *   - shm_last_error() returns a thread-local text for the last failure.
 */
#ifndef SHM_H
#define SHM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SHM_F32 = 0, /* float in, float out: FP32 arithmetic (FP64 for 1/r when r < 1e-2, float-float for the
                  m = 0, 1 recurrences) */
  SHM_F64 = 1  /* double in, double out.  Default arithmetic for l <= 9: binary64 for 1/r and the m = 0, 1
                  columns, float-float (two FP32 numbers, a ~48-bit significand, on the FP32 pipe) for the
                  m >= 2 columns, converted to binary64 once per value; within 1e-13 of the l-shell norm
                  sqrt((2l+1)/4pi) (measured <= 5.4e-14 at l = 9, all-binary64 rows: 1.4e-14).  With the
                  flag SHM_STRICT_FP64 every operation is binary64 (IEEE double add, multiply, fused
                  multiply-add; CUDA's binary64 rsqrt and sincos).  Rows above l = 9 are always
                  all-binary64. */
} shm_dtype;

typedef enum {
  SHM_OK = 0,
  SHM_EINVAL = 1,       /* bad argument (null/misaligned pointer, lmax, dtype, size) */
  SHM_ENOMEM = 2,       /* device or pinned memory exhausted */
  SHM_ECUDA = 3,        /* a CUDA call failed; shm_last_error() has its text */
  SHM_EBUSY = 4,        /* serving: request not admitted (queue or pool full) */
  SHM_ETIMEOUT = 5,     /* serving: wait expired / device wait gave up */
  SHM_EUNSUPPORTED = 6, /* valid request this build cannot do */
  SHM_ENOTFOUND = 7     /* serving: unknown ticket */
} shm_status;

#define SHM_LMAX_CAP 9  /* the paper's formulas stop at l = 9 (Sec. III) */
#define SHM_LMAX_EXT 16 /* shm_eval, shm_eval_ex, shm_eval_host and the tuner accept lmax up to this:
                           the recurrence behind the rows has no l limit (the paper's conclusion
                           points to recurrences for l > 9); l > 9 rows are all-FP64 for SHM_F64 */

/* shm_eval_ex flags */
#define SHM_NORMALIZED_INPUT 0x1u /* points are already x/r, y/r, z/r: skip the r work */
#define SHM_STRICT_FP64 0x2u      /* SHM_F64 only (ignored for SHM_F32): compute every value in binary64
                                     arithmetic -- no float-float -- with the same formulas (Sec. II
                                     Eq. 5-6 via the recurrence of the rows), as the paper does (Sec. IV:
                                     machine precision in double).  Accepted by shm_eval_ex,
                                     shm_eval_host_ex, shm_eval_complex, shm_eval_spinor,
                                     shm_eval_angles_ex and the tuner (shm_autotune_ex).  The all-binary64
                                     rows are bound by the FP64 pipe (about 2.4 FP64 instructions per
                                     harmonic at l = 9, against 0.74 for the default rows). */

/* Number of harmonics for lmax: (lmax+1)^2 (0 for lmax outside 0..16). */
int shm_num_harmonics(int lmax);

/*
 * shm_eval -- all R_l^m, 0 <= l <= lmax, at n points, in the default
 * arithmetic of the dtype (see shm_dtype: for SHM_F64 the hybrid
 * binary64/float-float rows at l <= 9; shm_eval_ex with SHM_STRICT_FP64 for
 * all-binary64 rows).
 *   points : device, [n][3] x, y, z (AoS) relative to the centre, element type
 *            per dtype, aligned to its element size.
 *   n      : number of points, >= 0 (0: returns SHM_OK, launches nothing).
 *   lmax   : 0..16 (SHM_LMAX_EXT; 0..9 is the paper's range).
 *   out    : device, [n][(lmax+1)^2] of dtype, aligned to its element size
 *            (16-byte alignment enables the vector store path).  Must not
 *            overlap points.
 * Caller owns both buffers; nothing is allocated.
 * Errors: SHM_EINVAL (null or misaligned pointer, lmax outside 0..16, n < 0,
 * bad dtype), SHM_ECUDA (launch failed).
 */
shm_status shm_eval(const void* points, int64_t n, int lmax, shm_dtype dtype, void* out, void* stream);

/* shm_eval with flags (SHM_NORMALIZED_INPUT, SHM_STRICT_FP64). Unknown flag bits: SHM_EINVAL. */
shm_status shm_eval_ex(const void* points, int64_t n, int lmax, shm_dtype dtype, unsigned flags,
                       void* out, void* stream);

/*
 * shm_eval_host -- shm_eval on HOST buffers, end to end: the points are copied
 * to the device, evaluated and the rows copied back, in chunks that flow
 * through a caller-provided device workspace, double-buffered on two internal
 * streams so that host->device copies, kernels and device->host copies of
 * consecutive chunks overlap.
 *   points_host : host, [n][3] of dtype (pinned memory gives full copy speed).
 *   out_host    : host, [n][(lmax+1)^2] of dtype.
 *   workspace   : device, >= shm_eval_host_workspace_size(lmax, dtype, 1)
 *                 bytes; larger workspaces give larger chunks.
 *   stream      : the work is ordered after prior work on `stream`, and
 *                 later work on `stream` waits for it; the call returns
 *                 once everything is enqueued (synchronise `stream` before
 *                 reading out_host).  The internal streams are created once
 *                 per device and kept until exit.
 * Nothing is allocated per call.  Errors: as shm_eval, plus SHM_EINVAL for a
 * workspace smaller than one point's worth.
 */
shm_status shm_eval_host(const void* points_host, int64_t n, int lmax, shm_dtype dtype, void* out_host,
                         void* workspace, size_t workspace_bytes, void* stream);

/* shm_eval_host with flags (SHM_NORMALIZED_INPUT, SHM_STRICT_FP64); unknown bits: SHM_EINVAL. */
shm_status shm_eval_host_ex(const void* points_host, int64_t n, int lmax, shm_dtype dtype, unsigned flags,
                            void* out_host, void* workspace, size_t workspace_bytes, void* stream);

/* Device workspace bytes shm_eval_host needs for chunks of `chunk_points` points. */
size_t shm_eval_host_workspace_size(int lmax, shm_dtype dtype, int64_t chunk_points);

/*
 * shm_autotune -- time every launch variant of the evaluator (store path x
 * CTA size) for (lmax, dtype) on n_probe synthetic points and keep the
 * fastest for later shm_eval / shm_eval_host calls in this process.  When
 * the environment variable SHM_TUNE_CACHE names a file, the choice is also
 * appended there, and every process reads that file before its first
 * evaluation.  Unlike shm_eval this call allocates (and frees) its probe
 * buffers with cudaMalloc and synchronises the device, so it must not be
 * called during stream capture.  best_ms (may be NULL) receives the fastest
 * time.  Errors: SHM_EINVAL (lmax, dtype, n_probe <= 0), SHM_ENOMEM, SHM_ECUDA.
 */
shm_status shm_autotune(int lmax, shm_dtype dtype, int64_t n_probe, double* best_ms);

/* shm_autotune for the rows a flag selects: with SHM_STRICT_FP64 (SHM_F64)
 * only the all-binary64 variants are timed and the choice is kept for calls
 * that pass that flag (a separate entry of the cache file).  Other bits:
 * SHM_EINVAL. */
shm_status shm_autotune_ex(int lmax, shm_dtype dtype, unsigned flags, int64_t n_probe, double* best_ms);

/* Text naming the launch variant shm_eval uses for (lmax, dtype) (always succeeds
 * for valid arguments; "" otherwise); _ex: for calls with these flags
 * (SHM_STRICT_FP64 selects the all-binary64 choice). */
const char* shm_eval_variant(int lmax, shm_dtype dtype);
const char* shm_eval_variant_ex(int lmax, shm_dtype dtype, unsigned flags);

/* Number of launch variants, and pinning one of them (0 .. count-1) for
 * (lmax, dtype) in this process; variant -1 restores the default choice.
 * _ex with SHM_STRICT_FP64 pins the choice of strict calls and accepts only
 * all-binary64 variants (staged-*, direct-*, phased-64/128, rows-tma-*; the
 * rows-tma-emu-* ones compute part of their binary64 products on the integer
 * pipes, bitwise the FP64 instructions' results, see shm_probe_dmul).
 * Errors: SHM_EINVAL. */
int shm_eval_variant_count(void);
shm_status shm_eval_set_variant(int lmax, shm_dtype dtype, int variant);
shm_status shm_eval_set_variant_ex(int lmax, shm_dtype dtype, unsigned flags, int variant);

/* ------------------------------------------------------------------------
 * Fused non-local projectors.  Sec. I of the paper motivates the method by
 * the projectors of pseudopotential and PAW methods, which need Y_lm at every
 * grid point of each atom's sphere; this entry point builds them directly:
 *
 *   out[out_offsets[a] + (p - point_offsets[a]) * (L_a+1)^2 + l*l + l + m]
 *       = f_{s,l}(|d|) * R_l^m(d / |d|)
 *
 * for every atom a (species s = atom_species[a], L_a = species_lmax[s]) and
 * every sphere point p of a, where grid point g = point_index[p] =
 * (i*ng + j)*ng + k sits at (i, j, k)*h, d = minimum image of (grid point -
 * atom_pos[a]) in the cubic periodic box of side `box` (each component
 * d_c -= box * rint(d_c / box)), and f_{s,l} is read from its table on the
 * log grid r_i = r_min * exp(i * dlog), i < n_rad, by 4-point Lagrange
 * interpolation at t = ln(|d| / r_min) / dlog clamped to [0, n_rad-1] (t = 0
 * for |d| = 0, where R follows the r = 0 convention), through the nodes
 * i0..i0+3, i0 = clamp(floor(t) - 1, 0, n_rad - 4).
 * ------------------------------------------------------------------------ */
#define SHM_PROJ_MAX_SPECIES 64

typedef struct {
  int64_t n_atoms;               /* 0 <= n_atoms < 2^31 */
  const double* atom_pos;        /* device [n_atoms][3], bohr */
  const int32_t* atom_species;   /* device [n_atoms], 0 <= s < n_species */
  int32_t n_species;             /* 1..SHM_PROJ_MAX_SPECIES */
  const int32_t* species_lmax;   /* HOST [n_species], each 0..9 */
  const double* radial;          /* device [n_species][radial_lstride][n_rad] */
  int32_t radial_lstride;        /* 1 + max species lmax .. 64 */
  int32_t n_rad;                 /* 4 .. 2^26 */
  double r_min;                  /* > 0 */
  double dlog;                   /* > 0 */
  double box;                    /* > 0, = ng * h */
  int32_t ng;                    /* 1..1290 (ng^3 < 2^31) */
  double h;                      /* > 0 */
  const int64_t* point_offsets;  /* device [n_atoms+1], non-decreasing, [0] = 0 */
  const int32_t* point_index;    /* device [n_points], each in [0, ng^3) */
  const int64_t* out_offsets;    /* device [n_atoms+1], out_offsets[a+1] - out_offsets[a] = n_a (L_a+1)^2 */
  int64_t n_points;              /* host copy of point_offsets[n_atoms], <= 2^40 */
  int64_t n_values;              /* host copy of out_offsets[n_atoms], <= 2^44 */
} shm_proj_problem;

/* Device workspace bytes shm_projectors needs for this problem and dtype; 0
 * for a problem shm_projectors would reject on its host-side checks (the
 * reason is then in shm_last_error()).  Host-side limits: n_rad 4..2^26,
 * radial_lstride (1 + max species lmax)..64, n_points <= 2^40, n_values <=
 * 2^44, n_atoms < 2^31 -- so no size product can overflow. */
size_t shm_projectors_workspace_size(const shm_proj_problem* prob, shm_dtype dtype);

/*
 * shm_projectors -- the fused projector values: shm_projectors_prepare then
 * shm_projectors_run on `stream` (the set-up's two launches, then the
 * persistent launch).
 *   dtype     : SHM_F64 (double out; binary64 for the displacement, r^2, 1/r
 *               and the unit vector, float-float (two FP32 numbers, ~48-bit
 *               significand) for the log-grid index, the radial cubic and
 *               the rows of lmax <= 4, hybrid rows above: within 1e-13 of
 *               F_sl sqrt((2l+1)/4pi); all-binary64 with shm_projectors_ex
 *               and SHM_STRICT_FP64; the 4-point Lagrange interpolation
 *               evaluated as the interval's cubic in the fractional index,
 *               the same polynomial up to rounding) or
 *               SHM_F32 (FP32 arithmetic on FP32 interval cubics of the
 *               tables, float out; grid displacements are formed exactly
 *               before rounding to float, 1/r in FP64 for |d| < 1e-2).
 *   out       : device [n_values] of dtype, caller-owned.
 *   workspace : device scratch of >= shm_projectors_workspace_size() bytes,
 *               caller-owned; it holds the per-atom tile table and atom
 *               order, one 32-byte descriptor per tile (n_points / 128 +
 *               n_atoms + 1 of them), an error word, the interval cubics of
 *               the radial tables (16 bytes per table node for SHM_F32, 32
 *               for SHM_F64) and the displacement tables (per atom, axis and
 *               grid coordinate: 3 ng values of dtype per atom).  One
 *               workspace must not be shared by calls that overlap on the GPU.
 * The kernel checks every index it reads through (species, grid index, table
 * stencil, output range) against the problem's sizes; an inconsistent problem
 * sets bits of the workspace error word (see shm_projectors_check) and the
 * offending rows are skipped -- no access goes out of bounds.
 * Errors (synchronous): SHM_EINVAL for bad scalars, null pointers, host
 * species_lmax out of range, or a workspace that is too small; SHM_ECUDA.
 */
shm_status shm_projectors(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* workspace,
                          size_t workspace_bytes, void* stream);

/* shm_projectors with flags.  SHM_STRICT_FP64 (SHM_F64; ignored for SHM_F32):
 * every value in binary64 arithmetic -- the interval cubics kept and
 * evaluated in binary64 (Horner), the log-grid index from CUDA's binary64 log
 * of |d|^2, the all-binary64 harmonic rows of shm_eval_ex with the flag, and
 * one binary64 product f_l x R_l^m per value -- instead of the default FP64
 * form's float-float log, cubics and short rows.  Other bits: SHM_EINVAL. */
shm_status shm_projectors_ex(const shm_proj_problem* prob, shm_dtype dtype, unsigned flags, void* out,
                             void* workspace, size_t workspace_bytes, void* stream);

/* Row form of the SHM_STRICT_FP64 projectors, for later prepares in this
 * process (a prepared workspace keeps the form it was prepared with):
 *   1 -- every binary64 product on the FP64 pipe;
 *   2 -- the products that leave the harmonic row (S_lm A_m, S_lm B_m,
 *        s A_m, s B_m of Sec. II Eq. 6) and f_l x R_l^m computed on the
 *        integer pipes: the IEEE-754 round-to-nearest-even product from
 *        32-bit integer multiply-adds, the same bits as the FP64 multiply; a
 *        row with a zero, subnormal or out-of-range product (an axis point,
 *        f_l = 0) is computed again with the FP64 instructions;
 *   3 -- (default) as 2, with every other product of the row as well (the
 *        scales S_lm Qh, the recurrence products G_lm Qh and the m = 0
 *        column).
 * All forms give the same bits; on a B300 the FP64 pipe binds form 1, and
 * forms 2 and 3 move 30-40 of its ~107 instructions per point to the
 * otherwise idle integer pipes.  shm_projectors_strict_form returns the
 * current form.  Errors: SHM_EINVAL for any other form. */
shm_status shm_projectors_set_strict_form(int form);
int shm_projectors_strict_form(void);

/*
 * shm_projectors_prepare -- the per-problem set-up of shm_projectors, done
 * once: two launches on `stream` that validate every atom's offsets and
 * species, order the atoms by species lmax (then species), build the tile
 * table and the tile descriptors (tiles of the current launch variant's
 * size), write the interval cubics of the radial tables and the
 * displacement tables into `workspace`, and clear the error word.  The
 * workspace is then "prepared" for this problem and dtype, and
 * shm_projectors_run computes the values with one launch per call.  Prepare
 * again after changing any array of the problem or the variant choice.
 *   prob, dtype, workspace, workspace_bytes, stream : as shm_projectors.
 * Errors: as shm_projectors.
 */
shm_status shm_projectors_prepare(const shm_proj_problem* prob, shm_dtype dtype, void* workspace,
                                  size_t workspace_bytes, void* stream);

/* shm_projectors_prepare with flags (SHM_STRICT_FP64 as for shm_projectors_ex);
 * the runs of the workspace then use that arithmetic. */
shm_status shm_projectors_prepare_ex(const shm_proj_problem* prob, shm_dtype dtype, unsigned flags, void* workspace,
                                     size_t workspace_bytes, void* stream);

/*
 * shm_projectors_run -- the projector values on a prepared workspace: ONE
 * persistent launch on `stream` (SMs x resident CTAs taking the tiles round
 * robin; it writes only the output and the error word, so every run is the
 * same launch).  It allocates nothing and enqueues only that kernel, so it
 * can be captured into a CUDA graph and replayed.  Runs of one workspace on
 * different streams may overlap on the GPU only with different outputs
 * (they share the error word).
 * Every index the kernel follows is checked on the device against the
 * problem; tiles that do not match it set error bit 8 and are skipped.
 * Errors: as shm_projectors; SHM_EINVAL when the workspace has not been
 * prepared for this problem's sizes and dtype.
 */
shm_status shm_projectors_run(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* workspace,
                              size_t workspace_bytes, void* stream);

/*
 * shm_projectors_autotune -- times every projector launch variant (tiles of
 * 128/256/512 sphere points in rounds of 64/128/256 rows, register caps of
 * 48 or 64, bulk copy or copy-out of the staged rows) on this problem: for
 * each, a
 * prepare and four runs into `out` (the first a warm-up), keeping the fastest
 * for later prepares of this dtype in this process (and in the file
 * SHM_TUNE_CACHE names, if set).  Leaves `workspace` prepared for the chosen
 * variant.  It synchronises a private stream, so it must not run during
 * stream capture.  best_ms (may be NULL) receives the fastest run.
 * Errors: as shm_projectors_prepare.
 */
shm_status shm_projectors_autotune(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* workspace,
                                   size_t workspace_bytes, double* best_ms);

/* Projector launch variants: count, the name of the current choice for a
 * dtype, and pinning one (0 .. count-1; -1 restores the default) for later
 * prepares in this process.  Errors: SHM_EINVAL. */
int shm_projectors_variant_count(void);
const char* shm_projectors_variant(shm_dtype dtype);
shm_status shm_projectors_set_variant(shm_dtype dtype, int variant);

/* Error bits a projector launch found (0 = none); waits for `stream`.
 * 1: point_offsets not non-decreasing or beyond n_points (or valid atoms'
 * point ranges overlapping beyond the workspace's tile descriptors); 2:
 * species index out of range; 4: grid index out of range; 8: output block
 * beyond n_values or inconsistent with out_offsets (or a tile that does not
 * match the problem).
 * The bits accumulate from the last prepare on. */
shm_status shm_projectors_check(const void* workspace, void* stream, uint32_t* error_bits);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of evaluation requests on one GPU (not in the
 * paper; the paper's evaluator is the unit of work).  Requests of any size,
 * lmax and dtype are admitted as device memory (a pool allocated at create)
 * and request slots free up; a scheduler thread forms each GPU batch from
 * chunks of every admitted, unfinished request (round robin, at most
 * chunk_points per request and batch_points per batch), so requests that
 * arrive while others run join the next batch and their work shares the
 * same kernel launches.  Each request's rows are computed by the same device
 * code as shm_eval, so a result does not depend on what it was batched with.
 * There is no device-side polling: every batch is an ordinary launch and
 * completion is observed through CUDA events.
 * ------------------------------------------------------------------------ */
typedef struct shm_server shm_server;

typedef struct {
  size_t pool_bytes;        /* device memory for request outputs (one cudaMalloc at create) */
  int32_t max_slots;        /* requests admitted (on the device) at once, >= 1 */
  int32_t queue_capacity;   /* requests waiting for admission; beyond it submit returns SHM_EBUSY */
  int64_t batch_points;     /* points per GPU batch (all requests together), >= 1 */
  int64_t chunk_points;     /* points per request per batch, >= 1 */
  int32_t inflight_batches; /* batches enqueued ahead of completion, 1..8 */
  int32_t device;           /* CUDA device ordinal */
} shm_serve_config;

#define SHM_REQ_DISCARD 0x1u     /* free the output as soon as the request completes (no result rows) */
#define SHM_REQ_STRICT_FP64 0x2u /* SHM_F64 requests: all-binary64 rows (as SHM_STRICT_FP64 for shm_eval_ex) */

typedef struct {
  const void* points;       /* device [n][3] of dtype, kept alive by the caller until the request
                               completes; NULL: the server generates point i from `seed` (see
                               shm_serve_generated_point) */
  int64_t n;                /* >= 1 */
  int32_t lmax;             /* 0..9 */
  shm_dtype dtype;
  uint64_t seed;
  uint32_t flags;           /* SHM_REQ_DISCARD, SHM_REQ_STRICT_FP64 */
} shm_request;

typedef struct {
  shm_status status;        /* SHM_OK once complete */
  void* out;                /* device [n][(lmax+1)^2] of dtype, valid until shm_serve_release
                               (NULL for SHM_REQ_DISCARD) */
  int64_t n;
  int32_t lmax;
  shm_dtype dtype;
  double t_submit_ms;       /* server clock: ms since shm_serve_create */
  double t_admit_ms;
  double t_done_ms;         /* when the server saw the last batch holding the request finish */
} shm_result;

typedef struct {
  uint64_t submitted, rejected, admitted, completed, batches;
  uint64_t queued_now, active_now;
  double harmonics_done;    /* sum over completed requests of n (lmax+1)^2 */
  double busy_ms;           /* sum of batch GPU times (CUDA events) */
  double lat_p50_ms, lat_p99_ms, lat_max_ms;   /* submit -> done (as the scheduler saw it), over completed
                                                  requests */
  size_t pool_bytes, pool_in_use, pool_peak;
  uint64_t collected;                          /* requests a wait has returned to the client */
  double client_lat_p50_ms, client_lat_p99_ms, client_lat_max_ms;  /* submit -> the first shm_serve_wait or
                                                  shm_serve_wait_any returning the request, over collected
                                                  requests: the latency the client sees */
} shm_serve_stats;

/* Creates a server: allocates the pool and starts the scheduler thread.
 * Errors: SHM_EINVAL (config), SHM_ENOMEM (pool), SHM_ECUDA. */
shm_status shm_serve_create(const shm_serve_config* cfg, shm_server** server);

/* Queues a request and returns its ticket.  SHM_EBUSY when the queue is full
 * (the request is counted as rejected); SHM_EINVAL for a bad request or one
 * whose output can never fit the pool. */
shm_status shm_serve_submit(shm_server* server, const shm_request* req, uint64_t* ticket);

/* Waits up to timeout_ms (< 0: no limit) for the request; fills *result.
 * SHM_ETIMEOUT when it is still running; SHM_ENOTFOUND for an unknown or
 * released ticket. */
shm_status shm_serve_wait(shm_server* server, uint64_t ticket, int timeout_ms, shm_result* result);

/* Waits up to timeout_ms (< 0: no limit) for any request that has completed
 * and that no wait has returned yet, oldest completion first, and returns
 * its ticket and result (requests submitted with SHM_REQ_DISCARD are never
 * returned).  A client that collects its requests this way sees each one as
 * soon as it completes, whatever order they were submitted in.  SHM_ETIMEOUT
 * when none completed in time; SHM_ECUDA for a request whose batch failed
 * (ticket and result are still filled in). */
shm_status shm_serve_wait_any(shm_server* server, int timeout_ms, uint64_t* ticket, shm_result* result);

/* Returns a completed request's output memory to the pool and forgets the
 * ticket.  SHM_EBUSY if it has not completed. */
shm_status shm_serve_release(shm_server* server, uint64_t ticket);

/* Counters and latency percentiles since create (or the last reset). */
shm_status shm_serve_stats_get(shm_server* server, shm_serve_stats* stats);
shm_status shm_serve_stats_reset(shm_server* server);

/* Stops the scheduler after the admitted work drains, frees the pool. */
shm_status shm_serve_destroy(shm_server* server);

/* Point i of a generated request (points == NULL) with this seed, as double
 * x, y, z: SplitMix64 counter words 4i..4i+3 mapped with correctly rounded
 * IEEE +, -, * only (on doubles assembled from the words' bits), so any
 * binary64 implementation reproduces it exactly (host function; the device
 * uses the same arithmetic).  FP32 requests round these to float. */
void shm_serve_generated_point(uint64_t seed, int64_t i, double xyz[3]);

/*
 * shm_projectors_noalloc -- shm_projectors for callers that cannot allocate
 * device memory.  (The paper has no counterpart: it is a calling convention
 * of this library.)  Some callers own no allocation rights on the device:
 * a host code whose framework has already reserved the device memory in its
 * own pool (a further cudaMalloc fails or fragments that pool), or a time-step
 * loop with a fixed memory budget that may not grow or synchronise the device
 * through cudaMalloc/cudaFree.  They pass only the problem and the output;
 * the scratch (the workspace of shm_projectors: tile table, descriptors,
 * error word, interval cubics and displacement tables) lives in a static
 * device array of SHM_PROJ_NOALLOC_SCRATCH_BYTES bytes inside this library,
 * which every GPU that loads the library holds until the process exits.
 *   prob, dtype, out, stream : as shm_projectors.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and caches it; make that
 * first call before any stream capture.  No call allocates or frees memory.
 * The error word is cleared at the start of every call, on `stream`.  All calls share the one array: calls that overlap on the GPU
 * (on different streams or threads) race and must not be issued; calls on
 * one stream are ordered and safe.  The error word of this variant cannot be
 * read back (use shm_projectors with a workspace for that report); rows the
 * kernel finds inconsistent are skipped as in shm_projectors.
 * Errors: those of shm_projectors; SHM_EINVAL, with the byte counts in
 * shm_last_error(), when the problem needs more scratch than
 * SHM_PROJ_NOALLOC_SCRATCH_BYTES (shm_projectors_workspace_size tells how
 * much); SHM_ECUDA if the symbol lookup fails.
 */
#define SHM_PROJ_NOALLOC_SCRATCH_BYTES (1u << 25)
shm_status shm_projectors_noalloc(const shm_proj_problem* prob, shm_dtype dtype, void* out, void* stream);

/*
 * shm_eval_complex -- the complex harmonics Y_l^m, l <= lmax (Sec. II Eq. 5,
 * Condon-Shortley sign included, and Sec. III Eq. 10 for negative m), at n
 * points.  Equivalently, from the real harmonics of shm_eval: Y_l^0 = R_l^0,
 * Y_l^{+m} = (-1)^m (R_l^m + i R_l^{-m}) / sqrt2, Y_l^{-m} = (R_l^m - i R_l^{-m}) / sqrt2
 * for m > 0 (the Sec. III relation printed without the 1/sqrt2).
 *   points, n, lmax, dtype, flags, stream : as shm_eval_ex.
 *   out : device, [n][(lmax+1)^2][2] of dtype: (Re, Im) at k = l*l + l + m.
 * FP64 rows use binary64 for 1/r and the m = 0, 1 columns and float-float
 * arithmetic for m >= 2 (within 1e-13 of the l-shell norm), or binary64
 * throughout with SHM_STRICT_FP64; FP32 rows as shm_eval.  Nothing is
 * allocated.  Errors: as shm_eval.
 */
shm_status shm_eval_complex(const void* points, int64_t n, int lmax, shm_dtype dtype, unsigned flags, void* out,
                            void* stream);

/*
 * shm_eval_angles -- the angular interface (Sec. II: the paper offers angular,
 * Cartesian and normalised-Cartesian inputs): all R_l^m, l <= lmax, at n
 * directions given by their angles.
 *   angles : device, [n][2] (theta, phi) in radians, theta from +z (Eq. 3),
 *            phi = atan2(y, x) (Eq. 4), element type per dtype.
 *   out    : device, [n][(lmax+1)^2] of dtype, as shm_eval.
 * The unit vector (sin t cos p, sin t sin p, cos t): for SHM_F64, theta by
 * CUDA's binary64 sincos and phi by a float-float sine and cosine on the FP32
 * pipe (|phi| <= 800; binary64 sincos beyond), then the hybrid rows of
 * shm_eval; for SHM_F32, sincosf and the FP32 rows.  Nothing is allocated.
 * Errors: as shm_eval.
 */
shm_status shm_eval_angles(const void* angles, int64_t n, int lmax, shm_dtype dtype, void* out, void* stream);

/* shm_eval_angles with flags: SHM_STRICT_FP64 (SHM_F64) takes binary64 sincos
 * of both angles and the all-binary64 rows.  Other bits: SHM_EINVAL. */
shm_status shm_eval_angles_ex(const void* angles, int64_t n, int lmax, shm_dtype dtype, unsigned flags, void* out,
                              void* stream);

/*
 * shm_eval_spinor -- the spin-1/2 spinor harmonics (Sec. II Eq. 7) for every
 * orbital l <= lmax and both total angular momenta j = l + s/2 (s = +1; and
 * s = -1 when l >= 1), m_j = -j .. j, at n points:
 *   upper = s sqrt((l + s m_j + 1/2) / (2l+1)) Y_l^{m_j - 1/2}
 *   lower =   sqrt((l - s m_j + 1/2) / (2l+1)) Y_l^{m_j + 1/2}
 * with Y_l^m the complex harmonics of shm_eval_complex (Y_l^m = 0 for |m| > l).
 *   points, n, lmax (0..9), dtype, flags, stream : as shm_eval_ex.
 *   out : device, [n][2 (lmax+1)^2][2][2] of dtype: spinor q, component
 *         (0 = upper, 1 = lower), (Re, Im).  Spinor order: l ascending; in
 *         each l first j = l - 1/2, then j = l + 1/2; m_j ascending, i.e.
 *         q = 2 l^2 + (s < 0 ? 0 : 2l) + (m_j + j).  16-byte (FP64) or
 *         8-byte (FP32) alignment of out enables the vector store path.
 * FP64 rows: the hybrid real rows times the coupling coefficients, real
 * parts by binary64 products and imaginary parts by float-float products
 * (within 1e-13 of the l-shell norm sqrt((2l+1)/4pi)); with SHM_STRICT_FP64
 * the all-binary64 rows and binary64 products throughout.  FP32 rows as
 * shm_eval.  Nothing is allocated.  Errors: as shm_eval (lmax outside 0..9:
 * SHM_EINVAL).
 */
shm_status shm_eval_spinor(const void* points, int64_t n, int lmax, shm_dtype dtype, unsigned flags, void* out,
                           void* stream);

/* Spinor harmonics per point for lmax: 2 (lmax+1)^2 (-1 for lmax outside 0..9). */
int shm_num_spinors(int lmax);

/* Diagnostics (not part of the method).  The FP64 pipe's rate on the current
 * device, measured: a kernel of independent DFMA chains (8 per thread, the
 * resident maximum of 256-thread CTAs per SM, `iters` DFMAs per chain) timed
 * with CUDA events after a warm-up launch.  *dfma_per_s receives the DFMA
 * instructions per second summed over the GPU's lanes (x 2 = FP64 flop/s),
 * *ms (may be NULL) the timed launch.  It synchronises on a private stream,
 * so it must not run during stream capture; nothing is allocated.
 * Errors: SHM_EINVAL (iters outside 1..2^24, null result), SHM_ECUDA. */
shm_status shm_probe_fp64_rate(int64_t iters, double* dfma_per_s, double* ms);

/* Diagnostics: checks the library's binary64 multiplication on the integer
 * pipes (used by the rows-tma-emu-* variants of SHM_STRICT_FP64) against the
 * GPU's DMUL instruction on n operand pairs generated from `seed` (random
 * significands over most of the normal range, exact ties, all-ones
 * significands, products at the edges of the normal range, zeros and
 * subnormals).  *mismatches receives the pairs where the two results differ
 * in any bit (0 expected), *declined the pairs outside the emulation's range
 * (zero, subnormal or non-finite operands or results), which the row code
 * hands to the FP64 instructions.  Synchronises the device; nothing is
 * allocated.  Errors: SHM_EINVAL (n outside 0..2^40, null results),
 * SHM_ECUDA. */
shm_status shm_probe_dmul(int64_t n, uint64_t seed, int64_t* mismatches, int64_t* declined);

/* Thread-local description of the last error of this thread ("" if none). */
const char* shm_last_error(void);

/* Text name of a status code. */
const char* shm_status_string(shm_status s);

#ifdef __cplusplus
}
#endif

#endif /* SHM_H */
