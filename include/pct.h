/*
 * pct.h -- C ABI of libpct, a GB300 (sm_103a) implementation of the data-
 * parallel hot path of the proton-CT data simulator of Witt, Schultze,
 * Schulte, Schubert and Gomez, "A Proton Simulator for Testing
 * Implementations of Proton CT Reconstruction Algorithms on GPGPU Clusters".
 *
 * The simulator produces the linear system A x = b of Sec. II (Methods):
 *   x  -- the RSP of every voxel of an analytic NEO phantom (Sec. II-A),
 *   A  -- one row per proton, a_ij = chord length of proton i's path in
 *         voxel j (Sec. II-C), stored as CSR (Sec. II-C, Fig. 3),
 *   b  -- WEPL of proton i, <a_i, x>, optionally with noise (Sec. II-C),
 * for protons entering as parallel beams from many angles, on straight or
 * cubic-spline paths with multiple-Coulomb-scattering exit draws (Sec. II-B).
 *
 * Conventions of every call:
 *   - Pointers named *_dev are CUDA device pointers; all others are host.
 *   - The caller owns every buffer.  The library allocates device memory only
 *     inside pct_simulate(), and only through the caller's pct_alloc_fn.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *     enqueue their GPU work on it and return without waiting, except where
 *     a call says it synchronises.
 *   - Every call returns a pct_status; on failure pct_last_error() returns a
 *     message for the calling thread.  The library never aborts the process.
 *   - Row i of A is proton p of angle k with i = k * paths_per_angle + p;
 *     column j = ix + nx * (iy + ny * iz); voxel ix covers
 *     [o_x + ix h_x, o_x + (ix+1) h_x) with o_x = -nx h_x / 2 (grid centred
 *     at the origin).  Beam frame of angle theta: u = (cos, sin, 0) beam
 *     direction, t = (-sin, cos, 0) lateral, v = (0, 0, 1) (Sec. II-C,
 *     Givens rotation of the tvu frame into xyz).
 *   - Results are a pure function of the arguments: the same arguments give
 *     the same bits.
 */
#ifndef PCT_H
#define PCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PCT_OK = 0,
  PCT_EINVAL = 1,       /* bad argument: nothing was enqueued */
  PCT_ENOMEM = 2,       /* the caller's allocator returned NULL / workspace too small */
  PCT_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
  PCT_ETIMEOUT = 4,     /* reserved: no call returns it (no kernel of the library waits on another) */
  PCT_EUNSUPPORTED = 5  /* valid request the library does not implement */
} pct_status;

enum { PCT_ELLIPSOID = 0, PCT_EXTRUDED = 1 };                /* phantom kind (3D) */
enum { PCT_RASTER_CENTER = 0, PCT_RASTER_CORNER = 1, PCT_RASTER_AREA = 2 }; /* Sec. II-A options */
enum { PCT_PATH_STRAIGHT = 0, PCT_PATH_STRAIGHT_MCS = 1, PCT_PATH_SPLINE = 2 };
enum { PCT_CHORD_EXACT = 0, PCT_CHORD_CONSTANT = 1 };        /* Sec. II-C */
enum { PCT_NOISE_NONE = 0, PCT_NOISE_GAUSS_REL = 1 };
enum { PCT_MCS_FIXED = 0, PCT_MCS_HIGHLAND = 1 };            /* Sec. II-B exit widths */
/* Arithmetic form of the path and traversal kernels.  All give identical
 * voxel indices and row pointers (every crossing decision equals the FP64
 * definition's); values and b agree within 1e-6 relative per row.
 *   PCT_PREC_MIXED: FP32 arithmetic with certified error bounds, exact FP64
 *                   evaluation only where a bound cannot decide; FP32 lengths,
 *                   FP32 Kahan-compensated WEPL.
 *   PCT_PREC_F64:   everything in FP64 (the comparison form).
 *   PCT_PREC_MIXED_LEAN: PCT_PREC_MIXED with about a fifth of its workspace
 *                   (the count keeps no per-segment records; the fill sets
 *                   each row's segments up again), same bits as
 *                   PCT_PREC_MIXED, slower fill: for systems whose workspace
 *                   would not fit beside the CSR.                         */
enum { PCT_PREC_MIXED = 0, PCT_PREC_F64 = 1, PCT_PREC_MIXED_LEAN = 2 };

#define PCT_MAX_REGIONS 16
#define PCT_MAX_SPLINE_SEGMENTS 1024

/* An ellipse (2D: z ignored) or ellipsoid with centre c and semi-axes a, mm.
 * Sec. II-A: the NEO phantom is a list of such regions, each with its RSP. */
typedef struct {
  double c[3];
  double a[3];
  double rsp;
} pct_region;

/* Sec. II-A.  Regions are painted in order (a later region overwrites an
 * earlier one where they overlap); region 0 is the phantom's outer boundary,
 * used as the entry/exit surface of the protons (Sec. II-B).  3D kind
 * PCT_EXTRUDED tests x, y only (the paper's stacked-slice elliptical
 * cylinder); PCT_ELLIPSOID tests x, y, z.  n[2] and h[2] are ignored in 2D. */
typedef struct {
  int32_t dim;    /* 2 or 3 */
  int32_t kind;   /* PCT_ELLIPSOID / PCT_EXTRUDED */
  int32_t raster; /* PCT_RASTER_CENTER / PCT_RASTER_CORNER / PCT_RASTER_AREA */
  int32_t n[3];   /* voxels per axis, >= 1, product < 2^31 */
  double h[3];    /* voxel size, mm, > 0 */
  int32_t n_regions;          /* 1..PCT_MAX_REGIONS */
  const pct_region* regions;  /* host array, copied by pct_phantom_create */
  int32_t area_samples;       /* PCT_RASTER_AREA: sub-samples per axis S, 1..64 */
} pct_phantom_desc;

/* Sec. II-B.  Lateral entry offsets are uniform on t_range (and v_range in
 * 3D).  MCS models draw, per proton, an entry slope ~ N(0, sigma_in) per
 * plane and a bivariate normal exit pair (displacement ~ N(0, sigma_lat) mm,
 * slope ~ N(0, sigma_out)) with correlation rho per plane.  With mcs =
 * PCT_MCS_HIGHLAND the exit widths follow the Highland formula with the PDG
 * constants instead, per proton, from its chord x through the hull (region
 * 0): theta0 = 13.6 MeV / (beta c p) sqrt(x / X0) (1 + 0.038 ln(x / (X0
 * beta^2))) for a proton of kinetic energy beam_mev in a medium of radiation
 * length x0_mm; sigma_out = theta0, sigma_lat = x theta0 / sqrt(3), rho =
 * sqrt(3) / 2 (a thin slab's displacement-angle covariance); sigma_lat,
 * sigma_out and rho are then ignored.  SPLINE paths are
 * cubic Hermite curves sampled at spline_segments pieces.  With
 * PCT_NOISE_GAUSS_REL, b_i is multiplied by (1 + noise_rel z_i), z_i ~ N(0,1)
 * (our stand-in for the PSTAR / Tschalar energy-straggling noise of
 * Sec. II-C, whose tables are not part of this library). */
typedef struct {
  int32_t model;           /* PCT_PATH_* */
  int32_t chord;           /* PCT_CHORD_*: CONSTANT stores h_x in A, b stays exact */
  int32_t spline_segments; /* 1..PCT_MAX_SPLINE_SEGMENTS (SPLINE only) */
  int32_t noise;           /* PCT_NOISE_* */
  double t_range[2];
  double v_range[2];
  double sigma_lat, sigma_in, sigma_out, rho; /* |rho| <= 1 */
  double noise_rel;
  int32_t mcs;       /* PCT_MCS_FIXED (the widths above) or PCT_MCS_HIGHLAND */
  double beam_mev;   /* PCT_MCS_HIGHLAND: proton kinetic energy, MeV, > 0 */
  double x0_mm;      /* PCT_MCS_HIGHLAND: radiation length, mm, > 0 (water: 360.8) */
} pct_path_model;

/* One simulated acquisition, or a contiguous block of one: angles (host,
 * radians), protons per angle, the path model, the generator key (seed,
 * stream_id) and the global index of its first row.  Random numbers come from
 * Philox4x64-10 (Salmon et al., SC'11) with key (seed, stream_id) and counter
 * (first_row + i, block, 0, 0) for row i of the call, replacing the paper's
 * rand().  A block of angles [k0, k1) of an acquisition with P protons per
 * angle (Sec. IV: an acquisition-structured partition over GPUs) passes
 * angles_rad + k0, n_angles = k1 - k0 and first_row = k0 P: its rows are then
 * bit for bit rows k0 P .. k1 P - 1 of the whole acquisition, and the blocks'
 * CSRs concatenate into the whole one.  first_row = 0 for a whole
 * acquisition; 0 <= first_row, first_row + rows <= 2^62. */
typedef struct {
  const double* angles_rad;
  int32_t n_angles;
  int64_t paths_per_angle;
  pct_path_model model;
  uint64_t seed;
  uint64_t stream_id;
  int64_t first_row;
} pct_geometry;

typedef struct pct_phantom pct_phantom; /* opaque, host memory only */

/* CSR A plus b and x (Sec. II-C, Fig. 3).  All pointers are device pointers.
 * row_ptr: int64 [n_rows + 1]; col: int32 [nnz]; val: float [nnz] (chord
 * lengths, mm); b: float [n_rows] (WEPL, mm); x_true: float [n_cols]. */
typedef struct {
  int64_t n_rows, n_cols, nnz;
  int64_t* row_ptr;
  int32_t* col;
  float* val;
  float* b;
  float* x_true;
} pct_csr;

typedef void* (*pct_alloc_fn)(size_t bytes, void* ctx); /* device memory or NULL */
typedef void (*pct_free_fn)(void* ptr, void* ctx);

/* ---- phantom (Sec. II-A) ---------------------------------------------- */

/* Validates and copies the description.  EINVAL on bad sizes, axes or
 * counts; ENOMEM if host memory runs out.  *out is released by
 * pct_phantom_destroy. */
pct_status pct_phantom_create(const pct_phantom_desc* desc, pct_phantom** out);
pct_status pct_phantom_destroy(pct_phantom* ph);
/* number of voxels (columns of A), or -1 for NULL */
int64_t pct_phantom_nvox(const pct_phantom* ph);

/* Sec. II-A: x_true_dev[j] = RSP of voxel j by the phantom's raster option,
 * in FP32: the centre point; the mean over the 4 / 8 corners; or the
 * weighted-area average sum_r RSP_r f_r, with f_r the fraction of the voxel's
 * S^dim sub-sample midpoints (o + (i + (k + 1/2) / S) h per axis) whose last
 * containing region is r.  The stored solution vector of the simulator. */
pct_status pct_phantom_rasterize(const pct_phantom* ph, float* x_true_dev, void* stream);

/* ---- simulation: A, b (Sec. II-B, II-C) -------------------------------- */

/* Bytes of device workspace that pct_simulate_count / _fill / pct_forward /
 * pct_adjoint need for this geometry (angle table, spline basis, per-row
 * path records, scan partials). */
pct_status pct_simulate_workspace_size(const pct_phantom* ph, const pct_geometry* geo,
                                       int32_t precision, size_t* bytes);

/* Phase 1: row_ptr_dev[0..n_rows] = exclusive scan of the row lengths (int64).
 * nnz = row_ptr_dev[n_rows] (read it back to size col / val).  Also leaves
 * the per-row path records in the workspace for phase 2.  Protons whose
 * path misses the grid get empty rows. */
pct_status pct_simulate_count(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                              void* workspace_dev, size_t workspace_bytes, int64_t* row_ptr_dev,
                              void* stream);

/* Phase 2, after pct_simulate_count with the same arguments and workspace:
 * writes col_dev / val_dev at row_ptr_dev (entries of a row in path order,
 * voxels re-entered later in a row appear again) and b_dev (WEPL from the
 * exact chord lengths and x_true_dev, then noise). */
pct_status pct_simulate_fill(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                             void* workspace_dev, size_t workspace_bytes,
                             const int64_t* row_ptr_dev, const float* x_true_dev,
                             int32_t* col_dev, float* val_dev, float* b_dev, void* stream);

/* Phase 2 into HOST memory (Sec. II-C: the simulator's output is the
 * system A, b), after pct_simulate_count with the same arguments and
 * workspace.  row_ptr_host[0..n_rows] receives a copy of row_ptr_dev,
 * col_host / val_host[0..nnz) and b_host[0..n_rows) the same values that
 * pct_simulate_fill writes to device memory.  The rows are filled block by
 * block into staging_dev (caller-owned device memory, 256-byte aligned, two
 * halves; each half holds up to E = (staging_bytes / 2) / 8.25 entries and
 * E / 16 rows), and each block's copies to the host run on two internal
 * streams (col; val and b) while the next block is filled.  Host buffers should be pinned
 * (page-locked) for the copies to overlap.  Synchronises: on return the
 * host buffers are complete.  EINVAL if a single row has more entries than
 * a half holds.  Caller owns every buffer. */
pct_status pct_simulate_fill_host(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                                  void* workspace_dev, size_t workspace_bytes, const int64_t* row_ptr_dev,
                                  const float* x_true_dev, void* staging_dev, size_t staging_bytes,
                                  int64_t* row_ptr_host, int32_t* col_host, float* val_host, float* b_host,
                                  void* stream);

/* The fill's row check (Sec. II-C: row i of A holds exactly the entries of
 * proton i's path).  Every fill compares, per row, the entries it writes with
 * the range row_ptr gives the row; stores never leave that range, and a row
 * whose counts differ (a row_ptr that is not the count of the same
 * arguments and workspace) is counted in the workspace's first word, which
 * pct_simulate_count and pct_simulate_host zero.  This call synchronises
 * `stream` and returns that count in *mismatched_rows (0 for a consistent
 * fill).  pct_simulate, pct_simulate_fill_host and pct_simulate_host make
 * the same check themselves and return PCT_EINVAL when rows disagree.
 * The batch calls do not report it (their row pointers come from their own
 * count). */
pct_status pct_simulate_check(const void* workspace_dev, int64_t* mismatched_rows, void* stream);

/* Bytes of device workspace for pct_simulate_host with blocks of
 * angles_per_block angles (>= 1): the layout of one block's simulation plus
 * the block's row pointers. */
pct_status pct_simulate_host_workspace_size(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                                            int32_t angles_per_block, size_t* bytes);

/* The whole simulation into HOST memory in one call (Sec. II-C: the
 * simulator's output is the system A, b, here for acquisitions whose CSR
 * need not, or cannot, stay on the device).  The acquisition is taken in
 * blocks of angles_per_block angles (the last may be shorter), each the
 * geometry's angle block k0..k1 with first_row + k0 P, so that its rows are
 * the acquisition's own.  Per block, on `stream`: the count and the scan
 * into the workspace (sized by pct_simulate_host_workspace_size), the
 * block's row pointers read back (one synchronisation per block), then the
 * fill through staging_dev exactly as pct_simulate_fill_host does; a block's
 * copies to the host run on two internal streams while the next block is
 * counted and filled.  x_true_dev: the rasterised phantom (device).
 * row_ptr_host[0..n_rows], b_host[0..n_rows) and, when the acquisition's
 * nonzero count fits nnz_capacity, col_host / val_host[0..nnz) receive the
 * values of pct_simulate_count + pct_simulate_fill.  *nnz_out receives the
 * nonzero count in every case.  When it exceeds nnz_capacity the remaining
 * blocks are only counted (col_host / val_host may be NULL; capacity 0 makes
 * the call a count with a one-block workspace), col / val / b hold nothing
 * defined and the call returns PCT_ENOMEM.  Host buffers should be pinned.
 * Synchronises: on return the host buffers are complete.  EINVAL for NULL
 * pointers, angles_per_block < 1 or a row with more entries than a staging
 * half holds; ENOMEM for a short workspace.  Caller owns every buffer. */
pct_status pct_simulate_host(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                             int32_t angles_per_block, void* workspace_dev, size_t workspace_bytes,
                             const float* x_true_dev, void* staging_dev, size_t staging_bytes,
                             int64_t* row_ptr_host, int32_t* col_host, float* val_host, float* b_host,
                             int64_t nnz_capacity, int64_t* nnz_out, void* stream);

/* Whole simulation: rasterises x_true, counts, reads nnz back (synchronises
 * the stream once), allocates through alloc_fn and fills.  out receives
 * device buffers owned by the caller (free them with free_fn).  On failure
 * everything allocated so far is freed. */
pct_status pct_simulate(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                        pct_alloc_fn alloc_fn, pct_free_fn free_fn, void* ctx, pct_csr* out,
                        void* stream);

/* ---- projectors: y = A x and g += A^T r (Sec. II, A x = b) -------------- */

/* Workspace for the matrix-free projectors on chunks of at most max_rows
 * rows (angle / basis tables and per-row records of one chunk). */
pct_status pct_projector_workspace_size(const pct_phantom* ph, const pct_geometry* geo, int32_t precision,
                                        int64_t max_rows, size_t* bytes);

/* y_dev[i - row0] = sum_j A_ij x_dev[j] for rows [row0, row0 + n_rows).
 * With A != NULL the CSR is used (HBM-bound, 8 bytes per nonzero; geo,
 * precision and the workspace are ignored).  With A == NULL the rows are
 * regenerated from the geometry (matrix-free: the same paths, voxels and
 * lengths as pct_simulate_fill, nothing stored) in the given precision, with
 * a workspace of pct_projector_workspace_size(..., n_rows) bytes; this is how
 * systems too large for HBM are projected, chunk by chunk. */
pct_status pct_forward(const pct_phantom* ph, const pct_geometry* geo, const pct_csr* A, int32_t precision,
                       int64_t row0, int64_t n_rows, const float* x_dev, float* y_dev,
                       void* workspace_dev, size_t workspace_bytes, void* stream);

/* g_dev[j] += sum_i A_ij r_dev[i - row0] over rows [row0, row0 + n_rows)
 * (accumulates, so chunks can be summed; the caller zeroes g_dev first).
 * FP32 atomic accumulation: the order of additions is not fixed.  Rows with
 * r_i = 0 are skipped.  Arguments as for pct_forward. */
pct_status pct_adjoint(const pct_phantom* ph, const pct_geometry* geo, const pct_csr* A, int32_t precision,
                       int64_t row0, int64_t n_rows, const float* r_dev, float* g_dev,
                       void* workspace_dev, size_t workspace_bytes, void* stream);

/* ---- batches: many simulations per launch -------------------------------
 * Several independent simulations (different phantoms, grids, 2D / 3D, path
 * models, sizes) share one persistent launch per phase: blocks take work
 * items (simulation, block of 128 rows) from a device counter.  The count
 * phase (raster, count, row pointers) and the fill phase are each captured
 * once as a CUDA graph and replayed.  Mixed precision; the outputs of each
 * simulation equal those of pct_simulate_count / pct_simulate_fill. */
typedef struct {
  const pct_phantom* phantom;  /* must outlive the batch */
  pct_geometry geo;            /* its angles are read by pct_batch_create */
  int64_t* row_ptr_dev;        /* [rows + 1], written by pct_batch_count */
  float* x_true_dev;           /* [nvox], rasterised by pct_batch_count */
} pct_batch_item;

typedef struct pct_batch pct_batch; /* opaque */

#define PCT_BATCH_AUTOTUNE 1 /* flags: time the launch shapes once and keep the fastest */
/* flags: items may take the PCT_PREC_MIXED_LEAN form (small workspace).  The
 * workspace size is then that of every item in the lean form; any workspace
 * given beyond it holds segment records, and the largest items take the
 * full PCT_PREC_MIXED form (whose fill is faster) while their records fit.
 * The outputs are the same bits either way. */
#define PCT_BATCH_LEAN 2

/* bytes of device workspace pct_batch_create needs for these items and flags
 * (with PCT_BATCH_LEAN: the all-lean minimum) */
pct_status pct_batch_workspace_size(const pct_batch_item* items, int32_t n, int32_t flags, size_t* bytes);

/* Uploads every simulation's tables into the workspace, orders the work
 * items, optionally autotunes the launch shape (runs the count phases a few
 * times and synchronises; see pct_batch_tuning) and captures the graphs.  The workspace and the item buffers must
 * stay valid until pct_batch_destroy. */
pct_status pct_batch_create(const pct_batch_item* items, int32_t n, void* workspace_dev, size_t workspace_bytes,
                            int32_t flags, void* stream, pct_batch** out);

/* count phase for all items (graph launch on stream) */
pct_status pct_batch_count(pct_batch* batch, void* stream);

/* nnz of every item after pct_batch_count: host array [n]; synchronises stream */
pct_status pct_batch_nnz(pct_batch* batch, int64_t* nnz, void* stream);

/* fill phase: col_dev[k], val_dev[k], b_dev[k] are item k's outputs (host
 * arrays of n device pointers).  With PCT_BATCH_AUTOTUNE the first call
 * times the fill's launch shapes on these outputs (synchronises). */
pct_status pct_batch_fill(pct_batch* batch, int32_t* const* col_dev, float* const* val_dev, float* const* b_dev,
                          void* stream);

/* The launch shape of a batch.  A phase's work items are blocks of
 * rows_per_item rows of one simulation; its persistent launch has
 * grid_mult x (SMs x resident blocks per SM) blocks.  With PCT_BATCH_AUTOTUNE
 * pct_batch_create times the item order on the count, then rows per item
 * {64, 128, 256} x grid multiplier {1, 2} for the path set-up and the count
 * phases; the first pct_batch_fill times the same for the fill phase, with
 * and without prefetching the next row's segment records into L2 (the
 * fill's staging depth, 1 row or none), and recaptures the fill graph.
 * Choices are cached per batch signature in the process. */
typedef struct {
  int32_t order;            /* 0: items as given, 1: largest simulation first (2D before 3D either way) */
  int32_t rows_per_item[3]; /* path set-up, count, fill */
  int32_t grid_mult[3];     /* path set-up, count, fill */
  int32_t fill_prefetch;    /* 1: next row's records prefetched into L2 */
} pct_batch_tuning;

pct_status pct_batch_params(const pct_batch* batch, pct_batch_tuning* out);

pct_status pct_batch_destroy(pct_batch* batch);

/* ---- allocation-free row pointers (no counterpart in the paper) ---------
 * For callers that cannot allocate device memory: code inside a host
 * application that owns every device allocation (a plugin with a fixed pool
 * and no cudaMalloc of its own), or a latency-critical loop where cudaMalloc
 * and cudaFree, which may synchronise the device, are not allowed.
 * On entry row_ptr_dev[1..n_rows] hold int64 per-row entry counts (for
 * example the differences of row pointers a caller already has, or counts it
 * computed); on completion, in stream order, row_ptr_dev[0] = 0 and
 * row_ptr_dev[i] = the sum of the first i counts -- the same result as the scan
 * inside pct_simulate_count, without a workspace.  The scratch (one int64 per
 * tile of rows) is a static device array sized for PCT_STATIC_SCAN_MAX_ROWS
 * rows, 512 KB that every GPU loading this library holds until the process
 * exits; larger n_rows return PCT_EINVAL with a message.  Every call looks up
 * that array's device address for the calling thread's current device
 * (cudaGetSymbolAddress, which allocates nothing), so the address stays right
 * after a cudaDeviceReset or in another context; the first call on a device
 * also loads the module that holds the array, so make that first call before
 * any stream capture.  All calls share the one array: calls whose work overlaps on the
 * GPU (other streams, other threads) race and corrupt each other's results --
 * serialise them.  A call writes every scratch slot it reads, so nothing has to
 * be cleared between calls.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
#define PCT_STATIC_SCAN_MAX_ROWS (1LL << 28)
pct_status pct_scan_counts_static(int64_t* row_ptr_dev, int64_t n_rows, void* stream);

/* ---- reconstruction: string-averaging projections (Sec. II-D) ----------
 * The paper's reconstruction algorithm (SAP, Censor et al.) on an explicit
 * CSR A and b, for checking the simulated systems.  The rows are split into
 * n_strings strings M, string t holding rows t, t + M, t + 2M, ... in
 * increasing order.  One iteration: every string starts from x and projects
 * its rows in order,
 *   y <- y + lambda (b_i - <a_i, y>) / ||a_i||^2 a_i   (rows with a_i = 0 skipped),
 * then x <- sum_t w_t y_t with w_t = weights[t] (host array of M doubles,
 * finite, summing to 1 within 1e-9) or 1 / M for weights = NULL.  (The
 * paper's printed update uses <a_i, x_k> and the opposite sign; this is the
 * projection of SAP as Censor et al. define it.)  FP32 iterates and sums,
 * FP64 averaging; summation order within a row is not fixed.  x_dev holds the
 * start on entry and the result on completion (in stream order); b_dev is
 * float [A->n_rows].  Workspace: pct_sap_workspace_size bytes (M copies of
 * x), caller-owned.  EINVAL on bad sizes, lambda not finite, weights not
 * summing to 1; ENOMEM when the workspace is too small. */
pct_status pct_sap_workspace_size(int64_t n_cols, int32_t n_strings, size_t* bytes);
pct_status pct_sap(const pct_csr* A, const float* b_dev, int32_t n_strings, const double* weights, double lambda,
                   int32_t iterations, float* x_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* ---- the system on disk (Sec. II-C: A written to a file read back as CSR) -
 * Host memory and host I/O only (no device work).  Layout: a 128-byte header
 * ("PCTCSR1\0", int64 n_rows, n_cols, nnz, then the byte offsets of the five
 * sections), then int64 row_ptr [n_rows + 1], int32 col [nnz], float val
 * [nnz], float b [n_rows], float x_true [n_cols], each section on a 4096-byte
 * boundary.  pct_csr_file_create makes the file for the whole system and
 * writes x_true; pct_csr_file_write_rows writes a block of rows (local
 * row_ptr[0..n_rows], any base, with its col / val / b) at global row row0
 * and global nonzero offset nz0 -- several writers (the angle blocks of an
 * acquisition split over GPUs, nz0 from the all-gathered block sizes) fill
 * one file that equals a single writer's.  EINVAL with the system's message
 * on I/O errors or a block beyond the file's sizes. */
pct_status pct_csr_file_create(const char* path, int64_t n_rows, int64_t n_cols, int64_t nnz, const float* x_true);
pct_status pct_csr_file_write_rows(const char* path, int64_t row0, int64_t n_rows, int64_t nz0,
                                   const int64_t* row_ptr, const int32_t* col, const float* val, const float* b);

/* message of the calling thread's last failure ("" if none) */
const char* pct_last_error(void);

/* library version string */
const char* pct_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PCT_H */
