/*
 * pct_oracle.h -- plain FP64 CPU oracle of the proton-CT data simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this code: only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py use it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it computes (Witt et al., "A Proton Simulator for Testing
 * Implementations of Proton CT Reconstruction Algorithms on GPGPU
 * Clusters"):
 *   - the NEO phantom raster x_true                      (Sec. II-A, Phantoms)
 *   - per proton: lateral entry offset, MCS exit displacement and angle from
 *     bivariate normals (Marsaglia polar + covariance), straight or cubic
 *     spline path                                        (Sec. II-B, Proton Paths)
 *   - row i of A: chord lengths of path i in each voxel it crosses, found by
 *     intersecting the path with the voxel planes      (Sec. II-C, Mathematical
 *     Formulation; the Ax=b statement of Sec. II)
 *   - b_i = <a_i, x_true> (+ relative Gaussian noise)   (Sec. II-C)
 *   - x from A, b by string-averaging projections        (Sec. II-D, SAP)
 * All floating point is IEEE binary64, compiled with -ffp-contract=off;
 * every fused multiply-add is an explicit fma() call.
 */
#ifndef PCT_ORACLE_H
#define PCT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ELLIPSOID = 0, ORC_EXTRUDED = 1 };
enum { ORC_CENTER = 0, ORC_CORNER = 1, ORC_AREA = 2 };
enum { ORC_STRAIGHT = 0, ORC_STRAIGHT_MCS = 1, ORC_SPLINE = 2 };
enum { ORC_CHORD_EXACT = 0, ORC_CHORD_CONSTANT = 1 };
enum { ORC_NOISE_NONE = 0, ORC_NOISE_GAUSS_REL = 1 };
enum { ORC_MCS_FIXED = 0, ORC_MCS_HIGHLAND = 1 };

typedef struct {
  int32_t dim;        /* 2 or 3 */
  int32_t kind;       /* ORC_ELLIPSOID or ORC_EXTRUDED (3D: z ignored) */
  int32_t raster;     /* ORC_CENTER, ORC_CORNER or ORC_AREA */
  int32_t n[3];       /* voxels per axis (n[2] = 1 in 2D) */
  double h[3];        /* voxel size per axis, mm */
  int32_t n_regions;  /* regions in painter's order; region 0 is the hull */
  const double* regions; /* n_regions x 7: cx cy cz ax ay az rsp */
  int32_t area_samples;  /* ORC_AREA: sub-samples per axis, S */
} orc_phantom;

typedef struct {
  int32_t model;           /* ORC_STRAIGHT / ORC_STRAIGHT_MCS / ORC_SPLINE */
  int32_t chord;           /* ORC_CHORD_EXACT / ORC_CHORD_CONSTANT */
  int32_t spline_segments; /* K, polyline pieces of the spline */
  int32_t noise;           /* ORC_NOISE_NONE / ORC_NOISE_GAUSS_REL */
  double t_lo, t_hi;       /* lateral entry interval (mm) */
  double v_lo, v_hi;       /* vertical entry interval (mm, 3D) */
  double sigma_lat;        /* exit lateral displacement sigma (mm) */
  double sigma_in;         /* entry slope sigma (rad) */
  double sigma_out;        /* exit slope sigma (rad) */
  double rho;              /* correlation of exit (displacement, slope) */
  double noise_rel;        /* relative WEPL noise sigma */
  int32_t mcs;             /* ORC_MCS_FIXED: the sigmas and rho above; ORC_MCS_HIGHLAND:
                              per proton from its chord through the hull (Highland / PDG) */
  double beam_mev;         /* proton kinetic energy, MeV (HIGHLAND) */
  double x0_mm;            /* radiation length of the (water-equivalent) medium, mm (HIGHLAND) */
} orc_model;

typedef struct {
  const orc_phantom* ph;
  const float* x_true;      /* [nvox] RSP values (FP32, as stored) */
  const double* angles;     /* [n_angles] projection angles, rad */
  int32_t n_angles;
  int64_t paths_per_angle;
  const orc_model* model;
  uint64_t seed;
  uint64_t stream;          /* second key word of the generator */
} orc_sim;

/* --- building blocks exposed for the pin tests --- */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double orc_log(double x);
/* uniform #j of proton `row` (j = 0: t offset, 1: v offset, 4.. normals) */
double orc_uniform(uint64_t seed, uint64_t stream, uint64_t row, uint64_t j);
/* standard normal pairs drawn by the polar method from proton `row`'s stream;
   writes 2*n_pairs normals, returns the next unused uniform index */
uint64_t orc_normal_pairs(uint64_t seed, uint64_t stream, uint64_t row, uint64_t j0,
                          int32_t n_pairs, double* z);
/* entry/exit parameters of a line A + lam*g through region r's ellipse or
   ellipsoid; returns 1 on a hit (lam_in < lam_out) */
int orc_hull_hit(const orc_phantom* ph, int32_t r, const double A[3], const double g[3],
                 double* lam_in, double* lam_out);

/* Highland / PDG multiple-scattering width theta0 (rad) of a proton of kinetic
   energy beam_mev after x_mm of a medium of radiation length x0_mm (Sec.
   II-B, MCS); *beta_cp receives beta c p in MeV.  Parity partly pinned: the
   kinematics by an independent route, the formula by its scaling. */
double orc_highland(double beam_mev, double x0_mm, double x_mm, double* beta_cp);

/* phantom raster: x[j] in FP64 (the stored x_true is its FP32 rounding).
   ORC_AREA (weighted-area average, Sec. II-A): x = sum_r rsp_r f_r over the
   regions in order, f_r the fraction of the voxel's S^dim sub-sample
   midpoints whose last containing region is r, evaluated as
   (sum_r rsp_r count_r) / S^dim. */
void orc_raster(const orc_phantom* ph, double* x);

/* one segment P->Q through the grid: voxel ids and FP64 chord lengths in path
   order; returns the count (entries beyond cap are counted, not written) */
int64_t orc_segment(const orc_phantom* ph, const double P[3], const double Q[3],
                    int32_t* cols, double* lens, int64_t cap);

/* polyline vertices of proton `row` (3 doubles each); returns the count */
int32_t orc_path(const orc_sim* sim, int64_t row, double* verts, int32_t cap);

/* row `row` of A: returns nnz; fills up to cap entries, FP64 lengths, and the
   clean / noisy WEPL */
int64_t orc_row(const orc_sim* sim, int64_t row, int32_t* cols, double* vals,
                int64_t cap, double* b_clean, double* b_noisy);

/* row counts for rows[0..n) (OpenMP over rows with `threads` threads) */
void orc_count_rows(const orc_sim* sim, const int64_t* rows, int64_t n, int64_t* counts,
                    int32_t threads);
/* rows[0..n) written at offsets off[0..n) of cols/vals; b per row */
void orc_fill_rows(const orc_sim* sim, const int64_t* rows, int64_t n, const int64_t* off,
                   int32_t* cols, double* vals, double* b_clean, double* b_noisy,
                   int32_t threads);

/* String-averaging projections (Sec. II-D, SAP; Censor et al.), the paper's
   reconstruction algorithm, in FP64.  Rows are partitioned into M strings,
   string t holding rows t, t + M, t + 2M, ... in increasing order.  One
   iteration: for every string, y = x, then for each of its rows i in order
     y <- y + lambda (b_i - <a_i, y>) / ||a_i||^2 a_i   (rows with a_i = 0 skipped);
   then x <- sum_t w_t y_t (w = NULL: w_t = 1 / M).  In place on x[n_cols]. */
void orc_sap(int64_t n_rows, int64_t n_cols, const int64_t* row_ptr, const int32_t* col,
             const double* val, const double* b, int32_t M, const double* w, double lambda,
             int32_t iterations, double* x);

#ifdef __cplusplus
}
#endif
#endif
