/*
 * pct_oracle.c -- plain FP64 CPU oracle of the proton-CT data simulator.
 *
 * TEST INFRASTRUCTURE ONLY (see pct_oracle.h).  Slow on purpose: every step
 * is the definition written out, in the order the paper describes it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared pct_oracle.c -lm
 * (-ffp-contract=off matters: GCC fuses a*b+c by default on aarch64).
 *
 * Readings of the paper that this file fixes (where the paper is silent or
 * ambiguous):
 *  - regions are painted in order, later regions overwrite earlier ones;
 *    region 0 is the phantom's outer boundary (the "hull");
 *  - rand() is replaced by the counter-based Philox4x64-10 generator of
 *    Salmon et al. (SC'11); key = (seed, stream), counter = (row, block, 0, 0);
 *  - the polar method keeps the paper's order: two uniforms -> two
 *    independent normals -> bivariate pair through the Cholesky factor of the
 *    covariance (Sec. II-B, bivariate normal density and BNRNG);
 *  - the logarithm inside the polar method is our own (argument reduction by
 *    frexp + the atanh series), so that two machines give identical bits;
 *  - a path is a polyline: a straight lead-in along the entry direction, the
 *    hull chord (straight) or the cubic Hermite spline sampled at K pieces,
 *    and a straight lead-out along the exit direction (Sec. II-B);
 *  - a_ij is the length of the polyline inside voxel j, found per segment
 *    from the sorted plane-crossing parameters (Sec. II-C); consecutive
 *    entries of one voxel across a polyline joint are merged;
 *  - b_i uses the exact lengths even when A stores the constant chord h.
 */
#include "pct_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers:
 * as easy as 1, 2, 3"): 10 rounds of two 64x64->128 multiplies; the key is
 * bumped by the Weyl constants (golden ratio, sqrt(3)-1) between rounds.     */
/* ------------------------------------------------------------------------- */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform on (0,1): the top 53 bits of a word, centred in their cell */
double orc_uniform(uint64_t seed, uint64_t stream, uint64_t row, uint64_t j) {
  uint64_t ctr[4] = {row, j / 4, 0, 0};
  uint64_t key[2] = {seed, stream};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  uint64_t w = out[j % 4];
  return ((double)(w >> 11) + 0.5) * 0x1p-53;
}

/* ------------------------------------------------------------------------- */
/* Natural logarithm by argument reduction and the atanh series:             */
/*   x = f 2^e with f in [sqrt(1/2), sqrt(2)),  u = f - 1 (exact),           */
/*   y = u / (f + 1),  ln f = 2 atanh(y) = 2y + 2y (y^2/3 + y^4/5 + ...),     */
/*   ln x = e ln2 + ln f with ln 2 split into a high part whose products with */
/*   e are exact and a low part (Cody & Waite, 1980).  |y| <= 0.1716, so the  */
/*   series is cut after y^24/25 (relative remainder below 2^-64).           */
/* ------------------------------------------------------------------------- */
static const double LN2_HI = 0x1.62e42fee00000p-1;  /* ln 2, top 32 bits */
static const double LN2_LO = 0x1.a39ef35793c76p-33; /* ln 2 - LN2_HI    */

double orc_log(double x) {
  int e;
  double f = frexp(x, &e); /* x = f * 2^e, f in [0.5, 1) */
  if (f < 0.70710678118654752440) {
    f = f * 2.0;
    e = e - 1;
  }
  double u = f - 1.0;
  double y = u / (f + 1.0);
  double y2 = y * y;
  double q = 1.0 / 25.0;
  for (int k = 11; k >= 1; --k) q = fma(q, y2, 1.0 / (double)(2 * k + 1));
  double ty = 2.0 * y;
  double lnf = fma(ty, y2 * q, ty);
  double de = (double)e;
  return fma(de, LN2_HI, fma(de, LN2_LO, lnf));
}

/* Marsaglia polar method, the paper's normal generator (Sec. II-B): draw
 * v1, v2 uniform on (-1,1) until 0 < s = v1^2 + v2^2 < 1, then
 * (z1, z2) = (v1, v2) sqrt(-2 ln s / s).  Attempts are capped at 64 (the
 * chance of reaching the cap is 0.2146^64 < 1e-42); a capped pair is (0,0). */
uint64_t orc_normal_pairs(uint64_t seed, uint64_t stream, uint64_t row, uint64_t j0,
                          int32_t n_pairs, double* z) {
  uint64_t j = j0;
  for (int32_t q = 0; q < n_pairs; ++q) {
    double z1 = 0.0, z2 = 0.0;
    for (int attempt = 0; attempt < 64; ++attempt) {
      double u1 = orc_uniform(seed, stream, row, j);
      double u2 = orc_uniform(seed, stream, row, j + 1);
      j += 2;
      double v1 = 2.0 * u1 - 1.0;
      double v2 = 2.0 * u2 - 1.0;
      double s = v1 * v1 + v2 * v2;
      if (s > 0.0 && s < 1.0) {
        double f = sqrt((-2.0 * orc_log(s)) / s);
        z1 = v1 * f;
        z2 = v2 * f;
        break;
      }
    }
    z[2 * q] = z1;
    z[2 * q + 1] = z2;
  }
  return j;
}

/* ------------------------------------------------------------------------- */
/* Grid and phantom                                                          */
/* ------------------------------------------------------------------------- */
typedef struct {
  int dim;
  int n[3];
  double h[3];
  double o[3]; /* lower corner: -n h / 2 */
} grid_t;

static grid_t grid_of(const orc_phantom* ph) {
  grid_t g;
  g.dim = ph->dim;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = ph->n[a];
    g.h[a] = ph->h[a];
    g.o[a] = -0.5 * ((double)ph->n[a] * ph->h[a]);
  }
  return g;
}

/* point-in-region test: sum of ((p - c)/a)^2 over the tested axes <= 1 */
static int inside(const orc_phantom* ph, int32_t r, const double p[3]) {
  const double* R = ph->regions + 7 * r;
  int axes = (ph->dim == 3 && ph->kind == ORC_ELLIPSOID) ? 3 : 2;
  double q = 0.0;
  for (int a = 0; a < axes; ++a) {
    double d = (p[a] - R[a]) / R[3 + a];
    q = q + d * d;
  }
  return q <= 1.0;
}

/* RSP at a point: the last region containing it (painter's order), else 0 */
static double rsp_at(const orc_phantom* ph, const double p[3]) {
  double v = 0.0;
  for (int32_t r = 0; r < ph->n_regions; ++r)
    if (inside(ph, r, p)) v = ph->regions[7 * r + 6];
  return v;
}

/* the last region containing a point (painter's order), else -1 */
static int32_t region_at(const orc_phantom* ph, const double p[3]) {
  int32_t v = -1;
  for (int32_t r = 0; r < ph->n_regions; ++r)
    if (inside(ph, r, p)) v = r;
  return v;
}

/* Sec. II-A: centre-point, corner-point-average or weighted-area RSP of every voxel */
void orc_raster(const orc_phantom* ph, double* x) {
  grid_t g = grid_of(ph);
  int nz = (g.dim == 3) ? g.n[2] : 1;
  int ncorner = (g.dim == 3) ? 8 : 4;
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < g.n[1]; ++iy)
      for (int ix = 0; ix < g.n[0]; ++ix) {
        int idx[3] = {ix, iy, iz};
        int64_t j = ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz);
        double p[3] = {0.0, 0.0, 0.0};
        if (ph->raster == ORC_CENTER) {
          for (int a = 0; a < g.dim; ++a) p[a] = g.o[a] + ((double)idx[a] + 0.5) * g.h[a];
          x[j] = rsp_at(ph, p);
        } else if (ph->raster == ORC_AREA) {
          /* area fractions from the sub-sample midpoints
             p_a = o_a + (i_a + (k_a + 1/2) / S) h_a, k_a = 0 .. S - 1 */
          int S = ph->area_samples;
          int64_t cnt[64];
          for (int r = 0; r < ph->n_regions; ++r) cnt[r] = 0;
          int kzn = (g.dim == 3) ? S : 1;
          for (int kz = 0; kz < kzn; ++kz)
            for (int ky = 0; ky < S; ++ky)
              for (int kx = 0; kx < S; ++kx) {
                int k[3] = {kx, ky, kz};
                for (int a = 0; a < g.dim; ++a)
                  p[a] = g.o[a] + ((double)idx[a] + ((double)k[a] + 0.5) / (double)S) * g.h[a];
                int32_t r = region_at(ph, p);
                if (r >= 0) cnt[r]++;
              }
          double nsub = (double)S * (double)S * (g.dim == 3 ? (double)S : 1.0);
          double sum = 0.0;
          for (int r = 0; r < ph->n_regions; ++r) sum = sum + ph->regions[7 * r + 6] * (double)cnt[r];
          x[j] = sum / nsub;
        } else {
          double sum = 0.0;
          for (int c = 0; c < ncorner; ++c) {
            for (int a = 0; a < g.dim; ++a)
              p[a] = g.o[a] + (double)(idx[a] + ((c >> a) & 1)) * g.h[a];
            sum = sum + rsp_at(ph, p);
          }
          x[j] = sum * (1.0 / (double)ncorner);
        }
      }
}

/* line A + lam g against region r: ((A + lam g - c)/a)^2 summed = 1 is
 * alpha lam^2 + 2 beta lam + gamma = 0 with e = g/a, f = (A - c)/a.         */
int orc_hull_hit(const orc_phantom* ph, int32_t r, const double A[3], const double g[3],
                 double* lam_in, double* lam_out) {
  const double* R = ph->regions + 7 * r;
  int axes = (ph->dim == 3 && ph->kind == ORC_ELLIPSOID) ? 3 : 2;
  double alpha = 0.0, beta = 0.0, gamma = 0.0;
  for (int a = 0; a < axes; ++a) {
    double ra = 1.0 / R[3 + a];
    double e = g[a] * ra;
    double f = (A[a] - R[a]) * ra;
    alpha = alpha + e * e;
    beta = beta + e * f;
    gamma = gamma + f * f;
  }
  gamma = gamma - 1.0;
  double delta = beta * beta - alpha * gamma;
  if (!(alpha > 0.0) || !(delta > 0.0)) return 0;
  double sq = sqrt(delta);
  double ia = 1.0 / alpha;
  *lam_in = (-beta - sq) * ia;
  *lam_out = (-beta + sq) * ia;
  return 1;
}

/* ------------------------------------------------------------------------- */
/* One segment through the voxel grid (Sec. II-C).                           */
/*                                                                           */
/* For an axis a with D_a = Q_a - P_a != 0 the crossing parameter of plane k  */
/* (k = 0..n_a, plane at o_a + k h_a) is                                     */
/*     sigma_a(k) = fma(k, h_a / D_a, (o_a - P_a) / D_a)                      */
/* with the reciprocal 1/D_a formed once.  The segment is inside the grid for */
/* sigma in (s_in, s_out), the intersection of [0,1] with every axis' slab.  */
/* The crossings strictly inside, sorted, cut it into intervals; interval m  */
/* lies in the voxel whose index along a is (planes with sigma <= its start) */
/* - 1 for D_a > 0, or n_a - (that count) for D_a < 0.  Its chord length is  */
/* |Q - P| times its parameter width.                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
  double s;
  int axis;
} event_t;

static int cmp_event(const void* a, const void* b) {
  double x = ((const event_t*)a)->s, y = ((const event_t*)b)->s;
  if (x < y) return -1;
  if (x > y) return 1;
  return ((const event_t*)a)->axis - ((const event_t*)b)->axis;
}

static int64_t segment_grid(const grid_t* g, const double P[3], const double Q[3],
                            int32_t* cols, double* lens, int64_t cap) {
  int dim = g->dim;
  double D[3] = {0, 0, 0}, inv[3] = {0, 0, 0}, dl[3] = {0, 0, 0}, s0[3] = {0, 0, 0};
  int idx[3] = {0, 0, 0}, active[3] = {0, 0, 0};
  double s_in = 0.0, s_out = 1.0;
  for (int a = 0; a < dim; ++a) {
    D[a] = Q[a] - P[a];
    if (D[a] == 0.0) {
      double fl = floor((P[a] - g->o[a]) / g->h[a]);
      if (fl < 0.0 || fl >= (double)g->n[a]) return 0;
      idx[a] = (int)fl;
    } else {
      active[a] = 1;
      inv[a] = 1.0 / D[a];
      dl[a] = g->h[a] * inv[a];
      s0[a] = (g->o[a] - P[a]) * inv[a];
      double sa = s0[a];
      double sb = fma((double)g->n[a], dl[a], s0[a]);
      double lo = sa < sb ? sa : sb;
      double hi = sa < sb ? sb : sa;
      if (lo > s_in) s_in = lo;
      if (hi < s_out) s_out = hi;
    }
  }
  if (!(s_in < s_out)) return 0;

  double len2 = 0.0;
  for (int a = 0; a < dim; ++a) len2 = len2 + D[a] * D[a];
  double seglen = sqrt(len2);

  int64_t max_ev = 0;
  for (int a = 0; a < dim; ++a)
    if (active[a]) max_ev += g->n[a] + 1;
  event_t* ev = (event_t*)malloc(sizeof(event_t) * (size_t)(max_ev > 0 ? max_ev : 1));
  int64_t nev = 0;
  for (int a = 0; a < dim; ++a) {
    if (!active[a]) continue;
    int64_t cnt = 0;
    for (int k = 0; k <= g->n[a]; ++k) {
      double s = fma((double)k, dl[a], s0[a]);
      if (s <= s_in) {
        cnt++;
      } else if (s < s_out) {
        ev[nev].s = s;
        ev[nev].axis = a;
        nev++;
      }
    }
    idx[a] = (D[a] > 0.0) ? (int)(cnt - 1) : (int)(g->n[a] - cnt);
  }
  qsort(ev, (size_t)nev, sizeof(event_t), cmp_event);

  int64_t m = 0;
  double s_prev = s_in;
  int64_t e = 0;
  for (;;) {
    double s_next = (e < nev) ? ev[e].s : s_out;
    for (int a = 0; a < dim; ++a) {
      if (idx[a] < 0 || idx[a] >= g->n[a]) {
        fprintf(stderr, "orc_segment: voxel index out of range (axis %d: %d)\n", a, idx[a]);
        abort();
      }
    }
    if (m < cap) {
      int64_t col = idx[0] + (int64_t)g->n[0] * (idx[1] + (int64_t)g->n[1] * (dim == 3 ? idx[2] : 0));
      cols[m] = (int32_t)col;
      lens[m] = seglen * (s_next - s_prev);
    }
    m++;
    if (e >= nev) break;
    /* every crossing at exactly this parameter moves its axis */
    while (e < nev && ev[e].s == s_next) {
      int a = ev[e].axis;
      idx[a] += (D[a] > 0.0) ? 1 : -1;
      e++;
    }
    s_prev = s_next;
  }
  free(ev);
  return m;
}

int64_t orc_segment(const orc_phantom* ph, const double P[3], const double Q[3],
                    int32_t* cols, double* lens, int64_t cap) {
  grid_t g = grid_of(ph);
  return segment_grid(&g, P, Q, cols, lens, cap);
}

/* ------------------------------------------------------------------------- */
/* Proton path (Sec. II-B)                                                   */
/*                                                                           */
/* Beam frame of angle theta: u = (cos, sin, 0) the beam direction,          */
/* t = (-sin, cos, 0) lateral, v = (0, 0, 1) vertical (Givens rotation about  */
/* z, Sec. II-C).  Uniform 0 -> t offset, uniform 1 -> v offset (3D); normals */
/* from uniform 4 on, in pairs: [MCS] exit ut-plane (displacement, slope),   */
/* [MCS, 3D] exit uv-plane, [MCS] entry slopes (t, v), [noise] (z, unused).  */
/* Entry direction g0 = u + slope_in_t t + slope_in_v v (not normalised).    */
/* Hull entry P0 / straight exit Q1 from region 0; exit P1 = Q1 + d_t n_t +  */
/* d_v n_v with n_t = (-g0y, g0x, 0), n_v = g0 x n_t; exit direction          */
/* g1 = g0 + slope_out_t n_t + slope_out_v n_v.  Spline: Hermite from P0 to  */
/* P1 with tangents l g0, l g1, l = (P1 - P0).g0, sampled at s = j/K.        */
/* Lead-in / lead-out: straight, 2 x grid diagonal long.  A line that misses */
/* the hull (or the STRAIGHT model) is one straight segment through A.       */
/* ------------------------------------------------------------------------- */
typedef struct {
  double t, v;
  double zt1, zt2, zv1, zv2;  /* exit pairs (ut-plane, uv-plane), standard normals */
  double in_t, in_v;
  double z_noise;
} draws_t;

/* Highland's formula with the PDG constants (Sec. II-B): theta0 =
   13.6 MeV / (beta c p) sqrt(x / X0) (1 + 0.038 ln(x / (X0 beta^2))) for a
   singly charged particle; beta c p = (pc)^2 / E with (pc)^2 = T (T + 2 m),
   E = T + m, m = 938.272088 MeV (proton). */
static const double ORC_MP_MEV = 938.272088;
double orc_highland(double beam_mev, double x0_mm, double x_mm, double* beta_cp) {
  double E = beam_mev + ORC_MP_MEV;
  double pc2 = beam_mev * (beam_mev + 2.0 * ORC_MP_MEV);
  double bcp = pc2 / E;
  double beta2 = pc2 / (E * E);
  if (beta_cp) *beta_cp = bcp;
  double t = x_mm / x0_mm;
  return (13.6 / bcp) * sqrt(t) * (1.0 + 0.038 * orc_log(t / beta2));
}

static draws_t draw_row(const orc_sim* sim, int64_t row) {
  const orc_model* md = sim->model;
  int dim = sim->ph->dim;
  draws_t d;
  memset(&d, 0, sizeof(d));
  double u0 = orc_uniform(sim->seed, sim->stream, (uint64_t)row, 0);
  d.t = md->t_lo + (md->t_hi - md->t_lo) * u0;
  if (dim == 3) {
    double u1 = orc_uniform(sim->seed, sim->stream, (uint64_t)row, 1);
    d.v = md->v_lo + (md->v_hi - md->v_lo) * u1;
  }
  uint64_t j = 4;
  double z[2];
  if (md->model != ORC_STRAIGHT) {
    j = orc_normal_pairs(sim->seed, sim->stream, (uint64_t)row, j, 1, z);
    d.zt1 = z[0];
    d.zt2 = z[1];
    if (dim == 3) {
      j = orc_normal_pairs(sim->seed, sim->stream, (uint64_t)row, j, 1, z);
      d.zv1 = z[0];
      d.zv2 = z[1];
    }
    j = orc_normal_pairs(sim->seed, sim->stream, (uint64_t)row, j, 1, z);
    d.in_t = md->sigma_in * z[0];
    d.in_v = md->sigma_in * z[1];
  }
  if (md->noise == ORC_NOISE_GAUSS_REL) {
    j = orc_normal_pairs(sim->seed, sim->stream, (uint64_t)row, j, 1, z);
    d.z_noise = z[0];
  }
  return d;
}

static double grid_diag(const grid_t* g) {
  double s = 0.0;
  for (int a = 0; a < g->dim; ++a) {
    double w = (double)g->n[a] * g->h[a];
    s = s + w * w;
  }
  return sqrt(s);
}

int32_t orc_path(const orc_sim* sim, int64_t row, double* verts, int32_t cap) {
  const orc_phantom* ph = sim->ph;
  const orc_model* md = sim->model;
  grid_t g = grid_of(ph);
  int dim = g.dim;
  int64_t k = row / sim->paths_per_angle;
  double c = cos(sim->angles[k]);
  double s = sin(sim->angles[k]);
  draws_t d = draw_row(sim, row);
  double R = 2.0 * grid_diag(&g);

  double A[3] = {-s * d.t, c * d.t, (dim == 3) ? d.v : 0.0};
  double g0[3];
  if (md->model == ORC_STRAIGHT) {
    g0[0] = c;
    g0[1] = s;
    g0[2] = 0.0;
  } else {
    g0[0] = c - d.in_t * s;
    g0[1] = s + d.in_t * c;
    g0[2] = (dim == 3) ? d.in_v : 0.0;
  }

  double V[4096][3];
  int32_t nv = 0;
  double lam_in = 0.0, lam_out = 0.0;
  int hit = (md->model != ORC_STRAIGHT) && ph->n_regions > 0 &&
            orc_hull_hit(ph, 0, A, g0, &lam_in, &lam_out);
  if (!hit) {
    for (int a = 0; a < 3; ++a) {
      V[0][a] = A[a] - R * g0[a];
      V[1][a] = A[a] + R * g0[a];
    }
    nv = 2;
  } else {
    double P0[3], Q1[3], P1[3], g1[3], nt[3], nvv[3];
    for (int a = 0; a < 3; ++a) {
      P0[a] = A[a] + lam_in * g0[a];
      Q1[a] = A[a] + lam_out * g0[a];
    }
    /* exit pair widths and correlation: fixed by the model, or (Highland)
       from the chord x through the hull: sigma_angle = theta0(x), sigma_lat
       = x theta0 / sqrt(3), correlation sqrt(3) / 2 (thin-slab MCS) */
    double s_lat = md->sigma_lat, s_ang = md->sigma_out, rho = md->rho;
    if (md->mcs == ORC_MCS_HIGHLAND) {
      double gl2 = 0.0;
      for (int a = 0; a < dim; ++a) gl2 = gl2 + g0[a] * g0[a];
      double x = (lam_out - lam_in) * sqrt(gl2);
      s_ang = orc_highland(md->beam_mev, md->x0_mm, x, NULL);
      s_lat = x * s_ang * (1.0 / sqrt(3.0));
      rho = 0.5 * sqrt(3.0);
    }
    double rc = sqrt(1.0 - rho * rho);
    double lat_t = s_lat * d.zt1;
    double ang_t = s_ang * (rho * d.zt1 + rc * d.zt2);
    double lat_v = s_lat * d.zv1;
    double ang_v = s_ang * (rho * d.zv1 + rc * d.zv2);
    nt[0] = -g0[1];
    nt[1] = g0[0];
    nt[2] = 0.0;
    if (dim == 3) {
      nvv[0] = -(g0[2] * g0[0]);
      nvv[1] = -(g0[2] * g0[1]);
      nvv[2] = g0[0] * g0[0] + g0[1] * g0[1];
      for (int a = 0; a < 3; ++a) {
        P1[a] = (Q1[a] + lat_t * nt[a]) + lat_v * nvv[a];
        g1[a] = (g0[a] + ang_t * nt[a]) + ang_v * nvv[a];
      }
    } else {
      for (int a = 0; a < 2; ++a) {
        P1[a] = Q1[a] + lat_t * nt[a];
        g1[a] = g0[a] + ang_t * nt[a];
      }
      P1[2] = 0.0;
      g1[2] = 0.0;
    }
    for (int a = 0; a < 3; ++a) V[0][a] = P0[a] - R * g0[a];
    for (int a = 0; a < 3; ++a) V[1][a] = P0[a];
    nv = 2;
    if (md->model == ORC_SPLINE) {
      int K = md->spline_segments;
      double l = 0.0;
      for (int a = 0; a < dim; ++a) l = l + (P1[a] - P0[a]) * g0[a];
      double m0[3], m1[3];
      for (int a = 0; a < 3; ++a) {
        m0[a] = l * g0[a];
        m1[a] = l * g1[a];
      }
      for (int jv = 1; jv < K; ++jv) {
        double sp = (double)jv / (double)K;
        double s2 = sp * sp;
        double s3 = s2 * sp;
        double h00 = (2.0 * s3 - 3.0 * s2) + 1.0;
        double h10 = (s3 - 2.0 * s2) + sp;
        double h01 = 3.0 * s2 - 2.0 * s3;
        double h11 = s3 - s2;
        for (int a = 0; a < 3; ++a)
          V[nv][a] = ((h00 * P0[a] + h10 * m0[a]) + h01 * P1[a]) + h11 * m1[a];
        if (dim == 2) V[nv][2] = 0.0;
        nv++;
      }
    }
    for (int a = 0; a < 3; ++a) V[nv][a] = P1[a];
    nv++;
    for (int a = 0; a < 3; ++a) V[nv][a] = P1[a] + R * g1[a];
    nv++;
  }
  for (int32_t i = 0; i < nv && i < cap; ++i)
    for (int a = 0; a < 3; ++a) verts[3 * i + a] = V[i][a];
  return nv;
}

/* ------------------------------------------------------------------------- */
/* Row i of A and its WEPL b_i (Sec. II-C)                                   */
/* ------------------------------------------------------------------------- */
int64_t orc_row(const orc_sim* sim, int64_t row, int32_t* cols, double* vals,
                int64_t cap, double* b_clean, double* b_noisy) {
  const orc_phantom* ph = sim->ph;
  const orc_model* md = sim->model;
  grid_t g = grid_of(ph);
  int32_t K = (md->model == ORC_SPLINE) ? md->spline_segments : 1;
  if (K < 1 || K > 4000) {
    fprintf(stderr, "orc_row: spline_segments out of range\n");
    abort();
  }
  double* verts = (double*)malloc(sizeof(double) * 3 * (size_t)(K + 4));
  int32_t nv = orc_path(sim, row, verts, K + 4);

  int64_t seg_cap = 0;
  for (int a = 0; a < g.dim; ++a) seg_cap += g.n[a];
  seg_cap += 2;
  int32_t* sc = (int32_t*)malloc(sizeof(int32_t) * (size_t)seg_cap);
  double* sl = (double*)malloc(sizeof(double) * (size_t)seg_cap);

  int64_t buf_cap = 1024;
  int32_t* rc = (int32_t*)malloc(sizeof(int32_t) * (size_t)buf_cap);
  double* rl = (double*)malloc(sizeof(double) * (size_t)buf_cap);
  int64_t m = 0;
  int prev_nonempty = 0;
  for (int32_t sg = 0; sg + 1 < nv; ++sg) {
    int64_t ns = segment_grid(&g, verts + 3 * sg, verts + 3 * (sg + 1), sc, sl, seg_cap);
    if (ns > seg_cap) {
      fprintf(stderr, "orc_row: segment longer than its bound\n");
      abort();
    }
    for (int64_t q = 0; q < ns; ++q) {
      if (q == 0 && prev_nonempty && m > 0 && rc[m - 1] == sc[0]) {
        rl[m - 1] = rl[m - 1] + sl[0];
        continue;
      }
      if (m == buf_cap) {
        buf_cap *= 2;
        rc = (int32_t*)realloc(rc, sizeof(int32_t) * (size_t)buf_cap);
        rl = (double*)realloc(rl, sizeof(double) * (size_t)buf_cap);
      }
      rc[m] = sc[q];
      rl[m] = sl[q];
      m++;
    }
    prev_nonempty = ns > 0;
  }

  double b = 0.0;
  for (int64_t q = 0; q < m; ++q) b = b + rl[q] * (double)sim->x_true[rc[q]];
  double bn = b;
  if (md->noise == ORC_NOISE_GAUSS_REL) {
    draws_t d = draw_row(sim, row);
    bn = b * (1.0 + md->noise_rel * d.z_noise);
  }
  if (b_clean) *b_clean = b;
  if (b_noisy) *b_noisy = bn;
  for (int64_t q = 0; q < m && q < cap; ++q) {
    cols[q] = rc[q];
    vals[q] = (md->chord == ORC_CHORD_CONSTANT) ? ph->h[0] : rl[q];
  }
  free(rc);
  free(rl);
  free(sc);
  free(sl);
  free(verts);
  return m;
}

void orc_count_rows(const orc_sim* sim, const int64_t* rows, int64_t n, int64_t* counts,
                    int32_t threads) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads > 0 ? threads : 1)
  for (int64_t q = 0; q < n; ++q) counts[q] = orc_row(sim, rows[q], NULL, NULL, 0, NULL, NULL);
}

void orc_fill_rows(const orc_sim* sim, const int64_t* rows, int64_t n, const int64_t* off,
                   int32_t* cols, double* vals, double* b_clean, double* b_noisy,
                   int32_t threads) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads > 0 ? threads : 1)
  for (int64_t q = 0; q < n; ++q) {
    double bc, bn;
    orc_row(sim, rows[q], cols + off[q], vals + off[q], (int64_t)1 << 40, &bc, &bn);
    if (b_clean) b_clean[q] = bc;
    if (b_noisy) b_noisy[q] = bn;
  }
}

/* ------------------------------------------------------------------------- */
/* Reconstruction: string-averaging projections (Sec. II-D, SAP)             */
/*                                                                           */
/* The paper's update reads <a^i, x_k> and adds lambda (<a^i, x_k> - b_i);   */
/* here the projection of the current string iterate y onto row i's         */
/* hyperplane is taken: y + lambda (b_i - <a_i, y>) / ||a_i||^2 a_i (Censor's */
/* SAP; with lambda = 1 the new y satisfies row i exactly).  Each string     */
/* starts from x; x becomes the weighted average of the string ends.         */
/* ------------------------------------------------------------------------- */
void orc_sap(int64_t n_rows, int64_t n_cols, const int64_t* row_ptr, const int32_t* col,
             const double* val, const double* b, int32_t M, const double* w, double lambda,
             int32_t iterations, double* x) {
  if (M < 1 || n_cols < 1) return;
  double* y = (double*)malloc(sizeof(double) * (size_t)n_cols);
  double* acc = (double*)malloc(sizeof(double) * (size_t)n_cols);
  for (int32_t it = 0; it < iterations; ++it) {
    for (int64_t j = 0; j < n_cols; ++j) acc[j] = 0.0;
    for (int32_t t = 0; t < M; ++t) {
      for (int64_t j = 0; j < n_cols; ++j) y[j] = x[j];
      for (int64_t i = t; i < n_rows; i += M) {
        double dot = 0.0, nrm = 0.0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
          dot = dot + val[q] * y[col[q]];
          nrm = nrm + val[q] * val[q];
        }
        if (!(nrm > 0.0)) continue;
        double c = lambda * (b[i] - dot) / nrm;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) y[col[q]] = y[col[q]] + c * val[q];
      }
      double wt = w ? w[t] : 1.0 / (double)M;
      for (int64_t j = 0; j < n_cols; ++j) acc[j] = acc[j] + wt * y[j];
    }
    for (int64_t j = 0; j < n_cols; ++j) x[j] = acc[j];
  }
  free(y);
  free(acc);
}
