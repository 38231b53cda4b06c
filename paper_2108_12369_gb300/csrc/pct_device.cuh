// pct_device.cuh -- device-side definitions shared by the libpct kernels:
// kernel-argument structs, the Philox4x64-10 generator, the logarithm and
// normal draws, the proton path set-up, and the FP64 voxel traversal.
//
// Every FP64 expression here is the definition the simulator computes; the
// library is compiled with -fmad=false so that no a*b+c is fused unless it
// is written as fma().  The FP32 fast path (pct_mixed.cuh) reproduces these
// decisions exactly and falls back to the functions below when its error
// bounds cannot decide.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/pct.h"

namespace pct {

constexpr int kMaxRegions = PCT_MAX_REGIONS;

// ---------------------------------------------------------------------------
// Kernel arguments (passed by value; a few KB at most)
// ---------------------------------------------------------------------------
struct GridDev {
  int dim;
  int n[3];
  double h[3];
  double o[3];  // lower corner, -n h / 2
};

struct PhantomDev {
  GridDev g;
  int kind, raster, n_regions;
  int area_s;  // weighted-area raster: sub-samples per axis
  double c[kMaxRegions][3];
  double a[kMaxRegions][3];
  double ra[kMaxRegions][3];  // 1 / a, formed on the host (IEEE division)
  double rsp[kMaxRegions];
};

struct ModelDev {
  int model, chord, K, noise;
  double t_lo, t_hi, v_lo, v_hi;
  double t_span, v_span;  // t_hi - t_lo, v_hi - v_lo (formed on the host, the same FP64 values)
  double sigma_lat, sigma_in, sigma_out, rho, rho_c;  // rho_c = sqrt(1 - rho^2)
  double noise_rel;
  // PCT_MCS_HIGHLAND: widths from the chord x through the hull, with host
  // constants hl_k = 13.6 / (beta c p), hl_x0, hl_beta2, hl_s3 = 1 / sqrt(3),
  // hl_rho = sqrt(3) / 2, hl_rho_c = sqrt(1 - hl_rho^2)
  int mcs;
  double hl_k, hl_x0, hl_beta2, hl_s3, hl_rho, hl_rho_c;
};

// cubic Hermite basis at one sample s = j / K
struct alignas(32) Basis4 {
  double h00, h10, h01, h11;
};

struct SimDev {
  PhantomDev ph;
  ModelDev md;
  int n_angles;
  long long P;  // paths per angle
  unsigned long long seed, stream;
  long long first_row;    // global index of row 0 (the generator's counter)
  double R;               // lead-in / lead-out length: 2 x grid diagonal
  const double2* cs;      // [n_angles] (cos, sin) from the host's libm
  const Basis4* basis;    // [K + 1] Hermite basis at s = j / K
  // rows whose fill wrote a different number of entries than row_ptr gives
  // them (the workspace's first word; zeroed by the count)
  unsigned long long* status;
};

// a row of the fill whose entry count differs from its row_ptr range
__device__ __forceinline__ void note_row_mismatch(const SimDev& S) {
  if (S.status) atomicAdd(S.status, 1ULL);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11).  key = (seed, stream),
// counter = (global row, block, 0, 0); uniform = (top 53 bits + 1/2) * 2^-53.
// ---------------------------------------------------------------------------
struct U4 {
  unsigned long long w[4];
};

__device__ __forceinline__ U4 philox4x64_10(unsigned long long c0, unsigned long long c1,
                                            unsigned long long c2, unsigned long long c3,
                                            unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  U4 o;
  o.w[0] = c0;
  o.w[1] = c1;
  o.w[2] = c2;
  o.w[3] = c3;
  return o;
}

// ((double)m + 0.5) * 2^-53 for m = w >> 11 < 2^53, assembled with integer
// operations (the FP64 pipe is this kernel's bottleneck) and bit-identical
// to that FP64 expression: for m < 2^52 the sum is exact, (2m + 1) 2^-54;
// above, m + 0.5 is a tie between m and m + 1 and rounds to the even one.
__device__ __forceinline__ double word_to_uniform(unsigned long long w) {
  const unsigned long long m = w >> 11;
  const bool exact = m < (1ULL << 52);
  const unsigned long long v = exact ? 2 * m + 1 : m + (m & 1ULL);  // value = v 2^-k, 0 < v <= 2^53
  const int k = exact ? 54 : 53;
  const int e = 63 - __clzll((long long)v);  // v in [2^e, 2^(e + 1))
  const unsigned long long mant = e >= 52 ? v >> (e - 52) : v << (52 - e);
  const unsigned long long bits =
      ((unsigned long long)(e - k + 1023) << 52) | (mant & ((1ULL << 52) - 1ULL));
  return __longlong_as_double((long long)bits);
}

// 2 u - 1 for u = word_to_uniform(w), which that FP64 expression forms
// exactly (for u < 1/2, 2u - 1 = (2m + 1 - 2^53) 2^-53, an integer of at most
// 53 bits; for u >= 1/2, Sterbenz), assembled with integer operations.
__device__ __forceinline__ double word_to_sym(unsigned long long w) {
  const unsigned long long m = w >> 11;
  const bool exact = m < (1ULL << 52);
  // magnitude n 2^-k, negative below 1/2
  const unsigned long long n = exact ? (1ULL << 53) - 1ULL - 2 * m : m + (m & 1ULL) - (1ULL << 52);
  const int k = exact ? 53 : 52;
  if (n == 0ULL) return 0.0;
  const int e = 63 - __clzll((long long)n);  // n in [2^e, 2^(e + 1)), e <= 52
  const unsigned long long mant = n << (52 - e);
  const unsigned long long bits = (exact ? (1ULL << 63) : 0ULL) | ((unsigned long long)(e - k + 1023) << 52) |
                                  (mant & ((1ULL << 52) - 1ULL));
  return __longlong_as_double((long long)bits);
}

// Sequential reader of one proton's uniform stream U_0, U_1, ...
struct UniformStream {
  unsigned long long row, k0, k1;
  long long block;
  U4 buf;
  __device__ void init(unsigned long long r, unsigned long long seed, unsigned long long stream) {
    row = r;
    k0 = seed;
    k1 = stream;
    block = -1;
  }
  __device__ double get(long long j) {
    long long b = j >> 2;
    if (b != block) {
      buf = philox4x64_10(row, (unsigned long long)b, 0ULL, 0ULL, k0, k1);
      block = b;
    }
    const int w = (int)(j & 3);
    unsigned long long x = buf.w[0];
    x = (w == 1) ? buf.w[1] : x;
    x = (w == 2) ? buf.w[2] : x;
    x = (w == 3) ? buf.w[3] : x;
    return word_to_uniform(x);
  }
  // 2 U_j - 1, the same FP64 value, without FP64 arithmetic
  __device__ double get_sym(long long j) {
    long long b = j >> 2;
    if (b != block) {
      buf = philox4x64_10(row, (unsigned long long)b, 0ULL, 0ULL, k0, k1);
      block = b;
    }
    const int w = (int)(j & 3);
    unsigned long long x = buf.w[0];
    x = (w == 1) ? buf.w[1] : x;
    x = (w == 2) ? buf.w[2] : x;
    x = (w == 3) ? buf.w[3] : x;
    return word_to_sym(x);
  }
};

// ---------------------------------------------------------------------------
// Natural logarithm (atanh series after argument reduction; Cody-Waite
// split of ln 2).  Same operations, in the same order, as the definition.
// ---------------------------------------------------------------------------
// Its argument is positive and normal (s of the polar method): frexp and the
// exact doubling are done on the bits (same values, no FP64 instructions).
__device__ __forceinline__ double own_log(double x) {
  const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
  int e = (int)((xb >> 52) & 0x7ffULL) - 1022;                       // x = f 2^e, f in [1/2, 1)
  unsigned long long fb = (xb & 0x800fffffffffffffULL) | (1022ULL << 52);
  if (fb < 0x3fe6a09e667f3bcdULL) {  // f < 0.70710678118654752440 (positive doubles order as integers)
    fb += 1ULL << 52;                 // f * 2
    e = e - 1;
  }
  const double f = __longlong_as_double((long long)fb);
  double u = f - 1.0;
  double y = u / (f + 1.0);
  double y2 = y * y;
  double q = 1.0 / 25.0;
#pragma unroll
  for (int k = 11; k >= 1; --k) q = fma(q, y2, 1.0 / (double)(2 * k + 1));
  double ty = 2.0 * y;
  double lnf = fma(ty, y2 * q, ty);
  double de = (double)e;
  return fma(de, 0x1.62e42fee00000p-1, fma(de, 0x1.a39ef35793c76p-33, lnf));
}

// Marsaglia polar method (Sec. II-B): pair of independent standard normals
// from the stream starting at uniform j; advances j.  64 attempts at most.
// The accepted point is found first and transformed after the loop: lanes
// accept at different attempts, and a transform inside the loop would run
// once per distinct attempt count in the warp (two to three times).
__device__ __forceinline__ void normal_pair(UniformStream& us, long long& j, double& z1,
                                            double& z2) {
  double v1 = 0.0, v2 = 0.0, s = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 64; ++attempt) {
    v1 = us.get_sym(j);  // 2 U - 1
    v2 = us.get_sym(j + 1);
    j += 2;
    s = v1 * v1 + v2 * v2;
    if (s > 0.0 && s < 1.0) {
      ok = true;
      break;
    }
  }
  z1 = 0.0;
  z2 = 0.0;
  if (ok) {
    double f = sqrt((-2.0 * own_log(s)) / s);
    z1 = v1 * f;
    z2 = v2 * f;
  }
}

// ---------------------------------------------------------------------------
// Proton path (Sec. II-B).  The polyline's vertices:
//   kind 0 (straight, or MCS model missing the hull): A - R g0, A + R g0
//   kind 1 (STRAIGHT_MCS): P0 - R g0, P0, P1, P1 + R g1
//   kind 2 (SPLINE):       P0 - R g0, P0, H(1/K) .. H((K-1)/K), P1, P1 + R g1
// ---------------------------------------------------------------------------
struct PathF64 {
  int kind;
  int nv;  // vertices
  double A[3], g0[3];
  double P0[3], P1[3], g1[3], m0[3], m1[3];
  double z_noise;
};

__device__ __forceinline__ bool hull_hit(const PhantomDev& ph, const double A[3],
                                         const double g[3], double& lam_in, double& lam_out) {
  int axes = (ph.g.dim == 3 && ph.kind == PCT_ELLIPSOID) ? 3 : 2;
  double alpha = 0.0, beta = 0.0, gamma = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= axes) break;
    double e = g[a] * ph.ra[0][a];
    double f = (A[a] - ph.c[0][a]) * ph.ra[0][a];
    alpha = alpha + e * e;
    beta = beta + e * f;
    gamma = gamma + f * f;
  }
  gamma = gamma - 1.0;
  double delta = beta * beta - alpha * gamma;
  if (!(alpha > 0.0) || !(delta > 0.0)) return false;
  double sq = sqrt(delta);
  double ia = 1.0 / alpha;
  lam_in = (-beta - sq) * ia;
  lam_out = (-beta + sq) * ia;
  return true;
}

// DIM: the grid's dimension when known at compile time (0: read from S)
template <int DIM = 0>
__device__ __forceinline__ PathF64 path_setup(const SimDev& S, long long row) {
  const ModelDev& md = S.md;
  const int dim = DIM ? DIM : S.ph.g.dim;
  PathF64 p;
  long long k = row / S.P;
  double2 cs = S.cs[k];
  double c = cs.x, s = cs.y;
  UniformStream us;
  us.init((unsigned long long)(S.first_row + row), S.seed, S.stream);
  double t = md.t_lo + md.t_span * us.get(0);
  double v = 0.0;
  if (dim == 3) v = md.v_lo + md.v_span * us.get(1);
  long long j = 4;
  double zt1 = 0.0, zt2 = 0.0, zv1 = 0.0, zv2 = 0.0, in_t = 0.0, in_v = 0.0;
  double z1, z2;
  if (md.model != PCT_PATH_STRAIGHT) {
    normal_pair(us, j, zt1, zt2);  // exit pair, ut-plane
    if (dim == 3) normal_pair(us, j, zv1, zv2);  // exit pair, uv-plane
    normal_pair(us, j, z1, z2);
    in_t = md.sigma_in * z1;
    in_v = md.sigma_in * z2;
  }
  p.z_noise = 0.0;
  if (md.noise == PCT_NOISE_GAUSS_REL) {
    normal_pair(us, j, z1, z2);
    p.z_noise = z1;
  }

  p.A[0] = -s * t;
  p.A[1] = c * t;
  p.A[2] = (dim == 3) ? v : 0.0;
  if (md.model == PCT_PATH_STRAIGHT) {
    p.g0[0] = c;
    p.g0[1] = s;
    p.g0[2] = 0.0;
  } else {
    p.g0[0] = c - in_t * s;
    p.g0[1] = s + in_t * c;
    p.g0[2] = (dim == 3) ? in_v : 0.0;
  }
  double lam_in = 0.0, lam_out = 0.0;
  bool hit = (md.model != PCT_PATH_STRAIGHT) && S.ph.n_regions > 0 &&
             hull_hit(S.ph, p.A, p.g0, lam_in, lam_out);
  if (!hit) {
    p.kind = 0;
    p.nv = 2;
    return p;
  }
  double Q1[3], nt[3], nv3[3];
  // in 2D the third coordinates are zero (A[2] = g0[2] = 0): not formed
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p.P0[a] = a < dim ? p.A[a] + lam_in * p.g0[a] : 0.0;
    Q1[a] = a < dim ? p.A[a] + lam_out * p.g0[a] : 0.0;
  }
  // exit pair widths: fixed, or (Highland) from the chord x through the hull
  double s_lat = md.sigma_lat, s_ang = md.sigma_out, rho = md.rho, rho_c = md.rho_c;
  if (md.mcs == PCT_MCS_HIGHLAND) {
    double gl2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) gl2 = gl2 + p.g0[a] * p.g0[a];
    const double x = (lam_out - lam_in) * sqrt(gl2);
    const double t = x / md.hl_x0;
    s_ang = md.hl_k * sqrt(t) * (1.0 + 0.038 * own_log(t / md.hl_beta2));
    s_lat = x * s_ang * md.hl_s3;
    rho = md.hl_rho;
    rho_c = md.hl_rho_c;
  }
  const double lat_t = s_lat * zt1, ang_t = s_ang * (rho * zt1 + rho_c * zt2);
  const double lat_v = s_lat * zv1, ang_v = s_ang * (rho * zv1 + rho_c * zv2);
  nt[0] = -p.g0[1];
  nt[1] = p.g0[0];
  nt[2] = 0.0;
  if (dim == 3) {
    nv3[0] = -(p.g0[2] * p.g0[0]);
    nv3[1] = -(p.g0[2] * p.g0[1]);
    nv3[2] = p.g0[0] * p.g0[0] + p.g0[1] * p.g0[1];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p.P1[a] = (Q1[a] + lat_t * nt[a]) + lat_v * nv3[a];
      p.g1[a] = (p.g0[a] + ang_t * nt[a]) + ang_v * nv3[a];
    }
  } else {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      p.P1[a] = Q1[a] + lat_t * nt[a];
      p.g1[a] = p.g0[a] + ang_t * nt[a];
    }
    p.P1[2] = 0.0;
    p.g1[2] = 0.0;
  }
  if (md.model == PCT_PATH_SPLINE) {
    double l = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) l = l + (p.P1[a] - p.P0[a]) * p.g0[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p.m0[a] = a < dim ? l * p.g0[a] : 0.0;
      p.m1[a] = a < dim ? l * p.g1[a] : 0.0;
    }
    p.kind = 2;
    p.nv = md.K + 3;
  } else {
    p.kind = 1;
    p.nv = 4;
  }
  return p;
}

// vertex q of the polyline (0 <= q < nv), FP64
__device__ __forceinline__ void path_vertex(const SimDev& S, const PathF64& p, int q, double V[3]) {
  const double R = S.R;
  if (p.kind == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = (q == 0) ? p.A[a] - R * p.g0[a] : p.A[a] + R * p.g0[a];
    return;
  }
  if (q == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = p.P0[a] - R * p.g0[a];
    return;
  }
  if (q == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = p.P0[a];
    return;
  }
  if (q == p.nv - 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = p.P1[a] + R * p.g1[a];
    return;
  }
  if (q == p.nv - 2) {
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a] = p.P1[a];
    return;
  }
  const Basis4 B = S.basis[q - 1];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    V[a] = ((B.h00 * p.P0[a] + B.h10 * p.m0[a]) + B.h01 * p.P1[a]) + B.h11 * p.m1[a];
  if (S.ph.g.dim == 2) V[2] = 0.0;
}

// ---------------------------------------------------------------------------
// Row assembly: merges the first entry of a segment into the previous
// entry when it is the same voxel and the previous segment ended there.
// Sink::put(col, len) receives the merged entries in path order;
// Sink::pend(col) is told each new pending voxel one step before its put().
// ---------------------------------------------------------------------------
template <class Len>
struct RowMerge {
  int pend_col;
  Len pend_len;
  bool has_pend, prev_nonempty, cur_any;
  __device__ void init() {
    has_pend = false;
    prev_nonempty = false;
    cur_any = false;
  }
  __device__ void seg_begin() { cur_any = false; }
  template <class Sink>
  __device__ void emit(int col, Len len, Sink& sink) {
    if (!cur_any && prev_nonempty && has_pend && col == pend_col) {
      pend_len = pend_len + len;
      cur_any = true;
      return;
    }
    if (has_pend) sink.put(pend_col, pend_len);
    pend_col = col;
    pend_len = len;
    has_pend = true;
    cur_any = true;
    sink.pend(col);  // lets a sink start loading what put() will need
  }
  __device__ void seg_end() { prev_nonempty = cur_any; }
  template <class Sink>
  __device__ void finish(Sink& sink) {
    if (has_pend) sink.put(pend_col, pend_len);
    has_pend = false;
  }
};

// ---------------------------------------------------------------------------
// FP64 traversal of segment P -> Q (Sec. II-C).  Plane k of axis a has the
// crossing parameter sigma_a(k) = fma(k, h_a / D_a, (o_a - P_a) / D_a); the
// segment is in the grid for sigma in (s_in, s_out); each interval between
// consecutive distinct crossings is one entry of length |Q-P| x width, in
// the voxel reached by counting crossed planes.  Incremental form of that
// definition (a digital differential analyser): every axis whose next
// crossing equals the smallest one steps.
// ---------------------------------------------------------------------------
struct SegF64 {
  double D[3], dl[3], s0[3];
  int idx[3], kn[3], step[3];
  bool act[3];
  double s_in, s_out, seglen;
};

__device__ __forceinline__ double sigma_at(const SegF64& sg, int a, int k) {
  return fma((double)k, sg.dl[a], sg.s0[a]);
}

// returns false when the segment does not meet the grid
__device__ __forceinline__ bool seg_setup_f64(const GridDev& g, const double P[3], const double Q[3],
                                              SegF64& sg) {
  const int dim = g.dim;
  sg.s_in = 0.0;
  sg.s_out = 1.0;
  for (int a = 0; a < 3; ++a) {
    sg.act[a] = false;
    sg.idx[a] = 0;
    sg.D[a] = 0.0;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= dim) break;
    sg.D[a] = Q[a] - P[a];
    if (sg.D[a] == 0.0) {
      double fl = floor((P[a] - g.o[a]) / g.h[a]);
      if (fl < 0.0 || fl >= (double)g.n[a]) return false;
      sg.idx[a] = (int)fl;
    } else {
      sg.act[a] = true;
      double inv = 1.0 / sg.D[a];
      sg.dl[a] = g.h[a] * inv;
      sg.s0[a] = (g.o[a] - P[a]) * inv;
      double sa = sg.s0[a];
      double sb = fma((double)g.n[a], sg.dl[a], sg.s0[a]);
      double lo = sa < sb ? sa : sb;
      double hi = sa < sb ? sb : sa;
      if (lo > sg.s_in) sg.s_in = lo;
      if (hi < sg.s_out) sg.s_out = hi;
    }
  }
  if (!(sg.s_in < sg.s_out)) return false;
  double len2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < dim) len2 = len2 + sg.D[a] * sg.D[a];
  sg.seglen = sqrt(len2);
  // start voxel: (planes with sigma <= s_in) - 1, or n - that count
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= dim) break;
    if (!sg.act[a]) continue;
    const int n = g.n[a];
    double x = P[a] + sg.s_in * sg.D[a];
    double u = floor((x - g.o[a]) / g.h[a]);
    int i = (u < 0.0) ? 0 : (u > (double)(n - 1) ? n - 1 : (int)u);
    if (sg.D[a] > 0.0) {
      while (i + 1 <= n - 1 && sigma_at(sg, a, i + 1) <= sg.s_in) ++i;
      while (i > 0 && sigma_at(sg, a, i) > sg.s_in) --i;
      sg.kn[a] = i + 1;
      sg.step[a] = 1;
    } else {
      while (i > 0 && sigma_at(sg, a, i) <= sg.s_in) --i;
      while (i < n - 1 && sigma_at(sg, a, i + 1) > sg.s_in) ++i;
      sg.kn[a] = i;
      sg.step[a] = -1;
    }
    sg.idx[a] = i;
  }
  return true;
}

__device__ __forceinline__ int vox_col(const GridDev& g, const int idx[3]) {
  return idx[0] + g.n[0] * (idx[1] + g.n[1] * (g.dim == 3 ? idx[2] : 0));
}

template <class Merge, class Sink>
__device__ __forceinline__ void seg_walk_f64(const GridDev& g, SegF64& sg, Merge& mg, Sink& sink) {
  const int dim = g.dim;
  double s_prev = sg.s_in;
  // a segment crosses at most sum(n) + 1 intervals; the bound keeps the loop finite
  int guard = g.n[0] + g.n[1] + (dim == 3 ? g.n[2] : 0) + 2;
  while (guard-- > 0) {
    double s_next = sg.s_out;
    double sa[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      sa[a] = (a < dim && sg.act[a]) ? sigma_at(sg, a, sg.kn[a]) : 2.0;
      if (a < dim && sg.act[a] && sa[a] < s_next) s_next = sa[a];
    }
    mg.emit(vox_col(g, sg.idx), sg.seglen * (s_next - s_prev), sink);
    if (!(s_next < sg.s_out)) break;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < dim && sg.act[a] && sa[a] == s_next) {
        sg.idx[a] += sg.step[a];
        sg.kn[a] += sg.step[a];
      }
    }
    s_prev = s_next;
  }
}

}  // namespace pct
