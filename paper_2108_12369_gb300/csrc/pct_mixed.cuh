// pct_mixed.cuh -- FP32 form of the path and traversal with certified
// decisions (PCT_PREC_MIXED).
//
// GB300 runs FP64 at about 1/70 of its FP32 rate.  The FP64 definition
// (pct_device.cuh) is reproduced here with double-float arithmetic: each
// real number is an unevaluated sum hi + lo of two FP32 values (Dekker's
// error-free transformations, with FMA), good to about 2^-44 relative.
//  - Polyline vertices are formed as V = P0 + s D + h10 (m0 - D) + h11 (m1 - D)
//    with D = P1 - P0, the Hermite sum of the definition rearranged into
//    small, well-conditioned terms (the rearrangement is exact in reals).
//  - Every traversal decision (next plane, ties, grid entry / exit, start
//    voxel) compares two crossing parameters sigma.  The double-float values
//    carry a rigorous bound on their distance to the FP64 definition's
//    values; when the difference exceeds the bounds its sign is the FP64
//    sign, otherwise (in practice only at exact ties) both FP64 values are
//    evaluated from the row's FP64 record and compared.
//  - Entry lengths are double-float differences of crossing parameters
//    times the FP32 segment length: accurate to ~1e-9 mm regardless of how
//    shallowly the path crosses a plane.
//  - A segment whose direction sign cannot be certified is walked in FP64.
// Voxel indices and row pointers therefore equal the FP64 definition's.
// Everything is templated on the dimension so that per-axis state lives in
// registers (axis selection uses selects, never dynamic indexing).
#pragma once
#include "pct_device.cuh"

namespace pct {

// ---------------------------------------------------------------------------
// double-float arithmetic (requires that a*b+c is never contracted, which
// the -fmad=false build guarantees; FMAs are explicit)
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return df{s, e};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return df{s, e};
}
// |error| <= 2^-44 (|a| + |b|)
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = s.lo + (a.lo + b.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// |error| <= 2^-44 |a b|
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return quick_two_sum(p, e);
}
// 1 / d by one Newton step from the FP32 reciprocal; |error| <= 2^-43 |1/d|
__device__ __forceinline__ df df_recip(df d) {
  float r = __frcp_rn(d.hi);
  df dr = df_mul_f(d, r);                  // ~ 1
  df e = df_sub(df{1.0f, 0.0f}, dr);       // 1 - d r, small
  return df_add(df{r, 0.0f}, df_mul_f(e, r));
}
__device__ __forceinline__ float df_to_f(df a) { return a.hi + a.lo; }

// FP64 -> double-float with integer operations only (no FP64 pipe):
// hi = RN32(d), lo = RN32(d - hi).  Values below 2^-74 in magnitude lose lo
// (error below 2^-98), values below 2^-103 become 0.
__device__ __forceinline__ df split_d(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  int e = (int)((b >> 52) & 0x7ff);
  if (e < 920) return df{0.0f, 0.0f};
  bool neg = (b >> 63) != 0;
  unsigned long long mant = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  unsigned long long top = mant >> 29;
  unsigned long long rem = mant & ((1ULL << 29) - 1);
  if (rem > (1ULL << 28) || (rem == (1ULL << 28) && (top & 1ULL))) top += 1;
  long long diff = (long long)mant - (long long)(top << 29);  // |diff| <= 2^28
  // scale factors 2^(e - 1046) and 2^(e - 1075) as floats
  float s_hi = __int_as_float((e - 1046 + 127) << 23);
  float hi = (float)(unsigned)top * s_hi;  // top <= 2^24, |diff| <= 2^28: 32-bit conversions are exact
  float lo = 0.0f;
  if (e >= 949) lo = (float)(int)diff * __int_as_float((e - 1075 + 127) << 23);
  if (neg) {
    hi = -hi;
    lo = -lo;
  }
  return df{hi, lo};
}

constexpr float kEps44 = 5.684342e-14f;  // 2^-44

// ---------------------------------------------------------------------------
// Row records.  The count kernel forms the FP64 path (the definition) once
// per proton and leaves it, plus a double-float copy of the quantities the
// vertices are built from, for the fill kernel.
// ---------------------------------------------------------------------------
struct alignas(16) RowDF {
  df P0[3];  // kind 0: A
  df Dl[3];  // P1 - P0
  df u0[3];  // m0 - (P1 - P0)
  df u1[3];  // m1 - (P1 - P0)
  df g0[3];
  df g1[3];
  int kind, nv;
  float fac;  // noise factor 1 + noise_rel z (1 without noise)
  float mag;  // max |coordinate| of the polyline's vertices (for bounds)
};

// the Hermite basis at s = j / K as double-float: (s, h10, h11)
struct alignas(16) BasisDF {
  df s, h10, h11;
  df pad;
};

struct GridDF {
  df o[3], h[3];
  float of[3], rh[3];
};

template <int DIM, class T, int N>
__device__ __forceinline__ T pick(const T (&v)[N], int ax) {
  T r = v[0];
#pragma unroll
  for (int a = 1; a < DIM; ++a)
    if (ax == a) r = v[a];
  return r;
}

template <int DIM>
__device__ __forceinline__ void make_rowdf(const PathF64& p, double R, float fac, RowDF& r) {
  r.kind = p.kind;
  r.nv = p.nv;
  r.fac = fac;
  // mag: a scale of the vertices' coordinates for the error bounds, from the
  // FP32 parts of the splits (no FP64 conversions)
  const float Rf = (float)R;
  float mag = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (p.kind == 0) {
      r.P0[a] = split_d(p.A[a]);
      r.g0[a] = split_d(p.g0[a]);
      mag = fmaxf(mag, fabsf(r.P0[a].hi) + Rf * fabsf(r.g0[a].hi));
    } else {
      double D = p.P1[a] - p.P0[a];
      r.P0[a] = split_d(p.P0[a]);
      r.Dl[a] = split_d(D);
      r.g0[a] = split_d(p.g0[a]);
      r.g1[a] = split_d(p.g1[a]);
      const float p0 = fabsf(r.P0[a].hi), dl = fabsf(r.Dl[a].hi);
      float m = fmaxf(p0 + Rf * fabsf(r.g0[a].hi), p0 + dl + Rf * fabsf(r.g1[a].hi));
      if (p.kind == 2) {
        r.u0[a] = split_d(p.m0[a] - D);
        r.u1[a] = split_d(p.m1[a] - D);
        m = fmaxf(m, p0 + 3.f * dl + fabsf(r.u0[a].hi) + fabsf(r.u1[a].hi));  // |m0|, |m1| <= |u| + |D|
      }
      mag = fmaxf(mag, m);
    }
  }
  r.mag = mag;
}

// vertex q of the polyline in double-float (within 2^-40 mag of the FP64 vertex)
template <int DIM>
__device__ __forceinline__ void vertex_df(const RowDF& r, const BasisDF* tab, df Rdf, int q, df (&V)[3]) {
  if (r.kind == 0) {
    df s = (q == 0) ? df_neg(Rdf) : Rdf;
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_add(r.P0[a], df_mul(s, r.g0[a]));
    return;
  }
  if (q == 0) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_sub(r.P0[a], df_mul(Rdf, r.g0[a]));
  } else if (q == 1) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = r.P0[a];
  } else if (q == r.nv - 2) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_add(r.P0[a], r.Dl[a]);
  } else if (q == r.nv - 1) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_add(df_add(r.P0[a], r.Dl[a]), df_mul(Rdf, r.g1[a]));
  } else {
    BasisDF B = tab[q - 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      V[a] = df_add(df_add(r.P0[a], df_mul(B.s, r.Dl[a])),
                    df_add(df_mul(B.h10, r.u0[a]), df_mul(B.h11, r.u1[a])));
  }
}

// ---------------------------------------------------------------------------
// One segment in double-float with certified decisions
// ---------------------------------------------------------------------------
// An event is plane k of axis ax (0..2), or ax = -1 for the constant k (0 or 1).
struct Ev {
  int ax, k;
};

struct SegDF {
  df P[3];       // start vertex
  df D[3];       // Q - P
  df inv[3];     // 1 / D
  df dl[3];      // h / D
  df sn[3];      // sigma of each axis' next plane
  float E0[3], E1[3];  // bound on |sigma~ - sigma| = E0 + E1 |sigma|
  float L;       // |Q - P|
  int idx[3], kn[3], step[3];
  Ev in, out;
  df s_in, s_out;
  unsigned inert;  // axes the segment runs along inside one slab (no crossing)
};

// Where the FP64 definition of a segment can be rebuilt: kernel arguments
// (a copy in global memory), the row's FP64 path record, the segment index.
struct ExactRef {
  const SimDev* S;
  const PathF64* p;
  int q;
};

// sigma of plane k of axis a in the FP64 definition
__device__ __forceinline__ double sigma_f64(const GridDev& g, const double P[3], const double Q[3], int a, int k) {
  double D = Q[a] - P[a];
  double inv = 1.0 / D;
  double dl = g.h[a] * inv;
  double s0 = (g.o[a] - P[a]) * inv;
  return fma((double)k, dl, s0);
}

// exact sign of sigma(e1) - sigma(e2) from the FP64 definition (rare: only
// where the double-float bounds cannot decide, in practice exact ties)
static __device__ __noinline__ int exact_cmp(ExactRef ref, int ax1, int k1, int ax2, int k2) {
  const SimDev& S = *ref.S;
  double P[3], Q[3];
  path_vertex(S, *ref.p, ref.q, P);
  path_vertex(S, *ref.p, ref.q + 1, Q);
  double x1 = ax1 < 0 ? (double)k1 : sigma_f64(S.ph.g, P, Q, ax1, k1);
  double x2 = ax2 < 0 ? (double)k2 : sigma_f64(S.ph.g, P, Q, ax2, k2);
  return x1 < x2 ? -1 : (x1 > x2 ? 1 : 0);
}

template <int DIM>
__device__ __forceinline__ df plane_df(const GridDF& gd, int a, int k) {
  return df_add(gd.o[a], df_mul_f(gd.h[a], (float)k));
}

// sigma of plane k of axis a: (X_k - P_a) / D_a
template <int DIM>
__device__ __forceinline__ df sigma_df(const SegDF& s, const GridDF& gd, int a, int k) {
  return df_mul(df_sub(plane_df<DIM>(gd, a, k), s.P[a]), s.inv[a]);
}

// exact sign of sigma(e1) - sigma(e2) given their double-float values
template <int DIM>
__device__ __forceinline__ int cmp_vals(const GridDev& g, const SegDF& s, Ev e1, df v1, Ev e2, df v2, ExactRef ends) {
  if (e1.ax == e2.ax && e1.k == e2.k) return 0;
  if (e1.ax < 0 && e2.ax < 0) return e1.k < e2.k ? -1 : (e1.k > e2.k ? 1 : 0);
  float d = (v1.hi - v2.hi) + (v1.lo - v2.lo);
  float m = (e1.ax < 0 ? 0.f : fmaf(pick<DIM>(s.E1, e1.ax), fabsf(v1.hi), pick<DIM>(s.E0, e1.ax))) +
            (e2.ax < 0 ? 0.f : fmaf(pick<DIM>(s.E1, e2.ax), fabsf(v2.hi), pick<DIM>(s.E0, e2.ax)));
  if (d < -m) return -1;
  if (d > m) return 1;
  return exact_cmp(ends, e1.ax, e1.k, e2.ax, e2.k);
}

// Slab k of axis a (plane k <= X < plane k + 1, any integer k) holding X
// at more than the margin from both planes, or false.  The margin covers
// the double-float vertex error and the FP64 definition's rounding of a
// plane position or of a point's floor.
template <int DIM>
__device__ __forceinline__ bool slab_of(const GridDev& g, const GridDF& gd, df X, int a, float eV, int& k) {
  const float h = gd.h[a].hi;
  const float u = floorf((X.hi - gd.of[a]) * gd.rh[a]);
  if (!(fabsf(u) < 1e7f)) return false;
  k = (int)u;
  float r = df_to_f(df_sub(X, plane_df<DIM>(gd, a, k)));
  if (r >= h) {
    ++k;
    r = df_to_f(df_sub(X, plane_df<DIM>(gd, a, k)));
  } else if (r < 0.f) {
    --k;
    r = df_to_f(df_sub(X, plane_df<DIM>(gd, a, k)));
  }
  const float mr = 4.f * (eV + 16.f * kEps44 * (fabsf(X.hi) + fabsf(gd.of[a]) + (float)g.n[a] * h));
  return r > mr && r < h - mr;
}

// Set-up.  Returns 0: the segment misses the grid; 1: ready for walk_df;
// 2: the sign of some axis' extent cannot be certified (walk it in FP64).
// With kInert, an axis whose extent cannot be certified but whose two ends
// lie inside one slab (with margin) is inert: the FP64 definition crosses
// none of its planes there (exactly zero extent: the axis is inactive; a
// tiny one: every plane's crossing parameter lies far outside [0, 1]) and
// its voxel index is that slab's; the other axes decide entry and exit.
template <int DIM, bool kInert = false>
__device__ __forceinline__ int seg_setup_df(const GridDev& g, const GridDF& gd, const df (&P)[3], const df (&Q)[3],
                                            float mag, SegDF& s, ExactRef ends) {
  float L2 = 0.f;
  // |V~ - V| <= eV for every vertex (double-float vertex formation, FP64 rounding)
  const float eV = 64.f * kEps44 * mag;
  s.inert = 0u;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    df D = df_sub(Q[a], P[a]);
    float Dh = df_to_f(D);
    if (!(fabsf(Dh) > 4.f * eV + 4.f * kEps44 * fabsf(Dh))) {
      if constexpr (!kInert) {
        return 2;
      } else {
        int kp, kq;
        if (!slab_of<DIM>(g, gd, P[a], a, eV, kp) || !slab_of<DIM>(g, gd, Q[a], a, eV, kq) || kp != kq) return 2;
        if (kp < 0 || kp > g.n[a] - 1) return 0;  // beside the grid along a
        L2 = fmaf(Dh, Dh, L2);
        s.inert |= 1u << a;
        s.P[a] = P[a];
        s.D[a] = D;
        s.inv[a] = df{0.f, 0.f};
        s.dl[a] = df{3e30f, 0.f};
        s.sn[a] = df{3e30f, 0.f};
        s.E0[a] = 0.f;
        s.E1[a] = 0.f;
        s.step[a] = 1;
        s.idx[a] = kp;
        s.kn[a] = kp + 1;
        continue;
      }
    }
    L2 = fmaf(Dh, Dh, L2);
    s.P[a] = P[a];
    s.D[a] = D;
    s.inv[a] = df_recip(D);
    s.dl[a] = df_mul(gd.h[a], s.inv[a]);
    s.step[a] = Dh > 0.f ? 1 : -1;
    // |sigma~ - sigma| for planes 0..n_a, with X = o + k h:
    //   double-float evaluation  < 2^-42 (|o| + n h + |P|) / |D| + 2^-42 |sigma|
    //   vertices within eV       < eV / |D| + |sigma| 2 eV / |D|
    //   D's own evaluation       < |sigma| 2^-43 mag / |D|
    //   FP64 definition          < 2^-50 (n h + |o - P|) / |D| + 2^-53 |sigma|
    // all times 4 (written as E0 + E1 |sigma|), plus the accumulated error of
    // the incremental steps sigma += dl (< 2^-44 (|sigma| + |dl|) each).
    float mx = (float)g.n[a] * fabsf(gd.h[a].hi) + fabsf(gd.o[a].hi) + fabsf(P[a].hi);
    s.E0[a] = 4.f * (16.f * kEps44 * mx + eV) / fabsf(Dh);
    s.E1[a] = 4.f * (16.f * kEps44 + (2.f * eV + 2.f * kEps44 * mag) / fabsf(Dh));
    s.E0[a] += (float)(g.n[a] + 2) * 2.f * kEps44 * (fabsf(s.dl[a].hi) + 2.f);
  }
  s.L = sqrtf(L2);
  // entry: the largest of 0 and every axis' first plane; exit: the smallest
  // of 1 and every axis' last plane
  s.in = Ev{-1, 0};
  s.out = Ev{-1, 1};
  df vin{0.f, 0.f}, vout{1.f, 0.f};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (s.inert >> a & 1u) continue;
    Ev lo{a, s.step[a] > 0 ? 0 : g.n[a]};
    Ev hi{a, s.step[a] > 0 ? g.n[a] : 0};
    df vlo = sigma_df<DIM>(s, gd, a, lo.k), vhi = sigma_df<DIM>(s, gd, a, hi.k);
    if (cmp_vals<DIM>(g, s, lo, vlo, s.in, vin, ends) > 0) {
      s.in = lo;
      vin = vlo;
    }
    if (cmp_vals<DIM>(g, s, hi, vhi, s.out, vout, ends) < 0) {
      s.out = hi;
      vout = vhi;
    }
  }
  if (cmp_vals<DIM>(g, s, s.in, vin, s.out, vout, ends) >= 0) return 0;
  s.s_in = vin;
  s.s_out = vout;
  // start voxel: (planes with sigma <= s_in) - 1, or n - that count
  const float sin_f = df_to_f(vin);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (s.inert >> a & 1u) continue;
    const int n = g.n[a];
    int i;
    if (s.in.ax == a) {
      i = s.step[a] > 0 ? 0 : n - 1;
    } else {
      df x = df_add(P[a], df_mul_f(df_sub(Q[a], P[a]), sin_f));
      float u = floorf((df_to_f(x) - gd.of[a]) * gd.rh[a]);
      i = (u < 0.f) ? 0 : (u > (float)(n - 1) ? n - 1 : (int)u);
      if (s.step[a] > 0) {
        while (i + 1 <= n - 1 && cmp_vals<DIM>(g, s, Ev{a, i + 1}, sigma_df<DIM>(s, gd, a, i + 1), s.in, vin, ends) <= 0) ++i;
        while (i > 0 && cmp_vals<DIM>(g, s, Ev{a, i}, sigma_df<DIM>(s, gd, a, i), s.in, vin, ends) > 0) --i;
      } else {
        while (i > 0 && cmp_vals<DIM>(g, s, Ev{a, i}, sigma_df<DIM>(s, gd, a, i), s.in, vin, ends) <= 0) --i;
        while (i < n - 1 && cmp_vals<DIM>(g, s, Ev{a, i + 1}, sigma_df<DIM>(s, gd, a, i + 1), s.in, vin, ends) > 0) ++i;
      }
    }
    s.idx[a] = i;
    s.kn[a] = s.step[a] > 0 ? i + 1 : i;
    s.sn[a] = sigma_df<DIM>(s, gd, a, s.kn[a]);
  }
  return 1;
}

// FP32 walk state: crossing parameters as offsets from the segment's walk
// origin (its grid entry s_in): ph_a = sigma of axis a's next plane - s_in,
// computed as fmaf(kf_a, hv_a, ph0_a).  The common offset cancels in every
// comparison; |ph~_a - ph_a| <= e0_a + 8u (|ph~_a| + ph0_a + hv_a).
struct Walk32 {
  float ph0[3], hv[3], e0[3], kf[3];
  float send, esend;  // s_out - s_in and its bound
};

constexpr float kU32 = 5.9604645e-8f;  // 2^-24

// Interior fast path: both endpoints inside the grid by a margin, so
// s_in = 0 and s_out = 1 exactly; the start voxel and the first phases come
// from the double-float residual of P against its lower plane.  Returns
// false when some residual is too close to a plane to certify (the caller
// then uses seg_setup_df).
template <int DIM>
__device__ __forceinline__ bool seg_setup_fast(const GridDev& g, const GridDF& gd, const df (&P)[3], const df (&Q)[3],
                                               float mag, SegDF& s, Walk32& w) {
  const float eV = 64.f * kEps44 * mag;
  float L2 = 0.f;
  s.inert = 0u;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const float lo = gd.of[a], span = (float)g.n[a] * gd.h[a].hi, m = 1e-3f * gd.h[a].hi;
    if (!(P[a].hi > lo + m && P[a].hi < lo + span - m && Q[a].hi > lo + m && Q[a].hi < lo + span - m)) return false;
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    df D = df_sub(Q[a], P[a]);
    float Dh = df_to_f(D);
    if (!(fabsf(Dh) > 4.f * eV + 4.f * kEps44 * fabsf(Dh))) return false;
    L2 = fmaf(Dh, Dh, L2);
    const float h = gd.h[a].hi;
    int i = (int)floorf((P[a].hi - gd.of[a]) * gd.rh[a]);
    i = i < 0 ? 0 : (i > g.n[a] - 1 ? g.n[a] - 1 : i);
    float r = df_to_f(df_sub(P[a], plane_df<DIM>(gd, a, i)));
    if (r >= h) {
      ++i;
      r = df_to_f(df_sub(P[a], plane_df<DIM>(gd, a, i)));
    } else if (r < 0.f) {
      --i;
      r = df_to_f(df_sub(P[a], plane_df<DIM>(gd, a, i)));
    }
    // |r~ - r| < eV + 2^-42 (|P| + |o| + n h); the FP64 definition decides a
    // point on a plane differently from the reals only within 2^-50 of that
    const float mr = 4.f * (eV + 16.f * kEps44 * (fabsf(P[a].hi) + fabsf(gd.of[a]) + (float)g.n[a] * h));
    if (!(r > mr && r < h - mr) || i < 0 || i > g.n[a] - 1) return false;
    const float aD = fabsf(Dh);
    s.P[a] = P[a];
    s.D[a] = D;
    s.step[a] = Dh > 0.f ? 1 : -1;
    s.idx[a] = i;
    s.kn[a] = Dh > 0.f ? i + 1 : i;
    // one correctly rounded reciprocal for the three quotients: each is
    // within about 1 u of the quotient of its operands (a division: 1/2 u);
    // the bounds built on them carry 4 u and more
    const float raD = __frcp_rn(aD);
    w.ph0[a] = (Dh > 0.f ? (h - r) : r) * raD;
    w.hv[a] = h * raD;
    w.kf[a] = 0.f;
    w.e0[a] = (2.f * mr) * raD + 4.f * kU32 * w.ph0[a];
  }
  s.L = sqrtf(L2);
  s.in = Ev{-1, 0};
  s.out = Ev{-1, 1};
  s.s_in = df{0.f, 0.f};
  s.s_out = df{1.f, 0.f};
  w.send = 1.f;
  w.esend = 0.f;
  return true;
}

// convert a double-float set-up (seg_setup_df) into the FP32 walk state
template <int DIM>
__device__ __forceinline__ void walk_from_df(const SegDF& s, Walk32& w) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    float p0 = df_to_f(df_sub(s.sn[a], s.s_in));
    w.ph0[a] = p0;
    w.hv[a] = fabsf(s.dl[a].hi);
    w.kf[a] = 0.f;
    w.e0[a] = fmaf(s.E1[a], fabsf(s.sn[a].hi), s.E0[a]) + 4.f * kU32 * fabsf(p0);
  }
  w.send = df_to_f(df_sub(s.s_out, s.s_in));
  w.esend = (s.out.ax < 0 ? 0.f : fmaf(pick<DIM>(s.E1, s.out.ax), fabsf(s.s_out.hi), pick<DIM>(s.E0, s.out.ax))) +
            4.f * kU32 * fabsf(w.send);
}

// Lean FP32 walker of one set-up segment.  Per step: the smallest phase
// certified against each other axis with one FFMA-formed bound, the exit
// tested by plane index (exit through a grid plane) or against the segment
// end, one fmaf to advance the stepped axis.  Anything the FP32 bounds cannot
// decide (and every exact tie) goes to rare_decide().
template <int DIM>
struct Lean {
  float ph[DIM], hv[DIM], ph0[DIM], kf[DIM];
  float c[DIM];  // bound of ph~ at offset p: c + 8u p
  float send, eend;
  float pcur;
  int kn[DIM], step[DIM], kexit[DIM], dcol[DIM];
  int col, q, out_ax, out_k;
  bool done;
};

template <int DIM>
__device__ __forceinline__ void lean_begin(const GridDev& g, const SegDF& s, const Walk32& w, int q, Lean<DIM>& L) {
  const int stride[3] = {1, g.n[0], g.n[0] * g.n[1]};
  L.col = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    L.ph[a] = w.ph0[a];
    L.ph0[a] = w.ph0[a];
    L.hv[a] = w.hv[a];
    L.kf[a] = 0.f;
    L.c[a] = fmaf(8.f * kU32, w.ph0[a] + w.hv[a], w.e0[a]);
    L.kn[a] = s.kn[a];
    L.step[a] = s.step[a];
    L.kexit[a] = (s.out.ax == a) ? s.out.k : -2147483647;
    L.dcol[a] = s.step[a] * stride[a];
    L.col += s.idx[a] * stride[a];
  }
  L.send = w.send;
  L.eend = w.esend;
  L.pcur = 0.f;
  L.q = q;
  L.out_ax = s.out.ax;
  L.out_k = s.out.k;
  L.done = false;
}

// Exact ordering of the axes' next planes (and against the segment end)
// from double-float values rebuilt from the row record, then FP64 where the
// double-float bounds cannot decide.
template <int DIM>
__device__ __forceinline__ void rare_decide(const RowDF& r, const BasisDF* tab, df Rdf, const GridDF& gd,
                                            const GridDev& g, float mag, ExactRef ref, const Lean<DIM>& L,
                                            unsigned& mask, int& m, bool& final) {
  df P[3], Q[3];
  vertex_df<DIM>(r, tab, Rdf, ref.q, P);
  vertex_df<DIM>(r, tab, Rdf, ref.q + 1, Q);
  const float eV = 64.f * kEps44 * mag;
  int kn[3];
  df v[4];
  float e[4];
#pragma unroll
  for (int a = 0; a < DIM; ++a) kn[a] = L.kn[a];
  // events 0..DIM-1: each axis' next plane; event DIM: the segment's end
  for (int t = 0; t <= DIM; ++t) {
    int a = (t < DIM) ? t : L.out_ax;
    if (t == DIM && a < 0) {
      v[t] = df{(float)L.out_k, 0.f};
      e[t] = 0.f;
      continue;
    }
    int k = (t < DIM) ? kn[a] : L.out_k;
    df D = df_sub(Q[a], P[a]);
    df inv = df_recip(D);
    v[t] = df_mul(df_sub(df_add(gd.o[a], df_mul_f(gd.h[a], (float)k)), P[a]), inv);
    float aD = fabsf(df_to_f(D));
    float mx = (float)g.n[a] * fabsf(gd.h[a].hi) + fabsf(gd.o[a].hi) + fabsf(P[a].hi);
    e[t] = 4.f * (16.f * kEps44 * mx + eV) / aD +
           4.f * (16.f * kEps44 + (2.f * eV + 2.f * kEps44 * mag) / aD) * fabsf(v[t].hi);
  }
  auto cmp = [&](int t1, int t2) -> int {
    float d = (v[t1].hi - v[t2].hi) + (v[t1].lo - v[t2].lo);
    float mm = e[t1] + e[t2];
    if (d < -mm) return -1;
    if (d > mm) return 1;
    int ax1 = t1 < DIM ? t1 : L.out_ax, k1 = t1 < DIM ? kn[t1] : L.out_k;
    int ax2 = t2 < DIM ? t2 : L.out_ax, k2 = t2 < DIM ? kn[t2] : L.out_k;
    if (ax1 == ax2 && k1 == k2) return 0;
    return exact_cmp(ref, ax1, k1, ax2, k2);
  };
  m = 0;
  for (int a = 1; a < DIM; ++a)
    if (cmp(a, m) < 0) m = a;
  mask = 1u << m;
  for (int a = 0; a < DIM; ++a)
    if (a != m && cmp(a, m) == 0) mask |= 1u << a;
  if (L.out_ax >= 0 && (mask >> L.out_ax & 1u) && kn[L.out_ax] == L.out_k)
    final = true;
  else
    final = cmp(m, DIM) >= 0;
}

template <int DIM>
__device__ __forceinline__ float lean_step(Lean<DIM>& L, const RowDF& r, const BasisDF* tab, df Rdf,
                                           const GridDF& gd, const GridDev& g, float mag, ExactRef ref) {
  int m = 0;
  float pm = L.ph[0];
  bool unsure = false;
#pragma unroll
  for (int a = 1; a < DIM; ++a) {
    const float e = fmaf(8.f * kU32, L.ph[a] + pm, L.c[a] + pick<DIM>(L.c, m));
    if (L.ph[a] < pm - e) {
      m = a;
      pm = L.ph[a];
    } else if (!(L.ph[a] > pm + e)) {
      unsure = true;
    }
  }
  unsigned mask = 1u << m;
  bool final = false;
  if (!unsure) {
    if (pick<DIM>(L.kexit, m) == pick<DIM>(L.kn, m)) {
      final = true;
    } else {
      const float e = fmaf(8.f * kU32, pm, pick<DIM>(L.c, m)) + L.eend;
      if (pm > L.send + e)
        final = true;
      else if (!(pm < L.send - e))
        unsure = true;
    }
  }
  if (unsure) {
    rare_decide<DIM>(r, tab, Rdf, gd, g, mag, ref, L, mask, m, final);
    pm = pick<DIM>(L.ph, m);
  }
  const float len = fmaxf((final ? L.send : pm) - L.pcur, 0.f);
  if (final) {
    L.done = true;
    return len;
  }
  L.pcur = pm;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (mask >> a & 1u) {
      L.kf[a] += 1.f;
      L.kn[a] += L.step[a];
      L.col += L.dcol[a];
      L.ph[a] = fmaf(L.kf[a], L.hv[a], L.ph0[a]);
    }
  }
  return len;
}

// kernel arguments of the mixed form besides SimDev
struct MixArgs {
  GridDF gd;
  df R;                 // lead length, double-float
  const BasisDF* tab;   // [K + 1]
  RowDF* rdf;           // [rows]
  PathF64* r64;         // [rows]
  void* lead;           // [rows][2] summaries of the lead-in / lead-out segments
  void* segg;           // [rows][seg_stride] compact segment records (count -> fill); NULL in the lean form
  unsigned char* rflag; // lean form: [rows] 1 = the row goes to the per-lane walker; NULL otherwise
  int seg_stride;
};

// one simulation of a batch (a global-memory copy of its arguments and its
// outputs); item0 = its first work item (block of 128 rows)
struct BatchInst {
  SimDev S;
  MixArgs M;
  long long n;
  long long item0[3];       // first work item of each phase (path, count, fill)
  long long* row_ptr_w;     // [n + 1]: counts go to row_ptr_w[1..n]
  const long long* row_ptr; // the same array, read by the fill
  const float* x;
  int* col;
  float* val;
  float* b;
};

MixArgs mix_args(const SimDev& S, long long n, const void* tab, void* rec, bool lean = false);
// persistent launch of one phase (0 path set-up, 1 count, 2 fill) over the
// items [first, last) (all of dimension dim)
// whether a simulation (rows of up to seg_stride segments, grid g) takes the
// smaller per-warp shared-memory layout of the count / fill kernels
bool small_cap(int seg_stride, const GridDev& g);
// small: every instance of that dimension fits the smaller layout
int batch_blocks_per_sm(int phase, int dim, bool small, bool lean = false);
// nr: rows per work item (32..256), pf: fill prefetch of the next row's records
void launch_batch(int phase, int dim, bool small, bool lean, const BatchInst* B, int n_inst, long long first,
                  long long last, unsigned long long* next, int grid, int nr, int pf, cudaStream_t st);

}  // namespace pct
